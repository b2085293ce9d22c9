"""Python binding of liblbm3 (the C ABI in include/lbm3.h), via ctypes.

The functions below carry the C names and only marshal arguments: every step
of the lattice Boltzmann update runs in the library's CUDA kernels.  PyTorch
supplies device memory (``Simulation`` binds two torch tensors as the
population buffers) and the CUDA stream (torch's current stream).  There is
no CPU fallback: if the library is missing, loading fails with an error.

Array conventions (see include/lbm3.h): colour densities (3, ny, nx) and
post-streaming populations (3, 9, ny, nx), FP64, C order; host arrays are
numpy arrays or CPU tensors, device arrays are CUDA float64 tensors.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm3.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENUMERIC, ETIMEOUT = range(7)
_STATUS = {OK: "LBM3_OK", EINVAL: "LBM3_EINVAL", ENOMEM: "LBM3_ENOMEM", ECUDA: "LBM3_ECUDA",
           ESTATE: "LBM3_ESTATE", ENUMERIC: "LBM3_ENUMERIC", ETIMEOUT: "LBM3_ETIMEOUT"}
BETA_PAPER, BETA_FU, BETA_SPENCER, BETA_LECLAIRE = range(4)
RECOLOR_COSINE, RECOLOR_LITERAL = range(2)
FP32, FP16_DEV, BF16_DEV, REDUCED = 0, 1, 2, 3
FORCE_BODY, FORCE_PERTURBATION = 0, 1


class Lbm3Error(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class lbm3_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double * 3), ("rho0", ctypes.c_double * 3),
        ("sigma12", ctypes.c_double), ("sigma13", ctypes.c_double), ("sigma23", ctypes.c_double),
        ("beta0", ctypes.c_double),
        ("beta_form", ctypes.c_int32), ("recolor_form", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("force_form", ctypes.c_int32),
        ("normal_delta", ctypes.c_double),
    ]


@dataclass
class Params:
    """Problem statement of one simulation (arXiv 1808.08555, Sec. 2)."""

    nx: int
    ny: int
    tau: tuple = (1.0, 1.0, 1.0)
    rho0: tuple = (1.0, 1.0, 1.0)
    sigma: tuple = (0.01, 0.01, 0.01)  # (sigma_12, sigma_13, sigma_23)
    beta0: float = 0.7
    beta_form: int = BETA_PAPER
    recolor_form: int = RECOLOR_COSINE
    storage: int = FP32
    force_form: int = FORCE_BODY  # 1: perturbation operator (Eqs. phi1 / phi_old)
    # recolouring normal G / max(|G|, normal_delta phi_k phi_l) in Eq. 6;
    # 0 is the paper's unit normal G/|G|
    normal_delta: float = 0.1

    def to_c(self) -> lbm3_params:
        p = lbm3_params()
        p.nx, p.ny = int(self.nx), int(self.ny)
        for k in range(3):
            p.tau[k] = float(self.tau[k])
            p.rho0[k] = float(self.rho0[k])
        p.sigma12, p.sigma13, p.sigma23 = (float(s) for s in self.sigma)
        p.beta0 = float(self.beta0)
        p.beta_form, p.recolor_form = int(self.beta_form), int(self.recolor_form)
        p.storage, p.force_form = int(self.storage), int(self.force_form)
        p.normal_delta = float(self.normal_delta)
        return p


class lbm3_interfaces(ctypes.Structure):
    _fields_ = [
        ("varphi", ctypes.c_double * 3), ("varphi_junction", (ctypes.c_double * 3) * 2),
        ("junction", (ctypes.c_double * 2) * 2), ("circle", (ctypes.c_double * 3) * 3),
        ("points", ctypes.c_double * 3), ("p_bulk", ctypes.c_double * 3), ("n_bulk", ctypes.c_double * 3),
        ("flags", ctypes.c_int32),
    ]


_lib = None


def load() -> ctypes.CDLL:
    """Load liblbm3.so (built by ``paper_1808_08555_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblbm3.so is not built ({LIB_PATH}); run paper_1808_08555_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, vp, dp = ctypes.POINTER(lbm3_params), ctypes.c_void_p, ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "lbm3_buffer_bytes": (st, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "lbm3_create": (st, [P, vp, ctypes.POINTER(vp)]),
        "lbm3_bind_buffers": (st, [vp, vp, vp, ctypes.c_size_t]),
        "lbm3_init": (st, [vp, dp, ctypes.c_int]),
        "lbm3_set_populations": (st, [vp, dp, ctypes.c_int]),
        "lbm3_set_rows_per_cta": (st, [vp, ctypes.c_int32]),
        "lbm3_debug_stall_row": (st, [vp, ctypes.c_int32]),
        "lbm3_step": (st, [vp, ctypes.c_int64]),
        "lbm3_fields": (st, [vp, dp, dp, dp, dp, ctypes.c_int]),
        "lbm3_populations": (st, [vp, dp, ctypes.c_int]),
        "lbm3_mass": (st, [vp, dp, dp]),
        "lbm3_sync": (st, [vp]),
        "lbm3_time": (ctypes.c_int64, [vp]),
        "lbm3_destroy": (st, [vp]),
        "lbm3_last_error": (ctypes.c_char_p, [vp]),
        "lbm3_mass_noalloc": (st, [vp, ctypes.c_int32, ctypes.c_int32, vp, vp]),
        "lbm3_set_params": (st, [vp, P]),
        "lbm3_phi": (st, [vp, dp, ctypes.c_int]),
        "lbm3_interface_diagnostics": (st, [vp, ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(lbm3_interfaces)]),
        "lbm3_tape_forward": (st, [vp, ctypes.c_int64, ctypes.c_int32]),
        "lbm3_tape_backward": (st, [vp, dp, ctypes.c_int, dp, dp, ctypes.c_int, dp]),
        "lbm3_batch_create": (st, [P, ctypes.c_int32, vp, ctypes.c_int32, ctypes.POINTER(vp)]),
        "lbm3_batch_count": (ctypes.c_int32, [vp]),
        "lbm3_batch_autotune": (st, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_double), dp]),
        "lbm3_batch_work_items": (ctypes.c_int32, [vp]),
        "lbm3_batch_init": (st, [vp, ctypes.c_int32, dp, ctypes.c_int]),
        "lbm3_batch_set_populations": (st, [vp, ctypes.c_int32, dp, ctypes.c_int]),
        "lbm3_batch_fields": (st, [vp, ctypes.c_int32, dp, dp, dp, dp, ctypes.c_int]),
        "lbm3_batch_populations": (st, [vp, ctypes.c_int32, dp, ctypes.c_int]),
        "lbm3_batch_mass": (st, [vp, ctypes.c_int32, dp, dp]),
        "lbm3_batch_step": (st, [vp, ctypes.c_int64]),
        "lbm3_batch_sync": (st, [vp]),
        "lbm3_batch_time": (ctypes.c_int64, [vp]),
        "lbm3_batch_destroy": (st, [vp]),
        "lbm3_batch_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _check(ctx, status: int):
    if status != OK:
        msg = load().lbm3_last_error(ctx).decode() if ctx else "(no context)"
        raise Lbm3Error(status, msg)


def _ptr(a):
    """(pointer, on_device) for a numpy array or torch tensor of float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError("expected a contiguous float64 tensor")
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    except ImportError:  # pragma: no cover
        pass
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float64 numpy array")
    return ctypes.c_void_p(a.ctypes.data), 0


# ------------------------------------------------------------ C-named calls

def lbm3_buffer_bytes(params: Params) -> int:
    n = ctypes.c_size_t()
    p = params.to_c()
    _check(None, load().lbm3_buffer_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def lbm3_create(params: Params, stream: int | None = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    p = params.to_c()
    s = load().lbm3_create(ctypes.byref(p), ctypes.c_void_p(stream or 0), ctypes.byref(ctx))
    if s != OK:
        raise Lbm3Error(s, "lbm3_create failed (parameters invalid or CUDA unavailable)")
    return ctx


def lbm3_bind_buffers(ctx, f0_ptr: int, f1_ptr: int, nbytes: int):
    _check(ctx, load().lbm3_bind_buffers(ctx, ctypes.c_void_p(f0_ptr), ctypes.c_void_p(f1_ptr), nbytes))


def lbm3_init(ctx, rho):
    p, dev = _ptr(rho)
    _check(ctx, load().lbm3_init(ctx, p, dev))


def lbm3_set_populations(ctx, f):
    p, dev = _ptr(f)
    _check(ctx, load().lbm3_set_populations(ctx, p, dev))


def lbm3_set_rows_per_cta(ctx, rows: int):
    _check(ctx, load().lbm3_set_rows_per_cta(ctx, int(rows)))


def lbm3_debug_stall_row(ctx, row: int):
    """Testing hook: the next step's CTA 0 never receives march row `row`,
    so its bounded waits run out (LBM3_ETIMEOUT at the next sync)."""
    _check(ctx, load().lbm3_debug_stall_row(ctx, int(row)))


def lbm3_step(ctx, n: int = 1):
    _check(ctx, load().lbm3_step(ctx, int(n)))


def lbm3_fields(ctx, rho=None, ux=None, uy=None, p=None):
    ptrs, devs = [], set()
    for a in (rho, ux, uy, p):
        if a is None:
            ptrs.append(None)
        else:
            q, d = _ptr(a)
            ptrs.append(q)
            devs.add(d)
    if len(devs) > 1:
        raise ValueError("outputs must be all host or all device arrays")
    _check(ctx, load().lbm3_fields(ctx, *ptrs, devs.pop() if devs else 0))


def lbm3_populations(ctx, f):
    p, dev = _ptr(f)
    _check(ctx, load().lbm3_populations(ctx, p, dev))


def lbm3_mass(ctx):
    m = np.zeros(3)
    mo = np.zeros(2)
    _check(ctx, load().lbm3_mass(ctx, ctypes.c_void_p(m.ctypes.data), ctypes.c_void_p(mo.ctypes.data)))
    return m, mo


def lbm3_mass_noalloc(dev_f_ptr: int, nx: int, ny: int, stream: int | None, dev_out_ptr: int):
    """Allocation-free reduction (see include/lbm3.h): device pointers in and
    out, enqueued on `stream`, no synchronisation."""
    s = load().lbm3_mass_noalloc(ctypes.c_void_p(dev_f_ptr), int(nx), int(ny), ctypes.c_void_p(stream or 0),
                                 ctypes.c_void_p(dev_out_ptr))
    if s != OK:
        raise Lbm3Error(s, "lbm3_mass_noalloc failed")


def lbm3_set_params(ctx, params: Params):
    p = params.to_c()
    _check(ctx, load().lbm3_set_params(ctx, ctypes.byref(p)))


def lbm3_phi(ctx, phi):
    p, dev = _ptr(phi)
    _check(ctx, load().lbm3_phi(ctx, p, dev))


def lbm3_interface_diagnostics(ctx, third_max: float = 1e-3, bulk_min: float = 0.99) -> dict:
    """FP64 device diagnostics of the current state (see include/lbm3.h):
    contact angles varphi_kl (degrees), junctions, fitted interface circles,
    bulk pressures per fluid."""
    r = lbm3_interfaces()
    _check(ctx, load().lbm3_interface_diagnostics(ctx, float(third_max), float(bulk_min), ctypes.byref(r)))
    return {"varphi": list(r.varphi), "varphi_junction": [list(v) for v in r.varphi_junction],
            "junctions": [tuple(v) for v in r.junction], "circles": [tuple(v) for v in r.circle],
            "points": list(r.points), "p_bulk": list(r.p_bulk), "n_bulk": list(r.n_bulk), "flags": int(r.flags)}


def lbm3_tape_forward(ctx, nsteps: int, checkpoint_every: int):
    _check(ctx, load().lbm3_tape_forward(ctx, int(nsteps), int(checkpoint_every)))


def lbm3_tape_backward(ctx, dphi, dpop0=None, drho0=None, want_dsigma: bool = True):
    """Returns dJ/dsigma (numpy (3,)) or None; fills dpop0 / drho0 if given
    (both host or both device arrays)."""
    pd, ddev = _ptr(dphi)
    outs, devs = [], set()
    for a in (dpop0, drho0):
        if a is None:
            outs.append(None)
        else:
            q, d = _ptr(a)
            outs.append(q)
            devs.add(d)
    if len(devs) > 1:
        raise ValueError("dpop0 and drho0 must be both host or both device arrays")
    ds = np.zeros(3)
    dsp = ctypes.c_void_p(ds.ctypes.data) if want_dsigma else None
    _check(ctx, load().lbm3_tape_backward(ctx, pd, ddev, outs[0], outs[1], devs.pop() if devs else 0, dsp))
    return ds if want_dsigma else None


def lbm3_sync(ctx):
    _check(ctx, load().lbm3_sync(ctx))


def lbm3_time(ctx) -> int:
    return int(load().lbm3_time(ctx))


def lbm3_destroy(ctx):
    load().lbm3_destroy(ctx)


def lbm3_last_error(ctx) -> str:
    return load().lbm3_last_error(ctx).decode()


# ---------------------------------------------------------- convenience

class Simulation:
    """One simulation on the current CUDA device: torch-owned population
    buffers bound to a library context on torch's current stream."""

    def __init__(self, params: Params, device=None, rows_per_cta: int = 0):
        import torch

        self.params = params
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            nbytes = lbm3_buffer_bytes(params)
            self._bufs = [torch.empty(nbytes // 4, dtype=torch.float32, device=self.device) for _ in range(2)]
            self.ctx = lbm3_create(params, self.stream.cuda_stream)
            lbm3_bind_buffers(self.ctx, self._bufs[0].data_ptr(), self._bufs[1].data_ptr(), nbytes)
            if rows_per_cta:
                lbm3_set_rows_per_cta(self.ctx, rows_per_cta)

    def init(self, rho):
        lbm3_init(self.ctx, rho)
        return self

    def set_populations(self, f):
        lbm3_set_populations(self.ctx, f)
        return self

    def step(self, n: int = 1):
        lbm3_step(self.ctx, n)
        return self

    def populations(self) -> np.ndarray:
        f = np.empty((3, 9, self.params.ny, self.params.nx))
        lbm3_populations(self.ctx, f)
        return f

    def fields(self) -> dict:
        ny, nx = self.params.ny, self.params.nx
        out = {"rho": np.empty((3, ny, nx)), "ux": np.empty((ny, nx)), "uy": np.empty((ny, nx)),
               "p": np.empty((ny, nx))}
        lbm3_fields(self.ctx, out["rho"], out["ux"], out["uy"], out["p"])
        return out

    def mass(self):
        return lbm3_mass(self.ctx)

    def phi(self) -> np.ndarray:
        out = np.empty((3, self.params.ny, self.params.nx))
        lbm3_phi(self.ctx, out)
        return out

    def interfaces(self, third_max: float = 1e-3, bulk_min: float = 0.99) -> dict:
        return lbm3_interface_diagnostics(self.ctx, third_max, bulk_min)

    def set_params(self, params: Params):
        lbm3_set_params(self.ctx, params)
        self.params = params
        return self

    def tape_forward(self, nsteps: int, checkpoint_every: int):
        lbm3_tape_forward(self.ctx, nsteps, checkpoint_every)
        return self

    def tape_backward(self, dphi, dpop0=None, drho0=None):
        return lbm3_tape_backward(self.ctx, dphi, dpop0, drho0)

    def sync(self):
        lbm3_sync(self.ctx)

    @property
    def t(self) -> int:
        return lbm3_time(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lbm3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches

def _bcheck(b, status: int):
    if status != OK:
        raise Lbm3Error(status, load().lbm3_batch_last_error(b).decode())


def lbm3_batch_create(params_list, stream: int | None = None, rows_per_cta: int = 0) -> ctypes.c_void_p:
    arr = (lbm3_params * len(params_list))(*[p.to_c() for p in params_list])
    b = ctypes.c_void_p()
    s = load().lbm3_batch_create(arr, len(params_list), ctypes.c_void_p(stream or 0), int(rows_per_cta),
                                 ctypes.byref(b))
    if s != OK:
        raise Lbm3Error(s, "lbm3_batch_create failed (an instance's parameters are invalid or CUDA failed)")
    return b


def lbm3_batch_init(b, i: int, rho):
    p, dev = _ptr(rho)
    _bcheck(b, load().lbm3_batch_init(b, int(i), p, dev))


def lbm3_batch_set_populations(b, i: int, f):
    p, dev = _ptr(f)
    _bcheck(b, load().lbm3_batch_set_populations(b, int(i), p, dev))


def lbm3_batch_step(b, n: int = 1):
    _bcheck(b, load().lbm3_batch_step(b, int(n)))


def lbm3_batch_populations(b, i: int, f):
    p, dev = _ptr(f)
    _bcheck(b, load().lbm3_batch_populations(b, int(i), p, dev))


def lbm3_batch_fields(b, i: int, rho=None, ux=None, uy=None, p=None):
    ptrs, devs = [], set()
    for a in (rho, ux, uy, p):
        if a is None:
            ptrs.append(None)
        else:
            q, d = _ptr(a)
            ptrs.append(q)
            devs.add(d)
    if len(devs) > 1:
        raise ValueError("outputs must be all host or all device arrays")
    _bcheck(b, load().lbm3_batch_fields(b, int(i), *ptrs, devs.pop() if devs else 0))


def lbm3_batch_mass(b, i: int):
    m = np.zeros(3)
    mo = np.zeros(2)
    _bcheck(b, load().lbm3_batch_mass(b, int(i), ctypes.c_void_p(m.ctypes.data), ctypes.c_void_p(mo.ctypes.data)))
    return m, mo


def lbm3_batch_sync(b):
    _bcheck(b, load().lbm3_batch_sync(b))


def lbm3_batch_destroy(b):
    load().lbm3_batch_destroy(b)


def lbm3_batch_autotune(b, candidates: int = 5, steps: int = 20) -> dict:
    """Time candidate tile heights on the current state (see include/lbm3.h)
    and keep the fastest.  Returns the winner and every candidate's time."""
    rows = ctypes.c_int32()
    ms = ctypes.c_double()
    table = np.zeros(2 * (candidates + 2))
    s = load().lbm3_batch_autotune(b, int(candidates), int(steps), ctypes.byref(rows), ctypes.byref(ms),
                                   ctypes.c_void_p(table.ctypes.data))
    if s != OK:
        raise Lbm3Error(s, load().lbm3_batch_last_error(b).decode())
    cands = [(int(r), float(t)) for r, t in table.reshape(-1, 2) if r > 0]
    return {"rows": int(rows.value), "ms_per_step": float(ms.value), "candidates": cands}


class Batch:
    """Independent simulations advanced together on the current device and
    torch's current stream (one launch per step, replayed from a CUDA graph)."""

    def __init__(self, params_list, rows_per_cta: int = 0):
        import torch

        self.params = list(params_list)
        self.stream = torch.cuda.current_stream()
        self.b = lbm3_batch_create(self.params, self.stream.cuda_stream, rows_per_cta)

    def __len__(self):
        return len(self.params)

    @property
    def work_items(self) -> int:
        return int(load().lbm3_batch_work_items(self.b))

    @property
    def t(self) -> int:
        return int(load().lbm3_batch_time(self.b))

    def init(self, i, rho):
        lbm3_batch_init(self.b, i, rho)
        return self

    def set_populations(self, i, f):
        lbm3_batch_set_populations(self.b, i, f)
        return self

    def step(self, n: int = 1):
        lbm3_batch_step(self.b, n)
        return self

    def autotune(self, candidates: int = 5, steps: int = 20) -> dict:
        return lbm3_batch_autotune(self.b, candidates, steps)

    def populations(self, i) -> np.ndarray:
        p = self.params[i]
        f = np.empty((3, 9, p.ny, p.nx))
        lbm3_batch_populations(self.b, i, f)
        return f

    def fields(self, i) -> dict:
        p = self.params[i]
        out = {"rho": np.empty((3, p.ny, p.nx)), "ux": np.empty((p.ny, p.nx)), "uy": np.empty((p.ny, p.nx)),
               "p": np.empty((p.ny, p.nx))}
        lbm3_batch_fields(self.b, i, out["rho"], out["ux"], out["uy"], out["p"])
        return out

    def mass(self, i):
        return lbm3_batch_mass(self.b, i)

    def sync(self):
        lbm3_batch_sync(self.b)

    def close(self):
        if getattr(self, "b", None):
            lbm3_batch_destroy(self.b)
            self.b = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- autograd

def phi_after(sim: "Simulation", rho0, sigma, nsteps: int, checkpoint_every: int = 0):
    """phi(t = nsteps) of a run from the rest state f = w_i rho0_k, as a
    differentiable torch function of rho0 ((3, ny, nx) float64 CUDA tensor)
    and sigma ((3,) float64 tensor of sigma_12, sigma_13, sigma_23).  The
    backward pass is the library's reverse mode (lbm3_tape_backward);
    checkpoint_every = 0 picks about sqrt(nsteps)."""
    import torch

    class _PhiAfter(torch.autograd.Function):
        @staticmethod
        def forward(ctx, rho0, sigma):
            p = sim.params
            s = [float(v) for v in sigma.detach().cpu()]
            if tuple(s) != tuple(p.sigma):
                sim.set_params(dataclasses.replace(p, sigma=tuple(s)))
            sim.init(rho0.detach().contiguous())
            every = checkpoint_every or max(1, int(round(nsteps ** 0.5)))
            sim.tape_forward(nsteps, every)
            phi = torch.empty_like(rho0)
            lbm3_phi(sim.ctx, phi)
            ctx.sigma_device = sigma.device
            return phi

        @staticmethod
        def backward(ctx, gphi):
            drho = torch.empty_like(gphi)
            ds = lbm3_tape_backward(sim.ctx, gphi.contiguous(), None, drho)
            return drho, torch.from_numpy(ds).to(ctx.sigma_device)

    return _PhiAfter.apply(rho0, sigma)


# ------------------------------------------------------------- N fluids

class lbm3n_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nfluids", ctypes.c_int32),
        ("tau", ctypes.c_void_p), ("rho0", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
        ("beta0", ctypes.c_double), ("beta_form", ctypes.c_int32), ("recolor_form", ctypes.c_int32),
        ("normal_delta", ctypes.c_double), ("storage", ctypes.c_int32),
    ]


def _load_n():
    lib = load()
    if not hasattr(lib, "_n_bound"):
        vp, dp, st = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
        sig = {
            "lbm3n_create": (st, [ctypes.POINTER(lbm3n_params), vp, ctypes.POINTER(vp)]),
            "lbm3n_init": (st, [vp, dp, ctypes.c_int]),
            "lbm3n_set_populations": (st, [vp, dp, ctypes.c_int]),
            "lbm3n_step": (st, [vp, ctypes.c_int64]),
            "lbm3n_populations": (st, [vp, dp, ctypes.c_int]),
            "lbm3n_mass": (st, [vp, dp, dp]),
            "lbm3n_fields": (st, [vp, dp, dp, dp, dp, ctypes.c_int]),
            "lbm3n_destroy": (st, [vp]),
            "lbm3n_last_error": (ctypes.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        lib._n_bound = True
    return lib


class NSimulation:
    """N-fluid simulation (include/lbm3.h, lbm3n_*) on the current device and
    torch's current stream.  sigma: (N, N) symmetric tension matrix with a
    zero diagonal; tau, rho0: length N.  storage: FP32 (populations) or
    REDUCED (phi_k, V_k, f^dagger_i per node; the same results, bit for
    bit)."""

    def __init__(self, nx: int, ny: int, sigma, tau, rho0=None, beta0: float = 0.7, beta_form: int = 0,
                 recolor_form: int = RECOLOR_COSINE, normal_delta: float = 0.1, storage: int = FP32):
        import torch

        self.sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        n = self.sigma.shape[0]
        self.tau = np.ascontiguousarray(tau, dtype=np.float64)
        self.rho0 = np.ascontiguousarray(rho0 if rho0 is not None else np.ones(n), dtype=np.float64)
        self.nx, self.ny, self.n = int(nx), int(ny), n
        p = lbm3n_params()
        p.nx, p.ny, p.nfluids = self.nx, self.ny, n
        p.tau, p.rho0, p.sigma = self.tau.ctypes.data, self.rho0.ctypes.data, self.sigma.ctypes.data
        p.beta0, p.beta_form, p.recolor_form, p.normal_delta = float(beta0), int(beta_form), int(recolor_form), \
            float(normal_delta)
        p.storage = int(storage)
        self.ctx = ctypes.c_void_p()
        self.stream = torch.cuda.current_stream()
        s = _load_n().lbm3n_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.ctx))
        if s != OK:
            raise Lbm3Error(s, "lbm3n_create failed (parameters invalid or CUDA unavailable)")

    def _check(self, s):
        if s != OK:
            raise Lbm3Error(s, _load_n().lbm3n_last_error(self.ctx).decode())

    def init(self, rho):
        q, dev = _ptr(np.ascontiguousarray(rho, dtype=np.float64))
        self._check(_load_n().lbm3n_init(self.ctx, q, dev))
        return self

    def set_populations(self, f):
        q, dev = _ptr(f if not isinstance(f, np.ndarray) else np.ascontiguousarray(f, dtype=np.float64))
        self._check(_load_n().lbm3n_set_populations(self.ctx, q, dev))
        return self

    def step(self, n: int = 1):
        self._check(_load_n().lbm3n_step(self.ctx, int(n)))
        return self

    def populations(self) -> np.ndarray:
        f = np.empty((self.n, 9, self.ny, self.nx))
        self._check(_load_n().lbm3n_populations(self.ctx, ctypes.c_void_p(f.ctypes.data), 0))
        return f

    def mass(self):
        m = np.zeros(self.n)
        mo = np.zeros(2)
        self._check(_load_n().lbm3n_mass(self.ctx, ctypes.c_void_p(m.ctypes.data), ctypes.c_void_p(mo.ctypes.data)))
        return m, mo

    def fields(self) -> dict:
        """rho (N, ny, nx), ux, uy, p (ny, nx), FP64."""
        rho = np.empty((self.n, self.ny, self.nx))
        ux, uy, p = (np.empty((self.ny, self.nx)) for _ in range(3))
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        self._check(_load_n().lbm3n_fields(self.ctx, ptr(rho), ptr(ux), ptr(uy), ptr(p), 0))
        return {"rho": rho, "ux": ux, "uy": uy, "p": p}

    def close(self):
        if getattr(self, "ctx", None):
            _load_n().lbm3n_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- D3Q19

class lbm3d_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("nfluids", ctypes.c_int32),
        ("tau", ctypes.c_void_p), ("rho0", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
        ("beta0", ctypes.c_double), ("beta_form", ctypes.c_int32), ("recolor_form", ctypes.c_int32),
        ("normal_delta", ctypes.c_double), ("storage", ctypes.c_int32),
    ]


def _load_d():
    lib = load()
    if not hasattr(lib, "_d_bound"):
        vp, dp, st = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
        sig = {
            "lbm3d_create": (st, [ctypes.POINTER(lbm3d_params), vp, ctypes.POINTER(vp)]),
            "lbm3d_init": (st, [vp, dp, ctypes.c_int]),
            "lbm3d_set_populations": (st, [vp, dp, ctypes.c_int]),
            "lbm3d_step": (st, [vp, ctypes.c_int64]),
            "lbm3d_populations": (st, [vp, dp, ctypes.c_int]),
            "lbm3d_mass": (st, [vp, dp, dp]),
            "lbm3d_fields": (st, [vp, dp, dp, dp, ctypes.c_int]),
            "lbm3d_destroy": (st, [vp]),
            "lbm3d_last_error": (ctypes.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        lib._d_bound = True
    return lib


class D3Q19Simulation:
    """N-fluid simulation on the D3Q19 lattice (include/lbm3.h, lbm3d_*) on
    the current device and torch's current stream.  sigma: (N, N) symmetric
    tension matrix with a zero diagonal; tau, rho0: length N.  Densities are
    (N, nz, ny, nx), populations (N, 19, nz, ny, nx), post-streaming.
    storage: FP32 (populations) or REDUCED (phi_k, f^dagger_i, V_k per node;
    the same results, bit for bit)."""

    def __init__(self, nx: int, ny: int, nz: int, sigma, tau, rho0=None, beta0: float = 0.7, beta_form: int = 0,
                 recolor_form: int = RECOLOR_COSINE, normal_delta: float = 0.1, storage: int = FP32):
        import torch

        self.sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        n = self.sigma.shape[0]
        self.tau = np.ascontiguousarray(tau, dtype=np.float64)
        self.rho0 = np.ascontiguousarray(rho0 if rho0 is not None else np.ones(n), dtype=np.float64)
        self.nx, self.ny, self.nz, self.n = int(nx), int(ny), int(nz), n
        p = lbm3d_params()
        p.nx, p.ny, p.nz, p.nfluids = self.nx, self.ny, self.nz, n
        p.tau, p.rho0, p.sigma = self.tau.ctypes.data, self.rho0.ctypes.data, self.sigma.ctypes.data
        p.beta0, p.beta_form, p.recolor_form, p.normal_delta = float(beta0), int(beta_form), int(recolor_form), \
            float(normal_delta)
        p.storage = int(storage)
        self.ctx = ctypes.c_void_p()
        self.stream = torch.cuda.current_stream()
        s = _load_d().lbm3d_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.ctx))
        if s != OK:
            raise Lbm3Error(s, "lbm3d_create failed (parameters invalid or CUDA unavailable)")

    def _check(self, s):
        if s != OK:
            raise Lbm3Error(s, _load_d().lbm3d_last_error(self.ctx).decode())

    def init(self, rho):
        q, dev = _ptr(np.ascontiguousarray(rho, dtype=np.float64))
        self._check(_load_d().lbm3d_init(self.ctx, q, dev))
        return self

    def set_populations(self, f):
        q, dev = _ptr(f if not isinstance(f, np.ndarray) else np.ascontiguousarray(f, dtype=np.float64))
        self._check(_load_d().lbm3d_set_populations(self.ctx, q, dev))
        return self

    def step(self, n: int = 1):
        self._check(_load_d().lbm3d_step(self.ctx, int(n)))
        return self

    def populations(self) -> np.ndarray:
        f = np.empty((self.n, 19, self.nz, self.ny, self.nx))
        self._check(_load_d().lbm3d_populations(self.ctx, ctypes.c_void_p(f.ctypes.data), 0))
        return f

    def mass(self):
        m = np.zeros(self.n)
        mo = np.zeros(3)
        self._check(_load_d().lbm3d_mass(self.ctx, ctypes.c_void_p(m.ctypes.data), ctypes.c_void_p(mo.ctypes.data)))
        return m, mo

    def fields(self) -> dict:
        """rho (N, nz, ny, nx), u (3, nz, ny, nx) and p (nz, ny, nx), FP64."""
        rho = np.empty((self.n, self.nz, self.ny, self.nx))
        u = np.empty((3, self.nz, self.ny, self.nx))
        p = np.empty((self.nz, self.ny, self.nx))
        self._check(_load_d().lbm3d_fields(self.ctx, ctypes.c_void_p(rho.ctypes.data), ctypes.c_void_p(u.ctypes.data),
                                           ctypes.c_void_p(p.ctypes.data), 0))
        return {"rho": rho, "u": u, "p": p}

    def close(self):
        if getattr(self, "ctx", None):
            _load_d().lbm3d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
