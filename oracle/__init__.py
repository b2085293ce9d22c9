"""FP64 CPU oracle of the ternary colour-gradient LBM step (arXiv 1808.08555, Sec. 2).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: the arithmetic lives in ``lbm3_oracle.c`` (plain loops,
double precision), compiled here with gcc and called through ctypes.

Array conventions (numpy, float64, C order):
  f    : (3, 9, ny, nx)  post-streaming populations f_{i,k}(x, t), k = r, g, b
  rho  : (3, ny, nx)     colour densities rho_k
  sigma: (sigma_12, sigma_13, sigma_23)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

# Threads of the oracle's node loops wait passively between loops, so that a
# busy host (other processes, a second threaded library) does not turn each
# loop's barrier into spinning threads that starve the working ones (read by
# the OpenMP runtime when the oracle's library first loads it).
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm3_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm3_oracle.so")
_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("tau", ctypes.c_double * 3),
        ("rho0", ctypes.c_double * 3),
        ("sigma", ctypes.c_double * 3),
        ("beta0", ctypes.c_double),
        ("beta_form", ctypes.c_int),
        ("recolor_form", ctypes.c_int),
        ("force_form", ctypes.c_int),
        ("normal_delta", ctypes.c_double),
    ]


@dataclass
class Params:
    """Physical parameters of one simulation (Sec. 2)."""

    nx: int
    ny: int
    tau: tuple = (1.0, 1.0, 1.0)
    rho0: tuple = (1.0, 1.0, 1.0)
    sigma: tuple = (0.01, 0.01, 0.01)
    beta0: float = 0.7
    beta_form: int = 0
    recolor_form: int = 0
    force_form: int = 0  # 0: Eq. 11 force via Eq. 5; 1: perturbation operator (Eqs. phi1, phi_old)
    # recolouring normal n = G / max(|G|, normal_delta phi_k phi_l) in Eq. 6;
    # 0 is the paper's unit normal G/|G| (Sec. 2, after Eq. 11)
    normal_delta: float = 0.1
    extra: dict = field(default_factory=dict)

    def _c(self) -> _Params:
        p = _Params()
        p.nx, p.ny = int(self.nx), int(self.ny)
        for j in range(3):
            p.tau[j] = float(self.tau[j])
            p.rho0[j] = float(self.rho0[j])
            p.sigma[j] = float(self.sigma[j])
        p.beta0 = float(self.beta0)
        p.beta_form = int(self.beta_form)
        p.recolor_form = int(self.recolor_form)
        p.force_form = int(self.force_form)
        p.normal_delta = float(self.normal_delta)
        return p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vector or host-specific flags), with
    OpenMP over the node loops when the compiler supports it (the results do
    not depend on the thread count)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        lib.orc_g.restype = ctypes.c_double
        lib.orc_g.argtypes = [ctypes.c_double]
        lib.orc_X.argtypes = [dp, dp]
        lib.orc_feq.argtypes = [ctypes.c_double] * 3 + [dp]
        lib.orc_guo.argtypes = [ctypes.c_double] * 5 + [dp]
        lib.orc_perturbation.argtypes = [dp, dp, dp, ctypes.c_double, dp]
        lib.orc_grad.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_colour_gradients.argtypes = [pp, dp, dp, dp]
        lib.orc_force.argtypes = [pp, dp, dp, dp, dp]
        lib.orc_beta.argtypes = [pp, dp, dp]
        lib.orc_fields.argtypes = [pp, dp, dp, dp, dp, dp]
        lib.orc_step.argtypes = [pp, dp, ctypes.c_int]
        lib.orc_init.argtypes = [pp, dp, dp]
        lib.orc_mass.argtypes = [pp, dp, dp, dp]
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def threads(n: int = 0) -> int:
    """Host threads of the oracle's node loops: n > 0 sets them, 0 only
    reads them.  Returns the number in effect (1 for a build without OpenMP)."""
    return int(_load().orc_threads(int(n)))


# ------------------------------------------------------------------ pieces

def g(X: float) -> float:
    """Eq. 20."""
    return _load().orc_g(float(X))


def X_of(sigma) -> np.ndarray:
    """Eq. 18: (X_12, X_13, X_23)."""
    s = _f64(sigma)
    out = np.zeros(3)
    _load().orc_X(_ptr(s), _ptr(out))
    return out


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. 3 for one node."""
    out = np.zeros(9)
    _load().orc_feq(rho, ux, uy, _ptr(out))
    return out


def guo(tau: float, ux: float, uy: float, Fx: float, Fy: float) -> np.ndarray:
    """Eq. 5 for one node."""
    out = np.zeros(9)
    _load().orc_guo(tau, ux, uy, Fx, Fy, _ptr(out))
    return out



def perturbation(sigma, G, C, tauf: float) -> np.ndarray:
    """Eqs. phi1 / phi_old for one node.  G: (3, 3, 2) colour gradients
    G_kl (G_lk = -G_kl), C: (3, 3) concentration factors."""
    out = np.zeros(9)
    _load().orc_perturbation(_ptr(_f64(sigma)), _ptr(_f64(G)), _ptr(_f64(C)), float(tauf), _ptr(out))
    return out


def grad(v) -> tuple[np.ndarray, np.ndarray]:
    """Eq. fd1 on a periodic (ny, nx) field; returns (d_x v, d_y v)."""
    v = _f64(v)
    ny, nx = v.shape
    gx = np.zeros_like(v)
    gy = np.zeros_like(v)
    _load().orc_grad(nx, ny, _ptr(v), _ptr(gx), _ptr(gy))
    return gx, gy


def colour_gradients(p: Params, rho) -> tuple[np.ndarray, np.ndarray]:
    """G_kl (3,3,2,ny,nx) and C_kl (3,3,ny,nx) from colour densities."""
    rho = _f64(rho)
    G = np.zeros((3, 3, 2) + rho.shape[1:])
    C = np.zeros((3, 3) + rho.shape[1:])
    cp = p._c()
    _load().orc_colour_gradients(ctypes.byref(cp), _ptr(rho), _ptr(G), _ptr(C))
    return G, C


def force(p: Params, rho) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Eq. 11: (F_x, F_y, T) with T = (T_xx, T_xy, T_yy)."""
    rho = _f64(rho)
    shape = rho.shape[1:]
    Fx = np.zeros(shape)
    Fy = np.zeros(shape)
    T = np.zeros((3,) + shape)
    cp = p._c()
    _load().orc_force(ctypes.byref(cp), _ptr(rho), _ptr(Fx), _ptr(Fy), _ptr(T))
    return Fx, Fy, T


def beta(p: Params, rk) -> np.ndarray:
    """Segregation parameters (beta_12, beta_13, beta_23) at one node."""
    rk = _f64(rk)
    out = np.zeros(3)
    cp = p._c()
    _load().orc_beta(ctypes.byref(cp), _ptr(rk), _ptr(out))
    return out


def init(p: Params, rho) -> np.ndarray:
    """f_{i,k} = w_i rho_k (rest equilibrium per colour)."""
    rho = _f64(rho)
    f = np.zeros((3, 9) + rho.shape[1:])
    cp = p._c()
    _load().orc_init(ctypes.byref(cp), _ptr(rho), _ptr(f))
    return f


def step(p: Params, f, n: int = 1) -> np.ndarray:
    """Advance post-streaming populations by n steps; returns a new array."""
    f = _f64(f).copy()
    assert f.shape == (3, 9, p.ny, p.nx)
    cp = p._c()
    _load().orc_step(ctypes.byref(cp), _ptr(f), int(n))
    return f


def fields(p: Params, f) -> dict:
    """rho_k, u (with the F_s/2 correction of Eq. uk1) and p = rho/3."""
    f = _f64(f)
    shape = f.shape[2:]
    rho = np.zeros((3,) + shape)
    ux = np.zeros(shape)
    uy = np.zeros(shape)
    pr = np.zeros(shape)
    cp = p._c()
    _load().orc_fields(ctypes.byref(cp), _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(pr))
    return {"rho": rho, "ux": ux, "uy": uy, "p": pr}


def mass(p: Params, f) -> tuple[np.ndarray, np.ndarray]:
    """Per-colour mass (3,) and lattice momentum sum f_i e_i (2,)."""
    f = _f64(f)
    m = np.zeros(3)
    mo = np.zeros(2)
    cp = p._c()
    _load().orc_mass(ctypes.byref(cp), _ptr(f), _ptr(m), _ptr(mo))
    return m, mo
