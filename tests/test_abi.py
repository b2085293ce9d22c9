"""C-ABI checks that need no GPU: the library builds/loads, exports every
symbol its header declares, and validates parameters on the host."""
import ctypes
import os
import re

import pytest

from paper_1808_08555_gb300 import build as B
from paper_1808_08555_gb300 import lbm3 as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbm3[nd]?_\w+)\s*\(", txt))
    return names


def test_header_symbols_exported(lib):
    names = _declared()
    assert "lbm3_step" in names and "lbm3_create" in names
    assert "lbm3n_step" in names and "lbm3d_step" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_params_struct_layout_matches_header():
    # int32 nx, ny; 3+3 doubles; 3 sigmas; beta0; 4 int32 (beta, recolour, storage, force
    # forms); normal_delta -> 4*2 + 8*10 + 4*4 + 8 = 112 bytes
    assert ctypes.sizeof(L.lbm3_params) == 112
    assert L.lbm3_params.normal_delta.offset == 104
    # lbm3_interfaces: 31 doubles and an int32 flag word, padded to 8 bytes
    assert ctypes.sizeof(L.lbm3_interfaces) == 256 and L.lbm3_interfaces.flags.offset == 248
    # lbm3n_params: 3 int32, 3 pointers, beta0, 2 int32, normal_delta, storage
    assert ctypes.sizeof(L.lbm3n_params) == 72 and L.lbm3n_params.tau.offset == 16
    assert L.lbm3n_params.normal_delta.offset == 56 and L.lbm3n_params.storage.offset == 64
    # lbm3d_params: 4 int32, 3 pointers, beta0, 2 int32, normal_delta, storage
    assert ctypes.sizeof(L.lbm3d_params) == 72 and L.lbm3d_params.tau.offset == 16
    assert L.lbm3d_params.beta0.offset == 40 and L.lbm3d_params.normal_delta.offset == 56
    assert L.lbm3d_params.storage.offset == 64


@pytest.mark.parametrize("kw", [
    dict(nx=6, ny=8), dict(nx=0, ny=8), dict(nx=8, ny=0), dict(nx=8, ny=8, tau=(0.5, 1, 1)),
    dict(nx=8, ny=8, rho0=(1, 0, 1)), dict(nx=8, ny=8, sigma=(0.01, -1, 0.01)),
    dict(nx=8, ny=8, beta0=0.0), dict(nx=8, ny=8, beta0=1.5), dict(nx=8, ny=8, beta_form=7),
    dict(nx=8, ny=8, recolor_form=2), dict(nx=8, ny=8, storage=9), dict(nx=8, ny=8, storage=-1),
    dict(nx=8, ny=8, force_form=2), dict(nx=8, ny=8, force_form=-1), dict(nx=8, ny=8, force_form=1, storage=1),
    dict(nx=8, ny=8, normal_delta=-0.1), dict(nx=8, ny=8, normal_delta=1.5),
    dict(nx=8, ny=8, normal_delta=float("nan")),
    # nx*ny below 2^31, but one padded FP32 plane reaches 4 GiB
    dict(nx=4, ny=2 ** 28), dict(nx=32768, ny=32768),
])
def test_invalid_params_rejected(lib, kw):
    with pytest.raises(L.Lbm3Error) as e:
        L.lbm3_buffer_bytes(L.Params(**kw))
    assert e.value.status == L.EINVAL


def test_buffer_bytes(lib):
    # 27 planes of ny rows, pitch max(nx + 8, 136) rounded up to 8 (ghost columns for the periodic wrap)
    assert L.lbm3_buffer_bytes(L.Params(8, 4)) == 27 * 4 * 136 * 4
    assert L.lbm3_buffer_bytes(L.Params(2048, 2048)) == 27 * 2048 * 2056 * 4
    assert L.lbm3_buffer_bytes(L.Params(2044, 10)) == 27 * 10 * 2056 * 4
    # 16-bit deviations plus three FP32 rho' planes
    assert L.lbm3_buffer_bytes(L.Params(2048, 2048, storage=1)) == (27 * 2 + 3 * 4) * 2048 * 2056
    assert L.lbm3_buffer_bytes(L.Params(2048, 2048, storage=2)) == (27 * 2 + 3 * 4) * 2048 * 2056
    # reduced state: three float4 planes and six float planes
    assert L.lbm3_buffer_bytes(L.Params(2048, 2048, storage=3)) == 18 * 4 * 2048 * 2056
    with pytest.raises(L.Lbm3Error):
        L.lbm3_buffer_bytes(L.Params(8, 8, storage=4))
    with pytest.raises(L.Lbm3Error):   # the perturbation operator runs on FP32 storage only
        L.lbm3_buffer_bytes(L.Params(8, 8, storage=3, force_form=1))


def test_largest_plane_accepted(lib):
    # 32768 x 32760 x 4 bytes per padded plane: just below the 4 GiB plane limit
    assert L.lbm3_buffer_bytes(L.Params(32760, 32760)) == 27 * 32760 * 32768 * 4


def test_null_context_is_einval(lib):
    assert lib.lbm3_step(None, 1) == L.EINVAL
    assert lib.lbm3_mass(None, None, None) == L.EINVAL
    assert lib.lbm3_destroy(None) == L.OK
    assert lib.lbm3_last_error(None)


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.Lbm3Error) as e:
        L.lbm3_create(L.Params(8, 8))
    assert e.value.status in (L.ECUDA, L.ENOMEM)


def _params_nd(cls, dims, n=3, **kw):
    """An lbm3n_params / lbm3d_params with valid defaults, then kw applied;
    the arrays it points to are returned too (they must outlive the call)."""
    import numpy as np

    sig = np.full((n, n), 0.01)
    np.fill_diagonal(sig, 0.0)
    if kw.pop("asym", False):
        sig[0, 1] += 0.001
    tau = np.full(n, kw.pop("tau0", 1.0))
    rho0 = np.ones(n)
    p = cls()
    for name, v in dims.items():
        setattr(p, name, v)
    p.nfluids = kw.pop("nfluids", n)
    p.tau, p.rho0, p.sigma = tau.ctypes.data, rho0.ctypes.data, sig.ctypes.data
    p.beta0, p.beta_form, p.recolor_form, p.normal_delta = 0.7, 0, 0, 0.1
    for name, v in kw.items():
        setattr(p, name, v)
    return p, (sig, tau, rho0)


@pytest.mark.parametrize("kw", [dict(nfluids=1), dict(nfluids=5), dict(nz=0), dict(ny=70000), dict(nz=70000),
                                dict(asym=True), dict(tau0=0.5), dict(beta0=0.0), dict(beta_form=2),
                                dict(recolor_form=-1), dict(normal_delta=2.0), dict(storage=1), dict(storage=2),
                                dict(storage=4)])
def test_d3q19_create_validates_on_the_host(lib, kw):
    """lbm3d_create rejects invalid parameters before any CUDA call."""
    n = 3 if kw.get("nfluids", 3) in (1, 5) else kw.get("nfluids", 3)
    p, keep = _params_nd(L.lbm3d_params, {"nx": 8, "ny": 8, "nz": 8}, n=n, **kw)
    ctx = ctypes.c_void_p()
    assert L._load_d().lbm3d_create(ctypes.byref(p), None, ctypes.byref(ctx)) == L.EINVAL
    assert not ctx.value


@pytest.mark.parametrize("kw", [dict(nfluids=1), dict(nfluids=7), dict(ny=0), dict(asym=True), dict(tau0=0.5),
                                dict(beta_form=2), dict(normal_delta=-0.1), dict(storage=1), dict(storage=2),
                                dict(storage=4)])
def test_nfluid_create_validates_on_the_host(lib, kw):
    """lbm3n_create rejects invalid parameters before any CUDA call."""
    p, keep = _params_nd(L.lbm3n_params, {"nx": 8, "ny": 8}, n=3, **kw)
    ctx = ctypes.c_void_p()
    assert L._load_n().lbm3n_create(ctypes.byref(p), None, ctypes.byref(ctx)) == L.EINVAL
    assert not ctx.value
