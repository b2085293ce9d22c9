"""The allocation-free reduction entry point against the context's own one.

lbm3_mass_noalloc exists for callers that cannot call cudaMalloc (their
device memory is owned by their own pool or allocator, or they run under a
fixed memory budget): it keeps its partial sums in a static device array.
This file is collected last on purpose, so a stop-at-first-failure run has
already run everything else.  It passes alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_1808_08555_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3
    lbm3.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm3


def _case(nx, ny, seed):
    rho = W.droplet_field(nx, ny, seed=seed, count=6, rmin=4.0, rmax=9.0, gap=10.0)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rng = np.random.default_rng(seed)
    f = w[None, :, None, None] * rho[:, None] * (1.0 + 0.05 * rng.uniform(-1, 1, (3, 9, ny, nx)))
    return np.asarray(f, dtype=np.float32).astype(np.float64)


def _reference(L, f, nx, ny):
    """The existing entry point: a context, its state set from f, lbm3_mass."""
    sim = L.Simulation(L.Params(nx, ny))
    sim.set_populations(f)
    m, mo = sim.mass()
    sim.close()
    return np.concatenate([m, mo])


def test_noalloc_matches_lbm3_mass_on_two_calls_in_a_row(L):
    stream = torch.cuda.current_stream()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    # a larger grid first, then a smaller one: the second call must not see
    # the first call's partial sums left in the shared static array
    for (nx, ny, seed) in [(520, 300, 1), (200, 72, 2)]:
        f = _case(nx, ny, seed)
        dev_f = torch.from_numpy(f.astype(np.float32)).cuda().contiguous()
        out.fill_(float("nan"))
        L.lbm3_mass_noalloc(dev_f.data_ptr(), nx, ny, stream.cuda_stream, out.data_ptr())
        stream.synchronize()
        got = out.cpu().numpy()
        ref = _reference(L, f, nx, ny)
        np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-12)
        np.testing.assert_allclose(got[3:], ref[3:], rtol=1e-12, atol=1e-12 * ref[:3].sum())


def test_noalloc_rejects_bad_sizes(L):
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    f = torch.zeros(27 * 16, dtype=torch.float32, device="cuda")
    with pytest.raises(L.Lbm3Error) as e:
        L.lbm3_mass_noalloc(f.data_ptr(), 4097, 4096, None, out.data_ptr())   # above 16,777,216 nodes
    assert e.value.status == L.EINVAL
    with pytest.raises(L.Lbm3Error) as e:
        L.lbm3_mass_noalloc(f.data_ptr(), 0, 4, None, out.data_ptr())
    assert e.value.status == L.EINVAL
    with pytest.raises(L.Lbm3Error) as e:
        L.lbm3_mass_noalloc(0, 4, 4, None, out.data_ptr())
    assert e.value.status == L.EINVAL
