"""se2ot_barycenter_noalloc: the barycenter for callers that cannot allocate device memory (a
host framework that owns the memory budget, a loop that cannot afford cudaMalloc's
synchronisation, a plugin limited to the buffers it is handed).  Its result must match the
ordinary se2ot_barycenter on the same inputs, on consecutive calls that share the library's
static scratch array.  Collected last on purpose (file name), and self-contained so that it also
passes alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rel_l1(a, b):
    a = a.double().cpu()
    b = b.double().cpu()
    return float((a - b).abs().sum() / b.abs().sum())


@pytest.mark.parametrize("nx,ny,nt,r,eps,n,lam,iters", [
    (32, 32, 8, 3, 5e-4, 2, [0.5, 0.5], 40),
    (37, 29, 16, 4, 1e-3, 3, [0.2, 0.3, 0.5], 25),
])
def test_noalloc_matches_barycenter_on_consecutive_calls(nx, ny, nt, r, eps, n, lam, iters):
    desc = se2ot.make_desc(nx, ny, nt, r, (1.0, 3.0, 0.5), eps)
    k = se2ot.se2ot_kernel_build(desc)
    opts = se2ot.solve_opts(iters)
    for call in range(2):
        mu = synth.coupled_measures(n, nx, ny, nt, config_seed=31 + call, max_shift=1, nbumps=3)
        mu = torch.from_numpy(mu.astype(np.float32)).cuda()
        want, wst, _ = se2ot.se2ot_barycenter(k, mu, lam, opts)
        got, gst, status = se2ot.se2ot_barycenter_noalloc(desc, mu, lam, opts)
        torch.cuda.synchronize()
        assert status == se2ot.SE2OT_OK
        assert rel_l1(got, want) <= 1e-5
        assert gst["iters"] == wst["iters"] == iters
        assert abs(gst["mass"] - wst["mass"]) <= 1e-6 * wst["mass"]
    k.close()


def test_noalloc_rejects_problems_larger_than_its_array():
    desc = se2ot.make_desc(128, 128, 16, 10, (1.0, 3.0, 0.5), 1e-4)
    mu = torch.full((4, 128, 128, 16), 1.0 / (128 * 128 * 16), dtype=torch.float32, device="cuda")
    _, _, status = se2ot.se2ot_barycenter_noalloc(desc, mu, [0.25] * 4, se2ot.solve_opts(2),
                                                  raise_on_error=False)
    assert status == se2ot.SE2OT_EINVAL
    assert "scratch" in se2ot.se2ot_last_error()
    _, _, status = se2ot.se2ot_barycenter_noalloc(desc, mu.cpu()[:1, :32, :32, :8].contiguous(),
                                                  [1.0], se2ot.solve_opts(2), raise_on_error=False)
    assert status == se2ot.SE2OT_EINVAL
