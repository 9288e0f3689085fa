"""Serving with continuous batching (se2ot_serve_*): requests admitted by slots and a device-memory
budget, their chunks overlapping on the device.  A request's result must be the same alone and in
the mix (bit-for-bit: every request runs its own deterministic kernel sequence) and equal to
se2ot_barycenter with the same options."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)

REQUESTS = [  # nx, ny, nt, r, eps, n, max_iters, check_every, tol
    (32, 32, 8, 3, 0.1, 2, 600, 10, 5e-3),
    (48, 40, 16, 4, 0.1, 3, 600, 10, 5e-3),
    (40, 40, 8, 5, 1e-3, 4, 60, 0, 0.0),
    (64, 48, 16, 6, 0.1, 2, 600, 20, 5e-3),
    (36, 36, 4, 3, 5e-3, 5, 80, 0, 0.0),
    (33, 29, 16, 4, 0.1, 2, 600, 10, 5e-3),
    (56, 56, 8, 7, 0.1, 3, 600, 10, 5e-3),
    (30, 30, 32, 3, 2e-2, 2, 50, 0, 0.0),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def make(k):
    nx, ny, nt, r, eps, n, iters, check, tol = REQUESTS[k]
    desc = se2ot.make_desc(nx, ny, nt, r, W, eps)
    mu = synth.coupled_measures(n, nx, ny, nt, config_seed=40 + k, max_shift=1, nbumps=3).astype(np.float32)
    lam = np.linspace(1.0, 2.0, n)
    lam = (lam / lam.sum()).tolist()
    return desc, torch.from_numpy(mu), lam, se2ot.solve_opts(iters, check, tol)


def serve(reqs, budget, slots):
    sv = se2ot.Server(budget, slots)
    tickets = [sv.submit(d, mu, lam, o) for (d, mu, lam, o) in reqs]
    results = []
    for (d, mu, lam, o), t in zip(reqs, tickets):
        out = torch.empty(mu.shape[1:], dtype=torch.float32)
        st, status = sv.wait(t, out)
        results.append((out, st, status))
    sv.close()
    return results


def test_mix_equals_alone_and_single_solves():
    reqs = [make(k) for k in range(len(REQUESTS))]
    mixed = serve(reqs, budget=1 << 30, slots=4)
    for k, (d, mu, lam, o) in enumerate(reqs):
        alone = serve([reqs[k]], budget=1 << 30, slots=1)[0]
        assert mixed[k][2] == alone[2] == se2ot.SE2OT_OK, (k, mixed[k][2], alone[2])
        assert torch.equal(mixed[k][0], alone[0]), k
        assert mixed[k][1]["iters"] == alone[1]["iters"]
        kern = se2ot.se2ot_kernel_build(d)
        single, sst, status = se2ot.se2ot_barycenter(kern, mu.cuda(), lam, o)
        assert status == se2ot.SE2OT_OK
        assert torch.equal(single.cpu(), mixed[k][0]), k
        assert sst["iters"] == mixed[k][1]["iters"]
        if o.tol_viol > 0:
            assert mixed[k][1]["viol"] <= o.tol_viol
        kern.close()


# A sample of the literal serving mix (grids up to 512^2, 32 orientations, the radii and eps range
# of the batched workload), served together; 20 iterations each so that the oracle can run the
# small ones in full.  nx, nt, r, eps, n
LITERAL_SAMPLE = [(64, 16, 7, 3.2e-4, 3), (64, 32, 7, 5e-5, 2), (256, 32, 15, 1.1e-4, 2), (512, 16, 8, 2.4e-4, 2),
                  (128, 32, 11, 7e-5, 4)]


def test_literal_mix_sample_matches_oracle_and_single_solves():
    """Served together, each request of the sample equals its single solve bit for bit, and the two
    smallest match the FP64 oracle's barycenter within 1e-5 rel L1 (Appendix A)."""
    reqs = []
    for k, (nx, nt, r, eps, n) in enumerate(LITERAL_SAMPLE):
        mu = synth.coupled_measures(n, nx, nx, nt, config_seed=70 + k, max_shift=r // 2, nbumps=3).astype(np.float32)
        lam = np.linspace(1.0, 3.0, n)
        reqs.append((se2ot.make_desc(nx, nx, nt, r, W, eps), torch.from_numpy(mu), (lam / lam.sum()).tolist(),
                     se2ot.solve_opts(20)))
    mixed = serve(reqs, budget=32 << 30, slots=8)
    for k, (d, mu, lam, o) in enumerate(reqs):
        assert mixed[k][2] == se2ot.SE2OT_OK
        kern = se2ot.se2ot_kernel_build(d)
        single, _, status = se2ot.se2ot_barycenter(kern, mu.cuda(), lam, o)
        assert status == se2ot.SE2OT_OK
        assert torch.equal(single.cpu(), mixed[k][0]), k
        kern.close()
    for k in (0, 1):
        nx, nt, r, eps, n = LITERAL_SAMPLE[k]
        d, mu, lam, _ = reqs[k]
        want = oracle.barycenter_log(oracle.Grid(nx, nx, nt, r, W, eps), mu.numpy().astype(np.float64), lam, 20)
        got = mixed[k][0].numpy().astype(np.float64)
        assert np.abs(got - want).sum() / np.abs(want).sum() <= 1e-5, k


def test_budget_admits_as_memory_frees_up():
    """A budget that holds about one request at a time: everything still completes, in order."""
    reqs = [make(k) for k in (0, 1, 3, 5)]
    big = max(4 * 90 * r[0].nx * r[0].ny * r[0].ntheta * r[1].shape[0] for r in reqs)
    res = serve(reqs, budget=big, slots=4)
    ref = serve(reqs, budget=1 << 30, slots=4)
    for (a, sa, ka), (b, sb, kb) in zip(res, ref):
        assert ka == kb == se2ot.SE2OT_OK
        assert torch.equal(a, b)


def test_request_larger_than_budget_is_refused_and_timeouts():
    d, mu, lam, o = make(6)
    sv = se2ot.Server(1 << 20, 2)   # 1 MiB: too small for this request
    with pytest.raises(se2ot.SE2OTError):
        sv.submit(d, mu, lam, o)
    sv.close()
    sv = se2ot.Server(1 << 30, 2)
    t = sv.submit(*make(6))
    _, status = sv.wait(t, None, timeout_ms=0)
    assert status in (se2ot.SE2OT_ETIMEOUT, se2ot.SE2OT_OK)
    if status == se2ot.SE2OT_ETIMEOUT:
        out = torch.empty(mu.shape[1:], dtype=torch.float32)
        _, status = sv.wait(t, out)
        assert status == se2ot.SE2OT_OK and torch.isfinite(out).all()
    sv.close()


def test_injected_admission_failure_rejects_only_that_request():
    os.environ["SE2OT_TEST_FAIL_ADMISSION"] = "1"    # the second admission fails
    try:
        reqs = [make(k) for k in (0, 2, 4)]
        res = serve(reqs, budget=1 << 30, slots=1)
    finally:
        del os.environ["SE2OT_TEST_FAIL_ADMISSION"]
    assert [r[2] for r in res] == [se2ot.SE2OT_OK, se2ot.SE2OT_ENOMEM, se2ot.SE2OT_OK]
    assert torch.isfinite(res[0][0]).all() and torch.isfinite(res[2][0]).all()


def test_submit_refuses_inputs_that_are_not_equal_mass_measures():
    """The server runs se2ot_barycenter's input check on its host copy of the request."""
    d, mu, lam, o = make(0)
    sv = se2ot.Server(1 << 30, 2)
    for edit, words in ((lambda m: m[0, 1, 1].__setitem__(0, float("nan")), "non-finite"),
                        (lambda m: m[1].mul_(1.0 + 1e-5), "masses differ")):
        bad = mu.clone()
        edit(bad)
        with pytest.raises(se2ot.SE2OTError) as ei:
            sv.submit(d, bad, lam, o)
        assert ei.value.status == se2ot.SE2OT_EINVAL and words in str(ei.value)
    with pytest.raises(ValueError):
        sv.submit(d, mu[:, :5], lam, o)
    t = sv.submit(d, mu, lam, o)
    out = torch.empty(mu.shape[1:], dtype=torch.float32)
    st, status = sv.wait(t, out)
    assert status == se2ot.SE2OT_OK and st["logscale_min"] <= st["logscale_max"]
    sv.close()


def test_server_on_a_fresh_process_races_a_solve_on_another_thread():
    """Kernel attributes are set once per device under a lock: a server's worker thread and a
    caller thread that launch their first convolutions at the same time in a fresh process both get
    correct results (each equal to a later single-threaded solve)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r'''
import sys, threading, numpy as np, torch
sys.path.insert(0, %r)
from paper_2402_15322_gb300 import se2ot, synth
torch.cuda.set_device(0)
W = (1.0, 3.0, 0.5)
d1 = se2ot.make_desc(40, 36, 16, 10, W, 1e-3)
d2 = se2ot.make_desc(48, 40, 8, 7, W, 2e-3)
mu1 = torch.from_numpy(synth.coupled_measures(3, 40, 36, 16, 5, 1, nbumps=3).astype(np.float32))
mu2 = torch.from_numpy(synth.coupled_measures(2, 48, 40, 8, 6, 1, nbumps=3).astype(np.float32))
lam1, lam2 = [0.2, 0.3, 0.5], [0.5, 0.5]
res = {}
def solve():
    k = se2ot.se2ot_kernel_build(d1)
    res["solve"] = se2ot.se2ot_barycenter(k, mu1.cuda(), lam1, se2ot.solve_opts(30))[0].cpu()
    k.close()
th = threading.Thread(target=solve)
sv = se2ot.Server(1 << 30, 2)
th.start()
t = sv.submit(d2, mu2, lam2, se2ot.solve_opts(30))
out = torch.empty((40, 48, 8), dtype=torch.float32)
st, status = sv.wait(t, out)
th.join()
sv.close()
assert status == se2ot.SE2OT_OK
k = se2ot.se2ot_kernel_build(d1)
want1 = se2ot.se2ot_barycenter(k, mu1.cuda(), lam1, se2ot.solve_opts(30))[0].cpu()
k = se2ot.se2ot_kernel_build(d2)
want2 = se2ot.se2ot_barycenter(k, mu2.cuda(), lam2, se2ot.solve_opts(30))[0].cpu()
assert torch.equal(res["solve"], want1), "threaded solve differs"
assert torch.equal(out, want2), "served result differs"
print("race ok")
''' % root
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "race ok" in r.stdout, r.stdout + r.stderr
