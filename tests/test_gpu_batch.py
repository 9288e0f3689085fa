"""Batched interpolations of uneven sizes (se2ot_interpolate_batched): every problem of the batch
must give bit-for-bit the result of the same problem solved alone (same tile code, same order of
operations), and the single solves themselves match the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)

PROBLEMS = [  # nx, ny, nt, r, eps, t
    (32, 32, 8, 3, 5e-4, 0.5),
    (48, 40, 16, 5, 1e-3, 0.25),
    (64, 64, 8, 7, 2e-3, 0.8),
    (40, 56, 4, 4, 5e-3, 0.0),
    (33, 17, 32, 4, 4e-3, 1.0),
    (50, 50, 16, 7, 1e-3, 0.6),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def inputs(seed):
    out = []
    for k, (nx, ny, nt, r, eps, t) in enumerate(PROBLEMS):
        mu = synth.coupled_measures(2, nx, ny, nt, config_seed=seed, problem=k, max_shift=max(1, r // 2),
                                    nbumps=3).astype(np.float32)
        out.append(mu)
    return out


def test_batch_equals_single_solves_and_oracle():
    iters = 25
    descs = [se2ot.make_desc(nx, ny, nt, r, W, eps) for (nx, ny, nt, r, eps, t) in PROBLEMS]
    ts = [p[5] for p in PROBLEMS]
    for call, seed in enumerate((3, 4)):   # the second call reuses the cached batch
        mus = inputs(seed)
        mu0 = [torch.from_numpy(m[0]).cuda() for m in mus]
        mu1 = [torch.from_numpy(m[1]).cuda() for m in mus]
        outs, stats, status = se2ot.se2ot_interpolate_batched(descs, mu0, mu1, ts, se2ot.solve_opts(iters))
        torch.cuda.synchronize()
        assert status == se2ot.SE2OT_OK
        for k, d in enumerate(descs):
            kern = se2ot.se2ot_kernel_build(d)
            single, sst, _ = se2ot.se2ot_interpolate(kern, mu0[k], mu1[k], ts[k], se2ot.solve_opts(iters))
            assert torch.equal(outs[k], single), k
            assert stats[k]["mass"] == sst["mass"] and stats[k]["viol"] == sst["viol"]
            kern.close()
    # the small problems against the FP64 oracle
    for k in (0, 3):
        nx, ny, nt, r, eps, t = PROBLEMS[k]
        want = oracle.interpolate_log(oracle.Grid(nx, ny, nt, r, W, eps), mus[k][0].astype(np.float64),
                                      mus[k][1].astype(np.float64), t, iters)
        got = outs[k].cpu().double().numpy()
        assert np.abs(got - want).sum() / want.sum() <= 1e-5


def test_both_launch_forms_are_bit_identical_and_the_tuner_measures_them():
    """The batch's convolutions as one launch per radius class or as one launch per line (every
    radius in it) give the same bits; an unforced first call times both and keeps the faster."""
    iters = 12
    descs = [se2ot.make_desc(nx, ny, nt, r, W, eps) for (nx, ny, nt, r, eps, t) in PROBLEMS]
    ts = [p[5] for p in PROBLEMS]
    mus = inputs(7)
    mu0 = [torch.from_numpy(m[0]).cuda() for m in mus]
    mu1 = [torch.from_numpy(m[1]).cuda() for m in mus]
    res = {}
    for flag in (se2ot.SE2OT_FLAG_BATCH_PER_RADIUS, se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH, 0):
        outs, stats, _ = se2ot.se2ot_interpolate_batched(descs, mu0, mu1, ts, se2ot.solve_opts(iters, flags=flag))
        res[flag] = ([o.clone() for o in outs], stats)
    for k in range(len(descs)):
        assert torch.equal(res[se2ot.SE2OT_FLAG_BATCH_PER_RADIUS][0][k], res[se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH][0][k]), k
        assert torch.equal(res[0][0][k], res[se2ot.SE2OT_FLAG_BATCH_PER_RADIUS][0][k]), k
    # 6 problems of 4 distinct radii: 4 + 4 convolution launches per iteration against 2
    per, one = (res[f][1][0]["kernel_launches"] for f in (se2ot.SE2OT_FLAG_BATCH_PER_RADIUS,
                                                          se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH))
    assert per - one == 6 * iters
    form, ms_per, ms_one = se2ot.se2ot_batch_tuning()
    assert form in (1, 2) and ms_per > 0 and ms_one > 0
    assert form == (2 if ms_one < ms_per else 1)
    _, _, st = se2ot.se2ot_interpolate_batched(descs, mu0, mu1, ts, se2ot.solve_opts(
        iters, flags=se2ot.SE2OT_FLAG_BATCH_PER_RADIUS | se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH), raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL


def test_batch_rejects_what_it_does_not_support():
    d = se2ot.make_desc(32, 32, 8, 3, W, 5e-4, periodic=True)
    mu = torch.full((32, 32, 8), 1.0 / 8192, device="cuda")
    _, _, st = se2ot.se2ot_interpolate_batched([d], [mu], [mu], [0.5], raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    d = se2ot.make_desc(32, 32, 8, 3, W, 5e-4)
    _, _, st = se2ot.se2ot_interpolate_batched([d], [mu], [mu], [0.5], se2ot.solve_opts(10, 5, 1e-3),
                                               raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    # host tensors: refused by the binding, and by the C entry point itself
    with pytest.raises(ValueError):
        se2ot.se2ot_interpolate_batched([d], [mu.cpu()], [mu], [0.5], raise_on_error=False)
    import ctypes
    host = mu.cpu()
    arr = lambda *ts: (ctypes.c_void_p * 1)(*[t.data_ptr() for t in ts])
    st = se2ot.lib().se2ot_interpolate_batched(1, (se2ot.se2ot_kernel_desc * 1)(d), arr(host), arr(mu),
                                               (ctypes.c_double * 1)(0.5), None, arr(mu), None, None)
    assert st == se2ot.SE2OT_EINVAL


def test_batch_checks_every_problems_inputs():
    """Each problem's pair must be measures of equal mass (Appendix A): a negative entry or unequal
    masses in one problem of the batch is refused, naming that problem, before any iteration."""
    d = se2ot.make_desc(32, 32, 8, 3, W, 5e-4)
    good = torch.full((32, 32, 8), 1.0 / 8192, device="cuda")
    neg = good.clone()
    neg[3, 4, 5] = -1e-9
    heavy = good * (1.0 + 1e-5)
    for bad, words in ((neg, "negative"), (heavy, "masses differ")):
        _, _, st = se2ot.se2ot_interpolate_batched([d, d], [good, good], [good, bad], [0.5, 0.5],
                                                   se2ot.solve_opts(5), raise_on_error=False)
        assert st == se2ot.SE2OT_EINVAL
        msg = se2ot.se2ot_last_error()
        assert "problem 1" in msg and words in msg
    outs, stats, st = se2ot.se2ot_interpolate_batched([d, d], [good, good], [good, good], [0.5, 0.5],
                                                      se2ot.solve_opts(5))
    assert st == se2ot.SE2OT_OK and all(torch.isfinite(o).all() for o in outs)
    assert all(s["logscale_min"] <= s["logscale_max"] for s in stats)


def test_largest_radius_class_in_both_launch_forms_against_oracle():
    """Radii 11 and 15 (the largest the batched workload draws) in both launch forms: the forms agree
    bit for bit and the r = 15 problem matches the FP64 oracle (Appendix A, n = 2)."""
    probs = [(40, 40, 8, 15, 2e-3, 0.3), (48, 44, 16, 11, 1e-3, 0.7)]
    iters = 15
    descs = [se2ot.make_desc(nx, ny, nt, r, W, eps) for (nx, ny, nt, r, eps, t) in probs]
    ts = [p[5] for p in probs]
    mus = [synth.coupled_measures(2, nx, ny, nt, config_seed=9, problem=k, max_shift=3, nbumps=3).astype(np.float32)
           for k, (nx, ny, nt, r, eps, t) in enumerate(probs)]
    mu0 = [torch.from_numpy(m[0]).cuda() for m in mus]
    mu1 = [torch.from_numpy(m[1]).cuda() for m in mus]
    outs = {}
    for flag in (se2ot.SE2OT_FLAG_BATCH_PER_RADIUS, se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH):
        o, _, _ = se2ot.se2ot_interpolate_batched(descs, mu0, mu1, ts, se2ot.solve_opts(iters, flags=flag))
        outs[flag] = [x.clone() for x in o]
    for k in range(2):
        assert torch.equal(outs[se2ot.SE2OT_FLAG_BATCH_PER_RADIUS][k], outs[se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH][k]), k
    nx, ny, nt, r, eps, t = probs[0]
    want = oracle.interpolate_log(oracle.Grid(nx, ny, nt, r, W, eps), mus[0][0].astype(np.float64),
                                  mus[0][1].astype(np.float64), t, iters)
    got = outs[se2ot.SE2OT_FLAG_BATCH_ONE_LAUNCH][0].cpu().double().numpy()
    assert np.abs(got - want).sum() / want.sum() <= 1e-5
