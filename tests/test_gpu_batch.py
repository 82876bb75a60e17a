"""GPU parity of the batched solver (many independent NNCP-HALS problems).

Each tensor of a batch is checked against the FP64 oracle run on that tensor
alone with the same root split (1) and stopping rule; a tensor's result must
be bitwise identical whether it is solved alone or inside a larger batch.
"""

import numpy as np
import pytest

import oracle
from paper_1806_07985_gb300 import synth
from tests._util import ensure_built, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nn():
    ensure_built()
    from paper_1806_07985_gb300 import nncp
    return nncp


def _problems(count, seed0=0, N=3, lo=8, hi=40, ranks=(2, 3, 4, 8)):
    rng = np.random.default_rng(seed0)
    probs = []
    for t in range(count):
        dims = tuple(int(d) for d in rng.integers(lo, hi + 1, size=N))
        R = int(ranks[int(rng.integers(len(ranks)))])
        x, _ = synth.lowrank_plus_noise(dims, R, seed=1000 + seed0 * 97 + t, noise=0.01)
        H0 = synth.init_factors(dims, R, seed=5000 + seed0 * 97 + t)
        probs.append((dims, R, x, H0))
    return probs


def _run_batch(nn, probs, iters, tol=0.0):
    b = nn.Batch([p[0] for p in probs], [p[1] for p in probs], max_iters=max(iters, 1))
    try:
        X = [torch.from_numpy(p[2]).cuda() for p in probs]
        H = [[torch.from_numpy(h.copy()).cuda() for h in p[3]] for p in probs]
        b.set_data(X, H)
        k, fits, lams = b.solve(iters, tol)
        return k, fits, lams, [[h.cpu().numpy() for h in hs] for hs in H]
    finally:
        b.close()


@pytest.mark.parametrize("N", [3, 4, 2])
def test_batch_matches_oracle(nn, N):
    probs = _problems(12 if N == 3 else 6, seed0=N, N=N, hi=40 if N < 4 else 14)
    iters = 10
    k, fits, lams, Hs = _run_batch(nn, probs, iters)
    for t, (dims, R, x, H0) in enumerate(probs):
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=iters, use_dimtree=True, s=1)
        assert k[t] == iters
        assert abs(fits[t] - ref["fits"][-1]) <= 1e-4, (t, dims, R, fits[t], ref["fits"][-1])
        for n in range(N):
            assert rel_fro(Hs[t][n], ref["H"][n]) <= 1e-3, (t, n)
        assert rel_fro(np.array(lams[t]), ref["lam"]) <= 1e-3


def test_batch_results_do_not_depend_on_the_batch(nn):
    probs = _problems(9, seed0=11)
    k_all, f_all, l_all, H_all = _run_batch(nn, probs, 6)
    for t in (0, 4, 8):
        k1, f1, l1, H1 = _run_batch(nn, [probs[t]], 6)
        assert k1[0] == k_all[t] and f1[0] == f_all[t] and l1[0] == l_all[t]
        for a, b in zip(H1[0], H_all[t]):
            assert np.array_equal(a, b)


def test_batch_stops_each_tensor_on_its_own(nn):
    # The rule |fit_k - fit_(k-1)| < tol is a threshold on a float32 fit
    # difference: where the oracle's own change sits within the float32 noise
    # band of tol (the fit identity cancels; ~1e-5 at eps ~ 0.1 on these
    # shapes), the two may stop an iteration or two apart.  Each tensor must
    # stop at an iteration where the oracle's change is below tol + band, and
    # not before one where it is still above tol + band.
    tol, band = 1e-4, 1e-5
    probs = _problems(8, seed0=21)
    k, fits, lams, Hs = _run_batch(nn, probs, 300, tol=tol)
    for t, (dims, R, x, H0) in enumerate(probs):
        H0d = [h.astype(np.float64) for h in H0]
        ref = oracle.nncp_hals(x.astype(np.float64), dims, H0d, max_iters=300, tol=tol,
                               use_dimtree=True, s=1)
        assert k[t] < 300 and 2 <= k[t]
        full = oracle.nncp_hals(x.astype(np.float64), dims, H0d, max_iters=max(k[t], ref["iters"]),
                                tol=0.0, use_dimtree=True, s=1)["fits"]
        change = np.abs(np.diff(full))  # change[j - 2]: iteration j against j - 1
        assert change[k[t] - 2] < tol + band, (t, k[t], change[k[t] - 2])
        assert (change[:k[t] - 2] >= tol - band).all(), (t, k[t])
        assert abs(fits[t] - full[k[t] - 1]) <= 1e-4


def test_batch_rejects_out_of_range_shapes(nn):
    with pytest.raises(nn.NNCPError):
        nn.Batch([(300, 4, 4)], [4], max_iters=4)   # mode longer than 256
    with pytest.raises(nn.NNCPError):
        nn.Batch([(10, 4, 4)], [65], max_iters=4)   # rank above 64


def test_batch_wide_ranks_and_long_modes(nn):
    # ranks up to 64 (the widest kernel instances), a 256-long first mode and
    # ragged shapes; checked against the oracle after a few iterations
    rng = np.random.default_rng(77)
    probs = []
    for t, (dims, R) in enumerate([((256, 9, 7), 5), ((33, 40, 17), 64), ((70, 3, 130), 33),
                                   ((1, 50, 60), 12), ((129, 64, 5), 20)]):
        x, _ = synth.lowrank_plus_noise(dims, R, seed=3000 + t, noise=0.01)
        probs.append((dims, R, x, synth.init_factors(dims, R, seed=4000 + t)))
    iters = 5
    k, fits, lams, Hs = _run_batch(nn, probs, iters)
    for t, (dims, R, x, H0) in enumerate(probs):
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=iters, use_dimtree=True, s=1)
        assert abs(fits[t] - ref["fits"][-1]) <= 1e-4, (t, dims, R)
        for n in range(3):
            assert rel_fro(Hs[t][n], ref["H"][n]) <= 1e-3, (t, n)


@pytest.mark.parametrize("N,lo,hi", [(4, 6, 30), (5, 3, 12)])
def test_batch_higher_orders_larger_nodes(nn, N, lo, hi):
    probs = _problems(5, seed0=40 + N, N=N, lo=lo, hi=hi, ranks=(3, 16, 40))
    iters = 4
    k, fits, lams, Hs = _run_batch(nn, probs, iters)
    for t, (dims, R, x, H0) in enumerate(probs):
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=iters, use_dimtree=True, s=1)
        assert abs(fits[t] - ref["fits"][-1]) <= 1e-4, (t, dims, R)
        for n in range(N):
            assert rel_fro(Hs[t][n], ref["H"][n]) <= 1e-3, (t, n)


def test_batch_bits_do_not_depend_on_the_widest_rank(nn):
    # the same small-rank tensor alone (16-wide kernels) and beside an R=64
    # tensor (64-wide kernels) gives the same bits
    small = _problems(2, seed0=91, ranks=(4,))
    wide = _problems(1, seed0=92, ranks=(64,))
    k1, f1, l1, H1 = _run_batch(nn, small, 6)
    k2, f2, l2, H2 = _run_batch(nn, small + wide, 6)
    for t in range(2):
        assert k1[t] == k2[t] and f1[t] == f2[t] and l1[t] == l2[t]
        for a, b in zip(H1[t], H2[t]):
            assert np.array_equal(a, b)


def test_one_call_batch_solve_mixed_orders(nn):
    # nncp_batch_solve: tensors of orders 3 and 4 interleaved in one call; each
    # order is solved as its own batch, so the bits equal the batch path's, and
    # the results match the oracle
    p3 = _problems(4, seed0=11, N=3, hi=30)
    p4 = _problems(3, seed0=12, N=4, hi=12)
    mixed = [p3[0], p4[0], p3[1], p3[2], p4[1], p4[2], p3[3]]
    iters = 8
    X = [torch.from_numpy(p[2]).cuda() for p in mixed]
    H = [[torch.from_numpy(h.copy()).cuda() for h in p[3]] for p in mixed]
    k, fits, lams = nn.nncp_batch_solve([p[0] for p in mixed], [p[1] for p in mixed], X, H,
                                        iters, 0.0)
    Hs = [[h.cpu().numpy() for h in hs] for hs in H]
    for probs in (p3, p4):
        kb, fb, lb, Hb = _run_batch(nn, probs, iters)
        for i, p in enumerate(probs):
            t = next(j for j, q in enumerate(mixed) if q is p)
            assert k[t] == kb[i] == iters
            assert fits[t] == fb[i]
            assert lams[t] == lb[i]
            for n in range(len(p[0])):
                assert np.array_equal(Hs[t][n], Hb[i][n])
    for t, (dims, R, x, H0) in enumerate(mixed):
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=iters, use_dimtree=True, s=1)
        assert abs(fits[t] - ref["fits"][-1]) <= 1e-4, t
        assert rel_fro(np.array(lams[t]), ref["lam"]) <= 1e-3, t


def test_one_call_batch_solve_rejects_bad_orders(nn):
    dims, R = (8, 6, 5), 2
    X = [torch.zeros(240, device="cuda")]
    H = [[torch.zeros(d, R, device="cuda") for d in dims]]
    with pytest.raises(nn.NNCPError) as info:
        nn.nncp_batch_solve([(8,)], [R], X, [H[0][:1]], 2, 0.0)  # order 1
    assert info.value.status == nn.NNCP_ERR_INVALID_ARG


def _run_batch_sched(nn, probs, iters, sched):
    b = nn.Batch([p[0] for p in probs], [p[1] for p in probs], max_iters=iters)
    try:
        b.set_schedule(*sched)
        X = [torch.from_numpy(p[2]).cuda() for p in probs]
        H = [[torch.from_numpy(h.copy()).cuda() for h in p[3]] for p in probs]
        b.set_data(X, H)
        k, fits, lams = b.solve(iters, 0.0)
        assert b.schedule() == sched
        return k, fits, lams, [[h.cpu().numpy() for h in hs] for hs in H]
    finally:
        b.close()


# batch compositions for the schedule tests: few items; more items than
# resident CTAs (each streamed CTA takes several, its stage ring wraps inside
# and across items); ranks up to 40 (64-wide rank blocks) with first modes
# above 128 (one column group, no group sum); order 4; order 2
_SCHED_SETS = {
    "small": dict(count=10, seed0=31, hi=60),
    "many_items": dict(count=48, seed0=33, lo=40, hi=128, ranks=(4, 8, 16)),
    "wide_rank": dict(count=8, seed0=35, lo=20, hi=200, ranks=(12, 24, 40)),
    "order4": dict(count=8, seed0=37, N=4, lo=6, hi=20, ranks=(3, 5, 8)),
    "order2": dict(count=8, seed0=39, N=2, lo=16, hi=250, ranks=(2, 7, 16)),
    "order5": dict(count=6, seed0=41, N=5, lo=3, hi=11, ranks=(2, 6, 16)),
    "edges": None,   # _edge_problems: first modes 1, 2, 3, 4, 255, 256; ranks 1 and 64
}


def _edge_problems():
    probs = []
    for t, (dims, R) in enumerate([((1, 50, 60), 12), ((256, 9, 7), 5), ((255, 3, 17), 64),
                                   ((2, 2, 2), 1), ((3, 40, 41), 33), ((4, 128, 3), 16),
                                   ((256, 64, 2), 1), ((7, 1, 200), 8)]):
        x, _ = synth.lowrank_plus_noise(dims, R, seed=6000 + t, noise=0.01)
        probs.append((dims, R, x, synth.init_factors(dims, R, seed=7000 + t)))
    return probs


@pytest.mark.parametrize("sched", [(1, 1), (0, 1), (1, 0), (2, 0), (0, 2), (2, 2), (1, 2)])
@pytest.mark.parametrize("which", sorted(_SCHED_SETS))
def test_root_phase_schedules_give_the_same_bits(nn, which, sched):
    # one CTA per work item, persistent CTAs taking items from a counter, or
    # the streamed kernels: which CTA (and which warp) computes a product
    # changes, the order of every output's sums does not
    probs = _edge_problems() if which == "edges" else _problems(**_SCHED_SETS[which])
    ref = _run_batch_sched(nn, probs, 5, (0, 0))
    got = _run_batch_sched(nn, probs, 5, sched)
    assert got[0] == ref[0] and got[1] == ref[1] and got[2] == ref[2]
    for a, c in zip(got[3], ref[3]):
        for x, y in zip(a, c):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("sched", [(2, 0), (0, 2)])
def test_streamed_schedule_reports_an_expired_wait(nn, sched):
    # the failure path without any fault or hang: a wait limit of one cycle
    # makes the streamed kernel's waits that are merely not yet satisfied
    # expire; the run reports NNCP_ERR_TIMEOUT naming the wait site, and the
    # same batch, limit restored, then solves to schedule 0's bits
    probs = _problems(**_SCHED_SETS["many_items"])
    iters = 3
    ref = _run_batch_sched(nn, probs, iters, (0, 0))
    b = nn.Batch([p[0] for p in probs], [p[1] for p in probs], max_iters=iters)
    try:
        with pytest.raises(nn.NNCPError):
            b.set_wait_limit(-1)
        b.set_schedule(*sched)
        X = [torch.from_numpy(p[2]).cuda() for p in probs]
        H = [[torch.from_numpy(h.copy()).cuda() for h in p[3]] for p in probs]
        b.set_data(X, H)
        b.set_wait_limit(1)
        with pytest.raises(nn.NNCPError) as info:
            b.solve(iters, 0.0)
        assert info.value.status == nn.NNCP_ERR_TIMEOUT
        assert "wait site" in str(info.value)
        for hs, p in zip(H, probs):
            for h, h0 in zip(hs, p[3]):
                h.copy_(torch.from_numpy(h0))
        b.set_wait_limit(0)
        k, fits, lams = b.solve(iters, 0.0)
        Hs = [[h.cpu().numpy() for h in hs] for hs in H]
    finally:
        b.close()
    assert k == ref[0] and fits == ref[1] and lams == ref[2]
    for a, c in zip(Hs, ref[3]):
        for x, y in zip(a, c):
            assert np.array_equal(x, y)


def test_streamed_schedule_matches_the_oracle_at_wide_ranks(nn):
    probs = _problems(count=4, seed0=43, lo=24, hi=150, ranks=(24, 40))
    iters = 6
    k, fits, lams, Hs = _run_batch_sched(nn, probs, iters, (2, 2))
    for t, (dims, R, x, H0) in enumerate(probs):
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=iters, use_dimtree=True, s=1)
        assert k[t] == iters
        assert abs(fits[t] - ref["fits"][-1]) <= 1e-4, (t, dims, R)
        assert rel_fro(np.array(lams[t]), ref["lam"]) <= 1e-3, t


def test_schedule_tuner_picks_a_valid_schedule(nn):
    probs = _problems(6, seed0=41)
    b = nn.Batch([p[0] for p in probs], [p[1] for p in probs], max_iters=3)
    try:
        with pytest.raises(nn.NNCPError):
            b.schedule()                     # before the first run
        with pytest.raises(nn.NNCPError):
            b.set_schedule(3, 0)
        with pytest.raises(nn.NNCPError):
            b.set_schedule(0, 3)
        X = [torch.from_numpy(p[2]).cuda() for p in probs]
        H = [[torch.from_numpy(h.copy()).cuda() for h in p[3]] for p in probs]
        b.set_data(X, H)
        b.solve(3, 0.0)
        r, l = b.schedule()
        assert r in (0, 1, 2) and l in (0, 1, 2)
    finally:
        b.close()
