"""GPU tests of the serving loop (continuous batching of solve requests).

Each request is one NNCP-HALS problem.  Small requests share the batched
iteration (root split 1): they are checked against the FP64 oracle, against
the batched solver (the same kernels, so the same bits) and for independence
from whatever else the server is running.  Large requests run the
single-problem solver: the same bits as nncp_solve_host.
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


def _request(seed, N, lo, hi, ranks):
    rng = np.random.default_rng(seed)
    dims = tuple(int(d) for d in rng.integers(lo, hi + 1, size=N))
    R = int(ranks[int(rng.integers(len(ranks)))])
    x, _ = synth.lowrank_plus_noise(dims, R, seed=seed + 1, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=seed + 2)
    return dims, R, x, H0


def _mix():
    return [_request(100 + 7 * q, N, lo, hi, ranks) for q, (N, lo, hi, ranks) in enumerate(
        [(3, 8, 40, (3, 8)), (4, 5, 16, (4, 16)), (5, 3, 8, (2, 5)), (3, 20, 60, (16, 33)),
         (4, 4, 12, (8,)), (3, 2, 9, (1, 2))])]


def _solve_all(nn, reqs, iters, tol=0.0, budget=1 << 30, slots=64):
    srv = nn.Server(budget, slots)
    try:
        tickets = [srv.submit(d, R, x, H0, iters, tol) for d, R, x, H0 in reqs]
        out = [srv.wait(t, 120000) for t in tickets]
        stats = srv.stats()
        for t in tickets:
            srv.release(t)
        return out, stats
    finally:
        srv.close()


def test_server_matches_oracle(nn):
    reqs = _mix()
    iters = 6
    out, stats = _solve_all(nn, reqs, iters)
    assert stats["completed"] == len(reqs)
    for (dims, R, x, H0), res in zip(reqs, out):
        assert res["status"] == 0 and res["iters"] == iters
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=iters, use_dimtree=True, s=1)
        assert abs(res["fit"] - ref["fits"][-1]) <= 1e-4, (dims, R)
        for n in range(len(dims)):
            assert rel_fro(res["H"][n], ref["H"][n]) <= 1e-3, (dims, R, n)
        assert rel_fro(res["lambda"], ref["lam"]) <= 1e-3
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]


def test_server_stops_each_request_on_its_own_rule(nn):
    reqs = _mix()[:4]
    out, _ = _solve_all(nn, reqs, 300, tol=1e-4)
    for (dims, R, x, H0), res in zip(reqs, out):
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=300, tol=1e-4, use_dimtree=True, s=1)
        assert res["iters"] < 300
        assert abs(res["iters"] - ref["iters"]) <= 1, (dims, R, res["iters"], ref["iters"])
        assert abs(res["fit"] - ref["fits"][min(res["iters"], ref["iters"]) - 1]) <= 1e-4


def test_server_bits_match_batch_and_do_not_depend_on_the_mix(nn):
    reqs = _mix()
    target = reqs[3]
    alone, _ = _solve_all(nn, [target], 7)
    mixed, _ = _solve_all(nn, reqs[:3] + [target] + reqs[4:], 7, slots=3)
    a, m = alone[0], mixed[3]
    assert a["iters"] == m["iters"] and a["fit"] == m["fit"]
    assert np.array_equal(a["lambda"], m["lambda"])
    for u, v in zip(a["H"], m["H"]):
        assert np.array_equal(u, v)
    # the batched solver runs the same kernels: same bits
    dims, R, x, H0 = target
    b = nn.Batch([dims], [R], max_iters=7)
    try:
        H = [torch.from_numpy(h.copy()).cuda() for h in H0]
        b.set_data([torch.from_numpy(x).cuda()], [H])
        k, fits, lams = b.solve(7, 0.0)
    finally:
        b.close()
    assert k[0] == a["iters"] and fits[0] == a["fit"]
    for u, v in zip(H, a["H"]):
        assert np.array_equal(u.cpu().numpy(), v)


def test_server_admission_respects_budget_and_slots(nn):
    reqs = [_request(900 + q, 3, 30, 40, (8,)) for q in range(6)]
    probe = nn.Server(1 << 30, 1)
    need = max(probe.footprint(d, R, 5) for d, R, _, _ in reqs)
    probe.close()
    out, stats = _solve_all(nn, reqs, 5, budget=2 * need + 4096)
    assert stats["completed"] == 6
    assert stats["peak_bytes_in_use"] <= stats["budget"]
    assert stats["peak_active"] <= 2
    assert all(r["status"] == 0 for r in out)
    out, stats = _solve_all(nn, reqs, 5, slots=1)
    assert stats["peak_active"] == 1 and stats["completed"] == 6
    # FIFO with one slot: each request is admitted after the previous one is done
    for p, q in zip(out, out[1:]):
        assert q["t_admit"] >= p["t_done"]


def test_server_rejects_what_cannot_run(nn):
    srv = nn.Server(1 << 20, 4)
    try:
        d, R, x, H0 = _request(5, 3, 60, 64, (16,))
        with pytest.raises(nn.NNCPError):          # footprint above the 1 MiB budget
            srv.submit(d, R, x, H0, 5, 0.0)
        with pytest.raises(nn.NNCPError):          # mode longer than 256
            srv.submit((300, 2, 2), 2, np.ones(1200, np.float32),
                       [np.ones((300, 2), np.float32), np.ones((2, 2), np.float32),
                        np.ones((2, 2), np.float32)], 5, 0.0)
        with pytest.raises(nn.NNCPError):          # rank above 64
            srv.submit((4, 4, 4), 65, np.ones(64, np.float32),
                       [np.ones((4, 65), np.float32)] * 3, 5, 0.0)
    finally:
        srv.close()


def test_server_poll_and_bounded_wait(nn):
    srv = nn.Server(1 << 30, 8)
    try:
        d, R, x, H0 = _request(11, 3, 60, 64, (16,))
        t = srv.submit(d, R, x, H0, 3000, 0.0)
        assert srv.poll(t) is None
        with pytest.raises(TimeoutError):
            srv.wait(t, 0)
        res = srv.wait(t, 120000)
        assert res["status"] == 0 and res["iters"] == 3000
        assert srv.poll(t)["iters"] == 3000
        srv.release(t)
        with pytest.raises(nn.NNCPError):
            srv.release(t)
    finally:
        srv.close()


@pytest.mark.parametrize("precision", ["fp32_simt", "split_bf16x3"])
def test_server_solo_lane_is_the_single_problem_solver(nn, precision):
    # a request of >= NNCP_SERVER_SOLO_ELEMS elements runs the single-problem
    # solver on its own stream: same bits as nncp_solve_host with root_split 0
    if precision != "fp32_simt" and "tcgen05" not in nn.nncp_version():
        pytest.skip("no tensor-core path in this build")
    dims, R = (160, 160, 170), 16
    assert dims[0] * dims[1] * dims[2] >= (1 << 22)
    x, _ = synth.lowrank_plus_noise(dims, R, seed=71, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=72)
    small = _mix()[:3]
    srv = nn.Server(1 << 32, 8)
    try:
        tk = [srv.submit(d, r, xx, h, 6, 0.0) for d, r, xx, h in small[:2]]
        big = srv.submit(dims, R, x, H0, 6, 0.0, precision=precision)
        tk.append(srv.submit(*small[2][:2], small[2][2], small[2][3], 6, 0.0))
        res = srv.wait(big, 120000)
        others = [srv.wait(t, 120000) for t in tk]
    finally:
        srv.close()
    assert res["status"] == 0 and res["iters"] == 6
    assert all(o["status"] == 0 and o["iters"] == 6 for o in others)
    Hh = [h.copy() for h in H0]
    lam, k, fit = nn.nncp_solve_host(dims, R, x, Hh, precision, 0, 6, 0.0)
    assert k == res["iters"] and fit == res["fit"]
    assert np.array_equal(np.array(lam), res["lambda"])
    for a, b in zip(Hh, res["H"]):
        assert np.array_equal(a, b)
    if precision == "fp32_simt":
        ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                               max_iters=6, use_dimtree=True, s=nn.nncp_default_split(dims))
        assert abs(res["fit"] - ref["fits"][-1]) <= 1e-4
        for n in range(3):
            assert rel_fro(res["H"][n], ref["H"][n]) <= 1e-3


def test_server_solo_lane_pads_like_solve_host(nn):
    # no root split of (161, 163, 165) tiles for tensor cores: the solo lane
    # pads mode 1 to 164 exactly as nncp_solve_host does (same bits)
    if "tcgen05" not in nn.nncp_version():
        pytest.skip("no tensor-core path in this build")
    dims, R = (161, 163, 165), 12
    assert dims[0] * dims[1] * dims[2] >= (1 << 22)
    x, _ = synth.lowrank_plus_noise(dims, R, seed=81, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=82)
    srv = nn.Server(1 << 32, 4)
    try:
        res = srv.wait(srv.submit(dims, R, x, H0, 5, 0.0, precision="split_bf16x3"), 120000)
    finally:
        srv.close()
    Hh = [h.copy() for h in H0]
    lam, k, fit = nn.nncp_solve_host(dims, R, x, Hh, "split_bf16x3", 0, 5, 0.0)
    assert res["iters"] == k == 5 and res["fit"] == fit
    for a, b in zip(Hh, res["H"]):
        assert a.shape == b.shape and np.array_equal(a, b)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=5, use_dimtree=True, s=nn.nncp_default_split((164, 163, 165)))
    assert abs(res["fit"] - ref["fits"][-1]) <= 1e-4
    for n in range(3):
        assert rel_fro(res["H"][n], ref["H"][n]) <= 1e-3


def test_server_borrowed_tensor_gives_the_same_bits(nn):
    # borrow_x: the server uploads from the caller's (page-locked) tensor at
    # admission instead of copying it at submit; results are the same bits
    small = _mix()[:3]
    dims, R = (160, 160, 170), 16
    x, _ = synth.lowrank_plus_noise(dims, R, seed=91, noise=0.01)
    big = (dims, R, x, synth.init_factors(dims, R, seed=92))
    reqs = small + [big]
    outs = []
    for borrow in (False, True):
        srv = nn.Server(1 << 32, 8)
        try:
            xs = [torch.from_numpy(q[2]).pin_memory() if borrow else q[2] for q in reqs]
            tk = [srv.submit(q[0], q[1], xx, q[3], 6, 0.0, precision="split_bf16x3", borrow=borrow)
                  for q, xx in zip(reqs, xs)]
            outs.append([srv.wait(t, 120000) for t in tk])
        finally:
            srv.close()
    for a, b in zip(*outs):
        assert a["status"] == b["status"] == 0 and a["iters"] == b["iters"] == 6
        assert a["fit"] == b["fit"]
        for u, v in zip(a["H"], b["H"]):
            assert np.array_equal(u, v)
