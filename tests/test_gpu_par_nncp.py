"""GPU parity of Par-NNCP (Alg. 2) and of the cached dimension-tree MTTKRP.

Par-NNCP: every processor of a P_1 x ... x P_N grid is a library object
(nncp_par_*) with its own tensor block and workspace on this one GPU; the
driver's LocalComm runs the collectives among them inside the process (the
processors' kernels never wait on one another: the exchange is on the host
between launches).  The result is compared with the FP64 oracle on the whole
tensor (fit 1e-4, factors and lambda 1e-3).

nncp_mttkrp_cached: in BCD order, each factor changed and reported after its
MTTKRP, every M(n) equals the oracle's MTTKRP for the current factors.
"""

import numpy as np
import pytest

import oracle
from paper_1806_07985_gb300 import par_nncp, synth
from tests._util import ensure_built, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nn():
    ensure_built()
    from paper_1806_07985_gb300 import nncp
    return nncp


def _procs(nn, x, H0, dims, grid, R, precision="fp32_simt"):
    procs = {}
    for r in range(int(np.prod(grid))):
        coords = par_nncp.grid_coords(r, grid)
        eng = nn.ParRank(dims, grid, coords, R, precision=precision)
        layouts = [eng.layout(n + 1) for n in range(len(dims))]
        X = torch.from_numpy(par_nncp.local_block(x, dims, grid, coords)).cuda()
        H = []
        for n, h in enumerate(H0):
            lo, rows = layouts[n][0], layouts[n][1]
            H.append(torch.from_numpy(np.ascontiguousarray(h[lo:lo + rows])).cuda())
        procs[r] = par_nncp.Processor(eng, X, H, layouts)
    return procs


def _assemble(procs, dims, R):
    out = [np.full((I, R), np.nan, dtype=np.float32) for I in dims]
    for p in procs.values():
        for n in range(len(dims)):
            _, _, lo, rows, _, _ = p.layouts[n]
            out[n][lo:lo + rows] = p.owned(n).cpu().numpy()
    return out


@pytest.mark.parametrize("dims,grid,R,prec", [
    ((24, 20, 16), (2, 1, 1), 4, "fp32_simt"),
    ((24, 20, 16), (2, 2, 1), 5, "fp32_simt"),
    ((21, 19, 17), (1, 3, 2), 3, "fp32_simt"),      # ragged blocks, uneven owned pieces
    ((12, 10, 8, 6), (2, 1, 2, 1), 4, "fp32_simt"),
    ((64, 48, 40), (2, 1, 2), 8, "split_bf16x3"),    # tensor-core local MTTKRPs
    ((20, 16, 12), (1, 1, 1), 4, "fp32_simt"),       # one processor
])
def test_par_nncp_matches_the_oracle(nn, dims, grid, R, prec):
    if prec != "fp32_simt" and "tcgen05" not in nn.nncp_version():
        pytest.skip("no tensor-core path in this build")
    x, _ = synth.lowrank_plus_noise(dims, R, seed=21, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=22)
    iters = 8
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=iters, use_dimtree=False)
    procs = _procs(nn, x, H0, dims, grid, R, prec)
    try:
        lams, fits, k = par_nncp.solve(procs, par_nncp.LocalComm(grid), iters)
        assert k == iters
        for r in procs:
            assert np.max(np.abs(np.array(fits[r]) - np.array(ref["fits"]))) <= 1e-4, r
            assert rel_fro(np.array(lams[r]), ref["lam"]) <= 1e-3
        for n, Hn in enumerate(_assemble(procs, dims, R)):
            assert rel_fro(Hn, ref["H"][n]) <= 1e-3, n
    finally:
        for p in procs.values():
            p.engine.close()


def test_par_nncp_stops_like_the_oracle(nn):
    dims, grid, R = (20, 18, 16), (2, 2, 1), 3
    x, _ = synth.lowrank_plus_noise(dims, R, seed=31, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=32)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=300, tol=1e-4, use_dimtree=False)
    procs = _procs(nn, x, H0, dims, grid, R)
    try:
        lams, fits, k = par_nncp.solve(procs, par_nncp.LocalComm(grid), 300, tol=1e-4)
    finally:
        for p in procs.values():
            p.engine.close()
    assert 2 <= ref["iters"] < 300 and abs(k - ref["iters"]) <= 1
    assert abs(fits[0][min(k, ref["iters"]) - 1] - ref["fits"][min(k, ref["iters"]) - 1]) <= 1e-4


def test_par_create_rejects_bad_grids(nn):
    with pytest.raises(nn.NNCPError):
        nn.ParRank((8, 8, 8), (2, 2, 2), (2, 0, 0), 4)      # coordinate outside the grid
    with pytest.raises(nn.NNCPError):
        nn.ParRank((3, 8, 8), (4, 1, 1), (0, 0, 0), 4)      # more blocks than rows


@pytest.mark.parametrize("dims,R,split,prec", [((12, 10, 9, 8), 5, 2, "fp32_simt"),
                                                ((9, 8, 7, 6, 5), 3, 3, "fp32_simt"),
                                                ((64, 16, 12, 10), 8, 2, "split_bf16x3")])
def test_cached_tree_mttkrp_in_bcd_order(nn, dims, R, split, prec):
    if prec != "fp32_simt" and "tcgen05" not in nn.nncp_version():
        pytest.skip("no tensor-core path in this build")
    rng = np.random.default_rng(5)
    x = rng.random(int(np.prod(dims))).astype(np.float32)
    H = [rng.random((d, R)).astype(np.float32) for d in dims]
    c = nn.Context(dims, R, precision=prec, root_split=split)
    try:
        X = torch.from_numpy(x).cuda()
        Hd = [torch.from_numpy(h.copy()).cuda() for h in H]
        c.set_tensor(X)
        c.set_factors(Hd)
        tol = 1e-5
        for sweep in range(2):
            for n in range(len(dims)):
                M = torch.empty((dims[n], R), device="cuda")
                c.mttkrp_cached(n + 1, M)
                torch.cuda.synchronize()
                ref = oracle.mttkrp_direct(x.astype(np.float64), dims,
                                           [h.cpu().numpy().astype(np.float64) for h in Hd], n)
                assert rel_fro(M.cpu().numpy(), ref) <= tol, (sweep, n)
                # a new factor n, as a BCD update would leave it
                Hd[n].copy_(torch.from_numpy(rng.random((dims[n], R)).astype(np.float32)))
                c.factor_changed(n + 1)
    finally:
        c.close()


def test_cached_tree_keeps_nodes_until_a_factor_is_reported(nn):
    # without the report, a node contracted with the old factor is reused:
    # the documented contract (and the saving) of the cache
    dims, R = (10, 9, 8, 7), 3
    rng = np.random.default_rng(9)
    x = rng.random(int(np.prod(dims))).astype(np.float32)
    H = [rng.random((d, R)).astype(np.float32) for d in dims]
    c = nn.Context(dims, R, root_split=2)
    try:
        X = torch.from_numpy(x).cuda()
        Hd = [torch.from_numpy(h.copy()).cuda() for h in H]
        c.set_tensor(X)
        c.set_factors(Hd)
        M = torch.empty((dims[1], R), device="cuda")
        c.mttkrp_cached(2, M)
        old = M.clone()
        Hd[3].mul_(2.0)             # mode 4 lies outside node {1, 2}
        c.mttkrp_cached(2, M)
        assert torch.equal(M, old)  # not reported: the cached node is reused
        c.factor_changed(4)
        c.mttkrp_cached(2, M)
        torch.testing.assert_close(M, 2.0 * old, rtol=1e-5, atol=0)
    finally:
        c.close()
