"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (from the method's accuracy targets): MTTKRP relative Frobenius
error <= 1e-5 in the float32-equivalent modes; final fit within 1e-4
(absolute); factors after a short solve within 1e-3 relative Frobenius.
"""

import numpy as np
import pytest

import oracle
from paper_1806_07985_gb300 import synth
from tests._util import ensure_built, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MTTKRP_TOL = 1e-5
FIT_TOL = 1e-4


@pytest.fixture(scope="module")
def nn():
    ensure_built()
    from paper_1806_07985_gb300 import nncp
    return nncp


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ctx(nn, dims, R, x, H, precision=0, split=0):
    c = nn.Context(dims, R, precision=precision, root_split=split)
    X = _dev(x)
    Hd = [_dev(h) for h in H]
    c.set_tensor(X)
    c.set_factors(Hd)
    return c, X, Hd


def _check_mttkrp(nn, dims, R, seed=0, split=0, tol=MTTKRP_TOL):
    rng = np.random.default_rng(seed)
    x = rng.random(int(np.prod(dims))).astype(np.float32)
    H = [rng.random((d, R)).astype(np.float32) for d in dims]
    c, X, Hd = _ctx(nn, dims, R, x, H, split=split)
    s = split or oracle.default_root_split(dims)
    try:
        for n in range(len(dims)):
            ref = oracle.mttkrp_direct(x.astype(np.float64), dims,
                                       [h.astype(np.float64) for h in H], n)
            for tree in (0, 1):
                M = torch.empty((dims[n], R), device="cuda")
                c.mttkrp(n + 1, tree, M)
                torch.cuda.synchronize()
                err = rel_fro(M.cpu().numpy(), ref)
                assert err <= tol, (dims, R, n, tree, s, err)
    finally:
        c.close()


@pytest.mark.parametrize("dims,R", [
    ((64, 64, 64), 8),
    ((37, 23, 29), 5),        # ragged, not multiples of any tile
    ((130, 7, 65), 33),       # R just above one rank tile
    ((1, 9, 1), 1),           # unit modes, R = 1
    ((200, 3), 4),            # N = 2 (matrix)
    ((16, 12, 6, 5), 24),
    ((6, 5, 4, 3, 7), 3),
    ((40, 40, 41), 128),      # maximum rank
])
def test_mttkrp_direct_and_tree_match_oracle(nn, dims, R):
    _check_mttkrp(nn, dims, R)


@pytest.mark.parametrize("split", [1, 2, 3])
def test_mttkrp_every_root_split(nn, split):
    _check_mttkrp(nn, (12, 10, 9, 11), 6, seed=3, split=split)


def test_mttkrp_split_k_many_chunks(nn):
    # I_L small, I_R large: the root->left partial MTTKRP is split over many CTAs
    _check_mttkrp(nn, (8, 300, 300), 16, seed=5)


def _solve_both(nn, dims, R, iters, x, H0, split=0, tol=0.0):
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=iters, tol=tol, use_dimtree=True, s=split or None)
    c, X, Hd = _ctx(nn, dims, R, x, H0, split=split)
    try:
        lam, k, fit = c.solve(iters, tol)
        hist = c.fit_history()
        exact = c.fit(exact=True)
        Hg = [h.cpu().numpy() for h in Hd]
    finally:
        c.close()
    return ref, (np.array(lam), k, fit, hist, exact, Hg)


def test_config1_solve_matches_oracle(nn):
    # 64^3, R = 8, rank-8 U[0,1) + U[0,0.01) noise, init seed 1, 20 iterations
    dims, R = (64, 64, 64), 8
    x, _ = synth.lowrank_plus_noise(dims, R, seed=0, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=1)
    ref, (lam, k, fit, hist, exact, Hg) = _solve_both(nn, dims, R, 20, x, H0)
    assert k == 20
    assert abs(fit - ref["fits"][-1]) <= FIT_TOL
    assert np.max(np.abs(np.array(hist) - np.array(ref["fits"]))) <= FIT_TOL
    for n in range(3):
        assert rel_fro(Hg[n], ref["H"][n]) <= 1e-3
    assert rel_fro(lam, ref["lam"]) <= 1e-3
    eps_oracle = oracle.explicit_residual(x.astype(np.float64), dims, ref["lam"], ref["H"])
    assert abs((1 - exact) - eps_oracle) <= FIT_TOL
    # the identity and the explicit residual agree on the GPU too
    assert abs(exact - fit) <= 1e-5


def test_one_iteration_tight(nn):
    # after a single outer iteration the factors still agree tightly
    dims, R = (33, 47, 21), 7
    x, _ = synth.lowrank_plus_noise(dims, R, seed=8, noise=0.05)
    H0 = synth.init_factors(dims, R, seed=9)
    ref, (lam, k, fit, hist, exact, Hg) = _solve_both(nn, dims, R, 1, x, H0)
    assert k == 1
    for n in range(3):
        assert rel_fro(Hg[n], ref["H"][n]) <= 1e-4, n
    assert rel_fro(lam, ref["lam"]) <= 1e-4
    assert abs(fit - ref["fits"][-1]) <= 1e-6


@pytest.mark.parametrize("dims,R,split", [((32, 32, 8, 4), 6, 2), ((9, 8, 7, 6, 5), 4, 2),
                                          ((50, 3), 2, 1), ((20, 20, 20), 3, 2)])
def test_solve_other_orders_and_splits(nn, dims, R, split):
    x, _ = synth.lowrank_plus_noise(dims, R, seed=11, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=12)
    ref, (lam, k, fit, hist, exact, Hg) = _solve_both(nn, dims, R, 10, x, H0, split=split)
    assert k == 10
    assert np.max(np.abs(np.array(hist) - np.array(ref["fits"]))) <= FIT_TOL
    for n in range(len(dims)):
        assert rel_fro(Hg[n], ref["H"][n]) <= 1e-3, n


def test_convergence_stops_early_like_oracle(nn):
    # the stopping test |fit_k - fit_(k-1)| < tol is a discrete decision: it is
    # compared at a tol well above the float32 noise of the fit identity
    # (eps^2 = (alpha - 2 beta + gamma) / alpha cancels, ~1e-6 at eps ~ 1e-2)
    dims, R = (20, 18, 16), 3
    x, _ = synth.lowrank_plus_noise(dims, R, seed=21, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=22)
    ref, (lam, k, fit, hist, exact, Hg) = _solve_both(nn, dims, R, 500, x, H0, tol=1e-4)
    assert 2 <= ref["iters"] < 500
    assert abs(k - ref["iters"]) <= 1
    # the stop may land one iteration either side; compare at the common iteration
    assert abs(fit - ref["fits"][min(k, ref["iters"]) - 1]) <= FIT_TOL


def test_solve_is_bitwise_reproducible(nn):
    dims, R = (40, 30, 20), 5
    x, _ = synth.lowrank_plus_noise(dims, R, seed=2, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=3)
    outs = []
    for _ in range(2):
        c, X, Hd = _ctx(nn, dims, R, x, H0)
        lam, k, fit = c.solve(8)
        outs.append((lam, fit, [h.cpu().numpy().copy() for h in Hd]))
        c.close()
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1]
    for a, b in zip(outs[0][2], outs[1][2]):
        assert np.array_equal(a, b)


def test_invalid_calls_report_errors(nn):
    c = nn.Context((8, 8, 8), 4)
    try:
        with pytest.raises(nn.NNCPError):
            c.solve(5)  # tensor and factors not set
        X = torch.rand(512, device="cuda")
        c.set_tensor(X)
        H = [torch.rand(8, 4, device="cuda") for _ in range(3)]
        c.set_factors(H)
        M = torch.empty(8, 4, device="cuda")
        with pytest.raises(nn.NNCPError):
            c.mttkrp(4, 0, M)
        with pytest.raises(nn.NNCPError):
            c.mttkrp(0, 1, M)
        with pytest.raises(nn.NNCPError):
            nn.nncp_set_options(c.ctx, 9, 0, None)
    finally:
        c.close()


@pytest.mark.slow
def test_full_size_512cubed_sampled_rows(nn):
    # configs' 512^3, R = 32 tensor: sampled rows of every MTTKRP, direct and tree
    dims, R = (512, 512, 512), 32
    x, _ = synth.lowrank_plus_noise(dims, R, seed=0, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=1)
    c, X, Hd = _ctx(nn, dims, R, x, H0)
    rows = [0, 1, 255, 300, 511]
    xd = x.astype(np.float64)
    Hd64 = [h.astype(np.float64) for h in H0]
    try:
        for n in range(3):
            ref = oracle.mttkrp_rows(xd, dims, Hd64, n, rows)
            for tree in (0, 1):
                M = torch.empty((512, R), device="cuda")
                c.mttkrp(n + 1, tree, M)
                torch.cuda.synchronize()
                err = rel_fro(M.cpu().numpy()[rows], ref)
                assert err <= MTTKRP_TOL, (n, tree, err)
    finally:
        c.close()


@pytest.mark.parametrize("dims,R", [((20, 17, 13), 5), ((9, 7, 8, 6), 4)])
def test_solve_without_dimension_tree_matches_oracle(nn, dims, R):
    # every M(n) by a full MTTKRP (Sec. V-C's comparison): same iteration,
    # checked against the oracle's own direct path
    x, _ = synth.lowrank_plus_noise(dims, R, seed=31, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=32)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=8, use_dimtree=False)
    c, X, Hd = _ctx(nn, dims, R, x, [h.copy() for h in H0])
    try:
        c.set_dimtree(False)
        lam, k, fit = c.solve(8)
        assert k == 8 and abs(fit - ref["fits"][-1]) <= FIT_TOL
        for n in range(len(dims)):
            assert rel_fro(Hd[n].cpu().numpy(), ref["H"][n]) <= 1e-3, n
    finally:
        c.close()


def test_without_dimension_tree_is_fp32_only(nn):
    if "tcgen05" not in nn.nncp_version():
        pytest.skip("no tensor-core path in this build")
    c = nn.Context((32, 16, 8), 4, precision=nn.NNCP_SPLIT_BF16X3)
    try:
        with pytest.raises(nn.NNCPError) as info:
            c.set_dimtree(False)
        assert info.value.status == nn.NNCP_ERR_UNSUPPORTED
    finally:
        c.close()


# Mode-update configurations: the cluster update (I_n <= 1024) with 1-8 CTAs
# of 32, 64 or 128 rows (ragged last CTA), every RMAX variant (R <= 16, <= 32,
# <= 64; R = 1; odd R takes the scalar staging path; R = 33 rotates 64 register
# columns of which 31 are padding), its largest case (1024 rows) and the
# multi-CTA kernel just above it (1025 rows).  FP32 SIMT, so the update is the
# only tensor-core-independent difference from the FP64 oracle.
UPDATE_SHAPES = [
    ((3, 40, 30), 5),       # a 3-row mode: one CTA of 32 rows, 3 used
    ((31, 33, 20), 7),      # odd R, 31- and 33-row modes (1 and 2 CTAs)
    ((100, 64, 10), 16),    # 4 CTAs of 32 rows
    ((512, 20, 8), 24),     # 8 CTAs of 64 rows, R in the 32-column variant
    ((1000, 12, 8), 32),    # 8 CTAs of 128 rows, the last one partial
    ((1024, 10, 6), 33),    # 64-column variant at the largest cluster mode
    ((1025, 10, 6), 8),     # one row more: the multi-CTA kernel
    ((40, 30, 20), 64),     # the maximum rank
    ((64, 48, 20), 1),      # rank one
]


@pytest.mark.parametrize("dims,R", UPDATE_SHAPES)
def test_update_configurations_match_oracle(nn, dims, R):
    x, _ = synth.lowrank_plus_noise(dims, min(R, 8), seed=31, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=32)
    ref, (lam, k, fit, hist, exact, Hg) = _solve_both(nn, dims, R, 3, x, H0, split=1)
    assert k == 3
    assert np.max(np.abs(np.array(hist) - np.array(ref["fits"]))) <= FIT_TOL
    for n in range(len(dims)):
        assert rel_fro(Hg[n], ref["H"][n]) <= 1e-4, n
    assert rel_fro(lam, ref["lam"]) <= 1e-4


def test_solve_with_tensor_and_factors_in_the_call(nn):
    # nncp_solve(ctx, X, H, ...) binds the tensor and factors itself: the same
    # bits as binding them first and calling nncp_solve_bound, and the oracle's
    # result
    dims, R = (30, 26, 22), 5
    x, _ = synth.lowrank_plus_noise(dims, R, seed=41, noise=0.01)
    H0 = synth.init_factors(dims, R, seed=42)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=6, use_dimtree=True)
    c, X, Hd = _ctx(nn, dims, R, x, H0)
    try:
        lam_a, k_a, fit_a = c.solve(6)
        Ha = [h.cpu().numpy() for h in Hd]
        H2 = [_dev(h) for h in H0]
        X2 = _dev(x)
        lam_b, k_b, fit_b = c.solve_on(X2, H2, 6)
        Hb = [h.cpu().numpy() for h in H2]
        # the pointers just bound again: graphs kept, same bits
        for h, h0 in zip(H2, H0):
            h.copy_(torch.from_numpy(h0))
        lam_c, k_c, fit_c = c.solve_on(X2, H2, 6)
    finally:
        c.close()
    assert k_a == k_b == k_c == 6
    assert lam_a == lam_b == lam_c and fit_a == fit_b == fit_c
    for a, b in zip(Ha, Hb):
        assert np.array_equal(a, b)
    assert abs(fit_b - ref["fits"][-1]) <= FIT_TOL
    for n in range(3):
        assert rel_fro(Hb[n], ref["H"][n]) <= 1e-3
