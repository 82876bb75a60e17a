"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one oracle function to a brute-force definition, a closed form,
a library routine on the equivalent problem, or an invariant the mathematics
fixes, so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails here.  The last tests plant such mistakes in the oracle and
check that a pin catches each one.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1806_07985_gb300 import synth


def _flat_pos(idx, dims):
    # mode-1-fastest position, written out for the test (Sec. IV-C layout)
    pos = 0
    for k in reversed(range(len(dims))):
        pos = pos * dims[k] + idx[k]
    return pos


def _brute_mttkrp(x, dims, H, n):
    """M(n)(i, r) = sum over all other indices of X(i_1..i_N) prod_{k!=n} H_k(i_k, r)."""
    R = H[0].shape[1]
    M = np.zeros((dims[n], R))
    for idx in itertools.product(*[range(d) for d in dims]):
        v = x[_flat_pos(idx, dims)]
        for r in range(R):
            p = v
            for k in range(len(dims)):
                if k != n:
                    p *= H[k][idx[k], r]
            M[idx[n], r] += p
    return M


def _random_case(rng, N, R):
    dims = tuple(int(d) for d in rng.integers(1, 6, size=N))
    x = rng.standard_normal(int(np.prod(dims)))
    H = [rng.standard_normal((d, R)) for d in dims]
    return dims, x, H


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_mttkrp_direct_and_tree_match_brute_force(N):
    rng = np.random.default_rng(100 + N)
    for trial in range(4):
        R = int(rng.integers(1, 5))
        dims, x, H = _random_case(rng, N, R)
        if trial == 0:
            dims = tuple(range(2, 2 + N))  # all lengths distinct
            x = rng.standard_normal(int(np.prod(dims)))
            H = [rng.standard_normal((d, R)) for d in dims]
        for n in range(N):
            ref = _brute_mttkrp(x, dims, H, n)
            scale = max(1.0, np.abs(ref).max())
            got = oracle.mttkrp_direct(x, dims, H, n)
            assert np.abs(got - ref).max() <= 1e-12 * scale
            for s in range(1, N):
                got_t = oracle.mttkrp_dimtree(x, dims, H, n, s)
                assert np.abs(got_t - ref).max() <= 1e-12 * scale
            got_rows = oracle.mttkrp_rows(x, dims, H, n, list(range(dims[n])))
            assert np.abs(got_rows - ref).max() <= 1e-12 * scale


def test_mttkrp_rank_one_closed_form():
    # X = a_1 o ... o a_N  =>  M(n)(i, r) = a_n(i) * prod_{k!=n} <a_k, H_k(:, r)>
    rng = np.random.default_rng(7)
    dims = (7, 5, 6, 4)
    a = [rng.random(d) for d in dims]
    x = np.zeros(int(np.prod(dims)))
    for idx in itertools.product(*[range(d) for d in dims]):
        x[_flat_pos(idx, dims)] = np.prod([a[k][idx[k]] for k in range(4)])
    R = 3
    H = [rng.random((d, R)) for d in dims]
    for n in range(4):
        coef = np.ones(R)
        for k in range(4):
            if k != n:
                coef *= a[k] @ H[k]
        expect = np.outer(a[n], coef)
        assert np.allclose(oracle.mttkrp_direct(x, dims, H, n), expect, rtol=1e-13, atol=0)
        for s in (1, 2, 3):
            assert np.allclose(oracle.mttkrp_dimtree(x, dims, H, n, s), expect,
                               rtol=1e-13, atol=0)


def test_partial_mttkrp_nodes_are_contractions_of_the_tensor():
    # T_L(i_1..i_s, r) = sum_{i_{s+1}..i_N} X * prod_{k>s} H_k ; T_R likewise
    rng = np.random.default_rng(11)
    dims = (3, 4, 2, 5)
    R = 2
    x = rng.standard_normal(int(np.prod(dims)))
    H = [rng.standard_normal((d, R)) for d in dims]
    for s in (1, 2, 3):
        IL = int(np.prod(dims[:s]))
        TL = np.zeros((IL, R))
        TR = np.zeros((x.size // IL, R))
        for idx in itertools.product(*[range(d) for d in dims]):
            v = x[_flat_pos(idx, dims)]
            left = _flat_pos(idx[:s], dims[:s])
            right = _flat_pos(idx[s:], dims[s:])
            for r in range(R):
                TL[left, r] += v * np.prod([H[k][idx[k], r] for k in range(s, 4)])
                TR[right, r] += v * np.prod([H[k][idx[k], r] for k in range(s)])
        assert np.allclose(oracle.partial_mttkrp_right(x, dims, H, s), TL, rtol=1e-12, atol=1e-12)
        assert np.allclose(oracle.partial_mttkrp_left(x, dims, H, s), TR, rtol=1e-12, atol=1e-12)


def test_default_root_split_balances_halves():
    assert oracle.default_root_split((512, 512, 512)) == 1
    assert oracle.default_root_split((512, 512, 32, 16)) == 1  # tie -> smaller s
    assert oracle.default_root_split((100, 512, 32, 16)) == 2
    assert oracle.default_root_split((64,) * 5) == 2
    assert oracle.default_root_split((10, 20)) == 1


def test_hals_rank_one_is_scalar_nnls():
    # R = 1: one column step is the exact minimiser w = max(0, m / s)
    rng = np.random.default_rng(3)
    for _ in range(20):
        I = 9
        M = rng.standard_normal((I, 1))
        S = np.array([[rng.random() + 0.1]])
        W = rng.random((I, 1)) * 5
        oracle.hals_sweep(W, M, S)
        assert np.allclose(W[:, 0], np.maximum(0.0, M[:, 0] / S[0, 0]), rtol=1e-14, atol=0)


def _nnls_by_active_sets(S, m):
    """Exact min_{w>=0} 1/2 w^T S w - m^T w by enumerating passive sets."""
    R = len(m)
    for k in range(R + 1):
        for P in itertools.combinations(range(R), k):
            w = np.zeros(R)
            if P:
                P = list(P)
                w[P] = np.linalg.solve(S[np.ix_(P, P)], m[P])
            if np.all(w >= -1e-12) and np.all(S @ w - m >= -1e-10):
                return w
    raise AssertionError("no KKT point")


@pytest.mark.parametrize("R", [2, 3, 4, 5, 6])
def test_hals_converges_to_exact_nnls(R):
    scipy_optimize = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(20 + R)
    A0 = rng.random((3 * R, R)) + 0.2 * np.eye(3 * R, R)
    S = A0.T @ A0
    I = 6
    M = rng.standard_normal((I, R)) * 3
    W = rng.random((I, R))
    for _ in range(4000):
        oracle.hals_sweep(W, M, S)
    # equivalent least squares: A^T A = S, A^T b = m
    A = np.linalg.cholesky(S).T
    for i in range(I):
        b = np.linalg.solve(A.T, M[i])
        w_ref, _ = scipy_optimize.nnls(A, b)
        assert np.allclose(W[i], w_ref, atol=1e-8)
        if R <= 5:
            assert np.allclose(W[i], _nnls_by_active_sets(S, M[i]), atol=1e-8)
    # KKT: W >= 0, Q = W S - M >= 0, complementarity
    Q = W @ S - M
    assert W.min() >= 0
    assert Q.min() >= -1e-9
    assert np.abs(W * Q).max() <= 1e-9


def test_hals_sweep_never_increases_objective():
    rng = np.random.default_rng(5)
    for _ in range(200):
        R = int(rng.integers(1, 8))
        A0 = rng.random((2 * R + 1, R))
        S = A0.T @ A0
        M = rng.standard_normal((5, R))
        W = rng.random((5, R))
        before = oracle.hals_objective(W, M, S)
        oracle.hals_sweep(W, M, S)
        after = oracle.hals_objective(W, M, S)
        assert after <= before + 1e-12 * max(1.0, abs(before))
        assert W.min() >= 0


def test_normalization_leaves_model_unchanged():
    rng = np.random.default_rng(9)
    dims = (4, 3, 5)
    R = 3
    W = [rng.random((d, R)) for d in dims]
    x_before = oracle.reconstruct(np.ones(R), W, dims)
    lam = np.ones(R)
    H = []
    for w in W:
        h, c = oracle.normalize_columns(w)
        H.append(h)
        lam = lam * c
    assert np.allclose(oracle.reconstruct(lam, H, dims), x_before, rtol=1e-13)
    for h in H:
        assert np.allclose(np.linalg.norm(h, axis=0), 1.0, rtol=1e-14)


def test_reconstruct_matches_generator_layout():
    # the generator's model tensor and the oracle's reconstruction agree entrywise
    # with the written-out definition at a few positions
    rng = np.random.default_rng(1)
    dims = (3, 4, 2)
    F = [rng.random((d, 2)) for d in dims]
    x = synth.model_tensor(F, dims)
    y = oracle.reconstruct(np.ones(2), F, dims)
    for idx in itertools.product(*[range(d) for d in dims]):
        v = sum(F[0][idx[0], r] * F[1][idx[1], r] * F[2][idx[2], r] for r in range(2))
        assert abs(x[_flat_pos(idx, dims)] - v) < 1e-14
        assert abs(y[_flat_pos(idx, dims)] - v) < 1e-14


def _small_noisy(dims, R, seed=0):
    x, _ = synth.lowrank_plus_noise(dims, R, seed, noise=0.05)
    H0 = synth.init_factors(dims, R, seed + 1)
    return x.astype(np.float64), H0


def test_fit_identity_matches_explicit_residual():
    dims, R = (6, 7, 5), 3
    x, H0 = _small_noisy(dims, R)
    for use_tree in (False, True):
        res = oracle.nncp_hals(x, dims, H0, max_iters=15, use_dimtree=use_tree)
        eps_exact = oracle.explicit_residual(x, dims, res["lam"], res["H"])
        assert eps_exact > 1e-3
        assert abs(res["eps"][-1] - eps_exact) < 1e-10


def test_objective_nonincreasing_over_inner_iterations():
    dims, R = (5, 6, 4, 3), 3
    x, H0 = _small_noisy(dims, R, seed=4)
    trace = []

    def cb(event, H, lam, **_):
        trace.append(np.sum((x - oracle.reconstruct(lam, H, dims)) ** 2))

    oracle.nncp_hals(x, dims, H0, max_iters=10, use_dimtree=True, s=2, callback=cb)
    assert len(trace) == 40
    for a, b in zip(trace, trace[1:]):
        assert b <= a * (1 + 1e-12)


def test_tree_and_direct_solves_agree():
    dims, R = (6, 5, 4, 3), 4
    x, H0 = _small_noisy(dims, R, seed=2)
    direct = oracle.nncp_hals(x, dims, H0, max_iters=12, use_dimtree=False)
    for s in (1, 2, 3):
        tree = oracle.nncp_hals(x, dims, H0, max_iters=12, use_dimtree=True, s=s)
        assert np.allclose(tree["fits"], direct["fits"], rtol=0, atol=1e-12)
        for a, b in zip(tree["H"], direct["H"]):
            assert np.allclose(a, b, rtol=0, atol=1e-10)


def _recovery_run(dims, R, seed, max_iters=5000):
    rng = np.random.default_rng(seed)
    F = [rng.random((d, R)) for d in dims]
    x = synth.model_tensor(F, dims)  # exact, noise free, float64
    H0 = [f + 1e-2 * rng.random(f.shape) for f in F]
    res = oracle.nncp_hals(x, dims, H0, max_iters=max_iters, tol=0.0, use_dimtree=True)
    return oracle.explicit_residual(x, dims, res["lam"], res["H"]), res


@pytest.mark.parametrize("dims,R", [((8, 9, 10), 3), ((6, 7, 5, 4), 2)])
def test_exact_low_rank_recovery(dims, R):
    # noise-free nonnegative rank-R tensor, started from the truth perturbed by 1e-2
    # (the paper only states that the residual goes to zero, Sec. V-A)
    eps, res = _recovery_run(dims, R, seed=31)
    assert eps < 1e-10, eps


def test_exact_low_rank_recovery_random_start():
    # a random start on an exact rank-2 model also drives the residual to zero
    dims, R = (8, 9, 10), 2
    rng = np.random.default_rng(17)
    F = [rng.random((d, R)) for d in dims]
    x = synth.model_tensor(F, dims)
    H0 = synth.init_factors(dims, R, 18)
    res = oracle.nncp_hals(x, dims, H0, max_iters=3000, tol=0.0)
    assert oracle.explicit_residual(x, dims, res["lam"], res["H"]) < 1e-10


# ---- the pins have teeth: plant a mistake in the oracle, a pin must fail ----

def test_planted_krp_order_mistake_is_caught(monkeypatch):
    def wrong_krp(A, B):
        A = np.asarray(A, dtype=np.float64)
        B = np.asarray(B, dtype=np.float64)
        K = np.empty((A.shape[0] * B.shape[0], A.shape[1]))
        for c in range(A.shape[1]):
            K[:, c] = np.kron(B[:, c], A[:, c])  # operands swapped
        return K

    monkeypatch.setattr(oracle.nncp, "khatri_rao", wrong_krp)
    with pytest.raises(AssertionError):
        test_mttkrp_direct_and_tree_match_brute_force(3)


def test_planted_hals_sign_mistake_is_caught(monkeypatch):
    def wrong_sweep(W, M, S):
        for r in range(W.shape[1]):
            W[:, r] = np.maximum(0.0, W[:, r] + (M[:, r] + W @ S[:, r]) / S[r, r])
        return W

    monkeypatch.setattr(oracle, "hals_sweep", wrong_sweep)
    with pytest.raises(AssertionError):
        test_hals_rank_one_is_scalar_nnls()


def test_planted_fit_mistake_is_caught(monkeypatch):
    def wrong_fit(alpha, M_N, W_N, lam, S_N, G_N):
        beta = float(np.sum(M_N * W_N))
        gamma = float(lam @ (S_N * G_N) @ lam)
        return math.sqrt(max(0.0, alpha - beta + gamma) / alpha), beta, gamma

    monkeypatch.setattr(oracle.nncp, "fit_identity", wrong_fit)
    with pytest.raises(AssertionError):
        test_fit_identity_matches_explicit_residual()


# ---- block principal pivoting (Alg. 1's NLS-Update solved exactly) --------

@pytest.mark.parametrize("R", [1, 2, 3, 5, 8, 16, 32])
def test_bpp_satisfies_kkt_and_matches_library_nnls(R):
    # the NNLS solution is unique for positive definite S: KKT conditions,
    # scipy's Lawson-Hanson NNLS on the equivalent least squares, and (small
    # R) the brute-force enumeration of active sets must all agree
    scipy_optimize = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(70 + R)
    for _ in range(20):
        A = rng.standard_normal((2 * R + 3, R))
        b = rng.standard_normal(2 * R + 3)
        S, m = A.T @ A, A.T @ b
        x = oracle.nnls_bpp(S, m)
        y = S @ x - m
        scale = max(1.0, float(np.abs(m).max()))
        assert x.min() >= 0.0
        assert y.min() >= -1e-9 * scale
        assert np.abs(x * y).max() <= 1e-9 * scale * scale
        x_ref, _ = scipy_optimize.nnls(A, b)
        assert np.allclose(x, x_ref, atol=1e-8)
        if R <= 5:
            assert np.allclose(x, _nnls_by_active_sets(S, m), atol=1e-8)


def test_bpp_special_cases():
    rng = np.random.default_rng(81)
    A = rng.random((12, 6)) + np.eye(12, 6)
    S = A.T @ A
    # m <= 0: x = 0 satisfies KKT (y = -m >= 0)
    assert np.array_equal(oracle.nnls_bpp(S, -rng.random(6)), np.zeros(6))
    # an interior unconstrained minimiser is the solution
    x_int = rng.random(6) + 0.5
    assert np.allclose(oracle.nnls_bpp(S, S @ x_int), x_int, atol=1e-10)
    # a zero-curvature column (S_rr = 0) stays at zero, the rest is solved
    S0 = S.copy()
    S0[2, :] = 0.0
    S0[:, 2] = 0.0
    m = S @ x_int
    x = oracle.nnls_bpp(S0, m)
    assert x[2] == 0.0
    keep = [0, 1, 3, 4, 5]
    assert np.allclose(x[keep], oracle.nnls_bpp(S0[np.ix_(keep, keep)], m[keep]), atol=1e-12)


def test_bpp_is_the_fixed_point_of_hals_sweeps():
    # repeated HALS sweeps (each a descent step on the same objective)
    # converge to the exact row-wise NNLS solution that BPP computes directly
    rng = np.random.default_rng(83)
    R = 5
    A0 = rng.random((3 * R, R)) + 0.3 * np.eye(3 * R, R)
    S = A0.T @ A0
    M = rng.standard_normal((7, R)) * 2
    W = rng.random((7, R))
    for _ in range(4000):
        oracle.hals_sweep(W, M, S)
    assert np.allclose(oracle.bpp_update(M, S), W, atol=1e-8)


def test_bpp_solve_fit_never_decreases():
    # BCD with exact block minimisation: the objective never increases, so
    # the fit never decreases (up to rounding), unlike a single HALS sweep
    # which is only a descent step
    dims, R = (12, 10, 9), 4
    x, _ = synth.lowrank_plus_noise(dims, R, seed=85, noise=0.05)
    H0 = synth.init_factors(dims, R, seed=86)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=15, nls="bpp")
    fits = np.array(ref["fits"])
    assert np.all(np.diff(fits) >= -1e-10)
    exact = 1.0 - oracle.explicit_residual(x.astype(np.float64), dims, ref["lam"], ref["H"])
    assert abs(exact - fits[-1]) <= 1e-10


def test_planted_bpp_mistake_is_caught(monkeypatch):
    # clipping the unconstrained minimiser is a plausible wrong NNLS
    def wrong(S, m, max_steps=None):
        return np.maximum(0.0, np.linalg.solve(S, m))

    monkeypatch.setattr(oracle, "nnls_bpp", wrong)
    with pytest.raises(AssertionError):
        test_bpp_satisfies_kkt_and_matches_library_nnls(8)


# ---- ADMM (AO-ADMM's NLS-Update, Sec. II-B's alternatives) ------------------

@pytest.mark.parametrize("R", [1, 3, 8, 16])
def test_admm_converges_to_library_nnls_with_its_dual(R):
    # ADMM's fixed point is the NNLS solution (scipy's Lawson-Hanson on the
    # equivalent least squares), and the scaled dual there is -y / rho with
    # y = S z - m the KKT multiplier: nonpositive, zero where z > 0
    scipy_optimize = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(90 + R)
    rows = 6
    A = rng.standard_normal((2 * R + 4, R))
    S = A.T @ A
    B = rng.standard_normal((rows, 2 * R + 4))
    M = B @ A
    Z, U = oracle.admm_update(M, S, rng.random((rows, R)), np.zeros((rows, R)), 6000)
    rho = np.trace(S) / R
    for i in range(rows):
        z_ref, _ = scipy_optimize.nnls(A, B[i])
        assert np.allclose(Z[i], z_ref, atol=1e-7)
    scale = max(1.0, float(np.abs(M).max()))
    assert np.allclose(Z @ S - M, -rho * U, atol=1e-7 * scale)
    assert U.max() <= 1e-9 * scale
    assert np.abs(Z * U).max() <= 1e-9 * scale * scale


def test_admm_interior_solution_is_a_fixed_point():
    # M = Z* S with Z* > 0: the unconstrained minimiser is feasible; from
    # z = Z*, u = 0 every iteration returns the same point
    rng = np.random.default_rng(95)
    R = 7
    A = rng.random((15, R)) + np.eye(15, R)
    S = A.T @ A
    Zs = rng.random((5, R)) + 0.1
    Z, U = oracle.admm_update(Zs @ S, S, Zs, np.zeros_like(Zs), 25)
    assert np.allclose(Z, Zs, atol=1e-12)
    assert np.abs(U).max() <= 1e-12


def test_admm_solve_limit_is_the_exact_bcd_solve():
    # with enough inner iterations every NLS-Update is solved exactly, so the
    # AO-ADMM solve follows the BPP solve whatever dual it carries
    dims, R = (8, 7, 6), 3
    x, _ = synth.lowrank_plus_noise(dims, R, seed=96, noise=0.05)
    H0 = [h.astype(np.float64) for h in synth.init_factors(dims, R, seed=97)]
    xd = x.astype(np.float64)
    a = oracle.nncp_hals(xd, dims, H0, max_iters=4, nls="admm", admm_iters=3000)
    b = oracle.nncp_hals(xd, dims, H0, max_iters=4, nls="bpp")
    assert np.allclose(a["fits"], b["fits"], atol=1e-9)
    for n in range(3):
        assert np.allclose(a["H"][n], b["H"][n], atol=1e-7)


def test_planted_admm_mistake_is_caught(monkeypatch):
    # a dual step with the wrong sign is a plausible slip
    real = oracle.admm_update

    def wrong(M, S, Z, U, iters):
        Z = np.array(Z, dtype=np.float64, copy=True)
        U = np.array(U, dtype=np.float64, copy=True)
        R = S.shape[0]
        rho = float(np.trace(S)) / R
        A = S + rho * np.eye(R)
        for _ in range(iters):
            X = np.linalg.solve(A, (M + rho * (Z - U)).T).T
            Z = np.maximum(0.0, X + U)
            U = U - X + Z
        return Z, U

    assert real is not wrong
    monkeypatch.setattr(oracle, "admm_update", wrong)
    with pytest.raises(AssertionError), np.errstate(over="ignore", invalid="ignore"):
        test_admm_converges_to_library_nnls_with_its_dual(8)


# ---- accelerated projected gradient (the Nesterov-type NLS-Update) ---------

@pytest.mark.parametrize("R", [1, 3, 8, 16])
def test_apg_converges_to_library_nnls(R):
    scipy_optimize = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(100 + R)
    A = rng.standard_normal((2 * R + 4, R))
    S = A.T @ A
    B = rng.standard_normal((6, 2 * R + 4))
    Z = oracle.apg_update(B @ A, S, rng.random((6, R)), 2000)
    for i in range(6):
        z_ref, _ = scipy_optimize.nnls(A, B[i])
        assert np.allclose(Z[i], z_ref, atol=1e-9)


def test_apg_scalar_case_is_exact_in_one_step():
    # R = 1: L = s, so the first projected step is max(0, m / s) exactly
    rng = np.random.default_rng(105)
    for _ in range(20):
        s = float(rng.random() + 0.1)
        m = rng.standard_normal((4, 1))
        x = oracle.apg_update(m, np.array([[s]]), rng.random((4, 1)) * 3, 1)
        assert np.allclose(x, np.maximum(0.0, m / s), rtol=1e-14, atol=1e-15)


def test_apg_interior_solution_is_a_fixed_point():
    rng = np.random.default_rng(106)
    R = 7
    A = rng.random((15, R)) + np.eye(15, R)
    S = A.T @ A
    Zs = rng.random((5, R)) + 0.1
    assert np.allclose(oracle.apg_update(Zs @ S, S, Zs, 30), Zs, atol=1e-12)


def test_apg_solve_limit_is_the_exact_bcd_solve():
    dims, R = (8, 7, 6), 3
    x, _ = synth.lowrank_plus_noise(dims, R, seed=107, noise=0.05)
    H0 = [h.astype(np.float64) for h in synth.init_factors(dims, R, seed=108)]
    xd = x.astype(np.float64)
    a = oracle.nncp_hals(xd, dims, H0, max_iters=4, nls="apg", apg_iters=4000)
    b = oracle.nncp_hals(xd, dims, H0, max_iters=4, nls="bpp")
    assert np.allclose(a["fits"], b["fits"], atol=1e-9)
    for n in range(3):
        assert np.allclose(a["H"][n], b["H"][n], atol=1e-7)


def test_planted_apg_mistake_is_caught(monkeypatch):
    # a gradient with the wrong sign on m is a plausible slip
    def wrong(M, S, W0, iters):
        X = np.array(W0, dtype=np.float64, copy=True)
        L = float(np.max(np.sum(np.abs(S), axis=1)))
        Y, t = X.copy(), 1.0
        for _ in range(iters):
            Xn = np.maximum(0.0, Y - (Y @ S + M) / L)
            tn = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            Y = Xn + ((t - 1.0) / tn) * (Xn - X)
            X, t = Xn, tn
        return X

    monkeypatch.setattr(oracle, "apg_update", wrong)
    with pytest.raises(AssertionError):
        test_apg_converges_to_library_nnls(8)


def test_unknown_nls_update_is_refused():
    dims = (4, 3, 2)
    x, _ = synth.lowrank_plus_noise(dims, 2, seed=110, noise=0.0)
    H0 = synth.init_factors(dims, 2, seed=111)
    with pytest.raises(ValueError):
        oracle.nncp_hals(x.astype(np.float64), dims, H0, max_iters=1, nls="bp")
