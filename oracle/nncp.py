"""Plain FP64 NNCP-HALS oracle (test infrastructure only; see package docstring).

Conventions
-----------
* A tensor is a flat float64 vector ``x`` plus its mode lengths ``dims``
  (I_1, ..., I_N).  Entries are stored "mode-descending, generalising
  column-major" (Sec. IV-C, Data Distribution): mode 1 is fastest, so the
  0-based linear index of (i_1, ..., i_N) is i_1 + I_1*(i_2 + I_2*(i_3 + ...)).
* Modes are numbered 0..N-1 in code (the paper numbers them 1..N).
* A factor matrix H[n] is an I_n x R float64 array; lam is the weight vector
  of the model [[lam; H_1, ..., H_N]] (Sec. II-A).
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "linear_index",
    "matricize",
    "khatri_rao",
    "krp_chain",
    "mttkrp_direct",
    "mttkrp_rows",
    "partial_mttkrp_right",
    "partial_mttkrp_left",
    "mttv_leaf",
    "mttv_contract_first",
    "mttkrp_dimtree",
    "default_root_split",
    "gram",
    "hadamard_of_grams",
    "hals_sweep",
    "nnls_bpp",
    "bpp_update",
    "admm_update",
    "apg_update",
    "normalize_columns",
    "fit_identity",
    "reconstruct",
    "explicit_residual",
    "hals_objective",
    "nncp_hals",
]


# --------------------------------------------------------------------------
# Layout, matricization, Khatri-Rao product  (Sec. II-A; Sec. IV-C layout)
# --------------------------------------------------------------------------

def linear_index(idx, dims):
    """Linear position of multi-index ``idx`` with mode 1 fastest (Sec. IV-C)."""
    pos, stride = 0, 1
    for i, d in zip(idx, dims):
        pos += i * stride
        stride *= d
    return pos


def matricize(x, dims, row_modes):
    """Explicit matricization: a materialised copy, rows over ``row_modes``.

    Sec. II-A defines X_(n) (I_n x I/I_n, columns are the mode-n fibres); the
    dimension-tree root matricization X_(1:s) (Sec. IV-A, Fig. 2a) puts a set
    of leading modes on the rows.  Both are this function: the row index runs
    over ``row_modes`` and the column index over the remaining modes, each
    with the lowest mode fastest, which is the column order that pairs column
    j of X_(n) with row j of K(n) = H_N (.) ... (.) H_1 (minus mode n).
    """
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    row_modes = sorted(row_modes)
    col_modes = [m for m in range(N) if m not in row_modes]
    # numpy C-order array whose axis k is mode N-1-k (last axis = mode 0 fastest)
    arr = np.asarray(x, dtype=np.float64).reshape(dims[::-1])
    axis_of = lambda m: N - 1 - m  # noqa: E731
    # highest mode first so that, after a C-order reshape, the lowest is fastest
    order = [axis_of(m) for m in sorted(row_modes, reverse=True)] + \
            [axis_of(m) for m in sorted(col_modes, reverse=True)]
    rows = int(np.prod([dims[m] for m in row_modes], dtype=np.int64))
    return np.ascontiguousarray(arr.transpose(order)).reshape(rows, -1)


def khatri_rao(A, B):
    """K = A (.) B with K(:, c) = A(:, c) kron B(:, c) (Sec. II-A).

    The paper states two index conventions for the same product; this uses the
    column-wise Kronecker one, so B's row index is the fastest in K.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert A.shape[1] == B.shape[1]
    K = np.empty((A.shape[0] * B.shape[0], A.shape[1]))
    for c in range(A.shape[1]):
        K[:, c] = np.kron(A[:, c], B[:, c])
    return K


def krp_chain(H, modes):
    """H[m_k] (.) ... (.) H[m_1] for ascending ``modes`` (lowest mode fastest).

    With modes = all modes except n this is K(n) of Sec. II-A.
    """
    modes = sorted(modes)
    K = np.asarray(H[modes[-1]], dtype=np.float64)
    for m in reversed(modes[:-1]):
        K = khatri_rao(K, H[m])
    return K


def mttkrp_direct(x, dims, H, n):
    """M(n) = X_(n) K(n) (Sec. II-A), explicit matricization and explicit KRP."""
    others = [m for m in range(len(dims)) if m != n]
    return matricize(x, dims, [n]) @ krp_chain(H, others)


def mttkrp_rows(x, dims, H, n, rows):
    """Selected rows of M(n) = X_(n) K(n): same definition, fewer rows.

    Used to check full-size GPU results at sampled rows.
    """
    dims = tuple(int(d) for d in dims)
    others = [m for m in range(len(dims)) if m != n]
    K = krp_chain(H, others)
    arr = np.asarray(x, dtype=np.float64).reshape(dims[::-1])
    out = np.empty((len(rows), K.shape[1]))
    for t, i in enumerate(rows):
        # the i-th mode-n slice, laid out with the remaining modes lowest-fastest
        sl = np.take(arr, int(i), axis=len(dims) - 1 - n)
        out[t] = sl.reshape(-1) @ K
    return out


# --------------------------------------------------------------------------
# Dimension tree (Sec. IV-A, Fig. 1 and Fig. 2)
# --------------------------------------------------------------------------

def partial_mttkrp_right(x, dims, H, s):
    """Root -> left node {1..s}: T_L = X_(1:s) (H_N (.) ... (.) H_{s+1}).

    One GEMM on the memory-compatible matricization (Sec. IV-A, Fig. 2a).
    Rows of T_L run over (i_1, ..., i_s) with i_1 fastest.
    """
    N = len(dims)
    return matricize(x, dims, list(range(s))) @ krp_chain(H, list(range(s, N)))


def partial_mttkrp_left(x, dims, H, s):
    """Root -> right node {s+1..N}: T_R = X_(1:s)^T (H_s (.) ... (.) H_1)."""
    return matricize(x, dims, list(range(s))).T @ krp_chain(H, list(range(s)))


def mttv_leaf(T, node_dims, H_rest):
    """Leaf M(a) from node {a..b}: contract every mode but the first.

    ``T`` is (I_a*...*I_b) x R with i_a fastest; ``H_rest`` are the factors of
    modes a+1..b.  Computed as the paper's multi-TTV: R independent GEMVs, one
    per contiguous block T[r] (Sec. IV-A, Fig. 2b).
    """
    Ia = int(node_dims[0])
    R = T.shape[1]
    K = krp_chain(H_rest, list(range(len(H_rest))))
    M = np.empty((Ia, R))
    for r in range(R):
        Tr = T[:, r].reshape(-1, Ia).T  # I_a x (I_{a+1}...I_b), column-major view
        M[:, r] = Tr @ K[:, r]
    return M


def mttv_contract_first(T, node_dims, Ha):
    """Node {a+1..b} from node {a..b}: contract mode a with H_a (R GEMVs)."""
    Ia = int(node_dims[0])
    R = T.shape[1]
    out = np.empty((T.shape[0] // Ia, R))
    for r in range(R):
        Tr = T[:, r].reshape(-1, Ia).T
        out[:, r] = Tr.T @ Ha[:, r]
    return out


def default_root_split(dims):
    """Root split s in [1, N-1] balancing the two halves' sizes.

    Sec. IV-C (Memory) notes that splitting the root so the two halves have
    nearly equal geometric means keeps the tree's temporaries small; this
    picks the s minimising |log I_L - log I_R|, the smaller s on ties.
    """
    N = len(dims)
    best, best_s = None, 1
    for s in range(1, N):
        IL = float(np.prod(dims[:s]))
        IR = float(np.prod(dims[s:]))
        score = abs(math.log(IL) - math.log(IR))
        if best is None or score < best - 1e-12:
            best, best_s = score, s
    return best_s


def _visit_node(T, modes, dims, H, update):
    """Walk node {modes} in BCD order (Fig. 1 shape: split off the first mode)."""
    a = modes[0]
    node_dims = [dims[m] for m in modes]
    if len(modes) == 1:
        update(a, T)
        return
    rest = modes[1:]
    update(a, mttv_leaf(T, node_dims, [H[m] for m in rest]))
    # H[a] has just been updated: the child node uses the new factor
    _visit_node(mttv_contract_first(T, node_dims, H[a]), rest, dims, H, update)


def _dimtree_sweep(x, dims, H, s, update):
    """One outer iteration's MTTKRPs through the dimension tree.

    A node is rebuilt right before the first of its modes is updated, after
    every factor outside it has been updated, so the root is visited twice per
    outer iteration (Sec. IV-A; Sec. IV-C Computation).
    """
    N = len(dims)
    T_L = partial_mttkrp_right(x, dims, H, s)          # uses H_{s+1..N}
    _visit_node(T_L, list(range(s)), dims, H, update)
    T_R = partial_mttkrp_left(x, dims, H, s)           # uses the new H_{1..s}
    _visit_node(T_R, list(range(s, N)), dims, H, update)


def mttkrp_dimtree(x, dims, H, n, s=None):
    """M(n) for the current factors, computed through the dimension tree."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    s = default_root_split(dims) if s is None else s
    out = {}

    def record(m, M):
        if m == n:
            out["M"] = M

    # read-only walk: no factor changes, so the schedule's order is immaterial
    if n < s:
        _visit_node(partial_mttkrp_right(x, dims, H, s), list(range(s)), dims, H, record)
    else:
        _visit_node(partial_mttkrp_left(x, dims, H, s), list(range(s, N)), dims, H, record)
    return out["M"]


# --------------------------------------------------------------------------
# Gram matrices, HALS, normalisation, fit  (Alg. 1; Sec. II-B; Sec. IV-B; Alg. 3)
# --------------------------------------------------------------------------

def gram(Hn):
    """G = H^T H (Alg. 1, Local-SYRK in Alg. 2)."""
    Hn = np.asarray(Hn, dtype=np.float64)
    return Hn.T @ Hn


def hadamard_of_grams(G, n):
    """S(n) = G_1 * ... * G_{n-1} * G_{n+1} * ... * G_N (Alg. 1)."""
    R = G[0].shape[0]
    S = np.ones((R, R))
    for k, Gk in enumerate(G):
        if k != n:
            S = S * Gk
    return S


def hals_sweep(W, M, S):
    """One HALS sweep over the columns of W, in place (Sec. II-B).

    For r = 1..R in order and every row i:
        w_ir <- max(0, w_ir + (m_ir - sum_s w_is S_sr) / S_rr)
    The sum uses the columns already updated in this sweep.  The paper prints
    the rule without the division by S_rr, which is the same rule when the
    other factors are 2-norm column-normalised (S_rr = 1, Alg. 3); the
    division keeps each column step an exact minimisation in general.
    A column with S_rr = 0 is left as it is.
    """
    R = W.shape[1]
    for r in range(R):
        if S[r, r] == 0.0:
            continue
        W[:, r] = np.maximum(0.0, W[:, r] + (M[:, r] - W @ S[:, r]) / S[r, r])
    return W


def nnls_bpp(S, m, max_steps=None):
    """min_{x >= 0} x^T S x / 2 - m^T x for symmetric positive (semi)definite S,
    by block principal pivoting (the NLS solver the paper names, Sec. II-B).

    The solution is the x with x >= 0, y = S x - m >= 0 and x_i y_i = 0 (the
    KKT conditions; unique when S is positive definite).  Block principal
    pivoting keeps a passive set F (x_F free, x elsewhere 0), solves
    S_FF x_F = m_F, and moves every infeasible index (x_i < 0 in F, or
    y_i < 0 outside it) to the other set at once.  While the number of
    infeasible indices does not fall below its best value, at most three
    more full exchanges are tried, after which only the infeasible index of
    largest position moves (the backup rule that guarantees termination).
    Columns with S_rr = 0 stay at x_r = 0 (their step is undefined, as in the
    HALS sweep).
    """
    S = np.asarray(S, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    R = m.shape[0]
    usable = np.diag(S) > 0.0
    F = np.zeros(R, dtype=bool)
    x = np.zeros(R)
    y = -m.copy()
    y[~usable] = 0.0
    best, backups = R + 1, 3
    for _ in range(max_steps or 50 * R + 50):
        infeasible = ((F & (x < 0.0)) | (~F & (y < 0.0))) & usable
        count = int(np.count_nonzero(infeasible))
        if count == 0:
            return x
        if count < best:
            best, backups = count, 3
            flip = infeasible
        elif backups > 0:
            backups -= 1
            flip = infeasible
        else:
            flip = np.zeros(R, dtype=bool)
            flip[np.flatnonzero(infeasible)[-1]] = True
        F = F ^ flip
        x = np.zeros(R)
        if F.any():
            x[F] = np.linalg.solve(S[np.ix_(F, F)], m[F])
        y = S @ x - m
        y[F] = 0.0
        y[~usable] = 0.0
    raise RuntimeError("block principal pivoting did not terminate")


def bpp_update(M, S):
    """W = argmin_{W >= 0} ||M - W S||-style NLS of every row: row i of W is
    nnls_bpp(S, M(i, :)) (the exact block solve of Alg. 1's NLS-Update)."""
    M = np.asarray(M, dtype=np.float64)
    return np.stack([nnls_bpp(S, M[i]) for i in range(M.shape[0])]) if M.shape[0] else M.copy()


def admm_update(M, S, Z, U, iters):
    """`iters` iterations of ADMM on every row's NLS (AO-ADMM, one of the
    alternative NLS-Updates Sec. II-B names), in the scaled form of ADMM.

    Row problem: min_{x >= 0} 1/2 x^T S x - m^T x, split as x = z with the
    constraint on z and a scaled dual u.  With rho = trace(S) / R, each
    iteration is, for every row at once (the rows share S + rho I):
        x <- (S + rho I)^-1 (m + rho (z - u))
        z <- max(0, x + u)
        u <- u + x - z
    Z and U are the starting values (rows of z and u); returns the final
    (Z, U), Z being the updated factor.  At a fixed point x = z and
    S z - m = -rho u, which with z >= 0, u <= 0, z_i u_i = 0 are the NNLS
    KKT conditions.  trace(S) = 0 gives Z = U = 0.
    """
    M = np.asarray(M, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    Z = np.array(Z, dtype=np.float64, copy=True)
    U = np.array(U, dtype=np.float64, copy=True)
    R = S.shape[0]
    rho = float(np.trace(S)) / R
    if rho <= 0.0:
        return np.zeros_like(Z), np.zeros_like(U)
    A = S + rho * np.eye(R)
    for _ in range(iters):
        X = np.linalg.solve(A, (M + rho * (Z - U)).T).T
        Z = np.maximum(0.0, X + U)
        U = U + X - Z
    return Z, U


def apg_update(M, S, W0, iters):
    """`iters` steps of Nesterov's accelerated projected gradient on every
    row's NLS (the Nesterov-type NLS-Update Sec. II-B names), FISTA form.

    Row problem: min_{x >= 0} f(x) = 1/2 x^T S x - m^T x, gradient S x - m.
    L = max_i sum_j |S_ij| bounds the largest eigenvalue of S (Gershgorin),
    so 1/L is a valid step.  From x_0 = y_1 = w0 and t_1 = 1, step k is
        x_k     = max(0, y_k - (S y_k - m) / L)
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
        y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})
    for all rows at once; returns x after `iters` steps.  L = 0 (S = 0)
    returns W0 unchanged.
    """
    M = np.asarray(M, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    X = np.array(W0, dtype=np.float64, copy=True)
    L = float(np.max(np.sum(np.abs(S), axis=1))) if S.size else 0.0
    if L <= 0.0:
        return X
    Y = X.copy()
    t = 1.0
    for _ in range(iters):
        Xn = np.maximum(0.0, Y - (Y @ S - M) / L)
        tn = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        Y = Xn + ((t - 1.0) / tn) * (Xn - X)
        X, t = Xn, tn
    return X


def normalize_columns(W):
    """lambda_r = ||W(:, r)||_2 and H = W diag(lambda)^-1 (Alg. 3, column norms).

    A zero column stays zero with lambda_r = 0.
    """
    lam = np.sqrt(np.sum(W * W, axis=0))
    Hn = np.zeros_like(W)
    nz = lam > 0
    Hn[:, nz] = W[:, nz] / lam[nz]
    return Hn, lam


def fit_identity(alpha, M_N, W_N, lam, S_N, G_N):
    """Relative error from the Sec. IV-B identity (Alg. 3, last lines).

    beta = <M(N), W(N)>, gamma = lam^T (S(N) * G(N)) lam,
    eps = sqrt(max(0, alpha - 2 beta + gamma) / alpha), returns (eps, beta, gamma).
    The max(0, .) guards the cancellation of the identity near an exact fit.
    """
    beta = float(np.sum(M_N * W_N))
    gamma = float(lam @ (S_N * G_N) @ lam)
    eps = math.sqrt(max(0.0, alpha - 2.0 * beta + gamma) / alpha)
    return eps, beta, gamma


def reconstruct(lam, H, dims):
    """Model tensor sum_r lam_r h_1r o ... o h_Nr as a flat mode-1-fastest vector.

    Built rank-one term by rank-one term with outer products (Sec. II-A).
    """
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    total = np.zeros(int(np.prod(dims, dtype=np.int64)))
    for r in range(len(lam)):
        t = np.asarray(H[N - 1][:, r], dtype=np.float64)
        for m in range(N - 2, -1, -1):
            t = np.multiply.outer(t, H[m][:, r])  # axes: mode N-1, ..., mode m
        total += lam[r] * t.reshape(-1)
    return total


def explicit_residual(x, dims, lam, H):
    """||X - [[lam; H]]|| / ||X||, every entry reconstructed in FP64."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.linalg.norm(x - reconstruct(lam, H, dims)) / np.linalg.norm(x))


def hals_objective(W, M, S):
    """f(W) = 1/2 tr(W S W^T) - <M, W>: the NLS objective up to a constant."""
    return 0.5 * float(np.sum((W @ S) * W)) - float(np.sum(M * W))


def nncp_hals(x, dims, H_init, max_iters, tol=0.0, use_dimtree=True, s=None,
              callback=None, nls="hals", admm_iters=5, apg_iters=None):
    """NNCP by block coordinate descent with one HALS sweep per block (Alg. 1, Alg. 3).

    nls selects Alg. 1's NLS-Update: "hals" (one HALS sweep from W = H_n
    diag(lam), the default) or "bpp" (the exact nonnegative least-squares
    solve of every row by block principal pivoting, ``bpp_update``; its
    result does not depend on the starting W) or "admm" (``admm_iters``
    ADMM iterations, ``admm_update``, from z = H_n diag(lam) and the dual
    this mode's previous update left; the factor is z).  The dual is kept
    in the frame of the normalised factor: divided by the new lam when
    H_n is, multiplied by the current lam when the next update of mode n
    starts, as z is; it starts at 0), or "apg" (``apg_iters`` steps of
    the accelerated projected gradient, ``apg_update``, from W = H_n
    diag(lam); default ``admm_iters`` steps).

    Steps, in the paper's order:
      init   : normalise every initial factor, fold the norms into lam,
               G_n = H_n^T H_n, alpha = ||X||^2.  (The paper initialises
               n = 2..N only because BPP needs no start for H_1; HALS does.)
      repeat : for n = 1..N:
                 M   <- MTTKRP(X, {H}, n)           (direct or dimension tree)
                 S   <- Hadamard of G_k, k != n
                 W   <- H_n diag(lam); one HALS sweep on (W, M, S)
                 lam <- column 2-norms of W; H_n <- W diag(lam)^-1
                 G_n <- H_n^T H_n
               fit = 1 - eps with eps from the Sec. IV-B identity at n = N.
      stop   : |fit_k - fit_{k-1}| < tol for k >= 2, or k = max_iters.

    ``callback(event, **state)`` is called after every inner iteration
    (event "inner") with copies-free references to the live state.
    Returns a dict with H (normalised), lam, fits, iters, eps.
    """
    if nls not in ("hals", "bpp", "admm", "apg"):
        raise ValueError(f"unknown NLS update {nls!r}")
    dims = tuple(int(d) for d in dims)
    x = np.asarray(x, dtype=np.float64)
    N = len(dims)
    s = default_root_split(dims) if s is None else s
    H = [np.array(h, dtype=np.float64, copy=True) for h in H_init]
    R = H[0].shape[1]
    lam = np.ones(R)
    for n in range(N):
        H[n], c = normalize_columns(H[n])
        lam = lam * c
    G = [gram(h) for h in H]
    alpha = float(np.sum(x * x))
    state = {"lam": lam, "fit": None, "eps": None}
    fits, epss = [], []
    Uhat = [np.zeros_like(h) for h in H]  # ADMM duals, normalised frame

    def update(n, M):
        S = hadamard_of_grams(G, n)
        if nls == "bpp":
            W = bpp_update(M, S)
        elif nls == "admm":
            W, U = admm_update(M, S, H[n] * state["lam"], Uhat[n] * state["lam"], admm_iters)
        elif nls == "apg":
            W = apg_update(M, S, H[n] * state["lam"],
                           admm_iters if apg_iters is None else apg_iters)
        else:
            W = H[n] * state["lam"]
            hals_sweep(W, M, S)
        H[n], state["lam"] = normalize_columns(W)
        if nls == "admm":
            lam_n = state["lam"]
            Uhat[n] = np.zeros_like(U)
            nz = lam_n > 0
            Uhat[n][:, nz] = U[:, nz] / lam_n[nz]
        G[n] = gram(H[n])
        if n == N - 1:
            eps, _, _ = fit_identity(alpha, M, W, state["lam"], S, G[n])
            state["eps"], state["fit"] = eps, 1.0 - eps
        if callback is not None:
            callback("inner", n=n, M=M, S=S, W=W, H=H, lam=state["lam"], G=G)

    iters = 0
    for k in range(1, max_iters + 1):
        if use_dimtree:
            _dimtree_sweep(x, dims, H, s, update)
        else:
            for n in range(N):
                update(n, mttkrp_direct(x, dims, H, n))
        fits.append(state["fit"])
        epss.append(state["eps"])
        iters = k
        if k >= 2 and abs(fits[-1] - fits[-2]) < tol:
            break
    return {"H": H, "lam": state["lam"], "fits": fits, "eps": epss,
            "iters": iters, "G": G, "alpha": alpha}
