"""GPU parity of the block principal pivoting NLS update (nncp_set_nls BPP).

The solve with BPP as Alg. 1's NLS-Update is compared with the FP64 oracle's
(nncp_hals(nls="bpp")): every row's nonnegative least squares is solved
exactly on both sides (float32 Cholesky here, float64 there), so the
iterates agree to float32 rounding.
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


def _solve(nn, dims, R, iters, x, H0, prec, split=0, tol=0.0):
    c = nn.Context(dims, R, precision=prec, root_split=split)
    try:
        c.set_nls("bpp")
        Hd = [torch.from_numpy(h.copy()).cuda() for h in H0]
        c.set_tensor(torch.from_numpy(x).cuda())
        c.set_factors(Hd)
        lam, k, fit = c.solve(iters, tol)
        return np.array(lam), k, fit, c.fit_history(), [h.cpu().numpy() for h in Hd]
    finally:
        c.close()


SHAPES = [((20, 17, 13), 5, 0), ((40, 30, 20), 8, 0), ((9, 8, 7, 6), 4, 2),
          ((64, 48, 40), 32, 0), ((300, 40, 20), 12, 0), ((32, 25, 20), 1, 0),
          ((2504, 16, 12), 6, 0)]


@pytest.mark.parametrize("prec", ["fp32_simt", "split_bf16x3"])
@pytest.mark.parametrize("dims,R,split", SHAPES)
def test_bpp_solve_matches_oracle(nn, prec, dims, R, split):
    iters = 6
    x, _ = synth.lowrank_plus_noise(dims, min(R, 6), seed=51, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=52)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=iters, use_dimtree=True, s=split or None, nls="bpp")
    lam, k, fit, hist, H = _solve(nn, dims, R, iters, x, H0, prec, split)
    assert k == iters
    assert np.max(np.abs(np.array(hist) - np.array(ref["fits"]))) <= 1e-4
    for n in range(len(dims)):
        assert rel_fro(H[n], ref["H"][n]) <= 1e-3, n
    assert rel_fro(lam, ref["lam"]) <= 1e-3


def test_bpp_fit_never_decreases(nn):
    # exact block minimisation: the objective never increases (to float32 noise)
    dims, R = (40, 30, 20), 6
    x, _ = synth.lowrank_plus_noise(dims, R, seed=53, noise=0.05)
    H0 = synth.init_factors(dims, R, seed=54)
    _, k, _, hist, _ = _solve(nn, dims, R, 25, x, H0, "fp32_simt")
    assert k == 25
    assert np.all(np.diff(np.array(hist)) >= -2e-6)


def test_bpp_rank_limit(nn):
    c = nn.Context((10, 10, 10), 33)
    try:
        with pytest.raises(nn.NNCPError):
            c.set_nls("bpp")
        c.set_nls("hals")
    finally:
        c.close()
