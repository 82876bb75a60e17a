"""GPU parity of the AO-ADMM NLS update (nncp_set_nls ADMM).

The solve with a fixed number of ADMM iterations per mode update is compared
with the FP64 oracle's (nncp_hals(nls="admm")): both run the same steps from
the same start (the dual zero at the start of the solve, carried across outer
iterations in the frame of the normalised factor), so the iterates agree to
float32 rounding.  With many inner iterations every update is the exact NNLS
solution, so the solve follows the oracle's BPP solve.
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


def _solve(nn, dims, R, iters, x, H0, prec, admm_iters, split=0):
    c = nn.Context(dims, R, precision=prec, root_split=split)
    try:
        c.set_nls("admm")
        c.set_nls_iters(admm_iters)
        Hd = [torch.from_numpy(h.copy()).cuda() for h in H0]
        c.set_tensor(torch.from_numpy(x).cuda())
        c.set_factors(Hd)
        lam, k, fit = c.solve(iters, 0.0)
        return np.array(lam), k, c.fit_history(), [h.cpu().numpy() for h in Hd]
    finally:
        c.close()


SHAPES = [((20, 17, 13), 5, 0), ((40, 30, 20), 8, 0), ((9, 8, 7, 6), 4, 2),
          ((64, 48, 40), 32, 0), ((300, 40, 20), 12, 0), ((32, 25, 20), 1, 0),
          ((2504, 16, 12), 6, 0)]


@pytest.mark.parametrize("prec", ["fp32_simt", "split_bf16x3"])
@pytest.mark.parametrize("dims,R,split", SHAPES)
def test_admm_solve_matches_oracle(nn, prec, dims, R, split):
    iters, inner = 6, 5
    x, _ = synth.lowrank_plus_noise(dims, min(R, 6), seed=61, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=62)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=iters, use_dimtree=True, s=split or None, nls="admm",
                           admm_iters=inner)
    lam, k, hist, H = _solve(nn, dims, R, iters, x, H0, prec, inner, split)
    assert k == iters
    assert np.max(np.abs(np.array(hist) - np.array(ref["fits"]))) <= 1e-4
    for n in range(len(dims)):
        assert rel_fro(H[n], ref["H"][n]) <= 1e-3, n
    assert rel_fro(lam, ref["lam"]) <= 1e-3


@pytest.mark.parametrize("inner", [1, 30])
def test_admm_inner_iteration_counts(nn, inner):
    dims, R = (40, 30, 20), 8
    x, _ = synth.lowrank_plus_noise(dims, 6, seed=63, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=64)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=5, nls="admm", admm_iters=inner)
    lam, k, hist, H = _solve(nn, dims, R, 5, x, H0, "fp32_simt", inner)
    assert np.max(np.abs(np.array(hist) - np.array(ref["fits"]))) <= 1e-4
    for n in range(3):
        assert rel_fro(H[n], ref["H"][n]) <= 1e-3, n


def test_admm_many_inner_iterations_is_the_exact_solve(nn):
    dims, R = (40, 30, 20), 8
    x, _ = synth.lowrank_plus_noise(dims, 6, seed=51, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=52)
    ref = oracle.nncp_hals(x.astype(np.float64), dims, [h.astype(np.float64) for h in H0],
                           max_iters=3, nls="bpp")
    lam, k, hist, H = _solve(nn, dims, R, 3, x, H0, "fp32_simt", 1000)
    assert abs(hist[-1] - ref["fits"][-1]) <= 1e-4
    for n in range(3):
        assert rel_fro(H[n], ref["H"][n]) <= 1e-3, n


def test_admm_arguments(nn):
    c = nn.Context((10, 10, 10), 33)
    try:
        with pytest.raises(nn.NNCPError):
            c.set_nls("admm")
        for bad in (0, 10001):
            with pytest.raises(nn.NNCPError):
                c.set_nls_iters(bad)
        c.set_nls_iters(7)
    finally:
        c.close()
