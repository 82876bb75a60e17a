"""FP64 CPU oracle for nonnegative CP decomposition (NNCP) with HALS updates.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The GPU library never calls it, shares no code with
it, and fails loudly instead of falling back to it.

Every function here follows the paper "Parallel Nonnegative CP Decomposition
of Dense Tensors" (Ballard, Hayashi, Kannan; arXiv:1806.07985) step by step in
plain numpy float64: explicit matricizations, explicit Khatri-Rao products and
library matmuls only, with no blocking, fusion or reordering beyond what the
paper's definitions state.  Pins (tests that tie it to something other than
itself) live in ``tests/test_oracle_pins.py``.

Parity status per function (the pins are listed in each docstring):
  * mttkrp_direct, mttkrp_dimtree, khatri_rao, matricize: pinned
    (brute-force elementwise sums, rank-1 closed form, tree == direct).
  * hals_sweep: pinned (R=1 closed form, convergence to the exact NNLS
    solution from scipy.optimize.nnls, KKT conditions, monotone objective).
  * normalize / fit_identity / explicit_residual / nncp_hals: pinned
    (model invariance, identity == explicit residual, exact recovery of
    noise-free low-rank tensors to < 1e-10, non-increasing objective).
  * nnls_bpp / bpp_update: pinned (KKT conditions, scipy.optimize.nnls,
    enumeration of every passive set for small R, special cases, the limit
    of repeated HALS sweeps, non-decreasing fit of the solve).
  * admm_update: pinned (convergence to scipy.optimize.nnls with the scaled
    dual equal to -y / rho, interior fixed point, many-iteration solve equal
    to the BPP solve).  The carry of each mode's dual across outer
    iterations in nncp_hals(nls="admm") changes only the inner convergence
    speed and has no external reference ("parity unpinned" for that part).
  * apg_update: pinned (convergence to scipy.optimize.nnls, exact one-step
    scalar case, interior fixed point, many-step solve equal to the BPP
    solve).
  * The final-fit value of a noisy solve has no external pin: it is the
    oracle's own trajectory ("parity unpinned" for that number alone).
"""

from .nncp import *  # noqa: F401,F403
