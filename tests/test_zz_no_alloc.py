"""The MTTKRP entry point that allocates nothing (nncp_mttkrp_noalloc).

Callers that must not allocate device memory (a host whose caching allocator
already holds the free memory, a plugin host that only passes in its own
buffers, a serving loop where cudaMalloc would stall other streams) get a
direct MTTKRP whose split-K scratch is a fixed __device__ array inside the
library.  These tests call it through the C ABI and compare its output with
the FP64 oracle's direct MTTKRP (Sec. II-A definition) at the float32 path's
1e-5, on two calls in a row, since every call reuses the same scratch array.
The file name makes pytest collect it last.
"""

import numpy as np
import pytest

import oracle
from tests._util import ensure_built, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the MTTKRP tolerance of the float32 path


@pytest.fixture(scope="module")
def nn():
    ensure_built()
    from paper_1806_07985_gb300 import nncp
    return nncp


@pytest.mark.parametrize("dims,R", [((8, 300, 300), 16),   # mode 1 splits K = 90000 over many CTAs
                                    ((37, 23, 29, 5), 7),
                                    ((64, 64, 64), 32)])
def test_noalloc_matches_oracle_twice(nn, dims, R):
    rng = np.random.default_rng(123)
    x = rng.random(int(np.prod(dims))).astype(np.float32)
    Hh = [rng.random((d, R)).astype(np.float32) for d in dims]
    X = torch.from_numpy(x).cuda()
    H = [torch.from_numpy(h).cuda() for h in Hh]
    xd = x.astype(np.float64)
    Hd = [h.astype(np.float64) for h in Hh]
    for mode in range(1, len(dims) + 1):
        ref = oracle.mttkrp_direct(xd, dims, Hd, mode - 1)
        outs = []
        for _ in range(2):
            M = torch.full((dims[mode - 1], R), float("nan"), device="cuda")
            nn.nncp_mttkrp_noalloc(dims, R, X, H, mode, M)
            outs.append(M)
        torch.cuda.synchronize()
        for M in outs:
            m = M.cpu().numpy()
            assert np.isfinite(m).all()
            assert rel_fro(m, ref) <= TOL, (dims, mode)


def test_noalloc_rejects_sizes_beyond_its_scratch(nn):
    dims, R = (20000, 2, 2), 128  # I_1 * R = 2.56e6 > 2^21 / 2
    X = torch.zeros(int(np.prod(dims)), device="cuda")
    H = [torch.zeros(d, R, device="cuda") for d in dims]
    M = torch.zeros(dims[0], R, device="cuda")
    with pytest.raises(nn.NNCPError) as info:
        nn.nncp_mttkrp_noalloc(dims, R, X, H, 1, M)
    assert info.value.status == nn.NNCP_ERR_INVALID_ARG
    assert "no-alloc limit" in str(info.value)


def test_noalloc_binding_checks_shapes_before_the_call(nn):
    dims, R = (8, 6, 5), 3
    X = torch.zeros(int(np.prod(dims)), device="cuda")
    H = [torch.zeros(d, R, device="cuda") for d in dims]
    M = torch.zeros(dims[0], R, device="cuda")
    with pytest.raises(ValueError):
        nn.nncp_mttkrp_noalloc(dims, R, X, H[:2], 1, M)          # too few factors
    with pytest.raises(ValueError):
        nn.nncp_mttkrp_noalloc(dims, R, X[:-1], H, 1, M)         # X too short
    with pytest.raises(ValueError):
        nn.nncp_mttkrp_noalloc(dims, R, X, H, 2, M)              # M is I_1 x R, not I_2 x R
    with pytest.raises(ValueError):
        nn.nncp_mttkrp_noalloc(dims, R, X, [h.double() for h in H], 1, M)
