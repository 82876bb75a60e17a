"""Par-NNCP (Alg. 2) on CPU: the driver's collectives and data placement.

The driver (paper_1806_07985_gb300/par_nncp.py) moves data between the
processors of a P_1 x ... x P_N grid; the per-processor computation is the
library's (nncp_par_*), which needs a GPU.  Here each processor's library
object is replaced by a stand-in with the same protocol whose every step is
the FP64 oracle's (local MTTKRP of the block, HALS sweep of the owned rows,
the Gram, normalisation and fit sums), so a correct exchange reproduces the
oracle's sequential solve on the whole tensor to rounding: checked with every
processor in one process (LocalComm) and with 2 and 4 gloo ranks (DistComm).
"""

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1806_07985_gb300 import par_nncp, synth

torch = pytest.importorskip("torch")


class OracleRank:
    """Stand-in for nncp.ParRank: float64, every step from the oracle."""

    def __init__(self, dims, grid, coords, R):
        self.dims, self.grid, self.coords, self.R = tuple(dims), tuple(grid), tuple(coords), R
        self.N = len(dims)
        self.local = tuple(par_nncp.block_range(I, P, c)[1] for I, P, c in zip(dims, grid, coords))

    def layout(self, mode):
        n = mode - 1
        lo, L = par_nncp.block_range(self.dims[n], self.grid[n], self.coords[n])
        others = [(self.coords[k], self.grid[k]) for k in range(self.N) if k != n]
        q, Q = 0, 1
        for c, P in others:
            q += c * Q
            Q *= P
        return lo, L, lo + q * L // Q, (q + 1) * L // Q - q * L // Q, q, Q

    def set_data(self, X, H):
        self.X, self.H = X, H

    def alpha_local(self, X):
        return float((X.double() ** 2).sum())

    def begin(self, alpha, tol):
        self.alpha, self.tol = alpha, tol
        self.lam = np.ones(self.R)
        self.G = [np.zeros((self.R, self.R)) for _ in range(self.N)]
        self.fits = []

    def mttkrp(self, mode, M):
        Hb = [h.numpy() for h in self.H]
        M.copy_(torch.from_numpy(oracle.mttkrp_direct(self.X.numpy(), self.local, Hb, mode - 1)))

    def update(self, mode, M_owned, H_owned):
        n = mode - 1
        W = H_owned.numpy().copy()
        beta = 0.0
        if M_owned is not None:
            S = oracle.hadamard_of_grams(self.G, n)
            W = W * self.lam
            oracle.hals_sweep(W, M_owned.numpy(), S)
            beta = float(np.sum(M_owned.numpy() * W))
            H_owned.copy_(torch.from_numpy(W))
        return list((W.T @ W).reshape(-1)) + [beta]

    def normalize(self, mode, sums, H_owned, init):
        n, R = mode - 1, self.R
        WtW = np.array(sums[:R * R]).reshape(R, R)
        c = np.sqrt(np.diag(WtW))
        self.lam = self.lam * c if init else c
        inv = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 0.0)
        self.G[n] = WtW * inv[:, None] * inv[None, :]
        H_owned.mul_(torch.from_numpy(inv))
        if init or n != self.N - 1:
            return (self.fits[-1] if self.fits else 0.0), False
        S = oracle.hadamard_of_grams(self.G, n)
        gamma = float(np.sum(S * WtW))
        eps = np.sqrt(max(0.0, self.alpha - 2.0 * sums[R * R] + gamma) / self.alpha)
        fit = 1.0 - eps
        stop = bool(self.fits) and abs(fit - self.fits[-1]) < self.tol
        self.fits.append(fit)
        return fit, stop

    def result(self):
        return list(self.lam), list(self.fits)


def _processor(x, H0, dims, grid, rank, R):
    coords = par_nncp.grid_coords(rank, grid)
    eng = OracleRank(dims, grid, coords, R)
    X = torch.from_numpy(par_nncp.local_block(x, dims, grid, coords).astype(np.float64))
    layouts = [eng.layout(n + 1) for n in range(len(dims))]
    H = []
    for n, h in enumerate(H0):
        lo, rows = layouts[n][0], layouts[n][1]
        H.append(torch.from_numpy(np.ascontiguousarray(h[lo:lo + rows], dtype=np.float64)))
    return par_nncp.Processor(eng, X, H, layouts)


def _assemble(procs, dims, grid):
    """Global factors from the owned rows of every processor."""
    out = []
    for n, I in enumerate(dims):
        Hn = np.full((I, procs[0].H[n].shape[1]), np.nan)
        for p in procs.values():
            _, _, lo, rows, _, _ = p.layouts[n]
            Hn[lo:lo + rows] = p.owned(n).numpy()
        out.append(Hn)
    return out


def _problem(dims, R, seed):
    x, _ = synth.lowrank_plus_noise(dims, R, seed=seed, noise=0.02)
    H0 = synth.init_factors(dims, R, seed=seed + 1)
    return x.astype(np.float64), [h.astype(np.float64) for h in H0]


@pytest.mark.parametrize("dims,grid,R", [((12, 10, 9), (2, 1, 1), 3),
                                         ((12, 10, 9), (2, 2, 1), 4),
                                         ((9, 11, 7), (3, 1, 2), 3),
                                         ((8, 6, 7, 5), (2, 1, 2, 1), 2),
                                         ((7, 5, 6), (1, 1, 1), 3)])
def test_local_grid_reproduces_the_sequential_oracle(dims, grid, R):
    x, H0 = _problem(dims, R, 3)
    iters = 6
    ref = oracle.nncp_hals(x, dims, H0, max_iters=iters, use_dimtree=False)
    P = int(np.prod(grid))
    procs = {r: _processor(x, H0, dims, grid, r, R) for r in range(P)}
    lams, fits, k = par_nncp.solve(procs, par_nncp.LocalComm(grid), iters)
    assert k == iters
    for r in range(P):
        np.testing.assert_allclose(fits[r], ref["fits"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(lams[r], ref["lam"], rtol=1e-10)
    for Hn, Hr in zip(_assemble(procs, dims, grid), ref["H"]):
        np.testing.assert_allclose(Hn, Hr, rtol=0, atol=1e-10)
    # every member of a slice holds the same, complete factor block
    for n in range(len(dims)):
        for k in range(grid[n]):
            members = par_nncp.slice_ranks(grid, n, k)
            for r in members[1:]:
                assert torch.equal(procs[r].H[n], procs[members[0]].H[n])


def test_layout_partitions_rows_exactly_once():
    dims, grid = (13, 7, 10), (3, 2, 2)
    P = int(np.prod(grid))
    for n, I in enumerate(dims):
        owners = np.zeros(I, dtype=int)
        for r in range(P):
            eng = OracleRank(dims, grid, par_nncp.grid_coords(r, grid), 2)
            bl, br, lo, rows, q, Q = eng.layout(n + 1)
            assert bl <= lo and lo + rows <= bl + br and Q == P // grid[n]
            owners[lo:lo + rows] += 1
        assert (owners == 1).all()


def test_stopping_rule_like_the_oracle():
    dims, grid, R = (10, 9, 8), (2, 1, 2), 2
    x, H0 = _problem(dims, R, 5)
    ref = oracle.nncp_hals(x, dims, H0, max_iters=200, tol=1e-4, use_dimtree=False)
    procs = {r: _processor(x, H0, dims, grid, r, R) for r in range(4)}
    lams, fits, k = par_nncp.solve(procs, par_nncp.LocalComm(grid), 200, tol=1e-4)
    assert k == ref["iters"] < 200
    np.testing.assert_allclose(fits[0], ref["fits"], atol=1e-10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, dims, grid, R, iters, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, H0 = _problem(dims, R, 7)
        p = _processor(x, H0, dims, grid, rank, R)
        comm = par_nncp.DistComm(grid, rank)
        lams, fits, k = par_nncp.solve({rank: p}, comm, iters, device="cpu")
        owned = [(p.layouts[n][2], p.owned(n).numpy().copy()) for n in range(len(dims))]
        out.put((rank, lams[rank], fits[rank], k, owned))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("grid", [(2, 1, 1), (1, 2, 2)])
def test_gloo_ranks_reproduce_the_sequential_oracle(grid):
    import torch.multiprocessing as mp
    dims, R, iters = (10, 8, 9), 3, 5
    world = int(np.prod(grid))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, dims, grid, R, iters, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x, H0 = _problem(dims, R, 7)
    ref = oracle.nncp_hals(x, dims, H0, max_iters=iters, use_dimtree=False)
    Hs = [np.full_like(h, np.nan) for h in ref["H"]]
    for rank, lam, fits, k, owned in res:
        assert k == iters
        np.testing.assert_allclose(fits, ref["fits"], atol=1e-10)
        np.testing.assert_allclose(lam, ref["lam"], rtol=1e-10)
        for n, (lo, rows) in enumerate(owned):
            Hs[n][lo:lo + rows.shape[0]] = rows
    for Hn, Hr in zip(Hs, ref["H"]):
        np.testing.assert_allclose(Hn, Hr, atol=1e-10)
