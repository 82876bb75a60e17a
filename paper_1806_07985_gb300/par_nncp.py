"""Par-NNCP driver (Alg. 2; Sec. IV-C): the collectives between the
per-processor library calls (``nncp.ParRank``, the ``nncp_par_*`` C ABI).

Every computation -- the local MTTKRP through the local dimension tree, the
HALS update of the owned rows, the Grams, lambda, the fit -- runs in the
library; this module moves data between processors:

  * Reduce-Scatter of each processor's local MTTKRP block over its mode-n
    processor slice, giving every member the owned rows of M(n);
  * All-Reduce over every processor of the R*R + 1 partial sums (W^T W and
    <M, W>) from which each processor forms lambda, G_n and the fit;
  * All-Gather of the owned rows of H(n) over the mode-n slice into the
    factor block every slice member keeps.

Two communicators implement the three collectives: ``DistComm`` (one
processor per process, ``torch.distributed``: NCCL between GPUs, or gloo on
CPU tensors) and ``LocalComm`` (every processor of the grid inside this
process, run one after another).  ``solve`` drives a dict of processors
{rank: Processor} with either.

Ranks and grid coordinates: rank = p_1 + P_1 (p_2 + P_2 (...)), mode 1
fastest.  The members of a mode-n slice are listed in rank order, which is
the order of their other coordinates with mode 1 fastest: the order in which
the library cuts the block rows into owned pieces.
"""

from __future__ import annotations

import math


def grid_coords(rank, grid):
    coords = []
    for P in grid:
        coords.append(rank % P)
        rank //= P
    return tuple(coords)


def grid_rank(coords, grid):
    r, stride = 0, 1
    for c, P in zip(coords, grid):
        r += c * stride
        stride *= P
    return r


def slice_ranks(grid, n, k):
    """Ranks of the mode-n processor slice p_n = k, in slice order."""
    return [r for r in range(math.prod(grid)) if grid_coords(r, grid)[n] == k]


def block_range(I, P, k):
    """Rows [lo, lo + rows) of block k of a mode of length I cut in P blocks."""
    lo = k * I // P
    return lo, (k + 1) * I // P - lo


def local_block(x, dims, grid, coords):
    """The processor's block of a global tensor (flat, mode-1 fastest numpy
    array) as a flat mode-1-fastest array: data placement for callers that
    hold the whole tensor, such as tests."""
    import numpy as np
    arr = np.asarray(x).reshape(tuple(reversed(dims)))
    sl = []
    for n in reversed(range(len(dims))):
        lo, rows = block_range(dims[n], grid[n], coords[n])
        sl.append(slice(lo, lo + rows))
    return np.ascontiguousarray(arr[tuple(sl)]).reshape(-1)


class Processor:
    """One grid position: its library object and device buffers."""

    def __init__(self, engine, X_local, H_block, layouts):
        import torch
        self.engine = engine
        self.X = X_local
        self.H = list(H_block)             # N factor blocks, block_rows x R
        self.layouts = layouts             # per mode: the nncp_par_layout tuple
        self.M = [torch.empty_like(h) for h in self.H]
        engine.set_data(self.X, self.H)

    def owned(self, n):
        block_lo, _, owned_lo, owned_rows, _, _ = self.layouts[n]
        o = owned_lo - block_lo
        return self.H[n][o:o + owned_rows]


def _counts(layout):
    """Owned-row counts of every member of the processor's mode-n slice, and
    the offsets of their pieces in the block (the cut the library makes)."""
    _, L, _, _, _, Q = layout
    lo = [q * L // Q for q in range(Q + 1)]
    return [lo[q + 1] - lo[q] for q in range(Q)], lo[:Q]


class DistComm:
    """The collectives of this process's single processor over
    torch.distributed (every process creates every slice group, in the same
    order, as torch.distributed requires)."""

    def __init__(self, grid, rank):
        import torch.distributed as dist
        self.dist = dist
        self.grid = tuple(grid)
        self.rank = rank
        self.groups = {}
        for n in range(len(grid)):
            for k in range(grid[n]):
                members = slice_ranks(grid, n, k)
                g = dist.new_group(members)
                if rank in members:
                    self.groups[n] = (g, members)

    def reduce_scatter(self, n, blocks, layouts):
        import torch
        (r, Mb), = blocks.items()
        g, members = self.groups[n]
        counts, offs = _counts(layouts[r][n])
        q = members.index(r)
        width = max(counts) if counts else 0
        R = Mb.shape[1]
        inp = torch.zeros((len(members) * width, R), dtype=Mb.dtype, device=Mb.device)
        for i, (c, o) in enumerate(zip(counts, offs)):
            inp[i * width:i * width + c] = Mb[o:o + c]
        out = torch.empty((width, R), dtype=Mb.dtype, device=Mb.device)
        self.dist.reduce_scatter_tensor(out, inp, group=g)
        return {r: out[:counts[q]]}

    def all_gather(self, n, owned, layouts):
        import torch
        (r, Ho), = owned.items()
        g, members = self.groups[n]
        counts, _ = _counts(layouts[r][n])
        width = max(counts) if counts else 0
        R = Ho.shape[1]
        inp = torch.zeros((width, R), dtype=Ho.dtype, device=Ho.device)
        inp[:Ho.shape[0]] = Ho
        out = torch.empty((len(members) * width, R), dtype=Ho.dtype, device=Ho.device)
        self.dist.all_gather_into_tensor(out, inp, group=g)
        return {r: torch.cat([out[i * width:i * width + c] for i, c in enumerate(counts)])}

    def all_reduce(self, vals, device):
        import torch
        (r, v), = vals.items()
        t = torch.tensor(v, dtype=torch.float64, device=device)
        self.dist.all_reduce(t)
        return {r: t.tolist()}


class LocalComm:
    """Every processor of the grid in this process: the same collectives on
    the dict of all processors' buffers (sums in rank order)."""

    def __init__(self, grid):
        self.grid = tuple(grid)

    def reduce_scatter(self, n, blocks, layouts):
        out = {}
        for k in range(self.grid[n]):
            members = slice_ranks(self.grid, n, k)
            total = blocks[members[0]].clone()
            for r in members[1:]:
                total += blocks[r]
            counts, offs = _counts(layouts[members[0]][n])
            for q, r in enumerate(members):
                out[r] = total[offs[q]:offs[q] + counts[q]]
        return out

    def all_gather(self, n, owned, layouts):
        import torch
        out = {}
        for k in range(self.grid[n]):
            members = slice_ranks(self.grid, n, k)
            block = torch.cat([owned[r] for r in members])
            for r in members:
                out[r] = block
        return out

    def all_reduce(self, vals, device=None):
        ranks = sorted(vals)
        total = [0.0] * len(vals[ranks[0]])
        for r in ranks:
            total = [a + b for a, b in zip(total, vals[r])]
        return {r: list(total) for r in ranks}


def solve(procs, comm, max_iters, tol=0.0, device=None):
    """Par-NNCP (Alg. 2) on the processors `procs` ({rank: Processor}, the
    factor blocks holding the initial values of the owned rows) with the
    communicator `comm`.  Returns ({rank: lambda}, {rank: fits}, iterations);
    the factor blocks hold the column-normalised result."""
    N = len(next(iter(procs.values())).H)
    layouts = {r: p.layouts for r, p in procs.items()}
    alpha = comm.all_reduce({r: [p.engine.alpha_local(p.X)] for r, p in procs.items()}, device)
    for r, p in procs.items():
        p.engine.begin(alpha[r][0], tol)

    def finish_mode(n, parts, init):
        sums = comm.all_reduce(parts, device)
        stop = False
        for r, p in procs.items():
            _, s = p.engine.normalize(n + 1, sums[r], p.owned(n), init)
            stop = stop or s
        blocks = comm.all_gather(n, {r: p.owned(n) for r, p in procs.items()}, layouts)
        for r, p in procs.items():
            p.H[n].copy_(blocks[r])
        return stop

    # initialisation (Alg. 2, first loop, plus the normalisation of Alg. 3)
    for n in range(N):
        finish_mode(n, {r: p.engine.update(n + 1, None, p.owned(n)) for r, p in procs.items()}, True)
    iters = 0
    for _ in range(max_iters):
        iters += 1
        stop = False
        for n in range(N):
            for p in procs.values():
                p.engine.mttkrp(n + 1, p.M[n])
            owned_M = comm.reduce_scatter(n, {r: p.M[n] for r, p in procs.items()}, layouts)
            parts = {r: p.engine.update(n + 1, owned_M[r], p.owned(n)) for r, p in procs.items()}
            stop = finish_mode(n, parts, False)
        if stop:
            break
    lams, fits = {}, {}
    for r, p in procs.items():
        lams[r], fits[r] = p.engine.result()
    return lams, fits, iters
