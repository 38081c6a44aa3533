"""Algorithm 2 with its fine propagations split over ranks (the distributed
version of App. A, Algorithm 3), one process per GPU.

Each parareal iteration k (1-based; slices n < k are final, Algorithm 2)
has work = N - k + 1 fine propagations, one per slice n = k..N.  They are
split into contiguous blocks by App. A's integer arithmetic: with
chunk = floor(work / N_p) and remainder = work mod N_p, rank r takes the
positions start = r chunk + min(remainder, r) + 1 .. end = (r + 1) chunk +
min(remainder, r + 1) of the work list (end - start + 1 of them: App. A
writes myChunk = end - start, which undercounts by one), position p being
slice n = k - 1 + p.  Every rank computes the jumps
Delta^n = P F L(U^{n-1,k-1}) - G(U^{n-1,k-1}) of its block; the jumps are
gathered on rank 0, which runs the sequential correction
U^{n,k} = G(U^{n-1,k}) + Delta^n for n = k..N (Eq. 10) and the error of
Eq. 10, and broadcasts the new iterates and the error (App. A).  The
exchange per iteration is 5 Nx doubles per slice.

States are conserved moments V = (rho, rho u, E), float64 host arrays of
shape [5, Nx]; the propagators are supplied by the caller:

* ``fine(Vs)`` -- P F L of a stack of states [m, 5, Nx], all of one rank's
  block at once (the library runs them in one persistent launch:
  ``LibraryPropagators``);
* ``coarse(V)`` -- G over one coarse interval.

No propagator, collective or buffer of this module does any of the
method's arithmetic itself besides the jump difference, the correction sum
and the error maximum of Algorithm 2.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np


def slice_block(N: int, k: int, world: int, rank: int) -> tuple[int, int]:
    """First and last slice (1-based, inclusive) of rank's block at iteration
    k (1-based); last < first when the rank has no work.  App. A's start/end
    arithmetic on the work list n = k..N."""
    if N < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("need N >= 1, world >= 1 and 0 <= rank < world")
    work = max(N - k + 1, 0)
    chunk, rem = divmod(work, world)
    start = rank * chunk + min(rem, rank) + 1
    end = (rank + 1) * chunk + min(rem, rank + 1)
    return k - 1 + start, k - 1 + end


@dataclass
class Group:
    """The ranks taking part: a torch.distributed process group (or None for
    one process) and the device its collectives use ("cpu" for gloo, the
    rank's CUDA device for NCCL)."""
    pg: object = None
    device: str = "cpu"

    @property
    def world(self) -> int:
        if self.pg is None:
            return 1
        import torch.distributed as dist

        return dist.get_world_size(self.pg)

    @property
    def rank(self) -> int:
        if self.pg is None:
            return 0
        import torch.distributed as dist

        return dist.get_rank(self.pg)


def _bcast(group: Group, arr: np.ndarray) -> np.ndarray:
    if group.pg is None:
        return arr
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(arr)).to(group.device)
    dist.broadcast(t, src=0, group=group.pg)
    return t.cpu().numpy()


def _gather(group: Group, arr: np.ndarray):
    """Every rank's equally shaped arr, on rank 0 (None elsewhere)."""
    if group.pg is None:
        return [arr]
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(arr)).to(group.device)
    out = [torch.empty_like(t) for _ in range(group.world)] if group.rank == 0 else None
    dist.gather(t, out, dst=0, group=group.pg)
    return [o.cpu().numpy() for o in out] if out is not None else None


def parareal_sharded(V0: np.ndarray, N: int, K: int, fine: Callable[[np.ndarray], np.ndarray],
                     coarse: Callable[[np.ndarray], np.ndarray], group: Optional[Group] = None, tol: float = 0.0,
                     history: bool = False):
    """Algorithm 2 from the conserved initial state V0 [5, Nx] over N slices,
    K iterations (stopping early once the error of Eq. 10 is below tol > 0),
    with each iteration's fine propagations split over the ranks of group as
    App. A prescribes.  Collective: every rank of the group calls it with the
    same arguments.  Returns (U [N+1, 5, Nx], errors per iteration, and with
    history=True the iterates of every level [K+1, N+1, 5, Nx]); the same on
    every rank."""
    group = group or Group()
    world, rank = group.world, group.rank
    V0 = np.ascontiguousarray(V0, dtype=np.float64)
    nx = V0.shape[1]
    U = np.empty((N + 1, 5, nx))
    U[0] = V0
    if rank == 0:  # the first coarse guess U^{n,0} = G(U^{n-1,0})
        for n in range(1, N + 1):
            U[n] = coarse(U[n - 1])
    U = _bcast(group, U)
    hist = [U.copy()] if history else None
    errs = []
    for k in range(1, K + 1):
        work = max(N - k + 1, 0)
        cap = -(-work // world) if work else 0
        first, last = slice_block(N, k, world, rank)
        m = last - first + 1
        D = np.zeros((max(cap, 1), 5, nx))
        if m > 0:  # this rank's jumps Delta^n = P F L(U^{n-1,k-1}) - G(U^{n-1,k-1})
            F = np.asarray(fine(U[first - 1:last]), dtype=np.float64).reshape(m, 5, nx)
            for j in range(m):
                D[j] = F[j] - coarse(U[first - 1 + j])
        parts = _gather(group, D)
        Unew = np.empty_like(U)
        err = np.zeros(1)
        if rank == 0:
            Dall = np.zeros((N + 1, 5, nx))
            for r in range(world):
                fr, lr = slice_block(N, k, world, r)
                if lr >= fr:
                    Dall[fr:lr + 1] = parts[r][:lr - fr + 1]
            Unew[:] = U
            for n in range(k, N + 1):  # sequential correction (Eq. 10)
                Unew[n] = coarse(Unew[n - 1]) + Dall[n]
            err[0] = np.max(np.abs(Unew - U))
        Unew = _bcast(group, Unew)
        err = _bcast(group, err)
        U = Unew
        errs.append(float(err[0]))
        if history:
            hist.append(U.copy())
        if tol > 0.0 and errs[-1] < tol:
            break
    return (U, errs, np.stack(hist)) if history else (U, errs)


class LibraryPropagators:
    """One rank's propagators from the library: the fine propagations P F L
    of a block run as instances of one pr_batch (allocated once, for the
    largest block, as App. A advises) in one persistent launch over the
    block's instances (pr_batch_run_range); G is pr_coarse_step of a
    pr_init problem with the same grids (one resident slice state)."""

    def __init__(self, nx: int, nv: int, eps: float, T: float, N: int, max_block: int, L: float = 8.0,
                 x0: float = 0.0, x1: float = 1.0, bc: Optional[int] = None, scheme: Optional[int] = None,
                 precision: Optional[int] = None, cfl_f: float = 0.5, cfl_g: float = 0.5):
        import paper_2502_02704_gb300 as pr

        self.pr = pr
        bc = pr.PR_BC_OUTFLOW if bc is None else bc
        scheme = pr.PR_UPWIND if scheme is None else scheme
        precision = pr.PR_FP64 if precision is None else precision
        self.ctx = pr.pr_init(nx, x0, x1, bc, nv, L, eps, T, N, cfl_f, cfl_g, scheme, precision, max_batch=1)
        self.nf, self.dt = pr.pr_fine_steps_per_slice(self.ctx)
        self.dT = T / N
        inst = pr.instance(nx, nv, self.dt, L=L, x0=x0, x1=x1, bc=bc, eps=eps, scheme=scheme)
        self.batch = pr.pr_batch_create([inst] * max(1, max_block), precision)
        self.max_block = max(1, max_block)

    def fine(self, Vs: np.ndarray) -> np.ndarray:
        pr = self.pr
        m = len(Vs)
        if m > self.max_block:
            raise ValueError(f"block of {m} slices exceeds the {self.max_block} allocated")
        for j in range(m):
            pr.pr_batch_set_initial(self.batch, j, Vs[j], pr.PR_CONSERVED)
        pr.pr_batch_run_range(self.batch, 0, m, self.nf)
        return np.stack([pr.pr_batch_moments(self.batch, j) for j in range(m)])

    def coarse(self, V: np.ndarray) -> np.ndarray:
        return self.pr.pr_coarse_step(self.ctx, V, self.dT)

    def close(self) -> None:
        if self.batch is not None:
            self.pr.pr_batch_destroy(self.batch)
            self.batch = None
        if self.ctx is not None:
            self.pr.pr_destroy(self.ctx)
            self.ctx = None


def block_capacity(N: int, world: int) -> int:
    """Largest block any rank holds (the first iteration's): ceil(N / N_p)."""
    return -(-N // world)
