"""One problem's Parareal slices sharded over ranks, one GPU each.

Within a Parareal iteration the fine propagations of the N slices are
independent (Sec. 3.1, the parallel step of the method), so the slices are
cut into contiguous blocks, one per rank.  Every rank holds a context over
the whole problem and, per sweep k:

1. runs the fine phase on its own block (`mmp_sweep_fine`; slices before
   k - 1 are exact by Property 3.3 and skipped);
2. gathers the restriction records of every block (an all-gather of
   N x MMP_STAT_STRIDE doubles: the only data every rank needs);
3. runs the driver redundantly over all N slices (`mmp_sweep_coarse`: the
   sequential FP64 coarse sweep, iterator and convergence test), so every
   rank holds the same macro states and takes the same decisions;
4. hands the fine output at the end of its block (P values) to the next
   rank, which matches it into the first slice of its block in sweep k + 1.

The compute of every step runs in the library's kernels; this module only
moves records and one ensemble per rank and sweep.  `run_distributed` uses
torch.distributed (NCCL between GPUs, gloo on CPU); `run_lockstep` runs the
ranks of one process in turn, for checking the data flow on one GPU.
"""
from __future__ import annotations

import numpy as np

from . import mmp


def slice_block(N: int, rank: int, world: int) -> tuple[int, int]:
    """Slices [lo, hi) of a rank: contiguous blocks of sizes differing by at most one."""
    return N * rank // world, N * (rank + 1) // world


class Rank:
    """One rank's share of a sharded run.  Every rank calls the phases in
    the same order; which ranks send and receive the boundary ensemble
    follows from the sweep index alone, so the calls pair up."""

    def __init__(self, engine, rank: int, world: int):
        if world < 1 or not 0 <= rank < world:
            raise ValueError("rank outside the world")
        if engine.N < world:
            raise ValueError(f"{engine.N} slices cannot give each of {world} ranks a block")
        self.engine = engine
        self.rank, self.world = rank, world
        self.lo, self.hi = slice_block(engine.N, rank, world)
        self.width = -(-engine.N // world)  # the largest block
        self.k = 0
        self.done = False

    def start(self) -> None:
        self.engine.lift()
        self.k = 0
        self.done = False

    def fine(self) -> None:
        self.k += 1
        self.engine.fine(self.lo, self.hi)

    def records_out(self) -> np.ndarray:
        """This block's restriction records, padded to the largest block."""
        out = np.zeros((self.width, mmp.STAT_STRIDE))
        out[: self.hi - self.lo] = self.engine.records(self.lo, self.hi)
        return out

    def records_in(self, blocks) -> None:
        """Every rank's records (blocks[r] from records_out of rank r)."""
        for r, b in enumerate(blocks):
            if r == self.rank:
                continue
            lo, hi = slice_block(self.engine.N, r, self.world)
            self.engine.set_records(lo, hi, np.asarray(b)[: hi - lo])

    def coarse(self) -> bool:
        self.done = self.engine.coarse()
        return self.done

    def sends_boundary(self) -> bool:
        # the next rank's first slice hi is propagated in sweep k + 1 iff
        # hi >= k, and then reads this rank's output of slice hi - 1
        return not self.done and self.rank + 1 < self.world and self.hi >= self.k

    def receives_boundary(self) -> bool:
        return not self.done and self.rank > 0 and self.lo >= self.k

    def boundary_out(self):
        return self.engine.output(self.hi - 1)

    def boundary_in(self, ensemble) -> None:
        self.engine.set_output(self.lo - 1, ensemble)


def run_lockstep(engines) -> list:
    """All ranks in one process, phase by phase (a loop-back exchange):
    the data flow of run_distributed without a process group."""
    ranks = [Rank(e, i, len(engines)) for i, e in enumerate(engines)]
    for r in ranks:
        r.start()
    while True:
        for r in ranks:
            r.fine()
        blocks = [r.records_out() for r in ranks]
        for r in ranks:
            r.records_in(blocks)
        dones = [r.coarse() for r in ranks]
        if len(set(dones)) != 1:
            raise RuntimeError("ranks disagree on convergence")
        if dones[0]:
            break
        sent = {r.rank: r.boundary_out() for r in ranks if r.sends_boundary()}
        for r in ranks:
            if r.receives_boundary():
                r.boundary_in(sent[r.rank - 1])
    return [e.moments() for e in engines]


def run_distributed(engine, group=None):
    """This process's rank of a sharded run over a torch.distributed group
    (records all-gathered, the boundary ensemble sent to the next rank);
    returns the macro states, the same on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    r = Rank(engine, rank, world)
    dev = engine.comm_device()
    r.start()
    while True:
        r.fine()
        mine = torch.from_numpy(r.records_out()).to(dev)
        blocks = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(blocks, mine, group=group)
        r.records_in([b.cpu().numpy() for b in blocks])
        if r.coarse():
            break
        if r.sends_boundary():
            dist.send(r.boundary_out(), dist.get_global_rank(group, rank + 1) if group is not None else rank + 1,
                      group=group)
        if r.receives_boundary():
            buf = engine.empty_output()
            dist.recv(buf, dist.get_global_rank(group, rank - 1) if group is not None else rank - 1, group=group)
            r.boundary_in(buf)
    return engine.moments()


class LibraryEngine:
    """A rank's engine: a context of libmmp over the whole problem on this
    process's GPU; the fine phase covers the rank's block only."""

    def __init__(self, problem, stream=None):
        self.solver = mmp.Solver(problem, stream)
        self.problem = problem
        self.N = problem.N

    def _ctx(self):
        return self.solver.ctx

    def comm_device(self):
        import torch
        return torch.device("cuda", torch.cuda.current_device())

    def lift(self) -> None:
        mmp.mmp_lift(self._ctx())

    def fine(self, lo: int, hi: int) -> None:
        mmp.mmp_sweep_fine(self._ctx(), 0, lo, hi)

    def records(self, lo: int, hi: int) -> np.ndarray:
        return mmp.mmp_get_records(self._ctx(), 0, lo, hi)

    def set_records(self, lo: int, hi: int, rows) -> None:
        mmp.mmp_set_records(self._ctx(), 0, lo, hi, rows)

    def coarse(self) -> bool:
        return mmp.mmp_sweep_coarse(self._ctx(), 0)

    def empty_output(self):
        import torch
        return torch.empty(self.problem.P, dtype=self.solver.dtype(), device="cuda")

    def output(self, n: int):
        buf = self.empty_output()
        mmp.mmp_get_output(self._ctx(), 0, n, buf.data_ptr(), False)
        return buf

    def set_output(self, n: int, ensemble) -> None:
        import torch
        t = ensemble.to(device="cuda", dtype=self.solver.dtype()).contiguous()
        mmp.mmp_set_output(self._ctx(), 0, n, t.data_ptr(), False)
        torch.cuda.current_stream().synchronize()

    def moments(self) -> np.ndarray:
        return self.solver.moments(0)

    def status(self) -> dict:
        return self.solver.status(0)

    def close(self) -> None:
        self.solver.close()
