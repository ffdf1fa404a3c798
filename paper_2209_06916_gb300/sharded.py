"""Time-sharded MGRIT over the ranks of a torch.distributed process group.

The paper parallelises in time only (Sec. 6.3.2): each process holds a
contiguous block of time points.  Here rank r of R holds the level-0
C-points of the CF-intervals a_r .. a_r + K_r - 1 (K_r = nt / (m R)), i.e.
rows a_r .. a_r + K_r of the C-point iterate, and relaxes them with the
library's level-0 kernels in a handle of its own.  One iteration of the
linear method of Sec. 2.2 then needs these exchanges:

  * after every C-relaxation, one n_x row: the C-point that rank r's last
    interval produced is row 0 (the start of the first interval) of rank
    r + 1 (point-to-point send / receive);
  * the residual norm: the squared norms of the blocks are summed over the
    ranks (all-reduce), so every rank takes the same stop decision;
  * the coarse-grid correction: rank 0 gathers the residual rows (the
    level-1 right-hand side), runs the coarse levels of the full hierarchy
    (mgrit_coarse_correct on a handle of the whole problem) and scatters
    the correction rows, each rank receiving rows a_r .. a_r + K_r.

The level-0 work, which dominates, is divided by R; the coarse levels run
on one GPU (they hold 1/m of the level-0 rows and less).  Transport is the
group's backend: NCCL on GPUs (device tensors), gloo for CPU tests (host
tensors).  No rank reads another rank's memory.

An executor does the per-rank arithmetic; the default one calls the
library (FP64 handles).  The iteration is the single-GPU solve's: the same
pre-relaxation, residual, stop test and coarse correction, so the iterates
equal a one-rank solve's up to the order of the norm's summation.
"""
import math

import numpy as np

from . import FP64, Solver, make_params


class HandleExecutor:
    """Per-rank arithmetic through libmgrit: a handle for the rank's block
    (nt = K_r m, two levels; only its level-0 kernels run) and, on rank 0, a
    handle of the whole problem for the initial iterate and the coarse
    levels."""

    def __init__(self, params, rank, world, stream=0):
        import torch
        self.torch = torch
        if params.precision != FP64:
            raise ValueError("the time-sharded solve runs FP64 handles")
        self.nx, self.m = params.nx, params.m
        K = params.nt // params.m
        self.kr = K // world
        loc = make_params(params.nx, self.kr * params.m, params.cfl, params.order_p, kind=params.rk_kind,
                          q=params.rk_order_q, m=params.m, levels=2, nu=params.nu, tol=params.tol,
                          max_iter=params.max_iter, seed=params.seed, coarse_op=params.coarse_op,
                          coarse_solve=params.coarse_solve, m_coarse=params.m_coarse)
        self.block = Solver(loc, stream=stream)
        self.full = Solver(params, stream=stream) if rank == 0 else None
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def empty(self, rows):
        return self.torch.empty((rows, self.nx), dtype=self.torch.float64, device=self.dev)

    def global_initial(self, u0):
        """The C-point rows of the random initial iterate of the whole
        problem (the library's seeded generator), row 0 = u0."""
        self.full.set_initial(u0)
        rows = self.full.level_rows(0, 0)
        out = self.empty(rows)
        self.full.rows_io(0, 0, 0, rows, out, 0)
        return out

    def set_block(self, rows):
        # the whole level (row 0 into both C-point buffers, which the handle
        # swaps per C-relaxation: rank 0 keeps u0 there)
        self.block.level_put(0, 0, rows.contiguous())

    def get_block(self):
        out = self.empty(self.kr + 1)
        self.block.rows_io(0, 0, 0, self.kr + 1, out, 0)
        return out

    def c_relax(self):
        self.block.relax(0, 1)

    def last_row(self):
        out = self.empty(1)
        self.block.rows_io(0, 0, self.kr, 1, out, 0)
        return out

    def set_first_row(self, row):
        self.block.rows_io(0, 0, 0, 1, row.to(self.dev).contiguous(), 1)

    def residual(self):
        """Residual rows of the block into its level-1 RHS; the squared norm."""
        nrm = self.block.residual(0)
        return nrm * nrm

    def residual_rows(self):
        out = self.empty(self.kr)
        self.block.rows_io(1, 1, 1, self.kr, out, 0)
        return out

    def add_block(self, rows):
        self.block.rows_io(0, 0, 0, self.kr + 1, rows.contiguous(), 2)

    def coarse_correction(self, res):
        """Rank 0: the correction rows e (K + 1 rows) for the residual rows
        res (K + 1 rows, row 0 zero) of the whole problem."""
        K1 = res.shape[0]
        zero = self.torch.zeros_like(res)
        self.full.rows_io(0, 0, 0, K1, zero, 1)
        self.full.rows_io(1, 1, 0, K1, res.contiguous(), 1)
        self.full.coarse_correct()
        out = self.empty(K1)
        self.full.rows_io(0, 0, 0, K1, out, 0)
        return out

    def sync(self):
        self.torch.cuda.synchronize()

    def close(self):
        self.block.close()
        if self.full is not None:
            self.full.close()


class ShardedSolver:
    """MGRIT with the level-0 CF-intervals in contiguous blocks over the
    ranks of `group` (torch.distributed, initialised by the caller).  nt/m
    must be a multiple of the world size.  `executor` (default: a
    HandleExecutor) does the per-rank arithmetic; `comm_device` is where the
    backend takes its tensors ("cuda" for NCCL, "cpu" for gloo)."""

    def __init__(self, params, group=None, executor=None, comm_device=None, stream=0, timeout_s=600.0):
        import datetime

        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        # bound on every point-to-point wait: a rank that failed or left ends
        # the others' solve with an error instead of a hang
        self.timeout = datetime.timedelta(seconds=timeout_s)
        self.params = params
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        K = params.nt // params.m
        if params.nt % params.m or K % self.world:
            raise ValueError("nt / m = %d CF-intervals do not split evenly over %d ranks" % (K, self.world))
        self.K, self.kr = K, K // self.world
        self.a = self.rank * self.kr
        self.ex = executor if executor is not None else HandleExecutor(params, self.rank, self.world, stream)
        if comm_device is None:
            comm_device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        self.cdev = torch.device(comm_device)

    # -- transport ---------------------------------------------------------
    def _to_comm(self, t):
        return t.to(self.cdev).contiguous()

    def _exchange_boundary(self):
        """Rank r's last C-point row becomes row 0 of rank r + 1."""
        dist, torch = self.dist, self.torch
        req = None
        if self.rank + 1 < self.world:
            out = self._to_comm(self.ex.last_row())
            req = dist.isend(out, self.rank + 1, group=self.group)
        if self.rank > 0:
            inb = torch.empty((1, self.params.nx), dtype=torch.float64, device=self.cdev)
            if not dist.irecv(inb, self.rank - 1, group=self.group).wait(self.timeout):
                raise RuntimeError("boundary row from rank %d not received" % (self.rank - 1))
            self.ex.set_first_row(inb)
        if req is not None and not req.wait(self.timeout):
            raise RuntimeError("boundary row to rank %d not delivered" % (self.rank + 1))

    def _all_sum(self, x):
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.cdev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return float(t.item())

    def _gather_rows(self, rows):
        """Rows of every rank, in rank order, on rank 0 (None elsewhere)."""
        dist, torch = self.dist, self.torch
        src = self._to_comm(rows)
        if self.rank == 0:
            parts = [torch.empty_like(src) for _ in range(self.world)]
            dist.gather(src, parts, dst=0, group=self.group)
            return torch.cat(parts, 0)
        dist.gather(src, None, dst=0, group=self.group)
        return None

    def _scatter_blocks(self, full):
        """Rank r receives rows a_r .. a_r + K_r of `full` (rank 0's)."""
        dist, torch = self.dist, self.torch
        out = torch.empty((self.kr + 1, self.params.nx), dtype=torch.float64, device=self.cdev)
        if self.rank == 0:
            full = self._to_comm(full)
            parts = [full[r * self.kr:r * self.kr + self.kr + 1].contiguous() for r in range(self.world)]
            dist.scatter(out, parts, src=0, group=self.group)
        else:
            dist.scatter(out, None, src=0, group=self.group)
        return out

    # -- the method ------------------------------------------------------------
    def _pre_relax_and_residual(self):
        for _ in range(self.params.nu):
            self.ex.c_relax()
            self._exchange_boundary()
        sq = self._all_sum(self.ex.residual())
        # a NaN sum stays NaN (the stop test reads it as divergence); only a
        # rounding-negative sum is clamped
        return math.sqrt(sq) if sq >= 0.0 else (sq if math.isnan(sq) else 0.0)

    def solve(self, u0):
        """Solve from the initial condition u0 (host array or tensor of nx
        values; rank 0's is used).  Returns (C-point rows of the whole
        problem on rank 0, None elsewhere; stats dict on every rank)."""
        torch = self.torch
        u0 = torch.as_tensor(np.asarray(u0) if not torch.is_tensor(u0) else u0, dtype=torch.float64)
        init = self.ex.global_initial(u0) if self.rank == 0 else None
        self.ex.set_block(self._scatter_blocks(init).to(self._dev_of_executor()))
        p = self.params
        history = [self._pre_relax_and_residual()]
        it, status = 0, 0
        while True:
            nrm = history[-1]
            if not math.isfinite(nrm) or (it > 0 and nrm > 1e3 * history[0]):
                status = -4
                break
            if nrm <= p.tol * history[0]:
                break
            if it >= p.max_iter:
                status = -3
                break
            res = self._gather_rows(self.ex.residual_rows())
            corr = None
            if self.rank == 0:
                full = torch.zeros((self.K + 1, p.nx), dtype=torch.float64, device=res.device)
                full[1:] = res
                corr = self.ex.coarse_correction(full.to(self._dev_of_executor()))
            self.ex.add_block(self._scatter_blocks(corr).to(self._dev_of_executor()))
            history.append(self._pre_relax_and_residual())
            it += 1
        rows = self._gather_rows(self.ex.get_block()[1:])
        out = None
        if self.rank == 0:
            out = torch.cat([u0.reshape(1, -1).to(rows.device), rows], 0)
        stats = {"iterations": it, "converged": status == 0, "status": status, "history": history,
                 "ranks": self.world, "intervals_per_rank": self.kr}
        return out, stats

    def _dev_of_executor(self):
        dev = getattr(self.ex, "dev", None)
        return dev if dev is not None else self.torch.device("cpu")

    def close(self):
        if hasattr(self.ex, "close"):
            self.ex.close()
