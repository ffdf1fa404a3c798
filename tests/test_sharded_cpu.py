"""The time-sharded MGRIT driver on CPU (gloo, world size 2 and 4): level-0
CF-intervals in contiguous blocks over the ranks, one boundary row sent per
C-relaxation, the residual norm all-reduced, the coarse levels on rank 0.
The per-rank arithmetic comes from an executor the test builds on the
oracle (its fine operator and coarse cycle); the driver's iterates must then
equal the oracle's one-process MGRIT solve: the same residual history,
iteration count and C-points.  A rank that fails leaves the others with an
error from the process group instead of a hang."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleExecutor:
    """The per-rank arithmetic of the sharded solve done by the oracle: the
    rank's block of C-point rows in numpy, Phi^m by m applications of the
    fine operator, the coarse correction by the oracle's cycle."""

    def __init__(self, case, rank, world):
        from oracle import mgrit as omg
        self.omg = omg
        kind, p, q, c, m, levels, nu, nx, nt, seed = case
        self.h = omg.Hierarchy(p, kind, q, c, m, levels)
        self.m, self.nu, self.nt, self.seed = m, nu, nt, seed
        self.kr = nt // m // world

    def _phim(self, V):
        for _ in range(self.m):
            V = self.h.fine.apply(V)
        return V

    def global_initial(self, u0):
        u = self.omg.initial_iterate(u0.numpy(), self.nt, self.seed)
        return torch.from_numpy(np.ascontiguousarray(u[::self.m]))

    def set_block(self, rows):
        self.U = rows.numpy().copy()

    def get_block(self):
        return torch.from_numpy(self.U.copy())

    def c_relax(self):
        self.U[1:] = self._phim(self.U[:-1])

    def last_row(self):
        return torch.from_numpy(self.U[-1:].copy())

    def set_first_row(self, row):
        self.U[0] = row.numpy()[0]

    def residual(self):
        self.R = self._phim(self.U[:-1]) - self.U[1:]
        return float(np.sum(self.R * self.R))

    def residual_rows(self):
        return torch.from_numpy(self.R.copy())

    def add_block(self, rows):
        self.U += rows.numpy()

    def coarse_correction(self, res):
        r = res.numpy()
        e = np.zeros_like(r)
        self.omg.vcycle(self.h, 1, e, r, self.nu)
        return torch.from_numpy(e)


CASES = {  # kind, p, q, c, m, levels, nu, nx, nt, seed
    "erk3_vcycle": ("erk", 3, 3, 0.85, 4, 3, 1, 64, 256, 7),
    "sdirk3u5_two_level": ("sdirk", 5, 3, 4.0, 8, 2, 1, 64, 512, 3),
    "erk1_f_relax": ("erk", 1, 1, 0.85, 4, 3, 0, 32, 128, 1),
}


def _rank(rank, world, port, name, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import paper_2209_06916_gb300 as pkg
    from paper_2209_06916_gb300.sharded import ShardedSolver
    from workloads import ic_sin4
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = CASES[name]
        kind, p, qq, c, m, levels, nu, nx, nt, seed = case
        prm = pkg.make_params(nx, nt, c, p, kind=pkg.ERK if kind == "erk" else pkg.SDIRK, q=qq, m=m, levels=levels,
                              nu=nu, tol=1e-10, max_iter=40, seed=seed)
        s = ShardedSolver(prm, executor=OracleExecutor(case, rank, world), comm_device="cpu")
        out, st = s.solve(ic_sin4(nx))
        q.put((rank, None if out is None else out.numpy(), st))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(name, world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=600) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return got


@pytest.mark.parametrize("name,world", [("erk3_vcycle", 2), ("erk3_vcycle", 4), ("sdirk3u5_two_level", 2),
                                        ("erk1_f_relax", 4)])
def test_sharded_iterates_equal_one_process_solve(name, world):
    from oracle import mgrit as omg
    from workloads import ic_sin4
    got = _run(name, world)
    kind, p, q, c, m, levels, nu, nx, nt, seed = CASES[name]
    ref = omg.solve(omg.Hierarchy(p, kind, q, c, m, levels), ic_sin4(nx), nt, nu=nu, tol=1e-10, max_iter=40,
                    seed=seed)
    for rank, out, st in got:
        # every rank took the same stop decision on the same norms
        assert st["iterations"] == ref["iterations"] and st["converged"] == ref["converged"]
        h, hr = np.array(st["history"]), np.array(ref["history"])
        assert len(h) == len(hr)
        assert np.max(np.abs(h - hr) / hr[0]) < 1e-12
        assert st["ranks"] == world and st["intervals_per_rank"] == nt // m // world
    out = got[0][1]
    assert out.shape == (nt // m + 1, nx)
    assert np.max(np.abs(out - ref["u"][::m])) < 1e-12 * np.max(np.abs(ref["u"]))
    assert all(o is None for _, o, _ in got[1:])


def _rank_fails(rank, world, port, q):
    """Rank 1 raises before the first boundary exchange; rank 0 must get an
    error from the process group (short timeout), not wait forever."""
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import paper_2209_06916_gb300 as pkg
    from paper_2209_06916_gb300.sharded import ShardedSolver
    from workloads import ic_sin4
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    case = CASES["erk3_vcycle"]
    kind, p, qq, c, m, levels, nu, nx, nt, seed = case
    prm = pkg.make_params(nx, nt, c, p, m=m, levels=levels, nu=nu, tol=1e-10, max_iter=40, seed=seed)
    ex = OracleExecutor(case, rank, world)
    if rank == 1:
        def boom():
            raise RuntimeError("injected failure on rank 1")
        ex.c_relax = boom
    s = ShardedSolver(prm, executor=ex, comm_device="cpu", timeout_s=10.0)
    try:
        s.solve(ic_sin4(nx))
        q.put((rank, "finished"))
    except Exception as e:  # noqa: BLE001
        q.put((rank, type(e).__name__))
    q.close()
    q.join_thread()  # the result is in the pipe before the process ends
    os._exit(0)


def test_failed_rank_surfaces_as_error_on_the_others():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_fails, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    assert got[1] == "RuntimeError"
    assert got[0] != "finished"


def _rank_nan(rank, world, port, q):
    """Rank 1's residual turns NaN after the first iteration: every rank
    must stop with the divergence status, not read the norm as zero."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import paper_2209_06916_gb300 as pkg
    from paper_2209_06916_gb300.sharded import ShardedSolver
    from workloads import ic_sin4
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = CASES["erk3_vcycle"]
        kind, p, qq, c, m, levels, nu, nx, nt, seed = case
        prm = pkg.make_params(nx, nt, c, p, m=m, levels=levels, nu=nu, tol=1e-10, max_iter=40, seed=seed)
        ex = OracleExecutor(case, rank, world)
        if rank == 1:
            calls = {"n": 0}
            plain = ex.residual

            def residual():
                calls["n"] += 1
                v = plain()
                return float("nan") if calls["n"] > 1 else v
            ex.residual = residual
        s = ShardedSolver(prm, executor=ex, comm_device="cpu", timeout_s=60.0)
        _, st = s.solve(ic_sin4(nx))
        q.put((rank, st))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_nan_residual_is_divergence_on_every_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_nan, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, st in got.items():
        assert st["status"] == -4 and not st["converged"], (rank, st["status"])
        assert st["iterations"] == 1
