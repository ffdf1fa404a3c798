"""The time-sharded solve through the library (two ranks, each relaxing its
block of CF-intervals with libmgrit's level-0 kernels; rank 0 runs the
coarse levels of the whole problem) against the one-handle solve of the same
problem.  The ranks are two processes on the one GPU this runs on; they
exchange their rows on the host (gloo), so no kernel of one rank waits on
the other's.  Iteration counts are equal, the residual histories agree to
rounding (the norm is summed in another order), and the C-points agree with
the one-handle solve and with sequential stepping (oracle) within 1e-10."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {  # kind, p, q, c, m, levels, nx, nt
    "erk3u3": ("erk", 3, 3, 0.85, 8, 3, 512, 8 * 8 * 64),
    "sdirk3u5": ("sdirk", 5, 3, 4.0, 16, 3, 4096, 16 * 16 * 8),
}


def _params(pkg, case):
    kind, p, q, c, m, levels, nx, nt = case
    return pkg.make_params(nx, nt, c, p, kind=pkg.ERK if kind == "erk" else pkg.SDIRK, q=q, m=m, levels=levels,
                           nu=1, tol=1e-11, max_iter=40, seed=3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    import paper_2209_06916_gb300 as pkg
    from paper_2209_06916_gb300.sharded import ShardedSolver
    from workloads import ic_fourier
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = None
    try:
        case = CASES[name]
        s = ShardedSolver(_params(pkg, case), comm_device="cpu", timeout_s=300.0)
        out, st = s.solve(ic_fourier(case[6], seed=2))
        torch.cuda.synchronize()
        q.put((rank, None if out is None else out.cpu().numpy(), st))
    except Exception as e:  # noqa: BLE001
        q.put((rank, None, {"error": repr(e)}))
    finally:
        if s is not None:
            s.close()
        q.close()
        q.join_thread()
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["erk3u3", "sdirk3u5"])
def test_sharded_solve_equals_one_handle_solve(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2209_06916_gb300 as pkg
    from oracle import mgrit as omg
    from oracle import operators as oops
    from workloads import ic_fourier
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=900) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
    for _, _, st in got:
        assert "error" not in st, st
    case = CASES[name]
    kind, p, qq, c, m, levels, nx, nt = case
    torch.cuda.set_device(0)
    u0 = ic_fourier(nx, seed=2)
    s = pkg.Solver(_params(pkg, case), stream=torch.cuda.current_stream().cuda_stream)
    ref = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st1 = s.solve(torch.tensor(u0, device="cuda"), ref)
    ref = ref.cpu().numpy()
    s.close()
    for _, _, st in got:
        assert st["iterations"] == st1["iterations"] and st["converged"]
        h, h1 = np.array(st["history"]), np.array(st1["history"])
        big = h1 > 1e-8 * h1[0]
        assert np.max(np.abs(h[big] - h1[big]) / h1[big]) < 1e-8
    out = got[0][1]
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(out - ref)) < 1e-10 * scale
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(oops.FineOperator(p, kind, qq, c), g)[::m]
    assert np.max(np.abs(out - seq)) < 1e-10 * np.max(np.abs(seq))
