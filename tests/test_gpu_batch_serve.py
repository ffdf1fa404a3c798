"""Batched and served solves: every result is identical alone and in the mix
(the solves share the GPU but no data; their kernels are deterministic), the
server respects its in-flight limit and HBM budget, and latencies are
reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from workloads import batch_mix, ic_sin4_noise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _params(mix, precision):
    out = []
    for d in mix:
        out.append(pkg.make_params(d["nx"], d["nt"], d["cfl"], d["p"], kind=pkg.ERK, m=d["m"], levels=0, nu=1,
                                   tol=1e-10, max_iter=60, precision=precision, seed=d["seed"]))
    return out


def _alone(prm, u0):
    s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
    out = np.zeros((prm.nt // prm.m + 1, prm.nx))
    st = s.solve(u0, out, allow_unconverged=True)
    s.close()
    return out, st


SMALL = dict(nx_choices=(256, 512, 1024), nt_choices=(512, 1024, 2048))


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.MIXED])
def test_batch_results_equal_standalone(precision):
    mix = batch_mix(10, seed=100, **SMALL)
    prms = _params(mix, precision)
    u0s = [ic_sin4_noise(d["nx"], seed=d["seed"]) for d in mix]
    b = pkg.Batch(prms, nstreams=4)
    stats = b.solve(u0s, allow_unconverged=True)
    for i, (prm, u0) in enumerate(zip(prms, u0s)):
        want, st = _alone(prm, u0)
        got = b.get(i)
        assert stats[i]["iterations"] == st["iterations"]
        assert np.array_equal(got, want), i
    assert b.dof() == sum(d["nx"] * d["nt"] for d in mix)
    b.close()


def test_batch_sequential_equals_standalone_stepping():
    """The batched sequential-stepping baseline (all solves at once over the
    stream pool) gives each solve's standalone GPU sequential stepping bit for
    bit, and that agrees with the oracle's stepping."""
    from oracle import operators as oops
    mix = batch_mix(8, seed=11, **SMALL)
    prms = _params(mix, pkg.FP64)
    u0s = [torch.tensor(ic_sin4_noise(d["nx"], seed=d["seed"]), dtype=torch.float64, device="cuda") for d in mix]
    outs = [torch.empty(d["nx"], dtype=torch.float64, device="cuda") for d in mix]
    b = pkg.Batch(prms, nstreams=3)
    b.sequential(u0s, outs)
    for i, (prm, d) in enumerate(zip(prms, mix)):
        s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
        want = torch.empty_like(outs[i])
        s.fine_propagate(u0s[i], want, prm.nt)
        s.close()
        assert torch.equal(outs[i], want), i
        if i < 3:
            fine = oops.FineOperator(d["p"], "erk", d["p"], d["cfl"])
            u = u0s[i].cpu().numpy()
            for _ in range(prm.nt):
                u = fine.apply(u)
            got = outs[i].cpu().numpy()
            assert np.max(np.abs(got - u)) < 1e-12 * prm.nt * max(1.0, np.max(np.abs(u)))
    b.close()


def test_serving_continuous_batching():
    mix = batch_mix(16, seed=7, **SMALL)
    prms = _params(mix, pkg.MIXED)
    u0s = [ic_sin4_noise(d["nx"], seed=d["seed"]) for d in mix]
    arrivals = np.cumsum(np.random.default_rng(1).exponential(0.01, size=len(mix)))
    sizes = [pkg.estimate_bytes(p) for p in prms]
    budget = 3 * max(sizes)
    outs = [np.zeros((p.nt // p.m + 1, p.nx)) for p in prms]
    # the server times no launch geometry: tune the shapes first (on the idle
    # GPU), so the server and the standalone solves below use the same ones
    for p in prms:
        pkg.Solver(p).close()
    res, st = pkg.serve(prms, u0s, arrivals, budget, max_inflight=4, time_limit_s=120.0, u_outs=outs)
    assert st["completed"] + st["failed"] == len(mix)
    assert st["max_inflight"] <= 4 and st["max_mem_bytes"] <= budget and st["setup_s"] >= 0.0
    for i, (prm, u0) in enumerate(zip(prms, u0s)):
        want, s1 = _alone(prm, u0)
        if res[i]["status"] == 0:
            assert np.array_equal(outs[i], want), i
            assert res[i]["latency_ms"] > 0 and res[i]["finish_s"] >= arrivals[i]
    lat = sorted(r["latency_ms"] for r in res if r["status"] == 0)
    assert lat and np.percentile(lat, 99) >= np.percentile(lat, 50)
