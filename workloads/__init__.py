"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds no arithmetic of the method: only the spatial mesh of
Sec. 2.1, the initial conditions of the numerical experiments and the problem
mixes of the batched and served workloads.  Both the CUDA path's tests and
the oracle draw their inputs from here.

  mesh(nx)                 x_i = -1 + i h, h = 2/nx, i = 0..nx-1 (Sec. 2.1)
  ic_sin4(nx)              u_0(x) = sin^4(pi x) (Sec. 5.3 numerical setup)
  ic_sin4_noise(nx, seed)  sin^4(pi x) plus N(0, 1e-2) noise (variance 1e-2)
  ic_fourier(nx, seed)     sum_{k=1}^{20} (a_k cos(pi k x) + b_k sin(pi k x))/k^2,
                           a_k, b_k ~ N(0, 1): a smooth periodic random IC
  batch_mix(count, seed)   parameter sets of the 512-solve batched workload
  batch_mix_sdirk(count, seed)  an implicit batch: SDIRK with upwind order
                           p in {1, 3, 5} (stage order q = min(p, 3))
"""
import numpy as np


def mesh(nx):
    h = 2.0 / nx
    return -1.0 + h * np.arange(nx, dtype=np.float64)


def ic_sin4(nx):
    return np.sin(np.pi * mesh(nx)) ** 4


def ic_sin4_noise(nx, seed, variance=1e-2):
    r = np.random.default_rng(seed)
    return ic_sin4(nx) + np.sqrt(variance) * r.standard_normal(nx)


def ic_fourier(nx, seed, modes=20):
    r = np.random.default_rng(seed)
    x = mesh(nx)
    a = r.standard_normal(modes)
    b = r.standard_normal(modes)
    u = np.zeros(nx, dtype=np.float64)
    for k in range(1, modes + 1):
        u += (a[k - 1] * np.cos(np.pi * k * x) + b[k - 1] * np.sin(np.pi * k * x)) / k ** 2
    return u


def batch_mix(count, seed, nx_choices=(256, 512, 1024, 2048, 4096, 8192),
              nt_choices=(512, 1024, 2048, 4096, 8192, 16384), orders=(1, 3, 5),
              cfl_range=(0.5, 0.95), m_choices=(4, 8, 16)):
    """Independent advection problems for the batched workload: nx, nt
    powers of two, upwind order with ERK of the same order, CFL uniform in
    cfl_range, coarsening factor m, per-solve seed = seed + index."""
    r = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append({
            "nx": int(r.choice(nx_choices)), "nt": int(r.choice(nt_choices)),
            "p": int(r.choice(orders)), "cfl": float(r.uniform(*cfl_range)),
            "m": int(r.choice(m_choices)), "seed": seed + i,
        })
    return out


def serving_stream(rate, duration, seed, sdirk_fraction=0.1, nx_max_sdirk=65536, nt_max_sdirk=131072,
                   nx_choices=(256, 512, 1024, 2048, 4096, 8192),
                   nt_choices=(512, 1024, 2048, 4096, 8192, 16384)):
    """Poisson arrivals (rate per second over `duration` s) of solve requests:
    a fraction `sdirk_fraction` are SDIRK5+U5 with CFL uniform in [2, 8] and
    nx, nt powers of two up to nx_max_sdirk / nt_max_sdirk; the rest follow
    batch_mix.  Returns (arrival times, list of parameter dicts)."""
    r = np.random.default_rng(seed)
    t, arrivals, reqs = 0.0, [], []
    i = 0
    while True:
        t += r.exponential(1.0 / rate)
        if t > duration:
            break
        if r.uniform() < sdirk_fraction:
            nxs = [n for n in (256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536) if n <= nx_max_sdirk]
            nts = [n for n in (512, 1024, 2048, 4096, 8192, 16384, 32768, 65536, 131072) if n <= nt_max_sdirk]
            req = {"nx": int(r.choice(nxs)), "nt": int(r.choice(nts)), "p": 5, "kind": "sdirk", "q": 5,
                   "cfl": float(r.uniform(2.0, 8.0)), "m": 4, "seed": seed + i}
        else:
            req = {"nx": int(r.choice(nx_choices)), "nt": int(r.choice(nt_choices)),
                   "p": int(r.choice((1, 3, 5))), "kind": "erk", "cfl": float(r.uniform(0.5, 0.95)),
                   "m": int(r.choice((4, 8, 16))), "seed": seed + i}
            req["q"] = req["p"]
        arrivals.append(t)
        reqs.append(req)
        i += 1
    return np.array(arrivals), reqs


def batch_mix_sdirk(count, seed, nx_choices=(1024, 2048, 4096, 8192), nt_choices=(1024, 2048, 4096, 8192),
                    orders=(1, 3, 5), cfl_range=(1.0, 4.0), m_choices=(4, 8, 16)):
    """Independent implicit problems: nx, nt powers of two, upwind order p
    with SDIRK of order q = min(p, 3), CFL uniform in cfl_range, coarsening
    factor m, per-solve seed = seed + index."""
    r = np.random.default_rng(seed)
    out = []
    for i in range(count):
        p = int(r.choice(orders))
        out.append({
            "nx": int(r.choice(nx_choices)), "nt": int(r.choice(nt_choices)), "p": p, "q": min(p, 3),
            "cfl": float(r.uniform(*cfl_range)), "m": int(r.choice(m_choices)), "seed": seed + i,
        })
    return out
