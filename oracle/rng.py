"""SplitMix64 counter-based uniform numbers for the random initial iterate.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The numerical tests start MGRIT from a uniformly random iterate except at
t = 0, where it equals the initial condition (Sec. 5.3, numerical setup).  The
random value at time index n and grid index i is the SplitMix64 output
function (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the constants of Vigna's public-domain
splitmix64.c) applied to the state seed + (n * nx + i + 1) * 0x9E3779B97F4A7C15
(mod 2^64), mapped to [0, 1) by its top 53 bits.  The CUDA side implements
the same published function on its own.

Parity pin: the first outputs of the sequential generator with seed 1234567
(tests/golden/splitmix64.txt, from the published reference stream).
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def mix(z):
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def sequence(seed, count):
    """First ``count`` outputs of the sequential SplitMix64 stream."""
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + idx * GOLDEN
    return mix(state)


def uniform_grid(seed, n_index, nx):
    """U[0,1) values at time indices ``n_index`` (1-D array) and i = 0..nx-1,
    shape (len(n_index), nx)."""
    n_index = np.asarray(n_index, dtype=np.uint64)
    i = np.arange(nx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = n_index[:, None] * np.uint64(nx) + i[None, :] + np.uint64(1)
        state = np.uint64(seed) + ctr * GOLDEN
    z = mix(state)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
