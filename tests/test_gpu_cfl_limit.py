"""Sec. 6.3.3 on the GPU: two-level MGRIT (m = 4, corrected operator, FCF,
2^10 x 2^12) slows down as the CFL number approaches the stability limit --
ERK3+U3 from 0.7 to 0.99 c_max, ERK5+U5 from 60% of c_max and failing by
80% -- with measured factors at or below the oracle's LFA prediction."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import coefficients as oco
from oracle import lfa
from workloads import ic_sin4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _solve(p, c, m=4, nx=1 << 10, nt=1 << 12):
    prm = pkg.make_params(nx, nt, c, p, kind=pkg.ERK, m=m, levels=2, nu=1, tol=1e-10, max_iter=30, seed=0)
    s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(torch.tensor(ic_sin4(nx), dtype=torch.float64, device="cuda"), out, allow_unconverged=True)
    s.close()
    return st


def test_erk3_u3_slows_near_the_limit():
    cm = oco.cfl_limit(3)
    fac = {}
    for f in (0.7, 0.99):
        st = _solve(3, f * cm)
        pred = lfa.two_level_factor(3, "erk", f * cm, 4, omit=10)
        assert st["conv_factor"] < 1.05 * pred, (f, st["conv_factor"], pred)
        fac[f] = (st["conv_factor"], st["iterations"], st["converged"])
    assert fac[0.7][2] and fac[0.99][0] > 2 * fac[0.7][0]
    assert fac[0.99][1] > fac[0.7][1]


def test_erk5_u5_degrades_from_sixty_percent():
    cm = oco.cfl_limit(5)
    st5 = _solve(5, 0.5 * cm)
    st7 = _solve(5, 0.7 * cm)
    st8 = _solve(5, 0.8 * cm)
    assert st5["converged"] and st7["conv_factor"] > st5["conv_factor"] + 0.05
    assert not st8["converged"] and st8["history"][-1] > 1e-6 * st8["history"][0]
