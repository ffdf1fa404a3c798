"""mgrit_residual_noalloc: the level-0 residual and its norm for callers that
cannot allocate device memory (code being captured into a CUDA graph, or
applications whose device memory is owned by a pool that must not be
bypassed).  Checked through the C ABI against the oracle's F-relaxation and
C-point residual (the plain definition r_k = Phi^m u_{(k-1)m} - u_{km}) and
against the handle-based mgrit_residual(level 0) on the same C-points, on
two calls in a row (the shared static scratch array must not leak one
call's contents into the next).  Collected last on purpose: the other tests
have run if it fails.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import mgrit as omg
from oracle import operators as oops


def _lib():
    lib = pkg.load_library()
    lib.mgrit_residual_noalloc.argtypes = [ctypes.POINTER(pkg.Params), ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p]
    return lib


def _oracle_residual(p, c, m, uC):
    """r_k, k = 1..K, by the oracle: the fine ERK step applied m times
    (F-relaxation from each C-point), then the C-point residual."""
    K, nx = uC.shape[0] - 1, uC.shape[1]
    fine = oops.FineOperator(p, "erk", p, c)
    u = np.zeros((K * m + 1, nx))
    u[::m] = uC
    g = np.zeros_like(u)
    omg.f_relax(fine, u, g, m)
    return omg.c_residual(fine, u, g, m)[1:]


# p, c, m, nx, K, compare with the handle path too
CASES = [
    (3, 0.85, 8, 4096, 2048, True),   # the ERK3+U3 bench shape
    (1, 0.85, 4, 96, 37, True),       # ragged tile count
    (5, 0.9, 4, 512, 64, True),       # ERK5 (beta_6 = 1/1280 term)
    (5, 0.9, 64, 64, 5, False),       # Phi^64 has 1921 taps before folding mod nx = 64
]


@pytest.mark.gpu
@pytest.mark.parametrize("p,c,m,nx,K,with_handle", CASES)
def test_noalloc_residual_matches_oracle_and_handle(p, c, m, nx, K, with_handle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lib = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    prm = pkg.make_params(nx, m * K, c, p, m=m, levels=2)
    s = pkg.Solver(prm, stream=stream) if with_handle else None
    rs = np.random.default_rng(11)
    for call in range(2):
        uC = rs.standard_normal((K + 1, nx)) * (1.0 + call)
        d_uC = torch.tensor(uC, dtype=torch.float64, device="cuda")
        d_r = torch.full((K, nx), float("nan"), dtype=torch.float64, device="cuda")
        norm = ctypes.c_double(-1.0)
        rc = lib.mgrit_residual_noalloc(ctypes.byref(prm), d_uC.data_ptr(), K + 1, d_r.data_ptr(),
                                        ctypes.byref(norm), ctypes.c_void_p(stream))
        assert rc == 0, pkg.ERRORS.get(rc)
        torch.cuda.synchronize()
        got_r = d_r.cpu().numpy()
        scale = np.max(np.abs(uC))
        want_r = _oracle_residual(p, c, m, uC)
        assert np.max(np.abs(got_r - want_r)) < 1e-12 * scale
        want_norm = float(np.sqrt(np.sum(want_r * want_r)))
        assert abs(norm.value - want_norm) < 1e-12 * want_norm
        if s is not None:
            s.level_set(0, 0, uC)
            h_norm = s.residual(0)
            h_r = s.level_get(1, 1)[1:]
            assert np.max(np.abs(got_r - h_r)) < 1e-12 * scale
            assert abs(norm.value - h_norm) < 1e-12 * h_norm
    if s is not None:
        s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch_on_the_host():
    """The size limit is checked on the host before any CUDA call.  Run only
    on a machine without a GPU: the pointers are placeholders, so if the
    check ever regressed, the call could only fail at its first CUDA call
    (no device) and never reach a kernel."""
    if torch.cuda.is_available():
        pytest.skip("host-side check, run where no GPU is present")
    import os
    if not os.path.exists(pkg.LIB_PATH):
        pytest.skip("libmgrit.so not built")
    lib = _lib()
    nx = 4096
    rows = 65536 // 4 + 2  # (rows - 1) * 4 tiles > 65536 partial slots
    prm = pkg.make_params(nx, 8, 0.85, 3, m=8, levels=2)
    norm = ctypes.c_double(0.0)
    rc = lib.mgrit_residual_noalloc(ctypes.byref(prm), ctypes.c_void_p(16), rows, ctypes.c_void_p(16),
                                    ctypes.byref(norm), None)
    assert rc == -1
    # the largest accepted size passes the check and then fails at the first
    # CUDA call on this GPU-less machine
    rc = lib.mgrit_residual_noalloc(ctypes.byref(prm), ctypes.c_void_p(16), rows - 1, ctypes.c_void_p(16),
                                    ctypes.byref(norm), None)
    assert rc == -6
    # even p is refused on the host (the entry point takes odd orders only)
    prm2 = pkg.make_params(nx, 8, 0.3, 2, m=8, levels=2)
    rc = lib.mgrit_residual_noalloc(ctypes.byref(prm2), ctypes.c_void_p(16), 3, ctypes.c_void_p(16),
                                    ctypes.byref(norm), None)
    assert rc == -1
