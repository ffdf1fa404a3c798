"""mgrit_residual_noalloc: the level-0 residual and its norm for callers that
cannot allocate device memory (code being captured into a CUDA graph, or
applications whose device memory is owned by a pool that must not be
bypassed).  Checked through the C ABI against the handle-based
mgrit_residual(level 0) on the same C-points, on two calls in a row (the
shared static scratch array must not leak one call's contents into the
next).  Collected last on purpose: the other tests have run if it fails.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg

pytestmark = pytest.mark.gpu


def _lib():
    lib = pkg.load_library()
    lib.mgrit_residual_noalloc.argtypes = [ctypes.POINTER(pkg.Params), ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("p,c,m,nx,K", [(3, 0.85, 8, 4096, 2048), (1, 0.85, 4, 96, 37)])
def test_noalloc_residual_matches_handle_residual(p, c, m, nx, K):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lib = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    prm = pkg.make_params(nx, m * K, c, p, m=m, levels=2)
    s = pkg.Solver(prm, stream=stream)
    rs = np.random.default_rng(11)
    for call in range(2):
        uC = rs.standard_normal((K + 1, nx)) * (1.0 + call)
        s.level_set(0, 0, uC)
        want_norm = s.residual(0)
        want_r = s.level_get(1, 1)[1:]
        d_uC = torch.tensor(uC, dtype=torch.float64, device="cuda")
        d_r = torch.full((K, nx), float("nan"), dtype=torch.float64, device="cuda")
        norm = ctypes.c_double(-1.0)
        rc = lib.mgrit_residual_noalloc(ctypes.byref(prm), d_uC.data_ptr(), K + 1, d_r.data_ptr(),
                                        ctypes.byref(norm), ctypes.c_void_p(stream))
        assert rc == 0, pkg.ERRORS.get(rc)
        torch.cuda.synchronize()
        got_r = d_r.cpu().numpy()
        assert np.max(np.abs(got_r - want_r)) < 1e-12 * np.max(np.abs(uC))
        assert abs(norm.value - want_norm) < 1e-12 * want_norm
    s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib()
    nx = 4096
    rows = 65536 // 4 + 2  # (rows - 1) * 4 tiles > 65536 partial slots
    prm = pkg.make_params(nx, 8, 0.85, 3, m=8, levels=2)
    norm = ctypes.c_double(0.0)
    rc = lib.mgrit_residual_noalloc(ctypes.byref(prm), ctypes.c_void_p(16), rows, ctypes.c_void_p(16),
                                    ctypes.byref(norm), None)
    assert rc == -1
