"""The allocation-free residual entry point against the allocating one.

ps_op_residual_noalloc exists for callers that may not allocate device
memory (memory owned by an external pool or arena, latency-critical loops,
no-allocation policies).  It must give the same residual and norm as
ps_op_residual through the C ABI, on consecutive calls that share its fixed
scratch array.  This file is collected last so that a failure here comes
after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_03563_gb300 import capi as M
    M.lib()
    return M


def _call_both(capi, n, order, box, seed):
    lib = capi.lib()
    g = capi.make_grid(n, (0.0, 0.0, 0.0), box)
    gh = order // 2
    shape = tuple(v + 2 * gh - 1 for v in reversed(n))
    gen = np.random.Generator(np.random.PCG64(seed))
    phi = torch.from_numpy(gen.standard_normal(shape)).cuda()
    f = torch.from_numpy(gen.standard_normal(shape)).cuda()
    r_ref = torch.zeros_like(phi)
    r_new = torch.full_like(phi, 0.0)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n_ref, n_new = C.c_double(), C.c_double()
    assert lib.ps_op_residual(C.byref(g), order, capi.DT_F64, C.c_void_p(phi.data_ptr()),
                              C.c_void_p(f.data_ptr()), C.c_void_p(r_ref.data_ptr()),
                              C.byref(n_ref), s) == capi.PS_OK
    assert lib.ps_op_residual_noalloc(C.byref(g), order, C.c_void_p(phi.data_ptr()),
                                      C.c_void_p(f.data_ptr()), C.c_void_p(r_new.data_ptr()),
                                      C.byref(n_new), s) == capi.PS_OK, lib.poisson_last_error()
    torch.cuda.synchronize()
    h = [(box[a] / n[a]) for a in range(3)]
    scale = float(phi.abs().max()) * sum(4.0 / x ** 2 for x in h)
    diff = float((r_new - r_ref).abs().max())
    assert diff <= 1e-13 * scale, (diff, scale)
    assert abs(n_new.value - n_ref.value) <= 1e-12 * n_ref.value
    return n_new.value


def test_noalloc_residual_matches_allocating_entry_point_twice(capi):
    # two calls in a row: the second reuses the scratch the first left behind
    a = _call_both(capi, (34, 20, 18), 2, (1.0, 1.0, 1.0), 1)
    b = _call_both(capi, (24, 40, 16), 4, (1.0, 0.7, 1.3), 2)
    assert a > 0 and b > 0 and a != b


def test_noalloc_rejects_grids_beyond_its_scratch(capi):
    lib = capi.lib()
    g = capi.make_grid(1024)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.ps_op_residual_noalloc(C.byref(g), 2, p, p, p, None, None)
    assert st == capi.PS_ERR_INVALID_ARG
    assert b"reduction slots" in lib.poisson_last_error()


def test_noalloc_at_the_edge_of_its_scratch(capi):
    # (2, 2048, 2048) intervals at order 2 launch exactly 1 x 256 x 128 = 32768
    # blocks, every reduction slot of the fixed scratch: accepted, and equal to
    # the allocating entry point
    _call_both(capi, (2, 2048, 2048), 2, (1.0, 1.0, 1.0), 3)
    # one more z-chunk of blocks (1 x 256 x 129 = 33024) is rejected before any GPU work
    lib = capi.lib()
    g = capi.make_grid((2, 2048, 2050))
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.ps_op_residual_noalloc(C.byref(g), 2, p, p, p, None, None)
    assert st == capi.PS_ERR_INVALID_ARG
    assert b"33024 reduction slots" in lib.poisson_last_error()
