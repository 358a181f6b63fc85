"""Op-level entry points of the C ABI (single hot-path kernels on caller buffers).

dtype of the tensors selects the kernel instantiation: float64, float32 or
bfloat16 storage.  Grids are Cartesian with n intervals per axis.
"""
from __future__ import annotations

import ctypes as C

from . import capi
from .capi import check, lib

_DT = {"float64": capi.DT_F64, "float32": capi.DT_F32, "bfloat16": capi.DT_BF16}


def _dt(t):
    return _DT[str(t.dtype).replace("torch.", "")]


def _p(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("contiguous CUDA tensor required")
    return C.c_void_p(t.data_ptr())


def _s(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def apply(n, order, phi, out, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    g = capi.make_grid(n, lo, hi)
    check(lib().ps_op_apply(C.byref(g), order, _dt(phi), _p(phi), _p(out), _s(stream)), "ps_op_apply")


def residual(n, order, phi, f, r, lo=(0, 0, 0), hi=(1, 1, 1), stream=None) -> float:
    g = capi.make_grid(n, lo, hi)
    nrm = C.c_double()
    check(lib().ps_op_residual(C.byref(g), order, _dt(phi), _p(phi), _p(f), _p(r), C.byref(nrm),
                               _s(stream)), "ps_op_residual")
    return nrm.value


def sweep(n, order, phi, f, omega=1.0, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    g = capi.make_grid(n, lo, hi)
    check(lib().ps_op_sweep(C.byref(g), order, _dt(phi), _p(phi), _p(f), float(omega), _s(stream)),
          "ps_op_sweep")


def restrict(n, order, r_fine, f_coarse, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    g = capi.make_grid(n, lo, hi)
    check(lib().ps_op_restrict(C.byref(g), order, _dt(r_fine), _p(r_fine), _p(f_coarse), _s(stream)),
          "ps_op_restrict")


def restrict_red(n, order, r_fine, f_coarse, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    """Full weighting of a 7-point residual that is zero on the black nodes (ps_op_restrict_red)."""
    g = capi.make_grid(n, lo, hi)
    check(lib().ps_op_restrict_red(C.byref(g), order, _dt(r_fine), _p(r_fine), _p(f_coarse), _s(stream)),
          "ps_op_restrict_red")


def prolong(n, order, e_coarse, phi_fine, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    g = capi.make_grid(n, lo, hi)
    check(lib().ps_op_prolong(C.byref(g), order, _dt(phi_fine), _p(e_coarse), _p(phi_fine), _s(stream)),
          "ps_op_prolong")


def multipole_moments(n, order, rho, origin, lmax, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    g = capi.make_grid(n, lo, hi)
    q = (C.c_double * ((lmax + 1) ** 2))()
    o = (C.c_double * 3)(*origin)
    check(lib().ps_op_multipole_moments(C.byref(g), order, _p(rho), o, lmax, q, _s(stream)),
          "ps_op_multipole_moments")
    return list(q)


def multipole_boundary(n, order, q, origin, lmax, G, phi, lo=(0, 0, 0), hi=(1, 1, 1), stream=None):
    g = capi.make_grid(n, lo, hi)
    qq = (C.c_double * len(q))(*q)
    o = (C.c_double * 3)(*origin)
    check(lib().ps_op_multipole_boundary(C.byref(g), order, qq, o, lmax, float(G), _p(phi), _s(stream)),
          "ps_op_multipole_boundary")


def scale_to_fp32(x, e, out, stream=None):
    """out = x * 2^e rounded to FP32 (the refinement residual's conversion);
    x float64, out float32, both contiguous CUDA tensors of the same size."""
    import torch
    if x.dtype != torch.float64 or out.dtype != torch.float32 or x.numel() != out.numel():
        raise ValueError("x must be float64 and out float32 of the same size")
    check(lib().ps_op_scale_to_fp32(_p(x), x.numel(), int(e), _p(out), _s(stream)), "ps_op_scale_to_fp32")


def add_scaled_fp32(e, p, phi, stream=None):
    """phi += e * 2^p (the refinement's correction step); e float32, phi
    float64, both contiguous CUDA tensors of the same size."""
    import torch
    if e.dtype != torch.float32 or phi.dtype != torch.float64 or e.numel() != phi.numel():
        raise ValueError("e must be float32 and phi float64 of the same size")
    check(lib().ps_op_add_scaled_fp32(_p(e), e.numel(), int(p), _p(phi), _s(stream)), "ps_op_add_scaled_fp32")


def compact_operators(order, h, nlevels):
    """Level operators of the compact-stencil multigrid (Sec. 2.1.3) as a compact
    solve builds them, computed on the host: per level l (spacing h 2^l) the
    class weights (centre, faces, edges, corners) of the operator (compact L_h,
    then Galerkin products), the SPAI weights M and omega of Table 1.  Returns
    (a, m, omega) as nested lists [nlevels][4], [nlevels][4], [nlevels]."""
    a = (C.c_double * (4 * nlevels))()
    m = (C.c_double * (4 * nlevels))()
    w = (C.c_double * nlevels)()
    check(lib().poisson_compact_operators(int(order), float(h), int(nlevels), a, m, w),
          "poisson_compact_operators")
    return ([list(a[4 * l:4 * l + 4]) for l in range(nlevels)],
            [list(m[4 * l:4 * l + 4]) for l in range(nlevels)], list(w))


def probe_fp64(kind, blocks, iters, out, stream=None):
    """Launch the FP64 pipe throughput probe (kind 0: fused multiply-adds, 1:
    adds) on `stream`; out is a float64 CUDA tensor of at least `blocks`
    elements.  Returns the number of FP64 instructions the launch issues; the
    caller times it."""
    import torch
    if out.dtype != torch.float64 or out.numel() < blocks:
        raise ValueError("out must be float64 with at least `blocks` elements")
    n = C.c_double()
    check(lib().ps_probe_fp64(int(kind), int(blocks), int(iters), _p(out), C.byref(n), _s(stream)),
          "ps_probe_fp64")
    return n.value


def probe_bounded_wait(first_wait, out, stream=None):
    """Run the tile kernels' bounded mbarrier wait on a barrier nothing arrives
    at (first_wait True: the 2 s limit of a kernel's first failing wait; False:
    the 1 ms limit of later waits).  out: int64 CUDA tensor of at least 3
    elements.  Returns (status, waited_ms); status is capi.PS_ERR_TIMEOUT when
    the wait ran out as it must."""
    import torch
    if out.dtype != torch.int64 or out.numel() < 3:
        raise ValueError("out must be int64 with at least 3 elements")
    ms = C.c_double()
    st = lib().ps_probe_bounded_wait(1 if first_wait else 0, _p(out), C.byref(ms), _s(stream))
    return st, ms.value
