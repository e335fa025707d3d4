"""GPU test of srj_steps_f32_noalloc, the allocation-free FP32 sweep entry point.

Callers that cannot allocate device memory (a fixed memory pool that forbids
foreign cudaMalloc, latency-critical loops where an allocation would synchronise
the device) use this entry point; its work buffers live in a static device
array instead of a plan's workspaces.  It must give exactly what srj_steps gives
on a mixed-precision plan with the same weights, on consecutive calls (the
static array keeps the previous call's contents, so stale data must not leak
into the next call), in 2-D and 3-D and up to the array's size limit.

This file is collected last so that a failure here does not hide the other GPU
tests when pytest stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import srj_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1511_04292_gb300 as srj  # noqa: E402


def _noalloc(dims, h, seq, f, u):
    L = srj.lib()
    d = (ctypes.c_int64 * len(dims))(*dims)
    s = np.ascontiguousarray(seq, dtype=np.float64)
    rc = L.srj_steps_f32_noalloc(len(dims), d, h, len(s), s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.srj_noalloc_last_error()


@pytest.mark.parametrize("dims,n,P", [((128, 128), 128, 5), ((64, 64), 64, 6), ((40, 40, 40), 128, 5),
                                      ((1016, 1016), 1024, 6)])
def test_noalloc_matches_plan_steps_on_two_calls(dims, n, P):
    """Bit-identical to srj_steps on a mixed plan with the same weight order, on
    two calls in a row.  (40, 40, 40) runs the 3-D branch (its pitched layout
    includes the nz + 2 planes); 1016^2 needs 1,042,432 floats per buffer, just
    under the 2^20 limit, and must be accepted.  The weights of the smaller
    grids' table row are used where the grid has no row of its own."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    row = srj.schedules.lookup(2, n, P)
    seq = row["omega"][row["order"]]
    h = 1.0 / (max(dims) + 1)
    plan = srj.Plan(dims, h, row["omega"], row["q"], row["order"], "mixed")
    for call, (seed, count) in enumerate([(11, len(seq)), (12, 7)]):
        f = torch.from_numpy(W.random_field(dims, seed)).cuda()
        u0 = torch.from_numpy(W.random_field(dims, seed + 100)).cuda()
        ref = u0.clone()
        plan.steps(f, ref, 0, count)
        got = u0.clone()
        _noalloc(dims, h, seq[:count], f, got)
        assert torch.isfinite(ref).all()
        # same kernels, same weights: bit-identical (within any FP32 tolerance)
        assert torch.equal(got, ref), ("call", call)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims = (1100, 1100)
    f = torch.zeros((1102, 1102), dtype=torch.float64, device="cuda")
    L = srj.lib()
    d = (ctypes.c_int64 * 2)(*dims)
    s = np.ones(1)
    rc = L.srj_steps_f32_noalloc(2, d, 0.001, 1, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), None)
    assert rc == -1 and b"static scratch" in L.srj_noalloc_last_error()
