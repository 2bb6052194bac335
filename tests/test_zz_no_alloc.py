"""gbs_cumulants_noalloc: the click-cumulant entry point for callers that cannot
allocate device memory (inside allocator callbacks, plugins whose host owns all
device allocations, runtimes that forbid allocation after start-up). It keeps its
scratch in a fixed device array inside the library. Called through the C ABI,
its output must match gbs_cumulants (the caller-workspace entry point) within
the forward tests' tolerance, on consecutive calls. Named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu
ABS_TOL = 1e-12


def noalloc_fn():
    gbs.build()
    f = gbs.lib().gbs_cumulants_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def call_noalloc(f, V, M, kmax):
    out = torch.full((gbs.table_size(M, kmax),), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    rc = f(ctypes.c_void_p(V.data_ptr()), M, kmax, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    assert rc == 0, gbs.lib().gbs_last_error().decode()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("M,kmax,seed", [(60, 5, 301), (100, 5, 302)])
def test_noalloc_matches_workspace_entry_on_consecutive_calls(M, kmax, seed):
    f = noalloc_fn()
    inst = synthetic.random_instance(M, kmax, seed=seed, r_range=(0.4, 1.3), eta_range=(0.3, 0.6))
    V = torch.from_numpy(inst.V).cuda()
    ref = gbs.cumulants(V, kmax)
    for _ in range(2):
        got = call_noalloc(f, V, M, kmax)
        assert torch.isfinite(got).all()
        assert (got - ref).abs().max().item() <= ABS_TOL
    # a different input right after: nothing left over from the previous call leaks in
    other = synthetic.random_instance(M, kmax, seed=seed + 1000)
    V2 = torch.from_numpy(other.V).cuda()
    got2 = call_noalloc(f, V2, M, kmax)
    assert (got2 - gbs.cumulants(V2, kmax)).abs().max().item() <= ABS_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = noalloc_fn()
    inst = synthetic.config(2)  # M=144, kmax=5 needs more scratch than the fixed array holds
    V = torch.from_numpy(inst.V).cuda()
    out = torch.empty(8, dtype=torch.float64, device="cuda")  # never written: rejected first
    rc = f(ctypes.c_void_p(V.data_ptr()), 144, 5, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 5
    assert b"allocation-free" in gbs.lib().gbs_last_error()


def test_noalloc_shape_check_matches_the_workspace_entry():
    """kmax <= 3 tables take up to 4096 modes: a valid shape too large for the fixed
    array is a workspace error, as documented, not an argument error."""
    f = noalloc_fn()
    M = 2048
    V = torch.eye(2 * M, dtype=torch.float64, device="cuda")
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    assert f(ctypes.c_void_p(V.data_ptr()), M, 3, ctypes.c_void_p(out.data_ptr()), None) == 5
    assert f(ctypes.c_void_p(V.data_ptr()), M, 4, ctypes.c_void_p(out.data_ptr()), None) == 1


def test_noalloc_status_is_queryable():
    """gbs_noalloc_status reports the device status of the allocation-free calls,
    whose callers hold no workspace to pass to gbs_stream_status."""
    f = noalloc_fn()
    q = gbs.lib().gbs_noalloc_status
    q.argtypes = [ctypes.c_void_p]
    q.restype = ctypes.c_int
    inst = synthetic.random_instance(20, 4, seed=303)
    V = torch.from_numpy(inst.V).cuda()
    call_noalloc(f, V, 20, 4)
    assert q(None) == 0
    bad = V.clone()
    bad[3, 3] = -5.0  # (V_T + I)/2 not positive definite for every T holding mode 3
    out = call_noalloc(f, bad, 20, 4)
    assert q(None) == 2 and torch.isnan(out).any()
    call_noalloc(f, V, 20, 4)
    assert q(None) == 0
