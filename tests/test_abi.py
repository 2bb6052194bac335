"""The C ABI library loads and exports every entry point include/gbs.h declares;
host-only helpers (sizes, offsets, colex rank/unrank, argument checks) agree with
the oracle's enumeration. No kernel is launched. CPU only."""
import ctypes
import os
import re
from math import comb

import numpy as np
import pytest

import oracle
import paper_2511_14923_gb300 as gbs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    gbs.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbs_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "gbs_cumulants" in names and "gbs_rank" in names
    L = gbs.lib()
    for n in names:
        assert hasattr(L, n), n


def test_table_size_and_offsets():
    for M in (1, 2, 5, 8, 50, 144, 1024):
        for k in range(1, min(M, 5) + 1):
            assert gbs.table_size(M, k) == sum(comb(M, d) for d in range(1, k + 1))
            assert gbs.order_offset(M, k) == sum(comb(M, d) for d in range(1, k))
    assert gbs.table_size(144, 5) == 498685188
    assert gbs.table_size(0, 1) == 0 and gbs.table_size(4, 5) == 0 and gbs.table_size(10, 6) == 0
    assert gbs.table_size(4097, 1) == 0 and gbs.table_size(1025, 4) == 0


@pytest.mark.parametrize("M", [1, 6, 11, 20])
def test_rank_unrank_match_oracle_enumeration(M):
    for d in range(1, min(M, 5) + 1):
        for i, S in enumerate(oracle.enumerate_subsets(M, d)):
            assert gbs.rank(S) == i
            assert gbs.unrank(i, d) == list(S)


def test_rank_large_modes_bit_exact():
    rng = np.random.default_rng(0)
    for _ in range(200):
        d = int(rng.integers(1, 6))
        S = np.sort(rng.choice(1024, d, replace=False))
        r = gbs.rank(S)
        assert r == sum(comb(int(c), i + 1) for i, c in enumerate(S))
        assert gbs.unrank(r, d) == list(S)


def test_rank_rejects_bad_input():
    assert gbs.rank([3, 3]) == 2**64 - 1
    assert gbs.rank([4, 2]) == 2**64 - 1
    assert gbs.rank([-1]) == 2**64 - 1
    with pytest.raises(gbs.GbsError):
        gbs.unrank(comb(4096, 2), 2)


def test_workspace_bytes_rejects_invalid():
    assert gbs.workspace_bytes(8, 3) > 0
    assert gbs.lib().gbs_workspace_bytes(8, 9, 0) == 0
    assert gbs.lib().gbs_workspace_bytes(8, 3, 7) == 0


def test_sampler_workspace_bytes_limits():
    """Host-side shape checks of gbs_sample: K in 3..5, M >= K, batch a multiple of
    128 up to GBS_MAX_SAMPLE_BATCH (2^21), a known precision."""
    q = gbs.sampler_workspace_bytes
    assert q(144, 5, 8192) > 0 and q(144, 5, 8192, "fp64") > 0
    assert q(8, 5, 1 << 21) > 0 and q(8, 5, (1 << 21) + 128) == 0
    assert q(8, 5, 64) == 0 and q(8, 5, 200) == 0 and q(4, 5, 128) == 0 and q(8, 6, 128) == 0
    assert gbs.lib().gbs_sampler_workspace_bytes(8, 5, 128, 7) == 0


def test_compute_entry_rejects_bad_arguments_without_launching():
    L = gbs.lib()
    vp = ctypes.c_void_p
    # NULL pointers and bad sizes are caught on the host before any CUDA work
    assert L.gbs_cumulants(vp(0), 8, 3, vp(0), 0, vp(0), 0, vp(0)) == 1
    assert L.gbs_cumulants(vp(0), 8, 9, vp(0), 0, vp(0), 0, vp(0)) == 1
    assert L.gbs_vacuum_probs(vp(0), 8, 3, vp(0), 5, vp(0), 0, vp(0)) == 1
    assert b"kmax" in L.gbs_last_error() or b"precision" in L.gbs_last_error()
    # the schedule query checks its arguments before it looks for a device
    arr = (ctypes.c_int * 3)()
    assert L.gbs_schedule(144, 5, 1, None) == 1
    assert L.gbs_schedule(144, 6, 1, arr) == 1
    assert L.gbs_schedule(144, 5, 7, arr) == 1


def test_large_mode_counts_for_low_orders():
    """kmax <= 3 (and the K = 3 sampler) accept up to 4096 modes; kmax >= 4 stays
    at 1024. Ranks of mode sets up to 4095 are exact."""
    assert gbs.table_size(4096, 3) == comb(4096, 1) + comb(4096, 2) + comb(4096, 3)
    assert gbs.table_size(1152, 3) == 1152 + comb(1152, 2) + comb(1152, 3)
    assert gbs.table_size(4097, 3) == 0 and gbs.table_size(1025, 4) == 0 and gbs.table_size(1024, 4) > 0
    assert gbs.order_offset(4096, 3) == 4096 + comb(4096, 2)
    rng = np.random.default_rng(4)
    for _ in range(300):
        d = int(rng.integers(1, 6))
        S = np.sort(rng.choice(4096, d, replace=False))
        r = gbs.rank(S)
        assert r == sum(comb(int(c), i + 1) for i, c in enumerate(S))
        assert gbs.unrank(r, d) == [int(c) for c in S]
    assert gbs.rank([4096]) == 2 ** 64 - 1
    assert gbs.lib().gbs_backward_workspace_bytes(1152, 3) == 0


def test_python_workspace_checks_run_before_any_library_call():
    """The binding rejects host-memory workspaces, foreign objects and undersized
    workspaces on the host (GBS_ERR_WORKSPACE = 5 for the size, as the library
    would), so no host pointer ever reaches a kernel."""
    import torch
    cuda0 = torch.device("cuda", 0)
    with pytest.raises(TypeError):
        gbs.Workspace(8, 3, device="cpu")
    with pytest.raises(TypeError):
        gbs._workspace_tensor(torch.empty(64, dtype=torch.uint8), 64, cuda0)
    with pytest.raises(TypeError):
        gbs._workspace_for(torch.empty(64, dtype=torch.uint8), 8, 3, "fp64", cuda0)
    # a Workspace whose buffer is on another device than the inputs
    ws = object.__new__(gbs.Workspace)
    ws.buf, ws.nbytes = torch.empty(16, dtype=torch.uint8, device="meta"), 16
    with pytest.raises(ValueError):
        gbs._workspace_for(ws, 8, 3, "fp64", cuda0)
    # same device, too small
    with pytest.raises(gbs.GbsError) as ei:
        gbs._workspace_for(ws, 8, 3, "fp64", torch.device("meta"))
    assert ei.value.code == 5
    ws.nbytes = gbs.workspace_bytes(8, 3, "fp64")
    assert gbs._workspace_for(ws, 8, 3, "fp64", torch.device("meta")) is ws
    assert gbs._nbytes(torch.empty(3, dtype=torch.float64)) == 24
    # inputs on different devices are refused
    t = torch.empty(4)
    assert gbs._on(t, torch.device("cpu"), "t") is t
    with pytest.raises(ValueError):
        gbs._on(t, torch.device("meta"), "t")


def test_status_code_maps_status_words():
    """gbs_status_code interprets a status word copied to the host without a
    synchronisation (the deferred checks of the autograd Functions): the bits
    not-positive-definite (1), bounded-wait timeout (2) and device index check
    (4), timeout first."""
    f = gbs.lib().gbs_status_code
    assert f(0) == 0 and gbs.lib().gbs_last_error() == b""
    assert f(1) == 2 and b"positive definite" in gbs.lib().gbs_last_error()
    assert f(2) == 4 and f(3) == 4 and f(7) == 4
    assert f(4) == 1 and f(5) == 2
