"""Parity of the CUDA forward tables (through the C ABI) with the CPU oracle.

Tolerances (FP64 path): vacuum probabilities relative 1e-12, click moments and
click cumulants absolute 1e-12; the table layout (order groups, colex ranks) is
checked exactly by comparing entry by entry with the oracle's nested-loop
enumeration."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(p0_rel=1e-12, abs=1e-12), "fp32r": dict(p0_rel=1e-11, abs=1e-12)}
FUNCS = {"p0": gbs.vacuum_probs, "mu": gbs.click_moments, "kappa": gbs.cumulants}


@pytest.fixture(scope="module", autouse=True)
def built():
    gbs.build()


def gpu_tables(V, kmax, precision="fp64", which=("p0", "mu", "kappa")):
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    return {w: FUNCS[w](Vd, kmax, precision).cpu().numpy() for w in which}


def assert_tables(got, ref, precision):
    tol = TOL[precision]
    p0g, p0r = got["p0"], ref[0]
    rel = np.abs(p0g - p0r) / np.abs(p0r)
    assert np.all(np.isfinite(p0g))
    assert rel.max() <= tol["p0_rel"], f"P0 max rel err {rel.max():.3e} at {rel.argmax()}"
    for key, r in (("mu", ref[1]), ("kappa", ref[2])):
        err = np.abs(got[key] - r)
        assert err.max() <= tol["abs"], f"{key} max abs err {err.max():.3e} at {err.argmax()}"


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("cfg", [0, 1])
def test_full_tables_match_oracle(cfg, precision):
    inst = synthetic.config(cfg)
    ref = oracle.tables(inst.V, inst.kmax)
    assert_tables(gpu_tables(inst.V, inst.kmax, precision), ref, precision)


@pytest.mark.parametrize("M,kmax,seed", [(5, 5, 1), (6, 5, 2), (9, 5, 3), (37, 5, 4), (41, 4, 5), (12, 2, 6),
                                         (1, 1, 7), (2, 2, 8), (3, 3, 9), (4, 4, 10)])
@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_ragged_sizes_match_oracle(M, kmax, seed, precision):
    inst = synthetic.random_instance(M, kmax, seed=seed, r_range=(0.3, 1.4), eta_range=(0.2, 0.8))
    ref = oracle.tables(inst.V, kmax)
    assert_tables(gpu_tables(inst.V, kmax, precision), ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_config3_full_tables(precision):
    inst = synthetic.config(3)
    ref = oracle.tables(inst.V, inst.kmax)
    assert_tables(gpu_tables(inst.V, inst.kmax, precision), ref, precision)


def test_vacuum_input_gives_trivial_tables():
    V = np.eye(2 * 7)
    got = gpu_tables(V, 5)
    assert np.all(got["p0"] == 1.0)
    assert np.abs(got["mu"]).max() == 0.0
    assert np.abs(got["kappa"]).max() < 1e-15


def test_product_state_cumulants_vanish():
    # block-diagonal across modes: independent single-mode states
    M = 9
    rng = np.random.default_rng(3)
    V = np.zeros((2 * M, 2 * M))
    for k in range(M):
        r, ph, eta = rng.uniform(0.2, 1.2), rng.uniform(0, 3), rng.uniform(0.3, 0.9)
        c, s = np.cos(ph), np.sin(ph)
        R = np.array([[c, -s], [s, c]])
        b = eta * R @ np.diag([np.exp(-2 * r), np.exp(2 * r)]) @ R.T + (1 - eta) * np.eye(2)
        V[np.ix_([k, k + M], [k, k + M])] = b
    got = gpu_tables(V, 5, which=("kappa",))["kappa"]
    assert np.abs(got[M:]).max() < 1e-14


def test_not_positive_definite_is_reported():
    inst = synthetic.random_instance(8, 3, seed=5)
    V = inst.V.copy()
    V[3, 3] = -5.0  # (V_T + I)/2 loses positive definiteness for T containing mode 3
    Vd = torch.from_numpy(V).cuda()
    with pytest.raises(gbs.GbsError) as ei:
        gbs.vacuum_probs(Vd, 3)
    assert ei.value.code == 2
    out = gbs.vacuum_probs(Vd, 3, check=False)
    torch.cuda.synchronize()
    assert torch.isnan(out[3]).item()


def test_invalid_arguments_rejected_on_host():
    Vd = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError):
        gbs.cumulants(Vd, 6)
    with pytest.raises(gbs.GbsError) as ei:
        gbs.cumulants(Vd, 3, workspace=gbs.Workspace(2, 1))
    assert ei.value.code == 5
    # a host pointer is rejected rather than dereferenced
    import ctypes
    host = (ctypes.c_double * 64)()
    ws = gbs.Workspace(4, 2)
    out = torch.empty(gbs.table_size(4, 2), dtype=torch.float64, device="cuda")
    rc = gbs.lib().gbs_vacuum_probs(ctypes.cast(host, ctypes.c_void_p), 4, 2, ctypes.c_void_p(out.data_ptr()), 0,
                                    ctypes.c_void_p(ws.ptr), ws.nbytes, None)
    assert rc == 1


def test_workspace_reuse_and_stream_order():
    inst = synthetic.random_instance(30, 5, seed=9)
    Vd = torch.from_numpy(inst.V).cuda()
    ws = gbs.Workspace(30, 5)
    a = gbs.cumulants(Vd, 5, workspace=ws)
    b = gbs.cumulants(Vd, 5, workspace=ws)
    assert torch.equal(a, b)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = gbs.cumulants(Vd, 5, workspace=ws)
    s.synchronize()
    assert torch.equal(a, c)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_full_size_m144_k5_sampled(precision):
    """The M=144, kmax=5 workload in the configuration the benchmark times: all
    entries of orders <= 3 against the oracle tables, and a seeded sample of
    orders 4 and 5 against entries the oracle computes one by one."""
    inst = synthetic.config(2)
    M, kmax = inst.M, inst.kmax
    got = gpu_tables(inst.V, kmax, precision)
    ref3 = oracle.tables(inst.V, 3)
    n3 = oracle.table_size(M, 3)
    tol = TOL[precision]
    assert np.abs(got["p0"][:n3] / ref3[0] - 1).max() <= tol["p0_rel"]
    assert np.abs(got["mu"][:n3] - ref3[1]).max() <= tol["abs"]
    assert np.abs(got["kappa"][:n3] - ref3[2]).max() <= tol["abs"]
    for d, n in ((4, 20000), (5, 20000)):
        sets = synthetic.random_subsets(M, d, n, seed=100 + d)
        idx = np.array([gbs.order_offset(M, d) + gbs.rank(S) for S in sets])
        e = oracle.entries(inst.V, sets)
        assert np.abs(got["p0"][idx] / e["p0"] - 1).max() <= tol["p0_rel"]
        assert np.abs(got["mu"][idx] - e["mu"]).max() <= tol["abs"]
        assert np.abs(got["kappa"][idx] - e["kappa"]).max() <= tol["abs"]
    # properties that hold at any size: 0 < P0 <= 1, 0 <= mu <= 1
    assert got["p0"].min() > 0 and got["p0"].max() <= 1.0
    assert got["mu"].min() >= -1e-12 and got["mu"].max() <= 1.0


def test_refined_path_differs_from_fp64_only_by_rounding():
    """The refined path is a different computation (FP32 factorisation plus
    refinement), not a relabelled FP64 run: its order-4/5 entries differ from the
    FP64 path in the last bits, and stay within the refined tolerance."""
    inst = synthetic.random_instance(40, 5, seed=77, r_range=(0.8, 1.6), eta_range=(0.3, 0.5))
    a = gpu_tables(inst.V, 5, "fp64", which=("p0",))["p0"]
    b = gpu_tables(inst.V, 5, "fp32r", which=("p0",))["p0"]
    n3 = gbs.table_size(40, 3)
    assert np.any(a[n3:] != b[n3:])
    assert np.abs(b / a - 1).max() <= 1e-11


def test_injected_runtime_failure_is_reported(monkeypatch):
    """A runtime-call failure inside the library (injected on the host) comes
    back as GBS_ERR_CUDA with a message; the next call succeeds."""
    inst = synthetic.config(0)
    V = torch.from_numpy(inst.V).cuda()
    monkeypatch.setenv("GBS_FAULT_INJECT", "forward_memset")
    with pytest.raises(gbs.GbsError) as err:
        gbs.cumulants(V, inst.kmax)
    assert err.value.code == 3 and "injected" in str(err.value)
    monkeypatch.delenv("GBS_FAULT_INJECT")
    kt = gbs.cumulants(V, inst.kmax).cpu().numpy()
    assert np.abs(kt - oracle.tables(inst.V, inst.kmax)[2]).max() <= 1e-12
