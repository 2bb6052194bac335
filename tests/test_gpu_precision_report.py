"""Per-table error of both precisions against the CPU oracle, printed for the
record (run with -s), and asserted against the stated bounds. Workloads: the
M=50 kmax=4 table in full, and the M=144 kmax=5 table on all entries of orders
<= 3 plus a seeded sample of 10^7 ranks of each of orders 4 and 5."""
import json

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu
BOUNDS = {"fp64": (1e-12, 1e-12), "fp32r": (1e-11, 1e-12)}


def colex_ranks(sets):
    """Colex ranks sum_i C(S[:, i], i + 1) of sorted rows, vectorised (exact in int64)."""
    r = np.zeros(len(sets), dtype=np.int64)
    for i in range(sets.shape[1]):
        c = sets[:, i].astype(np.int64)
        num = np.ones_like(c)
        for j in range(i + 1):
            num = num * (c - j)
        den = 1
        for j in range(1, i + 2):
            den *= j
        r += np.where(c > i, num // den, 0)
    return r


def errors(got, ref_p0, ref_mu, ref_kt, idx=None):
    sel = (lambda x: x) if idx is None else (lambda x: x[idx])
    return {"p0_max_rel": float(np.max(np.abs(sel(got["p0"]) / ref_p0 - 1))),
            "mu_max_abs": float(np.max(np.abs(sel(got["mu"]) - ref_mu))),
            "kappa_max_abs": float(np.max(np.abs(sel(got["kappa"]) - ref_kt)))}


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_report_errors(precision):
    gbs.build()
    report = {"precision": precision}
    fns = {"p0": gbs.vacuum_probs, "mu": gbs.click_moments, "kappa": gbs.cumulants}
    inst = synthetic.config(1)
    Vd = torch.from_numpy(inst.V).cuda()
    got = {k: f(Vd, inst.kmax, precision).cpu().numpy() for k, f in fns.items()}
    report["M50_k4_full"] = errors(got, *oracle.tables(inst.V, inst.kmax))
    inst = synthetic.config(2)
    Vd = torch.from_numpy(inst.V).cuda()
    got = {k: f(Vd, inst.kmax, precision).cpu().numpy() for k, f in fns.items()}
    n3 = oracle.table_size(144, 3)
    report["M144_orders1-3_full"] = errors({k: v[:n3] for k, v in got.items()}, *oracle.tables(inst.V, 3))
    for d in (4, 5):
        sets = synthetic.random_subsets(144, d, 10_000_000, seed=900 + d)
        r = colex_ranks(sets)
        assert all(r[i] == gbs.rank(sets[i]) for i in range(0, len(sets), 999_983))
        idx = gbs.order_offset(144, d) + r
        e = oracle.entries(inst.V, sets)
        report[f"M144_order{d}_sample"] = errors(got, e["p0"], e["mu"], e["kappa"], idx)
    print("PRECISION_REPORT " + json.dumps(report))
    rel, ab = BOUNDS[precision]
    for key, v in report.items():
        if key == "precision":
            continue
        assert v["p0_max_rel"] <= rel and v["mu_max_abs"] <= ab and v["kappa_max_abs"] <= ab, (key, v)
