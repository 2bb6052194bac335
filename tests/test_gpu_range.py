"""Sharded tables: slices of the top order over consecutive top-element ranges,
concatenated, equal the whole table's top-order group bit for bit (the same
arithmetic runs on the same entries), for every table kind, both precisions,
the prefix-tree orders (4, 5) and the flat ones (1-3); the lower orders the
slices need are computed inside the workspace."""
import pytest
import torch

import synthetic
import paper_2511_14923_gb300 as gbs

pytestmark = pytest.mark.gpu
WHOLE = {"p0": gbs.vacuum_probs, "mu": gbs.click_moments, "kappa": gbs.cumulants,
         "spin_c": gbs.spin_correlators, "spin_kappa": gbs.spin_cumulants}


@pytest.fixture(scope="module", autouse=True)
def built():
    gbs.build()


def check_shards(M, kmax, table, precision, parts, seed):
    inst = synthetic.random_instance(M, kmax, seed=seed, r_range=(0.4, 1.3), eta_range=(0.3, 0.6))
    V = torch.from_numpy(inst.V).cuda()
    whole = WHOLE[table](V, kmax, precision)
    top = whole[gbs.order_offset(M, kmax):]
    bounds = gbs.range_split(M, kmax, parts)
    assert bounds[0] == 0 and bounds[-1] == M and all(a <= b for a, b in zip(bounds, bounds[1:]))
    pieces = [gbs.table_range(V, kmax, lo, hi, table, precision).clone() for lo, hi in zip(bounds, bounds[1:])]
    got = torch.cat(pieces)
    assert got.numel() == top.numel()
    assert torch.equal(got, top), (table, precision, (got - top).abs().max().item())


@pytest.mark.parametrize("precision", ["fp32r", "fp64"])
def test_order5_cumulant_shards_equal_whole_table(precision):
    check_shards(60, 5, "kappa", precision, 4, 61)


@pytest.mark.parametrize("table", ["p0", "mu", "spin_c", "spin_kappa"])
def test_order4_shards_every_table(table):
    check_shards(40, 4, table, "fp64", 3, 62)


@pytest.mark.parametrize("M,kmax,parts", [(200, 3, 5), (90, 2, 4), (30, 1, 3), (12, 5, 7)])
def test_flat_orders_and_tiny_tables(M, kmax, parts):
    check_shards(M, kmax, "kappa", "fp32r", parts, 63)


def test_single_range_equals_slice_and_bad_ranges_rejected():
    inst = synthetic.random_instance(50, 5, seed=64)
    V = torch.from_numpy(inst.V).cuda()
    whole = gbs.cumulants(V, 5, "fp32r")
    lo, hi = 37, 41
    got = gbs.table_range(V, 5, lo, hi, "kappa", "fp32r")
    off = gbs.order_offset(50, 5)
    from math import comb
    assert torch.equal(got, whole[off + comb(lo, 5): off + comb(hi, 5)])
    assert gbs.table_range(V, 5, 20, 20, "kappa").numel() == 0
    with pytest.raises(ValueError):
        gbs.table_range(V, 5, 30, 20)
    with pytest.raises(gbs.GbsError):
        gbs.range_split(50, 5, 0)
