"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

config0_tables.txt: P0, mu and click-cumulant tables (columns) for the M=8,
kmax=3 workload (4 squeezers r~U[0.3,0.8], Haar U, eta=0.5; 92 subsets in
order-then-colex order). The paper prints no numeric worked example; these
values anchor the oracle against regressions and are pinned by the closed-form
and Torontonian tests.

Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synthetic  # noqa: E402


def main():
    inst = synthetic.config(0)
    p0, mu, kt = oracle.tables(inst.V, inst.kmax)
    np.savetxt(os.path.join(HERE, "config0_tables.txt"), np.stack([p0, mu, kt], axis=1),
               fmt="%.17e", header="P0 mu kappa  (M=8, kmax=3, order then colex rank)")


if __name__ == "__main__":
    main()
