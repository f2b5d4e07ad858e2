"""Fixtures under tests/golden/.

* paper_constants.json: the constants the paper prints (Eqs. 3 and 4, C8 = C6 R0^2,
  R_pot and R_cn).  The default parameters use them, and a two-atom open
  structure with one-reference tables gives the Eq. 2 energy with
  C8 = C6 R0^2 (R0^2 = 3 sqrtQ_i sqrtQ_j, the reading of the geometric mean).
* oracle_bilayer_ab_64.json: written by tests/golden/make_golden.py from the
  oracle alone; the oracle must keep reproducing it.
"""
import json
import os

import numpy as np

from paper_2310_05279_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BOHR = 0.529177210903
HARTREE = 27.211386245988


def test_paper_constants(oracle_mod):
    c = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert wl.PBE_BJ["k1"] == c["k1"]["value"]
    assert wl.PBE_BJ["k3"] == c["k3"]["value"]
    assert wl.PBE_BJ["rc_disp"] == c["r_pot_A"]["value"]
    assert wl.PBE_BJ["rc_cn"] == c["r_cn_A"]["value"]
    # Eq. 2 for one pair at r = 7 A (beyond R_cn: no CN dependence either way)
    tabs = wl.random_tables(["C", "O"], 1021, nref_max=1)
    r = 7.0
    res = oracle_mod.compute(np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]]), [0, 1], np.eye(3) * 40.0,
                             [0, 0, 0], tabs, wl.PBE_BJ)
    p = wl.PBE_BJ
    c6 = tabs.c6_ref[0, 1, 0, 0]
    r0sq = 3.0 * tabs.sqrtq[0] * tabs.sqrtq[1]
    c8 = c["c8_over_c6_r0sq"]["value"] * c6 * r0sq
    R = p["a1"] * np.sqrt(r0sq) + p["a2"]
    rb = r / BOHR
    e = -(p["s6"] * c6 / (rb ** 6 + R ** 6) + p["s8"] * c8 / (rb ** 8 + R ** 8)) * HARTREE
    assert abs(res["E"] - e) <= 1e-13 * abs(e)


def test_oracle_regression(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "oracle_bilayer_ab_64.json")))
    b = wl.bilayer_ab_64()
    for name in ("two_body", "with_three_body"):
        ref = g[name]
        r = oracle_mod.compute(*b.structure(0), b.tables, ref["params"])
        assert abs(r["E"] - ref["E_eV"]) <= 1e-12 * abs(ref["E_eV"])
        np.testing.assert_allclose(r["F"], np.array(ref["F_eV_A"]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(r["W"], np.array(ref["W_eV"]), rtol=0, atol=1e-12 * np.abs(ref["W_eV"]).max())
        np.testing.assert_allclose(r["cn"], np.array(ref["cn"]), rtol=1e-13)
        np.testing.assert_allclose(r["e_atom"], np.array(ref["e_atom_eV"]), rtol=1e-12)
