"""Reference-table and damping-parameter files (host-side IO, no GPU)."""
import json

import numpy as np
import pytest

from paper_2310_05279_gb300 import tables as tio
from paper_2310_05279_gb300 import workloads as wl


def _same(a, b):
    assert a.names == b.names
    np.testing.assert_array_equal(a.nref, b.nref)
    np.testing.assert_array_equal(a.cn_ref, b.cn_ref)
    np.testing.assert_array_equal(a.c6_ref, b.c6_ref)
    np.testing.assert_array_equal(a.sqrtq, b.sqrtq)
    np.testing.assert_array_equal(a.rcov, b.rcov)


@pytest.mark.parametrize("ext", [".json", ".npz"])
def test_round_trip(tmp_path, ext):
    t = wl.random_tables(["H", "C", "N", "O", "Zn"], 41)
    p = str(tmp_path / ("t" + ext))
    tio.save_tables(t, p)
    _same(tio.load_tables(p), t)


def test_subset_and_order(tmp_path):
    t = wl.random_tables(["H", "C", "N", "O"], 42)
    p = str(tmp_path / "t.json")
    tio.save_tables(t, p)
    s = tio.load_tables(p, ["O", "H"])
    assert s.names == ["O", "H"]
    i, j = t.names.index("O"), t.names.index("H")
    R = s.max_ref
    np.testing.assert_array_equal(s.c6_ref[0, 1], t.c6_ref[i, j, :R, :R])
    np.testing.assert_array_equal(s.cn_ref[1, :t.nref[j]], t.cn_ref[j, :t.nref[j]])


def test_loaded_tables_give_the_same_oracle_result(tmp_path, oracle_mod):
    b = wl.uneven_batch(seed=5, nstruct=1, n_range=(30, 31))
    p = str(tmp_path / "t.json")
    tio.save_tables(b.tables, p)
    t2 = tio.load_tables(p)
    pos, typ, cell, pbc = b.structure(0)
    r1 = oracle_mod.compute(pos, typ, cell, pbc, b.tables, wl.PBE_BJ)
    r2 = oracle_mod.compute(pos, typ, cell, pbc, t2, wl.PBE_BJ)
    assert r1["E"] == r2["E"] and np.array_equal(r1["F"], r2["F"])


def test_records_errors():
    refs = {"C": [0.0, 2.0], "H": [0.0]}
    good = [["C", 0, "C", 0, 40.0], ["C", 0, "C", 1, 30.0], ["C", 1, "C", 1, 25.0],
            ["C", 0, "H", 0, 10.0], ["C", 1, "H", 0, 9.0], ["H", 0, "H", 0, 3.0]]
    t = tio.tables_from_records(["C", "H"], refs, good, [1.4, 0.6], [3.0, 1.5])
    assert t.c6_ref[0, 0, 1, 0] == 30.0 and t.c6_ref[1, 0, 0, 1] == 9.0
    with pytest.raises(ValueError, match="missing"):
        tio.tables_from_records(["C", "H"], refs, good[:-1], [1.4, 0.6], [3.0, 1.5])
    with pytest.raises(ValueError, match="contradictory"):
        tio.tables_from_records(["C", "H"], refs, good + [["H", 0, "C", 1, 9.5]], [1.4, 0.6], [3.0, 1.5])
    with pytest.raises(ValueError, match="out of range"):
        tio.tables_from_records(["C", "H"], refs, good + [["H", 1, "C", 0, 1.0]], [1.4, 0.6], [3.0, 1.5])
    with pytest.raises(ValueError, match="positive"):
        tio.tables_from_records(["C", "H"], refs, good + [["H", 0, "H", 0, -3.0]], [1.4, 0.6], [3.0, 1.5])


def test_damping_file(tmp_path):
    p = tmp_path / "damp.json"
    p.write_text(json.dumps({"format": "d3gb-damping-1",
                             "functionals": {"PBE": {"s6": 1.0, "s8": 0.7875, "a1": 0.4289, "a2_bohr": 4.4407}}}))
    d = tio.load_damping(str(p), "pbe")
    assert d == dict(s6=1.0, s8=0.7875, a1=0.4289, a2=4.4407)
    with pytest.raises(KeyError):
        tio.load_damping(str(p), "b3lyp")
    q = tmp_path / "bad.json"
    q.write_text(json.dumps({"format": "something-else"}))
    with pytest.raises(ValueError):
        tio.load_damping(str(q), "pbe")


def test_dftd3_input_line(tmp_path):
    """The paper's three inputs (functional, R_pot, R_cn) as an input line or a tuple."""
    p = str(tmp_path / "d.json")
    json.dump({"format": tio.DAMPING_FORMAT, "functionals": {
        "PBE": {"s6": 1.0, "s8": 0.7875, "a1": 0.4289, "a2_bohr": 4.4407},
        "other": {"s6": 1.0, "s8": 0.9, "a1": 0.5, "a2_bohr": 4.0}}}, open(p, "w"))
    a = tio.dftd3_params("dftd3 pbe 12 6", p)
    assert a == dict(s6=1.0, s8=0.7875, a1=0.4289, a2=4.4407, k1=16.0, k2=4.0 / 3.0, k3=4.0, rc_disp=12.0, rc_cn=6.0)
    b = tio.dftd3_params(("OTHER", 20, 10.5), p)
    assert (b["s8"], b["a1"], b["a2"], b["rc_disp"], b["rc_cn"]) == (0.9, 0.5, 4.0, 20.0, 10.5)
    with pytest.raises(ValueError):
        tio.dftd3_params("dftd3 pbe 12", p)
    with pytest.raises(ValueError):
        tio.dftd3_params("dftd3 pbe -1 6", p)
    with pytest.raises(KeyError):
        tio.dftd3_params("dftd3 b3lyp 12 6", p)

