"""Parity at the full workload sizes, in the launch configuration the bench uses.

* 128 x 1440 bilayer scan: every structure against the FP64 oracle, both forms.
* 1,048,576-atom MOF-like box: the oracle cannot evaluate the whole box, so
  forces and site energies of sampled atoms are checked against the oracle on
  open clusters cut around them (radius R_pot + 2 R_cn: the force on an atom
  depends on nothing farther, pinned in test_oracle_invariants), and E and W of
  the mixed form against the FP64 form (itself oracle-exact at smaller sizes).
* 512-structure uneven batch: sampled structures of every size class against
  the oracle; all structures mixed against FP64.
* the scan with the optional three-body term: every structure mixed against
  FP64, 16 structures against the oracle.
"""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import (TOL_E_PER_ATOM, TOL_F_MAX, TOL_W_REL, assert_fp64_ok, assert_mixed_ok, cluster_around,
                       to_dev)

pytestmark = pytest.mark.gpu
PRM = dict(wl.PBE_BJ)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run(b, precision, **kw):
    from paper_2310_05279_gb300 import D3
    d3 = D3(b.tables, precision=precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, **kw)
    d3.sync_status()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    del d3
    return res


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bilayer_scan_full(torch_cuda, oracle_mod, precision):
    b = wl.bilayer_scan()
    out = run(b, precision)
    ref = oracle_mod.compute_batch(b, PRM)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(
        {k: torch_cuda.tensor(v) for k, v in out.items()}, ref, b.offsets)
    # binding curve shape: at fixed slide, E rises (less negative) with distance beyond 4 A
    E = out["E"].reshape(16, 8)
    d = np.linspace(2.8, 8.0, 16)
    assert np.all(np.diff(E[d >= 4.0], axis=0) > 0)


def test_mof_like_box_full(torch_cuda, oracle_mod):
    b = wl.mof_like_box()
    mixed = run(b, "mixed", e_atom=True)
    fp64 = run(b, "fp64")
    n = b.natoms
    assert abs(mixed["E"][0] - fp64["E"][0]) / n <= TOL_E_PER_ATOM
    assert np.linalg.norm(mixed["W"] - fp64["W"]) / np.linalg.norm(fp64["W"]) <= TOL_W_REL
    assert np.abs(mixed["F"] - fp64["F"]).max() <= TOL_F_MAX
    assert abs(mixed["e_atom"].sum() - mixed["E"][0]) <= 1e-9 * abs(mixed["E"][0])
    pos, types, cell, pbc = b.structure(0)
    g = np.random.Generator(np.random.PCG64(8))
    for i in g.choice(n, 6, replace=False):
        cp, ct = cluster_around(pos, types, cell, int(i), 24.0 + 1e-6)
        r = oracle_mod.compute(cp, ct, np.eye(3) * 400.0, [0, 0, 0], b.tables, PRM)
        assert np.abs(r["F"][0] - mixed["F"][i]).max() <= TOL_F_MAX
        assert abs(r["e_atom"][0] - mixed["e_atom"][i]) <= 5e-7  # one site energy: no averaging over atoms


def test_uneven_batch_full(torch_cuda, oracle_mod):
    b = wl.uneven_batch()
    mixed = run(b, "mixed")
    fp64 = run(b, "fp64")
    sizes = np.diff(b.offsets)
    de = np.abs(mixed["E"] - fp64["E"]) / np.maximum(sizes, 1)
    assert de.max() <= TOL_E_PER_ATOM
    assert np.abs(mixed["F"] - fp64["F"]).max() <= TOL_F_MAX
    wn = np.linalg.norm(fp64["W"].reshape(-1, 9), axis=1)
    assert (np.linalg.norm((mixed["W"] - fp64["W"]).reshape(-1, 9), axis=1) / wn).max() <= TOL_W_REL
    order = np.argsort(sizes)
    sample = [int(order[k]) for k in np.linspace(0, len(order) - 1, 10).astype(int)]
    sub = b.subset(sample)
    ref = oracle_mod.compute_batch(sub, PRM)
    F = np.concatenate([mixed["F"][b.offsets[s]:b.offsets[s + 1]] for s in sample])
    F64 = np.concatenate([fp64["F"][b.offsets[s]:b.offsets[s + 1]] for s in sample])
    assert_mixed_ok({"E": torch_cuda.tensor(mixed["E"][sample]), "F": torch_cuda.tensor(F),
                     "W": torch_cuda.tensor(mixed["W"][sample])}, ref, sub.offsets)
    assert_fp64_ok({"E": torch_cuda.tensor(fp64["E"][sample]), "F": torch_cuda.tensor(F64),
                    "W": torch_cuda.tensor(fp64["W"][sample])}, ref, sub.offsets)


def test_bilayer_scan_full_three_body(torch_cuda, oracle_mod):
    """The bench's three-body leg (mixed, s9 = 1, alpha = 16, rc3 = 6 A) on the full
    128 x 1440 scan, in one batched call as timed; 16 structures spread over the
    distance / slide grid against the oracle, all against the FP64 form."""
    p = dict(PRM, s9=1.0, alpha9=16.0, rc3=6.0)
    b = wl.bilayer_scan()
    from paper_2310_05279_gb300 import D3
    pos, typ = to_dev(b)
    out = {}
    for prec in ("mixed", "fp64"):
        d3 = D3(b.tables, p, precision=prec)
        r = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
        d3.sync_status()
        out[prec] = {k: v.cpu().numpy() for k, v in r.items()}
        del d3
    m, f = out["mixed"], out["fp64"]
    n = np.diff(b.offsets)
    assert (np.abs(m["E"] - f["E"]) / n).max() <= TOL_E_PER_ATOM
    assert np.abs(m["F"] - f["F"]).max() <= TOL_F_MAX
    wn = np.linalg.norm(f["W"].reshape(-1, 9), axis=1)
    assert (np.linalg.norm((m["W"] - f["W"]).reshape(-1, 9), axis=1) / wn).max() <= TOL_W_REL
    sample = list(range(0, 128, 8))
    sub = b.subset(sample)
    ref = oracle_mod.compute_batch(sub, p)
    F = np.concatenate([m["F"][b.offsets[s]:b.offsets[s + 1]] for s in sample])
    F64 = np.concatenate([f["F"][b.offsets[s]:b.offsets[s + 1]] for s in sample])
    assert_mixed_ok({"E": torch_cuda.tensor(m["E"][sample]), "F": torch_cuda.tensor(F),
                     "W": torch_cuda.tensor(m["W"][sample])}, ref, sub.offsets)
    assert_fp64_ok({"E": torch_cuda.tensor(f["E"][sample]), "F": torch_cuda.tensor(F64),
                    "W": torch_cuda.tensor(f["W"][sample])}, ref, sub.offsets)
    # the three-body term raises the energy of every sampled structure (in-plane triangles dominate)
    E2 = oracle_mod.compute_batch(sub, PRM)["E"]
    assert np.all(ref["E"] > E2)
