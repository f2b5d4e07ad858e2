"""Pins of the oracle's per-atom virial (Eq. 7) that do not reuse its algebra.

* On an open cluster Eq. 7 can be evaluated from site energies alone: U_j is a
  function of the vectors from j, and moving atom i changes only r_ji among
  them, so dU_j/dr_ji = grad_{x_i} U_j.  Central differences of the oracle's
  site energies (Eq. 2) then give W_i = sum_j r_ij (x) grad_{x_i} U_j.
* The per-atom virials sum to the total virial W = -sum d (x) dE/dd, including
  periodic cells with self-images; their three-body parts cancel in the sum.
* Translation invariance and permutation covariance.
"""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

PRM = dict(wl.PBE_BJ)


def _cluster(seed, n, box, tabs):
    g = np.random.Generator(np.random.PCG64(seed))
    while True:
        pos = g.uniform(0, box, (n, 3))
        r = np.linalg.norm(pos[:, None] - pos[None], axis=2)[np.triu_indices(n, 1)]
        # no pair near a cutoff (the terms are hard-truncated) and none too close
        if r.min() > 1.0 and np.abs(r - 6.0).min() > 0.05 and np.abs(r - 12.0).min() > 0.05:
            return pos, g.integers(0, len(tabs.names), n).astype(np.int32)


@pytest.mark.parametrize("seed", [1, 2])
def test_eq7_from_site_energies_open_cluster(oracle_mod, seed):
    tabs = wl.random_tables(["H", "C", "O"], 7 + seed)
    pos, typ = _cluster(seed, 14, 11.0, tabs)
    cell, pbc = np.eye(3) * 400.0, np.zeros(3, np.int32)
    Wa = oracle_mod.atom_virial(pos, typ, cell, pbc, tabs, PRM)
    n, h = len(pos), 1e-4
    ref = np.zeros((n, 3, 3))
    for i in range(n):
        for b in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, b] += h
            pm[i, b] -= h
            gU = (oracle_mod.compute(pp, typ, cell, pbc, tabs, PRM)["e_atom"]
                  - oracle_mod.compute(pm, typ, cell, pbc, tabs, PRM)["e_atom"]) / (2 * h)  # d U_j / d x_i,b
            for j in range(n):
                if j != i:
                    ref[i, :, b] += (pos[j] - pos[i]) * gU[j]
    scale = np.abs(ref).max()
    assert np.abs(Wa - ref).max() <= 1e-6 * scale
    # the CN terms make the per-atom virial non-symmetric
    assert np.abs(Wa - Wa.transpose(0, 2, 1)).max() > 1e-6 * scale


@pytest.mark.parametrize("case", ["bilayer", "triclinic", "self_images"])
def test_atom_virials_sum_to_total(oracle_mod, case):
    if case == "bilayer":
        b = wl.bilayer_ab_64()
        pos, typ, cell, pbc = b.structure(0)
        tabs = b.tables
    elif case == "triclinic":
        b = wl.uneven_batch(seed=8, nstruct=1, n_range=(40, 41))
        pos, typ, cell, pbc = b.structure(0)
        tabs = b.tables
    else:
        tabs = wl.random_tables(["C", "O"], 3)
        pos = np.array([[0.3, 0.2, 0.1], [1.6, 1.1, 1.9]])
        typ = np.array([0, 1], np.int32)
        cell, pbc = np.diag([3.1, 3.3, 3.7]), np.ones(3, np.int32)
    Wa = oracle_mod.atom_virial(pos, typ, cell, pbc, tabs, PRM)
    W = oracle_mod.compute(pos, typ, cell, pbc, tabs, PRM)["W"]
    assert np.abs(Wa.sum(0) - W).max() <= 1e-10 * np.abs(W).max()


def test_atom_virial_invariances(oracle_mod):
    b = wl.uneven_batch(seed=9, nstruct=1, n_range=(30, 31))
    pos, typ, cell, pbc = b.structure(0)
    W0 = oracle_mod.atom_virial(pos, typ, cell, pbc, b.tables, PRM)
    W1 = oracle_mod.atom_virial(pos + [0.37, -1.2, 2.9], typ, cell, pbc, b.tables, PRM)
    assert np.abs(W1 - W0).max() <= 1e-9 * np.abs(W0).max()
    perm = np.random.Generator(np.random.PCG64(3)).permutation(len(pos))
    W2 = oracle_mod.atom_virial(pos[perm], typ[perm], cell, pbc, b.tables, PRM)
    assert np.abs(W2 - W0[perm]).max() <= 1e-9 * np.abs(W0).max()
