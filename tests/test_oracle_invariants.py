"""Pins of the FP64 oracle against invariants and finite differences.

Periodic images (including an atom's own images in cells smaller than the
cutoff), the force/virial chain rule and the parameter derivatives are
checked against properties fixed by the mathematics: extensivity over
supercells, translation/rotation/permutation invariance, Newton's third law,
F = -dE/dx and W = -dE/d(strain) by central differences, linearity in s6/s8,
and locality (a site's force depends only on atoms within R_pot + 2 R_cn).
"""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import cluster_around

PRM = dict(wl.PBE_BJ)


def small_triclinic(seed=11, n=6, scale=6.5):
    g = np.random.Generator(np.random.PCG64(seed))
    cell = np.array([[scale, 0.0, 0.0], [0.9, scale * 0.95, 0.0], [-0.7, 0.6, scale * 1.05]])
    f = g.uniform(0, 1, (n, 3))
    pos = f @ cell
    types = g.integers(0, 3, n).astype(np.int32)
    tabs = wl.random_tables(["H", "C", "O"], 1000 + seed)
    return pos, types, cell, tabs


def min_pair_ok(pos, cell, rcuts, h, pbc=(1, 1, 1)):
    """True if no instance distance lies within h of any cutoff (FD stencils stay on one side)."""
    inv = np.linalg.inv(cell)
    d = pos[None, :, :] - pos[:, None, :]
    rng = range(-4, 5)
    for n0 in rng:
        for n1 in rng:
            for n2 in rng:
                T = np.array([n0, n1, n2]) @ cell
                r = np.linalg.norm(d + T, axis=-1)
                for rc in rcuts:
                    if np.any(np.abs(r - rc) < 4 * h):
                        return False
    return True


def test_supercell_extensivity(oracle_mod):
    pos, types, cell, tabs = small_triclinic()
    r1 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, PRM)
    reps = (2, 1, 3)
    sp, st = [], []
    for a in range(reps[0]):
        for b in range(reps[1]):
            for c in range(reps[2]):
                sp.append(pos + np.array([a, b, c]) @ cell)
                st.append(types)
    sc = cell * np.array(reps)[:, None]
    r2 = oracle_mod.compute(np.concatenate(sp), np.concatenate(st), sc, [1, 1, 1], tabs, PRM)
    k = np.prod(reps)
    assert abs(r2["E"] - k * r1["E"]) <= 1e-12 * abs(k * r1["E"])
    np.testing.assert_allclose(r2["F"], np.tile(r1["F"], (k, 1)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(r2["W"], k * r1["W"], rtol=0, atol=1e-12 * np.abs(r1["W"]).max() * k)
    np.testing.assert_allclose(r2["cn"], np.tile(r1["cn"], k), rtol=1e-13)


def test_single_atom_self_images(oracle_mod):
    """One atom in a ~3 A cell interacts only with its own images; E doubles in a
    2x1x1 supercell.  (Edges chosen so that no image sits exactly on a cutoff.)"""
    tabs = wl.carbon_table(1000)
    cell = np.diag([3.1, 3.3, 3.7])
    r1 = oracle_mod.compute(np.array([[0.3, 0.2, 0.1]]), [0], cell, [1, 1, 1], tabs, PRM)
    assert r1["E"] < 0 and r1["cn"][0] > 0
    np.testing.assert_allclose(r1["F"], 0.0, atol=1e-14)
    r2 = oracle_mod.compute(np.array([[0.3, 0.2, 0.1], [3.4, 0.2, 0.1]]), [0, 0], np.diag([6.2, 3.3, 3.7]),
                            [1, 1, 1], tabs, PRM)
    assert abs(r2["E"] - 2 * r1["E"]) <= 1e-12 * abs(r1["E"])


def test_invariances(oracle_mod):
    pos, types, cell, tabs = small_triclinic(seed=5, n=7)
    r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, PRM)
    assert r0["E"] < 0
    np.testing.assert_allclose(r0["F"].sum(0), 0.0, atol=1e-12)
    np.testing.assert_allclose(r0["W"], r0["W"].T, atol=1e-12)
    # translation (including moves across the periodic boundary)
    rt = oracle_mod.compute(pos + np.array([3.7, -11.2, 25.1]), types, cell, [1, 1, 1], tabs, PRM)
    assert abs(rt["E"] - r0["E"]) <= 1e-12 * abs(r0["E"])
    np.testing.assert_allclose(rt["F"], r0["F"], atol=1e-12)
    np.testing.assert_allclose(rt["W"], r0["W"], atol=1e-12)
    # rotation of positions and cell
    th = 0.83
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    Q = Rz @ Rx
    rr = oracle_mod.compute(pos @ Q.T, types, cell @ Q.T, [1, 1, 1], tabs, PRM)
    assert abs(rr["E"] - r0["E"]) <= 1e-12 * abs(r0["E"])
    np.testing.assert_allclose(rr["F"], r0["F"] @ Q.T, atol=1e-12)
    np.testing.assert_allclose(rr["W"], Q @ r0["W"] @ Q.T, atol=1e-12)
    # permutation
    perm = np.random.Generator(np.random.PCG64(3)).permutation(len(pos))
    rp = oracle_mod.compute(pos[perm], types[perm], cell, [1, 1, 1], tabs, PRM)
    assert abs(rp["E"] - r0["E"]) <= 1e-12 * abs(r0["E"])
    np.testing.assert_allclose(rp["F"], r0["F"][perm], atol=1e-12)


def test_forces_are_minus_gradient(oracle_mod):
    pos, types, cell, tabs = small_triclinic(seed=21, n=6)
    h = 1e-5
    assert min_pair_ok(pos, cell, (12.0, 6.0), h)
    r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, PRM)
    for i in range(len(pos)):
        for a in range(3):
            p, m = pos.copy(), pos.copy()
            p[i, a] += h
            m[i, a] -= h
            Ep = oracle_mod.compute(p, types, cell, [1, 1, 1], tabs, PRM)["E"]
            Em = oracle_mod.compute(m, types, cell, [1, 1, 1], tabs, PRM)["E"]
            assert abs(-(Ep - Em) / (2 * h) - r0["F"][i, a]) < 2e-8


def test_virial_is_minus_strain_derivative(oracle_mod):
    pos, types, cell, tabs = small_triclinic(seed=21, n=6)
    h = 1e-6
    r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, PRM)
    for a in range(3):
        for b in range(a, 3):
            e = np.zeros((3, 3))
            e[a, b] = e[b, a] = h if a != b else h
            if a != b:
                e *= 0.5
            Ep = oracle_mod.compute(pos @ (np.eye(3) + e).T, types, cell @ (np.eye(3) + e).T, [1, 1, 1], tabs, PRM)["E"]
            Em = oracle_mod.compute(pos @ (np.eye(3) - e).T, types, cell @ (np.eye(3) - e).T, [1, 1, 1], tabs, PRM)["E"]
            # symmetric strain (e_ab = e_ba = h/2 off the diagonal): dE = -h W_ab
            expect = -(Ep - Em) / (2 * h)
            assert abs(r0["W"][a, b] - expect) < 1e-6 * max(1.0, abs(expect))


def test_parameter_derivatives(oracle_mod):
    pos, types, cell, tabs = small_triclinic(seed=9, n=6)
    r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, PRM)
    # E is linear in s6 and s8
    for k, idx in (("s6", 0), ("s8", 1)):
        p2 = dict(PRM)
        p2[k] = PRM[k] + 0.37
        E2 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, p2)["E"]
        assert abs((E2 - r0["E"]) / 0.37 - r0["dEdp"][idx]) < 1e-10 * abs(r0["dEdp"][idx])
    p0 = dict(PRM, s6=0.0, s8=0.0)
    assert oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, p0)["E"] == 0.0
    # a1, a2 by central differences
    for k, idx in (("a1", 2), ("a2", 3)):
        h = 1e-6
        pp, pm = dict(PRM), dict(PRM)
        pp[k] += h
        pm[k] -= h
        fd = (oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, pp)["E"] -
              oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, pm)["E"]) / (2 * h)
        assert abs(fd - r0["dEdp"][idx]) < 1e-7 * abs(fd)


def test_site_energies_sum(oracle_mod):
    pos, types, cell, tabs = small_triclinic(seed=13, n=8)
    r = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, PRM)
    assert abs(r["e_atom"].sum() - r["E"]) <= 1e-13 * abs(r["E"])
    assert np.all(r["e_atom"] < 0)


def test_locality_of_forces(oracle_mod):
    """The force on atom i depends only on atoms within R_pot + 2 R_cn = 24 A and
    its site energy only on atoms within R_pot + R_cn = 18 A: an open cluster
    cut at those radii reproduces the periodic results for the centre atom."""
    b = wl.mof_like_box(ncell=9)
    pos, types, cell, pbc = b.structure(0)
    ref = oracle_mod.compute(pos, types, cell, pbc, b.tables, PRM)
    for i in (5, 1711, 2900):
        cp, ct = cluster_around(pos, types, cell, i, 24.0 + 1e-6)
        rc = oracle_mod.compute(cp, ct, np.eye(3) * 200.0, [0, 0, 0], b.tables, PRM)
        np.testing.assert_allclose(rc["F"][0], ref["F"][i], rtol=0, atol=1e-12)
        assert abs(rc["e_atom"][0] - ref["e_atom"][i]) < 1e-13
        assert abs(rc["cn"][0] - ref["cn"][i]) < 1e-12
        # too small a cluster misses the chain-rule terms of distant neighbours' CNs
        cp2, ct2 = cluster_around(pos, types, cell, i, 14.0)
        rs = oracle_mod.compute(cp2, ct2, np.eye(3) * 200.0, [0, 0, 0], b.tables, PRM)
        assert np.abs(rs["F"][0] - ref["F"][i]).max() > 1e-9


@pytest.mark.slow
def test_cutoff_convergence(oracle_mod):
    """Fig. 1(d): with R_cn = R_pot / 2 the force RMSE against a long-cutoff
    evaluation (R_pot 50.2 A, R_cn 20 A, the VASP defaults) falls as R_pot grows."""
    b = wl.mof_like_box(ncell=3, seed=5)
    pos, types, cell, pbc = b.structure(0)
    ref = oracle_mod.compute(pos, types, cell, pbc, b.tables, dict(PRM, rc_disp=50.2, rc_cn=20.0))["F"]
    rmse = []
    for rp in (8.0, 12.0, 16.0, 20.0, 30.0):
        F = oracle_mod.compute(pos, types, cell, pbc, b.tables, dict(PRM, rc_disp=rp, rc_cn=rp / 2))["F"]
        rmse.append(float(np.sqrt(np.mean((F - ref) ** 2))))
    assert all(rmse[k + 1] < rmse[k] for k in range(len(rmse) - 1)), rmse
