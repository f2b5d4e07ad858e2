"""Pins of the oracle's optional three-body (Axilrod-Teller-Muto) term.

The paper leaves the three-body term out (Sec. II A); the oracle evaluates the
D3 triple-dipole form when s9 != 0.  It is pinned against things fixed
independently of its own code:

* an equilateral triangle with one-reference tables (C6 constant): the closed
  form s9 C6^(3/2) (11/8) / r^9 / (1 + 6 (R/r)^alpha), and its breathing-mode
  derivative;
* the angular factor against the dipole-tensor identity
  Tr(T_ab T_bc T_ca) = -3 (3 cos A cos B cos C + 1) / (r_ab r_bc r_ca)^3,
  T = (3 u u^T - 1) / r^3 (a formula with no cosines), on acute, obtuse and
  collinear triangles;
* a pure-Python triple loop over an open cluster (i < j < k, all three sides
  below rc3), which pins the enumeration, the cutoff on the third side and
  the weight of each triangle;
* F = -dE/dx and W = -dE/d(strain) by central differences with CN-dependent
  C6 (the chain rule through every pair of the triangle), supercell
  extensivity in a cell smaller than the cutoff, invariances, linearity in s9
  and dE/d(a1, a2) by finite differences.
"""
import itertools

import numpy as np

from paper_2310_05279_gb300 import workloads as wl

from .test_oracle_invariants import min_pair_ok, small_triclinic

BOHR = 0.529177210903
HARTREE = 27.211386245988
PRM = dict(wl.PBE_BJ)
OPEN = [0, 0, 0]
BOX = np.eye(3) * 60.0


def atm_only(**kw):
    p = dict(PRM, s6=0.0, s8=0.0, s9=1.0, alpha9=16.0)
    p.update(kw)
    return p


def one_ref_tables(names, seed):
    return wl.random_tables(names, seed, nref_max=1)


def damp_R(tabs, ti, tj, p):
    return p["a1"] * np.sqrt(3.0 * tabs.sqrtq[ti] * tabs.sqrtq[tj]) + p["a2"]


def tensor_factor(P):
    """(3 cos A cos B cos C + 1) / (r_ab r_bc r_ca)^3 from the dipole tensors, positions in bohr."""
    def T(a, b):
        d = P[b] - P[a]
        r = np.linalg.norm(d)
        u = d / r
        return (3.0 * np.outer(u, u) - np.eye(3)) / r ** 3
    return -np.trace(T(0, 1) @ T(1, 2) @ T(2, 0)) / 3.0


def test_equilateral_closed_form(oracle_mod):
    tabs = one_ref_tables(["C"], 1007)
    c6 = tabs.c6_ref[0, 0, 0, 0]
    p = atm_only()
    R = damp_R(tabs, 0, 0, p)
    for r_A in (1.6, 2.5, 3.3, 4.7):
        pos = np.array([[0, 0, 0], [r_A, 0, 0], [0.5 * r_A, np.sqrt(3) / 2 * r_A, 0]]) + 20.0
        res = oracle_mod.compute(pos, [0, 0, 0], BOX, OPEN, tabs, p)

        def closed(ra):
            r = ra / BOHR
            return c6 ** 1.5 * (11.0 / 8.0) / r ** 9 / (1.0 + 6.0 * (R / r) ** 16) * HARTREE
        assert res["E"] > 0  # the triple-dipole term is repulsive for an equilateral triangle
        assert abs(res["E"] - closed(r_A)) <= 1e-13 * abs(closed(r_A))
        np.testing.assert_allclose(res["e_atom"], closed(r_A) / 3, rtol=1e-13)
        # breathing mode: sum_i F_i . (x_i - centre) = -r dE/dr
        h = 1e-6
        dEdr = (closed(r_A + h) - closed(r_A - h)) / (2 * h)
        c = pos.mean(0)
        assert abs(np.sum(res["F"] * (pos - c)) + r_A * dEdr) <= 1e-7 * abs(r_A * dEdr)
        np.testing.assert_allclose(res["F"].sum(0), 0.0, atol=1e-14 * np.abs(res["F"]).max() + 1e-300)


def test_angular_factor_dipole_tensor(oracle_mod):
    tabs = one_ref_tables(["C"], 1007)
    c6 = tabs.c6_ref[0, 0, 0, 0]
    p = atm_only(a1=0.0, a2=1e-4, rc3=6.0)  # (R/r)^16 ~ 1e-64: f = 1 in FP64
    g = np.random.Generator(np.random.PCG64(31))
    shapes = [np.array([[0, 0, 0], [2.0, 0, 0], [4.0, 0, 0]]),            # collinear, equal spacing
              np.array([[0, 0, 0], [1.5, 0, 0], [4.4, 0, 0]]),            # collinear, uneven
              np.array([[0, 0, 0], [3.0, 0, 0], [1.4, 0.4, 0]])]          # obtuse
    shapes += [g.uniform(0, 3.2, (3, 3)) for _ in range(6)]
    for P in shapes:
        d = np.linalg.norm(P[:, None] - P[None], axis=-1)
        assert d[np.triu_indices(3, 1)].max() < 6.0 and d[np.triu_indices(3, 1)].min() > 0.8
        res = oracle_mod.compute(P + 20.0, [0, 0, 0], BOX, OPEN, tabs, p)
        expect = c6 ** 1.5 * tensor_factor(P / BOHR) * HARTREE
        assert abs(res["E"] - expect) <= 1e-12 * abs(expect)
    # the collinear, equally spaced chain: 3 (1)(1)(-1) + 1 = -2, attractive
    res = oracle_mod.compute(shapes[0] + 20.0, [0, 0, 0], BOX, OPEN, tabs, p)
    r = 2.0 / BOHR
    assert abs(res["E"] - c6 ** 1.5 * (-2.0) / (r * r * 2 * r) ** 3 * HARTREE) <= 1e-12 * abs(res["E"])


def test_brute_force_cluster(oracle_mod):
    names = ["H", "C", "O"]
    tabs = one_ref_tables(names, 1011)
    g = np.random.Generator(np.random.PCG64(5))
    n = 9
    pos = g.uniform(0, 6.0, (n, 3))
    types = g.integers(0, 3, n).astype(np.int32)
    for rc3 in (3.5, 4.5, 6.0):
        p = atm_only(rc3=rc3)
        res = oracle_mod.compute(pos + 20.0, types, BOX, OPEN, tabs, p)
        E = 0.0
        ntri = 0
        for i, j, k in itertools.combinations(range(n), 3):
            sides = [np.linalg.norm(pos[a] - pos[b]) for a, b in ((i, j), (i, k), (j, k))]
            if max(sides) >= rc3:
                continue
            ntri += 1
            t = types
            c9 = np.sqrt(tabs.c6_ref[t[i], t[j], 0, 0] * tabs.c6_ref[t[i], t[k], 0, 0] * tabs.c6_ref[t[j], t[k], 0, 0])
            Rbar = (damp_R(tabs, t[i], t[j], p) * damp_R(tabs, t[i], t[k], p) * damp_R(tabs, t[j], t[k], p)) ** (1 / 3)
            rbar = (np.prod(sides) / BOHR ** 3) ** (1 / 3)
            f = 1.0 / (1.0 + 6.0 * (Rbar / rbar) ** 16)
            E += c9 * tensor_factor(pos[[i, j, k]] / BOHR) * f
        assert ntri > 3
        assert abs(res["E"] - E * HARTREE) <= 1e-12 * abs(E * HARTREE)


def dense_triclinic(seed):
    pos, types, cell, tabs = small_triclinic(seed=seed, n=6, scale=4.6)
    return pos, types, cell, tabs


def test_forces_are_minus_gradient(oracle_mod):
    """CN-dependent C6 (multi-reference tables): the chain rule runs through all
    three pairs of every triangle; the cell is smaller than rc3, so triangles
    include images of one atom."""
    pos, types, cell, tabs = dense_triclinic(21)
    h = 1e-5
    for p in (atm_only(rc3=5.0), dict(PRM, s9=1.0, alpha9=16.0, rc3=6.0)):
        assert min_pair_ok(pos, cell, (12.0, 6.0, p["rc3"]), h)
        r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, p)
        ref = atm_only(rc3=p["rc3"], s9=0.0)
        assert r0["E"] != oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, dict(p, s9=0.0))["E"]
        fmax = np.abs(r0["F"]).max()
        assert fmax > 0
        for i in range(len(pos)):
            for a in range(3):
                pp, mm = pos.copy(), pos.copy()
                pp[i, a] += h
                mm[i, a] -= h
                Ep = oracle_mod.compute(pp, types, cell, [1, 1, 1], tabs, p)["E"]
                Em = oracle_mod.compute(mm, types, cell, [1, 1, 1], tabs, p)["E"]
                assert abs(-(Ep - Em) / (2 * h) - r0["F"][i, a]) < 1e-6 * fmax + 1e-11
        del ref


def test_virial_is_minus_strain_derivative(oracle_mod):
    pos, types, cell, tabs = dense_triclinic(21)
    p = atm_only(rc3=5.0)
    h = 1e-6
    r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, p)
    wmax = np.abs(r0["W"]).max()
    assert wmax > 0
    for a in range(3):
        for b in range(a, 3):
            e = np.zeros((3, 3))
            e[a, b] = e[b, a] = h if a == b else 0.5 * h
            Ep = oracle_mod.compute(pos @ (np.eye(3) + e).T, types, cell @ (np.eye(3) + e).T, [1, 1, 1], tabs, p)["E"]
            Em = oracle_mod.compute(pos @ (np.eye(3) - e).T, types, cell @ (np.eye(3) - e).T, [1, 1, 1], tabs, p)["E"]
            assert abs(r0["W"][a, b] + (Ep - Em) / (2 * h)) < 1e-6 * wmax


def test_supercell_and_invariances(oracle_mod):
    pos, types, cell, tabs = dense_triclinic(5)
    p = dict(PRM, s9=1.0, alpha9=16.0, rc3=6.0)
    r1 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, p)
    reps = (2, 1, 2)
    sp = [pos + np.array([a, b, c]) @ cell for a in range(reps[0]) for b in range(reps[1]) for c in range(reps[2])]
    k = int(np.prod(reps))
    r2 = oracle_mod.compute(np.concatenate(sp), np.tile(types, k), cell * np.array(reps)[:, None], [1, 1, 1], tabs, p)
    assert abs(r2["E"] - k * r1["E"]) <= 1e-12 * abs(k * r1["E"])
    np.testing.assert_allclose(r2["F"], np.tile(r1["F"], (k, 1)), rtol=0, atol=1e-12 * np.abs(r1["F"]).max())
    np.testing.assert_allclose(r2["W"], k * r1["W"], rtol=0, atol=1e-12 * np.abs(r1["W"]).max() * k)
    np.testing.assert_allclose(r1["F"].sum(0), 0.0, atol=1e-12 * np.abs(r1["F"]).max())
    np.testing.assert_allclose(r1["W"], r1["W"].T, atol=1e-13 * np.abs(r1["W"]).max())
    assert abs(r1["e_atom"].sum() - r1["E"]) <= 1e-12 * abs(r1["E"])
    th = 0.61
    Q = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    rr = oracle_mod.compute(pos @ Q.T + np.array([1.3, -7.9, 4.4]), types, cell @ Q.T, [1, 1, 1], tabs, p)
    assert abs(rr["E"] - r1["E"]) <= 1e-12 * abs(r1["E"])
    np.testing.assert_allclose(rr["F"], r1["F"] @ Q.T, atol=1e-12 * np.abs(r1["F"]).max())
    np.testing.assert_allclose(rr["W"], Q @ r1["W"] @ Q.T, atol=1e-12 * np.abs(r1["W"]).max())
    perm = np.random.Generator(np.random.PCG64(2)).permutation(len(pos))
    rp = oracle_mod.compute(pos[perm], types[perm], cell, [1, 1, 1], tabs, p)
    assert abs(rp["E"] - r1["E"]) <= 1e-12 * abs(r1["E"])
    np.testing.assert_allclose(rp["F"], r1["F"][perm], atol=1e-12 * np.abs(r1["F"]).max())


def test_linearity_and_damping_derivatives(oracle_mod):
    pos, types, cell, tabs = dense_triclinic(9)
    base = dict(PRM, alpha9=16.0, rc3=5.5)
    E0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, dict(base, s9=0.0))["E"]
    E1 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, dict(base, s9=1.0))["E"]
    E2 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, dict(base, s9=2.5))["E"]
    assert E1 != E0
    assert abs((E2 - E0) - 2.5 * (E1 - E0)) <= 1e-12 * abs(E2)
    p = dict(base, s9=1.0)
    r0 = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, p)
    for key, idx in (("a1", 2), ("a2", 3)):
        h = 1e-6
        pp, pm = dict(p), dict(p)
        pp[key] += h
        pm[key] -= h
        fd = (oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, pp)["E"] -
              oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, pm)["E"]) / (2 * h)
        assert abs(fd - r0["dEdp"][idx]) < 1e-7 * abs(fd)
    # the three-body part of dE/da differs from the two-body part alone
    r2b = oracle_mod.compute(pos, types, cell, [1, 1, 1], tabs, dict(p, s9=0.0))
    assert abs(r2b["dEdp"][2] - r0["dEdp"][2]) > 1e-9 * abs(r0["dEdp"][2])
