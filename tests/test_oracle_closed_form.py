"""Pins of the FP64 oracle against closed forms evaluated independently.

The reference here is sympy: Eqs. 2-4 typed in their printed form (Eq. 3 as
the double-sum ratio, not the per-atom factorisation the oracle uses, no
max-shift), differentiated symbolically for forces and strain, and evaluated
to 30 digits.  A dropped term, a wrong sign, a transposed C6 reference index,
a wrong unit conversion or a broken chain rule in the oracle fails here.
"""
import math

import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

sympy = pytest.importorskip("sympy")
mpmath = pytest.importorskip("mpmath")

BOHR = 0.529177210903
HA = 27.211386245988


def two_element_tables():
    """Two elements with 3 and 2 references and a C6 grid that is not symmetric
    in (a, b) within a pair, so a transposed index changes the result."""
    nref = np.array([3, 2], np.int32)
    cn = np.array([[0.2, 1.1, 2.0], [0.5, 1.4, 0.0]])
    c6 = np.zeros((2, 2, 3, 3))
    c6[0, 0, :3, :3] = [[12.0, 17.0, 23.0], [17.0, 30.0, 41.0], [23.0, 41.0, 55.0]]
    c6[1, 1, :2, :2] = [[6.0, 9.5], [9.5, 14.0]]
    c6[0, 1, :3, :2] = [[8.0, 19.0], [11.0, 27.0], [15.0, 36.0]]
    c6[1, 0] = np.transpose(c6[0, 1])
    return wl.Tables(["A", "B"], nref, cn, c6, np.array([3.1, 2.4]), np.array([1.44, 1.31]))


def sympy_model(types, tables, prm):
    """Symbolic E(x) in eV for an open cluster (all pairs inside both cutoffs)."""
    n = len(types)
    X = sympy.symbols(f"x0:{3 * n}", real=True)
    pos = [X[3 * i:3 * i + 3] for i in range(n)]
    k1, k2, k3 = (sympy.Float(prm[k], 40) for k in ("k1", "k2", "k3"))
    s6, s8, a1, a2 = (sympy.Float(prm[k], 40) for k in ("s6", "s8", "a1", "a2"))
    bohr = sympy.Float(BOHR, 40)

    def r(i, j):
        return sympy.sqrt(sum((pos[j][a] - pos[i][a]) ** 2 for a in range(3))) / bohr

    rc = [float(tables.rcov[t]) for t in types]
    cn = [sum(1 / (1 + sympy.exp(-k1 * (k2 * (rc[i] + rc[j]) / r(i, j) - 1))) for j in range(n) if j != i)
          for i in range(n)]
    E = 0
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            ti, tj = types[i], types[j]
            num = 0
            den = 0
            for a in range(int(tables.nref[ti])):
                for b in range(int(tables.nref[tj])):
                    L = sympy.exp(-k3 * ((cn[i] - tables.cn_ref[ti, a]) ** 2 + (cn[j] - tables.cn_ref[tj, b]) ** 2))
                    num += tables.c6_ref[ti, tj, a, b] * L
                    den += L
            C6 = num / den
            R0 = sympy.sqrt(3 * sympy.Float(tables.sqrtq[ti], 40) * sympy.Float(tables.sqrtq[tj], 40))
            C8 = C6 * R0 ** 2
            Rd = a1 * R0 + a2
            rr = r(i, j)
            E += -sympy.Rational(1, 2) * (s6 * C6 / (rr ** 6 + Rd ** 6) + s8 * C8 / (rr ** 8 + Rd ** 8))
    return X, E * sympy.Float(HA, 40)


@pytest.fixture(scope="module")
def trimer():
    tables = two_element_tables()
    types = [0, 1, 0]
    pos = np.array([[0.0, 0.0, 0.0], [1.93, 0.21, -0.07], [0.44, 2.05, 0.33]])
    prm = dict(wl.PBE_BJ)
    X, E = sympy_model(types, tables, prm)
    mpmath.mp.dps = 30
    subs = {X[k]: sympy.Float(repr(float(pos.ravel()[k])), 40) for k in range(len(X))}
    Ev = sympy.N(E.subs(subs), 30)
    Fv = np.array([float(-sympy.N(sympy.diff(E, X[k]).subs(subs), 30)) for k in range(len(X))]).reshape(-1, 3)
    return tables, types, pos, prm, float(Ev), Fv


def test_trimer_energy_forces_virial(oracle_mod, trimer):
    tables, types, pos, prm, E_ref, F_ref = trimer
    r = oracle_mod.compute(pos, types, np.eye(3) * 30.0, [0, 0, 0], tables, prm)
    assert r["E"] < 0
    assert abs(r["E"] - E_ref) <= 1e-12 * abs(E_ref)
    np.testing.assert_allclose(r["F"], F_ref, rtol=0, atol=1e-11 * np.abs(F_ref).max())
    # virial of an open system: W_ab = sum_i F_ia x_ib (strain derivative of E)
    W_ref = F_ref.T @ pos
    np.testing.assert_allclose(r["W"], W_ref, rtol=0, atol=1e-11 * np.abs(W_ref).max())
    # coordination numbers sit between references, so every weight and chain term matters
    assert np.all((r["cn"] > 0.3) & (r["cn"] < 2.0))


def test_dimer_closed_form_and_short_range_limit(oracle_mod):
    """Isolated dimer: n1 = n2 = f(r); E(r) and dE/dr from the closed form.
    As r -> 0 the BJ-damped energy tends to the finite value
    -(s6 C6/R^6 + s8 C8/R^8) and the force to zero (no spurious short-range force)."""
    tables = wl.carbon_table(1000)
    prm = dict(wl.PBE_BJ)
    X, E = sympy_model([0, 0], tables, prm)
    for rA in (0.9, 1.42, 2.46, 3.4, 5.5):
        pos = np.array([[0.0, 0.0, 0.0], [rA, 0.0, 0.0]])
        subs = {X[k]: sympy.Float(repr(float(pos.ravel()[k])), 40) for k in range(6)}
        Ev = float(sympy.N(E.subs(subs), 30))
        dE = float(sympy.N(sympy.diff(E, X[3]).subs(subs), 30))
        r = oracle_mod.compute(pos, [0, 0], np.eye(3) * 40.0, [0, 0, 0], tables, prm)
        assert abs(r["E"] - Ev) <= 1e-12 * abs(Ev)
        assert abs(r["F"][1, 0] + dE) <= 1e-11 * max(abs(dE), 1e-8)
        assert abs(r["F"][0, 0] - dE) <= 1e-11 * max(abs(dE), 1e-8)
    # short-range limit
    e_small = []
    f_small = []
    for rA in (1e-2, 1e-3):
        pos = np.array([[0.0, 0.0, 0.0], [rA, 0.0, 0.0]])
        r = oracle_mod.compute(pos, [0, 0], np.eye(3) * 40.0, [0, 0, 0], tables, prm)
        e_small.append(r["E"])
        f_small.append(abs(r["F"][1, 0]))
    assert abs(e_small[0] - e_small[1]) < 1e-6 * abs(e_small[1])
    assert f_small[1] < f_small[0] < 1e-5


def test_single_reference_limit(oracle_mod):
    """One reference per element: W = 1, so C6 = C6ref exactly, the coordination
    numbers drop out (E and F independent of Rcov), and D3 reduces to the plain
    pairwise Becke-Johnson-damped C6/C8 potential."""
    g = np.random.Generator(np.random.PCG64(7))
    tabs = wl.random_tables(["H", "C", "O"], 77, max_ref=1, nref_max=1)
    pos = g.uniform(0, 7.0, (9, 3))
    types = g.integers(0, 3, 9).astype(np.int32)
    prm = dict(wl.PBE_BJ)
    big = np.eye(3) * 50.0
    r1 = oracle_mod.compute(pos, types, big, [0, 0, 0], tabs, prm)
    tabs2 = wl.Tables(tabs.names, tabs.nref, tabs.cn_ref, tabs.c6_ref, tabs.sqrtq, tabs.rcov * 1.7)
    r2 = oracle_mod.compute(pos, types, big, [0, 0, 0], tabs2, prm)
    assert abs(r1["E"] - r2["E"]) <= 1e-14 * abs(r1["E"])
    np.testing.assert_allclose(r1["F"], r2["F"], rtol=0, atol=1e-14)
    assert np.all(r1["dEdn"] == 0.0)
    # textbook pairwise sum
    E = 0.0
    for i in range(9):
        for j in range(i + 1, 9):
            rr = np.linalg.norm(pos[j] - pos[i]) / BOHR
            if rr * BOHR >= 12.0:
                continue
            ti, tj = types[i], types[j]
            C6 = tabs.c6_ref[ti, tj, 0, 0]
            R0 = math.sqrt(3 * tabs.sqrtq[ti] * tabs.sqrtq[tj])
            Rd = prm["a1"] * R0 + prm["a2"]
            E -= prm["s6"] * C6 / (rr ** 6 + Rd ** 6) + prm["s8"] * C6 * R0 ** 2 / (rr ** 8 + Rd ** 8)
    assert abs(r1["E"] - E * HA) <= 1e-13 * abs(E * HA)


def test_weights_limits(oracle_mod):
    """Eq. 3 weights: equal to the unshifted normalised Gaussians where those are
    representable, a partition of unity, dW/dn matching finite differences, and
    all weight on the nearest reference where every Gaussian underflows."""
    tabs = two_element_tables()
    for n in (0.0, 0.7, 1.3, 2.6):
        W, dW = oracle_mod.weights(tabs, 0, n)
        L = np.exp(-4.0 * (n - tabs.cn_ref[0, :3]) ** 2)
        np.testing.assert_allclose(W[:3], L / L.sum(), rtol=1e-14, atol=1e-300)
        assert abs(W.sum() - 1.0) < 1e-15
        h = 1e-6
        Wp, _ = oracle_mod.weights(tabs, 0, n + h)
        Wm, _ = oracle_mod.weights(tabs, 0, n - h)
        np.testing.assert_allclose(dW, (Wp - Wm) / (2 * h), rtol=0, atol=1e-7)
    n = 40.0
    with np.errstate(invalid="ignore"):
        L = np.exp(-4.0 * (n - tabs.cn_ref[0, :3]) ** 2)   # every Gaussian underflows: Eq. 3 reads 0/0
        assert np.all(L == 0.0) and np.isnan((L / L.sum())[0])
    W, dW = oracle_mod.weights(tabs, 0, n)
    assert W[2] == 1.0 and W[0] < 1e-100 and W[1] < 1e-100
    assert np.all(np.abs(dW) < 1e-100)
