"""Planted mistakes in the oracle are caught by its pins.

Each mutant below is a copy of ``oracle/d3_oracle.c`` with one plausible
mistake: a dropped term, a wrong sign, index, factor or unit, a missing
periodic image, a broken chain rule.  The copy is compiled with the oracle's
own flags, and the pins of the other oracle tests are run against it:
- the closed forms typed in from Eqs. 2-4 (sympy);
- the single-reference limit;
- supercell extensivity and self-images;
- invariances;
- finite-difference forces, virial and parameter derivatives;
- the three-body closed forms;
- the per-atom virial sum;
- the constants the paper prints.
At least one pin must fail.  The regression fixture written by the oracle
itself is not among the pins: it would catch any change and prove nothing.

An unmodified copy built the same way must pass every pin, so the harness
cannot report a catch on its own.  The oracle itself is not changed by this
test.
"""
import pytest

import oracle

from . import test_golden as golden
from . import test_oracle_atm as atm
from . import test_oracle_atom_virial as av
from . import test_oracle_closed_form as cf
from . import test_oracle_invariants as inv

trimer = cf.trimer  # the sympy reference of the two-element trimer (module-scoped fixture)

# (name, mistake, original text, replacement, occurrences of the original text)
MUTANTS = [
    ("c8_term_dropped", "Eq. 2 without its s8 C8 term",
     "double e = -0.5 * (p->s6 * C6 / d6 + p->s8 * C8 / d8);", "double e = -0.5 * (p->s6 * C6 / d6);", 1),
    ("r0_without_factor_3", "R0^2 = sqrtQ_i sqrtQ_j (the literal geometric mean)",
     "double R0sq = 3.0 * t->sqrtq[ti] * t->sqrtq[tj];", "double R0sq = t->sqrtq[ti] * t->sqrtq[tj];", 1),
    ("bj_radius_without_a2", "damping radius a1 R0 instead of a1 R0 + a2",
     "double Rd = p->a1 * R0 + p->a2_bohr;", "double Rd = p->a1 * R0;", 1),
    ("cn_without_k2", "Eq. 4 with the tabulated covalent radii unscaled (k2 dropped everywhere)",
     "double rc_eff = p->k2 * (t->rcov[types[s->i]] + t->rcov[types[s->j]]);",
     "double rc_eff = (t->rcov[types[s->i]] + t->rcov[types[s->j]]);", 2),
    ("cn_exponent_sign", "Eq. 4 with the sign of the exponent flipped",
     "return 1.0 / (1.0 + exp(-k1 * (rc_eff / r - 1.0)));", "return 1.0 / (1.0 + exp(k1 * (rc_eff / r - 1.0)));",
     1),
    ("c6_reference_transposed", "Eq. 3 reading C6ref[b][a] instead of C6ref[a][b]",
     "double c = cref[a * R + b];\n                C6 += Wt[R * s->i + a] * Wt[R * s->j + b] * c;\n                dC6i",
     "double c = cref[b * R + a];\n                C6 += Wt[R * s->i + a] * Wt[R * s->j + b] * c;\n                dC6i",
     1),
    ("weights_not_normalised", "Eq. 3 without the normalising sum",
     "for (int a = 0; a < nr; ++a) W[a] /= sum;", ";", 1),
    ("weights_width", "Eq. 3 Gaussian exponent -k3/2 (n - nref)^2",
     "ex[a] = -k3 * z * z;", "ex[a] = -0.5 * k3 * z * z;", 1),
    ("dEdn_partner_dropped", "dE/dn collected for atom i only, not for its partner j",
     "dEdn[s->j] += de_dC6 * dC6j;", ";", 1),
    ("direct_force_newton", "pair force added to both atoms with the same sign",
     "Fb[3 * s->i + a] += g;\n            Fb[3 * s->j + a] -= g;\n            for (int b = 0; b < 3; ++b) Wv[3 * a + b] -= "
     "s->d[a] * de_dr",
     "Fb[3 * s->i + a] += g;\n            Fb[3 * s->j + a] += g;\n            for (int b = 0; b < 3; ++b) Wv[3 * a + b] -= "
     "s->d[a] * de_dr", 1),
    ("direct_virial_index", "direct virial d_a d_a instead of d_a d_b",
     "Wv[3 * a + b] -= s->d[a] * de_dr * s->d[b] / r;", "Wv[3 * a + b] -= s->d[a] * de_dr * s->d[a] / r;", 1),
    ("chain_virial_sign", "CN chain-rule virial with the wrong sign",
     "Wv[3 * a + b] -= s->d[a] * g_r * s->d[b] / s->r;", "Wv[3 * a + b] += s->d[a] * g_r * s->d[b] / s->r;", 1),
    ("images_one_short", "image range floor(r / width) instead of ceil",
     "m[k] = pbc[k] ? (int)ceil(rmax / plane_width(Hb, k)) : 0;\n\n    int64_t ni",
     "m[k] = pbc[k] ? (int)floor(rmax / plane_width(Hb, k)) : 0;\n\n    int64_t ni", 1),
    ("own_images_excluded", "j != i read as excluding an atom's own periodic images",
     "if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;", "if (i == j) continue;", 1),
    ("force_units", "forces in eV/bohr instead of eV/A",
     "eV_A = ORACLE_HARTREE_EV / ORACLE_BOHR_A;", "eV_A = ORACLE_HARTREE_EV;", 1),
    ("wrap_transposed_inverse", "fractional coordinates from the transposed inverse cell",
     "for (int k = 0; k < 3; ++k) f[k] = xb[0] * Hi[k] + xb[1] * Hi[3 + k] + xb[2] * Hi[6 + k];",
     "for (int k = 0; k < 3; ++k) f[k] = xb[0] * Hi[3 * k] + xb[1] * Hi[3 * k + 1] + xb[2] * Hi[3 * k + 2];", 2),
    ("atm_angular_sign", "three-body angular factor 3 cos cos cos - 1",
     "double ang = 3.0 * ci * cj * ck + 1.0;", "double ang = 3.0 * ci * cj * ck - 1.0;", 1),
    ("atm_damping_power", "three-body damping (R/r)^(alpha/3)",
     "double q = pow(Rbar / rbar, p->alpha9);", "double q = pow(Rbar / rbar, p->alpha9 / 3.0);", 1),
    ("atm_triangle_counted_thrice", "each of the three sightings of a triangle carries its whole energy",
     "Etot += third * e;", "Etot += e;", 1),
    ("atm_cosine_sides", "cosine at j from the wrong pair of sides",
     "double cj = (u * u + w * w - v * v) / (2.0 * u * w);", "double cj = (u * u + v * v - w * w) / (2.0 * u * w);",
     1),
    ("eq7_second_neighbour_term_dropped", "Eq. 7 without the terms through other partners' CNs",
     "Wa[9 * c + 3 * a + bb] += rij * Bq[q1] * fp * s2->d[bb] / s2->r;",
     "Wa[9 * c + 3 * a + bb] += 0.0 * rij * Bq[q1] * fp * s2->d[bb] / s2->r;", 1),
    ("eq7_partner_cn_sign", "Eq. 7 with the sign of the term through the partner's CN flipped",
     "g[a] += dUdr[q] * s->d[a] / s->r - Bq[q] * G[3 * i + a];",
     "g[a] += dUdr[q] * s->d[a] / s->r + Bq[q] * G[3 * i + a];", 1),
]


def battery(trimer_ref):
    """The pins, cheapest first: (name, callable taking the oracle module)."""
    return [
        ("dimer closed form", cf.test_dimer_closed_form_and_short_range_limit),
        ("trimer closed form", lambda o: cf.test_trimer_energy_forces_virial(o, trimer_ref)),
        ("single-reference limit", cf.test_single_reference_limit),
        ("Eq. 3 weight limits", cf.test_weights_limits),
        ("paper constants", golden.test_paper_constants),
        ("own images", inv.test_single_atom_self_images),
        ("supercell extensivity", inv.test_supercell_extensivity),
        ("invariances", inv.test_invariances),
        ("F = -dE/dx", inv.test_forces_are_minus_gradient),
        ("W = -dE/dstrain", inv.test_virial_is_minus_strain_derivative),
        ("dE/d(s6, s8, a1, a2)", inv.test_parameter_derivatives),
        ("three-body equilateral closed form", atm.test_equilateral_closed_form),
        ("three-body dipole-tensor form", atm.test_angular_factor_dipole_tensor),
        ("three-body F = -dE/dx", atm.test_forces_are_minus_gradient),
        ("per-atom virials sum to W (self-images)", lambda o: av.test_atom_virials_sum_to_total(o, "self_images")),
        ("per-atom virials sum to W (triclinic)", lambda o: av.test_atom_virials_sum_to_total(o, "triclinic")),
    ]


def run_battery(o, trimer_ref, stop_at_first):
    failed = []
    for name, pin in battery(trimer_ref):
        try:
            pin(o)
        except Exception as e:  # an assertion, or an error the planted mistake provokes
            failed.append((name, f"{type(e).__name__}: {str(e)[:160]}"))
            if stop_at_first:
                break
    return failed


def build_copy(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return oracle.compile_library(str(src), str(tmp_path / f"lib{name}.so"))


def test_unmodified_copy_passes_every_pin(oracle_mod, trimer, tmp_path):
    with open(oracle.source_path()) as f:
        lib = build_copy(tmp_path, "unmodified", f.read())
    with oracle.using_library(lib):
        assert run_battery(oracle_mod, trimer, stop_at_first=False) == []


@pytest.mark.parametrize("name,mistake,old,new,occurrences", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_mod, trimer, tmp_path, name, mistake, old, new, occurrences):
    with open(oracle.source_path()) as f:
        text = f.read()
    assert text.count(old) == occurrences, f"{name}: the mutated text no longer matches the oracle source"
    lib = build_copy(tmp_path, name, text.replace(old, new))
    with oracle.using_library(lib):
        failed = run_battery(oracle_mod, trimer, stop_at_first=True)
    assert failed, f"no pin catches: {mistake}"
