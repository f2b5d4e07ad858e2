/*
 * d3_oracle.c -- plain FP64 CPU oracle for the D3(BJ) "two-body" dispersion
 * correction of Ying & Fan, "Combining the D3 dispersion correction with the
 * neuroevolution machine-learned potential" (arXiv 2310.05279), Sec. II A,
 * Eqs. 1-7.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What it computes, in the paper's order, for one periodic (or open) structure:
 *
 *   1. every ordered pair instance (i, j, T): atom j shifted by the lattice
 *      translation T, distance r = |x_j + T - x_i| in bohr, excluding only
 *      (i, i, 0).  An atom's own periodic images are neighbours (Eqs. 2 and 4
 *      sum over "j != i", read as "every instance but the atom itself").
 *   2. Eq. 4: n_i = sum over instances with r < R_cn of
 *             1 / (1 + exp(-k1 * (k2 * (Rcov_i + Rcov_j) / r - 1)))
 *      (effective covalent radius = k2 * tabulated radius).
 *   3. Eq. 3: C6_ij(n_i, n_j) = sum_ab C6ref_ab L_ia L_jb / sum_ab L_ia L_jb with
 *      L_ia = exp(-k3 (n_i - nref_ia)^2).  The exponent is a sum of an i part and
 *      a j part, so the ratio equals sum_ab W_ia W_jb C6ref_ab with per-atom
 *      normalised weights W_ia = L_ia / sum_c L_ic.  Each atom's exponents are
 *      shifted by their maximum before exponentiating; this leaves Eq. 3
 *      unchanged wherever it is defined and gives its limit (all weight on the
 *      nearest reference) where every L_ia underflows.
 *   4. Eq. 2: E = -1/2 sum over ordered instances with r < R_pot of
 *             s6 C6 / (r^6 + R^6) + s8 C8 / (r^8 + R^8),
 *      R = a1 R0 + a2, R0^2 = 3 sqrtQ_i sqrtQ_j, C8 = C6 R0^2.
 *   5. Forces F = -dE/dx by the chain rule through r directly and through the
 *      coordination numbers (the dependence of U_i on n_j that makes D3
 *      many-body, Sec. II A after Eq. 4).
 *   6. Virial W = -sum over instances d (x) dE/dd, the sum of the per-atom
 *      virials of Eq. 7.
 *   7. Optionally (s9 != 0), the three-body term of the original D3 model, which
 *      the paper excludes; see atm_triangle.
 *
 * Units: positions and cells in Angstrom; a2, Rcov, sqrt(Q) in bohr; C6ref in
 * Ha*bohr^6; all formulae evaluated in bohr/Hartree; E in eV, F in eV/A, W in eV.
 * Cutoffs are hard: a term is included when r < cutoff.
 *
 * Every accumulation below is a plain loop in a fixed order; the only
 * parallel part is the instance search (OpenMP over i, each thread writing
 * its own rows), so results are deterministic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_BOHR_A 0.529177210903      /* Angstrom per bohr (CODATA 2018) */
#define ORACLE_HARTREE_EV 27.211386245988 /* eV per Hartree (CODATA 2018) */

typedef struct {
    double s6, s8, a1, a2_bohr; /* BJ damping of Eq. 2 */
    double k1, k2, k3;          /* Eq. 4 steepness, covalent-radius scale, Eq. 3 Gaussian width */
    double rc_disp_A, rc_cn_A;  /* R_pot and R_cn */
    double s9, alpha9, rc3_A;   /* optional three-body term (s9 = 0: off), see atm_triangle */
} oracle_params;

typedef struct {
    int ntypes, max_ref;
    const int32_t *nref;   /* [ntypes] */
    const double *cn_ref;  /* [ntypes][max_ref] */
    const double *c6_ref;  /* [ntypes][ntypes][max_ref][max_ref] */
    const double *rcov;    /* [ntypes], bohr */
    const double *sqrtq;   /* [ntypes], bohr */
} oracle_tables;

typedef struct {
    int64_t i, j;
    double d[3]; /* x_j + T - x_i, bohr */
    double r;
    int T[3];    /* lattice translation of j, in lattice vectors */
} instance;

/* ------------------------------------------------------------------ helpers */

static void inv3(const double *H, double *Hi) {
    double a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7], k = H[8];
    double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
    Hi[0] = (e * k - f * h) / det; Hi[1] = (c * h - b * k) / det; Hi[2] = (b * f - c * e) / det;
    Hi[3] = (f * g - d * k) / det; Hi[4] = (a * k - c * g) / det; Hi[5] = (c * d - a * f) / det;
    Hi[6] = (d * h - e * g) / det; Hi[7] = (b * g - a * h) / det; Hi[8] = (a * e - b * d) / det;
}

static double det3(const double *H) {
    return H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
           H[2] * (H[3] * H[7] - H[4] * H[6]);
}

/* Distance between the two lattice planes spanned by rows l and m of H. */
static double plane_width(const double *H, int k) {
    int l = (k + 1) % 3, m = (k + 2) % 3;
    const double *u = H + 3 * l, *v = H + 3 * m;
    double c0 = u[1] * v[2] - u[2] * v[1], c1 = u[2] * v[0] - u[0] * v[2], c2 = u[0] * v[1] - u[1] * v[0];
    return fabs(det3(H)) / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

/* Eq. 4 counting function and its derivative d/dr. */
static double cn_term(double r, double rc_eff, double k1) {
    return 1.0 / (1.0 + exp(-k1 * (rc_eff / r - 1.0)));
}
static double cn_term_dr(double r, double rc_eff, double k1) {
    double f = cn_term(r, rc_eff, k1);
    return -k1 * rc_eff / (r * r) * f * (1.0 - f);
}

/* Normalised Gaussian weights of Eq. 3 for one atom (max-shifted exponents)
 * and their derivatives with respect to the atom's coordination number. */
static void ref_weights(const oracle_tables *t, int ti, double n, double k3, double *W, double *dW) {
    int R = t->max_ref, nr = t->nref[ti];
    double ex[64], emax = -INFINITY, sum = 0.0;
    for (int a = 0; a < nr; ++a) {
        double z = n - t->cn_ref[ti * R + a];
        ex[a] = -k3 * z * z;
        if (ex[a] > emax) emax = ex[a];
    }
    for (int a = 0; a < R; ++a) W[a] = dW[a] = 0.0;
    for (int a = 0; a < nr; ++a) {
        W[a] = exp(ex[a] - emax);
        sum += W[a];
    }
    for (int a = 0; a < nr; ++a) W[a] /= sum;
    /* dW_a/dn = W_a * (g_a - sum_b W_b g_b), g_a = d(exponent_a)/dn = -2 k3 (n - nref_a) */
    double gbar = 0.0;
    for (int a = 0; a < nr; ++a) gbar += W[a] * (-2.0 * k3 * (n - t->cn_ref[ti * R + a]));
    for (int a = 0; a < nr; ++a) dW[a] = W[a] * (-2.0 * k3 * (n - t->cn_ref[ti * R + a]) - gbar);
}

/* C6 of one pair from the per-atom weights (Eq. 3) and its derivatives with
 * respect to the two atoms' coordination numbers. */
static double pair_c6(const oracle_tables *t, const double *Wt, const double *dWt, int64_t i, int ti, int64_t j,
                      int tj, double *dCi, double *dCj) {
    int R = t->max_ref;
    const double *cref = t->c6_ref + ((size_t)(ti * t->ntypes + tj) * R) * R;
    double C6 = 0.0, di = 0.0, dj = 0.0;
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            double c = cref[a * R + b];
            C6 += Wt[R * i + a] * Wt[R * j + b] * c;
            di += dWt[R * i + a] * Wt[R * j + b] * c;
            dj += Wt[R * i + a] * dWt[R * j + b] * c;
        }
    *dCi = di;
    *dCj = dj;
    return C6;
}

/* Damping radius R = a1 R0 + a2 of Eq. 2 for a type pair, and R0. */
static double damp_radius(const oracle_params *p, const oracle_tables *t, int ti, int tj, double *R0) {
    *R0 = sqrt(3.0 * t->sqrtq[ti] * t->sqrtq[tj]);
    return p->a1 * *R0 + p->a2_bohr;
}

/*
 * Optional three-body (Axilrod-Teller-Muto triple-dipole) term of the original
 * D3 model (Grimme et al., J. Chem. Phys. 132, 154104 (2010)).  The paper leaves
 * it out (Sec. II A); it is evaluated only when s9 != 0.  For a triangle of atoms
 * i, j, k with sides u = r_ij, v = r_ik, w = r_jk and interior angles A_i, A_j, A_k:
 *
 *   E = s9 sqrt(C6_ij C6_ik C6_jk) (3 cos A_i cos A_j cos A_k + 1) / (u v w)^3 * f,
 *   f = 1 / (1 + 6 q),   q = (Rbar / rbar)^alpha9,
 *
 * rbar = (u v w)^(1/3) and Rbar the geometric mean of the three damping radii
 * R = a1 R0 + a2 of Eq. 2 (the Becke-Johnson radii in the zero-damping form of
 * the three-body damping).  The cosines come from the law of cosines.
 *
 * Outputs the energy, dE/du, dE/dv, dE/dw, dE/dR for the three radii (in the
 * order ij, ik, jk; for the a1/a2 derivatives) given the three C6 values.
 */
static double atm_triangle(const oracle_params *p, double u, double v, double w, double C6ij, double C6ik,
                           double C6jk, double Rij, double Rik, double Rjk, double *dEdu, double *dEdv,
                           double *dEdw, double dEdR[3]) {
    double ci = (u * u + v * v - w * w) / (2.0 * u * v);
    double cj = (u * u + w * w - v * v) / (2.0 * u * w);
    double ck = (v * v + w * w - u * u) / (2.0 * v * w);
    /* partial derivatives of each cosine with respect to each side */
    double ci_u = 1.0 / (2.0 * v) - v / (2.0 * u * u) + w * w / (2.0 * u * u * v);
    double ci_v = 1.0 / (2.0 * u) - u / (2.0 * v * v) + w * w / (2.0 * u * v * v);
    double ci_w = -w / (u * v);
    double cj_u = 1.0 / (2.0 * w) - w / (2.0 * u * u) + v * v / (2.0 * u * u * w);
    double cj_w = 1.0 / (2.0 * u) - u / (2.0 * w * w) + v * v / (2.0 * u * w * w);
    double cj_v = -v / (u * w);
    double ck_v = 1.0 / (2.0 * w) - w / (2.0 * v * v) + u * u / (2.0 * v * v * w);
    double ck_w = 1.0 / (2.0 * v) - v / (2.0 * w * w) + u * u / (2.0 * v * w * w);
    double ck_u = -u / (v * w);
    double prod = u * v * w;
    double inv3 = 1.0 / (prod * prod * prod);
    double ang = 3.0 * ci * cj * ck + 1.0;
    double G = ang * inv3;
    double G_u = 3.0 * (ci_u * cj * ck + ci * cj_u * ck + ci * cj * ck_u) * inv3 - 3.0 * G / u;
    double G_v = 3.0 * (ci_v * cj * ck + ci * cj_v * ck + ci * cj * ck_v) * inv3 - 3.0 * G / v;
    double G_w = 3.0 * (ci_w * cj * ck + ci * cj_w * ck + ci * cj * ck_w) * inv3 - 3.0 * G / w;
    double Rbar = cbrt(Rij * Rik * Rjk), rbar = cbrt(prod);
    double q = pow(Rbar / rbar, p->alpha9);
    double f = 1.0 / (1.0 + 6.0 * q);
    /* dq/du = -(alpha/3) q / u, so df/du = 2 alpha q f^2 / u; dq/dR = (alpha/3) q / R */
    double fs = 2.0 * p->alpha9 * q * f * f;
    double c = p->s9 * sqrt(C6ij * C6ik * C6jk);
    *dEdu = c * (G_u * f + G * fs / u);
    *dEdv = c * (G_v * f + G * fs / v);
    *dEdw = c * (G_w * f + G * fs / w);
    dEdR[0] = -c * G * fs / Rij;
    dEdR[1] = -c * G * fs / Rik;
    dEdR[2] = -c * G * fs / Rjk;
    return c * G * f;
}

/* ------------------------------------------------------------------ instance search */

/* All ordered instances (i, j, T) with r < rc (bohr).  x holds wrapped positions
 * in bohr; m[k] is the image range along lattice vector k.  Brute force: every
 * atom pair and every translation in the range.  Each atom's instances are
 * collected in its own growable row, then the rows are concatenated in atom
 * order. */
static instance *find_instances(int64_t n, const double *x, const double *Hb, const int *m, double rc,
                                int64_t *count_out) {
    instance **rows = (instance **)calloc((size_t)(n > 0 ? n : 1), sizeof(instance *));
    int64_t *cnt = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0, cap = 64;
        instance *row = (instance *)malloc((size_t)cap * sizeof(instance));
        for (int64_t j = 0; j < n; ++j)
            for (int n0 = -m[0]; n0 <= m[0]; ++n0)
                for (int n1 = -m[1]; n1 <= m[1]; ++n1)
                    for (int n2 = -m[2]; n2 <= m[2]; ++n2) {
                        if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;
                        double d[3], d2 = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            double T = n0 * Hb[a] + n1 * Hb[3 + a] + n2 * Hb[6 + a];
                            d[a] = x[3 * j + a] + T - x[3 * i + a];
                            d2 += d[a] * d[a];
                        }
                        if (d2 < rc2) {
                            if (c == cap) {
                                cap *= 2;
                                row = (instance *)realloc(row, (size_t)cap * sizeof(instance));
                            }
                            instance *q = &row[c++];
                            q->i = i; q->j = j;
                            q->d[0] = d[0]; q->d[1] = d[1]; q->d[2] = d[2];
                            q->r = sqrt(d2);
                            q->T[0] = n0; q->T[1] = n1; q->T[2] = n2;
                        }
                    }
        rows[i] = row;
        cnt[i] = c;
    }
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += cnt[i];
    instance *out = (instance *)malloc((size_t)(total > 0 ? total : 1) * sizeof(instance));
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (cnt[i]) memcpy(out + o, rows[i], (size_t)cnt[i] * sizeof(instance));
        o += cnt[i];
        free(rows[i]);
    }
    free(rows);
    free(cnt);
    *count_out = total;
    return out;
}

/* ------------------------------------------------------------------ main entry */

/*
 * d3_oracle_compute: one structure.
 *   pos     [n][3] Angstrom          types [n] (0 <= t < ntypes)
 *   cell    [9] rows = lattice vectors, Angstrom     pbc [3]
 * Outputs (any may be NULL except E):
 *   E       total energy, eV
 *   F       [n][3] forces, eV/A
 *   W       [9] virial, eV (row-major 3x3)
 *   e_atom  [n] site energies U_i of Eq. 2, eV
 *   cn      [n] coordination numbers of Eq. 4
 *   dEdn    [n] dE/dn_i, eV
 *   dEdp    [4] dE/d(s6, s8, a1, a2) with a2 in bohr, eV (per unit parameter)
 * Returns 0 on success, negative on bad input.
 */
int d3_oracle_compute(const oracle_params *p, const oracle_tables *t, int64_t n, const double *pos,
                      const int32_t *types, const double *cell, const int32_t *pbc, double *E, double *F,
                      double *W, double *e_atom, double *cn, double *dEdn_out, double *dEdp) {
    if (n < 0 || !p || !t || !E) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= t->ntypes) return -2;
    const int R = t->max_ref;
    const double rcd = p->rc_disp_A / ORACLE_BOHR_A, rcn = p->rc_cn_A / ORACLE_BOHR_A;
    const int atm = p->s9 != 0.0;
    const double rc3 = atm ? p->rc3_A / ORACLE_BOHR_A : 0.0;
    double rmax = rcd > rcn ? rcd : rcn;
    if (rc3 > rmax) rmax = rc3;

    /* lattice in bohr, wrapped positions in bohr */
    double Hb[9], Hi[9];
    for (int k = 0; k < 9; ++k) Hb[k] = cell[k] / ORACLE_BOHR_A;
    if (fabs(det3(Hb)) < 1e-12) return -3;
    inv3(Hb, Hi);
    double *x = (double *)malloc((size_t)(3 * (n > 0 ? n : 1)) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        double xb[3] = {pos[3 * i] / ORACLE_BOHR_A, pos[3 * i + 1] / ORACLE_BOHR_A, pos[3 * i + 2] / ORACLE_BOHR_A};
        double f[3];
        for (int k = 0; k < 3; ++k) f[k] = xb[0] * Hi[k] + xb[1] * Hi[3 + k] + xb[2] * Hi[6 + k];
        for (int k = 0; k < 3; ++k)
            if (pbc[k]) {
                f[k] -= floor(f[k]);
                if (f[k] >= 1.0) f[k] -= 1.0; /* keep [0, 1) when the subtraction rounds up */
            }
        for (int a = 0; a < 3; ++a) x[3 * i + a] = f[0] * Hb[a] + f[1] * Hb[3 + a] + f[2] * Hb[6 + a];
    }
    /* translations needed: with wrapped fractional coordinates in [0,1) the
     * fractional separation along k is below 1, and an instance closer than
     * rmax has |dfrac_k + n_k| <= rmax / width_k, so |n_k| <= ceil(rmax / width_k) */
    int m[3];
    for (int k = 0; k < 3; ++k) m[k] = pbc[k] ? (int)ceil(rmax / plane_width(Hb, k)) : 0;

    int64_t ni = 0;
    instance *I = find_instances(n, x, Hb, m, rmax, &ni);

    /* Eq. 4: coordination numbers */
    double *nc = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t q = 0; q < ni; ++q) {
        const instance *s = &I[q];
        if (s->r < rcn) {
            double rc_eff = p->k2 * (t->rcov[types[s->i]] + t->rcov[types[s->j]]);
            nc[s->i] += cn_term(s->r, rc_eff, p->k1);
        }
    }

    /* Eq. 3: per-atom reference weights */
    double *Wt = (double *)calloc((size_t)(R * (n > 0 ? n : 1)), sizeof(double));
    double *dWt = (double *)calloc((size_t)(R * (n > 0 ? n : 1)), sizeof(double));
    for (int64_t i = 0; i < n; ++i) ref_weights(t, types[i], nc[i], p->k3, Wt + R * i, dWt + R * i);

    /* Eq. 2: energy, dE/dn, direct forces and virial, and the parameter derivatives */
    double Etot = 0.0, dp[4] = {0, 0, 0, 0}, Wv[9] = {0};
    double *eat = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *dEdn = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *Fb = (double *)calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
    for (int64_t q = 0; q < ni; ++q) {
        const instance *s = &I[q];
        if (!(s->r < rcd)) continue;
        int ti = types[s->i], tj = types[s->j];
        const double *cref = t->c6_ref + ((size_t)(ti * t->ntypes + tj) * R) * R;
        double C6 = 0.0, dC6i = 0.0, dC6j = 0.0;
        for (int a = 0; a < R; ++a)
            for (int b = 0; b < R; ++b) {
                double c = cref[a * R + b];
                C6 += Wt[R * s->i + a] * Wt[R * s->j + b] * c;
                dC6i += dWt[R * s->i + a] * Wt[R * s->j + b] * c;
                dC6j += Wt[R * s->i + a] * dWt[R * s->j + b] * c;
            }
        double R0sq = 3.0 * t->sqrtq[ti] * t->sqrtq[tj];
        double R0 = sqrt(R0sq);
        double Rd = p->a1 * R0 + p->a2_bohr;
        double C8 = C6 * R0sq;
        double r = s->r, r2 = r * r, r6 = r2 * r2 * r2, r8 = r6 * r2;
        double R6 = pow(Rd, 6.0), R8 = pow(Rd, 8.0);
        double d6 = r6 + R6, d8 = r8 + R8;
        /* this ordered instance carries half of the pair energy */
        double e = -0.5 * (p->s6 * C6 / d6 + p->s8 * C8 / d8);
        Etot += e;
        eat[s->i] += e;
        /* de/dC6 (C8 follows C6) */
        double de_dC6 = -0.5 * (p->s6 / d6 + p->s8 * R0sq / d8);
        dEdn[s->i] += de_dC6 * dC6i;
        dEdn[s->j] += de_dC6 * dC6j;
        /* de/dr */
        double de_dr = 0.5 * (p->s6 * C6 * 6.0 * r * r2 * r2 / (d6 * d6) + p->s8 * C8 * 8.0 * r6 * r / (d8 * d8));
        for (int a = 0; a < 3; ++a) {
            double g = de_dr * s->d[a] / r; /* de/dd_a; dd/dx_i = -1, dd/dx_j = +1 */
            Fb[3 * s->i + a] += g;
            Fb[3 * s->j + a] -= g;
            for (int b = 0; b < 3; ++b) Wv[3 * a + b] -= s->d[a] * de_dr * s->d[b] / r;
        }
        /* parameter derivatives of this half pair energy */
        dp[0] += -0.5 * C6 / d6;
        dp[1] += -0.5 * C8 / d8;
        double de_dR = 0.5 * (p->s6 * C6 * 6.0 * pow(Rd, 5.0) / (d6 * d6) + p->s8 * C8 * 8.0 * pow(Rd, 7.0) / (d8 * d8));
        dp[2] += de_dR * R0;
        dp[3] += de_dR;
    }
    /* optional three-body term: every triangle whose three sides are below rc3.
     * Atom i's instances are contiguous in I; each unordered pair of them (j, k)
     * with |d_k - d_j| < rc3 is one triangle seen from vertex i.  Every triangle
     * is seen once from each of its three vertices, so each sighting carries a
     * third of the energy and of every derivative, the derivatives taken with
     * respect to all three atoms. */
    if (atm) {
        int64_t *start = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
        for (int64_t q = 0; q < ni; ++q) start[I[q].i + 1]++;
        for (int64_t i = 0; i < n; ++i) start[i + 1] += start[i];
        const double third = 1.0 / 3.0;
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t qa = start[i]; qa < start[i + 1]; ++qa) {
                const instance *A = &I[qa];
                if (!(A->r < rc3)) continue;
                for (int64_t qb = qa + 1; qb < start[i + 1]; ++qb) {
                    const instance *Bq = &I[qb];
                    if (!(Bq->r < rc3)) continue;
                    double djk[3] = {Bq->d[0] - A->d[0], Bq->d[1] - A->d[1], Bq->d[2] - A->d[2]};
                    double w = sqrt(djk[0] * djk[0] + djk[1] * djk[1] + djk[2] * djk[2]);
                    if (!(w < rc3)) continue;
                    int64_t j = A->j, k = Bq->j;
                    int ti = types[i], tj = types[j], tk = types[k];
                    double dij_i, dij_j, dik_i, dik_k, djk_j, djk_k;
                    double C6ij = pair_c6(t, Wt, dWt, i, ti, j, tj, &dij_i, &dij_j);
                    double C6ik = pair_c6(t, Wt, dWt, i, ti, k, tk, &dik_i, &dik_k);
                    double C6jk = pair_c6(t, Wt, dWt, j, tj, k, tk, &djk_j, &djk_k);
                    double R0ij, R0ik, R0jk;
                    double Rij = damp_radius(p, t, ti, tj, &R0ij), Rik = damp_radius(p, t, ti, tk, &R0ik),
                           Rjk = damp_radius(p, t, tj, tk, &R0jk);
                    double Eu, Ev, Ew, ER[3];
                    double e = atm_triangle(p, A->r, Bq->r, w, C6ij, C6ik, C6jk, Rij, Rik, Rjk, &Eu, &Ev, &Ew, ER);
                    Etot += third * e;
                    eat[i] += third * e;
                    /* dE/dC6 = E / (2 C6) for each of the three pairs */
                    dEdn[i] += third * 0.5 * e * (dij_i / C6ij + dik_i / C6ik);
                    dEdn[j] += third * 0.5 * e * (dij_j / C6ij + djk_j / C6jk);
                    dEdn[k] += third * 0.5 * e * (dik_k / C6ik + djk_k / C6jk);
                    /* edge vectors d and dE/dd: ij = A->d, ik = Bq->d, jk = djk */
                    const double *dv[3] = {A->d, Bq->d, djk};
                    const double len[3] = {A->r, Bq->r, w}, dl[3] = {Eu, Ev, Ew};
                    const int64_t from[3] = {i, i, j}, to[3] = {j, k, k};
                    for (int ed = 0; ed < 3; ++ed)
                        for (int a = 0; a < 3; ++a) {
                            double g = third * dl[ed] * dv[ed][a] / len[ed];
                            Fb[3 * from[ed] + a] += g;
                            Fb[3 * to[ed] + a] -= g;
                            for (int b = 0; b < 3; ++b) Wv[3 * a + b] -= dv[ed][a] * third * dl[ed] * dv[ed][b] / len[ed];
                        }
                    /* dR/da1 = R0, dR/da2 = 1 */
                    dp[2] += third * (ER[0] * R0ij + ER[1] * R0ik + ER[2] * R0jk);
                    dp[3] += third * (ER[0] + ER[1] + ER[2]);
                }
            }
        }
        free(start);
    }
    /* chain rule through the coordination numbers (Eq. 4 inside Eq. 3) */
    for (int64_t q = 0; q < ni; ++q) {
        const instance *s = &I[q];
        if (!(s->r < rcn)) continue;
        double rc_eff = p->k2 * (t->rcov[types[s->i]] + t->rcov[types[s->j]]);
        double g_r = dEdn[s->i] * cn_term_dr(s->r, rc_eff, p->k1); /* d(E via n_i)/dr */
        for (int a = 0; a < 3; ++a) {
            double g = g_r * s->d[a] / s->r;
            Fb[3 * s->i + a] += g;
            Fb[3 * s->j + a] -= g;
            for (int b = 0; b < 3; ++b) Wv[3 * a + b] -= s->d[a] * g_r * s->d[b] / s->r;
        }
    }

    const double eV = ORACLE_HARTREE_EV, eV_A = ORACLE_HARTREE_EV / ORACLE_BOHR_A;
    *E = Etot * eV;
    if (F)
        for (int64_t i = 0; i < 3 * n; ++i) F[i] = Fb[i] * eV_A;
    if (W)
        for (int k = 0; k < 9; ++k) W[k] = Wv[k] * eV;
    if (e_atom)
        for (int64_t i = 0; i < n; ++i) e_atom[i] = eat[i] * eV;
    if (cn)
        for (int64_t i = 0; i < n; ++i) cn[i] = nc[i];
    if (dEdn_out)
        for (int64_t i = 0; i < n; ++i) dEdn_out[i] = dEdn[i] * eV;
    if (dEdp)
        for (int k = 0; k < 4; ++k) dEdp[k] = dp[k] * eV;

    free(x); free(I); free(nc); free(Wt); free(dWt); free(eat); free(dEdn); free(Fb);
    return 0;
}

/* ------------------------------------------------------------------ per-atom virial (Eq. 7) */

/*
 * d3_oracle_atom_virial: the per-atom virial of Eq. 7,
 *     W_i = sum_{j != i} r_ij (x) dU_j/dr_ji,   r_ij = x_j - x_i,
 * for every atom of one structure, with the site energy U_j of Eq. 2 written as
 * a function of the vectors from atom j (the representation the general
 * many-body formulation behind Eqs. 5-7 uses).  U_j depends on r_ji
 *   (1) directly, through its pair term with i (r < R_pot);
 *   (2) through n_j, whose term f(r_ji) is in Eq. 4 (r < R_cn);
 *   (3a) through n_i when i is a dispersion partner of j: every term of n_i is
 *        f(|r_jc - r_ji|), so dn_i/dr_ji = -sum_c f'(r_ic) r_ic/r_ic;
 *   (3b) through n_b of every other dispersion partner b of j that has i as a
 *        CN neighbour: the term f(|r_ji - r_jb|) of n_b.
 * Each term is taken per ordered instance (periodic images included) and
 * added to W of the instance's real atom.  w_atom [n][9] in eV, row-major
 * (row = component of r_ij, column = component of dU_j/dr_ji).
 */
int d3_oracle_atom_virial(const oracle_params *p, const oracle_tables *t, int64_t n, const double *pos,
                          const int32_t *types, const double *cell, const int32_t *pbc, double *w_atom) {
    if (n < 0 || !p || !t || !w_atom) return -1;
    if (p->s9 != 0.0) return -4; /* Eq. 7 is defined for the two-body site energies only */
    for (int64_t i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= t->ntypes) return -2;
    const int R = t->max_ref;
    const double rcd = p->rc_disp_A / ORACLE_BOHR_A, rcn = p->rc_cn_A / ORACLE_BOHR_A;
    const double rmax = rcd > rcn ? rcd : rcn;
    double Hb[9], Hi[9];
    for (int k = 0; k < 9; ++k) Hb[k] = cell[k] / ORACLE_BOHR_A;
    if (fabs(det3(Hb)) < 1e-12) return -3;
    inv3(Hb, Hi);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    double *x = (double *)malloc(3 * nn * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        double xb[3] = {pos[3 * i] / ORACLE_BOHR_A, pos[3 * i + 1] / ORACLE_BOHR_A, pos[3 * i + 2] / ORACLE_BOHR_A};
        double f[3];
        for (int k = 0; k < 3; ++k) f[k] = xb[0] * Hi[k] + xb[1] * Hi[3 + k] + xb[2] * Hi[6 + k];
        for (int k = 0; k < 3; ++k)
            if (pbc[k]) {
                f[k] -= floor(f[k]);
                if (f[k] >= 1.0) f[k] -= 1.0;
            }
        for (int a = 0; a < 3; ++a) x[3 * i + a] = f[0] * Hb[a] + f[1] * Hb[3 + a] + f[2] * Hb[6 + a];
    }
    int m[3];
    for (int k = 0; k < 3; ++k) m[k] = pbc[k] ? (int)ceil(rmax / plane_width(Hb, k)) : 0;
    int64_t ni = 0;
    instance *I = find_instances(n, x, Hb, m, rmax, &ni);
    /* first instance of every atom's row */
    int64_t *row = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    for (int64_t q = 0; q < ni; ++q) row[I[q].i + 1]++;
    for (int64_t i = 0; i < n; ++i) row[i + 1] += row[i];

    /* Eq. 4 and Eq. 3 */
    double *nc = (double *)calloc(nn, sizeof(double));
    for (int64_t q = 0; q < ni; ++q)
        if (I[q].r < rcn) nc[I[q].i] += cn_term(I[q].r, p->k2 * (t->rcov[types[I[q].i]] + t->rcov[types[I[q].j]]), p->k1);
    double *Wt = (double *)calloc((size_t)R * nn, sizeof(double));
    double *dWt = (double *)calloc((size_t)R * nn, sizeof(double));
    for (int64_t i = 0; i < n; ++i) ref_weights(t, types[i], nc[i], p->k3, Wt + R * i, dWt + R * i);

    /* per dispersion instance (j -> b): dU_j/dr of the pair term and
     * B = dU_j/dn_b; per atom: A_j = dU_j/dn_j */
    double *Bq = (double *)calloc((size_t)(ni > 0 ? ni : 1), sizeof(double));
    double *dUdr = (double *)calloc((size_t)(ni > 0 ? ni : 1), sizeof(double));
    double *A = (double *)calloc(nn, sizeof(double));
    for (int64_t q = 0; q < ni; ++q) {
        const instance *s = &I[q];
        if (!(s->r < rcd)) continue;
        int tj = types[s->i], tb = types[s->j];
        const double *cref = t->c6_ref + ((size_t)(tj * t->ntypes + tb) * R) * R;
        double C6 = 0.0, dC6own = 0.0, dC6partner = 0.0;
        for (int a = 0; a < R; ++a)
            for (int b = 0; b < R; ++b) {
                double c = cref[a * R + b];
                C6 += Wt[R * s->i + a] * Wt[R * s->j + b] * c;
                dC6own += dWt[R * s->i + a] * Wt[R * s->j + b] * c;
                dC6partner += Wt[R * s->i + a] * dWt[R * s->j + b] * c;
            }
        double R0sq = 3.0 * t->sqrtq[tj] * t->sqrtq[tb];
        double Rd = p->a1 * sqrt(R0sq) + p->a2_bohr;
        double C8 = C6 * R0sq;
        double r = s->r, r2 = r * r, r6 = r2 * r2 * r2, r8 = r6 * r2;
        double d6 = r6 + pow(Rd, 6.0), d8 = r8 + pow(Rd, 8.0);
        /* U_j contains -1/2 (s6 C6 / d6 + s8 C8 / d8) for this instance */
        double dU_dC6 = -0.5 * (p->s6 / d6 + p->s8 * R0sq / d8);
        A[s->i] += dU_dC6 * dC6own;
        Bq[q] = dU_dC6 * dC6partner;
        dUdr[q] = 0.5 * (p->s6 * C6 * 6.0 * r * r2 * r2 / (d6 * d6) + p->s8 * C8 * 8.0 * r6 * r / (d8 * d8));
    }
    /* G_i = sum over CN instances of i of f'(r) r_ic / r */
    double *G = (double *)calloc(3 * nn, sizeof(double));
    for (int64_t q = 0; q < ni; ++q) {
        const instance *s = &I[q];
        if (!(s->r < rcn)) continue;
        double fp = cn_term_dr(s->r, p->k2 * (t->rcov[types[s->i]] + t->rcov[types[s->j]]), p->k1);
        for (int a = 0; a < 3; ++a) G[3 * s->i + a] += fp * s->d[a] / s->r;
    }
    double *Wa = (double *)calloc(9 * nn, sizeof(double));
    /* (1), (2), (3a): instance j -> i with vector d = r_ji; r_ij = -d */
    for (int64_t q = 0; q < ni; ++q) {
        const instance *s = &I[q];
        int64_t j = s->i, i = s->j;
        double g[3] = {0.0, 0.0, 0.0}; /* dU_j/dr_ji */
        if (s->r < rcd)
            for (int a = 0; a < 3; ++a) g[a] += dUdr[q] * s->d[a] / s->r - Bq[q] * G[3 * i + a];
        if (s->r < rcn) {
            double fp = cn_term_dr(s->r, p->k2 * (t->rcov[types[j]] + t->rcov[types[i]]), p->k1);
            for (int a = 0; a < 3; ++a) g[a] += A[j] * fp * s->d[a] / s->r;
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Wa[9 * i + 3 * a + b] += -s->d[a] * g[b];
    }
    /* (3b): j -> b (dispersion), b -> c (CN), c an instance other than j itself */
    for (int64_t q1 = 0; q1 < ni; ++q1) {
        const instance *s1 = &I[q1];
        if (!(s1->r < rcd)) continue;
        int64_t j = s1->i, b = s1->j;
        for (int64_t q2 = row[b]; q2 < row[b + 1]; ++q2) {
            const instance *s2 = &I[q2];
            if (!(s2->r < rcn)) continue;
            int64_t c = s2->j;
            if (c == j && s1->T[0] + s2->T[0] == 0 && s1->T[1] + s2->T[1] == 0 && s1->T[2] + s2->T[2] == 0)
                continue; /* the term of n_b from atom j itself depends on r_jb only: it is part of (3a) */
            double fp = cn_term_dr(s2->r, p->k2 * (t->rcov[types[b]] + t->rcov[types[c]]), p->k1);
            for (int a = 0; a < 3; ++a) {
                double rij = -(s1->d[a] + s2->d[a]); /* vector from c's instance to j */
                for (int bb = 0; bb < 3; ++bb) Wa[9 * c + 3 * a + bb] += rij * Bq[q1] * fp * s2->d[bb] / s2->r;
            }
        }
    }
    for (int64_t k = 0; k < 9 * n; ++k) w_atom[k] = Wa[k] * ORACLE_HARTREE_EV;
    free(x); free(I); free(row); free(nc); free(Wt); free(dWt); free(Bq); free(dUdr); free(A); free(G); free(Wa);
    return 0;
}

/* Eq. 3 weights for one atom, exposed for unit checks. */
void d3_oracle_weights(const oracle_tables *t, int ti, double n, double k3, double *W, double *dW) {
    ref_weights(t, ti, n, k3, W, dW);
}

int d3_oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
