// d3gb_passes.cu -- per-step passes of the D3(BJ) pipeline (arXiv 2310.05279,
// Sec. II A), evaluated with full per-atom neighbour lists: the thread of atom i
// visits every ordered pair instance (i, j) and writes only atom i's results,
// so no pass needs atomics and every sum has a fixed order.
//
//   k_cn       Eq. 4  n_i = sum_j 1/(1 + exp(-k1 (k2 (Rcov_i + Rcov_j)/r - 1)))
//              and Eq. 3 per atom at the end of the same thread: normalised
//                     Gaussian weights W_ia, dW_ia/dn_i and the projections
//                     v_i^(t)_a = sum_b C6ref[t][t_i][a][b] W_ib, so that
//                     C6_ij = sum_a W_ia v_j^(t_i)_a
//   k_disp     Eq. 2  site energy, direct forces, virial and
//                     dE/dn_i = sum_j (dE/dC6_ij)(dC6_ij/dn_i) (FP64 form and per-atom
//                     virial; the mixed form's dispersion pass runs over cluster half
//                     lists, d3gb_cluster.cu)
//   k_atm             optional three-body term (not part of the paper's model;
//                     d3gb_atm.cu), between the dispersion and chain passes
//   k_chain           forces and virial of the coordination-number dependence:
//                     F_i += sum_j (dE/dn_i + dE/dn_j) f'(r_ij) r_ij/r
//   k_fin_*           per-structure energy and virial (fixed-order sums)
//
// MIXED = true: pair arithmetic in FP32 on split (hi + lo) positions, partial
// sums of kChunk pairs added into compensated float pairs (dispersion pass) or
// FP64 sums (chain pass); cutoff tests that fall within the FP32 error band of
// the cutoff are decided in FP64, so the set of pairs is the FP64 one.
// MIXED = false: FP64 throughout.
#include "d3gb_pair.cuh"

namespace d3gb {

namespace {

// Running sums of the dispersion pass: a compensated float pair in the mixed
// form (FP64 runs at 1/64 of the FP32 rate on GB300, and FP64 chunk sums cost
// the pass about 5%), FP64 in the FP64 form.
template <bool MIXED> struct PassAcc;
template <> struct PassAcc<true> {
    float h = 0.f, l = 0.f;
    __device__ void add(float x) { acc_add(h, l, x); }
    __device__ double value() const { return (double)h + (double)l; }
    __device__ float total() const { return h + l; }
};
template <> struct PassAcc<false> {
    double h = 0.0;
    __device__ void add(double x) { h += x; }
    __device__ double value() const { return h; }
    __device__ double total() const { return h; }
};

// Eq. 4 counting function f(r) and, optionally, df/dr, in FP64; r from 1/r.
// (The mixed form evaluates it in double-single, cn_ds below.)
__device__ __forceinline__ void cn_fun(double rinv, double rc_eff, double, double k1, double& f, double* dfdr) {
    const double t = exp(-k1 * (rc_eff * rinv - 1.0));
    f = 1.0 / (1.0 + t);
    if (dfdr) *dfdr = -k1 * rc_eff * rinv * rinv * t * f * f;
}
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float recip(float x) { return rcp_approx(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// ------------------------------------------------------------------ Eq. 3
// Per atom, right after its coordination number (fused into the CN pass): the
// exponents -k3 (n - nref_a)^2 minus their maximum are formed in FP64 (their
// absolute error sets the relative error of the weights), and exp(y) is taken
// as exp(y_hi) (1 + y_lo).  dW_a/dn is written as
// -2 k3 W_a sum_b W_b (nref_b - nref_a), which has no cancellation against n.
// Rows are padded to RP (4 or 8) and stored 4 values at a time.
template <class T>
__device__ __forceinline__ void store_row(T* dst, const T (&v)[8], int rp) {
    using T4 = typename Real<sizeof(T) == 4>::T4;
    T4* d = reinterpret_cast<T4*>(dst);
    d[0] = T4{v[0], v[1], v[2], v[3]};
    if (rp > 4) d[1] = T4{v[4], v[5], v[6], v[7]};
}

// W and dW/dn rows of atom p and its projections v_p^(u)_a = sum_b C6ref[u][t][a][b] W_b
// (and, for the cluster-list dispersion pass, the same rows next to
// dv_p^(u)_a = sum_b C6ref[u][t][a][b] dW_b in w.vd)
template <class T, int R>
__device__ __forceinline__ void store_weights(const Work& w, const Consts& c, const T* __restrict__ c6, int64_t p, int t,
                                              const T (&L)[R], const T (&Wr)[8], const T (&dWr)[8]) {
    store_row<T>((T*)w.W + p * c.RP, Wr, c.RP);
    store_row<T>((T*)w.dW + p * c.RP, dWr, c.RP);
    T* vp = (T*)w.v + p * c.T * c.RP;
    T* dvp = (sizeof(T) == 4 && w.vd) ? (T*)w.vd + p * c.T * 2 * c.RP : nullptr;  // [T][2][RP] per atom
    for (int u = 0; u < c.T; ++u) {
        const T* cu = c6 + ((size_t)(u * c.T + t) * R) * R;  // C6ref[u][t][a][b]
        T vr[8], dvr[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            T s = 0, ds = 0;
            if (a < R) {
#pragma unroll
                for (int b = 0; b < R; ++b) {
                    s += cu[a * R + b] * L[b];
                    ds += cu[a * R + b] * dWr[b];
                }
            }
            vr[a] = s;
            dvr[a] = ds;
        }
        store_row<T>(vp + u * c.RP, vr, c.RP);
        if (dvp) {
            store_row<T>(dvp + 2 * u * c.RP, vr, c.RP);
            store_row<T>(dvp + (2 * u + 1) * c.RP, dvr, c.RP);
        }
    }
    if (p == 0 && w.npairs) *w.npairs = 0ull;  // pair count of this call's dispersion pass
    if (w.acc) {  // clear the atom's fixed-point sums of the cluster-list dispersion pass
        ulonglong2* a = reinterpret_cast<ulonglong2*>(w.acc + 8 * p);
        const ulonglong2 z = make_ulonglong2(0ull, 0ull);
        a[0] = z; a[1] = z; a[2] = z; a[3] = z;
    }
}

template <bool MIXED, int R>
__device__ __forceinline__ void weights_atom(const Work& w, const Consts& c, const double* __restrict__ cnref,
                                             const int* __restrict__ nref,
                                             const typename Real<MIXED>::T* __restrict__ c6, int64_t p, int t,
                                             double n) {
    using T = typename Real<MIXED>::T;
    const int nr = nref[t];
    double cr[R], x[R];
    double xmax = -1e300;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        cr[a] = cnref[t * R + a];
        const double z = n - cr[a];
        x[a] = -c.k3 * z * z;
        if (a < nr && x[a] > xmax) xmax = x[a];
    }
    T L[R];
    T sum = 0;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        if (a < nr) {
            const double y = x[a] - xmax;
            if constexpr (MIXED) {
                const float yh = (float)y, yl = (float)(y - (double)yh);
                L[a] = expf(yh) * (1.0f + yl);
            } else {
                L[a] = exp(y);
            }
        } else {
            L[a] = 0;
        }
        sum += L[a];
    }
    const T inv = (T)1 / sum;
#pragma unroll
    for (int a = 0; a < R; ++a) L[a] *= inv;
    T Wr[8], dWr[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        if (a < R) {
            T s = 0;
#pragma unroll
            for (int b = 0; b < R; ++b) s += L[b] * (T)(cr[b] - cr[a]);
            Wr[a] = L[a];
            dWr[a] = -2 * (T)c.k3 * L[a] * s;
        } else {
            Wr[a] = dWr[a] = 0;
        }
    }
    store_weights<T, R>(w, c, c6, p, t, L, Wr, dWr);
}

// Mixed form of the above without FP64 (GB300 runs FP64 at 1/64 of the FP32
// rate): the exponents -k3 (n - nref_a)^2 are formed in float-float from
// n = Nh + Nl, nref_a = cnref2[t][a].x + .y and k3 = k3h + k3l, about 44
// significant bits, so their absolute error stays far below the FP32 rounding
// of exp itself; the differences nref_b - nref_a come from a host table
// (dcr[t][a][b], rounded once).
template <int R>
__device__ __forceinline__ void weights_atom_mixed(const Work& w, const Consts& c, const float2* __restrict__ cnref2,
                                                   const float* __restrict__ dcr, const int* __restrict__ nref,
                                                   const float* __restrict__ c6, int64_t p, int t, float Nh,
                                                   float Nl) {
    const int nr = nref[t];
    float xh[R], xl[R];
    float mh = -3.0e38f, ml = 0.0f;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const float2 cr = cnref2[t * R + a];
        float zh, ze, zl;
        two_sum(Nh, -cr.x, zh, ze);
        two_sum(zh, ze + (Nl - cr.y), zh, zl);  // z = n - nref_a
        const float ph = zh * zh, pl = fmaf(zh, zh, -ph) + 2.0f * zh * zl;
        xh[a] = -c.k3h * ph;
        xl[a] = fmaf(-c.k3h, ph, -xh[a]) - c.k3h * pl - c.k3l * ph;
        if (a < nr && (xh[a] > mh || (xh[a] == mh && xl[a] > ml))) {
            mh = xh[a];
            ml = xl[a];
        }
    }
    float L[R];
    float sum = 0.0f;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        L[a] = 0.0f;
        if (a < nr) {
            float yh, ye, yl;
            two_sum(xh[a], -mh, yh, ye);
            two_sum(yh, ye + (xl[a] - ml), yh, yl);
            L[a] = expf(yh) * (1.0f + yl);
        }
        sum += L[a];
    }
    const float inv = 1.0f / sum;
#pragma unroll
    for (int a = 0; a < R; ++a) L[a] *= inv;
    float Wr[8], dWr[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        if (a < R) {
            float s = 0.0f;
            const float* dr = dcr + (t * R + a) * R;
#pragma unroll
            for (int b = 0; b < R; ++b) s += L[b] * dr[b];
            Wr[a] = L[a];
            dWr[a] = -2.0f * c.k3f * L[a] * s;
        } else {
            Wr[a] = dWr[a] = 0.0f;
        }
    }
    store_weights<float, R>(w, c, c6, p, t, L, Wr, dWr);
}

// ------------------------------------------------------------------ Eq. 4
// The coordination numbers feed dC6/dn, which can be large, so the mixed form
// keeps n_i accurate to a few 1e-8: the pair vector is exact (D + e), r^2 and
// r are formed in double-single, the argument k1 (rc/r - 1) is evaluated as
// k1 (rc - r) / r from the double-single difference rc - r, and the sum over
// neighbours is compensated.  The mixed form also stores, per list entry, the
// chain-rule coefficient f'(r)/r of the pair (0 outside R_cn), which depends on
// the geometry only: the chain pass reads it instead of forming the
// double-single Eq. 4 term a second time; and, when image atoms have rows of
// their own, it writes the copies of the atom's v/dv rows for its images.
template <bool MIXED, int R>
__global__ void __launch_bounds__(128) k_cn(Work w, Consts c, const float4* __restrict__ rcpair,
                                           const float2* __restrict__ exptab, const double* __restrict__ cnref,
                                           const float2* __restrict__ cnref2, const float* __restrict__ dcr,
                                           const int* __restrict__ nref,
                                           const typename Real<MIXED>::T* __restrict__ c6) {
    using T = typename Real<MIXED>::T;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const Site<MIXED> S(w, p);
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const T rc2 = MIXED ? (T)c.rc_cn2f : (T)c.rc_cn2, k1 = MIXED ? (T)c.k1f : (T)c.k1;
    T nh = 0, nl = 0;
    if constexpr (MIXED) {
        const float4* rrow = rcpair + (S.tsrc() & 15) * c.T;
        int nint = 0;  // terms with f > 1/2 are summed as 1 - t/(1 + t): exact integer part plus a small complement
        const int* row = LV.p;
        float* grow = w.gcn + (row - w.nbr_cn);
        auto term = [&](int q, const float4* rec_q) -> float {  // the pair's CN term; returns f'(r)/r (0 outside R_cn)
            float D[3], r2, ah, al, rch, rcl, r2l, y;
            int tq;
            if (!cn_pair_precise(S, q, rrow, k1, rc2, c.rc_cn2, D, r2, ah, al, rch, tq, &rcl, &r2l, &y, rec_q))
                return 0.0f;
            const CnDS z = cn_ds(ah, al, exptab);
            if (z.th < 1.0f) {
                ++nint;
                acc_add(nh, nl, -z.ch);
                nl -= z.cl;
            } else {
                acc_add(nh, nl, z.fh);
                nl += z.fl;
            }
            return chain_coef(z, y, r2, r2l, rch, rcl, k1);
        };
        for (int k = 0; k < cnt; k += 4) {
            // the four entries' records are loaded before any of their arithmetic (entries past
            // the end of the list read atom p's own record, unused)
            const int4 q4 = __ldg(reinterpret_cast<const int4*>(row + list_off(k)));
            const int qq[4] = {q4.x, k + 1 < cnt ? q4.y : (int)p, k + 2 < cnt ? q4.z : (int)p,
                               k + 3 < cnt ? q4.w : (int)p};
            float4 rq[4][2];
#pragma unroll
            for (int e = 0; e < 4; ++e) rec_load(w, qq[e], rq[e][0], rq[e][1]);
            float4 g4;
            g4.x = term(qq[0], rq[0]);
            g4.y = k + 1 < cnt ? term(qq[1], rq[1]) : 0.0f;
            g4.z = k + 2 < cnt ? term(qq[2], rq[2]) : 0.0f;
            g4.w = k + 3 < cnt ? term(qq[3], rq[3]) : 0.0f;
            *reinterpret_cast<float4*>(grow + list_off(k)) = g4;
        }
        float Nh, Nl;  // n = nint + nh + nl as a float pair
        two_sum((float)nint, nh, Nh, Nl);
        Nl += nl;
        w.cn[p] = (double)Nh + (double)Nl;
        weights_atom_mixed<R>(w, c, cnref2, dcr, nref, (const float*)c6, p, S.tsrc() & 15, Nh, Nl);
        if (w.vd_images) {  // copies of the atom's v/dv rows for its image atoms (read back from this thread's writes)
            const int rows4 = c.T * 2 * c.RP / 4;
            const int i = w.perm[p];
            const int g0 = w.gfirst[i], ng = w.gcnt[i];
            const float4* from = reinterpret_cast<const float4*>(w.vd) + p * rows4;
            for (int k = 0; k < ng && g0 + k < w.ghost_cap; ++k) {
                float4* to = reinterpret_cast<float4*>(w.vd) + (w.Nr + w.ginv[g0 + k]) * (int64_t)rows4;
                for (int m = 0; m < rows4; ++m) to[m] = from[m];
            }
        }
    } else {
        const T rki = S.rk();
        LV.for_each(0, cnt, [&](int q) {
            T dx, dy, dz, r2, rkq;
            int tq;
            S.dist(q, dx, dy, dz, r2, tq, rkq);
            if (!S.inside(q, r2, rc2, c.rc_cn2)) return;
            T f;
            cn_fun(inv_sqrt(r2), rki + rkq, (T)0, k1, f, (T*)nullptr);
            nh += f;
        });
        w.cn[p] = (double)nh;
        weights_atom<MIXED, R>(w, c, cnref, nref, c6, p, S.tsrc() & 15, (double)nh);
    }
}

// ------------------------------------------------------------------ Eq. 2
// pair table per (t_i, t_j): x = R^6, y = R^8, z = s6, w = s8 R0^2 (bohr, R = a1 R0 + a2)
// ATOMV: also form P_i = sum_j (dU_j/dn_i) r_ij for the per-atom virial of Eq. 7
// (dU_j/dn_i = -1/2 (dE_ij/dC6) dC6_ij/dn_i for the pair term of U_j).
template <bool MIXED, int R, bool ATOMV>
__global__ void __launch_bounds__(128) k_disp(Work w, Consts c, const typename Real<MIXED>::T4* __restrict__ pair_tab) {
    using T = typename Real<MIXED>::T;
    using T4 = typename Real<MIXED>::T4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T4* tab = reinterpret_cast<T4*>(smem_raw);
    for (int k = threadIdx.x; k < c.T * c.T; k += blockDim.x) tab[k] = pair_tab[k];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const Site<MIXED> S(w, p);
    const int ti = S.tsrc() & 15;
    T Wi[R], dWi[R];
    load_vec<R>((const T*)w.W + p * c.RP, Wi);
    load_vec<R>((const T*)w.dW + p * c.RP, dWi);
    const T4* row = tab + ti * c.T;
    const T* vbase = (const T*)w.v + ti * c.RP;
    const int vstride = c.T * c.RP;
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_disp + list_row(G.list_base_disp, p - G.atom_base, G.cap_disp)};
    const int cnt = w.cnt_disp[p];
    const T rc2 = (T)c.rc_disp2;
    T fx = 0, fy = 0, fz = 0;
    T dnh = 0, dnl = 0;  // dE/dn_i, compensated (it scales the chain-rule forces)
    PassAcc<MIXED> E, Sxx, Syy, Szz, Sxy, Sxz, Syz, Px, Py, Pz;
    for (int k0 = 0; k0 < cnt; k0 += kChunk) {
        const int k1e = min(cnt, k0 + kChunk);
        T e = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
        T px = 0, py = 0, pz = 0;
        LV.for_each(k0, k1e, [&](int q) {
            T dx, dy, dz, r2, rkq;
            int tsq;
            S.dist(q, dx, dy, dz, r2, tsq, rkq);
            if (!S.inside(q, r2, rc2, c.rc_disp2)) return;
            const T4 tb = row[tsq & 15];
            T vq[R];
            load_vec<R>(vbase + (int64_t)(tsq >> 4) * vstride, vq);
            T C6 = 0, dC6 = 0;
#pragma unroll
            for (int a = 0; a < R; ++a) {
                C6 = fma(Wi[a], vq[a], C6);
                dC6 = fma(dWi[a], vq[a], dC6);
            }
            const T r4 = r2 * r2, r6 = r4 * r2, r8 = r4 * r4;
            const T d6 = r6 + tb.x, d8 = r8 + tb.y;
            const T pinv = recip(d6 * d8);
            const T i6 = d8 * pinv, i8 = d6 * pinv;
            const T t6 = tb.z * i6, t8 = tb.w * i8;
            const T g = t6 + t8;                     // -de/dC6
            e = fma(-C6, g, e);
            acc_add(dnh, dnl, -g * dC6);
            if constexpr (ATOMV) {
                const T b = (T)-0.5 * g * dC6;
                px = fma(b, dx, px); py = fma(b, dy, py); pz = fma(b, dz, pz);
            }
            // 2 de/d(r^2): F_i += (de/dr) d/r = fc d
            const T fc = C6 * fma((T)6 * r4, t6 * i6, (T)8 * r6 * (t8 * i8));
            const T tx = fc * dx, ty = fc * dy, tz = fc * dz;
            fx += tx; fy += ty; fz += tz;
            sxx = fma(tx, dx, sxx); syy = fma(ty, dy, syy); szz = fma(tz, dz, szz);
            sxy = fma(tx, dy, sxy); sxz = fma(tx, dz, sxz); syz = fma(ty, dz, syz);
        });
        E.add(e);
        Sxx.add(sxx); Syy.add(syy); Szz.add(szz);
        Sxy.add(sxy); Sxz.add(sxz); Syz.add(syz);
        if constexpr (ATOMV) {
            Px.add(px); Py.add(py); Pz.add(pz);
        }
    }
    if constexpr (ATOMV) ((T4*)w.Pv)[p] = T4{(T)Px.total(), (T)Py.total(), (T)Pz.total(), (T)0};
    ((T*)w.dEdn)[p] = dnh + dnl;
    ((T4*)w.Fd)[p] = T4{fx, fy, fz, (T)0};
    w.eat[p] = 0.5 * E.value();
    double* wv = w.wv + 6 * p;
    wv[0] = -0.5 * Sxx.value(); wv[1] = -0.5 * Syy.value(); wv[2] = -0.5 * Szz.value();
    wv[3] = -0.5 * Sxy.value(); wv[4] = -0.5 * Sxz.value(); wv[5] = -0.5 * Syz.value();
}

// ------------------------------------------------------------------ CN chain rule
// The chain-rule virial is accumulated per atom as -dE/dn_i sum_q f'(r) d(x)d/r
// (ordered pairs; equal to the symmetric form), whose diagonal terms all have
// one sign, so the cancellation between atoms and against the dispersion part
// happens in FP64 (per-atom sums and the per-structure reduction).  The force
// coefficient (dE/dn_i + dE/dn_q) f'(r)/r uses the double-single argument, the
// exact rc and 1/r from the double-single r^2.
//
// ATOMV: also the per-atom virial of Eq. 7 (row-major, eV) into w_atom:
//   W_i = D_i - sum_j dE/dn_j f'(r)/r d (x) d - P_i (x) G_i - sum_j f'(r)/r P_j (x) d,
// d = r_ij, G_i = sum_j f'(r)/r d, D_i the half-and-half direct pair virial of
// the dispersion pass and P from it.  The first sum is the dependence of the
// partners' site energies on r_ji through their own coordination numbers, the
// last two the dependence through n_i and through the CNs of other partners.
template <bool MIXED, bool ATOMV>
__global__ void __launch_bounds__(128) k_chain(Work w, Consts c, const float4* __restrict__ rcpair,
                                              const float2* __restrict__ exptab, double* __restrict__ F,
                                              double* __restrict__ e_atom, double* __restrict__ cn_out,
                                              double* __restrict__ w_atom) {
    using T = typename Real<MIXED>::T;
    using T4 = typename Real<MIXED>::T4;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const Site<MIXED> S(w, p);
    const T* dEdn = (const T*)w.dEdn;
    const T dni = dEdn[p];
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const T rc2 = MIXED ? (T)c.rc_cn2f : (T)c.rc_cn2, k1 = MIXED ? (T)c.k1f : (T)c.k1;
    T fx = 0, fy = 0, fz = 0;
    double Sxx = 0, Syy = 0, Szz = 0, Sxy = 0, Sxz = 0, Syz = 0;
    double Tm[6] = {0, 0, 0, 0, 0, 0}, Gv[3] = {0, 0, 0}, Mm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k0 = 0; k0 < cnt; k0 += kChunk) {
        const int k1e = min(cnt, k0 + kChunk);
        T sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
        T tm[6] = {0, 0, 0, 0, 0, 0}, gv[3] = {0, 0, 0}, mm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        // one pair's chain-rule terms: pair vector d, coefficient g = f'(r)/r, partner's dE/dn
        auto add_pair = [&](T dx, T dy, T dz, T g, T dnq, int srcq) {
            const T coef = (dni + dnq) * g;
            fx += coef * dx; fy += coef * dy; fz += coef * dz;
            // per-atom geometric sum for the virial (scaled by dE/dn_i below)
            const T gx = g * dx, gy = g * dy, gz = g * dz;
            sxx = fma(gx, dx, sxx); syy = fma(gy, dy, syy); szz = fma(gz, dz, szz);
            sxy = fma(gx, dy, sxy); sxz = fma(gx, dz, sxz); syz = fma(gy, dz, syz);
            if constexpr (ATOMV) {
                const T4 Pq = ((const T4*)w.Pv)[srcq];
                const T hx = dnq * gx, hy = dnq * gy, hz = dnq * gz;
                tm[0] = fma(hx, dx, tm[0]); tm[1] = fma(hy, dy, tm[1]); tm[2] = fma(hz, dz, tm[2]);
                tm[3] = fma(hx, dy, tm[3]); tm[4] = fma(hx, dz, tm[4]); tm[5] = fma(hy, dz, tm[5]);
                gv[0] += gx; gv[1] += gy; gv[2] += gz;
                const T ga = g * Pq.x, gb = g * Pq.y, gc = g * Pq.z;
                mm[0] = fma(ga, dx, mm[0]); mm[1] = fma(ga, dy, mm[1]); mm[2] = fma(ga, dz, mm[2]);
                mm[3] = fma(gb, dx, mm[3]); mm[4] = fma(gb, dy, mm[4]); mm[5] = fma(gb, dz, mm[5]);
                mm[6] = fma(gc, dx, mm[6]); mm[7] = fma(gc, dy, mm[7]); mm[8] = fma(gc, dz, mm[8]);
            }
        };
        if constexpr (MIXED) {
            // the stored coefficients (g = 0 outside R_cn and past the end of the list); the
            // loads of a group of kGroup entries are issued before any of their arithmetic, an
            // entry with g = 0 reading atom p's own record (d = 0: it adds nothing)
            constexpr int kGroup = 8;
            const float* grow = w.gcn + (LV.p - w.nbr_cn);
            for (int k = k0; k < k1e; k += kGroup) {
                int q[kGroup];
                float g[kGroup];
#pragma unroll
                for (int h = 0; h < kGroup; h += 4) {
                    int4 q4 = make_int4(0, 0, 0, 0);
                    float4 g4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k + h < k1e) {
                        q4 = __ldg(reinterpret_cast<const int4*>(LV.p + list_off(k + h)));
                        g4 = __ldg(reinterpret_cast<const float4*>(grow + list_off(k + h)));
                    }
                    q[h] = q4.x; q[h + 1] = q4.y; q[h + 2] = q4.z; q[h + 3] = q4.w;
                    g[h] = g4.x; g[h + 1] = g4.y; g[h + 2] = g4.z; g[h + 3] = g4.w;
                }
                float D[kGroup][3];
                int src[kGroup];
#pragma unroll
                for (int e = 0; e < kGroup; ++e) {
                    float er[3];
                    int tq;
                    S.dist_exact(g[e] != 0.0f ? q[e] : (int)p, D[e], er, tq);
                    src[e] = tq >> 4;
                }
                float dn[kGroup];
#pragma unroll
                for (int e = 0; e < kGroup; ++e) dn[e] = dEdn[src[e]];
#pragma unroll
                for (int e = 0; e < kGroup; ++e) add_pair(D[e][0], D[e][1], D[e][2], g[e], dn[e], src[e]);
            }
        } else {
            LV.for_each(k0, k1e, [&](int q) {
                T dx, dy, dz, r2, rkq;
                int tsq;
                S.dist(q, dx, dy, dz, r2, tsq, rkq);
                if (!S.inside(q, r2, rc2, c.rc_cn2)) return;
                const T rinv = inv_sqrt(r2);
                T f, dfdr;
                cn_fun(rinv, S.rk() + rkq, (T)0, k1, f, &dfdr);
                const int srcq = tsq >> 4;
                add_pair(dx, dy, dz, dfdr * rinv, dEdn[srcq], srcq);
            });
        }
        Sxx += (double)sxx; Syy += (double)syy; Szz += (double)szz;
        Sxy += (double)sxy; Sxz += (double)sxz; Syz += (double)syz;
        if constexpr (ATOMV) {
#pragma unroll
            for (int k = 0; k < 6; ++k) Tm[k] += (double)tm[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) Gv[k] += (double)gv[k];
#pragma unroll
            for (int k = 0; k < 9; ++k) Mm[k] += (double)mm[k];
        }
    }
    const T4 fd = ((const T4*)w.Fd)[p];
    const double u = kHartreeEV / kBohrA;
    const int i = w.perm[p];
    const double f0 = ((double)fd.x + (double)fx) * u, f1 = ((double)fd.y + (double)fy) * u,
                 f2 = ((double)fd.z + (double)fz) * u;
    double* Fi = F + 3 * (int64_t)i;
    if (c.accumulate) {
        Fi[0] += f0; Fi[1] += f1; Fi[2] += f2;
    } else {
        Fi[0] = f0; Fi[1] = f1; Fi[2] = f2;
    }
    double* wv = w.wv + 6 * p;
    if constexpr (ATOMV) {
        // wv holds the direct (dispersion) part here: xx yy zz xy xz yz
        const double Dm[9] = {wv[0], wv[3], wv[4], wv[3], wv[1], wv[5], wv[4], wv[5], wv[2]};
        const double Ts[9] = {Tm[0], Tm[3], Tm[4], Tm[3], Tm[1], Tm[5], Tm[4], Tm[5], Tm[2]};
        const T4 Pi = ((const T4*)w.Pv)[p];
        const double P[3] = {(double)Pi.x, (double)Pi.y, (double)Pi.z};
        double* out = w_atom + 9 * (int64_t)i;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                out[3 * a + b] = (Dm[3 * a + b] - Ts[3 * a + b] - P[a] * Gv[b] - Mm[3 * a + b]) * kHartreeEV;
    }
    // W -= sum over ordered pairs of dE/dn_i f'(r) d(x)d/r
    const double dn = (double)dni;
    wv[0] -= dn * Sxx; wv[1] -= dn * Syy; wv[2] -= dn * Szz;
    wv[3] -= dn * Sxy; wv[4] -= dn * Sxz; wv[5] -= dn * Syz;
    if (e_atom) e_atom[i] = w.eat[p] * kHartreeEV;
    if (cn_out) cn_out[i] = w.cn[p];
}

// ------------------------------------------------------------------ per-structure sums
// Two fixed-order levels: block (s, c) sums atoms [c*kFinChunk, (c+1)*kFinChunk)
// of structure s into part[fin_base_s + c][7]; then warp s adds its structure's
// chunk sums (a strided pass and a shuffle tree, both in a fixed order).
// Deterministic for any batch shape.
__global__ void __launch_bounds__(256) k_fin_chunks(Work w, double* __restrict__ part) {
    const int64_t cid = blockIdx.x;
    const int s = w.fin_sid[cid];
    const StructGeo& G = w.geo[s];
    const int64_t k0 = (cid - G.fin_base) * kFinChunk;
    const int64_t k1 = k0 + kFinChunk < (int64_t)G.natoms ? k0 + kFinChunk : (int64_t)G.natoms;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const int64_t p = G.atom_base + k;
        acc[0] += w.eat[p];
#pragma unroll
        for (int m = 0; m < 6; ++m) acc[1 + m] += w.wv[6 * p + m];
    }
    __shared__ double red[7][256];
#pragma unroll
    for (int m = 0; m < 7; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int m = 0; m < 7; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 7) part[cid * 7 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(128) k_fin_struct(Work w, const double* __restrict__ part,
                                                    double* __restrict__ E, double* __restrict__ Wout,
                                                    int accumulate) {
    const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= w.B) return;  // whole warps leave together
    const StructGeo& G = w.geo[s];
    const int nc = (int)((G.natoms + kFinChunk - 1) / kFinChunk);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int ch = lane; ch < nc; ch += 32)
#pragma unroll
        for (int m = 0; m < 7; ++m) acc[m] += part[(G.fin_base + ch) * 7 + m];
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int m = 0; m < 7; ++m) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (lane != 0) return;
    const double h = kHartreeEV;
    const double v[9] = {acc[1] * h, acc[4] * h, acc[5] * h, acc[4] * h, acc[2] * h, acc[6] * h,
                         acc[5] * h, acc[6] * h, acc[3] * h};
    double* Ws = Wout + 9 * (int64_t)s;
    if (accumulate) {
        E[s] += acc[0] * h;
#pragma unroll
        for (int k = 0; k < 9; ++k) Ws[k] += v[k];
    } else {
        E[s] = acc[0] * h;
#pragma unroll
        for (int k = 0; k < 9; ++k) Ws[k] = v[k];
    }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <bool MIXED, int R>
cudaError_t forward_impl(const Work& w, const Consts& c, const Tabs& tb, double* E, double* F, double* W,
                         double* e_atom, double* cn_out, double* w_atom, int B, cudaStream_t st,
                         cudaEvent_t* marks) {
    using T = typename Real<MIXED>::T;
    using T4 = typename Real<MIXED>::T4;
    auto mark = [&](int k) {
        if (marks) cudaEventRecord(marks[k], st);
    };
    mark(0);
    if (w.Nr > 0)
        k_cn<MIXED, R><<<nblk(w.Nr, w.blk_cn), w.blk_cn, 0, st>>>(w, c, tb.rcpair, tb.exptab, tb.cnref, tb.cnref2,
                                                                  tb.dcr, tb.nref, (const T*)tb.c6);
    mark(1);  // the weights (Eq. 3) are formed inside the CN pass
    mark(2);
    if (MIXED && w.cl_mode && !w_atom) {
        const cudaError_t e = launch_disp_cl(w, c, tb.pair, e_atom != nullptr, st);
        if (e != cudaSuccess) return e;
    } else if (w.Nr > 0) {
        const int TB = w.blk_disp;
        if (w_atom)
            k_disp<MIXED, R, true><<<nblk(w.Nr, TB), TB, c.T * c.T * sizeof(T4), st>>>(w, c, (const T4*)tb.pair);
        else
            k_disp<MIXED, R, false><<<nblk(w.Nr, TB), TB, c.T * c.T * sizeof(T4), st>>>(w, c, (const T4*)tb.pair);
    }
    mark(3);
    if (c.atm && w.Nr > 0) {
        const cudaError_t e = launch_atm(w, c, MIXED, tb.rtab, st);
        if (e != cudaSuccess) return e;
    }
    mark(4);
    if (w.Nr > 0) {
        const int TB = w.blk_chain;
        if (w_atom)
            k_chain<MIXED, true><<<nblk(w.Nr, TB), TB, 0, st>>>(w, c, tb.rcpair, tb.exptab, F, e_atom, cn_out, w_atom);
        else
            k_chain<MIXED, false><<<nblk(w.Nr, TB), TB, 0, st>>>(w, c, tb.rcpair, tb.exptab, F, e_atom, cn_out, nullptr);
    }
    mark(5);
    if (B > 0) {
        if (w.n_fin > 0) k_fin_chunks<<<(unsigned)w.n_fin, 256, 0, st>>>(w, w.fin_part);
        k_fin_struct<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(w, w.fin_part, E, W, c.accumulate);
    }
    mark(6);
    return cudaGetLastError();
}

// Eq. 8: J_i = W_i . v_i (row-major W_i)
__global__ void k_heat(int64_t n, const double* __restrict__ w_atom, const double* __restrict__ vel,
                       double* __restrict__ J) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* Wi = w_atom + 9 * i;
    const double v0 = vel[3 * i], v1 = vel[3 * i + 1], v2 = vel[3 * i + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) J[3 * i + a] = Wi[3 * a] * v0 + Wi[3 * a + 1] * v1 + Wi[3 * a + 2] * v2;
}

}  // namespace

cudaError_t launch_heat(int64_t n, const double* w_atom, const double* vel, double* J, cudaStream_t st) {
    if (n > 0) k_heat<<<nblk(n, 256), 256, 0, st>>>(n, w_atom, vel, J);
    return cudaGetLastError();
}

cudaError_t launch_forward(const Work& w, const Consts& c, bool mixed, const Tabs& tabs, double* E, double* F,
                           double* W, double* e_atom, double* cn_out, double* w_atom, int B, cudaStream_t st,
                           cudaEvent_t* marks) {
#define D3_FWD(M, RR) return forward_impl<M, RR>(w, c, tabs, E, F, W, e_atom, cn_out, w_atom, B, st, marks)
    if (mixed) {
        switch (c.R) {
            case 1: D3_FWD(true, 1);
            case 2: D3_FWD(true, 2);
            case 3: D3_FWD(true, 3);
            case 4: D3_FWD(true, 4);
            case 5: D3_FWD(true, 5);
            case 6: D3_FWD(true, 6);
            default: D3_FWD(true, 7);
        }
    } else {
        switch (c.R) {
            case 1: D3_FWD(false, 1);
            case 2: D3_FWD(false, 2);
            case 3: D3_FWD(false, 3);
            case 4: D3_FWD(false, 4);
            case 5: D3_FWD(false, 5);
            case 6: D3_FWD(false, 6);
            default: D3_FWD(false, 7);
        }
    }
#undef D3_FWD
}

}  // namespace d3gb
