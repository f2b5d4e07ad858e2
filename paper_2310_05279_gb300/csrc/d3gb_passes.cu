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
//                     dE/dn_i = sum_j (dE/dC6_ij)(dC6_ij/dn_i)
//   k_atm             optional three-body term (not part of the paper's model)
//   k_chain           forces and virial of the coordination-number dependence:
//                     F_i += sum_j (dE/dn_i + dE/dn_j) f'(r_ij) r_ij/r
//   k_fin_*           per-structure energy and virial (fixed-order sums)
//
// MIXED = true: pair arithmetic in FP32 on split (hi + lo) positions, partial
// sums promoted to FP64 every kChunk pairs; cutoff tests that fall within the
// FP32 error band of the cutoff are decided in FP64, so the set of pairs is
// the FP64 one.  MIXED = false: FP64 throughout.
#include "d3gb_internal.cuh"

namespace d3gb {

namespace {

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// one Newton step on the hardware estimates
__device__ __forceinline__ float rsqrt_nr(float x) {
    float y = rsqrt_approx(x);
    float h = 0.5f * x * y;
    return y * fmaf(-h, y, 1.5f);
}
__device__ __forceinline__ float rcp_nr(float x) {
    float y = rcp_approx(x);
    float e = fmaf(-x, y, 1.0f);
    return fmaf(y, e, y);
}

// s + err == a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}
// running compensated sum (value hi + lo)
__device__ __forceinline__ void acc_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}
__device__ __forceinline__ void acc_add(double& hi, double&, double x) { hi += x; }

template <bool MIXED> struct Real;
template <> struct Real<true> { using T = float; using T4 = float4; };
template <> struct Real<false> { using T = double; using T4 = dbl4; };

// Per-thread view of atom p's position and the distance to a neighbour q.
template <bool MIXED> struct Site;

template <> struct Site<true> {
    float4 h, l;
    const Work* w;
    int64_t p;
    __device__ Site(const Work& W, int64_t P) : w(&W), p(P) { rec_load(W, P, h, l); }
    __device__ int tsrc() const { return __float_as_int(h.w); }
    __device__ float rk() const { return l.w; }
    // distance vector to q; returns the neighbour's packed type/source and k2*Rcov
    __device__ void dist(int q, float& dx, float& dy, float& dz, float& r2, int& tq, float& rkq) const {
        float4 hq, lq;
        rec_load(*w, q, hq, lq);
        dx = (hq.x - h.x) + (lq.x - l.x);
        dy = (hq.y - h.y) + (lq.y - l.y);
        dz = (hq.z - h.z) + (lq.z - l.z);
        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        tq = __float_as_int(hq.w);
        rkq = lq.w;
    }
    // exact pair vector as D + e (hi parts lie on a common grid, so hq - hp is exact)
    __device__ void dist_exact(int q, float (&D)[3], float (&e)[3], int& tq) const {
        float4 hq, lq;
        rec_load(*w, q, hq, lq);
        const float A[3] = {hq.x - h.x, hq.y - h.y, hq.z - h.z};
        const float Bv[3] = {lq.x - l.x, lq.y - l.y, lq.z - l.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            D[k] = A[k] + Bv[k];
            e[k] = Bv[k] - (D[k] - A[k]);  // |A| >= |B| unless A == 0: Fast2Sum is exact
        }
        tq = __float_as_int(hq.w);
    }
    // r^2 < rc2 as FP64 decides it: FP32 outside the error band, FP64 inside
    __device__ bool inside(int q, float r2, float rc2f, double rc2d) const {
        if (fabsf(r2 - rc2f) > 4e-6f * rc2f) return r2 < rc2f;
        const dbl4 a = w->pos64[p], b = w->pos64[q];
        const double ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
        return ex * ex + ey * ey + ez * ez < rc2d;
    }
};

template <> struct Site<false> {
    dbl4 x;
    int ts;
    const Work* w;
    __device__ Site(const Work& W, int64_t P) : w(&W) { x = W.pos64[P]; ts = rec_tsrc(W, P); }
    __device__ int tsrc() const { return ts; }
    __device__ double rk() const { return x.w; }
    __device__ void dist(int q, double& dx, double& dy, double& dz, double& r2, int& tq, double& rkq) const {
        const dbl4 y = w->pos64[q];
        dx = y.x - x.x;
        dy = y.y - x.y;
        dz = y.z - x.z;
        r2 = dx * dx + dy * dy + dz * dz;
        tq = rec_tsrc(*w, q);
        rkq = y.w;
    }
    __device__ bool inside(int, double r2, double rc2, double) const { return r2 < rc2; }
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

template <int R, class T>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&x)[R]) {
#pragma unroll
    for (int a = 0; a < R; ++a) x[a] = p[a];
}
// p is 16-byte aligned for R <= 4 and 32-byte aligned (one 256-bit load) for R <= 8
template <int R>
__device__ __forceinline__ void load_vec(const float* __restrict__ p, float (&x)[R]) {
    if constexpr (R <= 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int a = 0; a < R; ++a) x[a] = tv[a];
    } else {
        float4 t0, t1;
        ld8(p, t0, t1);
        const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
        for (int a = 0; a < R; ++a) x[a] = tv[a];
    }
}


// Mixed form: pair vector D (FP32), r^2 and the Eq. 4 exponent a = k1 (rc/r - 1)
// as a double-single pair (ah + al) from the exact pair vector D + e:
//   r^2 = Sh + Sl (TwoProd/TwoSum), u = rc^2 - r^2, r = sqrt(r^2) with its
//   correction term, den = r^2 + r rc, a = k1 u / den with one residual step.
// Its error is a few units of 2^-48 relative, so exp(-a) is as accurate as
// expf itself.  Returns false when the pair is outside R_cn.
__device__ __forceinline__ bool cn_pair_precise(const Site<true>& S, int q, const float4* rrow, float k1, float rc2,
                                                double rc2d, float (&D)[3], float& r2, float& ah, float& al,
                                                float& rch, int& tq, float* rcl_out = nullptr,
                                                float* r2l_out = nullptr) {
    float e[3];
    S.dist_exact(q, D, e, tq);
    float P[3], pl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P[k] = D[k] * D[k];
        pl[k] = fmaf(D[k], D[k], -P[k]);
    }
    float S1, s1, Sh, s2;
    two_sum(P[0], P[1], S1, s1);
    two_sum(S1, P[2], Sh, s2);
    float Sl = (s1 + s2) + (pl[0] + pl[1] + pl[2]) + 2.0f * (D[0] * e[0] + D[1] * e[1] + D[2] * e[2]);
    two_sum(Sh, Sl, Sh, Sl);  // normalise
    r2 = Sh;
    if (!S.inside(q, r2, rc2, rc2d)) return false;
    const float4 rc = rrow[tq & 15];  // rc hi, rc lo, rc^2 hi, rc^2 lo
    float uh, ue;
    two_sum(rc.z, -Sh, uh, ue);
    const float ul = ue + (rc.w - Sl);
    const float rh = Sh * rsqrt_nr(Sh);
    const float rl = (fmaf(-rh, rh, Sh) + Sl) * (0.5f / rh);
    const float ph = rh * rc.x, pe = fmaf(rh, rc.x, -ph);
    float dh, de;
    two_sum(Sh, ph, dh, de);
    const float dl = de + Sl + pe + rh * rc.y + rl * rc.x;
    const float idh = rcp_nr(dh);
    const float qh = uh * idh;
    const float ql = (fmaf(-qh, dh, uh) + ul - qh * dl) * idh;
    ah = k1 * qh;
    al = fmaf(k1, qh, -ah) + k1 * ql;
    rch = rc.x;
    if (rcl_out) *rcl_out = rc.y;
    if (r2l_out) *r2l_out = Sl;
    return true;
}

// ------------------------------------------------------------------ Eq. 4 in double-single
// t = exp(-a), f = 1/(1 + t) and 1 - f = t f for a = ah + al, each as a
// double-single pair with a relative error near 1e-11.  The coordination number
// and its chain-rule forces are sums of many such terms; FP32 rounding of each
// would leave a small systematic error that the sums accumulate, so the terms
// are formed here from FP32 operations with error-free transformations.
//
// exp follows the table-driven method of P. T. P. Tang (ACM TOMS 15(2), 1989):
// x = (64 m + j) L + r with L = ln2/64 (carried in three FP32 parts so that the
// reduction is exact to ~1e-14), exp(x) = 2^m 2^(j/64) exp(r), |r| <= L/2, and
// exp(r) = 1 + r + r^2/2 + r^3/6 + r^4/24 (truncation below 4e-14).  The table
// holds 2^(j/64) as FP32 hi + lo pairs.
constexpr double kLnTwoOver64 = 0.693147180559945309417232121458 / 64.0;
constexpr float kExpL1 = 1420.0f / 131072.0f;  // 11 significant bits: k L1 is exact for |k| < 2^13
constexpr float kExpL2 = (float)(kLnTwoOver64 - (double)kExpL1);
constexpr float kExpL3 = (float)((kLnTwoOver64 - (double)kExpL1) - (double)kExpL2);
constexpr float kExpInvL = (float)(64.0 / 0.693147180559945309417232121458);

struct CnDS {
    float th, tl;  // t = exp(-a)
    float fh, fl;  // f = 1 / (1 + t)
    float ch, cl;  // 1 - f = t f
};

__device__ __forceinline__ CnDS cn_ds(float ah, float al, const float2* __restrict__ tab) {
    // x = -a, clamped so that 2^m stays a normal FP32 scale (|x| <= 87: t in [1.6e-38, 6e37])
    float xh = -ah, xl = -al;
    if (fabsf(xh) > 87.0f) { xh = copysignf(87.0f, xh); xl = 0.0f; }
    const float kf = rintf(xh * kExpInvL);
    const int k = (int)kf;
    const float r1 = fmaf(-kf, kExpL1, xh);  // exact (see kExpL1)
    const float p2 = kf * kExpL2, p2e = fmaf(kf, kExpL2, -p2);
    float rh, re;
    two_sum(r1, -p2, rh, re);
    const float rl = ((re - p2e) - kf * kExpL3) + xl;
    // exp(r) - 1 = rh + s
    const float s = rl + rh * rl + rh * rh * fmaf(rh, fmaf(rh, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
    const int j = k & 63, m = (k - j) / 64;
    const float2 T = __ldg(tab + j);
    const float ph = T.x * rh, pe = fmaf(T.x, rh, -ph);
    const float hh = T.x + ph, he = ph - (hh - T.x);  // |T.x| >= |ph|: Fast2Sum
    const float lo = he + pe + T.y + fmaf(T.x, s, T.y * rh);
    float th = hh + lo;
    float tl = lo - (th - hh);
    th = ldexpf(th, m);
    tl = ldexpf(tl, m);
    CnDS o;
    o.th = th;
    o.tl = tl;
    // f = 1/(1 + t) with one residual correction
    float dh, de;
    two_sum(1.0f, th, dh, de);
    const float dl = de + tl;
    const float y = rcp_nr(dh);
    const float rho = fmaf(-dh, y, 1.0f) - dl * y;
    o.fh = y;
    o.fl = y * rho;
    // 1 - f = t f
    const float ch = th * o.fh;
    o.ch = ch;
    o.cl = fmaf(th, o.fh, -ch) + fmaf(th, o.fl, tl * o.fh);
    return o;
}

// double-single product (ah + al)(bh + bl), result as hi + lo
__device__ __forceinline__ void ds_mul(float ah, float al, float bh, float bl, float& h, float& l) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);
    l = fmaf(ah, bl, fmaf(al, bh, e));
    h = p + l;
    l = l - (h - p);
}

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
    store_row<T>((T*)w.W + p * c.RP, Wr, c.RP);
    store_row<T>((T*)w.dW + p * c.RP, dWr, c.RP);
    T* vp = (T*)w.v + p * c.T * c.RP;
    for (int u = 0; u < c.T; ++u) {
        const T* cu = c6 + ((size_t)(u * c.T + t) * R) * R;  // C6ref[u][t][a][b]
        T vr[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            T s = 0;
            if (a < R) {
#pragma unroll
                for (int b = 0; b < R; ++b) s += cu[a * R + b] * L[b];
            }
            vr[a] = s;
        }
        store_row<T>(vp + u * c.RP, vr, c.RP);
    }
}

// ------------------------------------------------------------------ Eq. 4
// The coordination numbers feed dC6/dn, which can be large, so the mixed form
// keeps n_i accurate to a few 1e-8: the pair vector is exact (D + e), r^2 is
// formed in double-single, the argument k1 (rc/r - 1) is evaluated as
// k1 (rc^2 - r^2) / (r (rc + r)) so its error is relative to its own size,
// and the sum over neighbours is compensated.
template <bool MIXED, int R>
__global__ void __launch_bounds__(128) k_cn(Work w, Consts c, const float4* __restrict__ rcpair,
                                           const float2* __restrict__ exptab, const double* __restrict__ cnref,
                                           const int* __restrict__ nref,
                                           const typename Real<MIXED>::T* __restrict__ c6) {
    using T = typename Real<MIXED>::T;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const Site<MIXED> S(w, p);
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const T rc2 = (T)c.rc_cn2, k1 = (T)c.k1;
    T nh = 0, nl = 0;
    if constexpr (MIXED) {
        const float4* rrow = rcpair + (S.tsrc() & 15) * c.T;
        int nint = 0;  // terms with f > 1/2 are summed as 1 - t/(1 + t): exact integer part plus a small complement
        LV.for_each(0, cnt, [&](int q) {
            float D[3], r2, ah, al, rch;
            int tq;
            if (!cn_pair_precise(S, q, rrow, k1, rc2, c.rc_cn2, D, r2, ah, al, rch, tq)) return;
            const CnDS z = cn_ds(ah, al, exptab);
            if (z.th < 1.0f) {
                ++nint;
                acc_add(nh, nl, -z.ch);
                nl -= z.cl;
            } else {
                acc_add(nh, nl, z.fh);
                nl += z.fl;
            }
        });
        const double n = (double)nint + (double)nh + (double)nl;
        w.cn[p] = n;
        weights_atom<MIXED, R>(w, c, cnref, nref, c6, p, S.tsrc() & 15, n);
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
    double E = 0, Sxx = 0, Syy = 0, Szz = 0, Sxy = 0, Sxz = 0, Syz = 0;
    double Px = 0, Py = 0, Pz = 0;
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
        E += (double)e;
        Sxx += (double)sxx; Syy += (double)syy; Szz += (double)szz;
        Sxy += (double)sxy; Sxz += (double)sxz; Syz += (double)syz;
        Px += (double)px; Py += (double)py; Pz += (double)pz;
    }
    if constexpr (ATOMV) ((T4*)w.Pv)[p] = T4{(T)Px, (T)Py, (T)Pz, (T)0};
    ((T*)w.dEdn)[p] = (T)((double)dnh + (double)dnl);
    ((T4*)w.Fd)[p] = T4{fx, fy, fz, (T)0};
    w.eat[p] = 0.5 * E;
    double* wv = w.wv + 6 * p;
    wv[0] = -0.5 * Sxx; wv[1] = -0.5 * Syy; wv[2] = -0.5 * Szz;
    wv[3] = -0.5 * Sxy; wv[4] = -0.5 * Sxz; wv[5] = -0.5 * Syz;
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
    const T rc2 = (T)c.rc_cn2, k1 = (T)c.k1;
    T fx = 0, fy = 0, fz = 0;
    double Sxx = 0, Syy = 0, Szz = 0, Sxy = 0, Sxz = 0, Syz = 0;
    double Tm[6] = {0, 0, 0, 0, 0, 0}, Gv[3] = {0, 0, 0}, Mm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k0 = 0; k0 < cnt; k0 += kChunk) {
        const int k1e = min(cnt, k0 + kChunk);
        T sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
        T tm[6] = {0, 0, 0, 0, 0, 0}, gv[3] = {0, 0, 0}, mm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        LV.for_each(k0, k1e, [&](int q) {
            T dx, dy, dz, g, dnq;
            int srcq;
            if constexpr (MIXED) {
                float D[3], r2, ah, al, rch, rcl, r2l;
                int tq;
                if (!cn_pair_precise(S, q, rcpair + (S.tsrc() & 15) * c.T, k1, rc2, c.rc_cn2, D, r2, ah, al, rch, tq,
                                     &rcl, &r2l))
                    return;
                const CnDS z = cn_ds(ah, al, exptab);
                // 1/r from r^2 = r2 + r2l with one residual step (double-single)
                const float y0 = rsqrt_nr(r2);
                const float y2 = y0 * y0, y2e = fmaf(y0, y0, -y2);
                const float ry = fmaf(-r2, y2, 1.0f) - fmaf(r2, y2e, r2l * y2);
                const float yh = y0, yl = 0.5f * y0 * ry;
                // f'(r)/r = -k1 rc f (1 - f) / r^3, formed in double-single and rounded once
                float a2h, a2l, a3h, a3l, cfh, cfl, uh, ul, gh, gl;
                ds_mul(yh, yl, yh, yl, a2h, a2l);
                ds_mul(a2h, a2l, yh, yl, a3h, a3l);
                ds_mul(z.ch, z.cl, z.fh, z.fl, cfh, cfl);
                ds_mul(rch, rcl, cfh, cfl, uh, ul);
                ds_mul(uh, ul, a3h, a3l, gh, gl);
                g = -k1 * (gh + gl);
                srcq = tq >> 4;
                dnq = dEdn[srcq];
                dx = D[0]; dy = D[1]; dz = D[2];
            } else {
                T r2, rkq;
                int tsq;
                S.dist(q, dx, dy, dz, r2, tsq, rkq);
                if (!S.inside(q, r2, rc2, c.rc_cn2)) return;
                const T rinv = inv_sqrt(r2);
                T f, dfdr;
                cn_fun(rinv, S.rk() + rkq, (T)0, k1, f, &dfdr);
                g = dfdr * rinv;
                srcq = tsq >> 4;
                dnq = dEdn[srcq];
            }
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
        });
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

// ------------------------------------------------------------------ optional three-body term
// Triple-dipole (Axilrod-Teller-Muto) term of the original D3 model, which the
// paper leaves out (Sec. II A); off unless d3_set_three_body enables it.  For a
// triangle (i, j, k) with squared sides x = r_ij^2, y = r_ik^2, z = r_jk^2 and
// P = x y z:
//   E = s9 sqrt(C6_ij C6_ik C6_jk) A f,
//   A = (3 cos cos cos + 1) / (r_ij r_ik r_jk)^3 = P^(-3/2) (1 + 3 N / (8 P)),
//   N = (x + y - z)(x + z - y)(y + z - x)   (law of cosines),
//   f = 1 / (1 + 6 q),   q = (R_ij R_ik R_jk / sqrt(P))^(alpha/3),
// R the damping radii a1 R0 + a2 of Eq. 2.  Every side must be below rc3 <= R_cn,
// so the candidates come from the CN list.
//
// One warp per atom i.  The lanes stage i's neighbours within rc3 in shared
// memory (vector, r^2, C6_ij and its n_i-derivative, W_j), then test the
// unordered pairs (j, k) of them: lane-strided partners j, each with the n/2
// slots that follow it cyclically, so every pair is tested once.  Most pairs
// fail the third side's cutoff, so the pairs that pass are queued in shared
// memory (ballot compaction) and evaluated 32 at a time with every lane busy.
// The warp writes only atom i's results; every triangle is visited once from
// each of its vertices, and these parts add up to its totals:
//   U_i     += E / 3
//   F_i     += -dE/dr_i = 2 (E_x d_ij + E_y d_ik)          (E_x = dE/dx)
//   dE/dn_i += E/2 (dC6_ij/dn_i / C6_ij + dC6_ik/dn_i / C6_ik), with W_j, W_k fixed
//   virial  -= E_x d_ij (x) d_ij + E_y d_ik (x) d_ik      (half of each side at i)
// A list longer than the staging area is processed in tile pairs.
constexpr int kAtmWarps = 4;
constexpr int kAtmQueue = 64;  // triangle queue per warp (ring; at most 63 entries pending)

template <bool MIXED> struct AtmCap { static constexpr int C = MIXED ? 128 : 64; };

// Per-lane running sums of the three-body pass.  The mixed form keeps a
// compensated float pair (value hi + lo) on the FP32 pipe: GB300 executes FP64
// at 1/64 of the FP32 rate, so FP64 running sums and an FP64 warp reduction
// would bound the kernel.  The FP64 form sums in FP64.
template <bool MIXED> struct AtmAcc;
template <> struct AtmAcc<true> {
    float h = 0.f, l = 0.f;
    __device__ void add(float x) { acc_add(h, l, x); }
    // with the partner lane's sum (the same result on both lanes)
    __device__ void xor_reduce(int o) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
        float sh, e;
        two_sum(h, h2, sh, e);
        h = sh;
        l = (l + l2) + e;
    }
    __device__ float total() const { return h + l; }
};
template <> struct AtmAcc<false> {
    double h = 0.0;
    __device__ void add(double x) { h += x; }
    __device__ void xor_reduce(int o) { h += __shfl_xor_sync(0xffffffffu, h, o); }
    __device__ double total() const { return h; }
};

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// x^e for x > 0 (FP32: hardware base-2 logarithm and power, relative error ~1e-6
// for the exponents used here; FP64: the library functions)
__device__ __forceinline__ float pow_pos(float x, float e) { return ex2_approx(e * lg2_approx(x)); }
__device__ __forceinline__ double pow_pos(double x, double e) { return exp2(e * log2(x)); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrt_nr(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rcp_t(float x) { return rcp_nr(x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

template <bool MIXED, int R>
__global__ void __launch_bounds__(32 * kAtmWarps) k_atm(Work w, Consts c, const typename Real<MIXED>::T* __restrict__ rtab) {
    using T = typename Real<MIXED>::T;
    using T4 = typename Real<MIXED>::T4;
    constexpr int C = AtmCap<MIXED>::C;
    constexpr int RPc = R <= 4 ? 4 : 8;  // row padding of W and v (c.RP)
    __shared__ T4 sA[kAtmWarps][C];    // d_ij (bohr), r_ij^2
    __shared__ T4 sB[kAtmWarps][C];    // C6_ij, (dC6_ij/dn_i) / C6_ij, R_ij, 1 / r_ij^2
    __shared__ int2 sQ[kAtmWarps][C];  // atom index of the instance, packed type/source
    __shared__ __align__(32) T sW[kAtmWarps][C][RPc];  // W_j
    __shared__ int sJK[kAtmWarps][kAtmQueue];           // queued triangles: j slot << 8 | k slot
    __shared__ T sR[kMaxTypes * kMaxTypes];
    for (int k = threadIdx.x; k < c.T * c.T; k += blockDim.x) sR[k] = rtab[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t p = (int64_t)blockIdx.x * kAtmWarps + wid;
    if (p >= w.Nr) return;  // the whole warp
    T4* sa = sA[wid];
    T4* sb = sB[wid];
    int2* sq = sQ[wid];
    int* jk = sJK[wid];
    const Site<MIXED> S(w, p);
    const int ti = S.tsrc() & 15;
    T Wi[R], dWi[R];
    load_vec<R>((const T*)w.W + p * RPc, Wi);
    load_vec<R>((const T*)w.dW + p * RPc, dWi);
    const T* vb = (const T*)w.v;
    const int vstride = c.T * RPc;
    const StructGeo& G = w.geo[w.sid[p]];
    const int* row = w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn);
    const int cnt = w.cnt_cn[p];
    // FP32 copies from the host in the mixed form (a conversion is an FP64-pipe operation)
    const T rc3 = MIXED ? (T)c.rc3_2f : (T)c.rc3_2, s9 = MIXED ? (T)c.s9f : (T)c.s9;
    const T alpha = MIXED ? (T)c.alpha9f : (T)c.alpha9, a3 = MIXED ? (T)c.alpha9_3f : (T)(c.alpha9 / 3.0);
    AtmAcc<MIXED> aE, aDn, aFx, aFy, aFz, aV[6];
    T e_ = 0, dn_ = 0, fx_ = 0, fy_ = 0, fz_ = 0, v_[6] = {0, 0, 0, 0, 0, 0};  // FP32 partial sums
    int head = 0, tail = 0;  // queue positions (warp-uniform)

    // list entries [k0, k1) within rc3 into slots base, base + 1, ...; returns their number
    auto stage = [&](int k0, int k1, int base) -> int {
        int n = 0;
        for (int kk = k0; kk < k1; kk += 32) {
            const int k = kk + lane;
            bool in = false;
            int q = 0, tq = 0;
            T dx = 0, dy = 0, dz = 0, r2 = 0, rkq = 0;
            if (k < k1) {
                q = __ldg(row + k);
                S.dist(q, dx, dy, dz, r2, tq, rkq);
                in = S.inside(q, r2, rc3, c.rc3_2);
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (in) {
                const int slot = base + n + __popc(m & lt);
                T vq[R], Wq[R];
                load_vec<R>(vb + (int64_t)(tq >> 4) * vstride + ti * RPc, vq);
                load_vec<R>((const T*)w.W + (int64_t)(tq >> 4) * RPc, Wq);
                T C6 = 0, dC6 = 0;
#pragma unroll
                for (int a = 0; a < R; ++a) {
                    C6 = fma(Wi[a], vq[a], C6);
                    dC6 = fma(dWi[a], vq[a], dC6);
                    sW[wid][slot][a] = Wq[a];
                }
                sa[slot] = T4{dx, dy, dz, r2};
                sb[slot] = T4{C6, dC6 / C6, sR[ti * c.T + (tq & 15)], (T)1 / r2};
                sq[slot] = make_int2(q, tq);
            }
            n += __popc(m);
        }
        __syncwarp();
        return n;
    };

    // third side below rc3, decided as FP64 decides it
    auto close = [&](int js, int ks) -> bool {
        const T4 Aj = sa[js], Ak = sa[ks];
        const T ex = Ak.x - Aj.x, ey = Ak.y - Aj.y, ez = Ak.z - Aj.z;
        const T z = fma(ex, ex, fma(ey, ey, ez * ez));
        if constexpr (MIXED) {
            if (fabsf(z - rc3) <= 4e-6f * rc3) {
                const dbl4 a = w.pos64[sq[js].x], b = w.pos64[sq[ks].x];
                const double gx = b.x - a.x, gy = b.y - a.y, gz = b.z - a.z;
                return gx * gx + gy * gy + gz * gz < c.rc3_2;
            }
        }
        return z < rc3;
    };

    // one triangle (slots js, ks) into this lane's partial sums
    auto eval = [&](int js, int ks) {
        const T4 Aj = sa[js], Ak = sa[ks];
        const T ex = Ak.x - Aj.x, ey = Ak.y - Aj.y, ez = Ak.z - Aj.z;
        const T z = fma(ex, ex, fma(ey, ey, ez * ez));
        const T4 Bj = sb[js], Bk = sb[ks];
        const int tj = sq[js].y & 15, tsk = sq[ks].y;
        T vk[R];
        load_vec<R>(vb + (int64_t)(tsk >> 4) * vstride + tj * RPc, vk);
        T C6jk = 0;
#pragma unroll
        for (int a = 0; a < R; ++a) C6jk = fma(sW[wid][js][a], vk[a], C6jk);
        const T x = Aj.w, y = Ak.w, ix = Bj.w, iy = Bk.w;
        const T P = x * y * z;
        const T sP = rsqrt_t(P);
        const T iP = sP * sP, A0 = iP * sP;
        const T ua = x + y - z, ub = x + z - y, uc = y + z - x;
        const T N = ua * ub * uc;
        const T Ang = A0 * fma((T)0.375 * N, iP, (T)1);
        const T q = pow_pos(Bj.z * Bk.z * sR[tj * c.T + (tsk & 15)] * sP, a3);
        T f = 0, qf = 0;
        if (q < (T)1e30) {
            f = rcp_t(fma((T)6, q, (T)1));
            qf = alpha * q * f * f;  // x df/dx
        }
        const T cc = Bj.x * Bk.x * C6jk;
        const T c9 = s9 * cc * rsqrt_t(cc);
        const T e = c9 * Ang * f;
        const T Nx = ub * uc + ua * uc - ua * ub, Ny = ub * uc - ua * uc + ua * ub;
        const T h = (T)0.375 * iP;
        const T Ex = c9 * (A0 * fma(h, fma((T)-2.5 * N, ix, Nx), (T)-1.5 * ix) * f + Ang * qf * ix);
        const T Ey = c9 * (A0 * fma(h, fma((T)-2.5 * N, iy, Ny), (T)-1.5 * iy) * f + Ang * qf * iy);
        e_ += e;
        dn_ = fma((T)0.5 * e, Bj.y + Bk.y, dn_);
        const T gx = Ex * Aj.x, gy = Ex * Aj.y, gz = Ex * Aj.z;
        const T hx = Ey * Ak.x, hy = Ey * Ak.y, hz = Ey * Ak.z;
        fx_ += gx + hx; fy_ += gy + hy; fz_ += gz + hz;
        v_[0] = fma(gx, Aj.x, fma(hx, Ak.x, v_[0]));
        v_[1] = fma(gy, Aj.y, fma(hy, Ak.y, v_[1]));
        v_[2] = fma(gz, Aj.z, fma(hz, Ak.z, v_[2]));
        v_[3] = fma(gx, Aj.y, fma(hx, Ak.y, v_[3]));
        v_[4] = fma(gx, Aj.z, fma(hx, Ak.z, v_[4]));
        v_[5] = fma(gy, Aj.z, fma(hy, Ak.z, v_[5]));
    };
    auto flush = [&]() {
        aE.add(e_);
        aDn.add(dn_);
        aFx.add(fx_);
        aFy.add(fy_);
        aFz.add(fz_);
#pragma unroll
        for (int m = 0; m < 6; ++m) aV[m].add(v_[m]);
        e_ = dn_ = fx_ = fy_ = fz_ = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m) v_[m] = 0;
    };
    // queue the lanes' passing pairs; evaluate 32 whenever 32 are pending (the
    // FP32 partial sums then hold at most 16 triangles per lane)
    int nev = 0;
    auto push = [&](bool pass, int js, int ks) {
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) jk[(tail + __popc(m & lt)) & (kAtmQueue - 1)] = (js << 8) | ks;
        tail += __popc(m);
        __syncwarp();
        if (tail - head >= 32) {
            const int t = jk[(head + lane) & (kAtmQueue - 1)];
            eval(t >> 8, t & 255);
            head += 32;
            __syncwarp();
            if ((++nev & 15) == 0) flush();
        }
    };
    auto drain = [&]() {
        if (lane < tail - head) {
            const int t = jk[(head + lane) & (kAtmQueue - 1)];
            eval(t >> 8, t & 255);
        }
        head = tail;
        __syncwarp();
        flush();
    };
    // Candidate pairs are numbered and dealt to the lanes 32 at a time.  j = c / m
    // is formed as (c + 1/2) * (1/m) in FP32: c < 2^13 and (c + 1/2)/m lies at least
    // 1/(2m) >= 2^-8 from an integer, far above the rounding error (< 2^-10).
    //
    // every unordered pair of slots [base, base + n) once: (j, j + s mod n) for
    // s = 1 .. (n-1)/2, and for even n also (j, j + n/2) with j < n/2
    auto pairs_within = [&](int base, int n) {
        const int half = n >> 1, smax = (n - 1) >> 1;
        const int nc1 = n * smax, nc = nc1 + ((n & 1) ? 0 : half);
        const float inv = 1.0f / (float)(smax > 0 ? smax : 1);
        for (int c0 = 0; c0 < nc; c0 += 32) {
            const int ci = c0 + lane;
            bool pass = false;
            int js = 0, ks = 0;
            if (ci < nc) {
                int j, k;
                if (ci < nc1) {
                    j = (int)(((float)ci + 0.5f) * inv);
                    k = ci - j * smax + 1 + j;
                    if (k >= n) k -= n;
                } else {
                    j = ci - nc1;
                    k = j + half;
                }
                js = base + j;
                ks = base + k;
                pass = close(js, ks);
            }
            push(pass, js, ks);
        }
        drain();
    };
    // every pair (j, k), j in [baseA, baseA + na), k in [baseB, baseB + nb)
    auto pairs_across = [&](int baseA, int na, int baseB, int nb) {
        const int nc = na * nb;
        const float inv = 1.0f / (float)(nb > 0 ? nb : 1);
        for (int c0 = 0; c0 < nc; c0 += 32) {
            const int ci = c0 + lane;
            bool pass = false;
            int js = 0, ks = 0;
            if (ci < nc) {
                const int j = (int)(((float)ci + 0.5f) * inv);
                js = baseA + j;
                ks = baseB + ci - j * nb;
                pass = close(js, ks);
            }
            push(pass, js, ks);
        }
        drain();
    };

    if (cnt <= C) {
        pairs_within(0, stage(0, cnt, 0));
    } else {
        constexpr int H = C / 2;
        for (int a0 = 0; a0 < cnt; a0 += H) {
            __syncwarp();
            const int na = stage(a0, min(cnt, a0 + H), 0);
            pairs_within(0, na);
            for (int b0 = a0 + H; b0 < cnt; b0 += H) {
                __syncwarp();
                const int nb = stage(b0, min(cnt, b0 + H), H);
                pairs_across(0, na, H, nb);
            }
        }
    }
    // fixed-order warp sums (every lane ends with the totals); lanes 0-7 each
    // write one part of atom i's results
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        aE.xor_reduce(o);
        aDn.xor_reduce(o);
        aFx.xor_reduce(o);
        aFy.xor_reduce(o);
        aFz.xor_reduce(o);
#pragma unroll
        for (int m = 0; m < 6; ++m) aV[m].xor_reduce(o);
    }
    // (the mixed form rounds the totals to FP32: its F and dE/dn are FP32 anyway,
    // and the three-body site energy and virial are small parts of FP64 sums)
    if (lane == 0) {
        w.eat[p] += (double)(aE.total() * (T)(1.0 / 3.0));
        T4* fd = (T4*)w.Fd + p;
        const T4 f0 = *fd;
        *fd = T4{f0.x + (T)2 * aFx.total(), f0.y + (T)2 * aFy.total(), f0.z + (T)2 * aFz.total(), f0.w};
    } else if (lane == 1) {
        T* dn = (T*)w.dEdn + p;
        *dn += aDn.total();
    } else {
#pragma unroll
        for (int m = 0; m < 6; ++m)
            if (lane == 2 + m) w.wv[6 * p + m] -= (double)aV[m].total();
    }
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
    const int TB = 128;
    auto mark = [&](int k) {
        if (marks) cudaEventRecord(marks[k], st);
    };
    mark(0);
    if (w.Nr > 0)
        k_cn<MIXED, R><<<nblk(w.Nr, TB), TB, 0, st>>>(w, c, tb.rcpair, tb.exptab, tb.cnref, tb.nref, (const T*)tb.c6);
    mark(1);  // the weights (Eq. 3) are formed inside the CN pass
    mark(2);
    if (w.Nr > 0) {
        if (w_atom)
            k_disp<MIXED, R, true><<<nblk(w.Nr, TB), TB, c.T * c.T * sizeof(T4), st>>>(w, c, (const T4*)tb.pair);
        else
            k_disp<MIXED, R, false><<<nblk(w.Nr, TB), TB, c.T * c.T * sizeof(T4), st>>>(w, c, (const T4*)tb.pair);
    }
    mark(3);
    if (c.atm && w.Nr > 0)
        k_atm<MIXED, R><<<nblk(w.Nr, kAtmWarps), 32 * kAtmWarps, 0, st>>>(w, c, (const T*)tb.rtab);
    mark(4);
    if (w.Nr > 0) {
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
