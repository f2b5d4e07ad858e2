// d3gb_pair.cuh -- device helpers shared by the pair passes (d3gb_passes.cu),
// the optional three-body pass (d3gb_atm.cu) and the mixed form of the backward
// (d3gb_backward.cu): FP32 reciprocals with one Newton step, error-free sums,
// the per-precision real types, the per-thread view of an atom's position and
// its distance to a neighbour, the row loads of the per-atom weight vectors,
// and the double-single evaluation of the Eq. 4 counting function.
#pragma once
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

// s + err == a + b exactly when |a| >= |b| (Dekker's Fast2Sum); s, err may alias a, b
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& err) {
    const float t = a + b;
    err = b - (t - a);
    s = t;
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
        dist_exact(hq, lq, D, e, tq);
    }
    // the same from the neighbour's record, already loaded
    __device__ void dist_exact(const float4& hq, const float4& lq, float (&D)[3], float (&e)[3], int& tq) const {
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
//   r^2 = Sh + Sl (TwoProd/TwoSum), r = sqrt(r^2) with its correction term,
//   d = rc - r (TwoSum of the double-single rc and r), a = k1 d / r with one
//   residual step.
// Its absolute error is about 1e-11 over the range of pair distances (a CPU
// emulation against long double), far below the rounding of expf itself.
// Returns false when the pair is outside R_cn.
__device__ __forceinline__ bool cn_pair_precise(const Site<true>& S, int q, const float4* rrow, float k1, float rc2,
                                                double rc2d, float (&D)[3], float& r2, float& ah, float& al,
                                                float& rch, int& tq, float* rcl_out = nullptr,
                                                float* r2l_out = nullptr, float* y_out = nullptr,
                                                const float4* rec_q = nullptr) {
    float e[3];
    if (rec_q) S.dist_exact(rec_q[0], rec_q[1], D, e, tq);  // q's record, loaded by the caller
    else S.dist_exact(q, D, e, tq);
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
    fast_two_sum(Sh, Sl, Sh, Sl);  // normalise (|Sl| <= |Sh|)
    r2 = Sh;
    if (!S.inside(q, r2, rc2, rc2d)) return false;
    const float4 rc = rrow[tq & 15];  // rc hi, rc lo (, rc^2 hi, rc^2 lo)
    const float y = rsqrt_nr(Sh);  // 1/r to FP32 precision: enough for the correction terms below
    const float rh = Sh * y;
    const float rl = (fmaf(-rh, rh, Sh) + Sl) * (0.5f * y);
    float dh, de;
    two_sum(rc.x, -rh, dh, de);
    const float dl = de + (rc.y - rl);
    const float qh = dh * y;  // q = d / r
    const float ql = (fmaf(-qh, rh, dh) + dl - qh * rl) * y;
    ah = k1 * qh;
    al = fmaf(k1, qh, -ah) + k1 * ql;
    rch = rc.x;
    if (rcl_out) *rcl_out = rc.y;
    if (r2l_out) *r2l_out = Sl;
    if (y_out) *y_out = y;  // rsqrt_nr(r2), for chain_coef
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
    // k = rint(x/L) by the 1.5 2^23 trick (|x/L| < 2^13), from FP32 additions only
    const float kb = __fmul_rn(xh, kExpInvL) + 12582912.0f;
    const float kf = kb - 12582912.0f;
    const int k = __float_as_int(kb) - 0x4B400000;
    const float r1 = fmaf(-kf, kExpL1, xh);  // exact (see kExpL1)
    const float p2 = kf * kExpL2, p2e = fmaf(kf, kExpL2, -p2);
    float rh, re;
    two_sum(r1, -p2, rh, re);
    const float rl = ((re - p2e) - kf * kExpL3) + xl;
    // exp(r) - 1 = rh + s
    const float s = rl + rh * rl + rh * rh * fmaf(rh, fmaf(rh, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
    const int j = k & 63, m = k >> 6;  // k = 64 m + j, |m| <= 126
    const float2 T = __ldg(tab + j);
    const float ph = T.x * rh, pe = fmaf(T.x, rh, -ph);
    const float hh = T.x + ph, he = ph - (hh - T.x);  // |T.x| >= |ph|: Fast2Sum
    const float lo = he + pe + T.y + fmaf(T.x, s, T.y * rh);
    float th = hh + lo;
    float tl = lo - (th - hh);
    const float sc = __int_as_float((m + 127) << 23);  // 2^m, a normal FP32 number
    th *= sc;
    tl *= sc;
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


// Chain-rule coefficient f'(r)/r = -k1 rc f (1 - f) / r^3 of Eq. 4, formed in
// double-single and rounded once: 1/r from r^2 = r2 + r2l with one residual
// step, the exact rc = rch + rcl, f and 1 - f from cn_ds.
// (y0 = rsqrt_nr(r2), when the caller has it already)
__device__ __forceinline__ float chain_coef(const CnDS& z, float y0, float r2, float r2l, float rch, float rcl,
                                           float k1) {
    const float y2 = y0 * y0, y2e = fmaf(y0, y0, -y2);
    const float ry = fmaf(-r2, y2, 1.0f) - fmaf(r2, y2e, r2l * y2);
    const float yh = y0, yl = 0.5f * y0 * ry;
    float a2h, a2l, a3h, a3l, cfh, cfl, uh, ul, gh, gl;
    ds_mul(yh, yl, yh, yl, a2h, a2l);
    ds_mul(a2h, a2l, yh, yl, a3h, a3l);
    ds_mul(z.ch, z.cl, z.fh, z.fl, cfh, cfl);
    ds_mul(rch, rcl, cfh, cfl, uh, ul);
    ds_mul(uh, ul, a3h, a3l, gh, gl);
    return -k1 * (gh + gl);
}
__device__ __forceinline__ float chain_coef(const CnDS& z, float r2, float r2l, float rch, float rcl, float k1) {
    return chain_coef(z, rsqrt_nr(r2), r2, r2l, rch, rcl, k1);
}

}  // namespace
}  // namespace d3gb
