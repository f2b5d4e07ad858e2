// d3gb_pair.cuh -- device helpers shared by the pair passes (d3gb_passes.cu)
// and the optional three-body pass (d3gb_atm.cu): FP32 reciprocals with one
// Newton step, error-free sums, the per-precision real types, the per-thread
// view of an atom's position and its distance to a neighbour, and the row
// loads of the per-atom weight vectors.
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


}  // namespace
}  // namespace d3gb
