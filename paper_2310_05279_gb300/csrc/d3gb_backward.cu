// d3gb_backward.cu -- hand-written backward of (E, F) for damping refits.
// The handle's precision selects the form of the backward: FP64 dual numbers
// throughout, or (mixed form) the forward's mixed arithmetic for the values --
// the double-single Eq. 4 term and chain coefficient, float-float Eq. 3
// exponents, FP32 pair math on split positions -- with FP32 tangents.  GB300
// runs FP64 at 1/64 of the FP32 rate, so the FP64 passes bound the mixed form's
// time otherwise.
//
// For a loss L(E, F) with upstream gradients gE = dL/dE (per structure) and
// gF = dL/dF (per atom):
//   dL/dtheta = sum_s gE_s dE_s/dtheta + sum_i gF_i . dF_i/dtheta
//             = sum_s gE_s dE_s/dtheta - d/dtheta (d/dt E(x + t gF))
//   dL/dx     = -gE F + J^T gF,  J = dF/dx = -Hessian (symmetric), so J^T gF = d/dt F(x + t gF).
// Both second-order terms are directional derivatives along u = gF.  They are
// obtained by running the whole evaluation (Eq. 4 coordination numbers, Eq. 3
// weights, Eq. 2 pair terms with their analytic derivatives in s6, s8, a1, a2,
// and the coordination-number chain rule) once in dual numbers (value,
// derivative along u), in FP64.  The coordination numbers are recomputed and
// nothing is stored per pair.
#include "d3gb_pair.cuh"

namespace d3gb {

namespace {

struct Dual {
    double v, t;
};
__device__ __forceinline__ Dual dd(double v, double t = 0.0) { return Dual{v, t}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual{-a.v, -a.t}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.v * b.t + a.t * b.v}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return Dual{s * a.v, s * a.t}; }
__device__ __forceinline__ Dual operator+(Dual a, double s) { return Dual{a.v + s, a.t}; }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) {
    a.v += b.v;
    a.t += b.t;
    return a;
}
__device__ __forceinline__ Dual inv(Dual a) {
    const double r = 1.0 / a.v;
    return Dual{r, -a.t * r * r};
}
__device__ __forceinline__ Dual dexp(Dual a) {
    const double e = exp(a.v);
    return Dual{e, a.t * e};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
    const double s = sqrt(a.v);
    return Dual{s, 0.5 * a.t / s};
}

// per-atom dual arrays carved from one scratch block
struct BW {
    Dual* n;      // [Nr]
    Dual* W;      // [Nr][R]
    Dual* dW;     // [Nr][R]
    Dual* v;      // [Nr][T][R]
    Dual* dEdn;   // [Nr]
    Dual* F;      // [Nr][3]
    Dual* th;     // [Nr][4] dE_i/d(s6, s8, a1, a2), half pair sums
    double* xd;   // [(Nr + ghost_cap) * 3] tangent positions (bohr)
    double* sth;  // [B][8] per-structure dE/dtheta (value, tangent)
    // mixed form of the dispersion pass
    float* vf;    // [Nr][T][2 * RP]: R values of v padded to RP, then R tangents padded to RP
    float4* xdf;  // [Nr + ghost_cap] tangent positions as FP32
    float2* dEdnf;  // [Nr] dE/dn (value, tangent) as FP32 for the chain pass
    int RP;
};

__host__ __device__ inline BW carve(double* s, int64_t Nr, int64_t Ng, int T, int R, int B) {
    BW b;
    Dual* d = reinterpret_cast<Dual*>(s);
    b.n = d;
    d += Nr;
    b.W = d;
    d += Nr * R;
    b.dW = d;
    d += Nr * R;
    b.v = d;
    d += Nr * T * R;
    b.dEdn = d;
    d += Nr;
    b.F = d;
    d += 3 * Nr;
    b.th = d;
    d += 4 * Nr;
    double* x = reinterpret_cast<double*>(d);
    b.xd = x;
    x += 3 * (Nr + Ng);
    b.sth = x;
    x += 8 * (int64_t)B;
    b.RP = R <= 4 ? 4 : 8;
    x += (4 - ((reinterpret_cast<uintptr_t>(x) / sizeof(double)) & 3)) & 3;  // 32-byte alignment
    b.vf = reinterpret_cast<float*>(x);
    x += Nr * T * b.RP;
    b.xdf = reinterpret_cast<float4*>(x);
    x += 2 * (Nr + Ng);
    b.dEdnf = reinterpret_cast<float2*>(x);
    return b;
}

struct BConsts {
    double rc_disp2, rc_cn2, k1, k3, s6, s8;
    int T, R;
};

// tangent positions: x(t) = x + t * gF / bohr for real atoms, images follow their source
__global__ void kb_xdot(Work w, BW b, const double* __restrict__ gF, int64_t nt) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nt || q >= w.Nr + w.start_ghost[w.ncells]) return;
    const int src = rec_tsrc(w, q) >> 4;
    const int i = w.perm[src];
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        t[a] = gF[3 * (int64_t)i + a] * (1.0 / kBohrA);
        b.xd[3 * q + a] = t[a];
    }
    b.xdf[q] = make_float4((float)t[0], (float)t[1], (float)t[2], 0.0f);
}

__device__ __forceinline__ void ddist(const Work& w, const BW& b, int64_t p, int64_t q, Dual (&d)[3], Dual& r2) {
    const dbl4 x = w.pos64[p], y = w.pos64[q];
    d[0] = Dual{y.x - x.x, b.xd[3 * q] - b.xd[3 * p]};
    d[1] = Dual{y.y - x.y, b.xd[3 * q + 1] - b.xd[3 * p + 1]};
    d[2] = Dual{y.z - x.z, b.xd[3 * q + 2] - b.xd[3 * p + 2]};
    r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

__global__ void kb_cn(Work w, BW b, BConsts c) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const double rki = w.pos64[p].w;
    Dual n = dd(0.0);
    LV.for_each(0, cnt, [&](int q) {
        Dual d[3], r2;
        ddist(w, b, p, q, d, r2);
        if (!(r2.v < c.rc_cn2)) return;
        const Dual rinv = inv(dsqrt(r2));
        const double rc = rki + w.pos64[q].w;
        const Dual t = dexp(-c.k1 * (rc * rinv + (-1.0)));
        n += inv(t + 1.0);
    });
    b.n[p] = n;
}

template <int R>
__global__ void kb_weights(Work w, BW b, BConsts c, const double* __restrict__ cnref, const int* __restrict__ nref,
                           const double* __restrict__ c6) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const int t = rec_tsrc(w, p) & 15;
    const Dual n = b.n[p];
    const int nr = nref[t];
    Dual z[R], ex[R], L[R];
    double emax = -1e300;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        z[a] = n + (-cnref[t * R + a]);
        ex[a] = -c.k3 * (z[a] * z[a]);
        if (a < nr && ex[a].v > emax) emax = ex[a].v;
    }
    Dual sum = dd(0.0);
#pragma unroll
    for (int a = 0; a < R; ++a) {
        L[a] = a < nr ? dexp(ex[a] + (-emax)) : dd(0.0);
        sum += L[a];
    }
    const Dual is = inv(sum);
    Dual gbar = dd(0.0);
#pragma unroll
    for (int a = 0; a < R; ++a) {
        L[a] = L[a] * is;
        gbar += L[a] * (-2.0 * c.k3 * z[a]);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
        b.W[p * R + a] = L[a];
        b.dW[p * R + a] = L[a] * ((-2.0 * c.k3 * z[a]) - gbar);
    }
    for (int u = 0; u < c.T; ++u) {
        const double* cu = c6 + ((size_t)(u * c.T + t) * R) * R;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            Dual s = dd(0.0);
#pragma unroll
            for (int bb = 0; bb < R; ++bb) s += cu[a * R + bb] * L[bb];
            b.v[(p * c.T + u) * R + a] = s;
        }
    }
}

// pairb[ti*T + tj] = (R0, R, R0^2, 0) in bohr
template <int R>
__global__ void kb_disp(Work w, BW b, BConsts c, const dbl4* __restrict__ pairb) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const int ti = rec_tsrc(w, p) & 15;
    Dual Wi[R], dWi[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
        Wi[a] = b.W[p * R + a];
        dWi[a] = b.dW[p * R + a];
    }
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_disp + list_row(G.list_base_disp, p - G.atom_base, G.cap_disp)};
    const int cnt = w.cnt_disp[p];
    Dual dn = dd(0.0), F[3] = {dd(0.0), dd(0.0), dd(0.0)}, th[4] = {dd(0.0), dd(0.0), dd(0.0), dd(0.0)};
    LV.for_each(0, cnt, [&](int q) {
        Dual d[3], r2;
        ddist(w, b, p, q, d, r2);
        if (!(r2.v < c.rc_disp2)) return;
        const int tsq = rec_tsrc(w, q);
        const int src = tsq >> 4;
        const dbl4 pb = pairb[ti * c.T + (tsq & 15)];
        const double R0 = pb.x, Rd = pb.y, R0sq = pb.z;
        const double R2 = Rd * Rd, R4 = R2 * R2, R6 = R4 * R2, R8 = R4 * R4;
        Dual C6 = dd(0.0), dC6 = dd(0.0);
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const Dual vq = b.v[((int64_t)src * c.T + ti) * R + a];
            C6 += Wi[a] * vq;
            dC6 += dWi[a] * vq;
        }
        const Dual r4 = r2 * r2, r6 = r4 * r2, r8 = r4 * r4;
        const Dual i6 = inv(r6 + R6), i8 = inv(r8 + R8);
        const Dual t6 = c.s6 * i6, t8 = (c.s8 * R0sq) * i8;
        const Dual g = t6 + t8;
        dn += -(g * dC6);
        const Dual fc = C6 * (6.0 * (r4 * (t6 * i6)) + 8.0 * (r6 * (t8 * i8)));
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] += fc * d[a];
        // derivatives of this ordered instance's energy -C6 g (halved at the end)
        th[0] += -(C6 * i6);
        th[1] += -(R0sq * (C6 * i8));
        const Dual dR = C6 * ((c.s6 * 6.0 * R4 * Rd) * (i6 * i6) + (c.s8 * R0sq * 8.0 * R6 * Rd) * (i8 * i8));
        th[2] += R0 * dR;
        th[3] += dR;
    });
    b.dEdn[p] = dn;
#pragma unroll
    for (int a = 0; a < 3; ++a) b.F[3 * p + a] = F[a];
#pragma unroll
    for (int m = 0; m < 4; ++m) b.th[4 * p + m] = 0.5 * th[m];
}

// ---- mixed form of the dispersion pass of the backward: the same dual-number
// evaluation with FP32 pair arithmetic on the split positions (hi + lo) and
// FP32 tangents, FP32 partial sums promoted to FP64 every kChunk pairs and a
// compensated value part of dE/dn (it scales the chain-rule forces).
struct DF {
    float v, t;
};
__device__ __forceinline__ DF operator+(DF a, DF b) { return DF{a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ DF operator*(DF a, DF b) { return DF{a.v * b.v, fmaf(a.v, b.t, a.t * b.v)}; }
__device__ __forceinline__ DF operator*(float s, DF a) { return DF{s * a.v, s * a.t}; }
__device__ __forceinline__ DF finv(DF a) {
    const float r = 1.0f / a.v;
    return DF{r, -a.t * r * r};
}
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// compensated float-pair running sum (value h + l)
struct FF {
    float h = 0.f, l = 0.f;
    __device__ void add(float x) { acc_add(h, l, x); }
    __device__ double value() const { return (double)h + (double)l; }
};

template <int R>
__global__ void __launch_bounds__(128) kb_disp_mixed(Work w, BW b, BConsts c, const dbl4* __restrict__ pairb) {
    // per element pair: R^6, R^8, s8 R0^2, R0, 6 s6 R^4 R, 8 s8 R0^2 R^6 R, R0^2
    __shared__ float tab[kMaxTypes * kMaxTypes][8];
    for (int k = threadIdx.x; k < c.T * c.T; k += blockDim.x) {
        const dbl4 pb = pairb[k];
        const double Rd = pb.y, R2 = Rd * Rd, R4 = R2 * R2, R6 = R4 * R2, R8 = R4 * R4;
        tab[k][0] = (float)R6;
        tab[k][1] = (float)R8;
        tab[k][2] = (float)(c.s8 * pb.z);
        tab[k][3] = (float)pb.x;
        tab[k][4] = (float)(6.0 * c.s6 * R4 * Rd);
        tab[k][5] = (float)(8.0 * c.s8 * pb.z * R6 * Rd);
        tab[k][6] = (float)pb.z;
        tab[k][7] = 0.0f;
    }
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    float4 hp, lp;
    rec_load(w, p, hp, lp);
    const int ti = __float_as_int(hp.w) & 15;
    const float4 tp = b.xdf[p];
    DF Wi[R], dWi[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const Dual x = b.W[p * R + a], y = b.dW[p * R + a];
        Wi[a] = DF{(float)x.v, (float)x.t};
        dWi[a] = DF{(float)y.v, (float)y.t};
    }
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_disp + list_row(G.list_base_disp, p - G.atom_base, G.cap_disp)};
    const int cnt = w.cnt_disp[p];
    const float rc2f = (float)c.rc_disp2, s6 = (float)c.s6;
    constexpr int RP = R <= 4 ? 4 : 8;  // b.RP
    const int stride = c.T * 2 * RP;
    float dnh = 0.0f, dnl = 0.0f;
    // running sums as compensated float pairs (FP64 runs at 1/64 of the FP32 rate)
    FF dnt, Fv[3], Ft[3], thv[4], tht[4];
    for (int k0 = 0; k0 < cnt; k0 += kChunk) {
        const int k1e = min(cnt, k0 + kChunk);
        float dt = 0.0f, fv[3] = {0, 0, 0}, ft[3] = {0, 0, 0}, hv[4] = {0, 0, 0, 0}, ht[4] = {0, 0, 0, 0};
        LV.for_each(k0, k1e, [&](int q) {
            float4 hq, lq;
            rec_load(w, q, hq, lq);
            const float dx = (hq.x - hp.x) + (lq.x - lp.x), dy = (hq.y - hp.y) + (lq.y - lp.y),
                        dz = (hq.z - hp.z) + (lq.z - lp.z);
            const float r2v = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool in;
            if (fabsf(r2v - rc2f) > 4e-6f * rc2f) {
                in = r2v < rc2f;
            } else {  // within the FP32 error band of the cutoff: decide in FP64
                const dbl4 x = w.pos64[p], y = w.pos64[q];
                const double ex = y.x - x.x, ey = y.y - x.y, ez = y.z - x.z;
                in = ex * ex + ey * ey + ez * ez < c.rc_disp2;
            }
            if (!in) return;
            const int tsq = __float_as_int(hq.w);
            const float4 tq = b.xdf[q];
            const float ux = tq.x - tp.x, uy = tq.y - tp.y, uz = tq.z - tp.z;
            const DF r2 = DF{r2v, 2.0f * fmaf(dx, ux, fmaf(dy, uy, dz * uz))};
            const float* tb = tab[ti * c.T + (tsq & 15)];
            // the v row of q for type t_i: R values, then R tangents, each padded to RP (vector loads)
            const float* vq = b.vf + (int64_t)(tsq >> 4) * stride + ti * 2 * RP;
            float vv[R], vt[R];
            load_vec<R>(vq, vv);
            load_vec<R>(vq + RP, vt);
            DF C6 = DF{0.0f, 0.0f}, dC6 = DF{0.0f, 0.0f};
#pragma unroll
            for (int a = 0; a < R; ++a) {
                const DF v = DF{vv[a], vt[a]};
                C6 = C6 + Wi[a] * v;
                dC6 = dC6 + dWi[a] * v;
            }
            const DF r4 = r2 * r2, r6 = r4 * r2, r8 = r4 * r4;
            const DF i6 = finv(DF{r6.v + tb[0], r6.t}), i8 = finv(DF{r8.v + tb[1], r8.t});
            const DF t6 = s6 * i6, t8 = tb[2] * i8;
            const DF g = t6 + t8;
            const DF gd = g * dC6;
            float s, e;
            two_sum_f(dnh, -gd.v, s, e);
            dnh = s;
            dnl += e;
            dt -= gd.t;
            const DF fc = C6 * (6.0f * (r4 * (t6 * i6)) + 8.0f * (r6 * (t8 * i8)));
            fv[0] = fmaf(fc.v, dx, fv[0]); fv[1] = fmaf(fc.v, dy, fv[1]); fv[2] = fmaf(fc.v, dz, fv[2]);
            ft[0] += fmaf(fc.t, dx, fc.v * ux); ft[1] += fmaf(fc.t, dy, fc.v * uy); ft[2] += fmaf(fc.t, dz, fc.v * uz);
            // derivatives of this ordered instance's energy -C6 g in s6, s8, a1, a2 (halved at the end)
            const DF e6 = C6 * i6, e8 = C6 * i8;
            hv[0] -= e6.v; ht[0] -= e6.t;
            hv[1] = fmaf(-tb[6], e8.v, hv[1]); ht[1] = fmaf(-tb[6], e8.t, ht[1]);
            const DF dR = C6 * (tb[4] * (i6 * i6) + tb[5] * (i8 * i8));
            hv[2] = fmaf(tb[3], dR.v, hv[2]); ht[2] = fmaf(tb[3], dR.t, ht[2]);
            hv[3] += dR.v; ht[3] += dR.t;
        });
        dnt.add(dt);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Fv[a].add(fv[a]);
            Ft[a].add(ft[a]);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            thv[m].add(hv[m]);
            tht[m].add(ht[m]);
        }
    }
    b.dEdn[p] = Dual{(double)dnh + (double)dnl, dnt.value()};
    b.dEdnf[p] = make_float2(dnh + dnl, dnt.h + dnt.l);
#pragma unroll
    for (int a = 0; a < 3; ++a) b.F[3 * p + a] = Dual{Fv[a].value(), Ft[a].value()};
#pragma unroll
    for (int m = 0; m < 4; ++m) b.th[4 * p + m] = Dual{0.5 * thv[m].value(), 0.5 * tht[m].value()};
}

__global__ void kb_chain(Work w, BW b, BConsts c, const double* __restrict__ gE, double* __restrict__ dLdx) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const int s = w.sid[p];
    const StructGeo& G = w.geo[s];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const double rki = w.pos64[p].w;
    const Dual dni = b.dEdn[p];
    Dual F[3] = {b.F[3 * p], b.F[3 * p + 1], b.F[3 * p + 2]};
    LV.for_each(0, cnt, [&](int q) {
        Dual d[3], r2;
        ddist(w, b, p, q, d, r2);
        if (!(r2.v < c.rc_cn2)) return;
        const int src = rec_tsrc(w, q) >> 4;
        const Dual rinv = inv(dsqrt(r2));
        const double rc = rki + w.pos64[q].w;
        const Dual t = dexp(-c.k1 * (rc * rinv + (-1.0)));
        const Dual f = inv(t + 1.0);
        const Dual dfdr = (-c.k1 * rc) * (rinv * rinv * t * f * f);
        const Dual coef = (dni + b.dEdn[src]) * dfdr * rinv;
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] += coef * d[a];
    });
    if (dLdx) {
        const double u = kHartreeEV / kBohrA;
        const double ge = gE[s];
        const int i = w.perm[p];
#pragma unroll
        for (int a = 0; a < 3; ++a) dLdx[3 * (int64_t)i + a] = (-ge * F[a].v + F[a].t) * u;
    }
}

// ---- mixed form of the CN, weight and chain passes of the backward
// n (value) as in the forward's CN pass: double-single Eq. 4 term, integer
// count plus compensated complements; dn/dt = sum_q f'(r)/r (d . u), FP32
// (compensated), u the tangent of d.
__global__ void __launch_bounds__(128) kb_cn_mixed(Work w, BW b, Consts c, const float4* __restrict__ rcpair,
                                                   const float2* __restrict__ exptab) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const Site<true> S(w, p);
    const StructGeo& G = w.geo[w.sid[p]];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const float4* rrow = rcpair + (S.tsrc() & 15) * c.T;
    const float k1 = c.k1f, rc2 = c.rc_cn2f;
    const float4 tp = b.xdf[p];
    float nh = 0.f, nl = 0.f, th = 0.f, tl = 0.f;
    int nint = 0;
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
        const float4 uq = b.xdf[q];
        const float du = fmaf(D[0], uq.x - tp.x, fmaf(D[1], uq.y - tp.y, D[2] * (uq.z - tp.z)));
        const float ri = rsqrt_nr(r2);
        acc_add(th, tl, -k1 * rch * z.fh * z.ch * (ri * ri * ri) * du);
    });
    b.n[p] = Dual{(double)nint + (double)nh + (double)nl, (double)th + (double)tl};
}

// Weights (Eq. 3) as dual numbers: values with float-float exponents as in the
// forward, tangents in FP32; dW/dn = -2 k3 W_a sum_b W_b (nref_b - nref_a) from
// the table of reference differences (no cancellation against n).  The shift
// by the largest exponent is a constant: it cancels in the normalisation.
template <int R>
__global__ void __launch_bounds__(128) kb_weights_mixed(Work w, BW b, Consts c, const float2* __restrict__ cnref2,
                                                        const float* __restrict__ dcr, const int* __restrict__ nref,
                                                        const float* __restrict__ c6) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const int t = rec_tsrc(w, p) & 15;
    const Dual nd = b.n[p];
    const float Nh = (float)nd.v, Nl = (float)(nd.v - (double)Nh), nt = (float)nd.t;
    const int nr = nref[t];
    float xh[R], xl[R], xt[R];
    float mh = -3.0e38f, ml = 0.0f;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const float2 cr = cnref2[t * R + a];
        float zh, ze, zl;
        two_sum(Nh, -cr.x, zh, ze);
        two_sum(zh, ze + (Nl - cr.y), zh, zl);
        const float ph = zh * zh, pl = fmaf(zh, zh, -ph) + 2.0f * zh * zl;
        xh[a] = -c.k3h * ph;
        xl[a] = fmaf(-c.k3h, ph, -xh[a]) - c.k3h * pl - c.k3l * ph;
        xt[a] = -2.0f * c.k3f * zh * nt;
        if (a < nr && (xh[a] > mh || (xh[a] == mh && xl[a] > ml))) {
            mh = xh[a];
            ml = xl[a];
        }
    }
    DF L[R];
    DF sum = DF{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < R; ++a) {
        L[a] = DF{0.f, 0.f};
        if (a < nr) {
            float yh, ye, yl;
            two_sum(xh[a], -mh, yh, ye);
            two_sum(yh, ye + (xl[a] - ml), yh, yl);
            const float e = expf(yh) * (1.0f + yl);
            L[a] = DF{e, e * xt[a]};
        }
        sum = sum + L[a];
    }
    const DF is = finv(sum);
#pragma unroll
    for (int a = 0; a < R; ++a) L[a] = L[a] * is;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        DF sa = DF{0.f, 0.f};
        const float* dr = dcr + (t * R + a) * R;
#pragma unroll
        for (int bb = 0; bb < R; ++bb) sa = sa + dr[bb] * L[bb];
        const DF dW = (-2.0f * c.k3f) * (L[a] * sa);
        b.W[p * R + a] = Dual{(double)L[a].v, (double)L[a].t};
        b.dW[p * R + a] = Dual{(double)dW.v, (double)dW.t};
    }
    // v rows (values then tangents, each padded to RP = 4 or 8) as whole 16-byte stores
    constexpr int RP = R <= 4 ? 4 : 8;
    for (int u = 0; u < c.T; ++u) {
        const float* cu = c6 + ((size_t)(u * c.T + t) * R) * R;  // C6ref[u][t][a][b]
        float vv[RP], vt[RP];
#pragma unroll
        for (int a = 0; a < RP; ++a) {
            DF sv = DF{0.f, 0.f};
            if (a < R) {
#pragma unroll
                for (int bb = 0; bb < R; ++bb) sv = sv + cu[a * R + bb] * L[bb];
            }
            vv[a] = sv.v;
            vt[a] = sv.t;
        }
        float4* dst = reinterpret_cast<float4*>(b.vf + (p * c.T + u) * 2 * RP);
#pragma unroll
        for (int k = 0; k < RP / 4; ++k) {
            dst[k] = make_float4(vv[4 * k], vv[4 * k + 1], vv[4 * k + 2], vv[4 * k + 3]);
            dst[RP / 4 + k] = make_float4(vt[4 * k], vt[4 * k + 1], vt[4 * k + 2], vt[4 * k + 3]);
        }
    }
}

// Chain rule as dual numbers: the value of the coefficient f'(r)/r as in the
// forward's chain pass (double-single, rounded once), its tangent
// d(f'/r)/dt = -k1 rc [(1 - 2f) f' / r^3 - 3 f (1 - f) / r^4] (d . u) / r in FP32.
__global__ void __launch_bounds__(128) kb_chain_mixed(Work w, BW b, Consts c, const float4* __restrict__ rcpair,
                                                      const float2* __restrict__ exptab,
                                                      const double* __restrict__ gE, double* __restrict__ dLdx) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const Site<true> S(w, p);
    const int s = w.sid[p];
    const StructGeo& G = w.geo[s];
    const ListView LV{w.nbr_cn + list_row(G.list_base_cn, p - G.atom_base, G.cap_cn)};
    const int cnt = w.cnt_cn[p];
    const float4* rrow = rcpair + (S.tsrc() & 15) * c.T;
    const float k1 = c.k1f, rc2 = c.rc_cn2f;
    const float2 dnd = b.dEdnf[p];
    const float dni = dnd.x, dnit = dnd.y;
    const float4 tp = b.xdf[p];
    float fv[3] = {0.f, 0.f, 0.f}, ft[3] = {0.f, 0.f, 0.f};
    LV.for_each(0, cnt, [&](int q) {
        float D[3], r2, ah, al, rch, rcl, r2l;
        int tq;
        if (!cn_pair_precise(S, q, rrow, k1, rc2, c.rc_cn2, D, r2, ah, al, rch, tq, &rcl, &r2l)) return;
        const CnDS z = cn_ds(ah, al, exptab);
        const float g = chain_coef(z, r2, r2l, rch, rcl, k1);
        const float2 dqd = b.dEdnf[tq >> 4];
        const float dnq = dqd.x, dnqt = dqd.y;
        const float4 uq = b.xdf[q];
        const float u[3] = {uq.x - tp.x, uq.y - tp.y, uq.z - tp.z};
        const float du = fmaf(D[0], u[0], fmaf(D[1], u[1], D[2] * u[2]));
        const float ri = rsqrt_nr(r2), ri2 = ri * ri;
        const float f = z.fh, omf = z.ch;  // f and 1 - f
        const float fp = -k1 * rch * f * omf * ri2;  // f'(r)
        const float dgdr = -k1 * rch * ((1.0f - 2.0f * f) * fp * ri2 * ri - 3.0f * f * omf * ri2 * ri2);
        const float gt = dgdr * du * ri;
        const float cv = (dni + dnq) * g;
        const float ct = fmaf(dnit + dnqt, g, (dni + dnq) * gt);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            fv[a] = fmaf(cv, D[a], fv[a]);
            ft[a] = fmaf(ct, D[a], fmaf(cv, u[a], ft[a]));
        }
    });
    if (dLdx) {
        const double uc = kHartreeEV / kBohrA;
        const double ge = gE[s];
        const int i = w.perm[p];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const Dual Fd = b.F[3 * p + a];
            dLdx[3 * (int64_t)i + a] = (-ge * (Fd.v + (double)fv[a]) + (Fd.t + (double)ft[a])) * uc;
        }
    }
}

// per-structure sums of dE/dtheta (value and tangent), fixed order
__global__ void __launch_bounds__(256) kb_struct_sum(Work w, BW b) {
    const int s = blockIdx.x;
    const StructGeo& G = w.geo[s];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < G.natoms; k += blockDim.x) {
        const int64_t p = G.atom_base + k;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            acc[m] += b.th[4 * p + m].v;
            acc[4 + m] += b.th[4 * p + m].t;
        }
    }
    __shared__ double red[8][256];
#pragma unroll
    for (int m = 0; m < 8; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int m = 0; m < 8; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 8) b.sth[8 * s + threadIdx.x] = red[threadIdx.x][0];
}

// dL/dtheta = sum_s gE_s dE_s/dtheta - d/dtheta(dE/dt), in eV per unit parameter
__global__ void __launch_bounds__(256) kb_param_grad(BW b, int B, const double* __restrict__ gE, double* __restrict__ out) {
    double acc[4] = {0, 0, 0, 0};
    for (int s = threadIdx.x; s < B; s += blockDim.x) {
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] += gE[s] * b.sth[8 * s + m] - b.sth[8 * s + 4 + m];
    }
    __shared__ double red[4][256];
#pragma unroll
    for (int m = 0; m < 4; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int m = 0; m < 4; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0] * kHartreeEV;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int R>
cudaError_t backward_impl(const Work& w, const Consts& cc, const double* c6d, const dbl4* pairb, const double* cnref,
                          const int* nref, const Tabs& tbm, const double* gE, const double* gF, double* dLdp,
                          double* dLdx, double* scratch, int B, bool mixed, cudaStream_t st) {
    BW b = carve(scratch, w.Nr, w.ghost_cap, w.T, R, B);
    BConsts c{cc.rc_disp2, cc.rc_cn2, cc.k1, cc.k3, cc.s6, cc.s8, cc.T, R};
    const int TB = 128;
    if (w.Nr > 0) {
        // tangent positions for real atoms and every image actually built
        kb_xdot<<<nblk(w.Nr + w.ghost_cap, TB), TB, 0, st>>>(w, b, gF, w.Nr + w.ghost_cap);
        if (mixed) {
            kb_cn_mixed<<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, cc, tbm.rcpair, tbm.exptab);
            kb_weights_mixed<R><<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, cc, tbm.cnref2, tbm.dcr, tbm.nref,
                                                                (const float*)tbm.c6);
            kb_disp_mixed<R><<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, c, pairb);
            kb_chain_mixed<<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, cc, tbm.rcpair, tbm.exptab, gE, dLdx);
        } else {
            kb_cn<<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, c);
            kb_weights<R><<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, c, cnref, nref, c6d);
            kb_disp<R><<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, c, pairb);
            kb_chain<<<nblk(w.Nr, TB), TB, 0, st>>>(w, b, c, gE, dLdx);
        }
    }
    kb_struct_sum<<<B, 256, 0, st>>>(w, b);
    if (dLdp) kb_param_grad<<<1, 256, 0, st>>>(b, B, gE, dLdp);
    return cudaGetLastError();
}

}  // namespace

int64_t backward_scratch_doubles(const Work& w, int B) {
    const int64_t Nr = w.Nr, Ng = w.ghost_cap;
    const int64_t duals = Nr * (1 + 2 * (int64_t)w.R + (int64_t)w.T * w.R + 1 + 3 + 4);
    const int64_t rp = w.R <= 4 ? 4 : 8;
    // duals, tangent positions, per-structure sums, FP32 v rows and tangents (+ alignment)
    return 2 * duals + 3 * (Nr + Ng) + 8 * (int64_t)B + Nr * (int64_t)w.T * rp + 2 * (Nr + Ng) + Nr + 64;
}

cudaError_t launch_backward(const Work& w, const Consts& c, const double* c6d, const dbl4* pairb,
                            const double* cnref, const int* nref, const Tabs& tbm, const double* dLdE,
                            const double* dLdF, double* dLdp, double* dLdx, double* scratch, int B, bool mixed,
                            cudaStream_t st) {
#define D3_BWD(RR) \
    return backward_impl<RR>(w, c, c6d, pairb, cnref, nref, tbm, dLdE, dLdF, dLdp, dLdx, scratch, B, mixed, st)
    switch (c.R) {
        case 1: D3_BWD(1);
        case 2: D3_BWD(2);
        case 3: D3_BWD(3);
        case 4: D3_BWD(4);
        case 5: D3_BWD(5);
        case 6: D3_BWD(6);
        default: D3_BWD(7);
    }
#undef D3_BWD
}

}  // namespace d3gb
