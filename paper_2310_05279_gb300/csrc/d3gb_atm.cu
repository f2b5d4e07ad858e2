// d3gb_atm.cu -- optional three-body (triple-dipole) pass of the D3 model.
// Not part of the paper's model (Sec. II A leaves it out); d3_set_three_body
// enables it.  It runs between the dispersion pass and the chain pass and adds
// into their per-atom results, so its dependence on the coordination numbers
// reaches the forces through the chain pass.
#include "d3gb_pair.cuh"

namespace d3gb {

namespace {

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
// unordered pairs of them, numbered as (j, j + s mod n) for s = 1 .. n/2 and
// dealt to the lanes 32 at a time, so every pair is tested once.  Most pairs
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
                q = __ldg(row + list_off(k));
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
                // FP32: Newton-refined reciprocals instead of IEEE divisions
                const T gC6 = MIXED ? dC6 * rcp_t(C6) : dC6 / C6;
                sb[slot] = T4{C6, gC6, sR[ti * c.T + (tq & 15)], rcp_t(r2)};
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

}  // namespace

cudaError_t launch_atm(const Work& w, const Consts& c, bool mixed, const void* rtab, cudaStream_t st) {
    if (w.Nr == 0) return cudaGetLastError();
    const unsigned grid = (unsigned)((w.Nr + kAtmWarps - 1) / kAtmWarps);
#define D3_ATM(M, RR) k_atm<M, RR><<<grid, 32 * kAtmWarps, 0, st>>>(w, c, (const typename Real<M>::T*)rtab); break
    if (mixed) {
        switch (c.R) {
            case 1: D3_ATM(true, 1);
            case 2: D3_ATM(true, 2);
            case 3: D3_ATM(true, 3);
            case 4: D3_ATM(true, 4);
            case 5: D3_ATM(true, 5);
            case 6: D3_ATM(true, 6);
            default: D3_ATM(true, 7);
        }
    } else {
        switch (c.R) {
            case 1: D3_ATM(false, 1);
            case 2: D3_ATM(false, 2);
            case 3: D3_ATM(false, 3);
            case 4: D3_ATM(false, 4);
            case 5: D3_ATM(false, 5);
            case 6: D3_ATM(false, 6);
            default: D3_ATM(false, 7);
        }
    }
#undef D3_ATM
    return cudaGetLastError();
}

}  // namespace d3gb
