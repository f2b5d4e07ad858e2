// d3gb_cluster.cu -- dispersion pass of the mixed form over cluster half lists
// (arXiv 2310.05279, Sec. II A, Eq. 2 with the C6 of Eq. 3).
//
// Eq. 2 sums every unordered pair instance once (the 1/2 over ordered pairs).
// This pass evaluates each instance exactly once and adds its contributions to
// both atoms:
//   * one warp per cluster of 8 consecutive sorted real atoms (the i atoms);
//     lane = i + 8 j, so each lane keeps one i atom in registers for the whole
//     list and each step evaluates 8 i x 4 list entries (32 pairs);
//   * the four j records of a step are each read by 8 lanes at one address
//     (broadcast loads instead of per-lane gathers);
//   * a step whose 32 pairs all lie outside R_pot is skipped as a whole;
//   * the j-side sums of a step (force, dE/dn_j, half the pair energy) are
//     reduce-scattered over the 8 lanes of each j and added to per-atom
//     accumulators as 64-bit fixed-point integers (2^-40 Hartree or
//     Hartree/bohr).  Integer addition is associative, so the totals are the
//     same whatever order the warps run in: the pass is deterministic;
//   * the i-side sums stay in registers and are added the same way at the end;
//     the virial is summed per cluster (only its total is needed).
// The C6 coefficient and both of its coordination-number derivatives come from
// per-atom projections formed with the Eq. 3 weights:
//   C6_ij       = sum_a W_ia v_j^(t_i)_a     v_j^(t)_a  = sum_b C6ref[t][t_j][a][b] W_jb
//   dC6_ij/dn_i = sum_a dW_ia v_j^(t_i)_a
//   dC6_ij/dn_j = sum_a W_ia dv_j^(t_i)_a    dv_j^(t)_a = sum_b C6ref[t][t_j][a][b] dW_jb
#include "d3gb_pair.cuh"

namespace d3gb {

namespace {

constexpr double kUnfix = 1.0 / 1099511627776.0;  // Hartree (or Hartree/bohr) per fixed-point unit, 2^-40

// round(v * 2^40) as a two's-complement 64-bit integer, for |v| < 2^14, from FP32
// additions and integer operations only (conversions from FP32 to integers run on
// the FP64 pipe of this GPU): v 2^40 = h 2^32 + m 2^16 + n with each of h, m, n
// rounded by the 1.5 2^23 trick (exact for magnitudes below 2^22) and every
// remainder formed exactly.  A larger (or non-finite) |v| sets the flag bad (the
// caller turns it into ST_SUM_RANGE; the returned value is then meaningless).
__device__ __forceinline__ int magic_rint(float x, float& xr) {  // rint(x) for |x| < 2^22, and its float value
    const float f = x + 12582912.0f;
    xr = f - 12582912.0f;
    return __float_as_int(f) - 0x4B400000;
}
__device__ __forceinline__ unsigned long long fix40(float v, bool& bad) {
    bad |= !(fabsf(v) < 16384.0f);
    float hr, mr;
    const float a = v * 256.0f;                       // v 2^8
    const int h = magic_rint(a, hr);
    const float r1 = (a - hr) * 65536.0f;              // exact, |r1| <= 2^15
    const int m = magic_rint(r1, mr);
    const float r2 = (r1 - mr) * 65536.0f;             // exact, |r2| <= 2^15
    float nr;
    const int n = magic_rint(r2, nr);
    return ((unsigned long long)(long long)h << 32) + (unsigned long long)((long long)m << 16) +
           (unsigned long long)(long long)n;
}

__device__ __forceinline__ void red_add(unsigned long long* a, unsigned long long x) {
    atomicAdd(a, x);  // result unused: a reduction, no return trip
}
// the same under a predicate, without a branch around it
__device__ __forceinline__ void red_add_if(bool p, unsigned long long* a, unsigned long long x) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.relaxed.gpu.global.add.u64 [%0], %1;\n\t}"
                 :: "l"(a), "l"(x), "r"((unsigned)p) : "memory");
}

// Data of one list entry for the lane's step: the neighbour's split position and
// its rows v^(t_i), dv^(t_i) (its own, or its source atom's); q = -1 past the end
// of the list.
template <int R>
struct JData {
    float4 h, l;
    float v[R], dv[R];
    int q;
};

template <int R>
__device__ __forceinline__ void load_j(const Work& w, const float* __restrict__ vdb, int rows, int q, int src,
                                       JData<R>& J) {
    J.q = q;
    rec_load(w, q >= 0 ? q : 0, J.h, J.l);
    const float* r = vdb + (int64_t)(src >= 0 ? src : 0) * rows;
    load_vec<R>(r, J.v);
    load_vec<R>(r + (R <= 4 ? 4 : 8), J.dv);
}

// The lane's i atom and its running sums.  step2() evaluates two steps (8 i atoms x
// 4 list entries each) written as one block, so that their dependency chains
// interleave.
template <int R, bool SITE>
struct ClusterPass {
    Site<true> S;
    float Wi[R], dWi[R];
    const float4* trow;
    int pthr;             // a pair is used when q > pthr: later clusters, images, own cluster after i
    float rc2, band;
    double rc2d;
    int b0, b1, il, fshift;
    unsigned long long* acc;
    bool bad = false;     // a fixed-point value out of range (ST_SUM_RANGE at the end)
    unsigned npairs = 0;  // used pairs of the warp (warp-uniform)
    // running sums of the lane's i
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float dnc = 0.f, dnh = 0.f, dnl = 0.f;            // dE/dn_i: chunk partial and compensated sum
    float ec = 0.f, Eh = 0.f, El = 0.f;               // energy (half pair energies for SITE, else whole)
    float sv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};     // virial chunk partials (of -fc d (x) d)
    float Vh[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Vl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

    __device__ ClusterPass(const Work& w, int64_t p) : S(w, p) {}

    __device__ __forceinline__ void chunk() {
        acc_add(dnh, dnl, dnc);
        acc_add(Eh, El, ec);
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            acc_add(Vh[m], Vl[m], sv[m]);
            sv[m] = 0.f;
        }
        dnc = ec = 0.f;
    }

    __device__ __forceinline__ void pair_vec(const JData<R>& J, float& dx, float& dy, float& dz, float& r2,
                                             bool& use, bool& near) const {
        dx = (J.h.x - S.h.x) + (J.l.x - S.l.x);
        dy = (J.h.y - S.h.y) + (J.l.y - S.l.y);
        dz = (J.h.z - S.h.z) + (J.l.z - S.l.z);
        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool listed = J.q > pthr;
        near = listed && fabsf(r2 - rc2) <= band;
        use = listed && r2 < rc2;
    }

    // pair terms of a used pair (zero weight otherwise) and the i-side sums; returns
    // the j-side values: force on j (nt), dE/dn_j, energy share
    __device__ __forceinline__ void pair(const JData<R>& J, float dx, float dy, float dz, float r2, bool use,
                                         float& ntx, float& nty, float& ntz, float& dnj, float& e) {
        const float4 tb = trow[__float_as_int(J.h.w) & 15];
        float C6 = 0.f, dC6i = 0.f, dC6j = 0.f;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            C6 = fmaf(Wi[a], J.v[a], C6);
            dC6i = fmaf(dWi[a], J.v[a], dC6i);
            dC6j = fmaf(Wi[a], J.dv[a], dC6j);
        }
        const float r4 = r2 * r2, r6 = r4 * r2, r8 = r4 * r4;
        const float d6 = r6 + tb.x, d8 = r8 + tb.y;
        const float pinv = rcp_approx(d6 * d8);
        const float i6 = d8 * pinv, i8 = d6 * pinv;
        const float t6 = tb.z * i6, t8 = tb.w * i8;
        const float mg = use ? -(t6 + t8) : 0.f;  // de/dC6 of a used pair, zero otherwise
        e = SITE ? 0.5f * (mg * C6) : mg * C6;   // half (SITE) or whole pair energy
        // F_i = -(de/dr) d/r = -nfc d, nfc = -C6 (6 r^4 t6 i6 + 8 r^6 t8 i8); the force on j is nfc d
        const float nfc = use ? -C6 * fmaf(6.0f * r4, t6 * i6, 8.0f * r6 * (t8 * i8)) : 0.f;
        ntx = nfc * dx; nty = nfc * dy; ntz = nfc * dz;
        fx -= ntx; fy -= nty; fz -= ntz;
        dnc = fmaf(mg, dC6i, dnc);
        ec += e;
        sv[0] = fmaf(ntx, dx, sv[0]); sv[1] = fmaf(nty, dy, sv[1]); sv[2] = fmaf(ntz, dz, sv[2]);
        sv[3] = fmaf(ntx, dy, sv[3]); sv[4] = fmaf(ntx, dz, sv[4]); sv[5] = fmaf(nty, dz, sv[5]);
        dnj = mg * dC6j;
    }

    // j side: reduce-scatter (force on j, dE/dn_j) over the 8 lanes of j (lane il < 4 ends
    // with component 2 b0 + b1; with SITE lane 4 with the energy) and add it to j's sums
    __device__ __forceinline__ void flush_j(int tsq, unsigned um, float ntx, float nty, float ntz, float dnj,
                                            float e) {
        const float k0v = (b0 ? ntz : ntx) + __shfl_xor_sync(0xffffffffu, b0 ? ntx : ntz, 1);
        const float k1v = (b0 ? dnj : nty) + __shfl_xor_sync(0xffffffffu, b0 ? nty : dnj, 1);
        float mv = (b1 ? k1v : k0v) + __shfl_xor_sync(0xffffffffu, b1 ? k0v : k1v, 2);
        mv += __shfl_xor_sync(0xffffffffu, mv, 4);
        if constexpr (SITE) {
            float ej = e;
            ej += __shfl_xor_sync(0xffffffffu, ej, 1);
            ej += __shfl_xor_sync(0xffffffffu, ej, 2);
            ej += __shfl_xor_sync(0xffffffffu, ej, 4);
            if (il == 4) mv = ej;
        }
        const unsigned long long x = fix40(mv, bad);
        red_add_if(il < (SITE ? 5 : 4) && ((um >> fshift) & 0xffu),  // some pair of this j was used
                   acc + 8 * (int64_t)(tsq >> 4) + (il < 4 ? 2 * b0 + b1 : 4), x);
    }

    // j side of two steps at once (without SITE): the first two levels of each
    // reduce-scatter leave partial sums of one component per lane in each half of
    // the 8 lanes of j; one exchange between the halves then completes step A's
    // component on lanes il < 4 and step B's on lanes il >= 4 (the same additions as
    // flush_j), so every lane adds one value
    __device__ __forceinline__ float part_j(float ntx, float nty, float ntz, float dnj) const {
        const float k0v = (b0 ? ntz : ntx) + __shfl_xor_sync(0xffffffffu, b0 ? ntx : ntz, 1);
        const float k1v = (b0 ? dnj : nty) + __shfl_xor_sync(0xffffffffu, b0 ? nty : dnj, 1);
        return (b1 ? k1v : k0v) + __shfl_xor_sync(0xffffffffu, b1 ? k0v : k1v, 2);
    }
    __device__ __forceinline__ void flush_j2(int tsa, unsigned uma, float pa, int tsb, unsigned umb, float pb) {
        const bool hi = il >= 4;
        const float mv = (hi ? pb : pa) + __shfl_xor_sync(0xffffffffu, hi ? pa : pb, 4);
        const unsigned um = hi ? umb : uma;
        const int tsq = hi ? tsb : tsa;
        const unsigned long long x = fix40(mv, bad);
        red_add_if((um >> fshift) & 0xffu, acc + 8 * (int64_t)(tsq >> 4) + 2 * b0 + b1, x);
    }

    __device__ __forceinline__ void step2(const JData<R>& A, const JData<R>& B) {
        float ax, ay, az, ar2, bx, by, bz, br2;
        bool ause, anear, buse, bnear;
        pair_vec(A, ax, ay, az, ar2, ause, anear);
        pair_vec(B, bx, by, bz, br2, buse, bnear);
        if (__any_sync(0xffffffffu, anear || bnear)) {  // a pair within the FP32 error band of R_pot
            if (anear) ause = S.inside(A.q, ar2, rc2, rc2d);
            if (bnear) buse = S.inside(B.q, br2, rc2, rc2d);
        }
        const unsigned uma = __ballot_sync(0xffffffffu, ause), umb = __ballot_sync(0xffffffffu, buse);
        if ((uma | umb) == 0u) return;
        npairs += __popc(uma) + __popc(umb);
        float atx, aty, atz, adn, ae, btx, bty, btz, bdn, be;
        pair(A, ax, ay, az, ar2, ause, atx, aty, atz, adn, ae);
        pair(B, bx, by, bz, br2, buse, btx, bty, btz, bdn, be);
        if constexpr (SITE) {
            flush_j(__float_as_int(A.h.w), uma, atx, aty, atz, adn, ae);
            flush_j(__float_as_int(B.h.w), umb, btx, bty, btz, bdn, be);
        } else {
            const float pa = part_j(atx, aty, atz, adn), pb = part_j(btx, bty, btz, bdn);
            flush_j2(__float_as_int(A.h.w), uma, pa, __float_as_int(B.h.w), umb, pb);
        }
    }
};

// IMGSRC: image atoms have no rows of their own; each list entry's source atom is
// resolved once per block of 32 entries (from the image's compact record).
// The bound (128, 3) holds every instantiation to 168 registers, so that three
// 128-thread blocks (12 warps) stay resident per SM whatever R is.
template <int R, bool SITE, bool IMGSRC>
__global__ void __launch_bounds__(128, 3) k_disp_cl(Work w, Consts c, const float4* __restrict__ pair_tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* tab = reinterpret_cast<float4*>(smem_raw);
    for (int k = threadIdx.x; k < c.T * c.T; k += blockDim.x) tab[k] = pair_tab[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, il = lane & 7, js = lane >> 3;
    const int64_t I = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (I >= w.ncl) return;  // whole warps
    const int s = w.clu_sid[I];
    const StructGeo& G = w.geo[s];
    const int64_t p0 = G.atom_base + (I - G.clu_base) * kClusterAtoms;
    const int64_t rem = G.atom_base + G.natoms - p0;
    const int nI = rem < kClusterAtoms ? (int)rem : kClusterAtoms;
    const bool ilive = il < nI;
    const int64_t p = p0 + (ilive ? il : 0);  // lanes past the cluster's end mirror its first atom, unused
    ClusterPass<R, SITE> P(w, p);
    const int ti = P.S.tsrc() & 15;
    load_vec<R>((const float*)w.W + p * c.RP, P.Wi);
    load_vec<R>((const float*)w.dW + p * c.RP, P.dWi);
    P.trow = tab + ti * c.T;
    P.pthr = ilive ? (int)p : 0x7fffffff;
    P.rc2 = c.rc_disp2f;
    P.band = 4e-6f * c.rc_disp2f;  // FP32 error band of the cutoff test (as Site::inside)
    P.rc2d = c.rc_disp2;
    P.b0 = lane & 1;
    P.b1 = (lane >> 1) & 1;
    P.il = il;
    P.fshift = lane & 24;
    P.acc = w.acc;
    constexpr int RPc = R <= 4 ? 4 : 8;
    const int rows = c.T * 2 * RPc;          // floats of v/dv rows per atom
    const float* vdb = w.vd + ti * 2 * RPc;  // the rows for partner type t_i
    const int* row = w.nbr_cl + G.list_base_cl + (I - G.clu_base) * (int64_t)G.cap_cl;
    const int cnt = w.cnt_cl[I];
    const int nsteps = (cnt + 3) >> 2;
    // list entries of steps 8b..8b+7 (block b) come from one coalesced load, lane k
    // holding entry 32b + k, together with the entry's source atom (itself for a real
    // atom; with IMGSRC, an image's source from its compact record), a block ahead.
    // The neighbour data of the next two steps is loaded while two steps compute.
    // Whole blocks are processed: entries past the end of the list are -1 (unused).
    const int nr = (int)w.Nr;
    auto src_of = [&](int q) { return IMGSRC && q >= nr ? (__float_as_int(__ldg(&w.hi[q].w)) >> 4) : q; };
    int qa = lane < cnt ? __ldg(row + lane) : -1;
    int qb = 32 + lane < cnt ? __ldg(row + 32 + lane) : -1;
    int sa = src_of(qa), sb = src_of(qb);
    // this lane's entry of step s (0..7) of the current block
    auto load = [&](int st, JData<R>& J) {
        const int from = (st << 2) + js;
        const int q = __shfl_sync(0xffffffffu, qa, from);
        const int src = IMGSRC ? __shfl_sync(0xffffffffu, sa, from) : q;
        load_j<R>(w, vdb, rows, q, src, J);
    };
    JData<R> A, B, C, D;
    load(0, A);
    load(1, B);
    const int nblocks = (nsteps + 7) >> 3;
    for (int b = 0; b < nblocks; ++b) {
        load(2, C);
        load(3, D);
        P.step2(A, B);
        load(4, A);
        load(5, B);
        P.step2(C, D);
        load(6, C);
        load(7, D);
        P.step2(A, B);
        // next block: its entries become current, the one after is loaded
        qa = qb;
        sa = sb;
        const int k = 32 * (b + 2) + lane;
        qb = k < cnt ? __ldg(row + k) : -1;
        sb = src_of(qb);
        load(0, A);
        load(1, B);
        P.step2(C, D);
        if (b & 1) P.chunk();  // every 16 steps
    }
    P.chunk();
    if (lane == 0 && w.npairs) atomicAdd(w.npairs, (unsigned long long)P.npairs);
    // i side: sum the 4 lanes of each i (fixed order) and add to the accumulators
    float fx = P.fx, fy = P.fy, fz = P.fz, dnh = P.dnh, dnl = P.dnl, Eh = P.Eh, El = P.El;
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
        dnh += __shfl_xor_sync(0xffffffffu, dnh, o);
        dnl += __shfl_xor_sync(0xffffffffu, dnl, o);
        if (SITE) {
            Eh += __shfl_xor_sync(0xffffffffu, Eh, o);
            El += __shfl_xor_sync(0xffffffffu, El, o);
        }
    }
    unsigned long long* acc = w.acc;
    if (js == 0 && ilive) {
        unsigned long long* ai = acc + 8 * p;
        red_add(ai + 0, fix40(fx, P.bad));
        red_add(ai + 1, fix40(fy, P.bad));
        red_add(ai + 2, fix40(fz, P.bad));
        red_add(ai + 3, fix40(dnh, P.bad) + fix40(dnl, P.bad));
        if (SITE) red_add(ai + 4, fix40(Eh, P.bad) + fix40(El, P.bad));
    }
    if (P.bad) atomicOr(w.status, ST_SUM_RANGE);
    // the cluster's virial, -sum_pairs fc d (x) d (the partials are of nfc d (x) d), and
    // without SITE its energy: compensated float pairs summed over the warp in a fixed
    // order, then lane m converts value m to FP64 (one conversion for all seven: the
    // FP64 pipe takes a whole warp instruction however few lanes are active) and
    // writes it on the cluster's first atom; zero on the others
    float hm = 0.f, lm = 0.f;
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        if (m == 6 && SITE) break;
        float h = m < 6 ? P.Vh[m] : P.Eh, l = m < 6 ? P.Vl[m] : P.El;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            h += __shfl_xor_sync(0xffffffffu, h, o);
            l += __shfl_xor_sync(0xffffffffu, l, o);
        }
        if (lane == m) {
            hm = h;
            lm = l;
        }
    }
    const double Vm = (double)hm + (double)lm;
    if (lane < 6) w.wv[6 * p0 + lane] = Vm;
    if (!SITE && lane == 6) w.eat[p0] = Vm;
    if (js == 0 && ilive && il > 0) {
        double* wv = w.wv + 6 * p;
#pragma unroll
        for (int m = 0; m < 6; ++m) wv[m] = 0.0;
        if (!SITE) w.eat[p] = 0.0;
    }
}

// Per atom: the fixed-point totals of the dispersion pass into the arrays the
// chain pass (and the optional three-body pass) read.
__global__ void __launch_bounds__(256) k_disp_fin(Work w, int site) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.Nr) return;
    const ulonglong2* a = reinterpret_cast<const ulonglong2*>(w.acc + 8 * p);
    const ulonglong2 a01 = a[0], a23 = a[1], a45 = a[2];
    const double fx = (double)(long long)a01.x * kUnfix, fy = (double)(long long)a01.y * kUnfix;
    const double fz = (double)(long long)a23.x * kUnfix, dn = (double)(long long)a23.y * kUnfix;
    ((float4*)w.Fd)[p] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
    ((float*)w.dEdn)[p] = (float)dn;
    if (site) w.eat[p] = (double)(long long)a45.x * kUnfix;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_disp_cl(const Work& w, const Consts& c, const void* pair_tab, bool site, cudaStream_t st) {
    if (w.Nr == 0) return cudaGetLastError();
    // (with vd_images the CN pass has written the image atoms' rows of v and dv)
    if (w.ncl > 0) {
        const int TB = w.blk_disp;  // 64 or 128 threads: 2 or 4 clusters per block
        const unsigned grid = nblk(w.ncl, TB / 32);
        const size_t sm = (size_t)c.T * c.T * sizeof(float4);
        const float4* pt = (const float4*)pair_tab;
#define D3_CL(RR)                                                                  \
    if (w.vd_images) {                                                             \
        if (site) k_disp_cl<RR, true, false><<<grid, TB, sm, st>>>(w, c, pt);     \
        else k_disp_cl<RR, false, false><<<grid, TB, sm, st>>>(w, c, pt);         \
    } else {                                                                       \
        if (site) k_disp_cl<RR, true, true><<<grid, TB, sm, st>>>(w, c, pt);      \
        else k_disp_cl<RR, false, true><<<grid, TB, sm, st>>>(w, c, pt);          \
    }                                                                              \
    break
        switch (c.R) {
            case 1: D3_CL(1);
            case 2: D3_CL(2);
            case 3: D3_CL(3);
            case 4: D3_CL(4);
            case 5: D3_CL(5);
            case 6: D3_CL(6);
            default: D3_CL(7);
        }
#undef D3_CL
    }
    k_disp_fin<<<nblk(w.Nr, 256), 256, 0, st>>>(w, site ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace d3gb
