// d3gb_api.cu -- C ABI, handle and per-geometry plan of the D3(BJ) library.
//
// A plan holds everything that depends only on the batch geometry (offsets,
// cells, pbc): the per-structure cell grids and image ranges, and device
// buffers sized for them.  The first call for a new geometry runs the
// neighbour build once synchronously to measure image and neighbour counts
// and regrows the buffers if the estimates were short; every later call with
// the same geometry only enqueues kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/d3gb.h"
#include "d3gb_internal.cuh"

namespace d3gb {
cudaError_t launch_build_impl(const Work& w, const double* pos, const int32_t* types, const double* rk_tab,
                              int* bsum, cudaStream_t st, cudaEvent_t* lmarks = nullptr);
int64_t scan_scratch_ints(int64_t ncells);
cudaError_t launch_backward(const Work& w, const Consts& c, const double* c6d, const dbl4* paird,
                            const double* cnref, const int* nref, const Tabs& tbm, const double* dLdE,
                            const double* dLdF, double* dLdp, double* dLdx, double* scratch, int B, bool mixed,
                            cudaStream_t st);
int64_t backward_scratch_doubles(const Work& w, int B);
}  // namespace d3gb

using namespace d3gb;

namespace {

constexpr int kWindowCells = 3;  // list radius spans at most this many cells per axis
// profiled stages: build, CN (with the Eq. 3 weights), weights, dispersion, three-body, chain, finalize
// (d3_profile_read), and the list-builder kernel inside the build (d3_profile_stage)
constexpr int kStages = 7;
constexpr int kStagesAll = 8;
constexpr int kEvents = kStages + 3;  // kStages + 1 stage boundaries, 2 around the list builder

// Launch shapes: threads per block of the CN, dispersion and chain passes, and
// list-builder blocks per SM.  The defaults are the fastest shapes on the
// 128 x 1440 bilayer scan; the autotuner measures the candidates once per size
// class.  Every candidate gives bit-identical results: the passes run one
// thread per atom with per-thread sums, and each list row is written by one
// lane in a fixed walk order whichever warp takes it.
constexpr int32_t kDefaultShape[4] = {64, 128, 128, 16};
constexpr int32_t kBlockCand[2] = {64, 128};
constexpr int32_t kBuildCand[2] = {8, 16};
constexpr int64_t kTuneMinAtoms = 16384;  // below this launch overhead decides, not the shape
constexpr int kTuneReps = 3;

struct DevBuf {
    std::vector<void*> ptrs;
    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back((void*)*p);
        return e;
    }
    void release() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

// List layout of a build: the mixed form's forward takes its dispersion pairs
// from cluster half lists (per-atom lists only within R_cn); the FP64 form, the
// per-atom virial of Eq. 7 and the backward use full per-atom lists.
enum ListMode { kFullLists = 0, kClusterLists = 1 };

struct Plan {
    bool valid = false;
    bool sized[2] = {false, false};  // capacities measured for each list mode
    int last_mode = -1;              // list mode of the last build enqueued
    int B = 0;
    std::vector<int64_t> offsets;
    std::vector<double> cells;
    std::vector<int32_t> pbc;
    std::vector<StructGeo> geo;
    int64_t Nr = 0, ncells = 0, list_disp = 0, list_cn = 0, list_cl = 0, ncl = 0;
    int ghost_cap = 0;
    DevBuf mem;
    Work w{};
    int* bsum = nullptr;  // scan scratch
    int* gate = nullptr;  // list-reuse gate (device int)
    double* bwd_scratch = nullptr;
    int64_t bwd_scratch_n = 0;
    unsigned long long* acc = nullptr;  // fixed-point sums of the cluster-list dispersion pass
    unsigned long long* npairs = nullptr;  // pair count of the cluster-list dispersion pass
    float* vd = nullptr;                // C6 projections (v, dv) per atom of the cluster-list dispersion pass
};

// The plan's Work set up for a list mode (kernel arguments are taken by value).
void set_mode(Plan& P, int mode) {
    P.w.cl_mode = mode == kClusterLists ? 1 : 0;
    P.w.acc = mode == kClusterLists ? P.acc : nullptr;
    P.w.npairs = mode == kClusterLists ? P.npairs : nullptr;
    P.w.vd = mode == kClusterLists ? P.vd : nullptr;
}

}  // namespace

struct d3_handle {
    d3_params prm{};
    int T = 0, R = 0, RP = 0;
    std::vector<int32_t> nref;
    std::vector<double> cnref, c6, rcov, sqrtq;
    DevBuf tabmem;
    int* d_nref = nullptr;
    double* d_cnref = nullptr;
    float2* d_cnref2 = nullptr;  // reference CNs as FP32 hi, lo
    float* d_dcr = nullptr;      // [T][R][R] differences of reference CNs, FP32
    float* d_c6f = nullptr;
    double* d_c6d = nullptr;
    float4* d_pairf = nullptr;
    dbl4* d_paird = nullptr;
    dbl4* d_pairb = nullptr;  // (R0, R, R0^2, 0) per element pair, for the backward
    float* d_rtabf = nullptr;  // R = a1 R0 + a2 per element pair (three-body damping), both precisions
    double* d_rtabd = nullptr;
    // optional three-body term (d3_set_three_body); off while s9 == 0
    double s9 = 0.0, alpha9 = 16.0, rc3_A = 0.0;
    float4* d_rcpair = nullptr;  // k2 (Rcov_i + Rcov_j) and its square, FP32 hi + lo
    float2* d_exptab = nullptr;  // 2^(j/64), j = 0..63, FP32 hi + lo
    double* d_rk = nullptr;
    int* d_status = nullptr;
    int* h_status = nullptr;                 // pinned host word for the status read of the host-buffer path
    unsigned long long* d_nbuild = nullptr;  // builds executed on the device
    cudaStream_t last_stream = nullptr;
    std::string err;
    Plan plan;
    // staging buffers of the host-memory entry point
    DevBuf stage;
    size_t stage_atoms = 0, stage_structs = 0;
    double *s_pos = nullptr, *s_E = nullptr, *s_F = nullptr, *s_W = nullptr;
    int32_t* s_types = nullptr;
    // stage timing (d3_profile_*): kStages + 1 events per call, read back lazily
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::vector<cudaEvent_t>> ev_pending;
    double prof_ms[kStagesAll] = {};
    int64_t prof_calls[kStagesAll] = {};
    float tune_ms[8] = {};  // last autotuner measurement: build, CN, dispersion, chain x 2 candidates
    int64_t launches = 0;
    bool accumulate = false;  // d3_set_accumulate
    // replay of the steady-state call as one CUDA graph (captured on cap_stream)
    bool graphs = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t glaunches = 0;         // kernels in the captured call
    const void* gkey[10] = {};     // pointers and generations the graph was captured with
    int64_t plan_gen = 0, param_gen = 0;
    // launch shapes (d3_launch_shapes): chosen per size class by the autotuner unless fixed
    int32_t shape[4] = {kDefaultShape[0], kDefaultShape[1], kDefaultShape[2], kDefaultShape[3]};
    bool autotune = true;
    int64_t tunings = 0;
    std::map<std::array<int, 4>, std::array<int32_t, 4>> shape_cache;
};

namespace {

d3_status fail(d3_handle* h, d3_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

d3_status cuda_fail(d3_handle* h, cudaError_t e, const char* where) {
    return fail(h, D3_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void inv3(const double* H, double* Hi) {
    const double a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], hh = H[7], k = H[8];
    const double det = a * (e * k - f * hh) - b * (d * k - f * g) + c * (d * hh - e * g);
    Hi[0] = (e * k - f * hh) / det; Hi[1] = (c * hh - b * k) / det; Hi[2] = (b * f - c * e) / det;
    Hi[3] = (f * g - d * k) / det;  Hi[4] = (a * k - c * g) / det;  Hi[5] = (c * d - a * f) / det;
    Hi[6] = (d * hh - e * g) / det; Hi[7] = (b * g - a * hh) / det; Hi[8] = (a * e - b * d) / det;
}

double det3(const double* H) {
    return H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) + H[2] * (H[3] * H[7] - H[4] * H[6]);
}

// Upload the damping table (R^6, R^8, s6, s8 R0^2 per element pair) in both precisions.
d3_status upload_pair_table(d3_handle* h) {
    const int T = h->T;
    std::vector<dbl4> pd(T * T), pb(T * T);
    std::vector<float4> pf(T * T);
    std::vector<double> rd(T * T);
    std::vector<float> rf(T * T);
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            const double R0sq = 3.0 * h->sqrtq[a] * h->sqrtq[b];
            const double Rd = h->prm.a1 * std::sqrt(R0sq) + h->prm.a2_bohr;
            const double R2 = Rd * Rd, R6 = R2 * R2 * R2, R8 = R6 * R2;
            pd[a * T + b] = dbl4_make(R6, R8, h->prm.s6, h->prm.s8 * R0sq);
            pf[a * T + b] = make_float4((float)R6, (float)R8, (float)h->prm.s6, (float)(h->prm.s8 * R0sq));
            pb[a * T + b] = dbl4_make(std::sqrt(R0sq), Rd, R0sq, 0.0);
            rd[a * T + b] = Rd;
            rf[a * T + b] = (float)Rd;
        }
    cudaError_t e = cudaMemcpy(h->d_paird, pd.data(), pd.size() * sizeof(dbl4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_rtabd, rd.data(), rd.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_rtabf, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_pairf, pf.data(), pf.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_pairb, pb.data(), pb.size() * sizeof(dbl4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "pair table upload");
    return D3_OK;
}

// List radius (bohr) for a cutoff in A: the cutoff plus the skin plus a margin
// covering the FP32 grid positions the list build compares (<= sqrt(3) 2^-10 bohr).
double list_radius(const d3_handle* h, double rc_A) {
    return rc_A / kBohrA * (1.0 + 1e-5) + 4e-3 + std::max(0.0, h->prm.skin_A) / kBohrA;
}

Consts make_consts(const d3_handle* h) {
    Consts c{};
    const double rd = h->prm.rc_disp_A / kBohrA, rn = h->prm.rc_cn_A / kBohrA;
    c.rc_disp2 = rd * rd;
    c.rc_disp2f = (float)c.rc_disp2;
    c.rc_cn2 = rn * rn;
    c.k1 = h->prm.k1;
    c.k3 = h->prm.k3;
    c.s6 = h->prm.s6;
    c.s8 = h->prm.s8;
    c.a1 = h->prm.a1;
    c.a2 = h->prm.a2_bohr;
    c.T = h->T;
    c.R = h->R;
    c.RP = h->RP;
    c.accumulate = h->accumulate ? 1 : 0;
    c.atm = h->s9 != 0.0 ? 1 : 0;
    c.s9 = h->s9;
    c.alpha9 = h->alpha9;
    const double r3 = h->rc3_A / kBohrA;
    c.rc3_2 = r3 * r3;
    c.k1f = (float)c.k1;
    c.rc_cn2f = (float)c.rc_cn2;
    c.k3f = (float)c.k3;
    c.k3h = (float)c.k3;
    c.k3l = (float)(c.k3 - (double)c.k3h);
    c.s9f = (float)c.s9;
    c.alpha9f = (float)c.alpha9;
    c.alpha9_3f = (float)(c.alpha9 / 3.0);
    c.rc3_2f = (float)c.rc3_2;
    return c;
}

bool same_geometry(const Plan& P, int32_t B, const int64_t* offsets, const double* cells, const int32_t* pbc) {
    if (!P.valid || P.B != B) return false;
    if (B == 0) return P.offsets.size() == 1;
    return std::memcmp(P.offsets.data(), offsets, sizeof(int64_t) * (B + 1)) == 0 &&
           std::memcmp(P.cells.data(), cells, sizeof(double) * 9 * B) == 0 &&
           std::memcmp(P.pbc.data(), pbc, sizeof(int32_t) * 3 * B) == 0;
}

// Host geometry of every structure: cell grid over the fractional range
// [-delta, 1 + delta) along periodic axes (delta = list radius / plane
// spacing) and [0, 1) along open ones, window half-widths, image ranges and
// first estimates of the per-atom list lengths.
d3_status plan_geometry(d3_handle* h, Plan& P, int32_t B, const int64_t* offsets, const double* cells,
                        const int32_t* pbc, std::vector<double>& ghost_est) {
    const double rld = list_radius(h, h->prm.rc_disp_A), rln = list_radius(h, h->prm.rc_cn_A);
    const double rl = std::max(rld, rln);
    P.geo.assign(B, StructGeo{});
    ghost_est.assign(B, 0.0);
    int64_t cell_base = 0;
    for (int s = 0; s < B; ++s) {
        StructGeo& G = P.geo[s];
        for (int k = 0; k < 9; ++k) G.H[k] = cells[9 * s + k] / kBohrA;
        const double det = det3(G.H);
        double scale = 0;
        for (int k = 0; k < 9; ++k) scale = std::max(scale, std::fabs(G.H[k]));
        if (!(std::fabs(det) > 1e-9 * scale * scale * scale) || !std::isfinite(det))
            return fail(h, D3_ERR_ARG, "degenerate or non-finite cell for structure " + std::to_string(s));
        inv3(G.H, G.Hinv);
        // the far corner of the cell (where wrapped positions end) must stay in the coordinate range
        double corner = 0.0;
        for (int m = 0; m < 8; ++m) {
            double c2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double x = ((m & 1) ? G.H[a] : 0.0) + ((m & 2) ? G.H[3 + a] : 0.0) + ((m & 4) ? G.H[6 + a] : 0.0);
                c2 += x * x;
            }
            corner = std::max(corner, std::sqrt(c2));
        }
        if (!(corner + rl < (double)kMaxCoordBohr))
            return fail(h, D3_ERR_ARG, "cell of structure " + std::to_string(s) +
                                            " extends beyond the supported coordinate range (4200 A)");
        const int64_t n = offsets[s + 1] - offsets[s];
        if (n < 0) return fail(h, D3_ERR_ARG, "offsets must be non-decreasing");
        if (n > (int64_t)1 << 27) return fail(h, D3_ERR_ARG, "structure too large (max 2^27 atoms)");
        double vol_factor = 1.0;
        int64_t nc_total = 1;
        for (int k = 0; k < 3; ++k) {
            const double* u = G.H + 3 * ((k + 1) % 3);
            const double* v = G.H + 3 * ((k + 2) % 3);
            const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
            const double width = std::fabs(det) / std::sqrt(cx * cx + cy * cy + cz * cz);
            G.pbc[k] = pbc[3 * s + k] ? 1 : 0;
            if (G.pbc[k]) {
                const double delta = rl / width + 1e-9;
                G.img[k] = (int)std::ceil(delta);
                if (G.img[k] > 100) return fail(h, D3_ERR_ARG, "cell too thin for the cutoff (more than 100 images)");
                G.lo[k] = -delta;
                G.ext_lo[k] = -delta;
                G.ext_hi[k] = 1.0 + delta;
                vol_factor *= 1.0 + 2.0 * delta;
            } else {
                G.img[k] = 0;
                G.lo[k] = 0.0;
                G.ext_lo[k] = 0.0;
                G.ext_hi[k] = 1.0;
            }
            const double span = G.pbc[k] ? 1.0 + 2.0 * (-G.lo[k]) : 1.0;
            long long nck = (long long)std::floor(span * width * kWindowCells / rl);
            nck = std::max(1LL, std::min(nck, 2048LL));
            G.ncell[k] = (int)nck;
            G.fscale[k] = (double)nck / span;
            const double cw = span * width / (double)nck;
            G.win[k] = (int)std::min<long long>(nck, (long long)std::ceil(rl / cw));
            G.win_cn[k] = (int)std::min<long long>(nck, (long long)std::ceil(rln / cw));
            nc_total *= nck;
        }
        if (nc_total > ((int64_t)1 << 26)) return fail(h, D3_ERR_ARG, "too many cells for structure " + std::to_string(s));
        for (int k = 0; k < 9; ++k) {
            G.Hinvf[k] = (float)G.Hinv[k];
            const double g = std::nearbyint(G.H[k] * 1024.0) / 1024.0;
            G.Hh[k] = (float)g;
            G.Hl[k] = (float)(G.H[k] - g);
        }
        for (int k = 0; k < 3; ++k) {
            G.lof[k] = (float)G.lo[k];
            G.fscalef[k] = (float)G.fscale[k];
            G.ext_lof[k] = (float)G.ext_lo[k];
            G.ext_hif[k] = (float)G.ext_hi[k];
        }
        G.cell_base = cell_base;
        cell_base += nc_total;
        G.atom_base = offsets[s];
        G.natoms = (int32_t)n;
        const double vol = std::fabs(det);  // bohr^3
        const double rho = n > 0 ? (double)n / vol : 0.0;
        const double four_thirds_pi = 4.18879020478639;
        const double nd = four_thirds_pi * rld * rld * rld * rho, nn = four_thirds_pi * rln * rln * rln * rho;
        const double cap_all = (double)n * vol_factor + 8;
        G.cap_disp = round_cap(std::min(cap_all, std::ceil(1.3 * nd + 32.0)));
        G.cap_cn = round_cap(std::min(cap_all, std::ceil(1.3 * nn + 16.0)));
        // a cluster list holds about half the atoms within the list radius of the
        // cluster's bounding box (regrown by the sizing pass when short)
        G.cap_cl = round_cap(std::min(cap_all, std::ceil(4.5 * nd + 64.0)));
        ghost_est[s] = (double)n * (vol_factor - 1.0);
    }
    P.ncells = cell_base;
    return D3_OK;
}

// (Re)allocate every device buffer of the plan for the current capacities.
d3_status plan_alloc(d3_handle* h, Plan& P) {
    ++h->plan_gen;  // a captured graph refers to the old buffers
    P.mem.release();
    P.bwd_scratch = nullptr;
    P.bwd_scratch_n = 0;
    const int B = P.B;
    const int64_t Nr = P.Nr, C = P.ncells, Ng = P.ghost_cap, Nt = Nr + Ng;
    int64_t ld = 0, lc = 0, lcl = 0, ncl = 0;
    std::vector<int> clu_sid;
    for (int s = 0; s < B; ++s) {
        StructGeo& G = P.geo[s];
        G.list_base_disp = ld;
        G.list_base_cn = lc;
        ld += list_size(G.natoms, G.cap_disp);
        lc += list_size(G.natoms, G.cap_cn);
        const int64_t k = (G.natoms + kClusterAtoms - 1) / kClusterAtoms;
        G.clu_base = ncl;
        G.list_base_cl = lcl;
        ncl += k;
        lcl += k * (int64_t)G.cap_cl;
        clu_sid.insert(clu_sid.end(), (size_t)k, s);
    }
    P.list_disp = ld;
    P.list_cn = lc;
    P.list_cl = lcl;
    P.ncl = ncl;
    Work& w = P.w;
    w = Work{};
    w.B = B;
    w.Nr = Nr;
    w.ncells = C;
    w.ghost_cap = (int)Ng;
    w.T = h->T;
    w.R = h->R;
    w.RP = h->RP;
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        w.num_sms = sms > 0 ? sms : 1;
    }
    w.blk_cn = h->shape[0];
    w.blk_disp = h->shape[1];
    w.blk_chain = h->shape[2];
    w.build_per_sm = h->shape[3];
    const size_t rs = h->prm.precision == D3_MIXED ? sizeof(float) : sizeof(double);
    StructGeo* dgeo = nullptr;
    int64_t* doff = nullptr;
    DevBuf& m = P.mem;
    cudaError_t e = cudaSuccess;
#define A(ptr, T, n) \
    if (e == cudaSuccess) e = m.alloc((T**)&(ptr), (size_t)(n))
    A(dgeo, StructGeo, B);
    A(doff, int64_t, B + 1);
    int* dsid = nullptr;
    A(dsid, int, Nr);
    A(w.cnt_real, int, C + 1);
    A(w.cnt_ghost, int, C + 1);
    A(w.start_real, int, C + 1);
    A(w.start_ghost, int, C + 1);
    A(w.cell_of, int, Nr);
    A(w.slot_of, int, Nr);
    A(w.xw, double, 3 * Nr);
    A(w.ghost_src, int, Ng);
    A(w.ghost_shift, int, Ng);
    A(w.ghost_cell, int, Ng);
    A(w.ghost_slot, int, Ng);
    A(w.ghost_sid, int, Ng);
    A(w.ghost_count, int, 1);
    A(w.sorted_src, int, Nr);
    A(w.gsorted, int, Ng);
    A(w.ginv, int, Ng);
    A(w.gfirst, int, Nr);
    A(w.gcnt, int, Nr);
    A(w.usrc, int, Nr + Ng);
    A(w.ukey, long long, Nr + Ng);
    A(w.pos64, dbl4, Nt);
    A(w.rec, float4, 2 * Nt);
    A(w.hi, float4, Nt);
    A(w.fw, float, 3 * Nr);
    A(w.frange, int, 6 * (int64_t)B);
    A(w.perm, int, Nr);
    A(w.sid, int, Nr);
    A(w.cell_sorted, int, Nr);
    A(w.nbr_disp, int, ld);
    A(w.nbr_cn, int, lc);
    A(w.cnt_disp, int, Nr);
    A(w.cnt_cn, int, Nr);
    A(w.maxcnt, int, 3 * B);
    A(w.work_ctr, int, 2);
    A(w.skey, float, Nr);
    int* dclu = nullptr;
    A(dclu, int, std::max<int64_t>(1, ncl));
    A(w.nbr_cl, int, lcl);
    A(w.cnt_cl, int, std::max<int64_t>(1, ncl));
    A(w.acc, unsigned long long, 8 * Nr);
    A(w.npairs, unsigned long long, 1);
    // rows of v and dv for real and image atoms (whether images get copies of their
    // source's rows is decided after the sizing pass, from the image count)
    if (h->prm.precision == D3_MIXED) A(w.vd, float, Nt * h->T * 2 * h->RP);
    if (h->prm.precision == D3_MIXED) A(w.gcn, float, lc);
    A(w.gate, int, 1);
    A(w.xref, double, 3 * Nr);
    A(w.wshift, double, 3 * Nr);
    A(w.cn, double, Nr);
    A(w.W, char, Nr * h->RP * rs);
    A(w.dW, char, Nr * h->RP * rs);
    A(w.v, char, Nr * h->T * h->RP * rs);
    A(w.dEdn, char, Nr * rs);
    A(w.Fd, char, Nr * 4 * rs);
    A(w.eat, double, Nr);
    A(w.wv, double, 6 * Nr);
    A(w.Pv, char, Nr * 4 * rs);
    int64_t maxn = 0;
    for (int s = 0; s < B; ++s) maxn = std::max<int64_t>(maxn, P.geo[s].natoms);
    w.max_natoms = maxn;
    std::vector<int> fin_sid;
    int64_t nfin = 0;
    for (int s = 0; s < B; ++s) {
        P.geo[s].fin_base = nfin;
        const int64_t k = (P.geo[s].natoms + kFinChunk - 1) / kFinChunk;
        nfin += k;
        fin_sid.insert(fin_sid.end(), (size_t)k, s);
    }
    w.n_fin = nfin;
    A(w.fin_part, double, 7 * std::max<int64_t>(1, nfin));
    int* dfin = nullptr;
    A(dfin, int, std::max<int64_t>(1, nfin));
    A(P.bsum, int, scan_scratch_ints(C));
#undef A
    if (e != cudaSuccess) {
        P.mem.release();
        P.valid = false;
        return cuda_fail(h, e, "workspace allocation");
    }
    P.w.status = h->d_status;
    P.w.geo = dgeo;
    P.w.offsets = doff;
    P.w.sid_in = dsid;
    P.w.fin_sid = dfin;
    P.w.clu_sid = dclu;
    P.w.ncl = ncl;
    P.acc = w.acc;  // attached to the Work of cluster-mode calls only
    P.npairs = w.npairs;
    P.w.npairs = nullptr;
    P.vd = w.vd;
    P.w.acc = nullptr;
    P.w.vd = nullptr;
    P.w.cl_mode = 0;
    const double rld = list_radius(h, h->prm.rc_disp_A), rln = list_radius(h, h->prm.rc_cn_A);
    w.rl_disp2 = (float)(rld * rld);
    w.rl_cn2 = (float)(rln * rln);
    const double half_skin = 0.5 * std::max(0.0, h->prm.skin_A) / kBohrA;
    w.skin_half2 = half_skin * half_skin;
    w.nbuild = h->d_nbuild;
    int* gate = w.gate;
    w.gate = nullptr;  // the plan's own Work builds unconditionally; enqueue_build gates a copy
    P.gate = gate;
    e = cudaMemcpy(dgeo, P.geo.data(), sizeof(StructGeo) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nfin > 0)
        e = cudaMemcpy(dfin, fin_sid.data(), sizeof(int) * (size_t)nfin, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(doff, P.offsets.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ncl > 0)
        e = cudaMemcpy(dclu, clu_sid.data(), sizeof(int) * (size_t)ncl, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && Nr > 0) {
        std::vector<int> sid((size_t)Nr);
        for (int s = 0; s < B; ++s)
            for (int64_t i = P.offsets[s]; i < P.offsets[s + 1]; ++i) sid[(size_t)i] = s;
        e = cudaMemcpy(dsid, sid.data(), sizeof(int) * (size_t)Nr, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "geometry upload");
    return D3_OK;
}

std::vector<cudaEvent_t> take_events(d3_handle* h, int n) {
    std::vector<cudaEvent_t> v;
    while ((int)v.size() < n) {
        if (!h->ev_pool.empty()) {
            v.push_back(h->ev_pool.back());
            h->ev_pool.pop_back();
        } else {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) break;
            v.push_back(e);
        }
    }
    return v;
}

// Device tables of the forward passes for the handle's precision.
Tabs forward_tabs(const d3_handle* h) {
    const bool mixed = h->prm.precision == D3_MIXED;
    Tabs tb{};
    tb.c6 = mixed ? (const void*)h->d_c6f : (const void*)h->d_c6d;
    tb.pair = mixed ? (const void*)h->d_pairf : (const void*)h->d_paird;
    tb.cnref = h->d_cnref;
    tb.cnref2 = h->d_cnref2;
    tb.dcr = h->d_dcr;
    tb.nref = h->d_nref;
    tb.rcpair = h->d_rcpair;
    tb.exptab = h->d_exptab;
    tb.rtab = mixed ? (const void*)h->d_rtabf : (const void*)h->d_rtabd;
    return tb;
}

void set_shapes(d3_handle* h, const int32_t* shape) {
    bool changed = false;
    for (int k = 0; k < 4; ++k) {
        changed = changed || h->shape[k] != shape[k];
        h->shape[k] = shape[k];
    }
    Work& w = h->plan.w;
    w.blk_cn = shape[0];
    w.blk_disp = shape[1];
    w.blk_chain = shape[2];
    w.build_per_sm = shape[3];
    if (changed) ++h->param_gen;  // launch shapes are baked into a captured graph
}

// Size class of a plan for the autotuner: precision, three-body term on or
// off, and the binary orders of magnitude of the atom count and of the mean
// structure size.
std::array<int, 4> size_class(const d3_handle* h, const Plan& P) {
    auto lg = [](int64_t x) {
        int k = 0;
        while (x > 1) {
            x >>= 1;
            ++k;
        }
        return k;
    };
    return {h->prm.precision, h->s9 != 0.0 ? 1 : 0, lg(P.Nr), lg(P.Nr / std::max(P.B, 1))};
}

// Enqueue the neighbour build.  gated (list reuse, skin > 0): a displacement
// check first decides on the device whether the build runs; the sorted
// positions are rewritten either way.
d3_status enqueue_build(d3_handle* h, Plan& P, const double* pos, const int32_t* types, cudaStream_t st, int mode,
                        bool gated = false, cudaEvent_t* lmarks = nullptr) {
    // a build in the other list mode re-sorted the atoms: the first build in
    // this mode must run whatever the displacement check would decide
    if (P.last_mode != mode) gated = false;
    set_mode(P, mode);
    P.last_mode = mode;
    Work w = P.w;
    cudaError_t e = cudaSuccess;
    if (gated) {
        w.gate = P.gate;
        e = cudaMemsetAsync(w.gate, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_check(w, pos, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "displacement check");
        if (P.Nr > 0) h->launches += 1;
    }
    e = launch_build_impl(w, pos, types, h->d_rk, P.bsum, st, lmarks);
    if (e != cudaSuccess) return cuda_fail(h, e, "neighbour build launch");
    if (P.Nr > 0) h->launches += kBuildLaunches;
    return D3_OK;
}

// The autotuner: once per size class, right after a new geometry is sized,
// run the build and the forward passes kTuneReps times with each candidate
// shape (alternating) and keep, per kernel, the candidate with the shortest
// time; a candidate replaces the default only when it is more than 1% faster.
// Each stage is timed with events on the caller's stream.  The runs write
// only the plan's workspace and scratch outputs, and the device build counter
// is put back afterwards.
d3_status tune_shapes(d3_handle* h, Plan& P, const double* pos, const int32_t* types, cudaStream_t st, int mode) {
    if (!h->autotune) return D3_OK;
    if (P.Nr < kTuneMinAtoms) {
        set_shapes(h, kDefaultShape);
        return D3_OK;
    }
    const std::array<int, 4> key = size_class(h, P);
    const auto it = h->shape_cache.find(key);
    if (it != h->shape_cache.end()) {
        set_shapes(h, it->second.data());
        return D3_OK;
    }
    std::vector<cudaEvent_t> ev = take_events(h, kStages + 1);
    auto give_back = [&]() {
        for (cudaEvent_t x : ev) h->ev_pool.push_back(x);
    };
    if (ev.size() != kStages + 1) {
        give_back();
        return cuda_fail(h, cudaErrorMemoryAllocation, "autotuner events");
    }
    DevBuf scratch;
    double *E = nullptr, *F = nullptr, *W = nullptr;
    cudaError_t e = scratch.alloc(&E, (size_t)P.B);
    if (e == cudaSuccess) e = scratch.alloc(&F, 3 * (size_t)P.Nr);
    if (e == cudaSuccess) e = scratch.alloc(&W, 9 * (size_t)P.B);
    unsigned long long nbuild = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nbuild, h->d_nbuild, sizeof(nbuild), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    Consts c = make_consts(h);
    c.accumulate = 0;
    const Tabs tb = forward_tabs(h);
    const bool mixed = h->prm.precision == D3_MIXED;
    set_mode(P, mode);
    P.last_mode = mode;
    Work w = P.w;
    // t[kernel][candidate]: build, CN, dispersion, chain
    float t[4][2];
    for (auto& r : t) r[0] = r[1] = 1e30f;
    for (int rep = 0; rep < kTuneReps && e == cudaSuccess; ++rep) {
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            w.build_per_sm = kBuildCand[k];
            w.blk_cn = w.blk_disp = w.blk_chain = kBlockCand[k];
            e = cudaEventRecord(ev[0], st);
            if (e == cudaSuccess) e = launch_build_impl(w, pos, types, h->d_rk, P.bsum, st);
            // marks 0..6 of the forward land in ev[1..7]: CN 0-1, dispersion 2-3, chain 4-5
            if (e == cudaSuccess) e = launch_forward(w, c, mixed, tb, E, F, W, nullptr, nullptr, nullptr, P.B, st,
                                                     ev.data() + 1);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            h->launches += kBuildLaunches + kForwardLaunches + c.atm + w.cl_mode;
            const int from[4] = {0, 1, 3, 5};
            for (int m = 0; m < 4 && e == cudaSuccess; ++m) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, ev[from[m]], ev[from[m] + 1]);
                t[m][k] = std::min(t[m][k], ms);
            }
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_nbuild, &nbuild, sizeof(nbuild), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    scratch.release();
    give_back();
    if (e != cudaSuccess) return cuda_fail(h, e, "autotuner");
    // kernel m's default is candidate dflt[m]; the other must beat it by more than 1%
    const int dflt[4] = {kDefaultShape[3] == kBuildCand[0] ? 0 : 1, kDefaultShape[0] == kBlockCand[0] ? 0 : 1,
                         kDefaultShape[1] == kBlockCand[0] ? 0 : 1, kDefaultShape[2] == kBlockCand[0] ? 0 : 1};
    int pick[4];
    for (int m = 0; m < 4; ++m) pick[m] = t[m][1 - dflt[m]] < 0.99f * t[m][dflt[m]] ? 1 - dflt[m] : dflt[m];
    for (int m = 0; m < 4; ++m)
        for (int k = 0; k < 2; ++k) h->tune_ms[2 * m + k] = t[m][k];
    const std::array<int32_t, 4> chosen = {kBlockCand[pick[1]], kBlockCand[pick[2]], kBlockCand[pick[3]],
                                           kBuildCand[pick[0]]};
    h->shape_cache[key] = chosen;
    ++h->tunings;
    set_shapes(h, chosen.data());
    return D3_OK;
}

// Make the plan match the geometry; on a new geometry run the build once
// synchronously and grow image and list capacities until nothing overflows.
d3_status ensure_plan(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos, const int32_t* types,
                      const double* cells, const int32_t* pbc, cudaStream_t st, int mode) {
    Plan& P = h->plan;
    if (same_geometry(P, B, offsets, cells, pbc) && P.sized[mode]) return D3_OK;
    if (!same_geometry(P, B, offsets, cells, pbc)) {
        P.valid = false;
        P.sized[0] = P.sized[1] = false;
        P.last_mode = -1;
        P.B = B;
        P.offsets.assign(offsets, offsets + B + 1);
        P.cells.assign(cells, cells + 9 * (size_t)B);
        P.pbc.assign(pbc, pbc + 3 * (size_t)B);
        P.Nr = offsets[B];
        std::vector<double> gest;
        d3_status s = plan_geometry(h, P, B, offsets, cells, pbc, gest);
        if (s != D3_OK) return s;
        double g = 64.0;
        for (double x : gest) g += 1.15 * x + 8.0;
        if (g > 2.0e9) return fail(h, D3_ERR_ARG, "too many periodic images");
        P.ghost_cap = (int)g;
        s = plan_alloc(h, P);
        if (s != D3_OK) return s;
        P.valid = true;
    }
    for (int attempt = 0; attempt < 4; ++attempt) {
        cudaError_t e = cudaMemsetAsync(h->d_status, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
        d3_status s = enqueue_build(h, P, pos, types, st, mode);
        if (s != D3_OK) return s;
        int gcount = 0, status = 0;
        std::vector<int> mx(3 * (size_t)std::max(B, 1), 0);
        e = cudaMemcpyAsync(&gcount, P.w.ghost_count, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && B > 0) e = cudaMemcpyAsync(mx.data(), P.w.maxcnt, sizeof(int) * 3 * B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(h, e, "sizing pass");
        if (status & ST_NONFINITE) return fail(h, D3_ERR_NONFINITE, "non-finite coordinate");
        if (status & ST_TYPE) return fail(h, D3_ERR_TYPE, "atom type out of range");
        bool grow = false;
        if (gcount > P.ghost_cap) {
            P.ghost_cap = (int)std::min<double>(2.0e9, gcount * 1.1 + 64);
            grow = true;
        }
        for (int s2 = 0; s2 < B; ++s2) {
            StructGeo& G = P.geo[s2];
            if (mx[3 * s2] > G.cap_disp) { G.cap_disp = round_cap(mx[3 * s2] * 1.1 + 16); grow = true; }
            if (mx[3 * s2 + 1] > G.cap_cn) { G.cap_cn = round_cap(mx[3 * s2 + 1] * 1.1 + 8); grow = true; }
            if (mx[3 * s2 + 2] > G.cap_cl) { G.cap_cl = round_cap(mx[3 * s2 + 2] * 1.1 + 16); grow = true; }
        }
        if (!grow) {
            // image rows of v and dv are copies of their source's when that is cheap
            // (few images, or few types); otherwise the pass resolves each image's source
            P.w.vd_images = (int64_t)gcount * h->T <= 2 * P.Nr ? 1 : 0;
            P.sized[mode] = true;
            return tune_shapes(h, P, pos, types, st, mode);
        }
        P.sized[0] = P.sized[1] = false;  // the buffers are reallocated: both modes re-measure
        s = plan_alloc(h, P);
        if (s != D3_OK) return s;
    }
    return fail(h, D3_ERR_CAPACITY, "workspace sizing did not converge");
}

d3_status check_batch_args(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos, const int32_t* types,
                           const double* cells, const int32_t* pbc) {
    if (!h) return D3_ERR_ARG;
    if (B < 0 || !offsets || (B > 0 && (!cells || !pbc))) return fail(h, D3_ERR_ARG, "bad batch description");
    if (offsets[0] != 0) return fail(h, D3_ERR_ARG, "offsets[0] must be 0");
    for (int s = 0; s < B; ++s)
        if (offsets[s + 1] < offsets[s]) return fail(h, D3_ERR_ARG, "offsets must be non-decreasing");
    if (offsets[B] > ((int64_t)1 << 27)) return fail(h, D3_ERR_ARG, "too many atoms (max 2^27)");
    if (offsets[B] > 0 && (!pos || !types)) return fail(h, D3_ERR_ARG, "NULL positions or types");
    return D3_OK;
}

// List mode of a forward call: cluster lists for the mixed form, full per-atom
// lists for the FP64 form and for the per-atom virial of Eq. 7.
int list_mode(const d3_handle* h, const double* w_atom) {
    return h->prm.precision == D3_MIXED && !w_atom ? kClusterLists : kFullLists;
}

d3_status forward(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos, const int32_t* types,
                  const double* cells, const int32_t* pbc, double* E, double* F, double* W, double* e_atom,
                  double* cn, cudaStream_t st, double* w_atom = nullptr) {
    d3_status s = check_batch_args(h, B, offsets, pos, types, cells, pbc);
    if (s != D3_OK) return s;
    if (B > 0 && (!E || !W)) return fail(h, D3_ERR_ARG, "NULL E or W");
    if (offsets[B] > 0 && !F) return fail(h, D3_ERR_ARG, "NULL F");
    if (w_atom && h->s9 != 0.0)
        return fail(h, D3_ERR_ARG, "per-atom virials (Eq. 7) are defined for the two-body model only; "
                                   "disable the three-body term");
    h->last_stream = st;
    if (B == 0) return D3_OK;
    const int mode = list_mode(h, w_atom);
    s = ensure_plan(h, B, offsets, pos, types, cells, pbc, st, mode);
    if (s != D3_OK) return s;
    Plan& P = h->plan;
    std::vector<cudaEvent_t> ev;
    if (h->prof_on) {
        ev = take_events(h, kEvents);
        if (ev.size() == kEvents) cudaEventRecord(ev[0], st);
    }
    s = enqueue_build(h, P, pos, types, st, mode, h->prm.skin_A > 0,
                      ev.size() == kEvents ? ev.data() + kStages + 1 : nullptr);
    if (s != D3_OK) return s;
    const Consts c = make_consts(h);
    const bool mixed = h->prm.precision == D3_MIXED;
    const Tabs tb = forward_tabs(h);
    cudaError_t e = launch_forward(P.w, c, mixed, tb, E, F, W, e_atom, cn, w_atom, B, st,
                                   ev.size() == kEvents ? ev.data() + 1 : nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "forward launch");
    h->launches += (P.Nr > 0 ? kForwardLaunches + c.atm + (mode == kClusterLists ? 1 : 0) : 1);
    if (ev.size() == kEvents) h->ev_pending.push_back(ev);
    else for (cudaEvent_t x : ev) h->ev_pool.push_back(x);
    return D3_OK;
}

// The steady-state call (sized plan, no profiling) is the same sequence of
// kernels and memsets every time for the same pointers and parameters, so it
// is captured once as a CUDA graph on an internal stream and then replayed on
// the caller's stream with one launch.  Calls made while the caller's stream
// is itself being captured enqueue directly.
bool graph_key_match(const d3_handle* h, const void* const (&k)[10]) {
    if (!h->gexec) return false;
    for (int i = 0; i < 10; ++i)
        if (h->gkey[i] != k[i]) return false;
    return true;
}

d3_status forward_graph(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos, const int32_t* types,
                        const double* cells, const int32_t* pbc, double* E, double* F, double* W, double* e_atom,
                        double* cn, cudaStream_t st, double* w_atom) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool direct = !h->graphs || h->prof_on || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
                        cs != cudaStreamCaptureStatusNone;
    if (direct || B <= 0 || !offsets || offsets[B] <= 0)
        return forward(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, st, w_atom);
    d3_status s = check_batch_args(h, B, offsets, pos, types, cells, pbc);
    if (s != D3_OK) return s;
    if (!E || !W || !F) return fail(h, D3_ERR_ARG, "NULL E, F or W");
    const int mode = list_mode(h, w_atom);
    s = ensure_plan(h, B, offsets, pos, types, cells, pbc, st, mode);
    if (s != D3_OK) return s;
    h->last_stream = st;
    // the last build was in the other list mode: rebuild once directly (a
    // replayed graph would take the list-reuse decision on stale lists)
    if (h->plan.last_mode != mode)
        return forward(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, st, w_atom);
    const void* key[10] = {pos, types, E, F, W, e_atom, cn, w_atom, (const void*)(intptr_t)h->plan_gen,
                           (const void*)(intptr_t)(h->param_gen * 2 + (h->accumulate ? 1 : 0))};
    if (!graph_key_match(h, key)) {
        if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            h->graphs = false;
            return forward(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, st, w_atom);
        }
        // the captured work must start after everything already on the caller's stream
        cudaGraph_t g = nullptr;
        const int64_t before = h->launches;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            s = forward(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, h->cap_stream, w_atom);
            e = cudaStreamEndCapture(h->cap_stream, &g);
        }
        const int64_t captured = h->launches - before;
        h->launches = before;
        h->last_stream = st;
        cudaGraphExec_t x = nullptr;
        if (e == cudaSuccess && s == D3_OK && g) e = cudaGraphInstantiate(&x, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || s != D3_OK || !x) {
            cudaGetLastError();
            if (x) cudaGraphExecDestroy(x);
            h->graphs = false;  // fall back to direct enqueueing for this handle
            return forward(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, st, w_atom);
        }
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        h->gexec = x;
        h->glaunches = captured;
        for (int i = 0; i < 10; ++i) h->gkey[i] = key[i];
    }
    cudaError_t e = cudaGraphLaunch(h->gexec, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    h->launches += h->glaunches;
    return D3_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* d3_version(void) { return "d3gb 0.1 (sm_103a)"; }

d3_status d3_create(const d3_params* params, const d3_tables* tables, d3_handle** out) {
    if (!out) return D3_ERR_ARG;
    *out = nullptr;
    if (!params || !tables) return D3_ERR_ARG;
    const d3_tables& t = *tables;
    if (t.ntypes < 1 || t.ntypes > kMaxTypes || t.max_ref < 1 || t.max_ref > kMaxRef || !t.nref || !t.cn_ref ||
        !t.c6_ref || !t.rcov_bohr || !t.sqrtq)
        return D3_ERR_ARG;
    const d3_params& p = *params;
    if (!(p.rc_disp_A > 0) || !(p.rc_cn_A > 0) || !(p.k1 > 0) || !(p.k3 > 0) || p.skin_A < 0 ||
        (p.precision != D3_FP64 && p.precision != D3_MIXED) || !std::isfinite(p.s6) || !std::isfinite(p.s8) ||
        !std::isfinite(p.a1) || !std::isfinite(p.a2_bohr))
        return D3_ERR_ARG;
    const int T = t.ntypes, R = t.max_ref;
    for (int a = 0; a < T; ++a) {
        if (t.nref[a] < 1 || t.nref[a] > R) return D3_ERR_ARG;
        if (!(t.rcov_bohr[a] > 0) || !(t.sqrtq[a] > 0)) return D3_ERR_ARG;
    }
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b)
            for (int i = 0; i < R; ++i)
                for (int j = 0; j < R; ++j) {
                    const double x = t.c6_ref[((a * T + b) * R + i) * R + j];
                    const double y = t.c6_ref[((b * T + a) * R + j) * R + i];
                    if (!std::isfinite(x) || x != y) return D3_ERR_ARG;
                }
    d3_handle* h = new d3_handle();
    h->prm = p;
    h->T = T;
    h->R = R;
    h->RP = R <= 4 ? 4 : 8;
    h->nref.assign(t.nref, t.nref + T);
    h->cnref.assign(t.cn_ref, t.cn_ref + T * R);
    h->c6.assign(t.c6_ref, t.c6_ref + (size_t)T * T * R * R);
    h->rcov.assign(t.rcov_bohr, t.rcov_bohr + T);
    h->sqrtq.assign(t.sqrtq, t.sqrtq + T);
    // padding entries (a >= nref) of C6 are never weighted, zero them for safety
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b)
            for (int i = 0; i < R; ++i)
                for (int j = 0; j < R; ++j)
                    if (i >= h->nref[a] || j >= h->nref[b]) h->c6[((a * T + b) * R + i) * R + j] = 0.0;
    std::vector<float> c6f(h->c6.begin(), h->c6.end());
    std::vector<double> rk(T);
    for (int a = 0; a < T; ++a) rk[a] = p.k2 * h->rcov[a];
    cudaError_t e = cudaSuccess;
    DevBuf& m = h->tabmem;
    if (e == cudaSuccess) e = m.alloc(&h->d_nref, T);
    if (e == cudaSuccess) e = m.alloc(&h->d_cnref, T * R);
    if (e == cudaSuccess) e = m.alloc(&h->d_cnref2, T * R);
    if (e == cudaSuccess) e = m.alloc(&h->d_dcr, T * R * R);
    if (e == cudaSuccess) e = m.alloc(&h->d_c6f, h->c6.size());
    if (e == cudaSuccess) e = m.alloc(&h->d_c6d, h->c6.size());
    if (e == cudaSuccess) e = m.alloc(&h->d_pairf, T * T);
    if (e == cudaSuccess) e = m.alloc(&h->d_paird, T * T);
    if (e == cudaSuccess) e = m.alloc(&h->d_pairb, T * T);
    if (e == cudaSuccess) e = m.alloc(&h->d_rtabf, T * T);
    if (e == cudaSuccess) e = m.alloc(&h->d_rtabd, T * T);
    if (e == cudaSuccess) e = m.alloc(&h->d_rcpair, T * T);
    if (e == cudaSuccess) e = m.alloc(&h->d_exptab, 64);
    if (e == cudaSuccess) e = m.alloc(&h->d_rk, T);
    if (e == cudaSuccess) e = m.alloc(&h->d_status, 1);
    if (e == cudaSuccess) e = m.alloc(&h->d_nbuild, 1);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_nref, h->nref.data(), T * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_cnref, h->cnref.data(), T * R * sizeof(double), cudaMemcpyHostToDevice);
    {
        std::vector<float2> cr2(T * R);
        std::vector<float> dcr((size_t)T * R * R);
        for (int a = 0; a < T; ++a)
            for (int i = 0; i < R; ++i) {
                const double v = h->cnref[a * R + i];
                const float hi = (float)v;
                cr2[a * R + i] = make_float2(hi, (float)(v - (double)hi));
                for (int j = 0; j < R; ++j)
                    dcr[((size_t)a * R + i) * R + j] = (float)(h->cnref[a * R + j] - h->cnref[a * R + i]);
            }
        if (e == cudaSuccess) e = cudaMemcpy(h->d_cnref2, cr2.data(), cr2.size() * sizeof(float2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_dcr, dcr.data(), dcr.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h->d_c6f, c6f.data(), c6f.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_c6d, h->c6.data(), h->c6.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_rk, rk.data(), T * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<float4> rcp(T * T);
    for (int a2 = 0; a2 < T; ++a2)
        for (int b2 = 0; b2 < T; ++b2) {
            const double rc = p.k2 * (h->rcov[a2] + h->rcov[b2]);
            const float rh = (float)rc, rl = (float)(rc - (double)rh);
            const double rc2 = rc * rc;
            const float qh = (float)rc2, ql = (float)(rc2 - (double)qh);
            rcp[a2 * T + b2] = make_float4(rh, rl, qh, ql);
        }
    if (e == cudaSuccess) e = cudaMemcpy(h->d_rcpair, rcp.data(), rcp.size() * sizeof(float4), cudaMemcpyHostToDevice);
    std::vector<float2> ex2(64);
    for (int j = 0; j < 64; ++j) {
        const double v = std::exp2(j / 64.0);
        const float hi = (float)v;
        ex2[j] = make_float2(hi, (float)(v - (double)hi));
    }
    if (e == cudaSuccess) e = cudaMemcpy(h->d_exptab, ex2.data(), ex2.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_nbuild, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        h->tabmem.release();
        delete h;
        return D3_ERR_CUDA;
    }
    if (upload_pair_table(h) != D3_OK) {
        h->tabmem.release();
        delete h;
        return D3_ERR_CUDA;
    }
    *out = h;
    return D3_OK;
}

void d3_destroy(d3_handle* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (auto& v : h->ev_pending)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->plan.mem.release();
    h->stage.release();
    h->tabmem.release();
    if (h->h_status) cudaFreeHost(h->h_status);
    delete h;
}

d3_status d3_set_damping(d3_handle* h, double s6, double s8, double a1, double a2_bohr) {
    if (!h) return D3_ERR_ARG;
    if (!std::isfinite(s6) || !std::isfinite(s8) || !std::isfinite(a1) || !std::isfinite(a2_bohr))
        return fail(h, D3_ERR_ARG, "non-finite damping parameter");
    if (h->last_stream) cudaStreamSynchronize(h->last_stream);
    h->prm.s6 = s6;
    h->prm.s8 = s8;
    h->prm.a1 = a1;
    h->prm.a2_bohr = a2_bohr;
    ++h->param_gen;  // the damping parameters are kernel arguments of a captured graph
    return upload_pair_table(h);
}

d3_status d3_set_three_body(d3_handle* h, double s9, double alpha9, double rc3_A) {
    if (!h) return D3_ERR_ARG;
    if (!std::isfinite(s9)) return fail(h, D3_ERR_ARG, "non-finite s9");
    if (s9 != 0.0) {
        if (!(alpha9 > 0.0) || !(alpha9 <= 64.0)) return fail(h, D3_ERR_ARG, "alpha9 must lie in (0, 64]");
        if (!(rc3_A > 0.0) || !(rc3_A <= h->prm.rc_cn_A))
            return fail(h, D3_ERR_ARG, "rc3 must lie in (0, R_cn]: the triangles come from the CN lists");
    }
    if (h->last_stream) cudaStreamSynchronize(h->last_stream);
    h->s9 = s9;
    h->alpha9 = s9 != 0.0 ? alpha9 : 16.0;
    h->rc3_A = s9 != 0.0 ? rc3_A : 0.0;
    ++h->param_gen;  // kernel arguments of a captured graph
    return D3_OK;
}

d3_status d3_set_graphs(d3_handle* h, int32_t on) {
    if (!h) return D3_ERR_ARG;
    h->graphs = on != 0;
    return D3_OK;
}

d3_status d3_set_accumulate(d3_handle* h, int32_t on) {
    if (!h) return D3_ERR_ARG;
    h->accumulate = on != 0;
    return D3_OK;
}

d3_status d3_set_autotune(d3_handle* h, int32_t on) {
    if (!h) return D3_ERR_ARG;
    h->autotune = on != 0;
    return D3_OK;
}

d3_status d3_launch_shapes(d3_handle* h, int32_t* shapes, int64_t* tunings) {
    if (!h) return D3_ERR_ARG;
    if (shapes)
        for (int k = 0; k < 4; ++k) shapes[k] = h->shape[k];
    if (tunings) *tunings = h->tunings;
    return D3_OK;
}

d3_status d3_set_launch_shapes(d3_handle* h, const int32_t* shapes) {
    if (!h) return D3_ERR_ARG;
    if (!shapes) return fail(h, D3_ERR_ARG, "NULL shapes");
    for (int k = 0; k < 3; ++k)
        if (shapes[k] != kBlockCand[0] && shapes[k] != kBlockCand[1])
            return fail(h, D3_ERR_ARG, "pass blocks must have 64 or 128 threads");
    if (shapes[3] != kBuildCand[0] && shapes[3] != kBuildCand[1])
        return fail(h, D3_ERR_ARG, "the list builder takes 8 or 16 blocks per SM");
    h->autotune = false;
    set_shapes(h, shapes);
    return D3_OK;
}

d3_status d3_build_neighbors(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos,
                             const int32_t* types, const double* cells, const int32_t* pbc, void* stream) {
    d3_status s = check_batch_args(h, B, offsets, pos, types, cells, pbc);
    if (s != D3_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    if (B == 0) return D3_OK;
    const int mode = list_mode(h, nullptr);
    s = ensure_plan(h, B, offsets, pos, types, cells, pbc, st, mode);
    if (s != D3_OK) return s;
    s = enqueue_build(h, h->plan, pos, types, st, mode);
    if (s != D3_OK) return s;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "build");
    return d3_sync_status(h);
}

d3_status d3_compute_batch_ex(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos,
                              const int32_t* types, const double* cells, const int32_t* pbc, double* E, double* F,
                              double* W, double* e_atom, double* cn, void* stream) {
    return forward_graph(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, (cudaStream_t)stream, nullptr);
}

d3_status d3_compute_batch_atoms(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos,
                                 const int32_t* types, const double* cells, const int32_t* pbc, double* E,
                                 double* F, double* W, double* e_atom, double* cn, double* w_atom, void* stream) {
    if (h && B > 0 && offsets && offsets[B] > 0 && !w_atom) return fail(h, D3_ERR_ARG, "NULL w_atom");
    return forward_graph(h, B, offsets, pos, types, cells, pbc, E, F, W, e_atom, cn, (cudaStream_t)stream, w_atom);
}

d3_status d3_heat_current(int64_t n, const double* w_atom, const double* vel, double* J, void* stream) {
    if (n < 0 || (n > 0 && (!w_atom || !vel || !J))) return D3_ERR_ARG;
    return launch_heat(n, w_atom, vel, J, (cudaStream_t)stream) == cudaSuccess ? D3_OK : D3_ERR_CUDA;
}

d3_status d3_compute_batch(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos,
                           const int32_t* types, const double* cells, const int32_t* pbc, double* E, double* F,
                           double* W, void* stream) {
    return forward_graph(h, B, offsets, pos, types, cells, pbc, E, F, W, nullptr, nullptr, (cudaStream_t)stream,
                         nullptr);
}

d3_status d3_compute(d3_handle* h, const double* pos, const int32_t* types, int64_t n, const double* cell,
                     const int32_t* pbc, double* E, double* F, double* W, void* stream) {
    if (!h) return D3_ERR_ARG;
    if (n < 0 || !cell || !pbc) return fail(h, D3_ERR_ARG, "bad structure description");
    const int64_t off[2] = {0, n};
    return forward_graph(h, 1, off, pos, types, cell, pbc, E, F, W, nullptr, nullptr, (cudaStream_t)stream, nullptr);
}

static d3_status status_of_word(d3_handle* h, int st);

d3_status d3_compute_batch_host(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos,
                                const int32_t* types, const double* cells, const int32_t* pbc, double* E,
                                double* F, double* W, void* stream) {
    d3_status s = check_batch_args(h, B, offsets, pos, types, cells, pbc);
    if (s != D3_OK) return s;
    if (B == 0) return D3_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)offsets[B];
    if (N > h->stage_atoms || (size_t)B > h->stage_structs) {
        h->stage.release();
        h->stage_atoms = std::max(N, h->stage_atoms);
        h->stage_structs = std::max((size_t)B, h->stage_structs);
        cudaError_t e = h->stage.alloc(&h->s_pos, 3 * h->stage_atoms);
        if (e == cudaSuccess) e = h->stage.alloc(&h->s_F, 3 * h->stage_atoms);
        if (e == cudaSuccess) e = h->stage.alloc(&h->s_types, h->stage_atoms);
        if (e == cudaSuccess) e = h->stage.alloc(&h->s_E, h->stage_structs);
        if (e == cudaSuccess) e = h->stage.alloc(&h->s_W, 9 * h->stage_structs);
        if (e != cudaSuccess) {
            h->stage.release();
            h->stage_atoms = h->stage_structs = 0;
            return cuda_fail(h, e, "staging allocation");
        }
    }
    cudaError_t e = cudaMemcpyAsync(h->s_pos, pos, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->s_types, types, N * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "input copy");
    s = forward_graph(h, B, offsets, h->s_pos, h->s_types, cells, pbc, h->s_E, h->s_F, h->s_W, nullptr, nullptr, st,
                      nullptr);
    if (s != D3_OK) return s;
    if (!h->h_status) {
        e = cudaHostAlloc(&h->h_status, sizeof(int), cudaHostAllocDefault);
        if (e != cudaSuccess) {
            h->h_status = nullptr;
            return cuda_fail(h, e, "status word allocation");
        }
    }
    e = cudaMemcpyAsync(E, h->s_E, B * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, h->s_F, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W, h->s_W, 9 * (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, st);
    // the status word travels with the outputs and is cleared on the same stream: one synchronisation
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "output copy");
    return status_of_word(h, *h->h_status);
}

d3_status d3_backward(d3_handle* h, int32_t B, const int64_t* offsets, const double* pos, const int32_t* types,
                      const double* cells, const int32_t* pbc, const double* dLdE, const double* dLdF,
                      double* dLdparams, double* dLdpos, void* stream) {
    d3_status s = check_batch_args(h, B, offsets, pos, types, cells, pbc);
    if (s != D3_OK) return s;
    if (h->s9 != 0.0)
        return fail(h, D3_ERR_ARG, "the backward differentiates the two-body model; disable the three-body term");
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    if (B > 0 && !dLdE) return fail(h, D3_ERR_ARG, "NULL dLdE");
    if (offsets[B] > 0 && !dLdF) return fail(h, D3_ERR_ARG, "NULL dLdF");
    if (B == 0) {
        if (dLdparams) {
            cudaError_t e = cudaMemsetAsync(dLdparams, 0, 4 * sizeof(double), st);
            if (e != cudaSuccess) return cuda_fail(h, e, "memset");
        }
        return D3_OK;
    }
    s = ensure_plan(h, B, offsets, pos, types, cells, pbc, st, kFullLists);
    if (s != D3_OK) return s;
    Plan& P = h->plan;
    s = enqueue_build(h, P, pos, types, st, kFullLists);
    if (s != D3_OK) return s;
    const int64_t need = backward_scratch_doubles(P.w, B);
    if (need > P.bwd_scratch_n) {
        double* p = nullptr;
        cudaError_t e = P.mem.alloc(&p, (size_t)need);
        if (e != cudaSuccess) return cuda_fail(h, e, "backward scratch");
        P.bwd_scratch = p;
        P.bwd_scratch_n = need;
    }
    Consts c = make_consts(h);
    Tabs tbm{};  // FP32 tables of the mixed form
    tbm.c6 = h->d_c6f;
    tbm.nref = h->d_nref;
    tbm.rcpair = h->d_rcpair;
    tbm.exptab = h->d_exptab;
    tbm.cnref2 = h->d_cnref2;
    tbm.dcr = h->d_dcr;
    cudaError_t e = launch_backward(P.w, c, h->d_c6d, h->d_pairb, h->d_cnref, h->d_nref, tbm, dLdE, dLdF, dLdparams,
                                    dLdpos, P.bwd_scratch, B, h->prm.precision == D3_MIXED, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "backward launch");
    return D3_OK;
}

// The status word's flags as a library status (and the error text).
static d3_status status_of_word(d3_handle* h, int st) {
    if (st & ST_NONFINITE) return fail(h, D3_ERR_NONFINITE, "non-finite coordinate");
    if (st & ST_TYPE) return fail(h, D3_ERR_TYPE, "atom type out of range");
    if (st & ST_RANGE)
        return fail(h, D3_ERR_ARG, "a coordinate lies beyond the supported range (|x| < 4200 A after wrapping)");
    if (st & ST_SUM_RANGE)
        return fail(h, D3_ERR_ARG, "a dispersion partial sum exceeded its fixed-point range (|sum| < 2^23 Hartree "
                                   "or Hartree/bohr): the damping parameters or reference data are out of range");
    if (st & (ST_GHOST_CAP | ST_LIST_CAP)) {
        h->plan.sized[0] = h->plan.sized[1] = false;  // the next call re-measures and regrows
        return fail(h, D3_ERR_CAPACITY, "neighbour or image capacity exceeded; buffers will be regrown");
    }
    h->err.clear();
    return D3_OK;
}

d3_status d3_sync_status(d3_handle* h) {
    if (!h) return D3_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
    int st = 0;
    e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    return status_of_word(h, st);
}

const char* d3_last_error(const d3_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

d3_status d3_build_count(d3_handle* h, int64_t* builds) {
    if (!h || !builds) return D3_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    unsigned long long n = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&n, h->d_nbuild, sizeof(n), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "build count");
    *builds = (int64_t)n;
    return D3_OK;
}

d3_status d3_profile_enable(d3_handle* h, int32_t on) {
    if (!h) return D3_ERR_ARG;
    h->prof_on = on != 0;
    return D3_OK;
}

d3_status d3_profile_read(d3_handle* h, double* ms, int64_t* calls, int64_t* launches) {
    if (!h) return D3_ERR_ARG;
    for (auto& v : h->ev_pending) {
        cudaError_t e = cudaEventSynchronize(v[kStages]);
        if (e != cudaSuccess) return cuda_fail(h, e, "profile event");
        for (int k = 0; k < kStages; ++k) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, v[k], v[k + 1]) == cudaSuccess) {
                h->prof_ms[k] += t;
                h->prof_calls[k] += 1;
            }
        }
        float t = 0.f;  // the list builder (recorded when the build ran that kernel)
        if (cudaEventElapsedTime(&t, v[kStages + 1], v[kStages + 2]) == cudaSuccess) {
            h->prof_ms[kStages] += t;
            h->prof_calls[kStages] += 1;
        }
        cudaGetLastError();
        for (cudaEvent_t x : v) h->ev_pool.push_back(x);
    }
    h->ev_pending.clear();
    for (int k = 0; k < kStages; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (calls) calls[k] = h->prof_calls[k];
    }
    if (launches) *launches = h->launches;
    return D3_OK;
}

d3_status d3_profile_reset(d3_handle* h) {
    if (!h) return D3_ERR_ARG;
    d3_status s = d3_profile_read(h, nullptr, nullptr, nullptr);
    for (int k = 0; k < kStagesAll; ++k) {
        h->prof_ms[k] = 0;
        h->prof_calls[k] = 0;
    }
    h->launches = 0;
    return s;
}


d3_status d3_profile_stage(d3_handle* h, int32_t stage, double* ms, int64_t* calls) {
    if (!h || stage < 0 || stage >= kStagesAll) return D3_ERR_ARG;
    d3_status s = d3_profile_read(h, nullptr, nullptr, nullptr);
    if (s != D3_OK) return s;
    if (ms) *ms = h->prof_ms[stage];
    if (calls) *calls = h->prof_calls[stage];
    return D3_OK;
}

d3_status d3_list_stats(d3_handle* h, int64_t* stats) {
    if (!h || !stats) return D3_ERR_ARG;
    for (int k = 0; k < 8; ++k) stats[k] = 0;
    Plan& P = h->plan;
    if (!P.valid) return D3_OK;
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    auto sum_ints = [&](const int* d, int64_t n, int64_t* out) {
        if (e != cudaSuccess || !d || n <= 0) return;
        std::vector<int> v((size_t)n);
        e = cudaMemcpy(v.data(), d, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost);
        int64_t t = 0;
        for (int x : v) t += x;
        *out = t;
    };
    stats[0] = P.Nr;
    int ng = 0;
    if (e == cudaSuccess && P.ncells > 0)
        e = cudaMemcpy(&ng, P.w.start_ghost + P.ncells, sizeof(int), cudaMemcpyDeviceToHost);
    stats[1] = ng;
    stats[2] = P.ncl;
    const bool cl = P.last_mode == kClusterLists;
    if (cl) sum_ints(P.w.cnt_cl, P.ncl, &stats[3]);
    sum_ints(P.w.cnt_cn, P.Nr, &stats[4]);
    if (!cl) sum_ints(P.w.cnt_disp, P.Nr, &stats[5]);
    if (e == cudaSuccess && cl && P.npairs) {
        unsigned long long np = 0;
        e = cudaMemcpy(&np, P.npairs, sizeof(np), cudaMemcpyDeviceToHost);
        stats[6] = (int64_t)np;
    }
    stats[7] = P.last_mode;
    if (e != cudaSuccess) return cuda_fail(h, e, "list statistics");
    return D3_OK;
}

d3_status d3_tune_times(d3_handle* h, float* ms) {
    if (!h || !ms) return D3_ERR_ARG;
    for (int k = 0; k < 8; ++k) ms[k] = h->tune_ms[k];
    return D3_OK;
}

}  // extern "C"
