// d3gb_internal.cuh -- shared device-side types of the D3(BJ) library.
//
// Data layout in device memory (one "plan" per batch geometry):
//   real atoms   sorted by (structure, cell); structure s owns sorted slots
//                [atom_base_s, atom_base_s + natoms_s), the same range it has
//                in the caller's input order.
//   image atoms  ("ghosts") periodic images of real atoms that fall inside the
//                list radius of the cell; stored after the real atoms, sorted
//                by cell.  Atom index q < Nr is real, q >= Nr is an image.
//   per atom q   pos64[q] = (x, y, z, k2*Rcov) in bohr, FP64
//                rec[q] = 32-byte record {hi.xyz, tsrc, lo.xyz, k2*Rcov}: the FP32
//                split of the position (x = hi + lo, hi on a 2^-10 bohr grid),
//                tsrc = type | (data source << 4) as int bits.  One 256-bit
//                load fetches the whole record.
//   lists        per structure, one row of cap_s entries per atom:
//                entry k of sorted atom p is at list_base_s + (p - atom_base_s) * cap_s + k.
//                A thread appends to its own row, so every 32-byte sector is
//                filled by one thread, and reads it 4 entries per 16-byte load.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace d3gb {

// 32-byte aligned quadruple of doubles (one memory sector per load).
struct __align__(32) dbl4 {
    double x, y, z, w;
};
__host__ __device__ inline dbl4 dbl4_make(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

constexpr double kBohrA = 0.529177210903;       // A per bohr
constexpr double kHartreeEV = 27.211386245988;  // eV per Hartree
constexpr int kMaxTypes = 16;
constexpr int kMaxRef = 7;
constexpr int kChunk = 64;  // pairs summed in FP32 before an FP64 accumulate (mixed form)
constexpr int kFinChunk = 4096;  // atoms per first-level block of the per-structure sums

enum StatusBits : int {
    ST_GHOST_CAP = 1,
    ST_LIST_CAP = 2,
    ST_NONFINITE = 4,
    ST_TYPE = 8,
    ST_RANGE = 16,  // a wrapped coordinate beyond kMaxCoordBohr
    ST_SUM_RANGE = 32,  // a partial sum of the cluster-list dispersion pass beyond its fixed-point range
};
// Largest |coordinate| (bohr) after wrapping: the 2^-10 bohr grid split of a
// position is exact in FP32 below 2^13 bohr; the rest is margin for images.
constexpr float kMaxCoordBohr = 8000.0f;

// Per-structure geometry, computed on the host from the cell and pbc.
struct StructGeo {
    double H[9];      // lattice rows, bohr
    double Hinv[9];   // inverse: f = x * Hinv
    double lo[3];     // fractional coordinate of the grid origin along each axis
    double fscale[3]; // grid cells per unit of fractional coordinate
    double ext_lo[3], ext_hi[3];  // fractional window of image atoms (periodic axes)
    // FP32 copies for the binning and image decisions (the list radius margin
    // covers their rounding): inverse cell, grid origin and scale, image window
    float Hinvf[9], lof[3], fscalef[3], ext_lof[3], ext_hif[3];
    // lattice rows split like positions: Hh on the 2^-10 bohr grid, Hl = H - Hh (FP32)
    float Hh[9], Hl[9];
    int ncell[3];
    int win[3];       // window half-width (cells) covering the list radii
    int win_cn[3];    // window half-width (cells) covering the CN list radius
    int img[3];       // image range, 0 along open axes
    int pbc[3];
    int64_t cell_base;
    int64_t atom_base;
    int32_t natoms;
    int32_t cap_disp, cap_cn;
    int32_t cap_cl;     // entries per row of the cluster lists
    int64_t fin_base;   // first chunk of the structure in the per-structure sums
    int64_t list_base_disp, list_base_cn;
    int64_t clu_base;     // first cluster of the structure
    int64_t list_base_cl;  // first entry of the structure's cluster-list rows
};

// Cells are numbered in serpentine order within a structure: planes along z,
// rows along y in alternating direction from plane to plane, cells along x in
// alternating direction from row to row, so that consecutive cells are always
// neighbours and runs of consecutive sorted atoms stay compact.  A row of cells
// (fixed y, z) is still one contiguous range of ids.
__host__ __device__ inline int64_t cell_index(const StructGeo& G, int cx, int cy, int cz) {
    const int yy = (cz & 1) ? G.ncell[1] - 1 - cy : cy;
    const int64_t row = (int64_t)cz * G.ncell[1] + yy;
    const int xx = (row & 1) ? G.ncell[0] - 1 - cx : cx;
    return G.cell_base + row * G.ncell[0] + xx;
}
// (a structure has fewer than 2^26 cells, so 32-bit divisions suffice)
__host__ __device__ inline void cell_coords(const StructGeo& G, int64_t id, int& cx, int& cy, int& cz) {
    const int rel = (int)(id - G.cell_base);
    const int row = rel / G.ncell[0];
    const int xx = rel - row * G.ncell[0];
    cz = row / G.ncell[1];
    const int yy = row - cz * G.ncell[1];
    cy = (cz & 1) ? G.ncell[1] - 1 - yy : yy;
    cx = (row & 1) ? G.ncell[0] - 1 - xx : xx;
}
// first and last cell id of cells x0..x1 of row (cy, cz)
__host__ __device__ inline void row_cells(const StructGeo& G, int cy, int cz, int x0, int x1, int64_t& first,
                                          int64_t& last) {
    const int64_t a = cell_index(G, x0, cy, cz), b = cell_index(G, x1, cy, cz);
    first = a < b ? a : b;
    last = a < b ? b : a;
}
// Atoms per cluster of the cluster lists (consecutive sorted real atoms of a structure).
constexpr int kClusterAtoms = 8;

// Pointers and sizes of one plan's workspace, passed by value to kernels.
struct Work {
    const StructGeo* geo;
    const int64_t* offsets;  // [B+1]
    const int* sid_in;       // [Nr] structure of each atom in input order
    int B;
    int64_t Nr;              // real atoms
    int64_t ncells;          // total cells
    int ghost_cap;
    int T, R, RP;            // types, references, padded references
    // binning
    int* cnt_real;           // [ncells + 1]
    int* cnt_ghost;          // [ncells + 1]
    int* start_real;         // [ncells + 1]
    int* start_ghost;        // [ncells + 1]
    int* cell_of;            // [Nr] input order
    int* slot_of;            // [Nr]
    double* xw;              // [Nr*3] wrapped positions, bohr, input order
    int* ghost_src;          // [ghost_cap] input index of the source atom
    int* ghost_shift;        // [ghost_cap] packed lattice translation
    int* ghost_cell;         // [ghost_cap]
    int* ghost_slot;         // [ghost_cap]
    int* ghost_sid;          // [ghost_cap] structure of the image
    int* ghost_count;        // [1]
    int* sorted_src;         // [Nr] sorted -> input index
    int* gsorted;            // [ghost_cap] sorted image slot -> raw image record
    int* ginv;               // [ghost_cap] raw image record -> sorted image slot
    int* gfirst;             // [Nr] input atom -> its first raw image record (its images are consecutive)
    int* gcnt;               // [Nr] input atom -> its number of image records
    int* usrc;               // [Nr + ghost_cap] cell order before the in-cell sort: input index / image record
    long long* ukey;         // [Nr + ghost_cap] the in-cell sort key of each such slot
    // per atom, sorted
    dbl4* pos64;             // [Nr + ghost_cap]
    float4* rec;             // [2 * (Nr + ghost_cap)]: hi at 2q, lo at 2q + 1
    float4* hi;              // [Nr + ghost_cap] compact copy of the hi parts for the list build
    float* fw;               // [Nr * 3] wrapped fractional coordinates (FP32), input order
    int* frange;             // [2][B][3] float bits: min and max occupied fraction per axis
    int* perm;               // [Nr] sorted -> input index
    int* sid;                // [Nr] structure of sorted real atom
    int* cell_sorted;        // [Nr] global cell id of sorted real atom
    // neighbour lists
    int* nbr_disp;
    int* nbr_cn;
    int* cnt_disp;           // [Nr]
    int* cnt_cn;             // [Nr]
    int* maxcnt;             // [3*B] max list length per structure (disp, cn, cluster)
    int* work_ctr;           // [2] persistent-kernel work counters (zeroed before each build)
    // cluster lists of the dispersion pass (mixed form)
    int cl_mode;             // build: 1 = CN per-atom lists and cluster lists, 0 = both per-atom lists
    int64_t ncl;             // clusters over the batch
    const int* clu_sid;      // [ncl] structure of each cluster
    int* nbr_cl;             // rows of cap_cl entries per cluster
    int* cnt_cl;             // [ncl]
    unsigned long long* acc; // [Nr][8] fixed-point sums of the dispersion pass: F (3), dE/dn, site energy
    float* gcn;              // mixed form: per CN-list entry, the chain coefficient f'(r)/r of Eq. 4
                             // (written by the CN pass, 0 outside R_cn; read by the chain pass)
    float* vd;               // [Nr (+ ghost_cap)][T][2][RP] per atom q and partner type t: v_q^(t) and
                             // dv_q^(t)_a = sum_b C6ref[t][tq][a][b] dW_qb
    int vd_images;           // 1: image atoms have rows (copies of their source's, written by the CN pass),
                             // 0: the dispersion pass reads their source's
    float* skey;             // [Nr] within-cell sort key (position along the serpentine direction), input order
    unsigned long long* npairs;  // [1] unique pairs within R_pot of the last cluster-mode dispersion pass
    // list reuse (skin > 0): the build kernels run only while *gate != 0
    int* gate;               // nullptr: unconditional build; else set by k_check when an atom moved > skin/2
    double* xref;            // [Nr*3] positions (bohr, input order) at the last build
    double* wshift;          // [Nr*3] translation the wrap applied at the last build (bohr)
    double skin_half2;       // (skin / 2)^2, bohr^2
    unsigned long long* nbuild;  // [1] builds executed
    int num_sms;
    // launch shapes (read on the host when enqueueing; every choice gives the same results)
    int blk_cn, blk_disp, blk_chain;  // threads per block of the CN, dispersion and chain passes
    int build_per_sm;                 // list-builder blocks per SM
    float rl_disp2, rl_cn2;  // list radii squared, bohr^2
    // passes
    double* cn;              // [Nr]
    void* W;                 // [Nr][RP] real
    void* dW;                // [Nr][RP] real
    void* v;                 // [Nr][T][RP] real: v_q^(t)_a = sum_b C6ref[t][tq][a][b] W_qb (RP = 4 or 8)
    void* dEdn;              // [Nr] real
    void* Fd;                // [Nr][4] real (direct forces)
    double* eat;             // [Nr] site energies, Ha
    double* wv;              // [Nr][6] per-atom virial (xx yy zz xy xz yz), Ha
    void* Pv;                // [Nr][4] real: P_i = sum_j (dU_j/dn_i) r_ij (per-atom virial of Eq. 7 only)
    double* fin_part;        // [n_fin][7] chunk sums, structure s owning chunks [fin_base_s, fin_base_s + ceil(natoms_s / kFinChunk))
    const int* fin_sid;      // [n_fin] structure of each chunk
    int64_t n_fin;           // chunks over the batch
    int64_t max_natoms;
    int* status;
};

// Per-handle constants of the pair arithmetic.
struct Consts {
    double rc_disp2, rc_cn2;   // bohr^2
    float rc_disp2f;           // FP32 copy for the mixed form
    double k1, k3;
    double s6, s8, a1, a2;     // damping of Eq. 2 (a2 in bohr)
    int T, R, RP;
    int accumulate;            // add E, F, W into the outputs instead of overwriting them
    // optional three-body (triple-dipole) term, off when atm == 0
    int atm;
    double s9, alpha9;         // strength and damping exponent
    double rc3_2;              // every side of a triangle below rc3: rc3^2, bohr^2 (rc3 <= R_cn)
    float s9f, alpha9f, alpha9_3f, rc3_2f;  // FP32 copies (alpha9_3f = alpha9 / 3) for the mixed form
    float k1f, rc_cn2f, k3f;   // FP32 copies for the mixed form
    float k3h, k3l;            // k3 as a float pair (k3h + k3l)
};

// ---- neighbour lists: `cap` entries per atom (cap a multiple of 8).  The rows of
// 32 consecutive atoms of a structure are interleaved in groups of 4 entries:
// entry k of local atom a is at base + (a / 32) 32 cap + (k / 4) 128 + (a % 32) 4 + k % 4,
// so when the threads of a warp (consecutive atoms) each read entries k..k+3 of
// their own rows, the warp reads 512 contiguous bytes.  list_row gives the
// address of entry 0 of an atom's row, list_off(k) the offset of entry k from it.
__host__ __device__ inline int64_t list_row(int64_t base, int64_t local, int cap) {
    return base + (local >> 5) * 32 * (int64_t)cap + (local & 31) * 4;
}
__host__ __device__ inline int list_off(int k) { return (k >> 2) * 128 + (k & 3); }
__host__ __device__ inline int round_cap(double c) {
    int v = (int)c;
    return (v + 7) & ~7;
}
__host__ __device__ inline int64_t list_size(int64_t natoms, int cap) { return ((natoms + 31) >> 5) * 32 * (int64_t)cap; }

// 256-bit read-only load (sm_100 and later)
__device__ __forceinline__ void ld8(const float* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}
__device__ __forceinline__ void rec_load(const Work& w, int64_t q, float4& hi, float4& lo) {
    ld8(reinterpret_cast<const float*>(w.rec + 2 * q), hi, lo);
}
__device__ __forceinline__ float4 rec_hi(const Work& w, int64_t q) { return __ldg(w.rec + 2 * q); }
__device__ __forceinline__ int rec_tsrc(const Work& w, int64_t q) { return __float_as_int(__ldg(&w.rec[2 * q].w)); }

struct ListView {
    const int* p;  // the atom's row (list_row)
    // fn(q) for entries [k0, k1); k0 must be a multiple of 4
    template <class Fn>
    __device__ __forceinline__ void for_each(int k0, int k1, Fn&& fn) const {
        for (int k = k0; k < k1; k += 4) {
            const int4 q4 = __ldg(reinterpret_cast<const int4*>(p + list_off(k)));
            fn(q4.x);
            if (k + 1 < k1) fn(q4.y);
            if (k + 2 < k1) fn(q4.z);
            if (k + 3 < k1) fn(q4.w);
        }
    }
};

__host__ __device__ inline int pack_shift(int a, int b, int c) {
    return (a + 128) | ((b + 128) << 8) | ((c + 128) << 16);
}
__host__ __device__ inline void unpack_shift(int s, int& a, int& b, int& c) {
    a = (s & 255) - 128;
    b = ((s >> 8) & 255) - 128;
    c = ((s >> 16) & 255) - 128;
}

// Structure of input atom i (binary search over offsets).
__device__ inline int struct_of(const int64_t* off, int B, int64_t i) {
    int lo = 0, hi = B;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace d3gb

// Launchers implemented in the build and pass translation units.
namespace d3gb {
cudaError_t launch_build(const Work& w, const double* pos, const int32_t* types, cudaStream_t st);
// Displacement check of list reuse: sets *w.gate when an atom moved more than
// skin/2 since the last build (or is not finite) and moves every atom's
// wrapped position by its new displacement.
cudaError_t launch_check(const Work& w, const double* pos, cudaStream_t st);
// Device tables of one handle.
struct Tabs {
    const void* c6;        // [T][T][R][R] real (float or double by precision)
    const void* pair;      // [T][T] real4: R^6, R^8, s6, s8 R0^2
    const double* cnref;   // [T][R]
    const int* nref;       // [T]
    const float4* rcpair;  // [T][T] k2 (Rcov_i + Rcov_j) as hi, lo and its square as hi, lo (bohr)
    const float2* exptab;  // [64] 2^(j/64) as FP32 hi, lo
    const float2* cnref2;  // [T][R] reference CNs as FP32 hi, lo
    const float* dcr;      // [T][R][R] cnref[t][b] - cnref[t][a], rounded to FP32
    const void* rtab;      // [T][T] real: damping radius R = a1 R0 + a2 of Eq. 2 (bohr), for the three-body term
};

// marks (optional): 7 events recorded before the CN pass and after the CN,
// weight, dispersion, three-body, chain and finalize passes.
// w_atom (optional, device double[N][9]): per-atom virial of Eq. 7, eV.
cudaError_t launch_forward(const Work& w, const Consts& c, bool mixed, const Tabs& tabs, double* E, double* F,
                           double* W, double* e_atom, double* cn_out, double* w_atom, int B, cudaStream_t st,
                           cudaEvent_t* marks);
// Dispersion pass of the mixed form over the cluster lists (d3gb_cluster.cu):
// fills w.Fd, w.dEdn, w.eat and w.wv like the per-atom-list pass (with site =
// false, w.eat holds per-cluster sums on each cluster's first atom instead of
// site energies).
cudaError_t launch_disp_cl(const Work& w, const Consts& c, const void* pair_tab, bool site, cudaStream_t st);
// Optional three-body pass (d3gb_atm.cu): adds into w.eat, w.wv, w.Fd and
// w.dEdn after the dispersion pass; rtab as Tabs::rtab in the handle's precision.
cudaError_t launch_atm(const Work& w, const Consts& c, bool mixed, const void* rtab, cudaStream_t st);
// Eq. 8 per atom: J_i = W_i . v_i (device arrays).
cudaError_t launch_heat(int64_t n, const double* w_atom, const double* vel, double* J, cudaStream_t st);
constexpr int kForwardLaunches = 5;  // kernels per forward pass (B > 0, N > 0): CN, dispersion, chain, 2 sums
                                     // (one more with the three-body term; in cluster mode one more,
                                     // the fixed-point finish)
constexpr int kBuildLaunches = 10;   // kernels per neighbour build (N > 0): reset, wrap, images, 3 scan (both
                                     // count arrays), scatter, rank (in-cell sort), fill, lists (per-atom or
                                     // cluster lists)
}  // namespace d3gb
