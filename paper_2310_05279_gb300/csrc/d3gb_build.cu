// d3gb_build.cu -- neighbour build of the D3(BJ) pipeline (cell lists).
//
// The sums of Eq. 2 and Eq. 4 (arXiv 2310.05279, Sec. II A) run over the
// neighbours of each atom within R_pot and R_cn, periodic images included.
// This file turns caller-order positions into:
//   * wrapped positions and a cell index per atom in a fractional grid that
//     also covers a margin of one list radius around the cell,
//   * explicit image atoms ("ghosts") for every periodic image that falls in
//     that margin, so the pair kernels never apply lattice translations,
//   * a counting sort of real atoms and of image atoms by cell (serpentine
//     cell numbering), each cell then ordered by a unique key (rank sort),
//   * FP64 and split-FP32 (hi + lo) positions of every atom in sorted order,
//   * per-atom neighbour lists within the two list radii, or (cluster mode)
//     per-atom lists within the CN radius and, for the dispersion pass,
//     half lists per cluster of 8 consecutive sorted atoms.
// Every kernel writes only inside the capacities it is given and records an
// overflow in the status word instead.
#include <algorithm>

#include "d3gb_internal.cuh"

namespace d3gb {

namespace {

// A build kernel does nothing when list reuse is on and no atom has moved enough.
__device__ __forceinline__ bool skip_build(const Work& w) { return w.gate && *w.gate == 0; }

// The binning, wrap and image decisions below are taken in FP32: GB300 runs
// FP64 at 1/64 of the FP32 rate, and the list radius carries a margin (4e-3
// bohr plus 1e-5 relative) far above their rounding (about 3e-5 bohr at 500
// bohr), so an atom binned one cell off, or an image kept or dropped at the
// edge of its window, changes no pair within the cutoffs.  Positions
// themselves stay FP64.
// Cell of a fractional position (serpentine numbering, cell_index); *fx is the
// position along the cell's row in the direction the numbering runs, the key
// that orders atoms inside a cell.
__device__ inline int cell_id(const StructGeo& G, const float f[3], float* fx = nullptr) {
    int c[3];
    float u0 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float u = (f[k] - G.lof[k]) * G.fscalef[k];
        u = fminf(fmaxf(u, 0.0f), (float)(G.ncell[k] - 1));
        if (k == 0) u0 = u;
        c[k] = (int)u;
    }
    const int64_t id = cell_index(G, c[0], c[1], c[2]);
    if (fx) {
        const int row = (int)(id - G.cell_base) / G.ncell[0];  // fewer than 2^26 cells per structure
        *fx = (row & 1) ? -u0 : u0;
    }
    return (int)id;
}

__device__ __forceinline__ bool finite_bits(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// x += n0 H_0 + n1 H_1 + n2 H_2 (lattice rows, bohr).  Translations are nearly
// always 0 or +-1 per axis, so those cost one FP64 add per component.
__device__ __forceinline__ void add_lattice(double (&x)[3], const StructGeo& G, int n0, int n1, int n2) {
    const int n[3] = {n0, n1, n2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (n[k] == 0) continue;
        const double* Hk = G.H + 3 * k;
        if (n[k] == 1) {
            x[0] += Hk[0]; x[1] += Hk[1]; x[2] += Hk[2];
        } else if (n[k] == -1) {
            x[0] -= Hk[0]; x[1] -= Hk[1]; x[2] -= Hk[2];
        } else {
            const double d = n[k];
            x[0] += d * Hk[0]; x[1] += d * Hk[1]; x[2] += d * Hk[2];
        }
    }
}

// Wrap into the cell, bin, and record each structure's occupied fractional
// range per periodic axis (as float bits: the fractions are >= 0).  The
// lattice translation that wraps an atom is chosen from its FP32 fractional
// coordinates; the wrapped position is x - sum_k n_k H_k in FP64 (x itself
// when the atom is inside the cell).
__global__ void __launch_bounds__(256) k_wrap(Work w, const double* __restrict__ pos, const int32_t* __restrict__ types) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.Nr || skip_build(w)) return;
    const int s = w.sid_in[i];
    const StructGeo& G = w.geo[s];
    double xb[3];
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xb[a] = pos[3 * i + a] * (1.0 / kBohrA);
        fin = fin && finite_bits(xb[a]);
    }
    if (!fin) {
        atomicOr(w.status, ST_NONFINITE);
        xb[0] = xb[1] = xb[2] = 0.0;
    }
    const int t = types[i];
    if (t < 0 || t >= w.T) atomicOr(w.status, ST_TYPE);
    const float xf[3] = {(float)xb[0], (float)xb[1], (float)xb[2]};
    float f[3];
    int n[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        f[k] = xf[0] * G.Hinvf[k] + xf[1] * G.Hinvf[3 + k] + xf[2] * G.Hinvf[6 + k];
        if (G.pbc[k]) {
            const float fl = floorf(f[k]);
            n[k] = (int)fl;
            f[k] -= fl;  // exact, in [0, 1]
            if (f[k] >= 1.0f) {
                f[k] = 0.0f;
                n[k] += 1;
            }
        }
        w.fw[3 * i + k] = f[k];
    }
    double xw[3] = {xb[0], xb[1], xb[2]};
    if (n[0] | n[1] | n[2]) add_lattice(xw, G, -n[0], -n[1], -n[2]);
    // the exact FP32 split of positions needs |x| < 2^13 bohr (checked in FP32)
    bool far = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xr = xf[a] - ((float)n[0] * G.Hh[a] + (float)n[1] * G.Hh[3 + a] + (float)n[2] * G.Hh[6 + a]);
        far = far || !(fabsf(xr) < kMaxCoordBohr);
    }
    if (far && fin) atomicOr(w.status, ST_RANGE);
#pragma unroll
    for (int a = 0; a < 3; ++a) w.xw[3 * i + a] = xw[a];
    if (w.skin_half2 > 0.0) {  // references for list reuse
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            w.xref[3 * i + a] = xb[a];
            w.wshift[3 * i + a] = xw[a] - xb[a];
        }
    }
    float key;
    const int cid = cell_id(G, f, &key);
    w.cell_of[i] = cid;
    w.skey[i] = key;
    w.slot_of[i] = atomicAdd(&w.cnt_real[cid], 1);
    // occupied range: one atomic per group of lanes in the same structure
    const unsigned grp = __match_any_sync(__activemask(), s);
    const bool leader = (threadIdx.x & 31) == __ffs(grp) - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!G.pbc[k]) continue;
        const int lo = __reduce_min_sync(grp, __float_as_int(f[k]));
        const int hi = __reduce_max_sync(grp, __float_as_int(f[k]));
        if (leader) {
            atomicMin(&w.frange[3 * s + k], lo);
            atomicMax(&w.frange[3 * (w.B + s) + k], hi);
        }
    }
}

// Periodic images that can be within the list radius of a real atom: along a
// periodic axis an image is kept when its fraction lies within delta (list
// radius / plane spacing) of the structure's occupied range.  Slots are
// reserved once per block (each thread counts, the block scans, one atomic).
__global__ void __launch_bounds__(256) k_images(Work w) {
    if (skip_build(w)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < w.Nr;
    const int s = live ? w.sid_in[i] : 0;
    const StructGeo& G = w.geo[s];
    float f[3] = {0, 0, 0};
    int nlo[3] = {0, 0, 0}, nhi[3] = {0, 0, 0};
    float u0[3] = {0, 0, 0};
    if (live) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            f[k] = w.fw[3 * i + k];
            u0[k] = (f[k] - G.lof[k]) * G.fscalef[k];
            if (G.img[k] > 0) {
                const float delta = G.ext_hif[k] - 1.0f;
                const float omin = __int_as_float(w.frange[3 * s + k]);
                const float omax = __int_as_float(w.frange[3 * (w.B + s) + k]);
                nlo[k] = max(-G.img[k], (int)ceilf(fmaxf(G.ext_lof[k], omin - delta) - f[k]));
                nhi[k] = min(G.img[k], min((int)ceilf(G.ext_hif[k] - f[k]) - 1, (int)floorf(omax + delta - f[k])));
            }
        }
    }
    int mine = 0;
    if (live && nhi[0] >= nlo[0] && nhi[1] >= nlo[1] && nhi[2] >= nlo[2]) {
        mine = (nhi[0] - nlo[0] + 1) * (nhi[1] - nlo[1] + 1) * (nhi[2] - nlo[2] + 1);
        // the identity is always inside the range; it is the atom itself
        mine -= 1;
    }
    // block scan of the counts
    __shared__ int wsum[8];
    __shared__ int base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            const int v = wsum[k];
            wsum[k] = acc;
            acc += v;
        }
        base = acc > 0 ? atomicAdd(w.ghost_count, acc) : 0;
    }
    __syncthreads();
    if (live) {  // the atom's image records are consecutive from here
        w.gfirst[i] = base + wsum[wid] + x - mine;
        w.gcnt[i] = mine > 0 ? mine : 0;
    }
    if (!live || mine <= 0) return;
    int slot = base + wsum[wid] + x - mine;
    auto cell_of_axis = [&](int k, int n) {
        const int c = (int)floorf(u0[k] + (float)n * G.fscalef[k]);
        return min(max(c, 0), G.ncell[k] - 1);
    };
    for (int n0 = nlo[0]; n0 <= nhi[0]; ++n0) {
        const int cx = cell_of_axis(0, n0);
        for (int n1 = nlo[1]; n1 <= nhi[1]; ++n1) {
            const int cy = cell_of_axis(1, n1);
            for (int n2 = nlo[2]; n2 <= nhi[2]; ++n2) {
                if (n0 == 0 && n1 == 0 && n2 == 0) continue;
                if (slot >= w.ghost_cap) {
                    atomicOr(w.status, ST_GHOST_CAP);
                    return;
                }
                const int cz = cell_of_axis(2, n2);
                const int gc = (int)cell_index(G, cx, cy, cz);
                w.ghost_src[slot] = (int)i;
                w.ghost_shift[slot] = pack_shift(n0, n1, n2);
                w.ghost_cell[slot] = gc;
                w.ghost_slot[slot] = atomicAdd(&w.cnt_ghost[gc], 1);
                w.ghost_sid[slot] = s;
                ++slot;
            }
        }
    }
}

// ---- exclusive scan of int counts (n entries) into start[0..n], start[n] = total
constexpr int kScanBlock = 1024;

__device__ inline int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    int before = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// Two arrays at once (the real and the image counts per cell): array a = 0, 1 is
// cnt[a] -> start[a], with its block sums at bsum + a nb.
struct ScanPair {
    const int* cnt[2];
    int* start[2];
};

__global__ void k_scan_blocks(ScanPair sp, int* __restrict__ bsum, int nb, int64_t n, const int* gate) {
    if (gate && *gate == 0) return;
    const int a = blockIdx.y;
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int v = i < n ? sp.cnt[a][i] : 0;
    int tot;
    int ex = block_exclusive_scan(v, &tot);
    if (i < n) sp.start[a][i] = ex;
    if (threadIdx.x == 0) bsum[a * nb + blockIdx.x] = tot;
}

__global__ void k_scan_sums(ScanPair sp, int* bsum_all, int nb, int64_t n, const int* gate) {
    if (gate && *gate == 0) return;
    int* bsum = bsum_all + blockIdx.x * nb;
    int* start = sp.start[blockIdx.x];
    int carry = 0;
    for (int base = 0; base < nb; base += kScanBlock) {
        int i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, &tot);
        if (i < nb) bsum[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_scan_add(ScanPair sp, const int* __restrict__ bsum, int nb, int64_t n, const int* gate) {
    if (gate && *gate == 0) return;
    const int a = blockIdx.y;
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) sp.start[a][i] += bsum[a * nb + blockIdx.x];
}

// ---- cell order
// Deterministic order inside each cell: real atoms by their position along the
// cell's row in the direction the serpentine numbering runs (ties by input
// index), so that runs of consecutive sorted atoms, the clusters of the
// dispersion pass, are compact; images by (source, translation).  Both keys are
// unique 64-bit integers.
__device__ __forceinline__ long long image_key(const Work& w, int g) {
    return ((long long)w.ghost_src[g] << 24) | (long long)w.ghost_shift[g];
}
// order-preserving map of a float to an unsigned int
__device__ __forceinline__ unsigned float_order(float x) {
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ long long real_key(const Work& w, int i) {
    return (long long)(((unsigned long long)float_order(w.skey[i]) << 32) | (unsigned)i);
}

// Scatter into cell order by the slots the binning reserved (an arbitrary order
// inside each cell), with each slot's key: threads [0, Nr) the real atoms, then
// the images (slots Nr + ... of usrc and ukey).
__global__ void k_scatter(Work w) {
    if (skip_build(w)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < w.Nr) {
        const int k = w.start_real[w.cell_of[i]] + w.slot_of[i];
        w.usrc[k] = (int)i;
        w.ukey[k] = real_key(w, (int)i);
        return;
    }
    const int64_t g = i - w.Nr;
    const int ng = min(*w.ghost_count, w.ghost_cap);
    if (g >= ng) return;
    const int64_t k = w.Nr + w.start_ghost[w.ghost_cell[g]] + w.ghost_slot[g];
    w.usrc[k] = (int)g;
    w.ukey[k] = image_key(w, (int)g);
}

// Each slot's final place in its cell is the number of smaller keys in the cell
// (one thread per slot; the threads of a cell read the same keys).  Writes the
// sorted order and, for real atoms, its inverse (slot_of[i] = sorted slot of
// input atom i; until here slot_of held the atoms' places in their cells).
__global__ void __launch_bounds__(256) k_rank(Work w) {
    if (skip_build(w)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool real = t < w.Nr;
    const int ng = min(*w.ghost_count, w.ghost_cap);
    if (!real && t - w.Nr >= ng) return;
    const int u = w.usrc[t];
    const int c = real ? w.cell_of[u] : w.ghost_cell[u];
    const int* start = real ? w.start_real : w.start_ghost;
    const int64_t off = real ? 0 : w.Nr;
    const int b = start[c], e = start[c + 1];
    const long long mine = w.ukey[t];
    const long long* key = w.ukey + off;
    int rank = 0;
    for (int m = b; m < e; ++m) rank += key[m] < mine ? 1 : 0;
    if (real) {
        w.sorted_src[b + rank] = u;
        w.slot_of[u] = b + rank;
    } else {
        w.gsorted[b + rank] = u;
        w.ginv[u] = b + rank;
    }
}

// Zero the counters of a build (and count the build).
__global__ void k_reset(Work w) {
    if (skip_build(w)) return;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= w.ncells) {
        w.cnt_real[k] = 0;
        w.cnt_ghost[k] = 0;
    }
    if (k < 3 * (int64_t)w.B) w.maxcnt[k] = 0;
    // occupied-range minima start at a huge float, maxima at +0
    if (k < 3 * (int64_t)w.B) {
        w.frange[k] = 0x7f7f7f7f;
        w.frange[3 * w.B + k] = 0;
    }
    if (k == 0) {
        *w.ghost_count = 0;
        w.work_ctr[0] = 0;
        w.work_ctr[1] = 0;
        atomicAdd(w.nbuild, 1ull);
    }
}

// List reuse: gate the build on the largest displacement since the last
// build, and carry every atom's wrapped position along with its displacement
// (the wrap overwrites it when the build runs).
__global__ void __launch_bounds__(256) k_check(Work w, const double* __restrict__ pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.Nr) return;
    double d2 = 0.0;
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * i + a] * (1.0 / kBohrA);
        fin = fin && isfinite(x);
        const double d = x - w.xref[3 * i + a];
        d2 += d * d;
        w.xw[3 * i + a] = x + w.wshift[3 * i + a];
    }
    if (!fin || !(d2 <= w.skin_half2)) atomicOr(w.gate, 1);
}

// Split position: hi on a 2^-10 bohr grid (exact in FP32 for |x| < 2^13 bohr),
// lo = x - hi (|lo| <= 2^-11).  Differences of hi parts are then exact in
// FP32, so a pair vector is recovered as D + e with no rounding lost.
// hi is the grid point nearest x, found from the float pair x = xh + xl (xl
// exact to 2^-24 |xh|) without FP64 products: m = rint(1024 xh), then the
// remainder 1024 (xh - m/1024) + 1024 xl, exact in FP32 below 2^-10 by
// Sterbenz, moves m by one when it exceeds 1/2.
__device__ inline void split_pos(const double x[3], float (&h)[3], float (&l)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xh = (float)x[a];
        const float xl = (float)(x[a] - (double)xh);
        float m = rintf(xh * 1024.0f);
        const float r = (xh * 1024.0f - m) + xl * 1024.0f;
        if (r > 0.5f) m += 1.0f;
        else if (r < -0.5f) m -= 1.0f;
        h[a] = m * (1.0f / 1024.0f);
        l[a] = (xh - h[a]) + xl;
    }
}
__device__ inline void store_pos(Work& w, int64_t q, const double x[3], double rk, int tsrc) {
    w.pos64[q] = dbl4_make(x[0], x[1], x[2], rk);
    float h[3], l[3];
    split_pos(x, h, l);
    w.rec[2 * q] = make_float4(h[0], h[1], h[2], __int_as_float(tsrc));
    w.rec[2 * q + 1] = make_float4(l[0], l[1], l[2], (float)rk);
    w.hi[q] = make_float4(h[0], h[1], h[2], __int_as_float(tsrc));
}

// Sorted positions: threads [0, Nr) fill the real atoms' slots, the next ones the
// images'.  An image's FP64 position is its source's plus the lattice
// translation; its split is the source's split plus the translation's (grid
// parts add exactly), moved back to the nearest grid point (|lo| <= 2^-11) by
// whole grid steps.
__global__ void k_fill(Work w, const int32_t* __restrict__ types, const double* __restrict__ rk_tab) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < w.Nr) {
        const int i = w.sorted_src[p];
        int t = types[i];
        if (t < 0 || t >= w.T) t = 0;
        w.perm[p] = i;
        w.sid[p] = w.sid_in[i];
        w.cell_sorted[p] = w.cell_of[i];
        const double x[3] = {w.xw[3 * i], w.xw[3 * i + 1], w.xw[3 * i + 2]};
        store_pos(w, p, x, rk_tab[t], t | ((int)p << 4));
        return;
    }
    const int64_t q = p - w.Nr;
    const int ng = w.start_ghost[w.ncells];
    if (q >= ng) return;
    const int g = w.gsorted[q];
    const int i = w.ghost_src[g];
    int n0, n1, n2;
    unpack_shift(w.ghost_shift[g], n0, n1, n2);
    const StructGeo& G = w.geo[w.ghost_sid[g]];
    int t = types[i];
    if (t < 0 || t >= w.T) t = 0;
    const int ps = w.slot_of[i];  // the source's sorted slot (inverse permutation of the sort)
    const double rk = rk_tab[t];
    const double xs[3] = {w.xw[3 * i], w.xw[3 * i + 1], w.xw[3 * i + 2]};
    double x[3] = {xs[0], xs[1], xs[2]};
    add_lattice(x, G, n0, n1, n2);
    w.pos64[w.Nr + q] = dbl4_make(x[0], x[1], x[2], rk);
    float sh[3], sl[3];  // the source's split, as its own slot holds it
    split_pos(xs, sh, sl);
    const float f0 = (float)n0, f1 = (float)n1, f2 = (float)n2;
    float h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        h[a] = sh[a] + (f0 * G.Hh[a] + f1 * G.Hh[3 + a] + f2 * G.Hh[6 + a]);
        l[a] = sl[a] + (f0 * G.Hl[a] + f1 * G.Hl[3 + a] + f2 * G.Hl[6 + a]);
        const float m = rintf(l[a] * 1024.0f);
        h[a] += m * (1.0f / 1024.0f);
        l[a] -= m * (1.0f / 1024.0f);
    }
    const int tsrc = t | (ps << 4);
    w.rec[2 * (w.Nr + q)] = make_float4(h[0], h[1], h[2], __int_as_float(tsrc));
    w.rec[2 * (w.Nr + q) + 1] = make_float4(l[0], l[1], l[2], (float)rk);
    w.hi[w.Nr + q] = make_float4(h[0], h[1], h[2], __int_as_float(tsrc));
}

// ---- per-atom lists within the two list radii ------------------------------
// Positions used here are the grid-aligned hi parts (error <= sqrt(3) 2^-10
// bohr, covered by the list margin).  Both builders are persistent: each warp
// repeatedly takes the next piece of work from a global counter, which
// balances uneven structures across SMs.

// Shared per-atom state of a list builder lane.
struct ListLane {
    int64_t p;
    bool live;
    int s, c0, c1, c2;
    float4 hp;
    int* Ld;
    int* Lc;
    int* bd;  // 8 staged entries of each list (shared memory)
    int* bc;
    int capd, capc, nd, nc;
    __device__ void init(const Work& w, int64_t P, int* stage_d, int* stage_c) {
        bd = stage_d;
        bc = stage_c;
        p = P;
        live = P < w.Nr;
        s = live ? w.sid[P] : -1;
        c0 = c1 = c2 = 0;
        hp = make_float4(0.f, 0.f, 0.f, 0.f);
        Ld = Lc = nullptr;
        capd = capc = nd = nc = 0;
        if (!live) return;
        const StructGeo& G = w.geo[s];
        cell_coords(G, w.cell_sorted[P], c0, c1, c2);
        hp = rec_hi(w, P);
        const int64_t local = P - G.atom_base;
        Ld = w.nbr_disp + list_row(G.list_base_disp, local, G.cap_disp);
        Lc = w.nbr_cn + list_row(G.list_base_cn, local, G.cap_cn);
        capd = G.cap_disp;
        capc = G.cap_cn;
    }
    // stage q; the 8th entry of a group writes the group as two 16-byte stores
    // (capacities are multiples of 8, and groups of 4 entries are 16-byte aligned)
    __device__ __forceinline__ static void push(int* L, int cap, int& n, int* b, int q) {
        b[n & 7] = q;
        if ((n & 7) == 7 && n < cap) {
            *reinterpret_cast<int4*>(L + list_off(n - 7)) = *reinterpret_cast<const int4*>(b);
            *reinterpret_cast<int4*>(L + list_off(n - 3)) = *reinterpret_cast<const int4*>(b + 4);
        }
        ++n;
    }
    __device__ __forceinline__ static void drain(int* L, int cap, int n, const int* b) {
        const int base = n & ~7;
        for (int k = base; k < n; ++k)
            if (k < cap) L[list_off(k)] = b[k & 7];
    }
    __device__ __forceinline__ void add(int q, float r2, float rd2, float rn2) {
        if (r2 < rd2 && q != (int)p) {
            push(Ld, capd, nd, bd, q);
            if (r2 < rn2) push(Lc, capc, nc, bc, q);
        }
    }
    __device__ void finish(Work& w, int lane) {
        if (live) {
            drain(Ld, capd, nd, bd);
            w.cnt_disp[p] = min(nd, capd);
            drain(Lc, capc, nc, bc);
            w.cnt_cn[p] = min(nc, capc);
            if (nd > capd || nc > capc) atomicOr(w.status, ST_LIST_CAP);
        }
        // per-structure maxima (one atomic per group of lanes in the same structure)
        const unsigned grp = __match_any_sync(0xffffffffu, s);
        const int md = __reduce_max_sync(grp, nd), mc = __reduce_max_sync(grp, nc);
        if (live && lane == __ffs(grp) - 1) {
            atomicMax(&w.maxcnt[3 * s], md);
            atomicMax(&w.maxcnt[3 * s + 1], mc);
        }
    }
};

__device__ __forceinline__ int64_t next_chunk(const Work& w, int lane, int ctr) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(w.work_ctr + ctr, 1);
    return (int64_t)__shfl_sync(0xffffffffu, chunk, 0);
}

// Every thread walks the cell window of its own atom, rows of cells as
// contiguous index ranges, four candidates loaded per step.  Appends are
// staged in shared memory, 8 per list, and leave as whole 32-byte sectors.
__global__ void __launch_bounds__(128) k_build_lists(Work w) {
    if (skip_build(w)) return;
    const int lane = threadIdx.x & 31;
    const float rd2 = w.rl_disp2, rn2 = w.rl_cn2;
    const float4* __restrict__ H = w.hi;
    __shared__ __align__(16) int stage[2][128][8];
    for (;;) {
        const int64_t p0 = next_chunk(w, lane, 0) * 32;
        if (p0 >= w.Nr) return;
        ListLane L;
        L.init(w, p0 + lane, stage[0][threadIdx.x], stage[1][threadIdx.x]);
        if (L.live) {
            const StructGeo& G = w.geo[L.s];
            const int x0 = max(0, L.c0 - G.win[0]), x1 = min(G.ncell[0] - 1, L.c0 + G.win[0]);
            const int y0 = max(0, L.c1 - G.win[1]), y1 = min(G.ncell[1] - 1, L.c1 + G.win[1]);
            const int z0 = max(0, L.c2 - G.win[2]), z1 = min(G.ncell[2] - 1, L.c2 + G.win[2]);
            const float4 hp = L.hp;
            auto test = [&](int q, float4 hq) {
                const float dx = hq.x - hp.x, dy = hq.y - hp.y, dz = hq.z - hp.z;
                L.add(q, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), rd2, rn2);
            };
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y) {
                    int64_t cf, cl;
                    row_cells(G, y, z, x0, x1, cf, cl);
                    const int rb = __ldg(&w.start_real[cf]), re = __ldg(&w.start_real[cl + 1]);
                    const int gb = (int)w.Nr + __ldg(&w.start_ghost[cf]);
                    const int ge = (int)w.Nr + __ldg(&w.start_ghost[cl + 1]);
                    for (int pass = 0; pass < 2; ++pass) {
                        const int b = pass == 0 ? rb : gb, e = pass == 0 ? re : ge;
                        int u = b;
                        for (; u + 4 <= e; u += 4) {
                            const float4 h0 = __ldg(&H[u]), h1 = __ldg(&H[u + 1]);
                            const float4 h2 = __ldg(&H[u + 2]), h3 = __ldg(&H[u + 3]);
                            test(u, h0);
                            test(u + 1, h1);
                            test(u + 2, h2);
                            test(u + 3, h3);
                        }
                        for (; u < e; ++u) test(u, __ldg(&H[u]));
                    }
                }
        }
        L.finish(w, lane);
    }
}

// ---- cluster lists of the dispersion pass ---------------------------------
// Cluster I of structure s is the run of sorted real atoms
// [atom_base + 8 (I - clu_base), + 8) (fewer at the end of a structure).  Its
// list holds every atom q, real or image, whose hi position lies within the
// list radius of the cluster's bounding box and that the half rule assigns to
// I: each unordered pair instance of Eq. 2 must be listed exactly once.  With
// src the source real atom of q and n its lattice translation:
//   src in a later cluster                       listed (here, not there)
//   src in an earlier cluster                    not listed (listed there)
//   src in I, q real                             listed; the pass keeps only q > i
//   src in I, q an image                         listed when n > 0 (packed order):
//                                                (i, src, n) and (src, i, -n) are one instance
// The same walk writes the per-atom CN lists of the cluster's atoms (every
// atom within the CN list radius of each, both directions).
// One warp per cluster walks the union of its atoms' cell windows.  A row of
// cells whose real atoms all precede the cluster in sorted order holds no entry
// of its half list, so for it only the (smaller) window of the CN radius is
// walked.  The rows of cells (real and image atoms of each row: two index
// ranges per row) are flattened: 32 ranges at a time, their lengths scanned
// across the lanes and the non-empty ones compacted in shared memory, then 32
// candidates at a time, each lane finding its range by counting the range
// starts at or before its candidate (one OR-reduction of start bits, a popcount).  Candidates are appended in walk
// order (ballot compaction), so every list is deterministic.  Candidates within
// the CN list radius of the bounding box are first staged in shared memory, in
// walk order, and tested against the cluster's atoms 32 at a time.
__global__ void __launch_bounds__(128) k_build_clist(Work w) {
    if (skip_build(w)) return;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const float rd2 = w.rl_disp2, rn2 = w.rl_cn2;
    const float4* __restrict__ H = w.hi;
    const int zero_shift = pack_shift(0, 0, 0);
    __shared__ float4 sh_i[4][kClusterAtoms];  // the cluster's atoms (hi positions) per warp
    __shared__ float4 sh_ch[4][64];            // staged CN candidates per warp: position, index
    __shared__ int sh_cq[4][64];
    __shared__ int sh_rb[4][32], sh_re[4][32];  // the batch's non-empty ranges: first index (bit 31: images), start
    float4* hi8 = sh_i[threadIdx.x >> 5];
    int* rb = sh_rb[threadIdx.x >> 5];
    int* re = sh_re[threadIdx.x >> 5];
    float4* ch = sh_ch[threadIdx.x >> 5];
    int* cq = sh_cq[threadIdx.x >> 5];
    for (;;) {
        const int64_t I = next_chunk(w, lane, 1);
        if (I >= w.ncl) return;
        const int s = w.clu_sid[I];
        const StructGeo& G = w.geo[s];
        const int64_t p0 = G.atom_base + (I - G.clu_base) * kClusterAtoms;
        const int64_t rem = G.atom_base + G.natoms - p0;
        const int nI = rem < kClusterAtoms ? (int)rem : kClusterAtoms;
        // bounding box (hi positions) and cell range of the cluster's atoms
        const bool own = lane < nI;
        const float4 h = __ldg(&H[own ? p0 + lane : p0]);
        if (lane < kClusterAtoms) hi8[lane] = h;
        int cx, cy, cz;
        cell_coords(G, w.cell_sorted[own ? p0 + lane : p0], cx, cy, cz);
        float lo[3] = {h.x, h.y, h.z}, hi[3] = {h.x, h.y, h.z};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(full, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(full, hi[k], o));
            }
        __syncwarp();
        const int x0 = max(0, __reduce_min_sync(full, cx) - G.win[0]);
        const int x1 = min(G.ncell[0] - 1, __reduce_max_sync(full, cx) + G.win[0]);
        const int y0 = max(0, __reduce_min_sync(full, cy) - G.win[1]);
        const int y1 = min(G.ncell[1] - 1, __reduce_max_sync(full, cy) + G.win[1]);
        const int z0 = max(0, __reduce_min_sync(full, cz) - G.win[2]);
        const int z1 = min(G.ncell[2] - 1, __reduce_max_sync(full, cz) + G.win[2]);
        // the window of the CN list radius
        const int xc0 = max(0, __reduce_min_sync(full, cx) - G.win_cn[0]);
        const int xc1 = min(G.ncell[0] - 1, __reduce_max_sync(full, cx) + G.win_cn[0]);
        const int yc0 = max(0, __reduce_min_sync(full, cy) - G.win_cn[1]);
        const int yc1 = min(G.ncell[1] - 1, __reduce_max_sync(full, cy) + G.win_cn[1]);
        const int zc0 = max(0, __reduce_min_sync(full, cz) - G.win_cn[2]);
        const int zc1 = min(G.ncell[2] - 1, __reduce_max_sync(full, cz) + G.win_cn[2]);
        const int ny = y1 - y0 + 1, nranges = 2 * ny * (z1 - z0 + 1);
        int* row = w.nbr_cl + G.list_base_cl + (I - G.clu_base) * (int64_t)G.cap_cl;
        const int cap = G.cap_cl, capc = G.cap_cn;
        const int first = (int)p0, last = (int)p0 + nI;  // the cluster's own sorted slots
        int n = 0;
        int nc[kClusterAtoms] = {0, 0, 0, 0, 0, 0, 0, 0};  // CN list lengths (warp-uniform)
        int ns = 0;                                        // staged CN candidates (warp-uniform)
        // per-atom CN lists of the cluster's atoms from the first m staged candidates
        auto cn_round = [&](int m) {
            __syncwarp();
            const bool live = lane < m;
            const int q = live ? cq[lane] : -1;
            const float4 hq = ch[lane];
#pragma unroll
            for (int i = 0; i < kClusterAtoms; ++i) {
                if (i >= nI) break;
                const float4 hp = hi8[i];
                const float dx = hq.x - hp.x, dy = hq.y - hp.y, dz = hq.z - hp.z;
                const bool in = live && q != first + i && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rn2;
                const unsigned mi = __ballot_sync(full, in);
                const int kc = nc[i] + __popc(mi & ((1u << lane) - 1u));
                if (in && kc < capc)
                    w.nbr_cn[list_row(G.list_base_cn, (int64_t)first + i - G.atom_base, capc) + list_off(kc)] = q;
                nc[i] += __popc(mi);
            }
            // move the rest (fewer than 32) to the front
            const int rest = ns - m;
            float4 h2 = make_float4(0.f, 0.f, 0.f, 0.f);
            int q2 = 0;
            if (lane < rest) {
                h2 = ch[m + lane];
                q2 = cq[m + lane];
            }
            __syncwarp();
            if (lane < rest) {
                ch[lane] = h2;
                cq[lane] = q2;
            }
            ns = rest;
            __syncwarp();
        };
        for (int r0 = 0; r0 < nranges; r0 += 32) {
            // this lane's range: row (y, z) = (r / 2) and real (r even) or image atoms
            int b = 0, len = 0;
            const int r = r0 + lane;
            if (r < nranges) {
                const int rr = r >> 1;
                const int y = y0 + rr % ny, z = z0 + rr / ny;
                int64_t cf, cl;
                row_cells(G, y, z, x0, x1, cf, cl);
                if ((r & 1) == 0) {
                    b = __ldg(&w.start_real[cf]);
                    len = __ldg(&w.start_real[cl + 1]) - b;
                    if (b + len <= (int)p0) {  // the whole row precedes the cluster: CN candidates only
                        if (y < yc0 || y > yc1 || z < zc0 || z > zc1) {
                            len = 0;
                        } else {
                            row_cells(G, y, z, xc0, xc1, cf, cl);
                            b = __ldg(&w.start_real[cf]);
                            len = __ldg(&w.start_real[cl + 1]) - b;
                        }
                    }
                } else {
                    b = (int)w.Nr + __ldg(&w.start_ghost[cf]);
                    len = (int)w.Nr + __ldg(&w.start_ghost[cl + 1]) - b;
                }
            }
            int incl = len;  // inclusive scan of the lengths over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - len;
            const int total = __shfl_sync(full, incl, 31);
            // the non-empty ranges in order, in shared memory (their starts are distinct)
            const unsigned ne = __ballot_sync(full, len > 0);
            __syncwarp();
            if (len > 0) {
                const int k = __popc(ne & ((1u << lane) - 1u));
                rb[k] = (int)((unsigned)b | ((unsigned)(r & 1) << 31));
                re[k] = excl;
            }
            __syncwarp();
            int c0 = 0;  // non-empty ranges that start before f0
            for (int f0 = 0; f0 < total; f0 += 32) {
                const int f = f0 + lane;
                // the range holding flat candidate f: the last non-empty range starting at or
                // before f, counted from one bit per range start in [f0, f0 + 32)
                const int d = excl - f0;
                const unsigned M = __reduce_or_sync(full, (len > 0 && d >= 0 && d < 32) ? (1u << d) : 0u);
                const int k = c0 + __popc(M & (0xffffffffu >> (31 - lane))) - 1;
                c0 += __popc(M);
                const int kr = f < total ? k : 0;
                const int rbk = rb[kr];
                const int q = (rbk & 0x7fffffff) + (f - re[kr]);
                const bool img = rbk < 0;
                bool take = false, cn_cand = false;
                float4 hq = make_float4(0.f, 0.f, 0.f, 0.f);
                if (f < total) {
                    hq = __ldg(&H[q]);
                    const float gx = fmaxf(0.0f, fmaxf(lo[0] - hq.x, hq.x - hi[0]));
                    const float gy = fmaxf(0.0f, fmaxf(lo[1] - hq.y, hq.y - hi[1]));
                    const float gz = fmaxf(0.0f, fmaxf(lo[2] - hq.z, hq.z - hi[2]));
                    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
                    cn_cand = g2 < rn2;
                    if (g2 < rd2) {
                        const int src = __float_as_int(hq.w) >> 4;
                        if (src >= last) {
                            take = true;
                        } else if (src >= first) {
                            take = !img || w.ghost_shift[w.gsorted[q - (int)w.Nr]] > zero_shift;
                        }
                    }
                }
                const unsigned m = __ballot_sync(full, take);
                const int kk = n + __popc(m & ((1u << lane) - 1u));
                if (take && kk < cap) row[kk] = q;
                n += __popc(m);
                // stage the CN candidates in walk order
                const unsigned mcn = __ballot_sync(full, cn_cand);
                if (cn_cand) {
                    const int kk2 = ns + __popc(mcn & ((1u << lane) - 1u));
                    ch[kk2] = hq;
                    cq[kk2] = q;
                }
                ns += __popc(mcn);
                if (ns >= 32) cn_round(32);
            }
        }
        if (ns > 0) cn_round(ns);
        int mc = 0;
#pragma unroll
        for (int i = 0; i < kClusterAtoms; ++i)
            if (i < nI) {
                mc = max(mc, nc[i]);
                if (lane == i) w.cnt_cn[first + i] = min(nc[i], capc);
            }
        if (lane == 0) {
            w.cnt_cl[I] = min(n, cap);
            if (n > cap || mc > capc) atomicOr(w.status, ST_LIST_CAP);
            atomicMax(&w.maxcnt[3 * s + 2], n);
            atomicMax(&w.maxcnt[3 * s + 1], mc);
        }
        __syncwarp();
    }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t scan2(const ScanPair& sp, int* bsum, int64_t n, const int* gate, cudaStream_t st) {
    const int nb = (int)nblk(n, kScanBlock);
    k_scan_blocks<<<dim3(nb, 2), kScanBlock, 0, st>>>(sp, bsum, nb, n, gate);
    k_scan_sums<<<2, kScanBlock, 0, st>>>(sp, bsum, nb, n, gate);
    k_scan_add<<<dim3(nb, 2), kScanBlock, 0, st>>>(sp, bsum, nb, n, gate);
    return cudaGetLastError();
}

}  // namespace

// The cell-list build: counters, binning, images, sort, fill, lists.  With
// w.gate set, every step but the fill runs only when *w.gate != 0 (list
// reuse); the fill always rewrites the sorted positions from w.xw.
// bsum must hold nblk(ncells, 1024) ints; rk_tab holds k2*Rcov per type (bohr);
// lmarks (optional): two events recorded around the list-builder kernel.
cudaError_t launch_build_impl(const Work& w, const double* pos, const int32_t* types, const double* rk_tab,
                              int* bsum, cudaStream_t st, cudaEvent_t* lmarks) {
    if (w.Nr == 0) return cudaGetLastError();
    const int TB = 256;
    const int64_t nreset = std::max<int64_t>(w.ncells + 1, 3 * (int64_t)w.B);
    k_reset<<<nblk(nreset, TB), TB, 0, st>>>(w);
    k_wrap<<<nblk(w.Nr, TB), TB, 0, st>>>(w, pos, types);
    k_images<<<nblk(w.Nr, TB), TB, 0, st>>>(w);
    const ScanPair sp{{w.cnt_real, w.cnt_ghost}, {w.start_real, w.start_ghost}};
    const cudaError_t e = scan2(sp, bsum, w.ncells, w.gate, st);
    if (e != cudaSuccess) return e;
    k_scatter<<<nblk(w.Nr + w.ghost_cap, TB), TB, 0, st>>>(w);
    k_rank<<<nblk(w.Nr + w.ghost_cap, TB), TB, 0, st>>>(w);
    k_fill<<<nblk(w.Nr + w.ghost_cap, TB), TB, 0, st>>>(w, types, rk_tab);
    {
        // persistent warps: w.build_per_sm blocks per SM, work handed out per 32 atoms
        // (per-atom lists) and per cluster (cluster lists)
        const int chunks = (int)((w.Nr + 31) / 32);
        const int blocks = std::min((chunks + 3) / 4, w.num_sms * w.build_per_sm);
        if (lmarks) cudaEventRecord(lmarks[0], st);
        if (w.cl_mode) {  // cluster lists and, in the same walk, the per-atom CN lists
            const int bcl = (int)std::min<int64_t>((w.ncl + 3) / 4, (int64_t)w.num_sms * w.build_per_sm);
            if (w.ncl > 0) k_build_clist<<<bcl, 128, 0, st>>>(w);
        } else {
            k_build_lists<<<blocks, 128, 0, st>>>(w);
        }
        if (lmarks) cudaEventRecord(lmarks[1], st);
    }
    return cudaGetLastError();
}

int64_t scan_scratch_ints(int64_t ncells) { return 2 * nblk(ncells, kScanBlock) + 2; }

cudaError_t launch_check(const Work& w, const double* pos, cudaStream_t st) {
    if (w.Nr == 0) return cudaGetLastError();
    k_check<<<nblk(w.Nr, 256), 256, 0, st>>>(w, pos);
    return cudaGetLastError();
}

}  // namespace d3gb
