/*
 * d3gb.h -- C ABI of the GB300 D3(BJ) dispersion library.
 *
 * The library evaluates the environment-dependent D3 dispersion correction with
 * Becke-Johnson damping as used in NEP-D3 (Ying & Fan, arXiv 2310.05279,
 * Sec. II A): the total energy of Eq. 1 as a sum of the site energies of Eq. 2,
 * the C6 interpolation of Eq. 3 over the coordination numbers of Eq. 4, the
 * forces of Eqs. 5-6 (evaluated as F = -dE/dx including the dependence on
 * neighbours' coordination numbers) and the total of the per-atom virials of
 * Eq. 7.  The three-body term is excluded by default, as in the paper;
 * d3_set_three_body adds it as an option.
 *
 * Conventions shared by every entry point
 *  - Units: positions and cells in Angstrom; a2, covalent radii and sqrt(Q) in
 *    bohr; C6 references in Hartree*bohr^6.  Outputs: E in eV, F in eV/A,
 *    W in eV.  Internally everything is evaluated in bohr/Hartree
 *    (1 bohr = 0.529177210903 A, 1 Ha = 27.211386245988 eV).
 *  - Cell matrices are row-major 3x3 with rows = lattice vectors.  pbc[k] = 0
 *    means no periodic images along lattice vector k.
 *  - Batches are concatenated: structure s owns atoms [offsets[s], offsets[s+1]).
 *  - Pointer spaces are stated per argument: "device" pointers must be CUDA
 *    device (or managed) memory on the current device; "host" pointers are
 *    ordinary host memory.  The caller owns every input and output buffer; the
 *    library owns the handle, its tables, neighbour lists and workspace.
 *  - Work is enqueued on the caller's stream (a cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Unless stated otherwise a call does not
 *    synchronise.  The first call for a new batch geometry (offsets, cells,
 *    pbc) sizes the workspace and synchronises once (and, for the first
 *    geometry of a size class, measures the launch shapes: d3_set_autotune);
 *    later calls with the same
 *    geometry allocate nothing and do not synchronise, so they can be captured
 *    in a CUDA graph.
 *  - Errors: every call returns a d3_status.  Device-side problems (capacity
 *    overflow, non-finite coordinates, bad types, coordinates out of range) are
 *    recorded in a status word that d3_sync_status() reads.  The library never
 *    aborts or traps.
 *  - Coordinate range: after wrapping into its cell (periodic axes) every
 *    position must satisfy |x| < 4200 A (8000 bohr; the FP32 split of positions
 *    on a 2^-10 bohr grid is exact below 2^13 bohr).  A cell that reaches
 *    beyond it is rejected with D3_ERR_ARG at the call; a position beyond it is
 *    reported as D3_ERR_ARG by d3_sync_status().
 *  - Thread safety: one handle must not be used from two host threads at once.
 */
#ifndef D3GB_H
#define D3GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum d3_status {
    D3_OK = 0,
    D3_ERR_ARG = 1,       /* invalid argument: NULL pointer, negative size, degenerate cell, bad table */
    D3_ERR_CUDA = 2,      /* a CUDA runtime call failed (message in d3_last_error) */
    D3_ERR_CAPACITY = 3,  /* a neighbour or image buffer overflowed; it has been regrown, repeat the call */
    D3_ERR_NONFINITE = 4, /* a coordinate was NaN or infinite */
    D3_ERR_TIMEOUT = 5,   /* reserved: no entry point returns it (the library has no device-side waits) */
    D3_ERR_TYPE = 6,      /* an atom type outside [0, ntypes) */
    D3_ERR_STATE = 7      /* call out of sequence */
} d3_status;

/* precision of the pair arithmetic */
enum { D3_FP64 = 0, D3_MIXED = 1 };

/* Functional parameters of Eq. 2 (s6, s8, a1, a2), the constants of Eqs. 3-4
 * (k1 = 16, k2 = 4/3 scales the tabulated covalent radii, k3 = 4), and the two
 * cutoffs R_pot and R_cn of the paper (12 A and 6 A by default).  skin_A is
 * added to both list radii.  With skin_A = 0 every compute call rebuilds the
 * lists.  With skin_A > 0 a compute call first checks on the device whether
 * any atom moved more than skin_A/2 since the last build; only then does the
 * build run, otherwise the lists (and the periodic images) are reused and only
 * the positions are refreshed.  No host synchronisation is involved either way.
 * precision: D3_MIXED evaluates distances, damping, the C6 interpolation and
 * the coordination-number terms in FP32 with FP64 accumulation of energies,
 * virials and dE/dn; D3_FP64 evaluates everything in FP64. */
typedef struct d3_params {
    double s6, s8, a1, a2_bohr;
    double k1, k2, k3;
    double rc_disp_A, rc_cn_A, skin_A;
    int32_t precision;
} d3_params;

/* Reference data (Eq. 3 and Eq. 4), host memory, copied by d3_create.
 *  nref[t]                      references of element t (1..max_ref)
 *  cn_ref[t*max_ref + a]        reference coordination numbers
 *  c6_ref[((ti*ntypes + tj)*max_ref + a)*max_ref + b]
 *                               C6 reference grid (Ha*bohr^6); must satisfy
 *                               c6_ref[ti,tj,a,b] == c6_ref[tj,ti,b,a]
 *  rcov_bohr[t]                 tabulated covalent radius (Eq. 4 uses k2*rcov)
 *  sqrtq[t]                     sqrt(Q); R0^2 = 3 sqrtq_i sqrtq_j, C8 = C6 R0^2
 * Limits: 1 <= ntypes <= 16, 1 <= max_ref <= 7. */
typedef struct d3_tables {
    int32_t ntypes, max_ref;
    const int32_t *nref;
    const double *cn_ref;
    const double *c6_ref;
    const double *rcov_bohr;
    const double *sqrtq;
} d3_tables;

typedef struct d3_handle d3_handle;

/* Create a handle: validates and copies params and tables (host pointers) to
 * the current CUDA device.  *out receives the handle; NULL on failure. */
d3_status d3_create(const d3_params *params, const d3_tables *tables, d3_handle **out);

/* Free every resource of the handle (synchronises the device first). NULL is a no-op. */
void d3_destroy(d3_handle *h);

/* Replace the four damping parameters of Eq. 2 (s6, s8, a1, a2 in bohr).
 * Takes effect for work enqueued afterwards on the handle's last stream. */
d3_status d3_set_damping(d3_handle *h, double s6, double s8, double a1, double a2_bohr);

/* Graph replay (default on): after the first call for a geometry, a compute
 * call whose pointers and parameters match the previous one is replayed as one
 * CUDA graph (captured once on an internal stream, launched on the caller's
 * stream), which removes the per-kernel launch overhead.  Calls made while
 * profiling (d3_profile_enable) or while the caller's stream is being captured
 * enqueue their kernels directly.  on = 0 always enqueues directly.  Results
 * are identical either way. */
d3_status d3_set_graphs(d3_handle *h, int32_t on);

/* Accumulate mode for the NEP-D3 sum of Eq. 9 (U = U_NEP + U_D3, Sec. II A):
 * with on != 0, the compute calls ADD their E, F and W into the caller's
 * output arrays (which then hold, e.g., the short-range model's values)
 * instead of overwriting them.  Site energies, CNs and per-atom virials are
 * always overwritten.  Default off.  Applies to work enqueued afterwards. */
d3_status d3_set_accumulate(d3_handle *h, int32_t on);

/* Launch shapes of the hot kernels, as int32_t shapes[4]: threads per block
 * of the CN pass (Eq. 4 with the Eq. 3 weights), of the dispersion pass
 * (Eq. 2) and of the CN chain-rule pass (64 or 128 each), and blocks per SM of
 * the persistent neighbour-list builder (8 or 16).  Every choice gives
 * bit-identical results; only the time differs.
 *
 * Autotuning (default on): when a new geometry of at least 16384 atoms is
 * sized, the library runs the build and the passes three times with each
 * candidate, timed with CUDA events on the call's stream, and keeps per kernel
 * the faster shape (the default unless the other is more than 1% faster).  The
 * choice is cached per size class (precision, three-body term on or off, and
 * the binary orders of magnitude of the atom count and of the mean structure
 * size), so later geometries of the same class reuse it.  Smaller geometries
 * use the defaults {64, 128, 128, 16}.  The measurement runs write only the
 * library's workspace, leave the build count unchanged and count as launches.
 *
 * d3_set_autotune: on = 0 keeps the current shapes for later geometries.
 * d3_launch_shapes: the shapes used for work enqueued next (host int32_t[4],
 * may be NULL) and the number of measurements made so far (host, may be NULL).
 * d3_set_launch_shapes: fix the shapes (host int32_t[4]) and turn autotuning
 * off; D3_ERR_ARG if a value is not one of the candidates, and then nothing
 * changes.  Applies to work enqueued afterwards. */
d3_status d3_set_autotune(d3_handle *h, int32_t on);
d3_status d3_launch_shapes(d3_handle *h, int32_t *shapes, int64_t *tunings);
d3_status d3_set_launch_shapes(d3_handle *h, const int32_t *shapes);

/* Optional three-body term (off by default).  The paper's model is two-body:
 * Sec. II A leaves out the triple-dipole term of the original D3 model, and so
 * does every other entry point unless this one enables it.  With s9 != 0 the
 * compute calls add, for every triangle (i, j, k) whose three sides are below
 * rc3,
 *   E_ijk = s9 sqrt(C6_ij C6_ik C6_jk) (3 cos A_i cos A_j cos A_k + 1)
 *           / (r_ij r_ik r_jk)^3 / (1 + 6 (Rbar / rbar)^alpha9),
 * A_v the interior angles, rbar = (r_ij r_ik r_jk)^(1/3) and Rbar the geometric
 * mean of the three damping radii a1 R0 + a2 of Eq. 2 (bohr), with the
 * C6 of Eq. 3 (so the term also acts through the coordination numbers), to E,
 * F, W and the site energies (a third of E_ijk to each vertex).
 *  s9      strength (0 turns the term off; 1 is the usual D3 value)
 *  alpha9  damping exponent, 0 < alpha9 <= 64 (16 in the original model)
 *  rc3_A   cutoff on every side, 0 < rc3_A <= rc_cn_A, A (the triangles are
 *          taken from the CN neighbour lists)
 * With the term on, d3_compute_batch_atoms and d3_backward return D3_ERR_ARG
 * (per-atom virials and the gradients are those of the two-body model).
 * Synchronises with the handle's last stream; applies to work enqueued afterwards. */
d3_status d3_set_three_body(d3_handle *h, double s9, double alpha9, double rc3_A);

/* Build (or rebuild) the neighbour lists of a batch and size the workspace
 * for it; synchronises.  The cell-list build: wrap into the cell, periodic
 * image atoms within the list radius, counting sort by cell, and per-atom
 * lists within R_pot and R_cn (Eqs. 2 and 4 sum over neighbours within these
 * cutoffs).
 *  B        number of structures (>= 0)
 *  offsets  host int64[B+1], offsets[0] = 0, non-decreasing
 *  pos      device double[N][3], A        types  device int32[N]
 *  cells    host double[B][9], A          pbc    host int32[B][3]  */
d3_status d3_build_neighbors(d3_handle *h, int32_t B, const int64_t *offsets, const double *pos,
                             const int32_t *types, const double *cells, const int32_t *pbc, void *stream);

/* One structure of n atoms: energy E (device double[1], eV), forces F (device
 * double[n][3], eV/A) and virial W (device double[9], eV, symmetric,
 * W = -dE/d(strain) = sum over atoms of Eq. 7).  cell: host double[9];
 * pbc: host int32[3].  Equivalent to d3_compute_batch with B = 1. */
d3_status d3_compute(d3_handle *h, const double *pos, const int32_t *types, int64_t n, const double *cell,
                     const int32_t *pbc, double *E, double *F, double *W, void *stream);

/* A batch of B independent structures in one pass: E device double[B],
 * F device double[N][3] in input order, W device double[B][9]. */
d3_status d3_compute_batch(d3_handle *h, int32_t B, const int64_t *offsets, const double *pos,
                           const int32_t *types, const double *cells, const int32_t *pbc, double *E, double *F,
                           double *W, void *stream);

/* As d3_compute_batch, plus optional per-atom outputs (device, input order;
 * NULL to skip): e_atom double[N] site energies U_i of Eq. 2 in eV, cn
 * double[N] coordination numbers of Eq. 4. */
d3_status d3_compute_batch_ex(d3_handle *h, int32_t B, const int64_t *offsets, const double *pos,
                              const int32_t *types, const double *cells, const int32_t *pbc, double *E,
                              double *F, double *W, double *e_atom, double *cn, void *stream);

/* As d3_compute_batch_ex, plus the per-atom virial of Eq. 7 (Sec. II A):
 * w_atom device double[N][9], eV, input order, row-major 3x3 per atom,
 *     W_i[a][b] = sum_{j != i} (r_ij)_a (dU_j/dr_ji)_b,   r_ij = x_j - x_i,
 * with each site energy U_j of Eq. 2 written as a function of the vectors
 * from atom j.  Through the coordination numbers U_j depends on r_ji directly
 * (n_j), through n_i, and through the CNs of j's other partners; all three
 * are included, so W_i is in general not symmetric, and sum_i W_i equals W.
 * Requires w_atom != NULL when N > 0 (e_atom and cn may be NULL). */
d3_status d3_compute_batch_atoms(d3_handle *h, int32_t B, const int64_t *offsets, const double *pos,
                                 const int32_t *types, const double *cells, const int32_t *pbc, double *E,
                                 double *F, double *W, double *e_atom, double *cn, double *w_atom,
                                 void *stream);

/* Per-atom heat current of Eq. 8, J_i = W_i . v_i, for n atoms (no handle):
 * w_atom device double[n][9] as written by d3_compute_batch_atoms, vel device
 * double[n][3] (any velocity unit), J device double[n][3] (eV times that unit).
 * Enqueued on stream; D3_ERR_ARG on a negative n or NULL arrays. */
d3_status d3_heat_current(int64_t n, const double *w_atom, const double *vel, double *J, void *stream);

/* As d3_compute_batch with every array in HOST memory (page-locked memory
 * gives full copy speed): copies inputs to the device, computes, copies E, F,
 * W back and synchronises the stream before returning. */
d3_status d3_compute_batch_host(d3_handle *h, int32_t B, const int64_t *offsets, const double *pos,
                                const int32_t *types, const double *cells, const int32_t *pbc, double *E,
                                double *F, double *W, void *stream);

/* Hand-written backward of (E, F) for refitting the damping parameters.
 * Given upstream gradients dL/dE (device double[B], per eV) and dL/dF
 * (device double[N][3], per eV/A) it returns
 *   dLdparams  device double[4] = dL/d(s6, s8, a1, a2[bohr])
 *   dLdpos     device double[N][3] = dL/dx (per A), input order
 * The force term needs the Hessian-vector product H*(dL/dF); it is formed by
 * forward-mode differentiation of the whole force evaluation along dL/dF
 * (coordination numbers recomputed, no per-pair storage).  A D3_FP64 handle
 * differentiates in FP64 dual numbers; a D3_MIXED handle forms the values with
 * the mixed forward's arithmetic (double-single Eq. 4 terms, float-float Eq. 3
 * exponents, FP32 pair math on split positions, compensated sums) and the
 * tangents in FP32, several times faster with the mixed forward's relative
 * precision.  Either output may be NULL.  Inputs as in d3_compute_batch. */
d3_status d3_backward(d3_handle *h, int32_t B, const int64_t *offsets, const double *pos, const int32_t *types,
                      const double *cells, const int32_t *pbc, const double *dLdE, const double *dLdF,
                      double *dLdparams, double *dLdpos, void *stream);

/* Synchronise the handle's last stream and report the first recorded
 * device-side problem (then clear it). */
d3_status d3_sync_status(d3_handle *h);

/* Number of neighbour builds the handle has executed on the device, sizing
 * passes included (with skin_A > 0 this shows how often the lists were
 * rebuilt).  *builds is host memory.  Synchronises the handle's last stream.
 * The paper has no counterpart; this is a diagnostic of the list reuse. */
d3_status d3_build_count(d3_handle *h, int64_t *builds);

/* Human-readable description of the last error on this handle ("" if none). */
const char *d3_last_error(const d3_handle *h);

/* Stage timing for benchmarks and profiling.  While enabled, every later
 * compute call brackets its stages with CUDA events on the call's stream:
 * 0 neighbour build, 1 coordination numbers (Eq. 4), 2 reference weights
 * (Eq. 3), 3 dispersion pass (Eq. 2), 4 three-body term (d3_set_three_body),
 * 5 coordination-number chain rule, 6 per-structure sums.  Events are cheap
 * stream markers; they add no synchronisation.  The library also counts every
 * kernel it launches. */
d3_status d3_profile_enable(d3_handle *h, int32_t on);

/* Synchronise on the recorded events and return totals since the last reset:
 * ms[7] milliseconds per stage and calls[7] calls timed per stage (either may
 * be NULL); *launches = kernels launched by the library (may be NULL).  Stages:
 * neighbour build, CN (Eq. 4, with the Eq. 3 weights), weights (empty: formed
 * in the CN pass), dispersion (Eq. 2), three-body (empty unless enabled),
 * CN chain rule, per-structure sums. */
d3_status d3_profile_read(d3_handle *h, double *ms, int64_t *calls, int64_t *launches);

/* Zero the stage totals and the launch counter. */
d3_status d3_profile_reset(d3_handle *h);

/* Totals of one profiled stage since the last reset: stage 0..6 as in
 * d3_profile_read, stage 7 the list-builder kernel alone (inside stage 0).
 * ms and calls may be NULL.  D3_ERR_ARG for another stage number. */
d3_status d3_profile_stage(d3_handle *h, int32_t stage, double *ms, int64_t *calls);

/* Sizes of the current plan's neighbour data, for measurement (synchronises):
 * stats[0] real atoms, [1] image atoms, [2] clusters of the cluster lists,
 * [3] cluster-list entries (last build in cluster mode, else 0), [4] CN-list
 * entries, [5] per-atom dispersion-list entries (last build with full lists,
 * else 0), [6] unique pair instances within R_pot evaluated by the last
 * cluster-mode dispersion pass (Eq. 2), [7] list mode of the last build
 * (1 = cluster lists, 0 = full per-atom lists, -1 = none).  host int64_t[8]. */
d3_status d3_list_stats(d3_handle *h, int64_t *stats);

/* The autotuner's last measurement, host float[8] in ms: list build, CN pass,
 * dispersion pass and chain pass, each with the 64- and 128-thread (or 8 and
 * 16 blocks per SM) candidate.  Zeros before the first measurement. */
d3_status d3_tune_times(d3_handle *h, float *ms);

/* Measured arithmetic rates of the current device, the denominators of the
 * rooflines of the pair passes: rates[0] FP32 FMA lane operations per second,
 * rates[1] FP64 FMA lane operations per second, rates[2] MUFU reciprocals per
 * second (host double[3]).  Runs three short microbenchmark kernels on
 * `stream` and synchronises; allocates a small scratch buffer.  A measurement
 * helper: the paper has no counterpart. */
d3_status d3_peak_rates(double *rates, void *stream);

/* Per-structure energies from site energies, for callers that cannot allocate
 * device memory: a host program that keeps all device memory in its own pool
 * and hands libraries only the buffers it owns, or a loop that cannot take the
 * implicit device synchronisation a cudaMalloc may cause.  The paper has no
 * counterpart: this is a service entry point.
 *  B        number of structures, 0 <= B <= 16384
 *  offsets  host int64[B+1], offsets[0] = 0, non-decreasing
 *  e_atom   device double[offsets[B]] site energies (e.g. from d3_compute_batch_ex), eV
 *  E        device double[B] receives the per-structure sums, eV
 * Allocates nothing: its scratch is a fixed array of about 0.7 MB inside the
 * library that every device which loads the library holds until the process
 * exits.  Limit: B times ceil(largest structure / 4096) must not exceed 65536;
 * beyond that (or B > 16384) it returns D3_ERR_CAPACITY before enqueueing
 * anything.  The first call on a device looks up the array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  The address is kept for the life of the process, so
 * calls after cudaDeviceReset are not supported.  All calls share the array,
 * so calls that overlap on the GPU race; calls ordered on one stream are
 * safe.  Enqueued on `stream` (offsets is copied to the device by an
 * asynchronous copy on that stream: keep it valid and unchanged until the
 * stream has reached this call), no handle needed. */
d3_status d3_structure_energies_noalloc(int32_t B, const int64_t *offsets, const double *e_atom, double *E,
                                        void *stream);

/* Library version string. */
const char *d3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* D3GB_H */
