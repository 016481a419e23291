/*
 * ygs.h -- C ABI of libygs, a GB300 (sm_103a) solver for the gravitational
 * potential on multi-patch spherical grids by a single global spherical-
 * harmonics expansion (Wongwathanarat, arXiv:1903.08475).
 *
 * The operation (Sect. 3-4 of the paper):
 *
 *   Phi(r) = -G \int rho(r') / |r - r'| d^3r'                 (Eq. integralpoisson)
 *
 * on a grid of N_g rotated spherical-coordinate patches sharing one set of
 * radial shells.  With cell-constant density rho and overlap weight w, and the
 * expansion truncated at l_max, every solve runs the paper's steps 2-5:
 *
 *   B[i,c]   = sum_{g,j,k} rho_{g,i,j,k} U_{g,jk,c}            (Eq. B_CS)
 *   M[i,c]   = (r_i^+)^-(l+1) sum_{i'<=i} R_in,i' B[i',c]
 *            + (r_i^+)^l      sum_{i'>i}  R_out,i' B[i',c]     (Eq. M_C)
 *   Phi_{g,i,jk} = sum_c Q_{g,jk,c} M[i,c]                     (Eq. gravpotmult)
 *
 * with the angular weights U (Eqs. U_C/U_S: the global-frame real harmonic
 * of column c integrated over the patch cell through the Wigner-D rotation of
 * Eqs. ylm_transform/wigner-D, times w and 2/delta_m) and the prefactors Q
 * (Eqs. Q_C/Q_S: -G times the global-frame real harmonic at the evaluation
 * point), both built once per grid by ygs_create (step 1).
 *
 * Conventions
 *   - Real columns c = (l, m, C|S), m >= 0:  (l,0,C) -> l*l,
 *     (l,m,C) -> l*l + 2m - 1, (l,m,S) -> l*l + 2m;  K = (l_max+1)^2.
 *     Y^C_lm = N_lm P_l^m(cos t) cos(m p), Y^S_lm = N_lm P_l^m(cos t) sin(m p),
 *     N_lm = sqrt((l-m)!/(l+m)!), P_l^m without the Condon-Shortley phase.
 *   - Patch g maps local Cartesian coordinates xi to global ones by
 *     x = R^(g) xi, R^(g) the z-y'-z'' Euler matrix of Eq. rottransmatrix.
 *   - Cell (g, i, j, k): r in [edges[i], edges[i+1]],
 *     theta in theta_lo + [j, j+1] * dtheta, phi in phi_lo + [k, k+1] * dphi
 *     (local coordinates, dtheta = (theta_hi - theta_lo)/n_theta, same for phi).
 *   - Fields (rho, Phi and their gradients) are FP64 arrays laid out
 *     [g][i][j][k] (patch-major, then shell, then theta, phi fastest), patches
 *     concatenated in order: patch g starts at element n_r * sum_{g'<g} n_theta[g'] n_phi[g'].
 *   - Phi_{g,i,j,k} is the potential at radius edges[i+1] and at the upper
 *     angular vertex (theta_j^+, phi_k^+) of the cell (YGS_EVAL_UPPER_VERTEX,
 *     the paper's choice, Sect. 4.2) or at the cell's angular centre.
 *
 * Ownership and threading
 *   - A plan owns all device memory it allocates (weights, workspaces) from
 *     ygs_create to ygs_destroy.  Field buffers are owned by the caller.
 *   - Device pointers must be allocated on the plan's device and be 16-byte
 *     aligned.  A plan must not be used by two host threads at once, and two
 *     calls on one plan must not overlap on the GPU (they share workspaces):
 *     issue them on one stream or order the streams.
 *   - ygs_solve / ygs_solve_batched / ygs_backward only enqueue work on the
 *     given stream (NULL = the legacy default stream); they do not synchronise.
 *
 * Errors
 *   Every entry point returns a ygs_status and never aborts the process.
 *   Arguments are validated before any work is enqueued; a failing CUDA call
 *   returns YGS_ERR_CUDA.  ygs_last_error() gives a message for the most recent
 *   failure on the calling thread.
 */
#ifndef YGS_H
#define YGS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  YGS_OK = 0,
  YGS_ERR_INVALID_ARG = 1, /* bad descriptor, size, pointer or alignment */
  YGS_ERR_OOM = 2,         /* device allocation failed */
  YGS_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
  YGS_ERR_UNSUPPORTED = 4, /* valid request this build does not implement */
  YGS_ERR_NUMERIC = 5,     /* a weight self-check failed, or (YGS_FP64_EMU) a field value at
                              or above 2^127, beyond what the FP32 window sums can hold */
  YGS_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  YGS_ERR_BOUNDS = 7       /* checked builds only (ygs_checked_build): a kernel met a global index
                              outside the buffer it addresses and skipped the access */
} ygs_status;

/* Arithmetic of the two contractions (projection and synthesis).  Weight
 * building and the radial scans are FP64 in every mode. */
typedef enum {
  YGS_FP64 = 0,   /* FP64 FMA on the CUDA cores */
  YGS_BF16X3 = 1, /* tcgen05 BF16 tensor cores, 2-slice operands, 3 products */
  YGS_BF16X6 = 2, /* tcgen05 BF16 tensor cores, 3-slice operands, 6 products */
  YGS_FP16X3 = 3, /* tcgen05 FP16 tensor cores, 2-slice operands (22 significant bits), 3 products;
                     every operand row is scaled by a power of two into FP16's range (U per
                     column, the field per shell and group of 128 angular cells, M per
                     shell, Q as a whole) and unscaled exactly */
  YGS_FP64_TC = 4, /* the FP64 path with its contractions on the FP64 tensor cores (DMMA 8x8x4):
                     FP64 products and sums, another order of additions */
  YGS_FP32 = 5,    /* FP32 contractions on the CUDA cores (FP32 copies of U and Q, the field
                     truncated to FP32, FP32 accumulation), FP64 radial scans; the adjoint of
                     such a plan runs on its FP64 weights */
  YGS_TF32X3 = 6,  /* tcgen05 TF32 tensor cores (kind::tf32), 2-slice operands (each value split
                     into two TF32 values, 22 significant bits), 3 products; FP32's exponent range,
                     so no row scaling; twice the operand bytes and half the tensor rate of FP16x3.
                     Phi within 1e-6 of FP64 (as FP16x3); its adjoint within 2e-6 of the
                     largest |A^T w| (1.4e-6 measured at l_max = 32) */
  YGS_FP64_EMU = 7 /* FP64-accurate contractions on the BF16 tensor cores (Ozaki-type splitting):
                     every FP64 value cut exactly into six 8-bit slices on a fixed grid (per
                     weight row; per shell and window of 256 cells for the field; per shell
                     for M), the 21 slice products with s + t <= 5 each summed exactly in FP32
                     over windows of 256 k, the window sums added in float-float; FP64 radial
                     scans.  Phi within 1e-12 of FP64.  The FP32 window sums bound the field:
                     values (and their products with U) must stay well inside FP32's range */
} ygs_precision;

typedef enum {
  YGS_EVAL_UPPER_VERTEX = 0, /* (r_i^+, theta_j^+, phi_k^+), Sect. 4.2 */
  YGS_EVAL_CELL_CENTRE = 1   /* (r_i^+, angular centre of the cell) */
} ygs_eval;

enum {
  YGS_FLAG_NO_SYMMETRY = 1, /* never use the Yin-Yang sign symmetry of Sect. 4.2 */
  YGS_FLAG_AUTOTUNE = 2,    /* split precisions: ygs_create times, on this GPU, the projection
                               with several split-K counts (angular chunks per shell tile) and,
                               but for YGS_FP64_EMU, the synthesis at every distinct shell
                               tiling of full-tile widths 144, 96 and 48 shells, on one CTA
                               per 128-cell tile and on CTA pairs, and keeps the fastest of
                               each (a few ms more at create, and a scratch Phi of n_cells
                               doubles while it runs; ygs_info reports the choices).  The
                               synthesis's results do not depend on its tile shape; the
                               projection's differ from an untuned plan's within the
                               precision's bound, as the chunk sums are added in another
                               grouping */
  YGS_FLAG_CTA_PAIRS = 4    /* split precisions but YGS_FP64_EMU: run the synthesis on pairs of
                               CTAs that share each MMA (cta_group::2, 256 cells per tile, each
                               CTA staging half of the tile's shells of M) instead of one CTA
                               per 128-cell tile.  Bitwise the same results; on GB300 at the
                               1-degree, 400-shell grid 20% slower (the synthesis is held by its
                               epilogue, not by operand traffic), so it is off by default */
};

/* Grid descriptor.  All arrays are HOST memory, read during ygs_create only. */
/* Patch geometry (ygs_desc.patch_kind). */
typedef enum {
  YGS_PATCH_LATLON = 0,  /* local spherical coordinates (Sect. 2.1): theta_range and phi_range are the local
                            colatitude and azimuth extents; U by the Wigner-D route (Sect. 3) */
  YGS_PATCH_GNOMONIC = 1 /* a non-orthogonal patch (Sect. 6): a cube face in equiangular gnomonic
                            coordinates.  theta_range and phi_range hold the extents of xi and eta
                            (radians, inside (-pi/2, pi/2)); the local direction of (xi, eta) is
                            (tan xi, tan eta, 1) / sqrt(1 + tan^2 xi + tan^2 eta), turned by R^(g); cell
                            (j, k) spans the j-th xi and k-th eta interval, k fastest; U is integrated
                            numerically (10-point Gauss-Legendre panels in xi and eta with the solid-angle
                            density (1 + X^2)(1 + Y^2) / (1 + X^2 + Y^2)^(3/2), X = tan xi, Y = tan eta);
                            the evaluation point is the upper vertex (xi_{j+1}, eta_{k+1}) or the centre.
                            The six faces of a cube, xi, eta in [-pi/4, pi/4], tile the sphere (w = 1). */
} ygs_patch_kind;

typedef struct {
  int n_r;                    /* number of radial shells, >= 1 */
  const double* r_edges;      /* n_r + 1 edges, strictly increasing, r_edges[0] >= 0 */
  int n_patch;                /* number of patches N_g, >= 1 */
  const double* euler;        /* 3*n_patch: (alpha, beta, gamma) of Eq. rottransmatrix */
  const int* n_theta;         /* n_patch: cells in local colatitude, >= 1 */
  const int* n_phi;           /* n_patch: cells in local azimuth, >= 1 */
  const double* theta_range;  /* 2*n_patch: [theta_lo, theta_hi], 0 <= lo < hi <= pi */
  const double* phi_range;    /* 2*n_patch: [phi_lo, phi_hi], lo < hi, hi - lo <= 2 pi */
  const double* overlap_w;    /* sum_g n_theta*n_phi cell-constant weights w_jk (Sect. 4.2) */
  int l_max;                  /* expansion degree, 0 <= l_max <= 128 */
  double G;                   /* gravitational constant */
  int eval;                   /* ygs_eval */
  int precision;              /* ygs_precision */
  int flags;                  /* YGS_FLAG_* */
  const int* patch_kind;      /* n_patch ygs_patch_kind values, or NULL: every patch YGS_PATCH_LATLON */
} ygs_desc;

typedef struct ygs_plan ygs_plan;

/* Sizes and modes of a plan (for callers and tests). */
typedef struct {
  int n_r, n_patch, l_max, K;
  long long n_ang;        /* sum_g n_theta*n_phi */
  long long n_cells;      /* n_r * n_ang: elements of one field */
  int precision;
  int symmetric;          /* 1: the Yin-Yang sign symmetry halves the contractions */
  int split_k;            /* number of angular chunks the projection is split into */
  long long weight_bytes; /* device bytes held for U, Q and their split copies */
  long long work_bytes;   /* device bytes of per-solve workspace */
  int fp64_split_k;       /* angular chunks of the FP64 kernels' projection (= split_k on FP64
                             plans; ygs_solve_static always runs those kernels) */
  long long static_scratch_bytes; /* scratch ygs_solve_static needs for this plan:
                                     (fp64_split_k + 2) * n_r * K * 8 */
  int cta_pairs;          /* 1: the synthesis runs on CTA pairs (YGS_FLAG_CTA_PAIRS on a split
                             plan other than YGS_FP64_EMU, and the GPU can co-schedule them,
                             or the autotuner picked them) */
  int synth_tile_shells;  /* split plans: shells per full synthesis tile (144, 128 for
                             YGS_FP64_EMU, or the width YGS_FLAG_AUTOTUNE picked); 0 on FP64 plans */
} ygs_info;

/* Builds the plan: validates the descriptor, allocates device memory on
 * `device`, and evaluates the FP64 weights U (Wigner-D route, Eqs. U_C/U_S),
 * Q (Eqs. Q_C/Q_S) and the radial factors of Eqs. R_in/R_out on the GPU
 * (step 1 of Sect. 4.3).  Synchronous.  On failure *out is set to NULL and
 * nothing is leaked.  Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED.
 * Testing hook: with YGS_INJECT_ALLOC_FAILURE=k in the environment, the k-th
 * device allocation of this call fails as if the device were out of memory. */
ygs_status ygs_create(const ygs_desc* desc, int device, ygs_plan** out);

/* Frees every device buffer of the plan (waits for its pending work).
 * NULL is accepted. */
ygs_status ygs_destroy(ygs_plan* plan);

ygs_status ygs_get_info(const ygs_plan* plan, ygs_info* info);

/* Phi = A rho: steps 2-5 of Sect. 4.3 on device pointers.  rho and phi each
 * hold n_cells FP64 values in the field layout above and must not overlap.
 * `stream` is a cudaStream_t (NULL: legacy default stream).  Errors:
 * INVALID_ARG (NULL/misaligned pointer), CUDA (launch failure). */
ygs_status ygs_solve(ygs_plan* plan, const double* d_rho, double* d_phi, void* stream);

/* The same solve from and to HOST buffers: copies rho host->device, solves,
 * copies Phi device->host on `stream`, then synchronises the stream.  Host
 * buffers should be page-locked for full copy bandwidth. */
ygs_status ygs_solve_host(ygs_plan* plan, const double* h_rho, double* h_phi, void* stream);

/* n solves of one plan from and to HOST buffers, pipelined: field k + 1 is
 * copied host->device and Phi_{k-1} device->host (on two copy streams of the
 * plan, made on first use) while field k is solved on `stream`, through two
 * device staging pairs (4 * n_cells doubles, allocated on first use and kept
 * with the plan).  h_rho[k] and h_phi[k] (HOST arrays of n host pointers)
 * each hold n_cells doubles and should be page-locked, or the copies do not
 * overlap; an h_phi[k] must not overlap any h_rho[j] with j > k (those are
 * still being read while Phi_k is written).  The same h_rho or h_phi buffer
 * may appear several times.  Returns after the last Phi is in h_phi[n - 1] (synchronises
 * `stream`; not capturable into a CUDA graph).  n = 0 does nothing.
 * Errors: INVALID_ARG (NULL plan or pointer, n < 0), OOM, CUDA. */
ygs_status ygs_solve_host_many(ygs_plan* plan, int n, const double* const* h_rho, double* const* h_phi,
                               void* stream);

/* n independent solves (plans may differ in every size) as one unit of work
 * on `stream`: the fields are forked onto a pool of internal worker streams
 * (fields of the same plan stay in order on one worker, since they share its
 * workspaces) and joined back onto `stream` with events, so independent
 * fields run concurrently and the whole batch can be captured into one CUDA
 * graph.  plans, d_rho and d_phi are HOST arrays of n entries each; all plans
 * must live on one device.  Errors: as ygs_solve. */
ygs_status ygs_solve_batched(int n, ygs_plan* const* plans, const double* const* d_rho,
                             double* const* d_phi, void* stream);

/* A fixed set of plans whose solves run together (the paper solves one field;
 * batching many independent fields of uneven sizes is this library's).
 * ygs_batch_create prepares, once, device descriptors of every split-precision
 * plan's contractions; plans are grouped by operand kind (BF16 two-slice, FP16
 * two-slice, BF16 three-slice) and each group's projection and synthesis tiles then run
 * in ONE persistent launch each per ygs_batch_solve, instead of one launch per
 * field.  FP64 plans of the batch run their ordinary solves.  All plans must
 * live on one device and appear once; they must outlive the batch.  At most
 * 128 split plans per operand kind, 1024 plans in all.  Errors: INVALID_ARG,
 * OOM, CUDA, UNSUPPORTED. */
typedef struct ygs_batch ygs_batch;
ygs_status ygs_batch_create(int n, ygs_plan* const* plans, ygs_batch** out);
/* Solves every field of the batch on `stream`: d_rho[k] -> d_phi[k] for plan k
 * (HOST arrays of device pointers, layouts and pointer rules of ygs_solve).
 * Enqueues work only: no allocation and no synchronisation, so a whole batch
 * can be captured into one CUDA graph.  Results equal ygs_solve's bitwise. */
ygs_status ygs_batch_solve(ygs_batch* batch, const double* const* d_rho, double* const* d_phi, void* stream);
/* Frees the descriptors (waits for the device).  NULL is accepted. */
ygs_status ygs_batch_destroy(ygs_batch* batch);
/* Kernel launches one ygs_batch_solve enqueues. */
int ygs_batch_launches(const ygs_batch* batch);

/* Adjoint of the linear map rho -> Phi:  grad_rho = A^T grad_phi
 * (transposed synthesis, reversed radial scans, transposed projection).
 * Same layouts, pointer rules and errors as ygs_solve.  It runs in the plan's
 * precision: FP64 plans on the FP64 kernels; split-precision plans on the
 * tensor cores with slices of Q^T and U made at ygs_create (grad_phi Q, the
 * transposed scans in FP64, then U), within the same relative bound of the
 * FP64 adjoint as ygs_solve of the FP64 solve. */
ygs_status ygs_backward(ygs_plan* plan, const double* d_grad_phi, double* d_grad_rho, void* stream);

/* Copies the moments B and the radial weights M of the most recent solve on
 * this plan into device buffers of n_r*K FP64 values each, row-major
 * [i][c] in the column order above (either pointer may be NULL).
 * Accuracy per degree band (relative 2-norm of a degree's columns against
 * FP64): FP64, FP64_TC and FP64_EMU plans hold B and M to FP64 accuracy
 * (FP64_EMU: about 1e-14).  The split precisions reach their Phi bound on the
 * monopole and the low degrees, but the FP32 accumulation between flushes
 * costs the high degrees, whose terms cancel: at 0.5 degree, Nr = 800,
 * l_max = 64, FP16X3 (flushed every 128 k in the forward projection) left B
 * within 1.2e-6 .. 8.9e-6 for l >= 24 and M within 7.3e-7, while Phi stayed at
 * 1.6e-7.  A caller that consumes B or M beyond 1e-6 uses FP64_EMU (or FP64). */
ygs_status ygs_get_moments(ygs_plan* plan, double* d_B, double* d_M, void* stream);

/* ---- angular sharding (Sect. 4.3, steps 2-3) ------------------------------
 * The paper's distributed solve: every process projects its share of the
 * angular cells (Eq. B_CS), the partial moments are summed over all
 * processes (one reduction of n_r*K values), and every process finishes the
 * solve (radial scans, Eq. M_C, and synthesis, Eq. gravpotmult) from the
 * whole B.  The share is a range of the plan's FP64 split-K chunks
 * (ygs_info.fp64_split_k of them; chunk z covers a fixed block of one
 * patch's angular cells), so the ranges [0, c1), [c1, c2), ... [c_{n-1},
 * fp64_split_k) of n processes cover every cell once.  Both calls run on the
 * plan's FP64 weights and workspaces (whatever the plan's precision), enqueue
 * work only and do not synchronise; the reduction between them is the
 * caller's (an MPI or NCCL all-reduce, or gloo on host copies).  On an FP64
 * plan ygs_get_moments then returns the B and M of the finish. */

/* d_B (n_r*K FP64, device, row-major [i][c] in ygs_get_moments' column order)
 * = the moments of the cells of chunks [chunk_begin, chunk_end) of d_rho
 * (the layout of ygs_solve).  An empty range writes zeros.
 * Errors: INVALID_ARG for NULL or unaligned pointers (16 bytes) or a range
 * outside [0, fp64_split_k]. */
ygs_status ygs_project_partial(ygs_plan* plan, const double* d_rho, int chunk_begin, int chunk_end, double* d_B,
                               void* stream);
/* d_phi (the layout of ygs_solve) from the moments d_B of the whole field
 * (layout of ygs_project_partial): the radial scans and the synthesis.
 * Errors: INVALID_ARG for NULL, unaligned or overlapping pointers. */
ygs_status ygs_finish_from_moments(ygs_plan* plan, const double* d_B, double* d_phi, void* stream);

/* Copies the FP64 weights of patch `patch` to HOST memory as [n_theta*n_phi][K]
 * row-major: which = 0 -> U, which = 1 -> Q.  Synchronous. */
ygs_status ygs_get_weights(ygs_plan* plan, int which, int patch, double* h_out);

/* Reads and clears the plan's device error word (set by bounded waits and
 * device-side checks).  Synchronises the plan's last stream.  In a checked
 * build it also reads and clears the device's out-of-range record (shared by
 * every plan on the device; the first event since the last read) and returns
 * YGS_ERR_BOUNDS for it, ygs_last_error naming the kernel site and index. */
ygs_status ygs_get_status(ygs_plan* plan);

/* 1 in a checked build of the library: compiled with YGS_DEBUG_BOUNDS=1
 * (python -m paper_1903_08475_gb300.build --checked, into _build_checked/),
 * every per-solve kernel checks the global index of its main loads and
 * stores against the extent of the buffer it addresses and, outside it,
 * skips the access and records the event for ygs_get_status instead of
 * faulting.  0 in the release build, whose kernels carry no checks.  The
 * Python binding loads another build named by the environment variable
 * YGS_LIB.  (Sanitiser-style checking for development; no counterpart in
 * the paper.) */
int ygs_checked_build(void);

/* Checked builds only (YGS_ERR_UNSUPPORTED otherwise): the field extent the
 * kernels' checks hold rho and Phi to, normally n_cells, set to n in
 * [0, n_cells] for the calls that follow.  A smaller n makes the checks
 * report (and skip) the accesses to elements n and beyond, so a test can see
 * a check fire without any access leaving the buffers; ygs_get_status then
 * returns YGS_ERR_BOUNDS.  The results of such calls are incomplete. */
ygs_status ygs_debug_set_field_extent(ygs_plan* plan, long long n);

/* Phase timing for measurement.  While enabled, every ygs_solve and
 * ygs_backward on this plan records CUDA events on its stream around its four
 * phases (0: field preparation (BF16 slicing; empty on the FP64 path),
 * 1: projection, 2: radial scans, 3: synthesis); at most 4096 calls are kept.
 * ygs_read_phase_times synchronises on those events, writes the summed
 * milliseconds of each phase (ms[0..3]) and the number of calls recorded
 * since the previous read, and clears the record. */
ygs_status ygs_set_profiling(ygs_plan* plan, int enable);
ygs_status ygs_read_phase_times(ygs_plan* plan, double* ms, int* n_calls);

/* Diagnostic of the failure path.  Enqueues a kernel that polls an mbarrier
 * nothing arrives at, at most `spins` times (the bounded wait every kernel of
 * this library uses), and then records YGS_ERR_TIMEOUT in the plan's error
 * word; ygs_get_status reports it once and clears it.  No GPU fault is
 * involved and the context stays usable. */
ygs_status ygs_debug_wait_timeout(ygs_plan* plan, int spins, void* stream);

/* Size of the device array behind ygs_solve_static, in bytes. */
#define YGS_STATIC_SCRATCH_BYTES (32u << 20)

/* Phi = A rho like ygs_solve, always in FP64 on the plan's FP64 weights, with
 * no device allocation: the split-K partial sums and the moments B and M live
 * in one file-scope device array of YGS_STATIC_SCRATCH_BYTES (32 MiB) per
 * device instead of the plan's workspaces.  The paper has no counterpart; it
 * serves callers that may not allocate at solve time (a host code that has
 * given all free device memory to its own pool, a running time-step loop that
 * forbids allocator calls).
 * Limit: the plan must need at most YGS_STATIC_SCRATCH_BYTES of scratch,
 * ygs_info.static_scratch_bytes = (fp64_split_k + 2) * n_r * K * 8 bytes
 * (fp64_split_k, not split_k: a split-precision plan's tensor-core path chunks
 * its projection differently); a larger plan returns UNSUPPORTED with the
 * sizes in ygs_last_error() and enqueues nothing.
 * ygs_create loads the module that holds the array (allocating it, once per
 * device and process) and the FP64 kernels, so no call of this function
 * allocates; each call looks the array's address up on the current device.
 * The array is shared by all calls on a device in the process: calls whose GPU
 * work overlaps (unordered streams, concurrent host threads) race on it.  No
 * part of it has to start at zero.  The plan's own moments (ygs_get_moments)
 * are not updated.  Errors: as ygs_solve, plus UNSUPPORTED for the limit. */
ygs_status ygs_solve_static(ygs_plan* plan, const double* d_rho, double* d_phi, void* stream);

/* YGS_STATIC_SCRATCH_BYTES, for bindings that cannot read this header. */
size_t ygs_static_scratch_capacity(void);

/* Number of kernel launches one ygs_solve (or ygs_backward) enqueues. */
int ygs_launches_per_solve(const ygs_plan* plan);

const char* ygs_status_string(ygs_status s);
const char* ygs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* YGS_H */
