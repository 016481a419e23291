// Internal declarations of libygs (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ygs.h"

namespace ygs {

constexpr int kMaxPatch = 64;
constexpr int kMaxLmax = 128;

// Per-call description of the angular layout, passed to kernels by value.
struct PatchTable {
  long long fld_off[kMaxPatch];  // element offset of patch g in a field
  long long nang[kMaxPatch];     // angular cells of patch g
  long long ang_off[kMaxPatch];  // row offset of patch g in a weight matrix
  long long n_cells;             // elements of a whole field (the checked build's bound for rho and Phi)
  long long w_rows;              // rows of the stored FP64 weight matrices U and Q (each w_rows x K)
};

// ---- checked builds ----
// Built with -DYGS_DEBUG_BOUNDS=1 (build.py's debug library), every
// per-solve kernel checks the global index of its main loads and stores
// against the extent of the buffer it addresses, taken from the plan's sizes.
// An index outside [0, extent) skips the access and records the first such
// event (site, index) in a device word of the translation unit;
// ygs_get_status reports it as YGS_ERR_BOUNDS (ygs_last_error names the site
// and the index) and clears it.  In release builds the checks compile to
// nothing.
#ifndef YGS_DEBUG_BOUNDS
#define YGS_DEBUG_BOUNDS 0
#endif
enum BoundsSite {
  kSiteField16Rho = 1, kSiteField16Slices, kSiteField16Fac, kSiteField16U00, kSiteFieldSlicesRho,
  kSiteFieldSlicesOut, kSiteScanPart, kSiteScanBM, kSiteScanMs, kSiteSliceM16In, kSiteSliceM16Out, kSiteGemmPhi,
  kSiteGemmPart, kSiteGemmFac, kSiteProjField, kSiteProjW, kSiteProjPart, kSiteSynthX, kSiteSynthW, kSiteSynthPhi,
  kSiteScanFwd, kSiteScanAdj, kSiteEmuFieldRho, kSiteEmuFieldOut, kSiteEmuScan, kSiteBoundsSites
};
const char* bounds_site_name(int site);
#if YGS_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds[3];  // {flag, site, index} of this translation unit
__device__ __forceinline__ bool bounds_ok(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(&g_bounds[0], 0ull, 1ull) == 0ull) {
    g_bounds[1] = (unsigned long long)site;
    g_bounds[2] = (unsigned long long)i;
  }
  return false;
}
#define YGS_IN_BOUNDS(i, n, site) ::ygs::bounds_ok((long long)(i), (long long)(n), (site))
// Host: reads and clears this translation unit's word on the current device.
#define YGS_BOUNDS_READER(fn)                                                            \
  cudaError_t fn(int* site, long long* index) {                                          \
    unsigned long long h[3] = {0, 0, 0};                                                 \
    cudaError_t e = cudaMemcpyFromSymbol(h, g_bounds, sizeof(h));                        \
    if (e != cudaSuccess) return e;                                                      \
    *site = h[0] ? (int)h[1] : 0;                                                        \
    *index = (long long)h[2];                                                            \
    if (h[0]) {                                                                          \
      const unsigned long long z[3] = {0, 0, 0};                                         \
      e = cudaMemcpyToSymbol(g_bounds, z, sizeof(z));                                    \
    }                                                                                    \
    return e;                                                                            \
  }
#else
#define YGS_IN_BOUNDS(i, n, site) true
#define YGS_BOUNDS_READER(fn)                \
  cudaError_t fn(int* site, long long* index) { \
    *site = 0;                               \
    *index = 0;                              \
    return cudaSuccess;                      \
  }
#endif
// the readers of the translation units with per-solve kernels
cudaError_t bounds_read_tc(int* site, long long* index);
cudaError_t bounds_read_fp64(int* site, long long* index);
cudaError_t bounds_read_emu(int* site, long long* index);

// One split-K chunk of the projection: angular cells [a0, a1) of patch g.
struct Chunk {
  int g, a0, a1, pad;
};

}  // namespace ygs

struct ygs_plan {
  int device = 0;
  int n_r = 0, n_patch = 0, l_max = 0, K = 0;
  int precision = 0, eval = 0, flags = 0;
  double G = 1.0;
  bool symmetric = false;   // Yin-Yang sign symmetry in use
  int n_wpatch = 0;         // patches with stored weights (1 when symmetric)
  int K_even = 0;           // internal columns [0, K_even) have even m when symmetric, else K_even = K
  std::vector<int> nth, nph;
  std::vector<int> kind;    // ygs_patch_kind per patch
  std::vector<double> euler, theta_range, phi_range, edges, w_host;
  std::vector<long long> nang, ang_off, fld_off;
  long long nang_total = 0, nang_wtotal = 0, n_cells = 0;
  std::vector<int> col_perm;  // internal column -> natural column
  ygs::PatchTable pt{};

  // device buffers owned by the plan
  double* U = nullptr;      // [nang_wtotal][K] internal column order
  double* Q = nullptr;      // [nang_wtotal][K]
  double* rad = nullptr;    // [4][l_max+1][n_r]: a, b, f_in, f_out
  int* col_l = nullptr;     // [K] degree of each internal column
  int* col_nat = nullptr;   // [K] natural index of each internal column
  ygs::Chunk* chunks = nullptr;
  int S = 0;                // split-K chunks
  double* part = nullptr;   // [S][n_r][K] projection partials
  double* B = nullptr;      // [n_r][K]
  double* M = nullptr;      // [n_r][K]
  // FP32 CUDA-core path (YGS_FP32): FP32 copies of the weights, the field, partials and M
  float *U32 = nullptr, *Q32 = nullptr, *f32_field = nullptr, *part32 = nullptr, *M32 = nullptr;
  double* Mbar = nullptr;   // [n_r][K] adjoint workspace
  double* Bbar = nullptr;   // [n_r][K] adjoint workspace
  double* h2d_rho = nullptr;  // device staging for ygs_solve_host
  double* h2d_phi = nullptr;
  // ygs_solve_host_many: the second staging pair, the copy streams and their
  // events (start, in[2], comp[2], out[2]), made on first use
  double* h2d_rho2 = nullptr;
  double* h2d_phi2 = nullptr;
  cudaStream_t hm_in = nullptr, hm_out = nullptr;
  cudaEvent_t hm_ev[7] = {};
  int* d_err = nullptr;     // device error word
  cudaStream_t last_stream = nullptr;
  // phase profiling: 4 events per recorded call
  bool profiling = false;
  std::vector<cudaEvent_t> prof_events;
  int prof_used = 0;
  long long weight_bytes = 0, work_bytes = 0;

  // ---- split-precision (tcgen05) path
  int tc_nsl = 0;            // BF16 or FP16 slices per operand (0: FP64 path)
  int tc_N = 0;              // shells per full tile
  int tc_np_full = 0;        // full shell tiles of the projection
  int tc_np_tail = 0;        // width of the projection's tail shell tile (0: none)
  int tc_n_full = 0;         // full shell tiles of the synthesis
  int tc_n_tail = 0;         // width of the tail shell tile (0: none)
  int tc_sms = 0;            // CTAs of the persistent contraction kernels
  int tc_pairs = 0;          // >0: the synthesis runs on CTA pairs, at most this many clusters of two
  int tc_k_even = 0, tc_k_pad = 0;
  long long tc_n_pad = 0;
  std::vector<long long> tc_pad_off;
  int tc_S = 0, tc_scan_chunk = 0, tc_scan_P = 0;
  __nv_bfloat16 *tc_ut = nullptr, *tc_qs = nullptr, *tc_f = nullptr, *tc_ms = nullptr;
  float2* tc_part = nullptr;
  float2 *tc_B = nullptr, *tc_M = nullptr;  // [n_r][K_pad] float-float moments of the last solve
  double *tc_summ = nullptr, *tc_carry = nullptr;
  int2* tc_chunks = nullptr;
  int *tc_pc_int = nullptr, *tc_pc_l = nullptr, *tc_pc_nat = nullptr;
  long long* tc_pad_off_d = nullptr;
  float2* tc_mono = nullptr;  // -G M[i][0] per shell as (hi, lo)
  float2* tc_cp = nullptr;    // [2][l_max+1][P] radial ratio products per chunk of shells (float-float)
  float2* tc_radff = nullptr; // [4][l_max+1][n_r] the radial tables a, b, f_in, f_out as float-float
  int tc_tf32 = 0;            // TF32 slices (YGS_TF32X3): 4-byte elements behind the slice pointers
  // FP64-accurate slices (YGS_FP64_EMU): six exact 8-bit BF16 slices per
  // value (tc_nsl = 6), the field on per-window grids (factors in tc_fac), M
  // on per-shell grids (tc_sc); FP64 radial scans into tc_Bd / tc_Md
  int tc_emu = 0;
  double *tc_Bd = nullptr, *tc_Md = nullptr;  // [n_r][K_pad] FP64 B and M of the last solve
  // FP16 slices (YGS_FP16X3): power-of-two exponents that scale each operand row into FP16's range
  int tc_fp16 = 0;
  int tc_eq = 0;              // Q (all rows)
  int* tc_eu = nullptr;       // [K_pad] U^T row (column c)
  float* tc_fac = nullptr;    // [2][n_pad / 128][n_r] 2^-e of the field row (plane, exponent group, shell), per solve
  int* tc_em = nullptr;       // [n_r] M row (shell), written by every solve
  float4* tc_sc = nullptr;    // [n_r] the synthesis epilogue's per-shell {exponent rebase, 0, scaled monopole pair}, per solve
  float2* tc_u00 = nullptr;   // [n_pad] monopole weight of every stored cell (float-float), padded layout
  float2* tc_mpart = nullptr; // [S][n_r] exact monopole moment per split-K chunk, written by every solve
  CUtensorMap tc_map_ut, tc_map_f, tc_map_f_tail, tc_map_q, tc_map_m, tc_map_m_tail;
  // adjoint on the tensor cores: Q^T slices in the projection layout, U slices
  // in the synthesis layout (monopole column kept), their FP16 exponents, and
  // FP64 Mbar / Bbar in the padded column order (the field, partial, summary,
  // carry and M-slice buffers of the forward solve are reused)
  __nv_bfloat16 *tc_qt = nullptr, *tc_us = nullptr;
  int* tc_eqt = nullptr;      // [K_pad] Q^T row (column c)
  int tc_eus = 0;             // U (all rows)
  float2 *tc_Mbar = nullptr, *tc_Bbar = nullptr;  // float-float (EMU: n_r K_pad doubles each)
  CUtensorMap tc_map_qt, tc_map_us;
  CUtensorMap tc_map_m2, tc_map_m2_tail;  // M slices in boxes of half a synthesis tile's shells (CTA pairs)
};

namespace ygs {

// Thread-local error message for ygs_last_error().
void set_error(const std::string& msg);

// cudaMalloc through one door: when YGS_INJECT_ALLOC_FAILURE=k is set in the
// environment at ygs_create, the k-th device allocation of that create fails
// with cudaErrorMemoryAllocation (host-side fault injection for tests).
cudaError_t dev_malloc(void** ptr, size_t bytes);
void arm_alloc_injection();

// ---- weight builder (ygs_weights.cu) -------------------------------------
// Builds U, Q (FP64, internal column order) and the radial tables of `p`
// with every allocation it needs; synchronous.
ygs_status build_weights(ygs_plan* p);

// ---- FP64 contractions and scans (ygs_fp64.cu) ----------------------------
// part[z][i][c] = sum over chunk z of field(i, a) * W[a][c]  (projection shape)
cudaError_t launch_project_fp64(const ygs_plan* p, const double* field, const double* W, double* part,
                                cudaStream_t s);
// out(g, i, a) = sum_c X[i][c] W[a][c]  (synthesis shape)
cudaError_t launch_synth_fp64(const ygs_plan* p, const double* X, const double* W, double* out, cudaStream_t s);
// B = sum_z part[z]; M = scaled inner + outer radial scans of B.
cudaError_t launch_scan_fwd(const ygs_plan* p, const double* part, int S, double* B, double* M, cudaStream_t s);
// Mbar = sum_z part[z]; Bbar = transposed scans of Mbar.
cudaError_t launch_scan_adj(const ygs_plan* p, const double* part, int S, double* Bbar, cudaStream_t s);
// Loads the FP64 kernels' module on the current device (they are loaded
// lazily otherwise, at their first launch, which may allocate device memory).
cudaError_t preload_fp64_kernels();
// Makes the static scratch array of ygs_solve_static resident on the current
// device (ygs_noalloc.cu): its module is loaded, and its array allocated, here
// rather than at the first ygs_solve_static.
cudaError_t prepare_static_scratch();
// Scratch bytes ygs_solve_static needs for plan p: (S + 2) n_r K doubles.
long long static_scratch_bytes(const ygs_plan* p);
// out[i][col_nat[c]] = in[i][c]
cudaError_t launch_unpermute(const ygs_plan* p, const double* in, double* out, cudaStream_t s);
// out[i][c] = in[i][col_nat[c]] (natural column order -> internal)
cudaError_t launch_permute(const ygs_plan* p, const double* in, double* out, cudaStream_t s);
// The FP64 projection of the chunks [z0, z1) of the plan's list into part[0 .. z1 - z0).
cudaError_t launch_project_fp64_chunks(const ygs_plan* p, const double* field, const double* W, double* part, int z0,
                                      int z1, cudaStream_t s);
// B = sum_{z < S} part[z] (fixed order).
cudaError_t launch_sum_partials(const ygs_plan* p, const double* part, int S, double* B, cudaStream_t s);
// FP64 -> FP32 (rounded, or truncated by integer operations)
cudaError_t launch_to_f32(const double* in, float* out, long long n, bool trunc, cudaStream_t s);
// The FP32 CUDA-core solve (YGS_FP32): FP32 contractions, FP64 scans; ev optional phase events 1..3
cudaError_t solve_fp32(const ygs_plan* p, const double* rho, double* phi, cudaStream_t s, cudaEvent_t* ev);

// ---- split-precision tensor-core path (ygs_tc.cu) --------------------------
ygs_status tc_setup(ygs_plan* p, int sms);     // slices, tensor maps, workspaces (at create)
void tc_free(ygs_plan* p);
// forward: FP16 plans also sum the monopole moment's chunk partials (the
// adjoint's input needs none)
cudaError_t tc_field_slices(const ygs_plan* p, const double* rho, cudaStream_t s, bool forward = true);
cudaError_t tc_project(const ygs_plan* p, cudaStream_t s);
cudaError_t tc_scan(const ygs_plan* p, cudaStream_t s);
cudaError_t tc_synthesize(const ygs_plan* p, double* phi, cudaStream_t s);
cudaError_t tc_unpermute(const ygs_plan* p, const float2* in, double* out, cudaStream_t s);
// Batches: the split-precision plans of a batch grouped by operand kind; each
// group's projection and synthesis tiles run in one persistent launch, with
// the problems' tensor maps and arguments in device memory.
namespace tc {
struct TcProblem;
}
// One per-field pass of a batch run as a single grouped launch: its
// problems' argument structs and grid shapes (tc::GroupDims) in device memory.
struct TcGroupedPass {
  void* d_args = nullptr;
  void* d_dims = nullptr;
  int blocks = 0;  // blocks of all problems
};
struct TcBatchGroup {
  int nsl = 0, fp16 = 0, tf32 = 0, emu = 0, sms = 0, total_p = 0, total_s = 0;
  std::vector<ygs_plan*> members;
  tc::TcProblem *d_proj = nullptr, *d_synth = nullptr;
  int *d_start_p = nullptr, *d_start_s = nullptr;
  TcGroupedPass field, scan, mslice;  // field slices, scans, M slicing (FP16 and EMU)
};
// Uploads a grouped pass: n argument structs of arg_bytes each and the
// problems' grid shapes (gx, gy, gz per problem).
cudaError_t upload_grouped_pass(TcGroupedPass& P, const void* args, size_t arg_bytes, int n, const int* gx,
                                const int* gy, const int* gz);
struct TcBatch {
  std::vector<TcBatchGroup> groups;
};
ygs_status tc_batch_build(TcBatch* b, const std::vector<ygs_plan*>& plans);
void tc_batch_free(TcBatch* b);
// The field slices of every member (rho[k] for member k) in one grouped launch.
cudaError_t tc_batch_field(const TcBatchGroup& g, const double* const* rho, cudaStream_t s);
// The scans (and M slicing) of every member in one grouped launch each.
cudaError_t tc_batch_scan(const TcBatchGroup& g, cudaStream_t s);
cudaError_t tc_batch_project(const TcBatchGroup& g, cudaStream_t s);
// phi[k]: output of the group's k-th member
cudaError_t tc_batch_synthesize(const TcBatchGroup& g, double* const* phi, cudaStream_t s);

// grad_rho = A^T grad_phi on the tensor cores: slices of grad_phi, projection
// with Q, transposed scans, synthesis with U.
cudaError_t tc_backward(const ygs_plan* p, const double* gphi, double* grho, cudaStream_t s, cudaEvent_t* ev);
cudaError_t debug_wait_timeout(const ygs_plan* p, int spins, cudaStream_t s);

// ---- FP64-accurate splitting on the BF16 tensor cores (ygs_emu.cu) ----------
// Cells per exponent window of the field (the flush group of its contraction).
constexpr int kEmuWindow = 1024;
// The weights' slices of an EMU plan (tc_ut, tc_qs, tc_qt, tc_us: six each,
// on per-row grids, monopole columns kept); synchronous, at create.
cudaError_t emu_slice_weights(ygs_plan* p);
// Shared-memory limits of the EMU contraction kernels (at create).
cudaError_t emu_set_smem_attrs();
// Field slices sigma+- (or rho) on per-(plane, window, shell) grids and their
// factors 2^e in tc_fac.
cudaError_t emu_field_slices(const ygs_plan* p, const double* rho, cudaStream_t s);
// Forward scans in FP64 (B, M into tc_Bd / tc_Md, float-float copies into
// tc_B / tc_M), then M's slices and tc_sc.
cudaError_t emu_scan(const ygs_plan* p, cudaStream_t s);
// Adjoint scans in FP64 (Mbar, Bbar into tc_Mbar / tc_Bbar as doubles), then Bbar's slices.
cudaError_t emu_scan_adj(const ygs_plan* p, cudaStream_t s);
// out[i][natural column] = in[i][pc] for FP64 moments in the padded column order.
cudaError_t emu_unpermute(const ygs_plan* p, const double* in, double* out, cudaStream_t s);
// The grouped field, scan and M-slicing passes of a batch's EMU members.
cudaError_t emu_batch_passes(const std::vector<ygs_plan*>& members, TcBatchGroup& G);
cudaError_t emu_batch_field(const TcBatchGroup& G, const double* const* rho, cudaStream_t s);
cudaError_t emu_batch_scan(const TcBatchGroup& G, cudaStream_t s);
// The EMU contraction kernels (one problem, or a group of problems).
namespace tc {
struct TcArgs;
struct TcPhiList;
}
cudaError_t emu_dispatch_gemm(int mode, int grid, const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& bt,
                              const tc::TcArgs& args, cudaStream_t s);
cudaError_t emu_dispatch_group(int mode, int grid, const tc::TcProblem* probs, const int* start, int n, int total,
                               const tc::TcPhiList& phis, cudaStream_t s);

}  // namespace ygs
