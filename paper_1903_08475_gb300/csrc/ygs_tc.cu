// Split-precision path: BF16-slice operands on tcgen05 tensor cores for the
// two contractions (steps 2 and 5 of Sect. 4.3), FP64 radial scans (step 4).
//
// Layouts (K_pad: internal columns padded per parity block to multiples of 64;
// n_pad: angular cells of each stored patch padded to whole k-blocks of BK):
//   Ut  [s][K_pad][n_pad]  slices of U^T      (projection A operand)
//   F   [h*NSL+s][Nr][n_pad] slices of the field: h = 0 sigma+ (or rho), h = 1 sigma-
//   Qs  [s][n_wtotal][K_pad] slices of Q       (synthesis A operand)
//   Ms  [s][Nr][K_pad]       slices of M       (synthesis B operand)
//   part [z][Nr][K_pad] float2 (hi, lo) projection partials of chunk z
#include <algorithm>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_fp16.h>

#include "ygs_tc_gemm.cuh"

namespace ygs {

using tc::TcArgs;
using tc::TcCfg;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Operand kind of a plan's slices: BF16, FP16 (scaled rows) or TF32 (FP32 storage).
enum SliceKind { kSliceBF16 = 0, kSliceFP16 = 1, kSliceTF32 = 2 };
int slice_kind(const ygs_plan* p) { return p->tc_tf32 ? kSliceTF32 : (p->tc_fp16 ? kSliceFP16 : kSliceBF16); }
size_t slice_bytes(const ygs_plan* p) { return p->tc_tf32 ? 4 : 2; }

// 3-D slice tensor (kdim fastest, rows, planes) read in boxes of one 128-byte
// k-block row (BK 2-byte or BK / 2 TF32 elements) x box_rows x 1, swizzled to
// match the UMMA shared-memory descriptors (128-byte swizzle for BK = 64).
bool make_map(CUtensorMap* m, void* base, long long kdim, long long rows, long long planes, int box_rows, int kind) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t esz = kind == kSliceTF32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)kdim * esz, (cuuint64_t)kdim * esz * rows};
  cuuint32_t box[3] = {(cuuint32_t)(tc::BK * 2 / esz), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = kind == kSliceTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : kind == kSliceFP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return enc(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             tc::BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__device__ __forceinline__ void slices_of(double x, int nsl, __nv_bfloat16 (&s)[3]) {
  float hi, lo;
  tc::f64_to_ff_fast(x, hi, lo);
  tc::ff_to_bf16x3(hi, lo, s[0], s[1], s[2]);
  if (nsl == 2) {
    // two slices: the second carries the rounded remainder of hi + lo
    float r = (hi - __bfloat162float(s[0])) + lo;
    s[1] = __float2bfloat16_rn(r);
  }
}

// Ut[s][pc][apad] from U[row][ci] (FP64 internal order).
__global__ void slice_ut_kernel(int nsl, int K, int K_pad, long long n_pad, const int* __restrict__ pc_int,
                                const double* __restrict__ U, PatchTable pt, int nwp, const long long* __restrict__ pad_off,
                                __nv_bfloat16* __restrict__ Ut) {
  long long total = (long long)K_pad * n_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int pc = (int)(e / n_pad);
    long long ap = e % n_pad;
    int g = 0;
    while (g + 1 < nwp && pad_off[g + 1] <= ap) ++g;
    long long a = ap - pad_off[g];
    __nv_bfloat16 s[3] = {__float2bfloat16_rn(0.f), __float2bfloat16_rn(0.f), __float2bfloat16_rn(0.f)};
    int ci = pc_int[pc];
    if (ci >= 0 && a < pt.nang[g]) slices_of(U[(pt.ang_off[g] + a) * K + ci], nsl, s);
    for (int k = 0; k < nsl; ++k) Ut[(long long)k * total + e] = s[k];
  }
}

// Qs[s][row][pc] from W[row][ci] (Q, or U for the adjoint).  With zero_mono
// the monopole column (natural column 0) is left zero: the synthesis epilogue
// adds -G M[i][0] for it.
__global__ void slice_q_kernel(int nsl, int K, int K_pad, long long rows, const int* __restrict__ pc_int,
                               const int* __restrict__ pc_nat, const double* __restrict__ Q, int zero_mono,
                               __nv_bfloat16* __restrict__ Qs) {
  long long total = rows * K_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long row = e / K_pad;
    int pc = (int)(e % K_pad);
    __nv_bfloat16 s[3] = {__float2bfloat16_rn(0.f), __float2bfloat16_rn(0.f), __float2bfloat16_rn(0.f)};
    int ci = pc_int[pc];
    if (ci >= 0 && (!zero_mono || pc_nat[pc] != 0)) slices_of(Q[row * K + ci], nsl, s);
    for (int k = 0; k < nsl; ++k) Qs[(long long)k * total + e] = s[k];
  }
}

// ---- TF32 slices (two per value, 22 significant bits; FP32's exponent range, no scaling) ----
// hi = tf32(head), lo = tf32((head - hi) + tail) of a float-float value.
__device__ __forceinline__ void ff_tf32(float h, float l, float& s0, float& s1) {
  s0 = tc::to_tf32(h);
  s1 = tc::to_tf32((h - s0) + l);
}
__device__ __forceinline__ void tf32_slices_of(double x, float& s0, float& s1) {
  float h, l;
  tc::f64_to_ff_fast(x, h, l);
  ff_tf32(h, l, s0, s1);
}

// Ut[s][pc][apad] (TF32) from U[row][ci] (FP64 internal order), as slice_ut_kernel.
__global__ void slice_ut_tf32_kernel(int K, int K_pad, long long n_pad, const int* __restrict__ pc_int,
                                     const double* __restrict__ U, PatchTable pt, int nwp,
                                     const long long* __restrict__ pad_off, float* __restrict__ Ut) {
  long long total = (long long)K_pad * n_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int pc = (int)(e / n_pad);
    long long ap = e % n_pad;
    int g = 0;
    while (g + 1 < nwp && pad_off[g + 1] <= ap) ++g;
    long long a = ap - pad_off[g];
    float s0 = 0.0f, s1 = 0.0f;
    int ci = pc_int[pc];
    if (ci >= 0 && a < pt.nang[g]) tf32_slices_of(U[(pt.ang_off[g] + a) * K + ci], s0, s1);
    Ut[e] = s0;
    Ut[total + e] = s1;
  }
}

// Qs[s][row][pc] (TF32) from W[row][ci], as slice_q_kernel (zero_mono: the monopole column stays zero).
__global__ void slice_q_tf32_kernel(int K, int K_pad, long long rows, const int* __restrict__ pc_int,
                                    const int* __restrict__ pc_nat, const double* __restrict__ Q, int zero_mono,
                                    float* __restrict__ Qs) {
  long long total = rows * K_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long row = e / K_pad;
    int pc = (int)(e % K_pad);
    float s0 = 0.0f, s1 = 0.0f;
    int ci = pc_int[pc];
    if (ci >= 0 && (!zero_mono || pc_nat[pc] != 0)) tf32_slices_of(Q[row * K + ci], s0, s1);
    Qs[e] = s0;
    Qs[total + e] = s1;
  }
}

// Field slices.  Symmetric: sigma+- = rho_Yin +- rho_Yang in float-float, then
// sliced; otherwise every patch's rho is sliced into its padded column range.
// Grid: (x over angular cells in steps of 2 per thread, y over shells, z over
// stored patches); each thread handles two neighbouring cells (16-byte loads,
// 4-byte stores).
__device__ __forceinline__ void ff_slices(float hi, float lo, int nsl, __nv_bfloat16 (&sl)[3]) {
  tc::ff_to_bf16x3(hi, lo, sl[0], sl[1], sl[2]);
  if (nsl == 2) sl[1] = __float2bfloat16_rn((hi - __bfloat162float(sl[0])) + lo);
}

__device__ __forceinline__ void sigma_slices(double r0, double r1, int nsl, int symmetric,
                                             __nv_bfloat16 (&out)[2][3]) {
  float h0, l0;
  tc::f64_to_ff_fast(r0, h0, l0);
  if (!symmetric) {
    ff_slices(h0, l0, nsl, out[0]);
    return;
  }
  float h1, l1;
  tc::f64_to_ff_fast(r1, h1, l1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float s, err;
    tc::two_sum(h0, h ? -h1 : h1, s, err);
    float lo = err + (h ? (l0 - l1) : (l0 + l1));
    float hi = s + lo;  // renormalise
    lo = lo - (hi - s);
    ff_slices(hi, lo, nsl, out[h]);
  }
}

// Grid: (x over groups of 4 angular cells, y over shells, z over stored
// patches).  Rows of rho whose start is 16-byte aligned are read with 16-byte
// loads; slices are written 4 cells (8 bytes) at a time.
#if YGS_DEBUG_BOUNDS
// Checked builds: cells [a, a + nv) of both input rows lie in the field and
// those of every output plane in the slice buffer (planes x plane elements).
__device__ __forceinline__ bool field_row_ok(long long in0, long long in1, long long n_cells, long long out,
                                             long long planes, long long plane, int nv) {
  return YGS_IN_BOUNDS(in0, n_cells, kSiteFieldSlicesRho) && YGS_IN_BOUNDS(in0 + nv - 1, n_cells, kSiteFieldSlicesRho) &&
         YGS_IN_BOUNDS(in1, n_cells, kSiteFieldSlicesRho) && YGS_IN_BOUNDS(in1 + nv - 1, n_cells, kSiteFieldSlicesRho) &&
         YGS_IN_BOUNDS(out, planes * plane, kSiteFieldSlicesOut) &&
         YGS_IN_BOUNDS((planes - 1) * plane + out + nv - 1, planes * plane, kSiteFieldSlicesOut);
}
#endif

__device__ __forceinline__ void field_slices_kernel_body(const tc::VBlock& vb, int nsl, int n_r, int symmetric, const PatchTable& pt,
                                    const long long* __restrict__ pad_off, long long n_pad,
                                    const double* __restrict__ rho, __nv_bfloat16* __restrict__ F) {
  const long long plane = (long long)n_r * n_pad;
  const int g = vb.z;
  const int i = vb.y;
  const int na = (int)pt.nang[g];
  const long long row_in = pt.fld_off[g] + (long long)i * na;
  const long long row_in1 = symmetric ? pt.fld_off[1] + (long long)i * na : row_in;
  const long long row_out = (long long)i * n_pad + (symmetric ? 0 : pad_off[g]);
  const bool vec = ((row_in | row_in1) & 1) == 0;
  for (int a = 4 * (vb.x * blockDim.x + threadIdx.x); a < na; a += 4 * vb.gx * blockDim.x) {
#if YGS_DEBUG_BOUNDS
    if (!field_row_ok(row_in + a, row_in1 + a, pt.n_cells, row_out + a, (long long)(symmetric ? 2 : 1) * nsl, plane,
                      min(4, na - a)))
      continue;
#endif
    double v0[4], v1[4];
    if (vec && a + 4 <= na) {
      const double2 x0 = *reinterpret_cast<const double2*>(rho + row_in + a);
      const double2 x1 = *reinterpret_cast<const double2*>(rho + row_in + a + 2);
      v0[0] = x0.x; v0[1] = x0.y; v0[2] = x1.x; v0[3] = x1.y;
      if (symmetric) {
        const double2 y0 = *reinterpret_cast<const double2*>(rho + row_in1 + a);
        const double2 y1 = *reinterpret_cast<const double2*>(rho + row_in1 + a + 2);
        v1[0] = y0.x; v1[1] = y0.y; v1[2] = y1.x; v1[3] = y1.y;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        v0[c] = (a + c < na) ? rho[row_in + a + c] : 0.0;
        v1[c] = (symmetric && a + c < na) ? rho[row_in1 + a + c] : 0.0;
      }
    }
    __nv_bfloat16 out[4][2][3];
#pragma unroll
    for (int c = 0; c < 4; ++c) sigma_slices(v0[c], v1[c], nsl, symmetric, out[c]);
    const int nh = symmetric ? 2 : 1;
    const bool whole = a + 4 <= na;
    for (int h = 0; h < nh; ++h)
      for (int k = 0; k < nsl; ++k) {
        __nv_bfloat16* dst = F + (long long)(h * nsl + k) * plane + row_out + a;
        if (whole) {
          __nv_bfloat162 p0, p1;
          p0.x = out[0][h][k];
          p0.y = out[1][h][k];
          p1.x = out[2][h][k];
          p1.y = out[3][h][k];
          uint2 w;
          w.x = *reinterpret_cast<unsigned int*>(&p0);
          w.y = *reinterpret_cast<unsigned int*>(&p1);
          *reinterpret_cast<uint2*>(dst) = w;
        } else {
          for (int c = 0; c < 4 && a + c < na; ++c) dst[c] = out[c][h][k];
        }
      }
  }
}
__global__ void __launch_bounds__(128) field_slices_kernel(int nsl, int n_r, int symmetric, PatchTable pt,
                                    const long long* __restrict__ pad_off, long long n_pad,
                                    const double* __restrict__ rho, __nv_bfloat16* __restrict__ F) {
  field_slices_kernel_body(tc::vblock_self(), nsl, n_r, symmetric, pt, pad_off, n_pad, rho, F);
}

// The arguments of field_slices_kernel but the field, for a grouped launch.
struct FieldSlicesArgs {
  int nsl;
  int n_r;
  int symmetric;
  PatchTable pt;
  const long long* pad_off;
  long long n_pad;
  __nv_bfloat16* F;
};

// field_slices_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(128) field_slices_kernel_group(const FieldSlicesArgs* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n, const __grid_constant__ tc::RhoList rhos) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const FieldSlicesArgs& a = probs[k];
  const double* rho = rhos.p[k];
  field_slices_kernel_body(vb, a.nsl, a.n_r, a.symmetric, a.pt, a.pad_off, a.n_pad, rho, a.F);
}


// sigma+- (or rho) of one cell as float-float pairs from the two values'
// float-float forms (TwoSum of the heads, renormalised), as sigma_slices.
__device__ __forceinline__ void sigma_ff2(double r0, double r1, int symmetric, float (&hi)[2], float (&lo)[2]) {
  float h0, l0;
  tc::f64_to_ff_fast(r0, h0, l0);
  if (!symmetric) {
    hi[0] = h0;
    lo[0] = l0;
    hi[1] = lo[1] = 0.0f;
    return;
  }
  float h1, l1;
  tc::f64_to_ff_fast(r1, h1, l1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float s, err;
    tc::two_sum(h0, h ? -h1 : h1, s, err);
    float l = err + (h ? (l0 - l1) : (l0 + l1));
    float hh = s + l;  // renormalise
    lo[h] = l - (hh - s);
    hi[h] = hh;
  }
}

// TF32 field slices, organised like field_slices_kernel: 4 cells per thread,
// 16-byte loads where the rows allow, one 16-byte store per plane and slice.
__device__ __forceinline__ void field_slices_tf32_kernel_body(const tc::VBlock& vb, int n_r, int symmetric, const PatchTable& pt, const long long* __restrict__ pad_off,
                                         long long n_pad, const double* __restrict__ rho, float* __restrict__ F) {
  const long long plane = (long long)n_r * n_pad;
  const int g = vb.z;
  const int i = vb.y;
  const int na = (int)pt.nang[g];
  const long long row_in = pt.fld_off[g] + (long long)i * na;
  const long long row_in1 = symmetric ? pt.fld_off[1] + (long long)i * na : row_in;
  const long long row_out = (long long)i * n_pad + (symmetric ? 0 : pad_off[g]);
  const bool vec = ((row_in | row_in1) & 1) == 0;
  for (int a = 4 * (vb.x * blockDim.x + threadIdx.x); a < na; a += 4 * vb.gx * blockDim.x) {
#if YGS_DEBUG_BOUNDS
    if (!field_row_ok(row_in + a, row_in1 + a, pt.n_cells, row_out + a, (long long)(symmetric ? 2 : 1) * 2, plane,
                      min(4, na - a)))
      continue;
#endif
    double v0[4], v1[4];
    if (vec && a + 4 <= na) {
      const double2 x0 = *reinterpret_cast<const double2*>(rho + row_in + a);
      const double2 x1 = *reinterpret_cast<const double2*>(rho + row_in + a + 2);
      v0[0] = x0.x; v0[1] = x0.y; v0[2] = x1.x; v0[3] = x1.y;
      if (symmetric) {
        const double2 y0 = *reinterpret_cast<const double2*>(rho + row_in1 + a);
        const double2 y1 = *reinterpret_cast<const double2*>(rho + row_in1 + a + 2);
        v1[0] = y0.x; v1[1] = y0.y; v1[2] = y1.x; v1[3] = y1.y;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        v0[c] = (a + c < na) ? rho[row_in + a + c] : 0.0;
        v1[c] = (symmetric && a + c < na) ? rho[row_in1 + a + c] : 0.0;
      }
    }
    float sl[2][2][4];  // [plane][slice][cell]
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float hi[2], lo[2];
      sigma_ff2(v0[c], v1[c], symmetric, hi, lo);
#pragma unroll
      for (int h = 0; h < 2; ++h) ff_tf32(hi[h], lo[h], sl[h][0][c], sl[h][1][c]);
    }
    const int nh = symmetric ? 2 : 1;
    for (int h = 0; h < nh; ++h)
      for (int k = 0; k < 2; ++k) {
        float* dst = F + (long long)(h * 2 + k) * plane + row_out + a;
        if (a + 4 <= na) {
          *reinterpret_cast<float4*>(dst) = make_float4(sl[h][k][0], sl[h][k][1], sl[h][k][2], sl[h][k][3]);
        } else {
          for (int c = 0; c < 4 && a + c < na; ++c) dst[c] = sl[h][k][c];
        }
      }
  }
}
__global__ void __launch_bounds__(128) field_slices_tf32_kernel(int n_r, int symmetric, PatchTable pt, const long long* __restrict__ pad_off,
                                         long long n_pad, const double* __restrict__ rho, float* __restrict__ F) {
  field_slices_tf32_kernel_body(tc::vblock_self(), n_r, symmetric, pt, pad_off, n_pad, rho, F);
}

// The arguments of field_slices_tf32_kernel but the field, for a grouped launch.
struct FieldSlicesTf32Args {
  int n_r;
  int symmetric;
  PatchTable pt;
  const long long* pad_off;
  long long n_pad;
  float* F;
};

// field_slices_tf32_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(128) field_slices_tf32_kernel_group(const FieldSlicesTf32Args* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n, const __grid_constant__ tc::RhoList rhos) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const FieldSlicesTf32Args& a = probs[k];
  const double* rho = rhos.p[k];
  field_slices_tf32_kernel_body(vb, a.n_r, a.symmetric, a.pt, a.pad_off, a.n_pad, rho, a.F);
}


// ---- FP16 slices (two per value, 22 significant bits) of power-of-two-scaled rows ----

__device__ __forceinline__ void half2_slices(double v, __half& s0, __half& s1) {
  s0 = __double2half(v);
  s1 = __double2half(v - (double)__half2float(s0));
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
  const int w = threadIdx.x / 32, nw = blockDim.x / 32;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  T r = red[0];
  for (int k = 1; k < nw; ++k) r = max(r, red[k]);
  return r;
}

// eu[pc] for the row pc of U^T (column ci of U) over every stored cell; one CTA per padded column.
__global__ void colexp_u_kernel(int K, const int* __restrict__ pc_int, long long rows, const double* __restrict__ U,
                                int* __restrict__ eu) {
  __shared__ double red[32];
  const int pc = blockIdx.x, ci = pc_int[pc];
  double m = 0.0;
  if (ci >= 0)
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) m = fmax(m, fabs(U[r * K + ci]));
  m = block_max(m, red);
  if (threadIdx.x == 0) eu[pc] = tc::fp16_row_exp(m);
}

// Ut[s][pc][apad]: slices of U^T rows scaled by 2^eu[pc].
// With zero_mono, padded column 0 (the monopole, whose moment the field pass
// computes exactly) is left zero.
__global__ void slice_ut16_kernel(int K, int K_pad, long long n_pad, const int* __restrict__ pc_int,
                                  const double* __restrict__ U, PatchTable pt, int nwp,
                                  const long long* __restrict__ pad_off, const int* __restrict__ eu, int zero_mono,
                                  __half* __restrict__ Ut) {
  long long total = (long long)K_pad * n_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int pc = (int)(e / n_pad);
    long long ap = e % n_pad;
    int g = 0;
    while (g + 1 < nwp && pad_off[g + 1] <= ap) ++g;
    long long a = ap - pad_off[g];
    double v = 0.0;
    int ci = pc_int[pc];
    if (ci >= 0 && a < pt.nang[g] && !(zero_mono && pc == 0)) v = ldexp(U[(pt.ang_off[g] + a) * K + ci], eu[pc]);
    __half s0, s1;
    half2_slices(v, s0, s1);
    Ut[e] = s0;
    Ut[total + e] = s1;
  }
}

// u00[ap] = U[row][ci0] (the monopole weight of the stored cell at padded
// angular index ap) as a float-float pair; zero in the padding.
__global__ void u00_kernel(int K, int ci0, long long n_pad, PatchTable pt, int nwp,
                           const long long* __restrict__ pad_off, const double* __restrict__ U,
                           float2* __restrict__ u00) {
  for (long long ap = blockIdx.x * (long long)blockDim.x + threadIdx.x; ap < n_pad;
       ap += (long long)gridDim.x * blockDim.x) {
    int g = 0;
    while (g + 1 < nwp && pad_off[g + 1] <= ap) ++g;
    const long long a = ap - pad_off[g];
    float h = 0.0f, l = 0.0f;
    if (a < pt.nang[g]) tc::f64_to_ff(U[(pt.ang_off[g] + a) * K + ci0], h, l);
    u00[ap] = make_float2(h, l);
  }
}

// Largest |Q| over the real columns other than the monopole (bits of a positive double, atomically maxed).
__global__ void qmax_kernel(int K, int K_pad, long long rows, const int* __restrict__ pc_int,
                            const int* __restrict__ pc_nat, const double* __restrict__ Q, int skip_mono,
                            unsigned long long* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  const long long total = rows * K_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int pc = (int)(e % K_pad);
    const int ci = pc_int[pc];
    if (ci >= 0 && (!skip_mono || pc_nat[pc] != 0)) m = fmax(m, fabs(Q[(e / K_pad) * K + ci]));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Qs[s][row][pc]: slices of W * 2^eq (Q, or U for the adjoint); with
// zero_mono the monopole column stays zero.
__global__ void slice_q16_kernel(int K, int K_pad, long long rows, const int* __restrict__ pc_int,
                                 const int* __restrict__ pc_nat, const double* __restrict__ Q, int eq, int zero_mono,
                                 __half* __restrict__ Qs) {
  long long total = rows * K_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long row = e / K_pad;
    int pc = (int)(e % K_pad);
    int ci = pc_int[pc];
    double v = (ci >= 0 && (!zero_mono || pc_nat[pc] != 0)) ? ldexp(Q[row * K + ci], eq) : 0.0;
    __half s0, s1;
    half2_slices(v, s0, s1);
    Qs[e] = s0;
    Qs[total + e] = s1;
  }
}

// sigma+- (or rho) of one cell as float-float pairs: the exact sum and
// difference of the two values rounded to FP32 (TwoSum), so each is within
// 2^-24 (|rho_Yin| + |rho_Yang|) of the FP64 value, below the 2^-22 of the
// two FP16 slices it becomes.
__device__ __forceinline__ void sigma_ff(double r0, double r1, int symmetric, float (&hi)[2], float (&lo)[2]) {
  const float h0 = tc::f64_round_f32(r0);
  if (!symmetric) {
    hi[0] = h0;
    lo[0] = hi[1] = lo[1] = 0.0f;
    return;
  }
  const float h1 = tc::f64_round_f32(r1);
  tc::two_sum(h0, h1, hi[0], lo[0]);
  tc::two_sum(h0, -h1, hi[1], lo[1]);
}

// The FP16 field pass works on exponent groups of kGroup = 128 angular cells
// (two k-blocks, aligned to the padded layout, so never straddling a chunk or
// a patch): every (plane, group, shell) row of a group is scaled by its own
// power of two, and the projection applies the inverse at the flush that
// closes the group (its accumulator holds exactly one group's products).
constexpr int kGroup = 128;
constexpr int kF16Threads = 256;
#ifndef YGS_FIELD_BATCH
#define YGS_FIELD_BATCH 1
#endif
constexpr int kFieldBatch = YGS_FIELD_BATCH;  // exponent groups a warp loads at once
static_assert(kFieldBatch >= 1 && kFieldBatch <= 4, "field pass: 1 to 4 groups per warp step");

// Block sum of float-float partials (warp TwoSum tree, then warp 0's lane 0
// over the warps); the result is valid in thread 0.
__device__ __forceinline__ float2 block_ff_sum(float mh, float ml) {
  __shared__ float rh[32], rl[32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, mh, d), ol = __shfl_xor_sync(0xffffffffu, ml, d);
    float s2, e2;
    tc::two_sum(mh, oh, s2, e2);
    mh = s2;
    ml += ol + e2;
  }
  const int wid = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  if (lane == 0) {
    rh[wid] = mh;
    rl[wid] = ml;
  }
  __syncthreads();
  float h = 0.0f, l = 0.0f;
  if (threadIdx.x == 0) {
    for (int k = 0; k < nw; ++k) {
      float s2, e2;
      tc::two_sum(h, rh[k], s2, e2);
      h = s2;
      l += rl[k] + e2;
    }
  }
  return make_float2(h, l);
}

__device__ __forceinline__ uint32_t h2_bits(__half2 v) {
  uint32_t r;
  memcpy(&r, &v, sizeof(r));
  return r;
}

// Four consecutive values of a row (cells c .. c + 3 of n; zero past n), by
// two 16-byte loads where the row allows.
__device__ __forceinline__ void load4(const double* __restrict__ p, long long c, long long n, bool vec,
                                      double (&x)[4]) {
  if (vec && c + 4 <= n) {
    const double2 v0 = *reinterpret_cast<const double2*>(p + c);
    const double2 v1 = *reinterpret_cast<const double2*>(p + c + 2);
    x[0] = v0.x; x[1] = v0.y; x[2] = v1.x; x[3] = v1.y;
  } else {
#pragma unroll
    for (int d = 0; d < 4; ++d) x[d] = c + d < n ? p[c + d] : 0.0;
  }
}

// The exponent e that puts a group's largest |head| m into [2^14, 2^15),
// kept within FP32's normal range so that 2^e and 2^-e are single FP32
// factors (groups whose largest value is below 2^-111 keep fewer bits).
__device__ __forceinline__ int group_exp(float m) {
  const int e = tc::fp16_row_exp_f(m);
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Row length of the factor table: whole projection shell tiles, so that the
// contraction's TMA warp copies a tile's row (kNmaxProject floats) in bounds.
int fac_ld(const ygs_plan* p) { return (p->tc_np_full + (p->tc_np_tail > 0 ? 1 : 0)) * tc::kNmaxProject; }

// Field slices in FP16 in one pass over rho.  One CTA per (split-K chunk z,
// shell i); each warp takes whole exponent groups of the chunk, lane l the
// cells 4l .. 4l + 3 of a group.  Per group and plane: sigma+- (or rho) in
// float-float from the FP32-rounded values (sigma_ff), the largest |head| by a
// warp max, its exponent e, the two FP16 slices of sigma * 2^e (one 8-byte
// store per lane, plane and slice) and the factor 2^-e for the projection's
// flush in fac[h][G][i] (G: the group's index in the padded angular layout;
// rows of fac_ld floats).
// With u00 (forward solves), plane 0's sigma * u (the monopole weight) is
// summed in float-float per thread and reduced over the CTA into
// mpart[z][i]: the monopole moment of the chunk, exactly to float-float
// rounding.  Cells past the patch read as zero, so a group's padding is
// written as zero slices.
#ifndef YGS_F16_MINB
#define YGS_F16_MINB 4  // resident CTAs per SM the field pass's register budget is set for
#endif
// One exponent group of the FP16 field pass: lane l holds cells 4l .. 4l + 3
// of the group (x0: patch g or Yin, x1: Yang; zero past the patch) and the
// monopole weights of the same cells (ua, ub; zero without u00).
__device__ __forceinline__ void field16_group(const double (&x0)[4], const double (&x1)[4], float4 ua, float4 ub,
                                              bool mono, int symmetric, int lane, long long G, int i,
                                              long long ngroups_all, int fac_ld, float* __restrict__ fac,
                                              __half* __restrict__ out, long long plane, float& mh, float& ml,
                                              long long oidx = 0, long long f_len = 0) {
  // oidx, f_len: out's element index within the slice buffer and its length (the checked build's bounds)
  (void)oidx;
  (void)f_len;
  float hi[4][2], lo[4][2];
  float m0 = 0.0f, m1 = 0.0f;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    sigma_ff(x0[d], x1[d], symmetric, hi[d], lo[d]);
    m0 = fmaxf(m0, fabsf(hi[d][0]));
    m1 = fmaxf(m1, fabsf(hi[d][1]));
  }
  // non-negative floats order like their bit patterns
  m0 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m0)));
  m1 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m1)));
  const int e[2] = {group_exp(m0), symmetric ? group_exp(m1) : 0};
  if (lane < 2 && (lane == 0 || symmetric)) {
    const long long fi = ((long long)lane * ngroups_all + G) * fac_ld + i;
    if (YGS_IN_BOUNDS(fi, 2 * ngroups_all * fac_ld, kSiteField16Fac)) fac[fi] = pow2f(-e[lane]);
  }
  if (mono) {
    // sigma+ times the weight in float-float (padding cells carry sigma = 0):
    // the heads' product with its rounding error from an FMA, the tails'
    // cross terms, the running sum by FastTwoSum (exact while the sum
    // dominates, as it does for a positive density)
    const float uh[4] = {ua.x, ua.z, ub.x, ub.z}, ul[4] = {ua.y, ua.w, ub.y, ub.w};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const float pr = hi[d][0] * uh[d];
      const float pe = fmaf(hi[d][0], ul[d], fmaf(lo[d][0], uh[d], fmaf(hi[d][0], uh[d], -pr)));
      const float s2 = mh + pr;
      ml += (pr - (s2 - mh)) + pe;
      mh = s2;
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h == 1 && !symmetric) break;
    const float f = pow2f(e[h]);
    uint32_t w0[2], w1[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // both cells of a pair at once: s0 = fp16(a), s1 = fp16((a - s0) + b)
      const float a0 = hi[2 * u][h] * f, a1 = hi[2 * u + 1][h] * f;
      const float b0 = lo[2 * u][h] * f, b1 = lo[2 * u + 1][h] * f;
      const __half2 s0 = __floats2half2_rn(a0, a1);  // a0 in the low half
      const float2 back = __half22float2(s0);
      const __half2 s1 = __floats2half2_rn((a0 - back.x) + b0, (a1 - back.y) + b1);
      w0[u] = h2_bits(s0);
      w1[u] = h2_bits(s1);
    }
    if (YGS_IN_BOUNDS(oidx + (2 * h) * plane, f_len, kSiteField16Slices) &&
        YGS_IN_BOUNDS(oidx + (2 * h + 1) * plane + 3, f_len, kSiteField16Slices)) {
      *reinterpret_cast<uint2*>(out + (long long)(2 * h) * plane) = make_uint2(w0[0], w0[1]);
      *reinterpret_cast<uint2*>(out + (long long)(2 * h + 1) * plane) = make_uint2(w1[0], w1[1]);
    }
  }
}

__device__ __forceinline__ void field16_kernel_body(const tc::VBlock& vb, 
    int n_r, int symmetric, int nwp, const PatchTable& pt, const long long* __restrict__ pad_off, long long n_pad,
    const int2* __restrict__ chunks, const double* __restrict__ rho, __half* __restrict__ F,
    float* __restrict__ fac, int fac_ld, const float2* __restrict__ u00, float2* __restrict__ mpart) {
  const int z = vb.x, i = vb.y;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const long long plane = (long long)n_r * n_pad;
  const long long ngroups_all = n_pad / kGroup;
  const int2 ch = chunks[z];
  int g = 0;
  while (g + 1 < nwp && pad_off[g + 1] <= ch.x) ++g;
  const long long na = pt.nang[g];
  const double* x0p = rho + pt.fld_off[g] + (long long)i * na;
  const double* x1p = symmetric ? rho + pt.fld_off[1] + (long long)i * na : x0p;
  const bool vec = ((reinterpret_cast<uintptr_t>(x0p) | reinterpret_cast<uintptr_t>(x1p)) & 15) == 0;
  const long long c_chunk = ch.x - pad_off[g];  // first cell of the chunk within patch g (a multiple of kGroup)
  const int ngroups = (ch.y - ch.x) / kGroup;
  const float2* const uz = u00 ? u00 + pad_off[g] : nullptr;
  float mh = 0.0f, ml = 0.0f;
  // kFieldBatch groups per warp step, their loads issued together (more bytes
  // in flight per warp: the pass is bound by memory latency, not issue)
  for (int q0 = warp; q0 < ngroups; q0 += kFieldBatch * nw) {
    double x0[kFieldBatch][4], x1[kFieldBatch][4];
    float4 ua[kFieldBatch], ub[kFieldBatch];
#pragma unroll
    for (int b = 0; b < kFieldBatch; ++b) {
      const int q = q0 + b * nw;
      const long long c = c_chunk + (long long)q * kGroup + 4 * lane;  // this lane's first cell in patch g
      bool live = q < ngroups;
#if YGS_DEBUG_BOUNDS
      {
        // the first and last cell this lane reads of either row, within the field
        const long long nv = na - c < 4 ? na - c : 4, r0 = pt.fld_off[g] + (long long)i * na + c;
        const long long r1 = (symmetric ? pt.fld_off[1] : pt.fld_off[g]) + (long long)i * na + c;
        if (live && nv > 0)
          live = YGS_IN_BOUNDS(r0, pt.n_cells, kSiteField16Rho) && YGS_IN_BOUNDS(r0 + nv - 1, pt.n_cells, kSiteField16Rho) &&
                 YGS_IN_BOUNDS(r1, pt.n_cells, kSiteField16Rho) && YGS_IN_BOUNDS(r1 + nv - 1, pt.n_cells, kSiteField16Rho);
        if (live && uz) live = YGS_IN_BOUNDS(pad_off[g] + c + 3, n_pad, kSiteField16U00);
      }
#endif
      load4(x0p, c, live ? na : 0, vec, x0[b]);
      load4(x1p, c, (live && symmetric) ? na : 0, vec, x1[b]);
      // the monopole weights of the same cells (padded layout, zero in the padding)
      ua[b] = (uz && live) ? *reinterpret_cast<const float4*>(uz + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      ub[b] = (uz && live) ? *reinterpret_cast<const float4*>(uz + c + 2) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < kFieldBatch; ++b) {
      const int q = q0 + b * nw;
      if (q >= ngroups) break;  // warp-uniform
      const long long c = c_chunk + (long long)q * kGroup + 4 * lane;
      // 8-byte aligned: pad_off, c multiples of 4
      const long long oidx = (long long)i * n_pad + pad_off[g] + c;
      field16_group(x0[b], x1[b], ua[b], ub[b], uz != nullptr, symmetric, lane, (ch.x / kGroup) + q, i, ngroups_all,
                    fac_ld, fac, F + oidx, plane, mh, ml, oidx, (symmetric ? 4 : 2) * plane);
    }
  }
  if (!mpart) return;
  const float2 m = block_ff_sum(mh, ml);
  if (threadIdx.x == 0) mpart[(long long)z * n_r + i] = m;
}
__global__ void __launch_bounds__(kF16Threads, YGS_F16_MINB) field16_kernel(
    int n_r, int symmetric, int nwp, PatchTable pt, const long long* __restrict__ pad_off, long long n_pad,
    const int2* __restrict__ chunks, const double* __restrict__ rho, __half* __restrict__ F,
    float* __restrict__ fac, int fac_ld, const float2* __restrict__ u00, float2* __restrict__ mpart) {
  field16_kernel_body(tc::vblock_self(), n_r, symmetric, nwp, pt, pad_off, n_pad, chunks, rho, F, fac, fac_ld, u00, mpart);
}

// The arguments of field16_kernel but the field, for a grouped launch.
struct Field16Args {
  int n_r;
  int symmetric;
  int nwp;
  PatchTable pt;
  const long long* pad_off;
  long long n_pad;
  const int2* chunks;
  __half* F;
  float* fac;
  int fac_ld;
  const float2* u00;
  float2* mpart;
};

// field16_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(kF16Threads, YGS_F16_MINB) field16_kernel_group(const Field16Args* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n, const __grid_constant__ tc::RhoList rhos) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const Field16Args& a = probs[k];
  const double* rho = rhos.p[k];
  field16_kernel_body(vb, a.n_r, a.symmetric, a.nwp, a.pt, a.pad_off, a.n_pad, a.chunks, rho, a.F, a.fac, a.fac_ld, a.u00, a.mpart);
}



// Ms[s][i][pc]: FP16 slices of M's row i scaled by 2^em[i] (largest |M| over the
// row; without keep_mono the monopole, padded column 0, whose Q column is
// zero, is left out and written as 0; padded columns hold zeros).  One CTA per
// shell, a pair of adjacent columns per thread step (16-byte loads, 4-byte
// stores); FP64 values enter as float-float pairs.  Also writes the synthesis
// epilogue's per-shell constants sc[i].
constexpr int kSliceM16Threads = 256;
__device__ __forceinline__ void slice_m16_kernel_body(const tc::VBlock& vb, 
    int n_r, int K_pad, const float2* __restrict__ M, int keep_mono, __half* __restrict__ Ms, int* __restrict__ em,
    int q_exp, const float2* __restrict__ mono, float4* __restrict__ sc) {
  __shared__ float red[32];
  const int i = vb.x, npair = K_pad / 2;  // K_pad is a multiple of 64
  const long long splane = (long long)n_r * K_pad;
  const float4* row = reinterpret_cast<const float4*>(M + (long long)i * K_pad);  // two float-float columns each
  // (a CTA-uniform test: the whole row is in, or the CTA leaves before its reduction)
  if (!YGS_IN_BOUNDS((long long)i * K_pad, splane, kSiteSliceM16In) ||
      !YGS_IN_BOUNDS((long long)i * K_pad + K_pad - 1, splane, kSiteSliceM16In) ||
      !YGS_IN_BOUNDS(splane + (long long)i * K_pad + K_pad - 1, 2 * splane, kSiteSliceM16Out))
    return;
  float m = 0.0f;
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    const float4 v = row[q];
    const float a = (q == 0 && !keep_mono) ? 0.0f : fabsf(v.x);
    m = fmaxf(m, fmaxf(a, fabsf(v.z)));
  }
  // the largest head bounds every head below
  const int e = tc::fp16_row_exp_f(block_max(m, red));
  if (threadIdx.x == 0) {
    em[i] = e;
    // the synthesis epilogue's per-shell constants: the exponent rebase that
    // unscales its results as they are widened to FP64, and the monopole pair
    // brought into the scaled units
    float f1, f2;
    tc::pow2_pair(q_exp + e, f1, f2);
    const float2 mm = mono ? mono[i] : make_float2(0.0f, 0.0f);
    sc[i] = make_float4(__int_as_float((896 - (q_exp + e)) * (1 << 20)), 0.0f, (mm.x * f1) * f2, (mm.y * f1) * f2);
  }
  float f1, f2;
  tc::pow2_pair(e, f1, f2);
  uint32_t* out0 = reinterpret_cast<uint32_t*>(Ms + (long long)i * K_pad);
  uint32_t* out1 = reinterpret_cast<uint32_t*>(Ms + splane + (long long)i * K_pad);
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    const float4 v = row[q];
    const bool skip = q == 0 && !keep_mono;
    const float h0 = skip ? 0.0f : v.x, l0 = skip ? 0.0f : v.y, h1 = v.z, l1 = v.w;
    const float a0 = (h0 * f1) * f2, a1 = (h1 * f1) * f2, b0 = (l0 * f1) * f2, b1 = (l1 * f1) * f2;
    const __half2 s0 = __floats2half2_rn(a0, a1);  // the pair's first column in the low half
    const float2 back = __half22float2(s0);
    const __half2 s1 = __floats2half2_rn((a0 - back.x) + b0, (a1 - back.y) + b1);
    out0[q] = h2_bits(s0);
    out1[q] = h2_bits(s1);
  }
}
__global__ void __launch_bounds__(kSliceM16Threads) slice_m16_kernel(
    int n_r, int K_pad, const float2* __restrict__ M, int keep_mono, __half* __restrict__ Ms, int* __restrict__ em,
    int q_exp, const float2* __restrict__ mono, float4* __restrict__ sc) {
  slice_m16_kernel_body(tc::vblock_self(), n_r, K_pad, M, keep_mono, Ms, em, q_exp, mono, sc);
}

// The arguments of slice_m16_kernel but the field, for a grouped launch.
struct SliceM16Args {
  int n_r;
  int K_pad;
  const float2* M;
  int keep_mono;
  __half* Ms;
  int* em;
  int q_exp;
  const float2* mono;
  float4* sc;
};

// slice_m16_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(kSliceM16Threads) slice_m16_kernel_group(const SliceM16Args* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const SliceM16Args& a = probs[k];
  slice_m16_kernel_body(vb, a.n_r, a.K_pad, a.M, a.keep_mono, a.Ms, a.em, a.q_exp, a.mono, a.sc);
}


// Products of the radial ratios over every chunk of shells (per degree l),
// as float-float:
// cp[0][l][p] = prod_{i in chunk p} (r_{i-1}^+/r_i^+)^(l+1),
// cp[1][l][p] = prod_{i in chunk p} (r_{i-1}^+/r_i^+)^l   (0 for chunks that contain shell 0).
__global__ void chunk_prod_kernel(int n_r, int L, int chunk, int P, const double* __restrict__ rad,
                                  float2* __restrict__ cp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (L + 1) * P) return;
  int l = t / P, p = t % P;
  const long long rs = (long long)(L + 1) * n_r;
  const double* fin = rad + 2 * rs + (long long)l * n_r;
  const double* fout = rad + 3 * rs + (long long)l * n_r;
  double a = 1.0, b = 1.0;
  for (int i = p * chunk; i < min(n_r, (p + 1) * chunk); ++i) {
    a *= fin[i];
    b *= (i > 0) ? fout[i - 1] : 0.0;
  }
  cp[(long long)l * P + p] = tc::ff_from_f64(a);
  cp[(long long)(L + 1) * P + (long long)l * P + p] = tc::ff_from_f64(b);
}

// The radial tables a, b, f_in, f_out ([4][L + 1][n_r]) as float-float.
__global__ void rad_ff_kernel(long long n, const double* __restrict__ rad, float2* __restrict__ radff) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    radff[e] = tc::ff_from_f64(rad[e]);
}

// Carries between chunks.  The chunk summaries define affine maps c -> F c + s;
// one warp per column and direction composes them: each lane folds up to 32
// consecutive chunks, this shuffle scan joins the lanes (inner recurrence
// upward, outer downward), and each lane walks its chunks again.
__device__ __forceinline__ float2 shfl_up_ff(float2 v, int d) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ void affine_scan_up(float2& F, float2& s, int lane) {
  // inclusive scan: after it lane p holds the composition of chunks 0..p
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float2 Fo = shfl_up_ff(F, d), so = shfl_up_ff(s, d);
    if (lane >= d) {
      s = tc::ff_fma(F, so, s);
      F = tc::ff_mul(F, Fo);
    }
  }
}

// Phase 2 of both scans: one warp composes column cc's chunk summaries
// upward (dir 0: sm[1] the factor, sm[0] the offset) or downward (dir 1:
// sm[3], sm[2]) and writes each chunk's incoming carry to cr[dir]; the CTA's
// warps take the 2 kCols (column, direction) tasks in turn.
template <int kCols, int kMaxP>
__device__ __forceinline__ void carry_scan_one(const float2 (&sm)[4][kMaxP][kCols], float2 (&cr)[2][kMaxP][kCols],
                                               int P, int cc, int dir, int lane) {
  const int q = (P + 31) / 32, t0 = lane * q, t1 = min(P, t0 + q);
  const int kF = dir ? 3 : 1, ks = dir ? 2 : 0;
  float2 F = make_float2(1.0f, 0.0f), sv = make_float2(0.0f, 0.0f);
  for (int t = t0; t < t1; ++t) {
    const int pp = dir ? P - 1 - t : t;
    sv = tc::ff_fma(sm[kF][pp][cc], sv, sm[ks][pp][cc]);
    F = tc::ff_mul(sm[kF][pp][cc], F);
  }
  affine_scan_up(F, sv, lane);
  float2 cin = shfl_up_ff(sv, 1);
  if (lane == 0) cin = make_float2(0.0f, 0.0f);
  for (int t = t0; t < t1; ++t) {
    const int pp = dir ? P - 1 - t : t;
    cr[dir][pp][cc] = cin;
    cin = tc::ff_fma(sm[kF][pp][cc], cin, sm[ks][pp][cc]);
  }
}

template <int kCols, int kMaxP>
__device__ __forceinline__ void carry_scan(const float2 (&sm)[4][kMaxP][kCols], float2 (&cr)[2][kMaxP][kCols],
                                           int P) {
  const int lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int w = threadIdx.x / 32; w < 2 * kCols; w += nw)  // a (column, direction) task per warp
    carry_scan_one<kCols, kMaxP>(sm, cr, P, w >> 1, w & 1, lane);
}

// The chunk partials of shell i, column pc summed over the chunks z in z
// order (TwoSum), as float-float; FP16 plans' partials are unscaled by the
// column's exponent first, and the monopole column of a forward FP16 solve
// takes the field pass's exact chunk sums instead.
// ... for the shells ib .. ib + G - 1 below i1 (zero for the others), with
// the loads of kScanZ chunks of every shell of the group issued together, so
// that a thread waits for one round trip per kScanZ chunks instead of one per
// chunk (each shell's sum keeps its z order and operations).
#ifndef YGS_SCAN_Z
#define YGS_SCAN_Z 1  // chunks per round of loads (more spill at the 64-register cap)
#endif
constexpr int kScanZ = YGS_SCAN_Z;
template <int G>
__device__ __forceinline__ void sum_chunks_group(const float2* __restrict__ part, long long plane, int S, int ib,
                                                 int i1, int K_pad, int pc, int escale,
                                                 const float2* __restrict__ mp, int n_r, float2 (&out)[G]) {
  float hh[G], ll[G];
#pragma unroll
  for (int k = 0; k < G; ++k) hh[k] = ll[k] = 0.0f;
  for (int z0 = 0; z0 < S; z0 += kScanZ) {
    float2 v[kScanZ][G];
#pragma unroll
    for (int zz = 0; zz < kScanZ; ++zz)
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const int z = z0 + zz, i = ib + k;
        v[zz][k] = make_float2(0.0f, 0.0f);
        if (z < S && i < i1) {
          const long long ix = mp ? (long long)z * n_r + i : z * plane + (long long)i * K_pad + pc;
          if (YGS_IN_BOUNDS(ix, mp ? (long long)S * n_r : S * plane, kSiteScanPart)) v[zz][k] = mp ? mp[ix] : part[ix];
        }
      }
#pragma unroll
    for (int zz = 0; zz < kScanZ; ++zz)
#pragma unroll
      for (int k = 0; k < G; ++k) {
        if (z0 + zz < S) {
          float2 w = v[zz][k];
          if (!mp && escale) {
            w.x = tc::mul_pow2f(w.x, -escale);
            w.y = tc::mul_pow2f(w.y, -escale);
          }
          float s, e;
          tc::two_sum(hh[k], w.x, s, e);
          hh[k] = s;
          ll[k] += e + w.y;
        }
      }
  }
#pragma unroll
  for (int k = 0; k < G; ++k) out[k] = ib + k < i1 ? tc::ff_renorm(hh[k], ll[k]) : make_float2(0.0f, 0.0f);
}

__device__ __forceinline__ void ff_slices(float2 v, int nsl, __nv_bfloat16 (&sl)[3]) {
  tc::ff_to_bf16x3(v.x, v.y, sl[0], sl[1], sl[2]);
  if (nsl == 2) sl[1] = __float2bfloat16_rn((v.x - __bfloat162float(sl[0])) + v.y);
}

// All three phases of the forward radial sums (Eq. M_C, step 4 of Sect. 4.3)
// in one launch, in float-float: a CTA owns kScanCols columns and up to
// kScanMaxP chunks of shells (thread = column + kScanCols * chunk), keeps the
// chunk summaries and carries in shared memory and separates the phases with
// block barriers (no CTA waits on another).  Phase 1: B from the projection's
// chunk partials (step 3), each chunk's recurrences with zero carry
//   I_i = a_i B_i + f_in,i I_{i-1},   O_i = b_i B_i + f_out,i-1 O_{i+1},
// and its summary (an affine map); phase 2: the carries, a scan of those
// maps; phase 3: the recurrences with the carries, M_i = I_i + O_{i+1}, its
// BF16 slices (BF16 plans) and the monopole -G M[i][0].
#ifndef YGS_SCAN_COLS
#define YGS_SCAN_COLS 2  // columns per scan CTA (256 threads: several CTAs share an SM and overlap their phases)
#endif
#ifndef YGS_SCAN_MAXP
#define YGS_SCAN_MAXP 128  // chunks of shells per column (a thread each)
#endif
constexpr int kScanCols = YGS_SCAN_COLS, kScanMaxP = YGS_SCAN_MAXP, kScanThreads = kScanCols * kScanMaxP;
constexpr int kScanGroup = 4;  // shells whose loads a thread issues together
// CTAs of a scan kernel resident per SM (4 of 256 threads at <= 64 registers
// hold K_pad / kScanCols = 576 CTAs of the 1-degree grid in one wave)
constexpr int kScanMinBlocks = 1024 / kScanThreads >= 1 ? 1024 / kScanThreads : 1;
static_assert(kScanCols >= 1 && kScanThreads <= 1024 && kScanThreads % 32 == 0 && kScanMaxP >= 32,
              "scan: a CTA of whole warps, at most 1024 threads, at least 32 chunks per column");

// A float-float store of the scans (B, M), index-checked in checked builds.
__device__ __forceinline__ void st_ff(float2* __restrict__ p, long long i, long long n, float2 v) {
  if (YGS_IN_BOUNDS(i, n, kSiteScanBM)) p[i] = v;
}

__device__ __forceinline__ void scan_ff_kernel_body(const tc::VBlock& vb, 
    int n_r, int K_pad, int L, int S, int chunk, int P, const int* __restrict__ pc_l, const float2* __restrict__ part,
    const float2* __restrict__ rad, const float2* __restrict__ cp, float2* __restrict__ B, float2* __restrict__ M,
    __nv_bfloat16* __restrict__ Ms, int nsl, int write_slices, float2 neg_G, float2* __restrict__ mono,
    const int* __restrict__ eu, const float2* __restrict__ mpart) {
  __shared__ float2 sm[4][kScanMaxP][kScanCols];
  __shared__ float2 cr[2][kScanMaxP][kScanCols];
  const float2 zero = make_float2(0.0f, 0.0f), one = make_float2(1.0f, 0.0f);
  const int c = threadIdx.x % kScanCols, p = threadIdx.x / kScanCols;
  const int pc = vb.x * kScanCols + c;
  const int l = pc < K_pad ? pc_l[pc] : -1;
  const int i0 = p * chunk, i1 = min(n_r, i0 + chunk);
  const bool live = l >= 0 && p < P && i0 < n_r;
  const long long plane = (long long)n_r * K_pad, rs = (long long)(L + 1) * n_r;
  const bool exact_mono = mpart && pc == 0;  // the monopole moment summed exactly by the field pass
  const int lq = l < 0 ? 0 : l;
  const float2* at = rad + (long long)lq * n_r;
  const float2* bt = rad + rs + (long long)lq * n_r;
  const float2* fin = rad + 2 * rs + (long long)lq * n_r;
  const float2* fout = rad + 3 * rs + (long long)lq * n_r;
  // ---- phase 1: B from the partials, local recurrences with zero carry, summaries
  float2 bb[kScanGroup];  // the chunk's B, kept for phase 3 when it is one group
  {
    float2 I = zero, Pv = zero, FI = one, FP = one;
    if (live) {
      const int escale = (eu && !exact_mono) ? eu[pc] : 0;
      for (int ib = i0; ib < i1; ib += kScanGroup) {
        float2 bg[kScanGroup];
        sum_chunks_group<kScanGroup>(part, plane, S, ib, i1, K_pad, pc, escale, exact_mono ? mpart : nullptr, n_r, bg);
#pragma unroll
        for (int k = 0; k < kScanGroup; ++k) {
          if (ib + k < i1) {
            const int i = ib + k;
            st_ff(B, (long long)i * K_pad + pc, plane, bg[k]);
            I = tc::ff_add(tc::ff_mul(at[i], bg[k]), tc::ff_mul(fin[i], I));
          }
          if (ib == i0) bb[k] = bg[k];
        }
      }
      if (i1 - i0 <= kScanGroup) {
#pragma unroll
        for (int k = kScanGroup - 1; k >= 0; --k) {
          if (k < i1 - i0) {
            const int i = i0 + k;
            const float2 fo = (i > 0) ? fout[i - 1] : zero;
            Pv = tc::ff_add(tc::ff_mul(bt[i], bb[k]), tc::ff_mul(fo, Pv));
          }
        }
      } else {
        for (int i = i1 - 1; i >= i0; --i) {
          const float2 fo = (i > 0) ? fout[i - 1] : zero;
          Pv = tc::ff_add(tc::ff_mul(bt[i], B[(long long)i * K_pad + pc]), tc::ff_mul(fo, Pv));
        }
      }
      FI = cp[(long long)l * P + p];
      FP = cp[(long long)(L + 1) * P + (long long)l * P + p];
    } else if (pc < K_pad && l < 0) {
      for (int i = i0; i < i1; ++i) st_ff(B, (long long)i * K_pad + pc, plane, zero);
    }
    if (p < kScanMaxP) {
      sm[0][p][c] = I;
      sm[1][p][c] = FI;
      sm[2][p][c] = Pv;
      sm[3][p][c] = FP;
    }
  }
  __syncthreads();
  // ---- phase 2: carries
  carry_scan<kScanCols, kScanMaxP>(sm, cr, P);
  __syncthreads();
  // ---- phase 3: the recurrences with the carries; M, its BF16 slices, the monopole
  if (pc >= K_pad || p >= P || i0 >= n_r) return;
  if (l < 0) {
    for (int i = i0; i < i1; ++i) {
      st_ff(M, (long long)i * K_pad + pc, plane, zero);
      if (write_slices == 2)
        for (int k = 0; k < 2; ++k) reinterpret_cast<float*>(Ms)[k * plane + (long long)i * K_pad + pc] = 0.0f;
      else if (write_slices)
        for (int k = 0; k < nsl; ++k) Ms[k * plane + (long long)i * K_pad + pc] = __float2bfloat16_rn(0.f);
    }
    return;
  }
  auto emit = [&](int i, float2 m) {
    st_ff(M, (long long)i * K_pad + pc, plane, m);
    if (pc == 0) mono[i] = tc::ff_mul(neg_G, m);  // natural column 0 (l = 0) is padded column 0: the monopole
    if (write_slices == 2) {  // TF32 slices (4-byte elements)
      float s0, s1;
      ff_tf32(m.x, m.y, s0, s1);
      float* Mf = reinterpret_cast<float*>(Ms);
      if (YGS_IN_BOUNDS(plane + (long long)i * K_pad + pc, 2 * plane, kSiteScanMs)) {
        Mf[(long long)i * K_pad + pc] = s0;
        Mf[plane + (long long)i * K_pad + pc] = s1;
      }
    } else if (write_slices) {
      __nv_bfloat16 sl[3];
      ff_slices(m, nsl, sl);
#pragma unroll
      for (int k = 0; k < 3; ++k)  // constant indices keep sl in registers
        if (k < nsl && YGS_IN_BOUNDS(k * plane + (long long)i * K_pad + pc, nsl * plane, kSiteScanMs))
          Ms[k * plane + (long long)i * K_pad + pc] = sl[k];
    }
  };
  float2 Pv = cr[1][p][c];
  float2 I = cr[0][p][c];
  if (i1 - i0 <= kScanGroup) {
    // the chunk's B and outer sums in registers; M written once
    float2 pv[kScanGroup];
#pragma unroll
    for (int k = kScanGroup - 1; k >= 0; --k) {
      pv[k] = Pv;
      if (k < i1 - i0) {
        const int i = i0 + k;
        const float2 fo = (i > 0) ? fout[i - 1] : zero;
        Pv = tc::ff_add(tc::ff_mul(bt[i], bb[k]), tc::ff_mul(fo, Pv));
      }
    }
#pragma unroll
    for (int k = 0; k < kScanGroup; ++k) {
      if (k < i1 - i0) {
        const int i = i0 + k;
        I = tc::ff_add(tc::ff_mul(at[i], bb[k]), tc::ff_mul(fin[i], I));
        emit(i, tc::ff_add(pv[k], I));
      }
    }
    return;
  }
  for (int i = i1 - 1; i >= i0; --i) {
    st_ff(M, (long long)i * K_pad + pc, plane, Pv);
    const float2 fo = (i > 0) ? fout[i - 1] : zero;
    Pv = tc::ff_add(tc::ff_mul(bt[i], B[(long long)i * K_pad + pc]), tc::ff_mul(fo, Pv));
  }
  for (int i = i0; i < i1; ++i) {
    I = tc::ff_add(tc::ff_mul(at[i], B[(long long)i * K_pad + pc]), tc::ff_mul(fin[i], I));
    emit(i, tc::ff_add(M[(long long)i * K_pad + pc], I));
  }
}
__global__ void __launch_bounds__(kScanThreads, kScanMinBlocks) scan_ff_kernel(
    int n_r, int K_pad, int L, int S, int chunk, int P, const int* __restrict__ pc_l, const float2* __restrict__ part,
    const float2* __restrict__ rad, const float2* __restrict__ cp, float2* __restrict__ B, float2* __restrict__ M,
    __nv_bfloat16* __restrict__ Ms, int nsl, int write_slices, float2 neg_G, float2* __restrict__ mono,
    const int* __restrict__ eu, const float2* __restrict__ mpart) {
  scan_ff_kernel_body(tc::vblock_self(), n_r, K_pad, L, S, chunk, P, pc_l, part, rad, cp, B, M, Ms, nsl, write_slices, neg_G, mono, eu, mpart);
}

// The arguments of scan_ff_kernel but the field, for a grouped launch.
struct ScanFfArgs {
  int n_r;
  int K_pad;
  int L;
  int S;
  int chunk;
  int P;
  const int* pc_l;
  const float2* part;
  const float2* rad;
  const float2* cp;
  float2* B;
  float2* M;
  __nv_bfloat16* Ms;
  int nsl;
  int write_slices;
  float2 neg_G;
  float2* mono;
  const int* eu;
  const float2* mpart;
};

// scan_ff_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(kScanThreads, kScanMinBlocks) scan_ff_kernel_group(const ScanFfArgs* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const ScanFfArgs& a = probs[k];
  scan_ff_kernel_body(vb, a.n_r, a.K_pad, a.L, a.S, a.chunk, a.P, a.pc_l, a.part, a.rad, a.cp, a.B, a.M, a.Ms, a.nsl, a.write_slices, a.neg_G, a.mono, a.eu, a.mpart);
}


// ---- adjoint scans (transposes of the recurrences above) ----
// With Mbar the adjoint of M, the transposed recurrences are
//   X_i = Mbar_i + fin_{i+1} X_{i+1}      (downward; X_{Nr} = 0)
//   Z_i = Mbar_i + fout_{i-1} Z_{i-1}     (upward; Z_{-1} = 0, fout_{-1} = 0)
//   Bbar_i = a_i X_i + b_i Z_{i-1},
// chunked like the forward scans: the summaries [0] Z at the chunk's end and
// [1] the product of its fout factors (upward), [2] X at its start and [3] the
// product of its fin factors (downward), all with zero carry, are composed by
// the same carry scan, in float-float like the forward scan.
__global__ void __launch_bounds__(kScanThreads, kScanMinBlocks) scan_adj_ff_kernel(
    int n_r, int K_pad, int L, int S, int chunk, int P, const int* __restrict__ pc_l, const float2* __restrict__ part,
    const float2* __restrict__ rad, float2* __restrict__ Mbar, float2* __restrict__ Bbar,
    __nv_bfloat16* __restrict__ Bs, int nsl, int write_slices, const int* __restrict__ ew) {
  __shared__ float2 sm[4][kScanMaxP][kScanCols];
  __shared__ float2 cr[2][kScanMaxP][kScanCols];
  const float2 zero = make_float2(0.0f, 0.0f), one = make_float2(1.0f, 0.0f);
  const int c = threadIdx.x % kScanCols, p = threadIdx.x / kScanCols;
  const int pc = blockIdx.x * kScanCols + c;
  const int l = pc < K_pad ? pc_l[pc] : -1;
  const int i0 = p * chunk, i1 = min(n_r, i0 + chunk);
  const bool live = l >= 0 && p < P && i0 < n_r;
  const long long plane = (long long)n_r * K_pad, rs = (long long)(L + 1) * n_r;
  const int lq = l < 0 ? 0 : l;
  const float2* at = rad + (long long)lq * n_r;
  const float2* bt = rad + rs + (long long)lq * n_r;
  const float2* fin = rad + 2 * rs + (long long)lq * n_r;
  const float2* fout = rad + 3 * rs + (long long)lq * n_r;
  // ---- phase 1: Mbar from the partials, chains with zero carry, summaries
  float2 mg[kScanGroup];  // the chunk's Mbar, kept for phase 3 when it is one group
  {
    float2 Z = zero, FZ = one, X = zero, FX = one;
    if (live) {
      const int escale = ew ? ew[pc] : 0;  // FP16 plans: Q^T's row scale
      for (int ib = i0; ib < i1; ib += kScanGroup) {
        float2 gg[kScanGroup];
        sum_chunks_group<kScanGroup>(part, plane, S, ib, i1, K_pad, pc, escale, nullptr, n_r, gg);
#pragma unroll
        for (int k = 0; k < kScanGroup; ++k) {
          if (ib + k < i1) {
            const int i = ib + k;
            Mbar[(long long)i * K_pad + pc] = gg[k];
            const float2 hz = (i > 0) ? fout[i - 1] : zero;
            Z = tc::ff_fma(hz, Z, gg[k]);
            FZ = tc::ff_mul(FZ, hz);
          }
          if (ib == i0) mg[k] = gg[k];
        }
      }
      if (i1 - i0 <= kScanGroup) {
#pragma unroll
        for (int k = kScanGroup - 1; k >= 0; --k) {
          if (k < i1 - i0) {
            const int i = i0 + k;
            const float2 gx = (i + 1 < n_r) ? fin[i + 1] : zero;
            X = tc::ff_fma(gx, X, mg[k]);
            FX = tc::ff_mul(FX, gx);
          }
        }
      } else {
        for (int i = i1 - 1; i >= i0; --i) {
          const float2 gx = (i + 1 < n_r) ? fin[i + 1] : zero;
          X = tc::ff_fma(gx, X, Mbar[(long long)i * K_pad + pc]);
          FX = tc::ff_mul(FX, gx);
        }
      }
    } else if (pc < K_pad && l < 0) {
      for (int i = i0; i < i1; ++i) Mbar[(long long)i * K_pad + pc] = zero;
    }
    if (p < kScanMaxP) {
      sm[0][p][c] = Z;
      sm[1][p][c] = FZ;
      sm[2][p][c] = X;
      sm[3][p][c] = FX;
    }
  }
  __syncthreads();
  // ---- phase 2: carries (Z upward, X downward)
  carry_scan<kScanCols, kScanMaxP>(sm, cr, P);
  __syncthreads();
  // ---- phase 3: Bbar_i = a_i X_i + b_i Z_{i-1} with the carries, and its BF16 slices
  if (pc >= K_pad || p >= P || i0 >= n_r) return;
  if (l < 0) {
    for (int i = i0; i < i1; ++i) {
      Bbar[(long long)i * K_pad + pc] = zero;
      if (write_slices == 2)
        for (int k = 0; k < 2; ++k) reinterpret_cast<float*>(Bs)[k * plane + (long long)i * K_pad + pc] = 0.0f;
      else if (write_slices)
        for (int k = 0; k < nsl; ++k) Bs[k * plane + (long long)i * K_pad + pc] = __float2bfloat16_rn(0.f);
    }
    return;
  }
  auto emit = [&](int i, float2 b) {
    Bbar[(long long)i * K_pad + pc] = b;
    if (write_slices == 2) {  // TF32 slices (4-byte elements)
      float s0, s1;
      ff_tf32(b.x, b.y, s0, s1);
      float* Bf = reinterpret_cast<float*>(Bs);
      Bf[(long long)i * K_pad + pc] = s0;
      Bf[plane + (long long)i * K_pad + pc] = s1;
    } else if (write_slices) {
      __nv_bfloat16 sl[3];
      ff_slices(b, nsl, sl);
#pragma unroll
      for (int k = 0; k < 3; ++k)  // constant indices keep sl in registers
        if (k < nsl) Bs[k * plane + (long long)i * K_pad + pc] = sl[k];
    }
  };
  float2 X = cr[1][p][c];  // X_{i1}
  float2 Z = cr[0][p][c];  // Z_{i0-1}
  if (i1 - i0 <= kScanGroup) {
    // the chunk's Mbar and a_i X_i in registers; Bbar written once
    float2 ax[kScanGroup];
#pragma unroll
    for (int k = kScanGroup - 1; k >= 0; --k) {
      ax[k] = zero;
      if (k < i1 - i0) {
        const int i = i0 + k;
        const float2 gx = (i + 1 < n_r) ? fin[i + 1] : zero;
        X = tc::ff_fma(gx, X, mg[k]);
        ax[k] = tc::ff_mul(at[i], X);
      }
    }
#pragma unroll
    for (int k = 0; k < kScanGroup; ++k) {
      if (k < i1 - i0) {
        const int i = i0 + k;
        emit(i, tc::ff_fma(bt[i], Z, ax[k]));
        const float2 hz = (i > 0) ? fout[i - 1] : zero;
        Z = tc::ff_fma(hz, Z, mg[k]);
      }
    }
    return;
  }
  for (int i = i1 - 1; i >= i0; --i) {
    const float2 gx = (i + 1 < n_r) ? fin[i + 1] : zero;
    X = tc::ff_fma(gx, X, Mbar[(long long)i * K_pad + pc]);
    Bbar[(long long)i * K_pad + pc] = tc::ff_mul(at[i], X);
  }
  for (int i = i0; i < i1; ++i) {
    emit(i, tc::ff_fma(bt[i], Z, Bbar[(long long)i * K_pad + pc]));
    const float2 hz = (i > 0) ? fout[i - 1] : zero;
    Z = tc::ff_fma(hz, Z, Mbar[(long long)i * K_pad + pc]);
  }
}

// out[i][nat] = in[i][pc] (float-float, widened to FP64) for every real padded column.
__global__ void tc_unpermute_kernel(int n_r, int K, int K_pad, const int* __restrict__ pc_nat,
                                    const float2* __restrict__ in, double* __restrict__ out) {
  long long total = (long long)n_r * K_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / K_pad;
    int pc = (int)(e % K_pad);
    int c = pc_nat[pc];
    if (c >= 0) out[i * K + c] = (double)in[e].x + (double)in[e].y;
  }
}

template <int NSL, int MODE, bool SCALE, bool TF = false>
cudaError_t set_smem_attr() {
  cudaError_t e = cudaFuncSetAttribute(tc::tc_gemm_kernel<NSL, MODE, SCALE, TF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<NSL, MODE>::SMEM);
  if (e == cudaSuccess) e = tc::check_reg_split<MODE, false>((const void*)tc::tc_gemm_kernel<NSL, MODE, SCALE, TF>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc::tc_gemm_group_kernel<NSL, MODE, SCALE, TF>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<NSL, MODE>::SMEM);
  if (e == cudaSuccess)
    e = tc::check_reg_split<MODE, false>((const void*)tc::tc_gemm_group_kernel<NSL, MODE, SCALE, TF>);
  return e;
}

// scale: the projection of FP16 field slices (group factors applied at the
// flushes); tf: TF32 operands; both two slices only
template <int MODE>
cudaError_t dispatch_gemm(int nsl, bool scale, bool tf, int grid, const CUtensorMap& a, const CUtensorMap& b,
                          const CUtensorMap& bt, const TcArgs& args, cudaStream_t s) {
  constexpr int threads = tc::TileShape<MODE>::THREADS;
  if (nsl == 3 && !scale && !tf) {
    tc::tc_gemm_kernel<3, MODE, false><<<grid, threads, TcCfg<3, MODE>::SMEM, s>>>(a, b, bt, args);
  } else if (nsl == 2 && tf && !scale) {
    tc::tc_gemm_kernel<2, MODE, false, true><<<grid, threads, TcCfg<2, MODE>::SMEM, s>>>(a, b, bt, args);
  } else if (nsl == 2 && !scale) {
    tc::tc_gemm_kernel<2, MODE, false><<<grid, threads, TcCfg<2, MODE>::SMEM, s>>>(a, b, bt, args);
  } else if (nsl == 2 && !tf && MODE == tc::kProject) {
    tc::tc_gemm_kernel<2, MODE, MODE == tc::kProject><<<grid, threads, TcCfg<2, MODE>::SMEM, s>>>(a, b, bt, args);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The synthesis on CTA pairs: clusters of two CTAs, each pair one 256-cell
// tile per step of its walk (B's maps with half-tile boxes).
template <int NSL, bool TF>
cudaError_t launch_synth_pair(int grid, const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& bt,
                              const TcArgs& args, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)tc::TileShape<tc::kSynthesize>::THREADS);
  cfg.dynamicSmemBytes = TcCfg<NSL, tc::kSynthesize, false, 2>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc::tc_gemm_kernel<NSL, tc::kSynthesize, false, TF, false, 2>, a, b, bt, args);
}
template <int NSL, bool TF>
const void* synth_pair_fn() {
  return (const void*)tc::tc_gemm_kernel<NSL, tc::kSynthesize, false, TF, false, 2>;
}
cudaError_t dispatch_synth_pair(int nsl, bool tf, int grid, const CUtensorMap& a, const CUtensorMap& b,
                                const CUtensorMap& bt, const TcArgs& args, cudaStream_t s) {
  if (grid % 2 != 0) return cudaErrorInvalidValue;
  if (nsl == 3 && !tf) return launch_synth_pair<3, false>(grid, a, b, bt, args, s);
  if (nsl == 2 && tf) return launch_synth_pair<2, true>(grid, a, b, bt, args, s);
  if (nsl == 2) return launch_synth_pair<2, false>(grid, a, b, bt, args, s);
  return cudaErrorInvalidValue;
}
// Shared memory of the pair kernel of a plan's operand kind, and how many of
// its clusters fit on the GPU at once (0: none, then the single-CTA kernel runs).
cudaError_t setup_synth_pair(int nsl, bool tf, int sms, int& clusters) {
  clusters = 0;
  const void* fn = nullptr;
  int smem = 0;
  if (nsl == 3 && !tf) {
    fn = synth_pair_fn<3, false>();
    smem = TcCfg<3, tc::kSynthesize, false, 2>::SMEM;
  } else if (nsl == 2) {
    fn = tf ? synth_pair_fn<2, true>() : synth_pair_fn<2, false>();
    smem = TcCfg<2, tc::kSynthesize, false, 2>::SMEM;
  } else {
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = tc::check_reg_split<tc::kSynthesize, false>(fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * std::max(1, sms / 2)));
  cfg.blockDim = dim3((unsigned)tc::TileShape<tc::kSynthesize>::THREADS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
}

template <int MODE>
cudaError_t dispatch_group(int nsl, bool scale, bool tf, int grid, const tc::TcProblem* probs, const int* start,
                           int n, int total, const tc::TcPhiList& phis, cudaStream_t s) {
  constexpr int threads = tc::TileShape<MODE>::THREADS;
  if (nsl == 3 && !scale && !tf) {
    tc::tc_gemm_group_kernel<3, MODE, false><<<grid, threads, TcCfg<3, MODE>::SMEM, s>>>(probs, start, n, total, phis);
  } else if (nsl == 2 && tf && !scale) {
    tc::tc_gemm_group_kernel<2, MODE, false, true>
        <<<grid, threads, TcCfg<2, MODE>::SMEM, s>>>(probs, start, n, total, phis);
  } else if (nsl == 2 && !scale) {
    tc::tc_gemm_group_kernel<2, MODE, false><<<grid, threads, TcCfg<2, MODE>::SMEM, s>>>(probs, start, n, total, phis);
  } else if (nsl == 2 && !tf && MODE == tc::kProject) {
    tc::tc_gemm_group_kernel<2, MODE, MODE == tc::kProject>
        <<<grid, threads, TcCfg<2, MODE>::SMEM, s>>>(probs, start, n, total, phis);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// The synthesis's shell tiling at full-tile width w (a multiple of 16, at
// most the kernel's NMAX): tile counts and the M-slice tensor maps (boxes of
// w and of the tail width; with CTA pairs, `clusters` > 0, also boxes of half
// of each, one per CTA of a pair).
static bool set_synth_shape(ygs_plan* p, int w, int clusters) {
  const int kind = slice_kind(p);
  p->tc_N = w;
  p->tc_n_full = p->n_r / w;
  p->tc_n_tail = ((p->n_r % w) + 15) / 16 * 16;
  const int Nt = p->tc_n_tail > 0 ? p->tc_n_tail : w;
  p->tc_pairs = 0;
  if (!make_map(&p->tc_map_m, p->tc_ms, p->tc_k_pad, p->n_r, p->tc_nsl, w, kind) ||
      !make_map(&p->tc_map_m_tail, p->tc_ms, p->tc_k_pad, p->n_r, p->tc_nsl, Nt, kind))
    return false;
  if (clusters > 0) {
    if (!make_map(&p->tc_map_m2, p->tc_ms, p->tc_k_pad, p->n_r, p->tc_nsl, w / 2, kind) ||
        !make_map(&p->tc_map_m2_tail, p->tc_ms, p->tc_k_pad, p->n_r, p->tc_nsl, Nt / 2, kind))
      return false;
    p->tc_pairs = clusters;
  }
  return true;
}

ygs_status tc_setup(ygs_plan* p, int sms) {
  const int nsl = p->tc_nsl;
  const int K = p->K;
  auto r64 = [](long long x) { return (x + 63) / 64 * 64; };
  // angular padding to whole exponent groups (two k-blocks; EMU: windows of
  // four): chunk and patch starts then fall on group boundaries
  const long long grp = p->tc_emu ? kEmuWindow : kGroup;
  auto r32 = [grp](long long x) { return (x + grp - 1) / grp * grp; };
  static_assert(kGroup == 2 * tc::BK, "an exponent group is two k-blocks");
  // padded column layout: [even block | pad | odd block | pad]
  const int Ke = p->K_even, Ko = K - p->K_even;
  p->tc_k_even = (int)r64(Ke);
  p->tc_k_pad = p->tc_k_even + (int)r64(Ko);
  std::vector<int> pc_int(p->tc_k_pad, -1), pc_l(p->tc_k_pad, -1), pc_nat(p->tc_k_pad, -1);
  for (int ci = 0; ci < K; ++ci) {
    int pc = (ci < Ke) ? ci : p->tc_k_even + (ci - Ke);
    int c = p->col_perm[ci], l = 0;
    while ((l + 1) * (l + 1) <= c) ++l;
    pc_int[pc] = ci;
    pc_l[pc] = l;
    pc_nat[pc] = c;
  }
  // padded angular layout of the stored patches
  p->tc_pad_off.assign(p->n_wpatch + 1, 0);
  for (int g = 0; g < p->n_wpatch; ++g) p->tc_pad_off[g + 1] = p->tc_pad_off[g] + r32(p->nang[g]);
  p->tc_n_pad = p->tc_pad_off[p->n_wpatch];
  const int NP = tc::kNmaxProject, NS = p->tc_emu ? tc::kNmaxSynthEmu : tc::kNmaxSynth;
  p->tc_N = NS;
  p->tc_np_full = p->n_r / NP;
  p->tc_np_tail = ((p->n_r % NP) + 15) / 16 * 16;
  p->tc_n_full = p->n_r / NS;
  p->tc_n_tail = ((p->n_r % NS) + 15) / 16 * 16;
  p->tc_sms = sms;

  // split-K chunks: the projection's tiles (a tail tile counted by its width) fill about one wave
  const int tiles_m = (p->tc_k_even + tc::BM - 1) / tc::BM +
                      ((p->tc_k_pad - p->tc_k_even) + tc::BM - 1) / tc::BM;
  const double per_chunk = tiles_m * (p->tc_np_full + (double)p->tc_np_tail / NP);
  const int n_tiles_p = p->tc_np_full + (p->tc_np_tail > 0 ? 1 : 0);
  long long want = std::max(1LL, (long long)std::floor(sms / std::max(1.0, per_chunk) + 0.5));
  while (want > 1 && (long long)tiles_m * n_tiles_p * want > sms) --want;
  // candidate split-K targets: the one-wave rule, and, when autotuning, half, two and three waves
  std::vector<long long> wants = {want};
  if (p->flags & YGS_FLAG_AUTOTUNE)
    for (long long w2 : {std::max(1LL, want / 2), 2 * want, 3 * want})
      if (std::find(wants.begin(), wants.end(), w2) == wants.end()) wants.push_back(w2);
  std::vector<std::vector<int2>> cand;
  for (long long wv : wants) {
    std::vector<int2> chunks;
    for (int g = 0; g < p->n_wpatch; ++g) {
      const long long kb_g = r32(p->nang[g]) / tc::BK;
      long long sg = std::max(1LL, (wv * p->nang[g] + p->nang_wtotal - 1) / p->nang_wtotal);
      sg = std::min(sg, std::max(1LL, kb_g / 4));
      const long long gkb = grp / tc::BK;
      const long long per = ((kb_g + sg - 1) / sg + gkb - 1) / gkb * gkb;  // whole exponent groups per chunk
      for (long long k0 = 0; k0 < kb_g; k0 += per)
        chunks.push_back(make_int2((int)((p->tc_pad_off[g] + k0 * tc::BK)),
                                   (int)(p->tc_pad_off[g] + std::min(kb_g, k0 + per) * tc::BK)));
    }
    cand.push_back(chunks);
  }
  size_t s_max = 0;
  for (const auto& c : cand) s_max = std::max(s_max, c.size());
  std::vector<int2> chunks = cand[0];
  p->tc_S = (int)chunks.size();
  // chunks of 4 shells for the parallel scans (more when n_r > 4 kScanMaxP: at most kScanMaxP chunks)
  p->tc_scan_chunk = std::max(4, (p->n_r + kScanMaxP - 1) / kScanMaxP);
  p->tc_scan_P = (p->n_r + p->tc_scan_chunk - 1) / p->tc_scan_chunk;

  const size_t kp = (size_t)p->tc_k_pad;
  const size_t esz = slice_bytes(p);
  size_t bytes_ut = (size_t)nsl * kp * p->tc_n_pad * esz;
  size_t bytes_q = (size_t)nsl * p->nang_wtotal * kp * esz;
  size_t bytes_f = (size_t)(p->symmetric ? 2 : 1) * nsl * p->n_r * p->tc_n_pad * esz;
  size_t bytes_m = (size_t)nsl * p->n_r * kp * esz;
  size_t bytes_part = s_max * p->n_r * kp * sizeof(float2);
  size_t bytes_nk = (size_t)p->n_r * kp * sizeof(double);
  size_t bytes_sum = (size_t)4 * p->tc_scan_P * kp * sizeof(double);
  cudaError_t e;
#define TC_ALLOC(ptr, bytes)                                                          \
  if ((e = dev_malloc((void**)&(ptr), std::max<size_t>((bytes), 16))) != cudaSuccess) { \
    set_error(std::string("cudaMalloc ") + #ptr + ": " + cudaGetErrorString(e));      \
    return YGS_ERR_OOM;                                                                \
  }
  TC_ALLOC(p->tc_ut, bytes_ut);
  TC_ALLOC(p->tc_qs, bytes_q);
  TC_ALLOC(p->tc_qt, bytes_ut);
  TC_ALLOC(p->tc_us, bytes_q);
  TC_ALLOC(p->tc_Mbar, bytes_nk);
  TC_ALLOC(p->tc_Bbar, bytes_nk);
  TC_ALLOC(p->tc_f, bytes_f);
  TC_ALLOC(p->tc_ms, bytes_m);
  TC_ALLOC(p->tc_part, bytes_part);
  TC_ALLOC(p->tc_B, bytes_nk);
  TC_ALLOC(p->tc_M, bytes_nk);
  TC_ALLOC(p->tc_summ, bytes_sum);
  TC_ALLOC(p->tc_carry, bytes_sum / 2);
  TC_ALLOC(p->tc_chunks, s_max * sizeof(int2));
  TC_ALLOC(p->tc_pc_int, kp * sizeof(int));
  TC_ALLOC(p->tc_pc_l, kp * sizeof(int));
  TC_ALLOC(p->tc_pc_nat, kp * sizeof(int));
  TC_ALLOC(p->tc_pad_off_d, (p->n_wpatch + 1) * sizeof(long long));
  TC_ALLOC(p->tc_mono, (size_t)p->n_r * sizeof(float2));
  TC_ALLOC(p->tc_cp, (size_t)2 * (p->l_max + 1) * p->tc_scan_P * sizeof(float2));
  TC_ALLOC(p->tc_radff, (size_t)4 * (p->l_max + 1) * p->n_r * sizeof(float2));
  if (p->tc_fp16) {
    TC_ALLOC(p->tc_eqt, kp * sizeof(int));
    TC_ALLOC(p->tc_eu, kp * sizeof(int));
    TC_ALLOC(p->tc_fac, (size_t)2 * (p->tc_n_pad / kGroup) * fac_ld(p) * sizeof(float));
    TC_ALLOC(p->tc_u00, (size_t)p->tc_n_pad * sizeof(float2));
    TC_ALLOC(p->tc_mpart, s_max * p->n_r * sizeof(float2));
    TC_ALLOC(p->tc_em, (size_t)p->n_r * sizeof(int));
    TC_ALLOC(p->tc_sc, (size_t)p->n_r * sizeof(float4));
  }
  if (p->tc_emu) {
    TC_ALLOC(p->tc_fac, (size_t)2 * (p->tc_n_pad / kEmuWindow) * fac_ld(p) * sizeof(float));
    TC_ALLOC(p->tc_sc, (size_t)p->n_r * sizeof(float4));
    TC_ALLOC(p->tc_Bd, bytes_nk);
    TC_ALLOC(p->tc_Md, bytes_nk);
  }
#undef TC_ALLOC
  p->weight_bytes += (long long)(2 * (bytes_ut + bytes_q));
  p->work_bytes += (long long)(bytes_f + bytes_m + bytes_part + 4 * bytes_nk + bytes_sum * 3 / 2);
#define TC_TRY(x)                                                                  \
  if ((e = (x)) != cudaSuccess) {                                                  \
    set_error(std::string("tc setup: ") + #x + ": " + cudaGetErrorString(e));       \
    return YGS_ERR_CUDA;                                                           \
  }
  TC_TRY(cudaMemcpy(p->tc_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice));
  TC_TRY(cudaMemcpy(p->tc_pc_int, pc_int.data(), kp * sizeof(int), cudaMemcpyHostToDevice));
  TC_TRY(cudaMemcpy(p->tc_pc_l, pc_l.data(), kp * sizeof(int), cudaMemcpyHostToDevice));
  TC_TRY(cudaMemcpy(p->tc_pc_nat, pc_nat.data(), kp * sizeof(int), cudaMemcpyHostToDevice));
  TC_TRY(cudaMemcpy(p->tc_pad_off_d, p->tc_pad_off.data(), (p->n_wpatch + 1) * sizeof(long long),
                    cudaMemcpyHostToDevice));
  TC_TRY(cudaMemset(p->tc_f, 0, bytes_f));  // padding columns stay zero
  if (p->tc_fp16 || p->tc_emu)  // factors of the shells past n_r (read with a tile's row, never written) stay zero
    TC_TRY(cudaMemset(p->tc_fac, 0, (size_t)2 * (p->tc_n_pad / grp) * fac_ld(p) * sizeof(float)));
  chunk_prod_kernel<<<((p->l_max + 1) * p->tc_scan_P + 127) / 128, 128>>>(p->n_r, p->l_max, p->tc_scan_chunk,
                                                                          p->tc_scan_P, p->rad, p->tc_cp);
  TC_TRY(cudaGetLastError());
  rad_ff_kernel<<<256, 256>>>((long long)4 * (p->l_max + 1) * p->n_r, p->rad, p->tc_radff);
  TC_TRY(cudaGetLastError());
  if (p->tc_fp16) {
    colexp_u_kernel<<<p->tc_k_pad, 256>>>(K, p->tc_pc_int, p->nang_wtotal, p->U, p->tc_eu);
    TC_TRY(cudaGetLastError());
    slice_ut16_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->tc_n_pad, p->tc_pc_int, p->U, p->pt, p->n_wpatch,
                                     p->tc_pad_off_d, p->tc_eu, 1, reinterpret_cast<__half*>(p->tc_ut));
    u00_kernel<<<256, 256>>>(K, pc_int[0], p->tc_n_pad, p->pt, p->n_wpatch, p->tc_pad_off_d, p->U, p->tc_u00);
    TC_TRY(cudaGetLastError());
    TC_TRY(cudaGetLastError());
    // Q as a whole: its largest magnitude (through a scratch word in the M buffer) sets eq
    unsigned long long* qm = reinterpret_cast<unsigned long long*>(p->tc_M);
    TC_TRY(cudaMemset(qm, 0, sizeof(unsigned long long)));
    qmax_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->Q, 1, qm);
    TC_TRY(cudaGetLastError());
    unsigned long long bits = 0;
    TC_TRY(cudaMemcpy(&bits, qm, sizeof(bits), cudaMemcpyDeviceToHost));
    double qmax;
    memcpy(&qmax, &bits, sizeof(qmax));
    p->tc_eq = tc::fp16_row_exp(qmax);
    slice_q16_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->Q, p->tc_eq, 1,
                                    reinterpret_cast<__half*>(p->tc_qs));
    TC_TRY(cudaGetLastError());
    // adjoint operands: Q^T per column, U as a whole (monopole kept)
    colexp_u_kernel<<<p->tc_k_pad, 256>>>(K, p->tc_pc_int, p->nang_wtotal, p->Q, p->tc_eqt);
    TC_TRY(cudaGetLastError());
    slice_ut16_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->tc_n_pad, p->tc_pc_int, p->Q, p->pt, p->n_wpatch,
                                     p->tc_pad_off_d, p->tc_eqt, 0, reinterpret_cast<__half*>(p->tc_qt));
    TC_TRY(cudaGetLastError());
    TC_TRY(cudaMemset(qm, 0, sizeof(unsigned long long)));
    qmax_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->U, 0, qm);
    TC_TRY(cudaGetLastError());
    TC_TRY(cudaMemcpy(&bits, qm, sizeof(bits), cudaMemcpyDeviceToHost));
    memcpy(&qmax, &bits, sizeof(qmax));
    p->tc_eus = tc::fp16_row_exp(qmax);
    slice_q16_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->U, p->tc_eus, 0,
                                    reinterpret_cast<__half*>(p->tc_us));
    TC_TRY(cudaGetLastError());
  } else if (p->tc_emu) {
    TC_TRY(emu_slice_weights(p));
  } else if (p->tc_tf32) {
    slice_ut_tf32_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->tc_n_pad, p->tc_pc_int, p->U, p->pt, p->n_wpatch,
                                        p->tc_pad_off_d, reinterpret_cast<float*>(p->tc_ut));
    TC_TRY(cudaGetLastError());
    slice_q_tf32_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->Q, 1,
                                       reinterpret_cast<float*>(p->tc_qs));
    TC_TRY(cudaGetLastError());
    // adjoint operands: Q^T in the projection layout, U in the synthesis layout (monopole kept)
    slice_ut_tf32_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->tc_n_pad, p->tc_pc_int, p->Q, p->pt, p->n_wpatch,
                                        p->tc_pad_off_d, reinterpret_cast<float*>(p->tc_qt));
    TC_TRY(cudaGetLastError());
    slice_q_tf32_kernel<<<1024, 256>>>(K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->U, 0,
                                       reinterpret_cast<float*>(p->tc_us));
    TC_TRY(cudaGetLastError());
  } else {
    slice_ut_kernel<<<1024, 256>>>(nsl, K, p->tc_k_pad, p->tc_n_pad, p->tc_pc_int, p->U, p->pt, p->n_wpatch,
                                   p->tc_pad_off_d, p->tc_ut);
    TC_TRY(cudaGetLastError());
    slice_q_kernel<<<1024, 256>>>(nsl, K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->Q, 1, p->tc_qs);
    TC_TRY(cudaGetLastError());
    // adjoint operands: Q^T in the projection layout, U in the synthesis layout (monopole kept)
    slice_ut_kernel<<<1024, 256>>>(nsl, K, p->tc_k_pad, p->tc_n_pad, p->tc_pc_int, p->Q, p->pt, p->n_wpatch,
                                   p->tc_pad_off_d, p->tc_qt);
    TC_TRY(cudaGetLastError());
    slice_q_kernel<<<1024, 256>>>(nsl, K, p->tc_k_pad, p->nang_wtotal, p->tc_pc_int, p->tc_pc_nat, p->U, 0, p->tc_us);
    TC_TRY(cudaGetLastError());
  }
  TC_TRY(cudaDeviceSynchronize());

  const int N = NS;
  const int Nt = p->tc_n_tail > 0 ? p->tc_n_tail : N;
  const int Npt = p->tc_np_tail > 0 ? p->tc_np_tail : NP;
  const int fplanes = (p->symmetric ? 2 : 1) * nsl;
  const int kind = slice_kind(p);
  if (!make_map(&p->tc_map_ut, p->tc_ut, p->tc_n_pad, p->tc_k_pad, nsl, tc::BM, kind) ||
      !make_map(&p->tc_map_f, p->tc_f, p->tc_n_pad, p->n_r, fplanes, NP, kind) ||
      !make_map(&p->tc_map_f_tail, p->tc_f, p->tc_n_pad, p->n_r, fplanes, Npt, kind) ||
      !make_map(&p->tc_map_q, p->tc_qs, p->tc_k_pad, p->nang_wtotal, nsl, tc::BM, kind) ||
      !make_map(&p->tc_map_qt, p->tc_qt, p->tc_n_pad, p->tc_k_pad, nsl, tc::BM, kind) ||
      !make_map(&p->tc_map_us, p->tc_us, p->tc_k_pad, p->nang_wtotal, nsl, tc::BM, kind) ||
      !make_map(&p->tc_map_m, p->tc_ms, p->tc_k_pad, p->n_r, nsl, N, kind) ||
      !make_map(&p->tc_map_m_tail, p->tc_ms, p->tc_k_pad, p->n_r, nsl, Nt, kind)) {
    set_error("cuTensorMapEncodeTiled failed or is unavailable");
    return YGS_ERR_CUDA;
  }
  {
    cudaError_t a1 = cudaSuccess, a2 = cudaSuccess;
    if (p->tc_emu) {
      a1 = emu_set_smem_attrs();
    } else if (nsl == 3) {
      a1 = set_smem_attr<3, tc::kProject, false>();
      a2 = set_smem_attr<3, tc::kSynthesize, false>();
    } else {
      a1 = p->tc_fp16   ? set_smem_attr<2, tc::kProject, true>()
           : p->tc_tf32 ? set_smem_attr<2, tc::kProject, false, true>()
                        : set_smem_attr<2, tc::kProject, false>();
      a2 = p->tc_tf32 ? set_smem_attr<2, tc::kSynthesize, false, true>() : set_smem_attr<2, tc::kSynthesize, false>();
    }
    TC_TRY(a1);
    TC_TRY(a2);
  }
  // the synthesis on CTA pairs: M slices in boxes of half a tile's shells
  p->tc_pairs = 0;
  if (!p->tc_emu && (p->flags & YGS_FLAG_CTA_PAIRS) && N % 16 == 0 && Nt % 16 == 0) {
    int clusters = 0;
    TC_TRY(setup_synth_pair(nsl, p->tc_tf32 != 0, p->tc_sms, clusters));
    if (!set_synth_shape(p, N, clusters)) {
      set_error("cuTensorMapEncodeTiled failed or is unavailable");
      return YGS_ERR_CUDA;
    }
  }
  if (cand.size() > 1) {
    // time the projection of a zero field with each candidate; keep the fastest
    cudaEvent_t e0, e1;
    TC_TRY(cudaEventCreate(&e0));
    TC_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    size_t pick = 0;
    for (size_t c = 0; c < cand.size(); ++c) {
      TC_TRY(cudaMemcpy(p->tc_chunks, cand[c].data(), cand[c].size() * sizeof(int2), cudaMemcpyHostToDevice));
      p->tc_S = (int)cand[c].size();
      TC_TRY(tc_project(p, 0));
      TC_TRY(cudaEventRecord(e0, 0));
      for (int r = 0; r < 5; ++r) TC_TRY(tc_project(p, 0));
      TC_TRY(cudaEventRecord(e1, 0));
      TC_TRY(cudaEventSynchronize(e1));
      float ms = 0.0f;
      TC_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    chunks = cand[pick];
    p->tc_S = (int)chunks.size();
    TC_TRY(cudaMemcpy(p->tc_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice));
    TC_TRY(cudaDeviceSynchronize());
  }
  if ((p->flags & YGS_FLAG_AUTOTUNE) && !p->tc_emu) {
    // the synthesis's tile shape: every distinct shell tiling of full-tile
    // widths NS, NS - NH, ... (whole groups of an epilogue warp's NH columns:
    // 144, 96, 48), on one CTA per 128-cell tile and, where
    // the GPU co-schedules them, on CTA pairs (256-cell tiles); each timed over
    // 5 launches on zero M slices into a scratch Phi; the fastest is kept
    int clusters = 0;
    if (setup_synth_pair(nsl, p->tc_tf32 != 0, p->tc_sms, clusters) != cudaSuccess) clusters = 0;
    cudaGetLastError();
    struct Shape { int w, pair; };
    std::vector<Shape> shapes;
    std::vector<std::pair<int, int>> tilings;  // (full tiles, tail width) already listed
    for (int w = NS; w >= tc::kNhSynth; w -= tc::kNhSynth) {  // whole epilogue-warp column groups
      const std::pair<int, int> tl(p->n_r / w, ((p->n_r % w) + 15) / 16 * 16);
      if (std::find(tilings.begin(), tilings.end(), tl) != tilings.end()) continue;
      tilings.push_back(tl);
      shapes.push_back(Shape{w, 0});
      if (clusters > 0) shapes.push_back(Shape{w, 1});
    }
    const Shape keep{p->tc_N, p->tc_pairs > 0 ? 1 : 0};
    double* phi_tmp = nullptr;
    if (shapes.size() > 1) {
      TC_TRY(cudaMemset(p->tc_ms, 0, bytes_m));
      TC_TRY(cudaMemset(p->tc_mono, 0, (size_t)p->n_r * sizeof(float2)));
      if (p->tc_fp16) TC_TRY(cudaMemset(p->tc_sc, 0, (size_t)p->n_r * sizeof(float4)));
      if ((e = dev_malloc((void**)&phi_tmp, (size_t)p->n_cells * sizeof(double))) != cudaSuccess) {
        set_error(std::string("cudaMalloc (autotuner's scratch Phi): ") + cudaGetErrorString(e));
        return YGS_ERR_OOM;
      }
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaError_t te = cudaEventCreate(&e0);
      if (te == cudaSuccess) te = cudaEventCreate(&e1);
      float best = 1e30f;
      Shape pick = keep;
      for (size_t c = 0; c < shapes.size() && te == cudaSuccess; ++c) {
        if (!set_synth_shape(p, shapes[c].w, shapes[c].pair ? clusters : 0)) {
          te = cudaErrorInvalidValue;
          break;
        }
        if ((te = tc_synthesize(p, phi_tmp, 0)) != cudaSuccess) break;
        if ((te = cudaEventRecord(e0, 0)) != cudaSuccess) break;
        for (int r = 0; r < 5 && te == cudaSuccess; ++r) te = tc_synthesize(p, phi_tmp, 0);
        if (te != cudaSuccess || (te = cudaEventRecord(e1, 0)) != cudaSuccess) break;
        if ((te = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        if ((te = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (ms < best) {
          best = ms;
          pick = shapes[c];
        }
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaFree(phi_tmp);
      TC_TRY(te);
      if (!set_synth_shape(p, pick.w, pick.pair ? clusters : 0)) {
        set_error("cuTensorMapEncodeTiled failed or is unavailable");
        return YGS_ERR_CUDA;
      }
      TC_TRY(cudaDeviceSynchronize());
    }
  }

#undef TC_TRY
  return YGS_OK;
}

void tc_free(ygs_plan* p) {
  void* bufs[] = {p->tc_ut,    p->tc_qs,     p->tc_f,      p->tc_ms,     p->tc_part,      p->tc_B,
                  p->tc_M,     p->tc_summ,   p->tc_carry,  p->tc_chunks, p->tc_pc_int,    p->tc_pc_l,
                  p->tc_pc_nat, p->tc_pad_off_d, p->tc_mono, p->tc_cp, p->tc_radff, p->tc_eu, p->tc_fac, p->tc_em,
                  p->tc_qt,    p->tc_us,     p->tc_eqt,    p->tc_Mbar,   p->tc_Bbar,   p->tc_u00,
                  p->tc_mpart, p->tc_sc, p->tc_Bd, p->tc_Md};
  for (void* b : bufs)
    if (b) cudaFree(b);
}

// The arguments and grids of the per-field passes, shared by the plain
// launches below and the grouped launches of a batch.
static Field16Args field16_args(const ygs_plan* p, bool forward) {
  return Field16Args{p->n_r, p->symmetric ? 1 : 0, p->n_wpatch, p->pt, p->tc_pad_off_d, p->tc_n_pad, p->tc_chunks,
                     reinterpret_cast<__half*>(p->tc_f), p->tc_fac, fac_ld(p), forward ? p->tc_u00 : nullptr,
                     forward ? p->tc_mpart : nullptr};
}
static dim3 field16_grid(const ygs_plan* p) { return dim3(p->tc_S, p->n_r); }
constexpr int kFieldSlicesThreads = 128;
static dim3 field_slices_grid(const ygs_plan* p) {
  long long nmax = 0;
  for (int g = 0; g < p->n_wpatch; ++g) nmax = std::max(nmax, p->nang[g]);
  const int bx = (int)std::min<long long>(64, (nmax / 4 + kFieldSlicesThreads - 1) / kFieldSlicesThreads);
  return dim3(std::max(1, bx), p->n_r, p->n_wpatch);
}
static FieldSlicesArgs field_slices_args(const ygs_plan* p) {
  return FieldSlicesArgs{p->tc_nsl, p->n_r, p->symmetric ? 1 : 0, p->pt, p->tc_pad_off_d, p->tc_n_pad, p->tc_f};
}
static FieldSlicesTf32Args field_slices_tf32_args(const ygs_plan* p) {
  return FieldSlicesTf32Args{p->n_r, p->symmetric ? 1 : 0, p->pt, p->tc_pad_off_d, p->tc_n_pad,
                             reinterpret_cast<float*>(p->tc_f)};
}

cudaError_t tc_field_slices(const ygs_plan* p, const double* rho, cudaStream_t s, bool forward) {
  if (p->tc_emu) return emu_field_slices(p, rho, s);
  if (p->tc_fp16) {
    const Field16Args a = field16_args(p, forward);
    field16_kernel<<<field16_grid(p), kF16Threads, 0, s>>>(a.n_r, a.symmetric, a.nwp, a.pt, a.pad_off, a.n_pad,
                                                           a.chunks, rho, a.F, a.fac, a.fac_ld, a.u00, a.mpart);
    return cudaGetLastError();
  }
  if (p->tc_tf32) {
    const FieldSlicesTf32Args a = field_slices_tf32_args(p);
    field_slices_tf32_kernel<<<field_slices_grid(p), kFieldSlicesThreads, 0, s>>>(a.n_r, a.symmetric, a.pt,
                                                                                  a.pad_off, a.n_pad, rho, a.F);
    return cudaGetLastError();
  }
  const FieldSlicesArgs a = field_slices_args(p);
  field_slices_kernel<<<field_slices_grid(p), kFieldSlicesThreads, 0, s>>>(a.nsl, a.n_r, a.symmetric, a.pt,
                                                                           a.pad_off, a.n_pad, rho, a.F);
  return cudaGetLastError();
}

// The forward synthesis flushes its accumulators every 192 k-elements (three
// windows per 576-column segment at l_max = 32): its terms change sign (the
// monopole, the one coherent sum, is added exactly in the epilogue), so the
// FP32 accumulation drifts less than in the adjoint's synthesis with U, whose
// monopole column sums positive terms and keeps 64.  (Measured on config 1
// against FP64: 2.1e-7 at 64, 3.4e-7 at 128, 5.4e-7 at 256; 192 is 10% faster
// than 128.)  The FP16 forward projection, whose monopole is summed exactly
// in the field pass, flushes every 128: a flush window there must not span
// two of the field's exponent groups (kGroup cells), whose factors differ.
#ifndef YGS_PROJ_FLUSH_K_EXACT_MONO
#define YGS_PROJ_FLUSH_K_EXACT_MONO 128
#endif
#ifndef YGS_SYNTH_FLUSH_K
#define YGS_SYNTH_FLUSH_K 192
#endif
static_assert(kGroup % YGS_PROJ_FLUSH_K_EXACT_MONO == 0 && YGS_PROJ_FLUSH_K_EXACT_MONO % tc::BK == 0,
              "an FP16 projection flush covers whole k-blocks within one field exponent group");
static_assert(YGS_SYNTH_FLUSH_K % tc::BK == 0, "a synthesis flush covers whole k-blocks");

// k elements of one stage of the contractions: 64 two-byte or 32 TF32 values
static int kblock_elems(const ygs_plan* p) { return p->tc_tf32 ? tc::BK / 2 : tc::BK; }

static void fill_tiles(const ygs_plan* p, TcArgs& a, int n_w, int n_full, int n_tail) {
  a.err = p->d_err;
  a.ab_fmt = p->tc_tf32 ? 2 : (p->tc_fp16 ? 0 : 1);
  // flush the FP32 accumulators into the float-float sums every 64 k-elements
  // (EMU: every window of four k-blocks, whose sums are exact)
  a.flush_kb = p->tc_emu ? tc::kEmuWindowKb : std::max(1, 64 / kblock_elems(p));
  a.n_b = p->n_r;
  a.n_w = n_w;
  a.n_full = n_full;
  a.n_tail = n_tail;
  a.n_tiles = n_full + (n_tail > 0 ? 1 : 0);
}

// forward: FP16 plans take the monopole moment from the field pass (its U^T
// column is zero), so the remaining columns, whose terms change sign, flush
// every 128 k like the synthesis; BF16 plans and the adjoint keep 64
static void project_args(const ygs_plan* p, TcArgs& a, bool forward = true) {
  a = TcArgs{};
  fill_tiles(p, a, tc::kNmaxProject, p->tc_np_full, p->tc_np_tail);
  if (forward && p->tc_fp16) a.flush_kb = std::max(1, YGS_PROJ_FLUSH_K_EXACT_MONO / kblock_elems(p));
  if (!forward && p->tc_tf32) a.flush_kb = 1;  // the TF32 adjoint flushes every k-block (below)
  a.tiles_m_even = (p->tc_k_even + tc::BM - 1) / tc::BM;
  a.tiles_m = a.tiles_m_even + (p->tc_k_pad - p->tc_k_even + tc::BM - 1) / tc::BM;
  a.a_row_odd = p->tc_k_even;
  a.a_rows_total = p->tc_k_pad;
  a.b_plane_odd = p->symmetric ? p->tc_nsl : 0;
  a.n_chunks = p->tc_S;
  a.chunks = p->tc_chunks;
  a.part = p->tc_part;
  a.ldp = p->tc_k_pad;
  a.fac = (p->tc_fp16 || p->tc_emu) ? p->tc_fac : nullptr;
  a.fac_ld = fac_ld(p);
  a.fac_plane = (p->tc_n_pad / (p->tc_emu ? kEmuWindow : kGroup)) * (long long)a.fac_ld;
  a.total_tiles = a.tiles_m * a.n_chunks * a.n_tiles;
}

static cudaError_t project_with(const ygs_plan* p, const CUtensorMap& wmap, cudaStream_t s, bool forward = true) {
  TcArgs a;
  project_args(p, a, forward);
  const int grid = std::min(a.total_tiles, p->tc_sms);
  if (p->tc_emu) return emu_dispatch_gemm(tc::kProject, grid, wmap, p->tc_map_f, p->tc_map_f_tail, a, s);
  return dispatch_gemm<tc::kProject>(p->tc_nsl, a.fac != nullptr, p->tc_tf32 != 0, grid, wmap, p->tc_map_f,
                                     p->tc_map_f_tail, a, s);
}

cudaError_t tc_project(const ygs_plan* p, cudaStream_t s) { return project_with(p, p->tc_map_ut, s); }

static ScanFfArgs scan_ff_args(const ygs_plan* p) {
  const float neg_gh = (float)(-p->G);
  const float2 neg_g = make_float2(neg_gh, (float)(-p->G - (double)neg_gh));
  return ScanFfArgs{p->n_r, p->tc_k_pad, p->l_max, p->tc_S, p->tc_scan_chunk, p->tc_scan_P, p->tc_pc_l, p->tc_part,
                    p->tc_radff, p->tc_cp, p->tc_B, p->tc_M, p->tc_ms, p->tc_nsl,
                    p->tc_fp16 ? 0 : (p->tc_tf32 ? 2 : 1), neg_g, p->tc_mono, p->tc_fp16 ? p->tc_eu : nullptr,
                    p->tc_fp16 ? p->tc_mpart : nullptr};
}
static int scan_ff_blocks(const ygs_plan* p) { return (p->tc_k_pad + kScanCols - 1) / kScanCols; }
static SliceM16Args slice_m16_args(const ygs_plan* p) {
  return SliceM16Args{p->n_r, p->tc_k_pad, p->tc_M, 0, reinterpret_cast<__half*>(p->tc_ms), p->tc_em, p->tc_eq,
                      p->tc_mono, p->tc_sc};
}

cudaError_t tc_scan(const ygs_plan* p, cudaStream_t s) {
  if (p->tc_emu) return emu_scan(p, s);
  const ScanFfArgs a = scan_ff_args(p);
  scan_ff_kernel<<<scan_ff_blocks(p), kScanThreads, 0, s>>>(a.n_r, a.K_pad, a.L, a.S, a.chunk, a.P, a.pc_l, a.part,
                                                             a.rad, a.cp, a.B, a.M, a.Ms, a.nsl, a.write_slices,
                                                             a.neg_G, a.mono, a.eu, a.mpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !p->tc_fp16) return e;
  const SliceM16Args m = slice_m16_args(p);
  slice_m16_kernel<<<p->n_r, kSliceM16Threads, 0, s>>>(m.n_r, m.K_pad, m.M, m.keep_mono, m.Ms, m.em, m.q_exp, m.mono,
                                                       m.sc);
  return cudaGetLastError();
}

// pair: tiles of 2 x 128 cells for the CTA-pair kernel.
static void synth_args(const ygs_plan* p, TcArgs& a, double* phi, const float2* mono, bool pair = false) {
  a = TcArgs{};
  fill_tiles(p, a, p->tc_N, p->tc_n_full, p->tc_n_tail);
  // the forward synthesis excludes the monopole (added exactly) and may flush less
  // often; the adjoint's U has a positive monopole column and keeps 64
  a.flush_kb = p->tc_emu ? tc::kEmuWindowKb : std::max(1, (mono ? YGS_SYNTH_FLUSH_K : 64) / kblock_elems(p));
  // TF32 operands take K = 8 per MMA, so an accumulator is rounded twice as
  // often per k as with 2-byte slices: the adjoint's contractions (whose
  // synthesis sums U's positive monopole column) flush every k-block of 32 k
  if (!mono && p->tc_tf32) a.flush_kb = 1;
  a.k_even = p->symmetric ? p->tc_k_even : p->tc_k_pad;
  a.k_total = p->tc_k_pad;
  a.symmetric = p->symmetric ? 1 : 0;
  a.n_wpatch = p->n_wpatch;
  a.pt = p->pt;
  long long row = 0;
  int t = 0;
  for (int g = 0; g < p->n_wpatch; ++g) {
    a.a_row0[g] = row;
    a.tile0[g] = t;
    row += p->nang[g];
    const int cells = tc::BM * (pair ? 2 : 1);
    t += (int)((p->nang[g] + cells - 1) / cells) * a.n_tiles;  // cell tiles x shell tiles, shells fastest
  }
  a.tile0[p->n_wpatch] = t;
  a.total_tiles = t;
  a.phi = phi;
  // EMU: the monopole column is an ordinary one on the tensor cores
  a.mono = p->tc_emu ? nullptr : mono;
  a.sc = (p->tc_fp16 || p->tc_emu) ? p->tc_sc : nullptr;
}

static cudaError_t synthesize_with(const ygs_plan* p, const CUtensorMap& wmap, double* phi, const float2* mono,
                                   cudaStream_t s) {
  TcArgs a;
  const bool pair = p->tc_pairs > 0 && !p->tc_emu;
  synth_args(p, a, phi, mono, pair);
  if (pair)
    return dispatch_synth_pair(p->tc_nsl, p->tc_tf32 != 0, 2 * std::min(a.total_tiles, p->tc_pairs), wmap,
                               p->tc_map_m2, p->tc_map_m2_tail, a, s);
  const int grid = std::min(a.total_tiles, p->tc_sms);
  if (p->tc_emu) return emu_dispatch_gemm(tc::kSynthesize, grid, wmap, p->tc_map_m, p->tc_map_m_tail, a, s);
  return dispatch_gemm<tc::kSynthesize>(p->tc_nsl, false, p->tc_tf32 != 0, grid, wmap, p->tc_map_m,
                                        p->tc_map_m_tail, a, s);
}

cudaError_t tc_synthesize(const ygs_plan* p, double* phi, cudaStream_t s) {
  return synthesize_with(p, p->tc_map_q, phi, p->tc_mono, s);
}

// The adjoint: grad_phi's slices (sigma+- of the Yin/Yang rows, as the
// forward field: Q_Yang = (-1)^m Q_Yin), Mbar = grad_phi Q on the tensor
// cores, Bbar by the transposed scans, grad_rho = Bbar U^T with E +- O.  The
// monopole needs no special case here (its U column is an ordinary one).
// ev (optional) receives the phase events 1..4 after each phase.
cudaError_t tc_backward(const ygs_plan* p, const double* gphi, double* grho, cudaStream_t s, cudaEvent_t* ev) {
  cudaError_t e;
  if ((e = tc_field_slices(p, gphi, s, false)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
  if ((e = project_with(p, p->tc_map_qt, s, false)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
  if (p->tc_emu) {
    if ((e = emu_scan_adj(p, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
    return synthesize_with(p, p->tc_map_us, grho, nullptr, s);
  }
  scan_adj_ff_kernel<<<(p->tc_k_pad + kScanCols - 1) / kScanCols, kScanThreads, 0, s>>>(
      p->n_r, p->tc_k_pad, p->l_max, p->tc_S, p->tc_scan_chunk, p->tc_scan_P, p->tc_pc_l, p->tc_part, p->tc_radff,
      p->tc_Mbar, p->tc_Bbar, p->tc_ms, p->tc_nsl, p->tc_fp16 ? 0 : (p->tc_tf32 ? 2 : 1),
      p->tc_fp16 ? p->tc_eqt : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (p->tc_fp16) {
    slice_m16_kernel<<<p->n_r, kSliceM16Threads, 0, s>>>(p->n_r, p->tc_k_pad, p->tc_Bbar, 1,
                                                         reinterpret_cast<__half*>(p->tc_ms), p->tc_em, p->tc_eus,
                                                         nullptr, p->tc_sc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
  return synthesize_with(p, p->tc_map_us, grho, nullptr, s);
}

// ---- batches: the contractions of many plans in one persistent launch each ----

ygs_status tc_batch_build(TcBatch* b, const std::vector<ygs_plan*>& plans) {
  b->groups.clear();
  // one group per operand kind: BF16 two-slice, FP16 two-slice (whose
  // projection applies the field's group factors), BF16 three-slice, TF32
  // two-slice, EMU six-slice
  for (int kind = 0; kind < 5; ++kind) {
    const int nsl = kind == 4 ? tc::kEmuSlices : (kind == 2 ? 3 : 2), fp16 = kind == 1 ? 1 : 0,
              tf32 = kind == 3 ? 1 : 0, emu = kind == 4 ? 1 : 0;
    std::vector<ygs_plan*> mem;
    for (ygs_plan* p : plans)
      if (p->tc_nsl == nsl && p->tc_fp16 == fp16 && p->tc_tf32 == tf32 && p->tc_emu == emu) mem.push_back(p);
    if (mem.empty()) continue;
    if ((int)mem.size() > tc::kMaxGroup) {
      set_error("a batch holds at most 128 split-precision plans of one operand kind");
      return YGS_ERR_UNSUPPORTED;
    }
    TcBatchGroup G;
    G.nsl = nsl;
    G.fp16 = fp16;
    G.tf32 = tf32;
    G.emu = emu;
    G.members = mem;
    std::vector<tc::TcProblem> proj(mem.size()), syn(mem.size());
    std::vector<int> sp(mem.size() + 1, 0), ss(mem.size() + 1, 0);
    for (size_t k = 0; k < mem.size(); ++k) {
      const ygs_plan* p = mem[k];
      proj[k].a = p->tc_map_ut;
      proj[k].b = p->tc_map_f;
      proj[k].bt = p->tc_map_f_tail;
      project_args(p, proj[k].args);
      syn[k].a = p->tc_map_q;
      syn[k].b = p->tc_map_m;
      syn[k].bt = p->tc_map_m_tail;
      synth_args(p, syn[k].args, nullptr, p->tc_mono);  // outputs come per call
      sp[k + 1] = sp[k] + proj[k].args.total_tiles;
      ss[k + 1] = ss[k] + syn[k].args.total_tiles;
    }
    G.total_p = sp.back();
    G.total_s = ss.back();
    G.sms = mem[0]->tc_sms;
    const size_t pb = mem.size() * sizeof(tc::TcProblem), sb = (mem.size() + 1) * sizeof(int);
    cudaError_t e;
    if ((e = dev_malloc((void**)&G.d_proj, pb)) != cudaSuccess || (e = dev_malloc((void**)&G.d_synth, pb)) != cudaSuccess ||
        (e = dev_malloc((void**)&G.d_start_p, sb)) != cudaSuccess ||
        (e = dev_malloc((void**)&G.d_start_s, sb)) != cudaSuccess) {
      b->groups.push_back(G);
      set_error(std::string("batch descriptors: ") + cudaGetErrorString(e));
      return YGS_ERR_OOM;
    }
    if ((e = cudaMemcpy(G.d_proj, proj.data(), pb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(G.d_synth, syn.data(), pb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(G.d_start_p, sp.data(), sb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(G.d_start_s, ss.data(), sb, cudaMemcpyHostToDevice)) != cudaSuccess) {
      b->groups.push_back(G);
      set_error(std::string("batch descriptors: ") + cudaGetErrorString(e));
      return YGS_ERR_CUDA;
    }
    // the per-field passes (field slices, scans, M slicing), grouped the same way
    const int n = (int)mem.size();
    std::vector<int> gx(n), gy(n), gz(n), sx(n), one(n, 1), mx(n);
    for (int k = 0; k < n; ++k) {
      const dim3 d = fp16 ? field16_grid(mem[k]) : field_slices_grid(mem[k]);
      gx[k] = (int)d.x;
      gy[k] = (int)d.y;
      gz[k] = (int)d.z;
      sx[k] = scan_ff_blocks(mem[k]);
      mx[k] = mem[k]->n_r;
    }
    if (emu) {
      e = emu_batch_passes(mem, G);
    } else if (fp16) {
      std::vector<Field16Args> fa;
      std::vector<ScanFfArgs> sa;
      std::vector<SliceM16Args> ma;
      for (ygs_plan* p : mem) {
        fa.push_back(field16_args(p, true));
        sa.push_back(scan_ff_args(p));
        ma.push_back(slice_m16_args(p));
      }
      if ((e = upload_grouped_pass(G.field, fa.data(), sizeof(Field16Args), n, gx.data(), gy.data(), gz.data())) ==
              cudaSuccess &&
          (e = upload_grouped_pass(G.scan, sa.data(), sizeof(ScanFfArgs), n, sx.data(), one.data(), one.data())) ==
              cudaSuccess)
        e = upload_grouped_pass(G.mslice, ma.data(), sizeof(SliceM16Args), n, mx.data(), one.data(), one.data());
    } else {
      std::vector<ScanFfArgs> sa;
      for (ygs_plan* p : mem) sa.push_back(scan_ff_args(p));
      if (tf32) {
        std::vector<FieldSlicesTf32Args> fa;
        for (ygs_plan* p : mem) fa.push_back(field_slices_tf32_args(p));
        e = upload_grouped_pass(G.field, fa.data(), sizeof(FieldSlicesTf32Args), n, gx.data(), gy.data(), gz.data());
      } else {
        std::vector<FieldSlicesArgs> fa;
        for (ygs_plan* p : mem) fa.push_back(field_slices_args(p));
        e = upload_grouped_pass(G.field, fa.data(), sizeof(FieldSlicesArgs), n, gx.data(), gy.data(), gz.data());
      }
      if (e == cudaSuccess)
        e = upload_grouped_pass(G.scan, sa.data(), sizeof(ScanFfArgs), n, sx.data(), one.data(), one.data());
    }
    b->groups.push_back(G);
    if (e != cudaSuccess) {
      set_error(std::string("batch descriptors: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? YGS_ERR_OOM : YGS_ERR_CUDA;
    }
  }
  return YGS_OK;
}

cudaError_t upload_grouped_pass(TcGroupedPass& P, const void* args, size_t arg_bytes, int n, const int* gx,
                                const int* gy, const int* gz) {
  std::vector<tc::GroupDims> dims(n);
  int start = 0;
  for (int k = 0; k < n; ++k) {
    dims[k] = tc::GroupDims{gx[k], gy[k], gz[k], start};
    start += gx[k] * gy[k] * gz[k];
  }
  P.blocks = start;
  cudaError_t e;
  if ((e = dev_malloc(&P.d_args, std::max<size_t>(16, arg_bytes * n))) != cudaSuccess) return e;
  if ((e = dev_malloc(&P.d_dims, std::max<size_t>(16, sizeof(tc::GroupDims) * n))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(P.d_args, args, arg_bytes * n, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  return cudaMemcpy(P.d_dims, dims.data(), sizeof(tc::GroupDims) * n, cudaMemcpyHostToDevice);
}

cudaError_t tc_batch_field(const TcBatchGroup& G, const double* const* rho, cudaStream_t s) {
  if (G.emu) return emu_batch_field(G, rho, s);
  tc::RhoList list{};
  const int n = (int)G.members.size();
  for (int k = 0; k < n; ++k) list.p[k] = rho[k];
  const tc::GroupDims* dims = static_cast<const tc::GroupDims*>(G.field.d_dims);
  if (G.fp16)
    field16_kernel_group<<<G.field.blocks, kF16Threads, 0, s>>>(static_cast<const Field16Args*>(G.field.d_args), dims,
                                                                n, list);
  else if (G.tf32)
    field_slices_tf32_kernel_group<<<G.field.blocks, kFieldSlicesThreads, 0, s>>>(
        static_cast<const FieldSlicesTf32Args*>(G.field.d_args), dims, n, list);
  else
    field_slices_kernel_group<<<G.field.blocks, kFieldSlicesThreads, 0, s>>>(
        static_cast<const FieldSlicesArgs*>(G.field.d_args), dims, n, list);
  return cudaGetLastError();
}

cudaError_t tc_batch_scan(const TcBatchGroup& G, cudaStream_t s) {
  if (G.emu) return emu_batch_scan(G, s);
  const int n = (int)G.members.size();
  scan_ff_kernel_group<<<G.scan.blocks, kScanThreads, 0, s>>>(static_cast<const ScanFfArgs*>(G.scan.d_args),
                                                              static_cast<const tc::GroupDims*>(G.scan.d_dims), n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !G.fp16) return e;
  slice_m16_kernel_group<<<G.mslice.blocks, kSliceM16Threads, 0, s>>>(
      static_cast<const SliceM16Args*>(G.mslice.d_args), static_cast<const tc::GroupDims*>(G.mslice.d_dims), n);
  return cudaGetLastError();
}

void tc_batch_free(TcBatch* b) {
  for (TcBatchGroup& G : b->groups) {
    void* bufs[] = {G.d_proj,       G.d_synth,     G.d_start_p,    G.d_start_s,     G.field.d_args,
                    G.field.d_dims, G.scan.d_args, G.scan.d_dims, G.mslice.d_args, G.mslice.d_dims};
    for (void* q : bufs)
      if (q) cudaFree(q);
  }
  b->groups.clear();
}

cudaError_t tc_batch_project(const TcBatchGroup& G, cudaStream_t s) {
  tc::TcPhiList none{};
  if (G.emu)
    return emu_dispatch_group(tc::kProject, std::min(G.total_p, G.sms), G.d_proj, G.d_start_p, (int)G.members.size(),
                              G.total_p, none, s);
  return dispatch_group<tc::kProject>(G.nsl, G.fp16 != 0, G.tf32 != 0, std::min(G.total_p, G.sms), G.d_proj, G.d_start_p,
                                      (int)G.members.size(), G.total_p, none, s);
}

cudaError_t tc_batch_synthesize(const TcBatchGroup& G, double* const* phi, cudaStream_t s) {
  tc::TcPhiList out{};
  for (size_t k = 0; k < G.members.size(); ++k) out.p[k] = phi[k];
  if (G.emu)
    return emu_dispatch_group(tc::kSynthesize, std::min(G.total_s, G.sms), G.d_synth, G.d_start_s,
                              (int)G.members.size(), G.total_s, out, s);
  return dispatch_group<tc::kSynthesize>(G.nsl, false, G.tf32 != 0, std::min(G.total_s, G.sms), G.d_synth, G.d_start_s,
                                         (int)G.members.size(), G.total_s, out, s);
}

namespace {
// Waits on an mbarrier that nothing arrives at, with the same bounded polling
// as the contraction kernels, then records the timeout in the error word.
__global__ void wait_timeout_kernel(int spins, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    bool done = false;
    for (int it = 0; it < spins && !done; ++it) done = tc::mbar_try_wait(&bar, 0);
    if (!done) tc::set_err(err, YGS_ERR_TIMEOUT);
  }
}
}  // namespace

cudaError_t debug_wait_timeout(const ygs_plan* p, int spins, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(spins, p->d_err);
  return cudaGetLastError();
}

cudaError_t tc_unpermute(const ygs_plan* p, const float2* in, double* out, cudaStream_t s) {
  tc_unpermute_kernel<<<256, 256, 0, s>>>(p->n_r, p->K, p->tc_k_pad, p->tc_pc_nat, in, out);
  return cudaGetLastError();
}

// this translation unit's out-of-range record (checked builds; a no-op otherwise)
YGS_BOUNDS_READER(bounds_read_tc)

}  // namespace ygs
