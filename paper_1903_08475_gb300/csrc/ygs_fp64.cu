// FP64 (and FP32 CUDA-core) contractions and FP64 radial scans (steps 2-5 of Sect. 4.3).
//
// Projection  part[z][i][c] = sum_{a in chunk z} field(g_z, i, a) * W[a][c]
//   (Eq. B_CS; the split-K chunks z are the GPU image of the paper's
//   angular task decomposition, and their fixed-order sum is step 3).
// Synthesis   out(g, i, a) = sum_c X[i][c] * W[a][c]   (Eq. gravpotmult).
// Scans       Eq. M_C as recurrences over shells with every factor <= O(r^2):
//   I_i = a_i B_i + (r_{i-1}^+/r_i^+)^(l+1) I_{i-1},
//   O_i = b_{i+1} B_{i+1} + (r_i^+/r_{i+1}^+)^l O_{i+1},  M_i = I_i + O_i,
//   and their transposes for the adjoint.
//
// With the Yin-Yang sign symmetry (Sect. 4.2: U_Yang = (-1)^m U_Yin and
// Q_Yang = (-1)^m Q_Yin), only Yin's weights are stored, columns are ordered
// even-m first, the projection contracts (rho_Yin +- rho_Yang) against the
// even / odd column blocks, and the synthesis writes Phi_Yin = E + O and
// Phi_Yang = E - O from the even and odd partial sums: half the arithmetic.
#include <type_traits>

#include "ygs_internal.h"

namespace ygs {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// D (8x8) += A (8x4, row) B (4x8, col) on the FP64 tensor cores (DMMA).  Lane
// l holds A[l/4][l%4], B[l%4][l/4] and D[l/4][2(l%4) + {0, 1}].
__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// One BK-deep step of a 64 x 64 tile held in registers, from As[k][row] and
// Bs[k][col] in shared memory.  CUDA cores: 16 x 16 threads, 4 x 4 outputs
// each at (ty + 16 r, tx + 16 q).  Tensor cores (TC): 8 warps, each a 16 x 32
// block of 2 x 4 DMMA tiles; acc[2 mb + i][nb] is element i of the lane's pair
// in tile (mb, nb) (tile_out gives the position).  Both keep FP64 products and
// FP64 accumulation; only the order of the additions differs.
template <typename T, bool TC>
__device__ __forceinline__ void tile_step(const T (&As)[BK][BM + 1], const T (&Bs)[BK][BN + 1], T (&acc)[4][4]) {
  const int tid = threadIdx.x;
  if constexpr (TC) {
    const int lane = tid % 32, w = tid / 32, g = lane >> 2, t4 = lane & 3;
    const int wr = (w >> 1) * 16, wc = (w & 1) * 32;
#pragma unroll
    for (int k0 = 0; k0 < BK; k0 += 4) {
      T av[2], bv[4];
#pragma unroll
      for (int mb = 0; mb < 2; ++mb) av[mb] = As[k0 + t4][wr + mb * 8 + g];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) bv[nb] = Bs[k0 + t4][wc + nb * 8 + g];
#pragma unroll
      for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) dmma_8x8x4(acc[2 * mb][nb], acc[2 * mb + 1][nb], av[mb], bv[nb]);
    }
  } else {
    const int tx = tid % 16, ty = tid / 16;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
    }
  }
}

// Row and column within the 64 x 64 tile of acc[r][q].
template <bool TC>
__device__ __forceinline__ void tile_out(int r, int q, int& row, int& col) {
  const int tid = threadIdx.x;
  if (TC) {
    const int lane = tid % 32, w = tid / 32, g = lane >> 2, t4 = lane & 3;
    row = (w >> 1) * 16 + (r >> 1) * 8 + g;
    col = (w & 1) * 32 + q * 8 + 2 * t4 + (r & 1);
  } else {
    row = tid / 16 + 16 * r;
    col = tid % 16 + 16 * q;
  }
}

template <typename T>
struct ProjArgs {
  int n_r, K, K_even, tiles_e, symmetric;
  const T* field;
  const T* W;
  T* part;
  const Chunk* chunks;
  PatchTable pt;
};

template <typename T, bool TC>
__global__ void __launch_bounds__(NT) proj_fp64_kernel(ProjArgs<T> a) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tn = blockIdx.x, tm = blockIdx.y, z = blockIdx.z;
  int c0, c1;
  T sgn;
  if (tn < a.tiles_e) {
    c0 = tn * BN;
    c1 = min(a.K_even, c0 + BN);
    sgn = T(1);
  } else {
    c0 = a.K_even + (tn - a.tiles_e) * BN;
    c1 = min(a.K, c0 + BN);
    sgn = T(-1);
  }
  const int i0 = tm * BM;
  const Chunk ch = a.chunks[z];
  const long long lda = a.pt.nang[ch.g];
  const T* A0 = a.field + a.pt.fld_off[ch.g];
  const T* A1 = a.symmetric ? a.field + a.pt.fld_off[1] : nullptr;
  const T* Wg = a.W + a.pt.ang_off[ch.g] * (long long)a.K;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = T(0);

  for (int k0 = ch.a0; k0 < ch.a1; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * NT, row = e / BK, kk = e % BK;
      int i = i0 + row, k = k0 + kk;
      T v = T(0);
      if (i < a.n_r && k < ch.a1 &&
          YGS_IN_BOUNDS(a.pt.fld_off[ch.g] + i * lda + k, a.pt.n_cells, kSiteProjField) &&
          (!A1 || YGS_IN_BOUNDS(a.pt.fld_off[1] + i * lda + k, a.pt.n_cells, kSiteProjField))) {
        v = A0[i * lda + k];
        if (A1) v += sgn * A1[i * lda + k];
      }
      As[kk][row] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * NT, kk = e / BN, col = e % BN;
      int k = k0 + kk, c = c0 + col;
      Bs[kk][col] = (k < ch.a1 && c < c1 &&
                     YGS_IN_BOUNDS((a.pt.ang_off[ch.g] + k) * (long long)a.K + c, a.pt.w_rows * a.K, kSiteProjW))
                        ? Wg[(long long)k * a.K + c]
                        : T(0);
    }
    __syncthreads();
    tile_step<T, TC>(As, Bs, acc);
    __syncthreads();
  }
  T* out = a.part + (long long)z * a.n_r * a.K;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int row, col;
      tile_out<TC>(r, q, row, col);
      int i = i0 + row, c = c0 + col;
      if (i < a.n_r && c < c1 &&
          YGS_IN_BOUNDS(((long long)z * a.n_r + i) * a.K + c, (long long)gridDim.z * a.n_r * a.K, kSiteProjPart))
        out[(long long)i * a.K + c] = acc[r][q];
    }
}

template <typename T>
struct SynthArgs {
  int n_r, K, K_even, symmetric;
  const T* X;
  const T* W;
  double* out;
  PatchTable pt;
};

template <typename T, bool TC>
__device__ inline void synth_range(const SynthArgs<T>& s, const T* Wg, long long nang, int i0, int a0, int k_lo,
                                   int k_hi, T (&As)[BK][BM + 1], T (&Bs)[BK][BN + 1], T (&acc)[4][4]) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * NT, row = e / BK, kk = e % BK;
      int i = i0 + row, k = k0 + kk;
      As[kk][row] = (i < s.n_r && k < k_hi &&
                     YGS_IN_BOUNDS((long long)i * s.K + k, (long long)s.n_r * s.K, kSiteSynthX))
                        ? s.X[(long long)i * s.K + k]
                        : T(0);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * NT, n = e / BK, kk = e % BK;
      int a = a0 + n, k = k0 + kk;
      Bs[kk][n] = (a < nang && k < k_hi &&
                   YGS_IN_BOUNDS((Wg - s.W) + (long long)a * s.K + k, s.pt.w_rows * s.K, kSiteSynthW))
                      ? Wg[(long long)a * s.K + k]
                      : T(0);
    }
    __syncthreads();
    tile_step<T, TC>(As, Bs, acc);
    __syncthreads();
  }
}

template <typename T, bool TC>
__global__ void __launch_bounds__(NT) synth_fp64_kernel(SynthArgs<T> s) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int g = blockIdx.z;
  const long long nang = s.pt.nang[g];
  const int a0 = blockIdx.x * BN;
  if (a0 >= nang) return;
  const int i0 = blockIdx.y * BM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const T* Wg = s.W + s.pt.ang_off[g] * (long long)s.K;
  T ae[4][4], ao[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) ae[r][q] = ao[r][q] = T(0);
  synth_range<T, TC>(s, Wg, nang, i0, a0, 0, s.K_even, As, Bs, ae);
  if (s.K_even < s.K) synth_range<T, TC>(s, Wg, nang, i0, a0, s.K_even, s.K, As, Bs, ao);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int row, col;
      tile_out<TC>(r, q, row, col);
      int i = i0 + row;
      long long a = a0 + col;
      if (i >= s.n_r || a >= nang) continue;
      if (s.symmetric) {
        if (YGS_IN_BOUNDS(s.pt.fld_off[0] + i * nang + a, s.pt.n_cells, kSiteSynthPhi))
          s.out[s.pt.fld_off[0] + i * nang + a] = (double)(ae[r][q] + ao[r][q]);
        if (YGS_IN_BOUNDS(s.pt.fld_off[1] + i * nang + a, s.pt.n_cells, kSiteSynthPhi))
          s.out[s.pt.fld_off[1] + i * nang + a] = (double)(ae[r][q] - ao[r][q]);
      } else {
        if (YGS_IN_BOUNDS(s.pt.fld_off[g] + i * nang + a, s.pt.n_cells, kSiteSynthPhi))
          s.out[s.pt.fld_off[g] + i * nang + a] = (double)(ae[r][q] + ao[r][q]);
      }
    }
}

template <typename T>
__global__ void scan_fwd_kernel(int n_r, int K, int L, const int* __restrict__ col_l, const T* __restrict__ part,
                                int S, const double* __restrict__ rad, double* __restrict__ B, double* __restrict__ M) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K) return;
  const int l = col_l[c];
  const long long plane = (long long)n_r * K, rs = (long long)(L + 1) * n_r;
  // the column's radial tables and its last element of the partials
  if (!YGS_IN_BOUNDS(l, L + 1, kSiteScanFwd) || !YGS_IN_BOUNDS((S - 1) * plane + plane - K + c, S * plane, kSiteScanFwd))
    return;
  const double* at = rad + (long long)l * n_r;
  const double* bt = rad + rs + (long long)l * n_r;
  const double* fin = rad + 2 * rs + (long long)l * n_r;
  const double* fout = rad + 3 * rs + (long long)l * n_r;
  for (int i = 0; i < n_r; ++i) {
    double b = 0.0;
    for (int z = 0; z < S; ++z) b += (double)part[z * plane + (long long)i * K + c];
    B[(long long)i * K + c] = b;
  }
  double O = 0.0;
  M[(long long)(n_r - 1) * K + c] = 0.0;
  for (int i = n_r - 2; i >= 0; --i) {
    O = fma(bt[i + 1], B[(long long)(i + 1) * K + c], fout[i] * O);
    M[(long long)i * K + c] = O;
  }
  double I = 0.0;
  for (int i = 0; i < n_r; ++i) {
    I = fma(at[i], B[(long long)i * K + c], fin[i] * I);
    M[(long long)i * K + c] += I;
  }
}

__global__ void scan_adj_kernel(int n_r, int K, int L, const int* __restrict__ col_l, const double* __restrict__ part,
                                int S, const double* __restrict__ rad, double* __restrict__ Mb,
                                double* __restrict__ Bb) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K) return;
  const int l = col_l[c];
  const long long plane = (long long)n_r * K, rs = (long long)(L + 1) * n_r;
  if (!YGS_IN_BOUNDS(l, L + 1, kSiteScanAdj) || !YGS_IN_BOUNDS((S - 1) * plane + plane - K + c, S * plane, kSiteScanAdj))
    return;
  const double* at = rad + (long long)l * n_r;
  const double* bt = rad + rs + (long long)l * n_r;
  const double* fin = rad + 2 * rs + (long long)l * n_r;
  const double* fout = rad + 3 * rs + (long long)l * n_r;
  for (int i = 0; i < n_r; ++i) {
    double v = 0.0;
    for (int z = 0; z < S; ++z) v += part[z * plane + (long long)i * K + c];
    Mb[(long long)i * K + c] = v;
  }
  // X_i = Mb_i + (r_i^+/r_{i+1}^+)^(l+1) X_{i+1};  Bbar_i = a_i X_i + ...
  double X = 0.0;
  for (int i = n_r - 1; i >= 0; --i) {
    X = Mb[(long long)i * K + c] + ((i + 1 < n_r) ? fin[i + 1] * X : 0.0);
    Bb[(long long)i * K + c] = at[i] * X;
  }
  // Y_i = Mb_{i-1} + (r_{i-2}^+/r_{i-1}^+)^l Y_{i-1};  ... + b_i Y_i
  double Y = 0.0;
  for (int i = 1; i < n_r; ++i) {
    Y = Mb[(long long)(i - 1) * K + c] + ((i >= 2) ? fout[i - 2] * Y : 0.0);
    Bb[(long long)i * K + c] += bt[i] * Y;
  }
}

// B[i][c] = sum_{z < S} part[z][i][c], in order of z
__global__ void sum_partials_kernel(long long plane, int S, const double* __restrict__ part, double* __restrict__ B) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < plane; e += (long long)gridDim.x * blockDim.x) {
    double b = 0.0;
    for (int z = 0; z < S; ++z) b += part[z * plane + e];
    B[e] = b;
  }
}

// out[i][c] = in[i][col_nat[c]]: natural column order -> internal
__global__ void permute_kernel(int n_r, int K, const int* __restrict__ col_nat, const double* __restrict__ in,
                               double* __restrict__ out) {
  long long total = (long long)n_r * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / K;
    int c = (int)(e % K);
    out[e] = in[i * K + col_nat[c]];
  }
}

__global__ void unpermute_kernel(int n_r, int K, const int* __restrict__ col_nat, const double* __restrict__ in,
                                 double* __restrict__ out) {
  long long total = (long long)n_r * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / K;
    int c = (int)(e % K);
    out[i * K + col_nat[c]] = in[e];
  }
}

}  // namespace

namespace {

// Chunks [z0, z0 + nz) of the plan's list (all of them by default) into part[0 .. nz).
template <typename T>
cudaError_t project_t(const ygs_plan* p, const T* field, const T* W, T* part, bool tc, cudaStream_t s, int z0 = 0,
                      int nz = -1) {
  if (nz < 0) nz = p->S - z0;
  ProjArgs<T> a;
  a.n_r = p->n_r;
  a.K = p->K;
  a.K_even = p->K_even;
  a.tiles_e = (p->K_even + BN - 1) / BN;
  a.symmetric = p->symmetric ? 1 : 0;
  a.field = field;
  a.W = W;
  a.part = part;
  a.chunks = p->chunks + z0;
  a.pt = p->pt;
  int tiles_o = (p->K - p->K_even + BN - 1) / BN;
  dim3 grid(a.tiles_e + tiles_o, (p->n_r + BM - 1) / BM, nz);
  if constexpr (std::is_same<T, double>::value) {
    if (tc) {
      proj_fp64_kernel<T, true><<<grid, NT, 0, s>>>(a);
      return cudaGetLastError();
    }
  }
  proj_fp64_kernel<T, false><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t synth_t(const ygs_plan* p, const T* X, const T* W, double* out, bool tc, cudaStream_t s) {
  SynthArgs<T> a;
  a.n_r = p->n_r;
  a.K = p->K;
  a.K_even = p->K_even;
  a.symmetric = p->symmetric ? 1 : 0;
  a.X = X;
  a.W = W;
  a.out = out;
  a.pt = p->pt;
  long long nmax = 0;
  for (int g = 0; g < p->n_wpatch; ++g) nmax = std::max(nmax, p->nang[g]);
  dim3 grid((unsigned)((nmax + BN - 1) / BN), (p->n_r + BM - 1) / BM, p->n_wpatch);
  if constexpr (std::is_same<T, double>::value) {
    if (tc) {
      synth_fp64_kernel<T, true><<<grid, NT, 0, s>>>(a);
      return cudaGetLastError();
    }
  }
  synth_fp64_kernel<T, false><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

// FP64 -> FP32: round to nearest for the weights (once per plan), truncation
// by integer operations for per-solve data (GB300 converts FP64 on its narrow
// FP64 pipe); exponents outside FP32's normal range flush to zero / infinity.
__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, long long n, int trunc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double x = in[e];
    if (!trunc) {
      out[e] = __double2float_rn(x);
      continue;
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const int ex = (int)((b >> 52) & 0x7FF) - 1023;
    out[e] = ex < -126 ? __int_as_float((int)sign)
                       : ex > 127 ? __int_as_float((int)(sign | 0x7F800000u))
                                  : __int_as_float((int)(sign | ((unsigned int)(ex + 127) << 23) |
                                                         (unsigned int)((b >> 29) & 0x7FFFFFu)));
  }
}

}  // namespace

cudaError_t launch_project_fp64(const ygs_plan* p, const double* field, const double* W, double* part,
                                cudaStream_t s) {
  return project_t<double>(p, field, W, part, p->precision == YGS_FP64_TC, s);
}

cudaError_t launch_synth_fp64(const ygs_plan* p, const double* X, const double* W, double* out, cudaStream_t s) {
  return synth_t<double>(p, X, W, out, p->precision == YGS_FP64_TC, s);
}

cudaError_t preload_fp64_kernels() {
  // cudaFuncGetAttributes loads a lazily loaded kernel (and its module) now
  cudaFuncAttributes fa;
  cudaError_t e;
  if ((e = cudaFuncGetAttributes(&fa, proj_fp64_kernel<double, false>)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&fa, proj_fp64_kernel<double, true>)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&fa, synth_fp64_kernel<double, false>)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&fa, synth_fp64_kernel<double, true>)) != cudaSuccess) return e;
  return cudaFuncGetAttributes(&fa, scan_fwd_kernel<double>);
}

cudaError_t launch_scan_fwd(const ygs_plan* p, const double* part, int S, double* B, double* M, cudaStream_t s) {
  scan_fwd_kernel<double><<<(p->K + 63) / 64, 64, 0, s>>>(p->n_r, p->K, p->l_max, p->col_l, part, S, p->rad, B, M);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* in, float* out, long long n, bool trunc, cudaStream_t s) {
  to_f32_kernel<<<(int)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(in, out, n, trunc ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t solve_fp32(const ygs_plan* p, const double* rho, double* phi, cudaStream_t s, cudaEvent_t* ev) {
  cudaError_t e;
  if ((e = launch_to_f32(rho, p->f32_field, p->n_cells, true, s)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
  if ((e = project_t<float>(p, p->f32_field, p->U32, p->part32, false, s)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
  scan_fwd_kernel<float><<<(p->K + 63) / 64, 64, 0, s>>>(p->n_r, p->K, p->l_max, p->col_l, p->part32, p->S, p->rad,
                                                         p->B, p->M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_to_f32(p->M, p->M32, (long long)p->n_r * p->K, false, s)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
  return synth_t<float>(p, p->M32, p->Q32, phi, false, s);
}

cudaError_t launch_scan_adj(const ygs_plan* p, const double* part, int S, double* Bbar, cudaStream_t s) {
  scan_adj_kernel<<<(p->K + 63) / 64, 64, 0, s>>>(p->n_r, p->K, p->l_max, p->col_l, part, S, p->rad, p->Mbar, Bbar);
  return cudaGetLastError();
}

cudaError_t launch_project_fp64_chunks(const ygs_plan* p, const double* field, const double* W, double* part, int z0,
                                      int z1, cudaStream_t s) {
  return project_t<double>(p, field, W, part, p->precision == YGS_FP64_TC, s, z0, z1 - z0);
}

cudaError_t launch_sum_partials(const ygs_plan* p, const double* part, int S, double* B, cudaStream_t s) {
  sum_partials_kernel<<<256, 256, 0, s>>>((long long)p->n_r * p->K, S, part, B);
  return cudaGetLastError();
}

cudaError_t launch_permute(const ygs_plan* p, const double* in, double* out, cudaStream_t s) {
  permute_kernel<<<256, 256, 0, s>>>(p->n_r, p->K, p->col_nat, in, out);
  return cudaGetLastError();
}

cudaError_t launch_unpermute(const ygs_plan* p, const double* in, double* out, cudaStream_t s) {
  unpermute_kernel<<<256, 256, 0, s>>>(p->n_r, p->K, p->col_nat, in, out);
  return cudaGetLastError();
}

// this translation unit's out-of-range record (checked builds; a no-op otherwise)
YGS_BOUNDS_READER(bounds_read_fp64)

}  // namespace ygs
