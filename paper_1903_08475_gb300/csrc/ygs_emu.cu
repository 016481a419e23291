// FP64-accurate solves on the BF16 tensor cores (YGS_FP64_EMU).
//
// The contractions of Eqs. B_CS (projection) and gravpotmult (synthesis) are
// done in the Ozaki manner.  Every FP64 operand value x on a row (or row and
// window) with |x| < 2^e is rounded to the integer N = round(x 2^(47-e)),
// |N| <= 2^47, and N is written in six balanced base-256 digits,
//   N = sum_{i<6} d_i 256^(5-i),   |d_i| <= 128,
// so x = 2^e sum_i d_i 2^(-7-8i) + r with |r| <= 2^(e-48); each
// d_i 2^(e-7-8i) is one BF16 value, exactly.  The 26 products of digits with
// s + t <= 6 are summed on the tensor cores: a dropped product (s + t >= 7)
// is below 2^-56 of the two rows' scales and of either sign, so they do not
// pile up along k.  Within a flush window of 1024 k-elements one product's
// terms are integers of magnitude at most 2^14 on a common grid, so their
// FP32 sum is exact and only the float-float flushes round.  The radial
// scans (Eq. M_C, Sect. 4.3 step 4) run in FP64.
//
// Grids: the weights U^T, Q (and the adjoint's Q^T, U) per row of the
// contraction, over the whole k range; the field per (plane, shell, window of
// 1024 angular cells), from the largest |sigma| of the window (sigma+- are
// formed exactly first), scaled by 2^-e with the factor 2^e applied at the
// flush; M (and the adjoint's Bbar) per shell, scaled by 2^-e and unscaled in
// FP64 at the synthesis output.  All fixed-point conversions are integer
// operations on the FP64 bit patterns (no FP64 arithmetic).
#include "ygs_tc_gemm.cuh"

namespace ygs {

namespace {

constexpr int kS = tc::kEmuSlices;
static_assert(kEmuWindow == tc::kEmuWindowKb * tc::BK, "a field window is one flush group");

// Biased exponent field of a double (0 for zeros and subnormals, which the
// splitting treats as zero: they lie below 2^-1022).
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// round(|x| 2^(bits - e)) (half up) for |x| < 2^e, by shifting the
// significand: the shift 1075 - bits + e - bexp(x) is at least 0 for
// bits <= 53 (then the result is at most 2^bits).
__device__ __forceinline__ long long fixed_mag(double x, int e, int bits) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int bx = (int)((u >> 52) & 0x7FF);
  if (bx == 0) return 0;
  const int rs = 1075 - bits + e - bx;
  if (rs >= 64) return 0;
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  return (long long)(rs == 0 ? m : (m + (1ull << (rs - 1))) >> rs);
}
__device__ __forceinline__ long long fixed_signed(double x, int e, int bits) {
  const long long n = fixed_mag(x, e, bits);
  return x < 0.0 ? -n : n;
}

// Balanced base-256 digits of |N| <= 2^47: d[5] .. d[1] in [-128, 127], d[0]
// in [-128, 128].
__device__ __forceinline__ void bal_digits(long long N, int (&d)[kS]) {
#pragma unroll
  for (int i = kS - 1; i > 0; --i) {
    const int r = (int)((N + 128) & 255) - 128;
    d[i] = r;
    N = (N - r) >> 8;  // exact: N - r is a multiple of 256
  }
  d[0] = (int)N;
}

// BF16 bits of d * 2^(-7-8i) (|d| <= 128: at most eight significant bits, so
// the top half of the FP32 value is the BF16 value exactly).
__device__ __forceinline__ uint16_t digit_bf16(int d, int i) {
  const float f = (float)d * __int_as_float((127 - 7 - 8 * i) << 23);
  return (uint16_t)(__float_as_uint(f) >> 16);
}

// The BF16 value d * 2^(e-7-8i) (weights keep their magnitude; below BF16's
// normal range the value rounds, a change below 2^-126).
__device__ __forceinline__ __nv_bfloat16 digit_bf16_at(int d, int i, int e) {
  return __double2bfloat16((double)d * ldexp(1.0, e - 7 - 8 * i));
}

__device__ __forceinline__ unsigned int block_max_u(unsigned int v, unsigned int* red) {
  v = __reduce_max_sync(0xffffffffu, v);
  const int wid = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  unsigned int m = 0;
  for (int k = 0; k < nw; ++k) m = max(m, red[k]);
  return m;
}

// Grid exponent of a set whose largest biased exponent is bmax: |x| < 2^e.
__device__ __forceinline__ int grid_exp(unsigned int bmax) { return bmax == 0 ? 0 : (int)bmax - 1022; }

// ---- weights (at create) ---------------------------------------------------

// ecol[pc]: grid exponent of column ci = pc_int[pc] of W (all rows).
__global__ void emu_col_exp_kernel(int K, const int* __restrict__ pc_int, long long rows,
                                   const double* __restrict__ W, int* __restrict__ ecol) {
  __shared__ unsigned int red[32];
  const int pc = blockIdx.x, ci = pc_int[pc];
  unsigned int b = 0;
  if (ci >= 0)
    for (long long a = threadIdx.x; a < rows; a += blockDim.x) b = max(b, (unsigned int)bexp(W[a * K + ci]));
  b = block_max_u(b, red);
  if (threadIdx.x == 0) ecol[pc] = grid_exp(b);
}

// Ut[s][pc][apad] from W[row][ci] on the column grids ecol (the projection's
// A operand: rows are the padded columns pc, k the padded angular cells).
__global__ void emu_slice_ut_kernel(int K, int K_pad, long long n_pad, const int* __restrict__ pc_int,
                                    const double* __restrict__ W, PatchTable pt, int nwp,
                                    const long long* __restrict__ pad_off, const int* __restrict__ ecol,
                                    __nv_bfloat16* __restrict__ Ut) {
  const long long total = (long long)K_pad * n_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int pc = (int)(e / n_pad);
    const long long ap = e % n_pad;
    int g = 0;
    while (g + 1 < nwp && pad_off[g + 1] <= ap) ++g;
    const long long a = ap - pad_off[g];
    const int ci = pc_int[pc];
    double x = 0.0;
    if (ci >= 0 && a < pt.nang[g]) x = W[(pt.ang_off[g] + a) * K + ci];
    const int ex = ecol[pc];
    int d[kS];
    bal_digits(fixed_signed(x, ex, 47), d);
#pragma unroll
    for (int i = 0; i < kS; ++i) Ut[(long long)i * total + e] = digit_bf16_at(d[i], i, ex);
  }
}

// Ws[s][row][pc] from W[row][ci] on per-row grids (the synthesis's A
// operand), one warp per row.
__global__ void emu_slice_rows_kernel(int K, int K_pad, long long rows, const int* __restrict__ pc_int,
                                      const double* __restrict__ W, __nv_bfloat16* __restrict__ Ws) {
  const int lane = threadIdx.x % 32;
  const long long total = rows * K_pad;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; row < rows;
       row += (long long)gridDim.x * blockDim.x / 32) {
    const double* wr = W + row * K;
    unsigned int b = 0;
    for (int c = lane; c < K; c += 32) b = max(b, (unsigned int)bexp(wr[c]));
    const int ex = grid_exp(__reduce_max_sync(0xffffffffu, b));
    for (int pc = lane; pc < K_pad; pc += 32) {
      const int ci = pc_int[pc];
      const double x = ci >= 0 ? wr[ci] : 0.0;
      int d[kS];
      bal_digits(fixed_signed(x, ex, 47), d);
#pragma unroll
      for (int i = 0; i < kS; ++i) Ws[(long long)i * total + row * K_pad + pc] = digit_bf16_at(d[i], i, ex);
    }
  }
}

// ---- field (every solve) -----------------------------------------------------

__device__ __forceinline__ int bit_length(long long v) {
  const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
  return 64 - __clzll((long long)a);
}

// Rounds |v| / 2^r (half up), keeping the sign; r >= 0.
__device__ __forceinline__ long long shift_round(long long v, int r) {
  if (r == 0) return v;
  if (r >= 63) return 0;
  const long long a = v < 0 ? -v : v;
  const long long q = (a + (1ll << (r - 1))) >> r;
  return v < 0 ? -q : q;
}

constexpr int kFieldThreads = 256;
static_assert(kEmuWindow == 4 * kFieldThreads, "four cells per thread");

// F[(h * 6 + s)][i][pad] and fac[h][G][i].  One CTA per (window G of 1024
// padded cells, shell i); thread t takes the cells 4t .. 4t + 3.  The window's
// largest biased exponent of rho_Yin, rho_Yang gives Ef with |rho| < 2^Ef;
// both become integers on the grid 2^(Ef-53) (exact for the largest
// binade), sigma+- (or rho) their exact sum and difference (|sigma| <= 2^54).
// Per plane, the largest |sigma| of the window fixes a right shift r that
// brings the plane to |sigma'| <= 2^47 (rounded), whose balanced digits are the
// slices, with the factor 2^(Ef-6+r).  Factors are kept within FP32's normal
// range (a window whose largest value is below about 2^-120 keeps fewer
// bits; one at or above 2^127 sets the error word: the FP32 sums of the
// contraction could not hold it).
__device__ __forceinline__ void emu_field_kernel_body(const tc::VBlock& vb, 
    int n_r, int symmetric, int nwp, const PatchTable& pt, const long long* __restrict__ pad_off, long long n_pad,
    const double* __restrict__ rho, uint16_t* __restrict__ F, float* __restrict__ fac, int fac_ld,
    int* __restrict__ err) {
  __shared__ unsigned int red[32];
  const long long G = vb.x;
  const int i = vb.y;
  const long long plane = (long long)n_r * n_pad;
  const long long nwin_all = n_pad / kEmuWindow;
  const long long ap = G * kEmuWindow;  // first padded cell of the window
  int g = 0;
  while (g + 1 < nwp && pad_off[g + 1] <= ap) ++g;
  const long long na = pt.nang[g];
  const double* x0p = rho + pt.fld_off[g] + (long long)i * na;
  const double* x1p = symmetric ? rho + pt.fld_off[1] + (long long)i * na : x0p;
  const long long c = ap - pad_off[g] + 4 * threadIdx.x;  // this thread's first cell in patch g
  double x0[4], x1[4];
  const bool vec = ((reinterpret_cast<uintptr_t>(x0p) | reinterpret_cast<uintptr_t>(x1p)) & 15) == 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) x0[d] = x1[d] = 0.0;
  bool in = true;  // checked builds: this thread's cells of both rows lie in the field
#if YGS_DEBUG_BOUNDS
  {
    const long long nv = na - c < 4 ? na - c : 4;
    const long long r0 = pt.fld_off[g] + (long long)i * na + c, r1 = (symmetric ? pt.fld_off[1] : pt.fld_off[g]) + (long long)i * na + c;
    if (nv > 0)
      in = YGS_IN_BOUNDS(r0, pt.n_cells, kSiteEmuFieldRho) && YGS_IN_BOUNDS(r0 + nv - 1, pt.n_cells, kSiteEmuFieldRho) &&
           YGS_IN_BOUNDS(r1, pt.n_cells, kSiteEmuFieldRho) && YGS_IN_BOUNDS(r1 + nv - 1, pt.n_cells, kSiteEmuFieldRho);
  }
#endif
  if (!in) {
  } else if (vec && c + 4 <= na) {
    const double2 a0 = *reinterpret_cast<const double2*>(x0p + c), a1 = *reinterpret_cast<const double2*>(x0p + c + 2);
    x0[0] = a0.x; x0[1] = a0.y; x0[2] = a1.x; x0[3] = a1.y;
    if (symmetric) {
      const double2 b0 = *reinterpret_cast<const double2*>(x1p + c), b1 = *reinterpret_cast<const double2*>(x1p + c + 2);
      x1[0] = b0.x; x1[1] = b0.y; x1[2] = b1.x; x1[3] = b1.y;
    }
  } else {
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (c + d < na) {
        x0[d] = x0p[c + d];
        if (symmetric) x1[d] = x1p[c + d];
      }
    }
  }
  unsigned int b = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) b = max(b, (unsigned int)max(bexp(x0[d]), bexp(x1[d])));
  b = block_max_u(b, red);
  const int Ef = grid_exp(b);
  long long sg[2][4];
  unsigned int len0 = 0, len1 = 0;  // bit lengths of the planes' largest |sigma|
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const long long a = fixed_signed(x0[d], Ef, 53), bb = fixed_signed(x1[d], Ef, 53);
    sg[0][d] = a + bb;
    sg[1][d] = a - bb;
    len0 = max(len0, (unsigned int)bit_length(sg[0][d]));
    len1 = max(len1, (unsigned int)bit_length(sg[1][d]));
  }
  const unsigned int l0 = block_max_u(len0, red), l1 = block_max_u(len1, red);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h == 1 && !symmetric) break;
    const int L = h ? (int)l1 : (int)l0;
    int r = L > 47 ? L - 47 : 0;
    int fe = Ef - 6 + r;
    if (b == 0) {  // an all-zero window: zero digits
      r = 0;
      fe = -126;
    } else if (fe < -126) {
      r += -126 - fe;
      fe = -126;
    }
    if (fe > 127) {
      if (threadIdx.x == 0) atomicCAS(err, 0, (int)YGS_ERR_NUMERIC);
      fe = 127;
    }
    if (threadIdx.x == 0) fac[((long long)h * nwin_all + G) * fac_ld + i] = __int_as_float((127 + fe) << 23);
    int dg[4][kS];
#pragma unroll
    for (int d = 0; d < 4; ++d) bal_digits(shift_round(sg[h][d], r), dg[d]);
    uint16_t* out = F + (long long)(h * kS) * plane + (long long)i * n_pad + ap + 4 * threadIdx.x;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const uint32_t w0 = (uint32_t)digit_bf16(dg[0][s], s) | ((uint32_t)digit_bf16(dg[1][s], s) << 16);
      const uint32_t w1 = (uint32_t)digit_bf16(dg[2][s], s) | ((uint32_t)digit_bf16(dg[3][s], s) << 16);
      const long long oi = (long long)(h * kS + s) * plane + (long long)i * n_pad + ap + 4 * threadIdx.x;
      (void)oi;
      if (YGS_IN_BOUNDS(oi + 3, (long long)(symmetric ? 2 : 1) * kS * plane, kSiteEmuFieldOut))
        *reinterpret_cast<uint2*>(out + (long long)s * plane) = make_uint2(w0, w1);  // 8-byte aligned
    }
  }
}
__global__ void __launch_bounds__(256) emu_field_kernel(
    int n_r, int symmetric, int nwp, PatchTable pt, const long long* __restrict__ pad_off, long long n_pad,
    const double* __restrict__ rho, uint16_t* __restrict__ F, float* __restrict__ fac, int fac_ld,
    int* __restrict__ err) {
  emu_field_kernel_body(tc::vblock_self(), n_r, symmetric, nwp, pt, pad_off, n_pad, rho, F, fac, fac_ld, err);
}

// The arguments of emu_field_kernel but the field, for a grouped launch.
struct EmuFieldArgs {
  int n_r;
  int symmetric;
  int nwp;
  PatchTable pt;
  const long long* pad_off;
  long long n_pad;
  uint16_t* F;
  float* fac;
  int fac_ld;
  int* err;
};

// emu_field_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(256) emu_field_kernel_group(const EmuFieldArgs* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n, const __grid_constant__ tc::RhoList rhos) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const EmuFieldArgs& a = probs[k];
  const double* rho = rhos.p[k];
  emu_field_kernel_body(vb, a.n_r, a.symmetric, a.nwp, a.pt, a.pad_off, a.n_pad, rho, a.F, a.fac, a.fac_ld, a.err);
}


// ---- radial scans (every solve), FP64 ----------------------------------------
// One warp per padded column; lane p owns the shells [p c, (p + 1) c), c =
// ceil(n_r / 32).  A first-order recurrence x_i = c_i + f_i x_(i -+ 1) is
// solved per lane from a zero carry, the lanes' affine maps (x_end = b + A
// x_in) are joined by a shuffle scan, and each lane redoes its shells from
// its true carry.  Every step is an FP64 FMA.

// Inclusive scan of the lanes' maps toward higher lanes (upward recurrences):
// lane p ends with the composition of lanes 0..p.
__device__ __forceinline__ void aff_scan_up(double& A, double& b, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double Ao = __shfl_up_sync(0xffffffffu, A, d), bo = __shfl_up_sync(0xffffffffu, b, d);
    if (lane >= d) {
      b = fma(A, bo, b);
      A *= Ao;
    }
  }
}
// The same toward lower lanes (downward recurrences): lane p ends with lanes p..31.
__device__ __forceinline__ void aff_scan_down(double& A, double& b, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double Ao = __shfl_down_sync(0xffffffffu, A, d), bo = __shfl_down_sync(0xffffffffu, b, d);
    if (lane + d < 32) {
      b = fma(A, bo, b);
      A *= Ao;
    }
  }
}

constexpr int kScanWarps = 8;  // columns per CTA

// B_i = sum_z part[z][i][pc] (float-float pairs, summed in FP64); the outer
// and inner scaled recurrences of Eq. M_C, M = O + I:
//   O_i = b_(i+1) B_(i+1) + f_out,i O_(i+1)  (O_(n-1) = 0),
//   I_i = a_i B_i + f_in,i I_(i-1)            (I_(-1) = 0).
__device__ __forceinline__ void emu_scan_kernel_body(const tc::VBlock& vb, 
    int n_r, int K_pad, int L, int S, const int* __restrict__ pc_l, const float2* __restrict__ part,
    const double* __restrict__ rad, double* __restrict__ B, double* __restrict__ M, float2* __restrict__ Bff,
    float2* __restrict__ Mff) {
  const int lane = threadIdx.x % 32;
  const int c = vb.x * kScanWarps + threadIdx.x / 32;
  if (c >= K_pad) return;  // warp-uniform
  const int l = pc_l[c];
  const long long plane = (long long)n_r * K_pad;
  const int ch = (n_r + 31) / 32, i0 = min(n_r, lane * ch), i1 = min(n_r, i0 + ch);
  if (l < 0) {
    for (int i = i0; i < i1; ++i) {
      B[(long long)i * K_pad + c] = M[(long long)i * K_pad + c] = 0.0;
      Bff[(long long)i * K_pad + c] = Mff[(long long)i * K_pad + c] = make_float2(0.0f, 0.0f);
    }
    return;
  }
  // the column's radial tables and its last partial (warp-uniform: one column per warp)
  if (!YGS_IN_BOUNDS(l, L + 1, kSiteEmuScan) || !YGS_IN_BOUNDS((S - 1) * plane + plane - K_pad + c, S * plane, kSiteEmuScan))
    return;
  const long long rs = (long long)(L + 1) * n_r;
  const double* at = rad + (long long)l * n_r;
  const double* bt = rad + rs + (long long)l * n_r;
  const double* fin = rad + 2 * rs + (long long)l * n_r;
  const double* fout = rad + 3 * rs + (long long)l * n_r;
  for (int i = i0; i < i1; ++i) {
    double b = 0.0;
    for (int z = 0; z < S; ++z) {
      const float2 v = part[z * plane + (long long)i * K_pad + c];
      b += (double)v.x + (double)v.y;
    }
    B[(long long)i * K_pad + c] = b;
    Bff[(long long)i * K_pad + c] = tc::ff_from_f64(b);
  }
  __syncwarp();  // the next shell's B, read below, may belong to the lane above
  // outer (downward): the step at i reads B_(i+1)
  auto oc = [&](int i) { return i + 1 < n_r ? bt[i + 1] * B[(long long)(i + 1) * K_pad + c] : 0.0; };
  auto of = [&](int i) { return i + 1 < n_r ? fout[i] : 0.0; };
  double A = 1.0, x = 0.0;
  for (int i = i1 - 1; i >= i0; --i) {
    x = fma(of(i), x, oc(i));
    A *= of(i);
  }
  aff_scan_down(A, x, lane);
  double carry = __shfl_down_sync(0xffffffffu, x, 1);
  if (lane == 31) carry = 0.0;
  x = carry;
  for (int i = i1 - 1; i >= i0; --i) {
    x = fma(of(i), x, oc(i));
    M[(long long)i * K_pad + c] = x;
  }
  // inner (upward)
  A = 1.0;
  x = 0.0;
  for (int i = i0; i < i1; ++i) {
    x = fma(fin[i], x, at[i] * B[(long long)i * K_pad + c]);
    A *= fin[i];
  }
  aff_scan_up(A, x, lane);
  carry = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) carry = 0.0;
  x = carry;
  for (int i = i0; i < i1; ++i) {
    x = fma(fin[i], x, at[i] * B[(long long)i * K_pad + c]);
    const double m = M[(long long)i * K_pad + c] + x;
    M[(long long)i * K_pad + c] = m;
    Mff[(long long)i * K_pad + c] = tc::ff_from_f64(m);
  }
}
__global__ void __launch_bounds__(32 * kScanWarps) emu_scan_kernel(
    int n_r, int K_pad, int L, int S, const int* __restrict__ pc_l, const float2* __restrict__ part,
    const double* __restrict__ rad, double* __restrict__ B, double* __restrict__ M, float2* __restrict__ Bff,
    float2* __restrict__ Mff) {
  emu_scan_kernel_body(tc::vblock_self(), n_r, K_pad, L, S, pc_l, part, rad, B, M, Bff, Mff);
}

// The arguments of emu_scan_kernel but the field, for a grouped launch.
struct EmuScanArgs {
  int n_r;
  int K_pad;
  int L;
  int S;
  const int* pc_l;
  const float2* part;
  const double* rad;
  double* B;
  double* M;
  float2* Bff;
  float2* Mff;
};

// emu_scan_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(32 * kScanWarps) emu_scan_kernel_group(const EmuScanArgs* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const EmuScanArgs& a = probs[k];
  emu_scan_kernel_body(vb, a.n_r, a.K_pad, a.L, a.S, a.pc_l, a.part, a.rad, a.B, a.M, a.Bff, a.Mff);
}


// The transposed scans: Mbar_i = sum_z part[z][i][pc], then
//   X_i = Mbar_i + f_in,(i+1) X_(i+1)      (X_n = 0),
//   Y_i = Mbar_(i-1) + f_out,(i-2) Y_(i-1)  (Y_0 = 0, Y_1 = Mbar_0),
//   Bbar_i = a_i X_i + b_i Y_i.
__global__ void __launch_bounds__(32 * kScanWarps) emu_scan_adj_kernel(
    int n_r, int K_pad, int L, int S, const int* __restrict__ pc_l, const float2* __restrict__ part,
    const double* __restrict__ rad, double* __restrict__ Mb, double* __restrict__ Bb) {
  const int lane = threadIdx.x % 32;
  const int c = blockIdx.x * kScanWarps + threadIdx.x / 32;
  if (c >= K_pad) return;  // warp-uniform
  const int l = pc_l[c];
  const long long plane = (long long)n_r * K_pad;
  const int ch = (n_r + 31) / 32, i0 = min(n_r, lane * ch), i1 = min(n_r, i0 + ch);
  if (l < 0) {
    for (int i = i0; i < i1; ++i) Mb[(long long)i * K_pad + c] = Bb[(long long)i * K_pad + c] = 0.0;
    return;
  }
  const long long rs = (long long)(L + 1) * n_r;
  const double* at = rad + (long long)l * n_r;
  const double* bt = rad + rs + (long long)l * n_r;
  const double* fin = rad + 2 * rs + (long long)l * n_r;
  const double* fout = rad + 3 * rs + (long long)l * n_r;
  for (int i = i0; i < i1; ++i) {
    double v = 0.0;
    for (int z = 0; z < S; ++z) {
      const float2 w = part[z * plane + (long long)i * K_pad + c];
      v += (double)w.x + (double)w.y;
    }
    Mb[(long long)i * K_pad + c] = v;
  }
  __syncwarp();  // the previous shell's Mbar, read below, may belong to the lane below
  auto xf = [&](int i) { return i + 1 < n_r ? fin[i + 1] : 0.0; };
  double A = 1.0, x = 0.0;
  for (int i = i1 - 1; i >= i0; --i) {
    x = fma(xf(i), x, Mb[(long long)i * K_pad + c]);
    A *= xf(i);
  }
  aff_scan_down(A, x, lane);
  double carry = __shfl_down_sync(0xffffffffu, x, 1);
  if (lane == 31) carry = 0.0;
  x = carry;
  for (int i = i1 - 1; i >= i0; --i) {
    x = fma(xf(i), x, Mb[(long long)i * K_pad + c]);
    Bb[(long long)i * K_pad + c] = at[i] * x;
  }
  auto yc = [&](int i) { return i >= 1 ? Mb[(long long)(i - 1) * K_pad + c] : 0.0; };
  auto yf = [&](int i) { return i >= 2 ? fout[i - 2] : 0.0; };
  A = 1.0;
  x = 0.0;
  for (int i = i0; i < i1; ++i) {
    x = fma(yf(i), x, yc(i));
    A *= yf(i);
  }
  aff_scan_up(A, x, lane);
  carry = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) carry = 0.0;
  x = carry;
  for (int i = i0; i < i1; ++i) {
    x = fma(yf(i), x, yc(i));
    Bb[(long long)i * K_pad + c] = fma(bt[i], x, Bb[(long long)i * K_pad + c]);
  }
}

// Xs[s][i][pc]: the balanced digits of row i of X on the grid of the row's
// largest value (scaled by 2^-e), and sc[i] = {(896 + e) << 20, 0, 0, 0}, the
// exponent rebase that unscales the synthesis output as it is widened to
// FP64.  One CTA per shell.
constexpr int kSliceThreads = 256;
__device__ __forceinline__ void emu_slice_m_kernel_body(const tc::VBlock& vb, int n_r, int K_pad, const double* __restrict__ X,
                                                                    uint16_t* __restrict__ Xs,
                                                                    float4* __restrict__ sc) {
  __shared__ unsigned int red[32];
  const int i = vb.x;
  const double* row = X + (long long)i * K_pad;
  unsigned int b = 0;
  for (int c = threadIdx.x; c < K_pad; c += blockDim.x) b = max(b, (unsigned int)bexp(row[c]));
  // (rows below 2^-895 keep fewer bits: the rebase must stay a valid FP64 exponent)
  const int e = max(grid_exp(block_max_u(b, red)), -895);
  if (threadIdx.x == 0) sc[i] = make_float4(__int_as_float((896 + e) << 20), 0.0f, 0.0f, 0.0f);
  const long long plane = (long long)n_r * K_pad;
  for (int c = threadIdx.x; c < K_pad; c += blockDim.x) {
    int d[kS];
    bal_digits(fixed_signed(row[c], e, 47), d);
#pragma unroll
    for (int s = 0; s < kS; ++s) Xs[s * plane + (long long)i * K_pad + c] = digit_bf16(d[s], s);
  }
}
__global__ void __launch_bounds__(kSliceThreads) emu_slice_m_kernel(int n_r, int K_pad, const double* __restrict__ X,
                                                                    uint16_t* __restrict__ Xs,
                                                                    float4* __restrict__ sc) {
  emu_slice_m_kernel_body(tc::vblock_self(), n_r, K_pad, X, Xs, sc);
}

// The arguments of emu_slice_m_kernel but the field, for a grouped launch.
struct EmuSliceMArgs {
  int n_r;
  int K_pad;
  const double* X;
  uint16_t* Xs;
  float4* sc;
};

// emu_slice_m_kernel over the problems of a batch, one block per problem block.
__global__ void __launch_bounds__(kSliceThreads) emu_slice_m_kernel_group(const EmuSliceMArgs* __restrict__ probs,
    const tc::GroupDims* __restrict__ dims, int n) {
  tc::VBlock vb;
  const int k = tc::locate_block(dims, n, blockIdx.x, vb);
  const EmuSliceMArgs& a = probs[k];
  emu_slice_m_kernel_body(vb, a.n_r, a.K_pad, a.X, a.Xs, a.sc);
}


// out[i][pc_nat[pc]] = in[i][pc] (the FP64 moments in natural column order)
__global__ void emu_unpermute_kernel(int n_r, int K, int K_pad, const int* __restrict__ pc_nat,
                                     const double* __restrict__ in, double* __restrict__ out) {
  const long long total = (long long)n_r * K_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / K_pad;
    const int c = pc_nat[(int)(e % K_pad)];
    if (c >= 0) out[i * K + c] = in[e];
  }
}

}  // namespace

cudaError_t emu_unpermute(const ygs_plan* p, const double* in, double* out, cudaStream_t s) {
  emu_unpermute_kernel<<<256, 256, 0, s>>>(p->n_r, p->K, p->tc_k_pad, p->tc_pc_nat, in, out);
  return cudaGetLastError();
}

cudaError_t emu_slice_weights(ygs_plan* p) {
  const int K = p->K, kp = p->tc_k_pad;
  int* ecol = nullptr;
  cudaError_t e = dev_malloc((void**)&ecol, (size_t)kp * sizeof(int));
  if (e != cudaSuccess) return e;
  auto run = [&]() -> cudaError_t {
    cudaError_t r;
    // forward: U^T (projection), Q (synthesis); adjoint: Q^T (projection), U (synthesis)
    emu_col_exp_kernel<<<kp, 256>>>(K, p->tc_pc_int, p->nang_wtotal, p->U, ecol);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    emu_slice_ut_kernel<<<1024, 256>>>(K, kp, p->tc_n_pad, p->tc_pc_int, p->U, p->pt, p->n_wpatch, p->tc_pad_off_d,
                                       ecol, p->tc_ut);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    emu_col_exp_kernel<<<kp, 256>>>(K, p->tc_pc_int, p->nang_wtotal, p->Q, ecol);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    emu_slice_ut_kernel<<<1024, 256>>>(K, kp, p->tc_n_pad, p->tc_pc_int, p->Q, p->pt, p->n_wpatch, p->tc_pad_off_d,
                                       ecol, p->tc_qt);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    emu_slice_rows_kernel<<<1024, 256>>>(K, kp, p->nang_wtotal, p->tc_pc_int, p->Q, p->tc_qs);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    emu_slice_rows_kernel<<<1024, 256>>>(K, kp, p->nang_wtotal, p->tc_pc_int, p->U, p->tc_us);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    return cudaDeviceSynchronize();
  };
  e = run();
  cudaFree(ecol);
  return e;
}

// The arguments and grids of the per-field passes, shared by the plain
// launches and the grouped launches of a batch.
namespace {
EmuFieldArgs emu_field_args(const ygs_plan* p) {
  const int fld = (p->tc_np_full + (p->tc_np_tail > 0 ? 1 : 0)) * tc::kNmaxProject;
  return EmuFieldArgs{p->n_r, p->symmetric ? 1 : 0, p->n_wpatch, p->pt, p->tc_pad_off_d, p->tc_n_pad,
                      reinterpret_cast<uint16_t*>(p->tc_f), p->tc_fac, fld, p->d_err};
}
dim3 emu_field_grid(const ygs_plan* p) { return dim3((unsigned)(p->tc_n_pad / kEmuWindow), p->n_r); }
EmuScanArgs emu_scan_args(const ygs_plan* p) {
  return EmuScanArgs{p->n_r, p->tc_k_pad, p->l_max, p->tc_S, p->tc_pc_l, p->tc_part, p->rad,
                     p->tc_Bd, p->tc_Md, p->tc_B, p->tc_M};
}
int emu_scan_blocks(const ygs_plan* p) { return (p->tc_k_pad + kScanWarps - 1) / kScanWarps; }
EmuSliceMArgs emu_slice_m_args(const ygs_plan* p) {
  return EmuSliceMArgs{p->n_r, p->tc_k_pad, p->tc_Md, reinterpret_cast<uint16_t*>(p->tc_ms), p->tc_sc};
}
}  // namespace

cudaError_t emu_field_slices(const ygs_plan* p, const double* rho, cudaStream_t s) {
  const EmuFieldArgs a = emu_field_args(p);
  emu_field_kernel<<<emu_field_grid(p), kFieldThreads, 0, s>>>(a.n_r, a.symmetric, a.nwp, a.pt, a.pad_off, a.n_pad,
                                                               rho, a.F, a.fac, a.fac_ld, a.err);
  return cudaGetLastError();
}

cudaError_t emu_scan(const ygs_plan* p, cudaStream_t s) {
  const EmuScanArgs a = emu_scan_args(p);
  emu_scan_kernel<<<emu_scan_blocks(p), 32 * kScanWarps, 0, s>>>(a.n_r, a.K_pad, a.L, a.S, a.pc_l, a.part, a.rad,
                                                                 a.B, a.M, a.Bff, a.Mff);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const EmuSliceMArgs m = emu_slice_m_args(p);
  emu_slice_m_kernel<<<p->n_r, kSliceThreads, 0, s>>>(m.n_r, m.K_pad, m.X, m.Xs, m.sc);
  return cudaGetLastError();
}

cudaError_t emu_batch_passes(const std::vector<ygs_plan*>& mem, TcBatchGroup& G) {
  const int n = (int)mem.size();
  std::vector<EmuFieldArgs> fa;
  std::vector<EmuScanArgs> sa;
  std::vector<EmuSliceMArgs> ma;
  std::vector<int> gx, gy, one(n, 1), sx, mx;
  for (ygs_plan* p : mem) {
    fa.push_back(emu_field_args(p));
    sa.push_back(emu_scan_args(p));
    ma.push_back(emu_slice_m_args(p));
    const dim3 d = emu_field_grid(p);
    gx.push_back((int)d.x);
    gy.push_back((int)d.y);
    sx.push_back(emu_scan_blocks(p));
    mx.push_back(p->n_r);
  }
  cudaError_t e;
  if ((e = upload_grouped_pass(G.field, fa.data(), sizeof(EmuFieldArgs), n, gx.data(), gy.data(), one.data())) !=
      cudaSuccess)
    return e;
  if ((e = upload_grouped_pass(G.scan, sa.data(), sizeof(EmuScanArgs), n, sx.data(), one.data(), one.data())) !=
      cudaSuccess)
    return e;
  return upload_grouped_pass(G.mslice, ma.data(), sizeof(EmuSliceMArgs), n, mx.data(), one.data(), one.data());
}

cudaError_t emu_batch_field(const TcBatchGroup& G, const double* const* rho, cudaStream_t s) {
  tc::RhoList list{};
  const int n = (int)G.members.size();
  for (int k = 0; k < n; ++k) list.p[k] = rho[k];
  emu_field_kernel_group<<<G.field.blocks, kFieldThreads, 0, s>>>(static_cast<const EmuFieldArgs*>(G.field.d_args),
                                                                  static_cast<const tc::GroupDims*>(G.field.d_dims),
                                                                  n, list);
  return cudaGetLastError();
}

cudaError_t emu_batch_scan(const TcBatchGroup& G, cudaStream_t s) {
  const int n = (int)G.members.size();
  emu_scan_kernel_group<<<G.scan.blocks, 32 * kScanWarps, 0, s>>>(static_cast<const EmuScanArgs*>(G.scan.d_args),
                                                                  static_cast<const tc::GroupDims*>(G.scan.d_dims), n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  emu_slice_m_kernel_group<<<G.mslice.blocks, kSliceThreads, 0, s>>>(
      static_cast<const EmuSliceMArgs*>(G.mslice.d_args), static_cast<const tc::GroupDims*>(G.mslice.d_dims), n);
  return cudaGetLastError();
}

cudaError_t emu_scan_adj(const ygs_plan* p, cudaStream_t s) {
  // the adjoint workspaces hold n_r K_pad doubles: FP64 Mbar and Bbar here
  double* mb = reinterpret_cast<double*>(p->tc_Mbar);
  double* bb = reinterpret_cast<double*>(p->tc_Bbar);
  emu_scan_adj_kernel<<<(p->tc_k_pad + kScanWarps - 1) / kScanWarps, 32 * kScanWarps, 0, s>>>(p->n_r, p->tc_k_pad, p->l_max, p->tc_S, p->tc_pc_l,
                                                            p->tc_part, p->rad, mb, bb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  emu_slice_m_kernel<<<p->n_r, kSliceThreads, 0, s>>>(p->n_r, p->tc_k_pad, bb, reinterpret_cast<uint16_t*>(p->tc_ms),
                                                      p->tc_sc);
  return cudaGetLastError();
}

// ---- the contraction kernels -------------------------------------------------

namespace {
template <int MODE>
using EmuCfg = tc::TcCfg<1, MODE, true>;
}  // namespace

cudaError_t emu_set_smem_attrs() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(tc::tc_gemm_kernel<1, tc::kProject, true, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, EmuCfg<tc::kProject>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(tc::tc_gemm_group_kernel<1, tc::kProject, true, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, EmuCfg<tc::kProject>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(tc::tc_gemm_kernel<1, tc::kSynthesize, false, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, EmuCfg<tc::kSynthesize>::SMEM)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(tc::tc_gemm_group_kernel<1, tc::kSynthesize, false, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, EmuCfg<tc::kSynthesize>::SMEM)) !=
      cudaSuccess)
    return e;
  // the register split of each kernel (see check_reg_split)
  if ((e = tc::check_reg_split<tc::kProject, true>((const void*)tc::tc_gemm_kernel<1, tc::kProject, true, false, true>)) !=
          cudaSuccess ||
      (e = tc::check_reg_split<tc::kProject, true>(
           (const void*)tc::tc_gemm_group_kernel<1, tc::kProject, true, false, true>)) != cudaSuccess ||
      (e = tc::check_reg_split<tc::kSynthesize, true>(
           (const void*)tc::tc_gemm_kernel<1, tc::kSynthesize, false, false, true>)) != cudaSuccess)
    return e;
  return tc::check_reg_split<tc::kSynthesize, true>(
      (const void*)tc::tc_gemm_group_kernel<1, tc::kSynthesize, false, false, true>);
}

cudaError_t emu_dispatch_gemm(int mode, int grid, const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& bt,
                              const tc::TcArgs& args, cudaStream_t s) {
  if (mode == tc::kProject) {
    tc::tc_gemm_kernel<1, tc::kProject, true, false, true>
        <<<grid, tc::TileShape<tc::kProject, true>::THREADS, EmuCfg<tc::kProject>::SMEM, s>>>(a, b, bt, args);
  } else {
    tc::tc_gemm_kernel<1, tc::kSynthesize, false, false, true>
        <<<grid, tc::TileShape<tc::kSynthesize, true>::THREADS, EmuCfg<tc::kSynthesize>::SMEM, s>>>(a, b, bt, args);
  }
  return cudaGetLastError();
}

cudaError_t emu_dispatch_group(int mode, int grid, const tc::TcProblem* probs, const int* start, int n, int total,
                               const tc::TcPhiList& phis, cudaStream_t s) {
  if (mode == tc::kProject) {
    tc::tc_gemm_group_kernel<1, tc::kProject, true, false, true>
        <<<grid, tc::TileShape<tc::kProject, true>::THREADS, EmuCfg<tc::kProject>::SMEM, s>>>(probs, start, n, total,
                                                                                           phis);
  } else {
    tc::tc_gemm_group_kernel<1, tc::kSynthesize, false, false, true>
        <<<grid, tc::TileShape<tc::kSynthesize, true>::THREADS, EmuCfg<tc::kSynthesize>::SMEM, s>>>(
            probs, start, n, total, phis);
  }
  return cudaGetLastError();
}

// this translation unit's out-of-range record (checked builds; a no-op otherwise)
YGS_BOUNDS_READER(bounds_read_emu)

}  // namespace ygs
