// Split-precision tensor-core contraction for sm_103a (tcgen05 + TMEM + TMA).
//
//   D[r][n] = sum_k A[r][k] * B[n][k],  A and B given as NSL BF16 slices each
//   (A ~ A_0 + A_1 + A_2, likewise B), of which the products A_s B_t with
//   s + t <= NSL - 1 are formed (3 for two slices, 6 for three).
//
// One CTA owns a 128 x N output tile.  Warp 0 streams A/B slice tiles of
// 32 k-elements (64-byte rows, 64-byte swizzle) through a ring of shared-memory
// stages with TMA; warp 1 issues tcgen05.mma into FP32 TMEM accumulators;
// warps 2-9 drain them with tcgen05.ld.  The tensor core's FP32 accumulation
// loses about one unit in the last place per accumulation step, always in the
// same direction, so the leading product A_0 B_0 (full size) is accumulated
// only over a short "group" of k-blocks in one of several rotating TMEM
// buffers and then flushed into a float-float register sum, while the
// correction products (2^-8 smaller, so their rounding is negligible) share one
// accumulator for the whole k range of a segment.
//
//   kProject:    groups are consecutive runs of the chunk's k-blocks; the
//                epilogue keeps a float-float running sum (TwoSum, in the spirit
//                of the compensated sums of Sect. 4.3) and stores (hi, lo) pairs
//                of the chunk's partial moments: part[z][n][r].
//   kSynthesize: group 0 is the even-m column block, group 1 (Yin-Yang
//                symmetry) the odd block; the epilogue writes
//                Phi_Yin = E + O and Phi_Yang = E - O (or Phi_g = E) in FP64.
#pragma once

#include "ygs_internal.h"
#include "ygs_tc.cuh"

namespace ygs {
namespace tc {

#ifndef YGS_TC_BK
#define YGS_TC_BK 64
#endif
constexpr int BK = YGS_TC_BK;  // k elements per stage: 64 (128-byte rows, 128-byte swizzle) or 32 (64-byte)
constexpr int BM = 128;  // output rows per CTA (TMEM lanes)
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;

enum Mode { kProject = 0, kSynthesize = 1 };

struct TcArgs {
  int* err;
  int flush_kb;         // k-blocks per TMEM group (a flush into the float-float sums)
  int n_b;              // valid B rows (shells)
  // ---- projection: blockIdx = (m-tile, n-tile, chunk)
  int tiles_m_even;     // m-tiles of the even column block (the rest are odd)
  int a_row_odd;        // first A row of the odd column block (= rows of the even block)
  int a_rows_total;     // rows of A that hold data (even + odd blocks)
  int b_plane_odd;      // B plane of the odd block's field slices (sigma-) or 0
  const int2* chunks;   // k range [x, y) of chunk z, in elements (multiples of BK)
  float2* part;         // [z][n_b][ldp] (hi, lo)
  int ldp;
  // ---- synthesis: blockIdx = (n-tile, m-tile within the patch, patch)
  int k_even;           // length of the even column block (elements, multiple of BK)
  int k_total;          // total padded columns
  int symmetric;
  PatchTable pt;        // field offsets / angular sizes per patch
  long long a_row0[kMaxPatch];  // first A row of each patch
  double* phi;
  // Monopole term of Eq. gravpotmult: Q_00 = -G at every cell, so
  // mono[n] = -G M[n][0] (a float-float pair per shell) is added here instead
  // of being accumulated on the tensor cores (its column is zero in the Q
  // slices).  nullptr disables it.
  const float2* mono;
};

template <int N, int NSL>
struct TcCfg {
  static constexpr int NPROD = (NSL == 3) ? 6 : (NSL == 2 ? 3 : 1);
  static constexpr int NH = N / 2;  // columns per epilogue warp
  static constexpr int A_SLICE = BM * BK * 2;
  static constexpr int B_SLICE = N * BK * 2;
  static constexpr int STAGE = NSL * (A_SLICE + B_SLICE);
#ifdef YGS_TC_STAGES
  static constexpr int STAGES = YGS_TC_STAGES;
#else
  static constexpr int STAGES = (220 * 1024) / STAGE > 8 ? 8 : (220 * 1024) / STAGE;
#endif
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
  static constexpr uint32_t IDESC = idesc_f16(BM, N, 1);
  // TMEM columns: correction accumulators of up to two segments, then rotating
  // leading-product buffers.
  static constexpr int NCORR = 2;
  static constexpr int NBUF = (512 - NCORR * N) / N > 4 ? 4 : (512 - NCORR * N) / N;
  static_assert(N % 16 == 0 && N >= 16 && N <= 128, "N must be a multiple of 16 in [16, 128]");
  static_assert(STAGES >= 2, "not enough shared memory for two stages");
  static_assert(NBUF >= 2, "not enough TMEM for two leading-product buffers");
};

// (s, t) slice pairs in issue order; pair 0 is the leading product.
// NSL = 3: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0);  NSL = 2: (0,0) (0,1) (1,0).
__device__ __forceinline__ int prod_s(int p) { return (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ int prod_t(int p) { return (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0); }

__device__ __forceinline__ double f32_to_f64(float f) {
  unsigned int u = __float_as_uint(f);
  unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  unsigned int hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  unsigned int lo = u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Bounded wait that ignores the abort flag (used before releasing resources).
__device__ __forceinline__ void mbar_wait_final(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit && !mbar_try_wait(bar, parity); ++it) {
  }
}

template <int N, int NSL, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs args) {
  using C = TcCfg<N, NSL>;
  constexpr int NH = C::NH;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* tfull = empty + C::STAGES;  // [NBUF] leading-product buffer ready
  uint64_t* tempty = tfull + C::NBUF;   // [NBUF] leading-product buffer drained
  uint64_t* cfull = tempty + C::NBUF;   // [2] correction accumulator of segment s final
  uint64_t* mma_done = cfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  // ---- tile decode: A rows, B rows, k range split into one or two segments
  int a_row0, b_row0, b_plane0 = 0, a_rows_end;
  int kstart, seg_kb[2];  // k-blocks of segment 0 and 1
  int g_patch = 0;
  if (MODE == kProject) {
    const int mt = blockIdx.x;
    const bool odd = mt >= args.tiles_m_even;
    a_row0 = odd ? args.a_row_odd + (mt - args.tiles_m_even) * BM : mt * BM;
    a_rows_end = odd ? args.a_rows_total : args.a_row_odd;
    b_row0 = blockIdx.y * N;
    b_plane0 = odd ? args.b_plane_odd : 0;
    const int2 ch = args.chunks[blockIdx.z];
    kstart = ch.x;
    seg_kb[0] = (ch.y - ch.x) / BK;
    seg_kb[1] = 0;
  } else {
    g_patch = blockIdx.z;
    const long long nang = args.pt.nang[g_patch];
    if ((long long)blockIdx.y * BM >= nang) return;  // the whole CTA leaves before any setup
    a_row0 = (int)(args.a_row0[g_patch] + (long long)blockIdx.y * BM);
    a_rows_end = 0;
    b_row0 = blockIdx.x * N;
    kstart = 0;
    const bool two = args.symmetric && args.k_even < args.k_total;
    seg_kb[0] = (two ? args.k_even : args.k_total) / BK;
    seg_kb[1] = two ? (args.k_total - args.k_even) / BK : 0;
  }
  const int flush = args.flush_kb;
  const int ng0 = (seg_kb[0] + flush - 1) / flush, ng1 = (seg_kb[1] + flush - 1) / flush;
  const int n_groups = ng0 + ng1;
  // k-block range [kb0, kb1) of group g and whether it closes its segment
  auto group_range = [&](int g, int& kb0, int& kb1, bool& last) {
    if (g < ng0) {
      kb0 = g * flush;
      kb1 = min(seg_kb[0], kb0 + flush);
      last = (g == ng0 - 1);
    } else {
      const int h = g - ng0;
      kb0 = seg_kb[0] + h * flush;
      kb1 = min(seg_kb[0] + seg_kb[1], kb0 + flush);
      last = (g == n_groups - 1);
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < C::NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(&cfull[0], 1);
    mbar_init(&cfull[1], 1);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      const int nkb = seg_kb[0] + seg_kb[1];
      for (int kb = 0; kb < nkb; ++kb) {
        const int stage = issued % C::STAGES;
        const uint32_t ph = (issued / C::STAGES) & 1;
        if (!mbar_wait(&empty[stage], ph ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        uint8_t* sA = smem + stage * C::STAGE;
        uint8_t* sB = sA + NSL * C::A_SLICE;
        mbar_arrive_expect_tx(&full[stage], C::STAGE);
        const int kx = kstart + kb * BK;
#pragma unroll
        for (int s = 0; s < NSL; ++s) tma_load_3d(sA + s * C::A_SLICE, &mapA, &full[stage], kx, a_row0, s);
#pragma unroll
        for (int t = 0; t < NSL; ++t) tma_load_3d(sB + t * C::B_SLICE, &mapB, &full[stage], kx, b_row0, b_plane0 + t);
        ++issued;
      }
      if (!ok) {
        set_err(args.err, YGS_ERR_TIMEOUT);
        *abort_flag = 1;
      }
      // every issued copy has landed before shared memory can be released
      for (int d = max(0, issued - C::STAGES); d < issued; ++d)
        mbar_wait_final(&full[d % C::STAGES], (d / C::STAGES) & 1);
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0) {
      int consumed = 0;
      bool ok = true;
      bool corr_init = false;
      for (int g = 0; g < n_groups && ok; ++g) {
        const int buf = g % C::NBUF, use = g / C::NBUF;
        if (use >= 1 && !mbar_wait(&tempty[buf], (use - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        int kb0, kb1;
        bool last;
        group_range(g, kb0, kb1, last);
        const int seg = (g < ng0) ? 0 : 1;
        if (g == 0 || g == ng0) corr_init = false;
        const uint32_t d_corr = tmem + seg * N;
        const uint32_t d_main = tmem + (C::NCORR + buf) * N;
        bool main_init = false;
        for (int kb = kb0; kb < kb1; ++kb) {
          const int stage = consumed % C::STAGES;
          const uint32_t ph = (consumed / C::STAGES) & 1;
          if (!mbar_wait(&full[stage], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sA = smem_u32(smem + stage * C::STAGE);
          const uint32_t sB = sA + NSL * C::A_SLICE;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int p = 0; p < C::NPROD; ++p) {
              const uint64_t ad = BK == 64 ? sdesc_kmajor_sw128(sA + prod_s(p) * C::A_SLICE + kk * 32)
                                           : sdesc_kmajor_sw64(sA + prod_s(p) * C::A_SLICE + kk * 32);
              const uint64_t bd = BK == 64 ? sdesc_kmajor_sw128(sB + prod_t(p) * C::B_SLICE + kk * 32)
                                           : sdesc_kmajor_sw64(sB + prod_t(p) * C::B_SLICE + kk * 32);
              if (p == 0) {
                umma_f16(d_main, ad, bd, C::IDESC, main_init ? 1u : 0u);
                main_init = true;
              } else {
                umma_f16(d_corr, ad, bd, C::IDESC, corr_init ? 1u : 0u);
                corr_init = true;
              }
            }
          }
          umma_commit(&empty[stage]);
          ++consumed;
        }
        if (!ok) break;
        umma_commit(&tfull[buf]);
        if (last) umma_commit(&cfull[seg]);
      }
      if (!ok) {
        set_err(args.err, YGS_ERR_TIMEOUT);
        *abort_flag = 1;
      }
      umma_commit(mma_done);
      mbar_wait_final(mma_done, 0);  // every issued MMA has finished before TMEM is released
    }
  } else {
    // ================= epilogue warps 2..9 =================
    const int q = warp % 4;            // TMEM lane quadrant this warp may access
    const int half = (warp - 2) / 4;   // which half of the N columns
    const int r = q * 32 + lane;       // output row within the tile
    const uint32_t t_lane = (uint32_t)(q * 32) << 16;
    const int col0 = half * NH;
    float hi[NH], lo[NH], ev[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) hi[j] = lo[j] = ev[j] = 0.0f;
    bool ok = true;
    for (int g = 0; g < n_groups && ok; ++g) {
      const int buf = g % C::NBUF, use = g / C::NBUF;
      int kb0, kb1;
      bool last;
      group_range(g, kb0, kb1, last);
      if (!mbar_wait(&tfull[buf], use & 1, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int c0 = 0; c0 < NH; c0 += 8) {
        uint32_t vm[8];
        tmem_ld8(tmem + t_lane + (C::NCORR + buf) * N + col0 + c0, vm);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float s, e;
          two_sum(hi[c0 + j], __uint_as_float(vm[j]), s, e);
          hi[c0 + j] = s;
          lo[c0 + j] += e;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      if (last) {
        const int seg = (g < ng0) ? 0 : 1;
        if (NSL > 1) {
          if (!mbar_wait(&cfull[seg], 0, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int c0 = 0; c0 < NH; c0 += 8) {
            uint32_t vc[8];
            tmem_ld8(tmem + t_lane + seg * N + col0 + c0, vc);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 8; ++j) lo[c0 + j] += __uint_as_float(vc[j]);
          }
        }
        if (MODE == kSynthesize && seg == 0 && ng1 > 0) {
          // even block done: keep E, restart the sums for the odd block
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            ev[j] = hi[j] + lo[j];
            hi[j] = lo[j] = 0.0f;
          }
        }
      }
    }
    if (!ok) {
      set_err(args.err, YGS_ERR_TIMEOUT);
      *abort_flag = 1;
    } else if (MODE == kProject) {
      if (a_row0 + r < a_rows_end) {
        float2* out = args.part + (long long)blockIdx.z * args.n_b * args.ldp;
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          const int n = b_row0 + col0 + j;
          if (n < args.n_b) {
            float s, e;
            two_sum(hi[j], lo[j], s, e);
            out[(long long)n * args.ldp + a_row0 + r] = make_float2(s, e);
          }
        }
      }
    } else {
      const long long nang = args.pt.nang[g_patch];
      const long long a_loc = (long long)blockIdx.y * BM + r;
      if (a_loc < nang) {
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          const int n = b_row0 + col0 + j;
          if (n >= args.n_b) continue;
          float v = hi[j] + lo[j];
          if (args.mono) {
            // the monopole belongs to the even block (E) or, without the symmetry, to the only block
            const float2 mm = args.mono[n];
            const float mh = mm.x, ml = mm.y;
            if (ng1 > 0) {
              float s, e;
              two_sum(ev[j], mh, s, e);
              ev[j] = s + (e + ml);
            } else {
              float s, e;
              two_sum(hi[j], mh, s, e);
              v = s + (e + ml + lo[j]);
            }
          }
          if (args.symmetric) {
            // Yin-Yang: Phi_Yin = E + O, Phi_Yang = E - O (O = 0 when there are no odd columns)
            const float e = (ng1 > 0) ? ev[j] : v, o = (ng1 > 0) ? v : 0.0f;
            args.phi[args.pt.fld_off[0] + (long long)n * nang + a_loc] = f32_to_f64(e + o);
            args.phi[args.pt.fld_off[1] + (long long)n * nang + a_loc] = f32_to_f64(e - o);
          } else {
            args.phi[args.pt.fld_off[g_patch] + (long long)n * nang + a_loc] = f32_to_f64(v);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace tc
}  // namespace ygs
