// Split-precision tensor-core contraction for sm_103a (tcgen05 + TMEM + TMA).
//
//   D[r][n] = sum_k A[r][k] * B[n][k],  A and B given as NSL BF16 slices, or
//   NSL FP16 slices of power-of-two-scaled rows, each (A ~ A_0 + A_1 + A_2,
//   likewise B), of which the products A_s B_t with s + t <= NSL - 1 are
//   formed (3 for two slices, 6 for three).
//
// Persistent kernel: one CTA per SM walks a static list of 128 x n_eff output
// tiles (n_eff = n_w shells, NMAX = 144 by default or a narrower width picked
// by the autotuner, or the tail width for the last shell tile).  Warp 0
// streams A/B slice tiles of BK k-elements (128-byte rows, 128-byte swizzle)
// through a ring of shared-memory stages with TMA; warp 1 issues tcgen05.mma
// into FP32 TMEM accumulators; the epilogue warps (from warp 4, after the two
// idle warps that complete warpgroup 0; 4 per group of NH columns) drain them
// with tcgen05.ld.  The
// tensor core's FP32 accumulation loses about one unit in the last place per
// accumulation step, always in the same direction, so every product is
// accumulated only over a short "group" of k-blocks in one of NBUF rotating
// TMEM buffers and then flushed into a float-float register sum (TwoSum, in
// the spirit of the compensated sums of Sect. 4.3).  TMEM buffers are tracked
// across tiles, so the epilogue of one tile overlaps the MMAs of the next.
//
//   kProject:    tile = (column tile m, shell tile n, angular chunk z); the
//                epilogue stores (hi, lo) pairs of the chunk's partial
//                moments: part[z][n][r].
//   kSynthesize: tile = (cell tile m of patch g, shell tile n); segment 0 is
//                the even-m column block, segment 1 (Yin-Yang symmetry) the
//                odd block; E (with the monopole term, added in float-float)
//                is parked in TMEM, and the epilogue writes Phi_Yin = E + O
//                and Phi_Yang = E - O (or Phi_g = E + monopole) in FP64.
#pragma once

#include "ygs_internal.h"
#include "ygs_tc.cuh"

namespace ygs {
namespace tc {

#ifndef YGS_TC_BK
#define YGS_TC_BK 64
#endif
#ifndef YGS_TC_SETMAXNREG
#define YGS_TC_SETMAXNREG 1  // move registers from the TMA/MMA warpgroup to the epilogue warpgroups
#endif
#ifndef YGS_TC_REGS_LOW
#define YGS_TC_REGS_LOW 56  // registers per thread the TMA/MMA warpgroup keeps (multiple of 8)
#endif
#ifndef YGS_EPI_CHUNK
#define YGS_EPI_CHUNK 24  // TMEM columns an epilogue warp loads per wait (multiple of 8)
#endif
#ifndef YGS_EPI_CHUNK_SCALED
#define YGS_EPI_CHUNK_SCALED 8  // the same for the flushes that apply the field's group factors
#endif
constexpr int BK = YGS_TC_BK;  // 2-byte k elements per stage: 64 (128-byte rows, 128-byte swizzle) or 32 (64-byte)
// k elements per stage: BK for 2-byte operands, BK / 2 for TF32 (4-byte)
// operands, so that a stage holds the same bytes (and the same descriptors
// and k-steps: four of 32 bytes per product) for every operand type
template <bool TF>
struct KElems {
  static constexpr int KE = TF ? BK / 2 : BK;
};
constexpr int BM = 128;        // output rows per tile (TMEM lanes)
// Tile shapes (shells per tile, columns per epilogue warp).  144-shell tiles
// keep the tensor core compute-bound (a 128 x 80 x 16 MMA is bound by reading
// its operands from shared memory) and cut the operand bytes per flop.  The
// projection's epilogue (flushes only; its output is a small partial) runs
// best on 8 warps of 72 columns, the synthesis's (flushes, the parked E and
// the FP64 output) on 12 of 48 (measured: projection 79.4 -> 76.4 us with 72,
// synthesis 100.7 -> 156.7 us).
#ifndef YGS_PROJ_NH
#define YGS_PROJ_NH 72  // of a projection tile's 144 shells per epilogue warp (8 epilogue warps)
#endif
constexpr int kNmaxProject = 144, kNhProject = YGS_PROJ_NH;
constexpr int kNhProjectEmu = 48;  // the FP64-accurate projection keeps 12 epilogue warps
#ifndef YGS_SYNTH_N
#define YGS_SYNTH_N 144  // shells per synthesis tile
#endif
#ifndef YGS_SYNTH_NH
#define YGS_SYNTH_NH 48  // of them per epilogue warp
#endif
constexpr int kNmaxSynth = YGS_SYNTH_N, kNhSynth = YGS_SYNTH_NH;

// FP64-accurate mode (EMU, Ozaki-type splitting): every operand value is cut
// into kEmuSlices balanced base-256 digits (each in [-128, 128], exact in
// BF16) on a grid fixed per row (or per row and window of kEmuWindowKb
// k-blocks), and the kEmuProducts products A_s B_t with s + t <= kEmuSlices
// are accumulated one at a time over windows of kEmuWindowKb k-blocks.  A
// window's sum of one product is a sum of 1024 integers of magnitude at most
// 2^14 on a common grid, so the FP32 accumulator holds it exactly; only the
// flushes into the float-float sums round.  The synthesis tile is 128 shells
// wide so that E can be parked in TMEM as a (hi, lo) pair.
constexpr int kEmuSlices = 6, kEmuProducts = 26, kEmuWindowKb = 1024 / BK;
// k-blocks per shared-memory stage in EMU mode: one slice of each operand is
// 4 MMAs per k-block, and every barrier wait of the issuing thread drains its
// queued MMAs, so a stage carries two k-blocks (8 MMAs per wait)
constexpr int kEmuStageKb = 2;
static_assert(kEmuWindowKb % kEmuStageKb == 0, "a flush window holds whole stages");
constexpr int kNmaxSynthEmu = 128, kNhSynthEmu = 64;
static_assert(kEmuProducts == kEmuSlices * (kEmuSlices + 1) / 2 + kEmuSlices - 1,
              "products with s, t < kEmuSlices and s + t <= kEmuSlices");
static_assert(kEmuWindowKb * BK * 128 * 128 <= (1 << 24), "a window's products sum exactly in FP32");

// Product p of the EMU order: s-major (t from 0 to min(kEmuSlices - 1,
// kEmuSlices - s)), so that consecutive products share the A slice, which the
// L2 then serves again.
__device__ __forceinline__ void emu_pair(int p, int& s, int& t) {
  int first = 0;
  for (s = 0;; ++s) {
    const int n = min(kEmuSlices - 1, kEmuSlices - s) + 1;
    if (p < first + n) break;
    first += n;
  }
  t = p - first;
}

enum Mode { kProject = 0, kSynthesize = 1 };

template <int MODE, bool EMU = false>
struct TileShape {
  // shells per full tile; columns per epilogue warp
  static constexpr int NMAX = MODE == 0 ? kNmaxProject : (EMU ? kNmaxSynthEmu : kNmaxSynth);
  static constexpr int NH = MODE == 0 ? (EMU ? kNhProjectEmu : kNhProject) : (EMU ? kNhSynthEmu : kNhSynth);
  static constexpr int EPI_WARPS = 4 * (NMAX / NH);
  // warps: TMA producer, MMA issuer (with YGS_TC_SETMAXNREG two idle warps
  // complete their warpgroup), then the epilogue warpgroups
  static constexpr int FIRST_EPI = YGS_TC_SETMAXNREG ? 4 : 2;
  static constexpr int THREADS = 32 * FIRST_EPI + 32 * EPI_WARPS;
  static_assert(NMAX % 16 == 0 && NMAX <= 256 && NMAX % NH == 0 && NH % 8 == 0, "tile shape");
  // Registers per thread: at launch (the whole register file over THREADS,
  // in steps of 8), then, with YGS_TC_SETMAXNREG, warpgroup 0 (TMA, MMA)
  // gives up all but REGS_LOW and the epilogue warpgroups take the rest, so
  // their float-float sums stay in registers.  setmaxnreg.inc draws only on
  // the CTA's launch allocation, so the split must not exceed it.
  static constexpr int REGS_LAUNCH = (65536 / THREADS) / 8 * 8 > 248 ? 248 : (65536 / THREADS) / 8 * 8;
  static constexpr int REGS_LOW = YGS_TC_REGS_LOW;
  static constexpr int REGS_EPI_RAW = (THREADS * REGS_LAUNCH - 128 * REGS_LOW) / (32 * EPI_WARPS) / 8 * 8;
  static constexpr int REGS_EPI = REGS_EPI_RAW > 248 ? 248 : REGS_EPI_RAW;
  static_assert(!YGS_TC_SETMAXNREG || (EPI_WARPS % 4 == 0 && REGS_EPI >= REGS_LAUNCH &&
                                       128 * REGS_LOW + 32 * EPI_WARPS * REGS_EPI <= THREADS * REGS_LAUNCH),
                "register split: whole warpgroups, within the launch allocation");
  // TMEM (512 columns): NBUF rotating accumulators of NMAX columns, plus, in
  // the synthesis, NMAX columns that hold the even-block result E of a tile
  // (2 NMAX in EMU mode: its head and tail).
  static constexpr int E_COLS = MODE == 0 ? 0 : (EMU ? 2 : 1) * NMAX;
  static constexpr int NBUF = (512 - E_COLS) / NMAX > 4 ? 4 : (512 - E_COLS) / NMAX;
  static_assert(NBUF >= 2, "TMEM holds 512 columns: need two accumulators");
};

constexpr int kGroupKb = 2;  // k-blocks per exponent group of the FP16 field slices

struct TcArgs {
  int* err;
  int flush_kb;         // k-blocks per TMEM group (a flush into the float-float sums)
  int n_b;              // valid B rows (shells)
  int n_w;              // shells per full tile: NMAX, or (synthesis) a narrower width the
                        // autotuner picked: a multiple of NH, so that an epilogue warp's
                        // columns lie wholly inside a full tile or wholly past it (the
                        // tail tile is the last, its extra columns past n_b)
  int n_full;           // full shell tiles (n_w wide)
  int n_tail;           // width of the tail shell tile (multiple of 16) or 0
  int n_tiles;          // n_full + (n_tail > 0)
  int total_tiles;      // length of the tile list
  // ---- projection: tile = (chunk z, m-tile, n-tile), n fastest
  int tiles_m;          // column tiles (even block, then odd block)
  int tiles_m_even;     // m-tiles of the even column block
  int a_row_odd;        // first A row of the odd column block (= rows of the even block)
  int a_rows_total;     // rows of A that hold data (even + odd blocks)
  int b_plane_odd;      // B plane of the odd block's field slices (sigma-) or 0
  int n_chunks;         // S
  const int2* chunks;   // k range [x, y) of chunk z, in elements (multiples of the k-block)
  float2* part;         // [z][n_b][ldp] (hi, lo)
  int ldp;
  // FP16 field slices: fac[h][G][n] = 2^-e of the field row (plane h, exponent
  // group G of kGroupKb k-blocks, shell n), applied at each flush (a flush
  // covers one group, or half of one).  Rows of fac_ld >= n_tiles * NMAX
  // floats (zero past n_b), so that a tile's row is one 16-byte-aligned
  // bulk copy; fac_plane = the offset of plane 1.  nullptr: unscaled.
  const float* fac;
  long long fac_plane;
  int fac_ld;
  // ---- synthesis: tile = (patch g, m-tile, n-tile), n fastest
  int k_even;           // length of the even column block (elements, multiple of the k-block)
  int k_total;          // total padded columns
  int symmetric;
  int n_wpatch;
  PatchTable pt;        // field offsets / angular sizes per patch
  long long a_row0[kMaxPatch];   // first A row of each patch
  int tile0[kMaxPatch + 1];      // first tile index of each patch
  double* phi;
  // Monopole term of Eq. gravpotmult: Q_00 = -G at every cell, so
  // mono[n] = -G M[n][0] (a float-float pair per shell) is added here instead
  // of being accumulated on the tensor cores (its column is zero in the Q
  // slices).  nullptr disables it.
  const float2* mono;
  int ab_fmt;           // operand type of the slices: 1 = BF16, 0 = FP16, 2 = TF32 (then a TF32 kernel)
  // FP16 slices are scaled rows: sc[n] = {c20, 0, monopole head, tail}, with
  // c20 = (896 + d) << 20 (an int's bits) for d = -(q_exp + m_exp[n]), the
  // power of two that unscales the synthesis result of shell n, applied as it
  // is widened to FP64, and the monopole pair in the scaled units, read from
  // here instead of mono (which then only says whether to add it).
  // nullptr: unscaled (BF16).
  const float4* sc;
};

// CG = 2: a synthesis tile of 256 cells computed by a pair of CTAs (a
// cluster of two) with cta_group::2 MMAs issued by the even CTA; each CTA
// stages its own 128 cells of A and half of the tile's shells of B.
template <int NSL, int MODE, bool EMU = false, int CG = 1>
struct TcCfg {
  static_assert(!EMU || NSL == 1, "EMU stages hold one slice of each operand");
  static_assert(CG == 1 || (CG == 2 && MODE == kSynthesize && !EMU), "CTA pairs: the split synthesis only");
  static constexpr int NMAX = TileShape<MODE, EMU>::NMAX;
  static_assert((NMAX / CG) % 8 == 0, "a CTA's share of B is whole 8-row swizzle atoms");
  static constexpr int NPROD = (NSL == 3) ? 6 : (NSL == 2 ? 3 : 1);
  static constexpr int KBS = EMU ? kEmuStageKb : 1;  // k-blocks per stage
  static constexpr int A_SLICE = BM * BK * 2;      // one k-block of one slice (a 128-byte-swizzled block)
  static constexpr int B_SLICE = NMAX / CG * BK * 2;
  // [A: KBS k-blocks x NSL slices | B: the same]
  static constexpr int STAGE = KBS * NSL * (A_SLICE + B_SLICE);
#ifdef YGS_TC_STAGES
  static constexpr int STAGES = YGS_TC_STAGES;
#else
  static constexpr int STAGES = (220 * 1024) / STAGE > 8 ? 8 : (220 * 1024) / STAGE;
#endif
  // stages, alignment slack, barriers, and (projection) a ring of FAC_RING
  // slots for the field's group factors of a tile's NMAX shells, filled by
  // the TMA warp with each group's first k-block.  The ring cannot be lapped:
  // the TMA warp writes the slot of group g after the MMAs of the k-block
  // STAGES earlier have finished, i.e. after the epilogue has released group
  // g - ceil(STAGES / flush) - 1 - NBUF or later, which is more than
  // FAC_RING groups back for STAGES <= 3, NBUF <= 3, any flush >= 1.
  // (EMU: flush groups of kEmuWindowKb k-blocks, so the lead is
  // ceil(STAGES / kEmuWindowKb) + 1 + NBUF groups.)
  static constexpr int FAC_OFF = 512;
  static constexpr int FAC_RING = 8;
  static constexpr int FAC_BYTES = MODE == 0 ? FAC_RING * NMAX * 4 : 0;
  static_assert(MODE != 0 || FAC_RING > 3 + 1 + 3, "factor ring deeper than the pipeline's lead");
  static constexpr int SMEM = STAGES * STAGE + 1024 + FAC_OFF + FAC_BYTES;
  static constexpr int NBUF = TileShape<MODE, EMU>::NBUF;
  static constexpr int E_COL0 = NBUF * NMAX;  // first TMEM column of the parked E (synthesis)
  static_assert(STAGES >= 2, "not enough shared memory for two stages");
  static_assert(MODE != 0 || (EMU ? (STAGES * KBS + kEmuWindowKb - 1) / kEmuWindowKb + 1 + NBUF < FAC_RING
                                  : (STAGES <= 3 && NBUF <= 3)),
                "the factor ring is deeper than the pipeline's lead");
};

// (s, t) slice pairs in issue order; pair 0 is the leading product.
// NSL = 3: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0);  NSL = 2: (0,0) (0,1) (1,0).
__device__ __forceinline__ int prod_s(int p) { return (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ int prod_t(int p) { return (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0); }

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned int hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  // selects, no branches: FP32 zeros and subnormals give +-0
  return __hiloint2double((int)(e == 0 ? (u & 0x80000000u) : hi), (int)(e == 0 ? 0u : u << 29));
}
// f * 2^d exactly for a normal FP32 f: the magnitude bits shifted into the
// double's layout and the exponent rebased by c20 = (896 + d) << 20 (896 =
// 1023 - 127), so the power-of-two unscaling costs no arithmetic and cannot
// overflow FP32.  Zeros stay exact; an FP32 subnormal (which the scaled
// sums never produce) widens to a double subnormal.
__device__ __forceinline__ double f32_to_f64_pow2(float f, unsigned int c20) {
  const unsigned int u = __float_as_uint(f), mag = u & 0x7FFFFFFFu, sign = u & 0x80000000u;
  const unsigned int hi = mag < 0x00800000u ? sign : (((mag >> 3) + c20) | sign);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Bounded wait that ignores the abort flag (used before releasing resources).
__device__ __forceinline__ void mbar_wait_final(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit && !mbar_try_wait(bar, parity); ++it) {
  }
}

struct Tile {
  int a_row0, a_rows_end, b_row0, b_plane0, n_eff, use_tail;
  int kstart, seg_kb0, seg_kb1;  // k-blocks of segment 0 and 1
  int g_patch, m_loc, z;
};

// CG = 2: t is a pair tile of 2 x BM cells, of which this CTA (rank) takes
// the half `rank`.
template <int MODE, int KE, bool EMU = false, int CG = 1>
__device__ __forceinline__ Tile decode_tile(const TcArgs& a, int t, int rank = 0) {
  Tile T;
  int n;
  if (MODE == kProject) {
    // shell tiles fastest, then column tiles, then chunks: the tiles that read
    // one A block run side by side, and a chunk's field block serves every
    // column tile while it is in L2
    n = t % a.n_tiles;
    const int rem = t / a.n_tiles;
    T.z = rem / a.tiles_m;
    const int mt = rem % a.tiles_m;
    const bool odd = mt >= a.tiles_m_even;
    T.a_row0 = odd ? a.a_row_odd + (mt - a.tiles_m_even) * BM : mt * BM;
    T.a_rows_end = odd ? a.a_rows_total : a.a_row_odd;
    T.b_plane0 = odd ? a.b_plane_odd : 0;
    const int2 ch = a.chunks[T.z];
    T.kstart = ch.x;
    T.seg_kb0 = (ch.y - ch.x) / KE;
    T.seg_kb1 = 0;
    T.g_patch = 0;
    T.m_loc = mt;
  } else {
    int g = 0;
    while (g + 1 < a.n_wpatch && a.tile0[g + 1] <= t) ++g;
    const int rem = t - a.tile0[g];
    T.m_loc = CG * (rem / a.n_tiles) + rank;
    n = rem % a.n_tiles;
    T.g_patch = g;
    T.a_row0 = (int)(a.a_row0[g] + (long long)T.m_loc * BM);
    T.a_rows_end = 0;
    T.b_plane0 = 0;
    T.kstart = 0;
    const bool two = a.symmetric && a.k_even < a.k_total;
    T.seg_kb0 = (two ? a.k_even : a.k_total) / KE;
    T.seg_kb1 = two ? (a.k_total - a.k_even) / KE : 0;
    T.z = 0;
  }
  // full-tile width: the projection's is always NMAX (a constant here)
  const int nw = MODE == kProject ? TileShape<MODE, EMU>::NMAX : a.n_w;
  T.use_tail = (n >= a.n_full);
  T.n_eff = T.use_tail ? a.n_tail : nw;
  T.b_row0 = n * nw;
  return T;
}

// One problem of a grouped launch: its tensor maps and arguments (in global
// memory, written by the host before the launch; aligned like CUtensorMap).
struct alignas(128) TcProblem {
  CUtensorMap a, b, bt;
  TcArgs args;
};
constexpr int kMaxGroup = 128;          // problems per grouped launch
struct TcPhiList {                      // synthesis outputs of a grouped launch
  double* p[kMaxGroup];
};

// What a role needs for one tile: the problem's arguments and maps, its
// output and the tile's index within the problem.
struct TileRef {
  const TcArgs* A;
  const CUtensorMap *ma, *mb, *mbt;
  double* phi;
  int t;
};

struct SingleSrc {  // one problem, everything in kernel parameters
  const TcArgs* A;
  const CUtensorMap *ma, *mb, *mbt;
  __device__ __forceinline__ int total() const { return A->total_tiles; }
  __device__ __forceinline__ TileRef locate(int t) const { return TileRef{A, ma, mb, mbt, A->phi, t}; }
};

struct GroupSrc {  // tiles of several problems concatenated: problem k owns [start[k], start[k+1])
  const TcProblem* probs;
  const int* start;
  int n, tot;
  const TcPhiList* phis;
  __device__ __forceinline__ int total() const { return tot; }
  __device__ __forceinline__ TileRef locate(int t) const {
    int lo = 0, hi = n - 1;  // last problem with start <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const TcProblem& P = probs[lo];
    return TileRef{&P.args, &P.a, &P.b, &P.bt, phis->p[lo], t - start[lo]};
  }
};

// SCALE (projection of FP16 or EMU field slices only): undo the field's
// group factors at every flush.  A compile-time switch: each instance then
// holds only its own flush code, and the epilogue's float-float sums stay in
// registers.  EMU: one slice of each operand per stage, the kEmuProducts
// products one after another over the whole k range of a segment (each
// sweep its own flush groups), flushed by a renormalised float-float add.
//
// CG = 2 (CTA pairs, synthesis): both CTAs walk the same list of pair tiles;
// each loads its 128 cells of A and its half of B, the even CTA's TMA warp
// expects the bytes of both on its `full` barriers (the odd CTA's copies
// complete there), the even CTA issues every MMA and commits to the barriers
// of both CTAs, and the epilogue warps of both drain their own TMEM and
// release it on the even CTA's `tempty` barriers.
template <int NSL, int MODE, bool SCALE, bool TF, bool EMU, int CG, class Src>
__device__ __forceinline__ void gemm_body(const Src& src) {
  static_assert(!SCALE || MODE == kProject, "only the projection scales its flushes");
  static_assert(!(TF && SCALE), "TF32 operands need no scaling");
  static_assert(!(TF && EMU), "EMU slices are BF16");
  constexpr int KE = KElems<TF>::KE;
  using C = TcCfg<NSL, MODE, EMU, CG>;
  constexpr int NMAX = TileShape<MODE, EMU>::NMAX;
  constexpr int NH = TileShape<MODE, EMU>::NH;
  constexpr int kEpiWarps = TileShape<MODE, EMU>::EPI_WARPS;
  constexpr int NPASS = EMU ? kEmuProducts : 1;        // sweeps over a segment's k-blocks
  constexpr int GKB = EMU ? kEmuWindowKb : kGroupKb;   // k-blocks per exponent group of the field
  constexpr int kFirstEpi = TileShape<MODE, EMU>::FIRST_EPI;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* tfull = empty + C::STAGES;  // [NBUF] accumulator ready
  uint64_t* tempty = tfull + C::NBUF;   // [NBUF] accumulator drained
  uint64_t* mma_done = tempty + C::NBUF;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* fac_ring = (float*)(smem + C::STAGES * C::STAGE + C::FAC_OFF);  // [FAC_RING][NMAX] (projection)
  static_assert((2 * C::STAGES + 2 * C::NBUF + 2) * 8 + 8 <= C::FAC_OFF, "barriers fit below the factor slots");

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // this CTA's half of a pair tile; the first tile and the stride of its walk
  const int rank = CG == 2 ? (int)cluster_ctarank() : 0;
  const int unit0 = blockIdx.x / CG, units = gridDim.x / CG;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < C::NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], CG * kEpiWarps);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc<CG>(tmem_slot, 512);
    tmem_relinquish<CG>();
  }
  tc_fence_before();
  __syncthreads();
  // pairs: both CTAs' barriers exist before either signals the other's
  if constexpr (CG == 2) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kFirstEpi) {
    // warpgroup 0: TMA producer, MMA issuer (and, with YGS_TC_SETMAXNREG, two idle warps)
    if constexpr (YGS_TC_SETMAXNREG) setmaxnreg_dec<TileShape<MODE, EMU>::REGS_LOW>();
  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      int issued = 0, fgroups = 0;  // k-blocks issued; factor rows issued (the ring's position)
      bool ok = true;
      int* err = nullptr;
      for (int t = unit0; t < src.total() && ok; t += units) {
        const TileRef R = src.locate(t);
        const Tile T = decode_tile<MODE, KE, EMU, CG>(*R.A, R.t, rank);
        err = R.A->err;
        const CUtensorMap* mb = T.use_tail ? R.mbt : R.mb;
        // this CTA's bytes per k-block, and its first B row (pairs: half of the tile's shells each)
        const uint32_t bytes = NSL * (C::A_SLICE + T.n_eff / CG * BK * 2);
        const int b_row = T.b_row0 + rank * (T.n_eff / CG);
        const float* const fac = SCALE ? R.A->fac : nullptr;
        const int flush = R.A->flush_kb;
        // segments (even and odd column blocks of the synthesis), then the
        // products of an EMU tile, then the k-blocks of the segment
        for (int seg = 0; seg < 2 && ok; ++seg) {
          const int nkb = seg ? T.seg_kb1 : T.seg_kb0, kb0 = seg ? T.seg_kb0 : 0;
          for (int pp = 0; pp < NPASS && ok; ++pp) {
            int ps = 0, pt = 0;
            if (EMU) emu_pair(pp, ps, pt);
            for (int kb = 0; kb < nkb; kb += C::KBS) {
              const int stage = issued % C::STAGES;
              const uint32_t ph = (issued / C::STAGES) & 1;
              if (!mbar_wait(&empty[stage], ph ^ 1, abort_flag)) {
                ok = false;
                break;
              }
              uint8_t* sA = smem + stage * C::STAGE;
              uint8_t* sB = sA + C::KBS * NSL * C::A_SLICE;
              const int nks = min(C::KBS, nkb - kb);          // k-blocks in this stage
              const bool fac_now = SCALE && kb % flush == 0;  // first k-block of a flush group
              if (rank == 0) mbar_arrive_expect_tx(&full[stage], CG * nks * bytes + (fac_now ? NMAX * 4 : 0));
              if (fac_now) {
                const int G = (T.kstart / KE + kb0 + kb) / GKB;
                long long fo = (T.b_plane0 ? R.A->fac_plane : 0) + (long long)G * R.A->fac_ld + T.b_row0;
                // (checked builds: a row outside the table is reported and row 0 copied instead, so
                // the stage's byte count still completes)
                if (!YGS_IN_BOUNDS(fo + NMAX - 1, 2 * R.A->fac_plane, kSiteGemmFac) || !YGS_IN_BOUNDS(fo, 2 * R.A->fac_plane, kSiteGemmFac)) fo = 0;
                const float* src = fac + fo;
                bulk_load(fac_ring + (fgroups % C::FAC_RING) * NMAX, src, NMAX * 4, &full[stage]);
                ++fgroups;
              }
              const int kx = T.kstart + (kb0 + kb) * KE;
              if (EMU) {
                for (int j = 0; j < nks; ++j) {
                  tma_load_3d(sA + j * C::A_SLICE, R.ma, &full[stage], kx + j * KE, T.a_row0, ps);
                  tma_load_3d(sB + j * C::B_SLICE, mb, &full[stage], kx + j * KE, T.b_row0, T.b_plane0 + pt);
                }
              } else if (CG == 2) {
                const uint32_t bar0 = mapa_shared(&full[stage], 0);  // the even CTA's barrier
#pragma unroll
                for (int s = 0; s < NSL; ++s) tma_load_3d_pair(sA + s * C::A_SLICE, R.ma, bar0, kx, T.a_row0, s);
#pragma unroll
                for (int s = 0; s < NSL; ++s)
                  tma_load_3d_pair(sB + s * C::B_SLICE, mb, bar0, kx, b_row, T.b_plane0 + s);
              } else {
#pragma unroll
                for (int s = 0; s < NSL; ++s) tma_load_3d(sA + s * C::A_SLICE, R.ma, &full[stage], kx, T.a_row0, s);
#pragma unroll
                for (int s = 0; s < NSL; ++s)
                  tma_load_3d(sB + s * C::B_SLICE, mb, &full[stage], kx, b_row, T.b_plane0 + s);
              }
              ++issued;
            }
          }
        }
      }
      if (!ok) {
        set_err(err, YGS_ERR_TIMEOUT);
        *abort_flag = 1;
      }
      // every issued copy has landed before shared memory can be released
      // (the odd CTA of a pair: its copies complete on the even CTA's
      // barriers, and the MMAs that read them have finished when its own
      // `empty` barriers complete)
      for (int d = max(0, issued - C::STAGES); d < issued; ++d) {
        if (rank == 0)
          mbar_wait_final(&full[d % C::STAGES], (d / C::STAGES) & 1);
        else
          mbar_wait_final(&empty[d % C::STAGES], (d / C::STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer (pairs: in the even CTA) =================
    if (lane == 0 && rank == 0) {
      int consumed = 0, gglob = 0;
      bool ok = true;
      int* err = nullptr;
      for (int t = unit0; t < src.total() && ok; t += units) {
        const TileRef R = src.locate(t);
        const Tile T = decode_tile<MODE, KE, EMU, CG>(*R.A, R.t, rank);
        err = R.A->err;
        const uint32_t idesc = idesc_f16(BM * CG, T.n_eff, R.A->ab_fmt);
        const int flush = R.A->flush_kb;  // k-blocks per accumulator flush, per problem
        for (int sp = 0; sp < 2 * NPASS && ok; ++sp) {
          const int seg = sp / NPASS;
          const int nkb = seg ? T.seg_kb1 : T.seg_kb0;
          for (int kg = 0; kg < nkb && ok; kg += flush, ++gglob) {
            const int buf = gglob % C::NBUF, use = gglob / C::NBUF;
            if (use >= 1 && !(CG == 2 ? mbar_wait_cluster(&tempty[buf], (use - 1) & 1, abort_flag)
                                      : mbar_wait(&tempty[buf], (use - 1) & 1, abort_flag))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + buf * NMAX;
            bool init = false;
            const int kg1 = min(nkb, kg + flush);
            for (int kb = kg; kb < kg1; kb += C::KBS) {
              const int stage = consumed % C::STAGES;
              const uint32_t ph = (consumed / C::STAGES) & 1;
              if (!mbar_wait(&full[stage], ph, abort_flag)) {
                ok = false;
                break;
              }
              tc_fence_after();
              // one descriptor per operand and stage; slices and k-steps are compile-time
              // offsets added to the start-address field (addresses stay below 256 KB)
              const uint32_t sA = smem_u32(smem + stage * C::STAGE);
              const uint64_t a0 = BK == 64 ? sdesc_kmajor_sw128(sA) : sdesc_kmajor_sw64(sA);
              const uint64_t b0 = BK == 64 ? sdesc_kmajor_sw128(sA + C::KBS * NSL * C::A_SLICE)
                                           : sdesc_kmajor_sw64(sA + C::KBS * NSL * C::A_SLICE);
              if (EMU) {
                // one product, the stage's k-blocks one after another
                const int nks = min(C::KBS, kg1 - kb);
                for (int j = 0; j < nks; ++j) {
#pragma unroll
                  for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint64_t ad = a0 + (uint64_t)((j * C::A_SLICE + kk * 32) >> 4);
                    const uint64_t bd = b0 + (uint64_t)((j * C::B_SLICE + kk * 32) >> 4);
                    umma_f16<CG>(d, ad, bd, idesc, init ? 1u : 0u);
                    init = true;
                  }
                }
                umma_commit<CG>(&empty[stage]);
                ++consumed;
                continue;
              }
              // correction products first, while the accumulator is still small (their
              // rounding then stays ~2^-8 below the leading product's), the leading
              // product A_0 B_0 last: one FP32 rounding per MMA at its own scale
#pragma unroll
              for (int i = 0; i < C::NPROD * (BK / 16); ++i) {
                constexpr int NC = C::NPROD - 1, NCd = NC > 0 ? NC : 1;  // correction products
                const int p = (i < NC * (BK / 16)) ? 1 + i % NCd : 0;
                const int kk = (i < NC * (BK / 16)) ? i / NCd : i - NC * (BK / 16);
                const uint64_t ad = a0 + (uint64_t)((prod_s(p) * C::A_SLICE + kk * 32) >> 4);
                const uint64_t bd = b0 + (uint64_t)((prod_t(p) * C::B_SLICE + kk * 32) >> 4);
                if (TF)
                  umma_tf32<CG>(d, ad, bd, idesc, init ? 1u : 0u);
                else
                  umma_f16<CG>(d, ad, bd, idesc, init ? 1u : 0u);
                init = true;
              }
              umma_commit<CG>(&empty[stage]);
              ++consumed;
            }
            if (!ok) break;
            umma_commit<CG>(&tfull[buf]);
          }
        }
      }
      if (!ok) {
        set_err(err, YGS_ERR_TIMEOUT);
        *abort_flag = 1;
      }
      umma_commit<CG>(mma_done);
      mbar_wait_final(mma_done, 0);  // every issued MMA has finished before TMEM is released
    } else if (CG == 2 && lane == 0) {
      // the odd CTA of a pair: the even CTA's MMAs write this CTA's TMEM too
      mbar_wait_final(mma_done, 0);
    }
  }
  } else {
    if constexpr (YGS_TC_SETMAXNREG) setmaxnreg_inc<TileShape<MODE, EMU>::REGS_EPI>();
    // ================= epilogue warps kFirstEpi .. kFirstEpi + kEpiWarps - 1 =================
    const int ew = warp - kFirstEpi;
    const int q = warp % 4;                // TMEM lane quadrant this warp may access
    const int colq = ew / 4;               // which group of NH columns
    const int r = q * 32 + lane;           // output row within the tile
    const uint32_t t_lane = (uint32_t)(q * 32) << 16;
    const int col0 = colq * NH;
    int gglob = 0;
    bool ok = true;
    int* err = nullptr;
    for (int t = unit0; t < src.total() && ok; t += units) {
      const TileRef R = src.locate(t);
      const Tile T = decode_tile<MODE, KE, EMU, CG>(*R.A, R.t, rank);
      err = R.A->err;
      const int flush = R.A->flush_kb;
      const bool active = col0 < T.n_eff;  // this warp's columns exist in the tile (warp-uniform)
      // float-float sums of column pairs (2j, 2j+1), packed for the f32x2 pipes
      uint64_t H[NH / 2], L[NH / 2];
#pragma unroll
      for (int j = 0; j < NH / 2; ++j) H[j] = L[j] = 0ull;
      const int nseg = T.seg_kb1 > 0 ? 2 : 1;
      // FP16 projection: the field's group factors of the tile's shells, in
      // the ring slot the TMA warp filled with the group's first k-block
      for (int sp = 0; sp < nseg * NPASS && ok; ++sp) {
        const int seg = sp / NPASS;
        const int nkb = seg ? T.seg_kb1 : T.seg_kb0;
        for (int kg = 0; kg < nkb; kg += flush, ++gglob) {
          const int buf = gglob % C::NBUF, use = gglob / C::NBUF;
          if (!mbar_wait(&tfull[buf], use & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (active) {
            const float* const fslot = SCALE ? fac_ring + (gglob % C::FAC_RING) * NMAX + col0 : nullptr;
            // CH columns in flight per wait (fewer when scaling: each pair's
            // factors are live beside its values)
            constexpr int CH0 = SCALE ? YGS_EPI_CHUNK_SCALED : YGS_EPI_CHUNK;
            constexpr int CH = CH0 < NH ? CH0 : NH;
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += CH) {
              uint32_t vm[CH];
#pragma unroll
              for (int c1 = 0; c1 < CH && c0 + c1 < NH; c1 += 8)
                tmem_ld8(tmem + t_lane + buf * NMAX + col0 + c0 + c1, *reinterpret_cast<uint32_t(*)[8]>(&vm[c1]));
              tmem_ld_wait();
#pragma unroll
              for (int j = 0; j < CH / 2 && c0 + 2 * j < NH; ++j) {
                // FastTwoSum: the running sum dominates the flush after the first few
                // (always for same-sign terms); where it does not, the pair still
                // holds the sum within one rounding of that flush
                uint64_t s, e;
                const uint64_t v = pk2(__uint_as_float(vm[2 * j]), __uint_as_float(vm[2 * j + 1]));
                if (EMU) {
                  // the window sum is exact (times an exact power of two): TwoSum
                  // into the head, the tail folded in, renormalised
                  const uint64_t w = SCALE ? mul2(v, lds_pair(fslot + c0 + 2 * j)) : v;
                  two_sum2(H[c0 / 2 + j], w, s, e);
                  fast_two_sum2(s, add2(e, L[c0 / 2 + j]), H[c0 / 2 + j], L[c0 / 2 + j]);
                } else {
                  if (SCALE) {
                    fast_two_sum_scaled2(H[c0 / 2 + j], v, lds_pair(fslot + c0 + 2 * j), s, e);
                  } else {
                    fast_two_sum2(H[c0 / 2 + j], v, s, e);
                  }
                  H[c0 / 2 + j] = s;
                  L[c0 / 2 + j] = add2(L[c0 / 2 + j], e);
                }
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (CG == 2 && rank != 0)
              mbar_arrive_cluster(mapa_shared(&tempty[buf], 0));  // the issuing CTA's barrier
            else
              mbar_arrive(&tempty[buf]);
          }
        }
        if (!ok) break;
        if (EMU && MODE == kSynthesize && sp == NPASS - 1 && nseg == 2 && active) {
          // even block done (all products): park E = (hi, lo) in TMEM, restart the sums
#pragma unroll
          for (int c0 = 0; c0 < NH; c0 += 8) {
            uint32_t vh[8], vl[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float h0, h1, l0, l1;
              upk2(H[c0 / 2 + j], h0, h1);
              upk2(L[c0 / 2 + j], l0, l1);
              vh[2 * j] = __float_as_uint(h0);
              vh[2 * j + 1] = __float_as_uint(h1);
              vl[2 * j] = __float_as_uint(l0);
              vl[2 * j + 1] = __float_as_uint(l1);
              H[c0 / 2 + j] = L[c0 / 2 + j] = 0ull;
            }
            tmem_st8(tmem + t_lane + C::E_COL0 + col0 + c0, vh);
            tmem_st8(tmem + t_lane + C::E_COL0 + NMAX + col0 + c0, vl);
          }
          tmem_st_wait();
        }
        if (!EMU && MODE == kSynthesize && seg == 0 && nseg == 2 && active) {
          // even block done: park E = hi + lo (+ the monopole, which belongs to
          // E: its float-float pair is added before the one rounding to FP32)
          // in TMEM, restart the sums for the odd block
          const float4* const sce = R.A->sc;
          const float2* const monoe = R.A->mono;
          const int n_be = R.A->n_b;
#pragma unroll
          for (int c0 = 0; c0 < NH; c0 += 8) {
            uint32_t ve[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint64_t hh = H[c0 / 2 + j], ll = L[c0 / 2 + j];
              if (monoe) {
                const int n0 = T.b_row0 + col0 + c0 + 2 * j;
                float2 m0 = make_float2(0.0f, 0.0f), m1 = m0;
                if (sce) {
                  if (n0 < n_be) m0 = make_float2(sce[n0].z, sce[n0].w);
                  if (n0 + 1 < n_be) m1 = make_float2(sce[n0 + 1].z, sce[n0 + 1].w);
                } else {
                  if (n0 < n_be) m0 = monoe[n0];
                  if (n0 + 1 < n_be) m1 = monoe[n0 + 1];
                }
                uint64_t sm, em;
                two_sum2(hh, pk2(m0.x, m1.x), sm, em);
                hh = sm;
                ll = add2(ll, add2(em, pk2(m0.y, m1.y)));
              }
              float e0, e1;
              upk2(add2(hh, ll), e0, e1);
              ve[2 * j] = __float_as_uint(e0);
              ve[2 * j + 1] = __float_as_uint(e1);
              H[c0 / 2 + j] = L[c0 / 2 + j] = 0ull;
            }
            tmem_st8(tmem + t_lane + C::E_COL0 + col0 + c0, ve);
          }
          tmem_st_wait();
        }
      }
      if (!ok || !active) continue;
      // this tile's output arguments in registers (the stores below cannot alias them)
      const int n_b = R.A->n_b, ldp = R.A->ldp, symmetric = R.A->symmetric;
      float2* const part = R.A->part;
      const float4* const sc = R.A->sc;
      const float2* const mono = R.A->mono;
      double* const phi = R.phi;
      const long long nang = MODE == kSynthesize ? R.A->pt.nang[T.g_patch] : 0;
      const long long off0 = MODE == kSynthesize ? R.A->pt.fld_off[symmetric ? 0 : T.g_patch] : 0;
      const long long off1 = MODE == kSynthesize && symmetric ? R.A->pt.fld_off[1] : 0;
      const long long phi_len = R.A->pt.n_cells;  // the checked build's bound for Phi
      (void)phi_len;
      if (EMU && MODE == kSynthesize) {
        // output in float-float: Phi_Yin = E + O, Phi_Yang = E - O (or Phi_g),
        // each widened to FP64 as head + tail with the shell's power of two
        const long long a_loc = (long long)T.m_loc * BM + r;
#pragma unroll
        for (int c0 = 0; c0 < NH; c0 += 8) {
          uint32_t eh[8], el[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) eh[jj] = el[jj] = 0u;
          if (nseg == 2) {
            tmem_ld8(tmem + t_lane + C::E_COL0 + col0 + c0, eh);
            tmem_ld8(tmem + t_lane + C::E_COL0 + NMAX + col0 + c0, el);
            tmem_ld_wait();
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = c0 + jj;
            float h0, h1, l0, l1;
            upk2(H[j / 2], h0, h1);
            upk2(L[j / 2], l0, l1);
            const float oh = (j & 1) ? h1 : h0, ol = (j & 1) ? l1 : l0;
            const int n = T.b_row0 + col0 + j;
            if (n >= n_b || a_loc >= nang) continue;
            const unsigned int c20 = sc ? (unsigned int)__float_as_int(sc[n].x) : (896u << 20);
            if (nseg == 2 || symmetric) {
              // E from TMEM (zero without two column blocks: then the sums are E and O = 0)
              const float e_h = nseg == 2 ? __uint_as_float(eh[jj]) : oh;
              const float e_l = nseg == 2 ? __uint_as_float(el[jj]) : ol;
              const float o_h = nseg == 2 ? oh : 0.0f, o_l = nseg == 2 ? ol : 0.0f;
              float s, e;
              two_sum(e_h, o_h, s, e);
              float2 v = ff_renorm(s, e + (e_l + o_l));
              if (YGS_IN_BOUNDS(off0 + (long long)n * nang + a_loc, phi_len, kSiteGemmPhi)) phi[off0 + (long long)n * nang + a_loc] = f32_to_f64_pow2(v.x, c20) + f32_to_f64_pow2(v.y, c20);
              if (symmetric) {
                two_sum(e_h, -o_h, s, e);
                v = ff_renorm(s, e + (e_l - o_l));
                if (YGS_IN_BOUNDS(off1 + (long long)n * nang + a_loc, phi_len, kSiteGemmPhi)) phi[off1 + (long long)n * nang + a_loc] = f32_to_f64_pow2(v.x, c20) + f32_to_f64_pow2(v.y, c20);
              }
            } else {
              if (YGS_IN_BOUNDS(off0 + (long long)n * nang + a_loc, phi_len, kSiteGemmPhi)) phi[off0 + (long long)n * nang + a_loc] = f32_to_f64_pow2(oh, c20) + f32_to_f64_pow2(ol, c20);
            }
          }
        }
        continue;
      }
      // output, 8 columns at a time (keeps the register footprint of the sums)
#pragma unroll
      for (int c0 = 0; c0 < NH; c0 += 8) {
        float ev[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) ev[jj] = 0.0f;
        if (MODE == kSynthesize && nseg == 2) {
          uint32_t eu[8];
          tmem_ld8(tmem + t_lane + C::E_COL0 + col0 + c0, eu);
          tmem_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) ev[jj] = __uint_as_float(eu[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = c0 + jj;
          float h0, h1, l0, l1;
          upk2(H[j / 2], h0, h1);
          upk2(L[j / 2], l0, l1);
          const float hj = (j & 1) ? h1 : h0, lj = (j & 1) ? l1 : l0;
          const int n = T.b_row0 + col0 + j;
          if (n >= n_b) continue;
          if (MODE == kProject) {
            if (T.a_row0 + r < T.a_rows_end) {
              float s, e;
              two_sum(hj, lj, s, e);
              const long long pi = ((long long)T.z * n_b + n) * ldp + T.a_row0 + r;
              if (YGS_IN_BOUNDS(pi, (long long)R.A->n_chunks * n_b * ldp, kSiteGemmPart)) part[pi] = make_float2(s, e);
            }
          } else {
            const long long a_loc = (long long)T.m_loc * BM + r;
            if (a_loc >= nang) continue;
            const float hs = hj, ls = lj, e0 = ev[jj];
            // FP16 slices: the exact unscaling, applied when widening to FP64
            const unsigned int c20 = sc ? (unsigned int)__float_as_int(sc[n].x) : (896u << 20);
            float v = hs + ls;
            if (mono && nseg == 1) {
              // without two column blocks the monopole belongs to the only one
              // (with them, to E, where it was added when E was parked)
              const float2 mm = sc ? make_float2(sc[n].z, sc[n].w) : mono[n];
              float s, e;
              two_sum(hs, mm.x, s, e);
              v = s + (e + mm.y + ls);
            }
            if (symmetric) {
              // Yin-Yang: Phi_Yin = E + O, Phi_Yang = E - O (O = 0 when there are no odd columns)
              const float ee = (nseg == 2) ? e0 : v, oo = (nseg == 2) ? v : 0.0f;
              if (YGS_IN_BOUNDS(off0 + (long long)n * nang + a_loc, phi_len, kSiteGemmPhi)) phi[off0 + (long long)n * nang + a_loc] = f32_to_f64_pow2(ee + oo, c20);
              if (YGS_IN_BOUNDS(off1 + (long long)n * nang + a_loc, phi_len, kSiteGemmPhi)) phi[off1 + (long long)n * nang + a_loc] = f32_to_f64_pow2(ee - oo, c20);
            } else {
              if (YGS_IN_BOUNDS(off0 + (long long)n * nang + a_loc, phi_len, kSiteGemmPhi)) phi[off0 + (long long)n * nang + a_loc] = f32_to_f64_pow2(v, c20);
            }
          }
        }
      }
    }
    if (!ok) {
      set_err(err, YGS_ERR_TIMEOUT);
      *abort_flag = 1;
    }
  }

  tc_fence_before();
  __syncthreads();
  // pairs: neither CTA leaves while the other may still signal its barriers
  if constexpr (CG == 2) cluster_sync();
  tc_fence_after();
  if (warp == 0) tmem_dealloc<CG>(tmem, 512);
}

// setmaxnreg.inc waits for registers out of the CTA's launch allocation, so
// the split above holds only if the compiled kernel's register count is the
// REGS_LAUNCH it assumes: the host refuses a kernel whose count differs (a
// compiler that allocated fewer would otherwise leave the epilogue waiting).
template <int MODE, bool EMU>
inline cudaError_t check_reg_split(const void* fn) {
  if (!YGS_TC_SETMAXNREG) return cudaSuccess;
  cudaFuncAttributes at;
  const cudaError_t e = cudaFuncGetAttributes(&at, fn);
  if (e != cudaSuccess) return e;
  return at.numRegs == TileShape<MODE, EMU>::REGS_LAUNCH ? cudaSuccess : cudaErrorInvalidKernelImage;
}

// Registers: one CTA per SM takes the whole register file at launch
// (TileShape::REGS_LAUNCH per thread), which setmaxnreg then moves from
// warpgroup 0 to the epilogue warpgroups (TileShape::REGS_LOW, REGS_EPI).
// One problem: maps and arguments in kernel parameters.
// CG = 2: launched in clusters of two CTAs (the grid even), B's maps with
// boxes of half a tile's shells.
template <int NSL, int MODE, bool SCALE, bool TF = false, bool EMU = false, int CG = 1>
__global__ void __launch_bounds__(TileShape<MODE, EMU>::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapBt, const __grid_constant__ TcArgs args) {
  if (threadIdx.x == 0) {
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
    prefetch_tmap(&mapBt);
  }
  const SingleSrc src{&args, &mapA, &mapB, &mapBt};
  gemm_body<NSL, MODE, SCALE, TF, EMU, CG>(src);
}

// Several problems of one operand type in one persistent launch (a batch of
// fields): every CTA walks the concatenated tile list; TMEM accumulators and
// shared-memory stages carry over from one problem to the next.
template <int NSL, int MODE, bool SCALE, bool TF = false, bool EMU = false>
__global__ void __launch_bounds__(TileShape<MODE, EMU>::THREADS, 1)
    tc_gemm_group_kernel(const TcProblem* __restrict__ probs, const int* __restrict__ start, int n, int total,
                         const __grid_constant__ TcPhiList phis) {
  const GroupSrc src{probs, start, n, total, &phis};
  gemm_body<NSL, MODE, SCALE, TF, EMU, 1>(src);
}

}  // namespace tc
}  // namespace ygs
