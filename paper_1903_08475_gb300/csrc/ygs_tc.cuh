// tcgen05 (5th-generation tensor core) building blocks for sm_103a: mbarriers,
// TMA tile loads, TMEM allocation, UMMA descriptors and issue, TMEM loads.
// Every wait is bounded: on expiry the caller sets the plan's error word and
// leaves its loop instead of spinning forever.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ygs {
namespace tc {

constexpr uint32_t kSpinLimit = 1u << 26;  // try_wait polls (each may sleep ~us): seconds, not forever

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of `bar` with the given parity to complete.  Returns
// false if it did not within the spin limit or another role already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}

// 3-D tiled TMA load into shared memory, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Per-thread register allocation of a whole warpgroup (all its threads
// execute it together): .dec returns registers to the CTA's pool, .inc waits
// for them there.
template <int R>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(R));
}
template <int R>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(R));
}

// Plain bulk copy global -> shared (no tensor map): `bytes` a multiple of 16,
// both addresses 16-byte aligned; completion counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// ---- CTA pairs (a cluster of two CTAs sharing one MMA, cta_group::2) ----------
// Rank of this CTA in its cluster.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Shared::cluster address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Arrives on an mbarrier of another CTA of the cluster (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// try_wait with acquire at cluster scope: for barriers that other CTAs arrive on.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}
// Every thread of both CTAs of the cluster (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// 3-D tiled TMA load into this CTA's shared memory whose completion is counted
// on an mbarrier of either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x, int y,
                                                 int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
      "%5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(bar_cluster), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// ---- TMEM -------------------------------------------------------------------
// CG = 2: one warp of each CTA of the pair allocates; the same columns in both.
template <int CG = 1>
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {  // whole warp
  if constexpr (CG == 2)
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
  else
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
template <int CG = 1>
__device__ __forceinline__ void tmem_relinquish() {
  if constexpr (CG == 2)
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  else
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int CG = 1>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
  if constexpr (CG == 2)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (bf16 or fp16 operands, fp32 accumulate).
// CG = 2 (issued by the even CTA of a pair): M = 256, A's rows 0-127 from this
// CTA's shared memory and 128-255 from the peer's at the same address, B's
// first N/2 rows from this CTA and the rest from the peer, D's rows split the
// same way over the two CTAs' TMEM.
template <int CG = 1>
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  if constexpr (CG == 2)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The same with TF32 operands (kind::tf32: FP32 storage read as TF32, K = 8 per instruction).
template <int CG = 1>
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (CG == 2)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// x rounded to TF32 (nearest, ties away): the value the tensor core reads, exactly.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Arrives once on `bar` when every tcgen05.mma issued so far by this thread
// has completed; CG = 2: on the barrier at the same address in both CTAs of
// the pair.
template <int CG = 1>
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  if constexpr (CG == 2)
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Stores 8 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- descriptors --------------------------------------------------------------
// Shared-memory matrix descriptor, K-major, 64-byte swizzle: rows of 64 bytes
// (32 bf16), 8-row atoms of 512 bytes, atoms packed along M/N (SBO = 512 B).
__device__ __forceinline__ uint64_t sdesc_kmajor_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);       // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;               // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                        // layout: SWIZZLE_64B
  return d;
}

// Same for 128-byte rows (64 bf16) with 128-byte swizzle: 8-row atoms of 1 KB.
__device__ __forceinline__ uint64_t sdesc_kmajor_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);       // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                        // layout: SWIZZLE_128B
  return d;
}

// Instruction descriptor of kind::f16 / kind::tf32 with fp32 accumulation, both operands K-major.
// ab_fmt: 0 = fp16, 1 = bf16 (kind::f16); 2 = tf32 (kind::tf32).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int ab_fmt) {
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// ---- float-float helpers -------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Packed FP32 pairs (two lanes in one 64-bit register, IEEE round-to-nearest
// per lane, no flush to zero): half the issue slots of the scalar forms.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Lane-wise TwoSum: s = fl(a + b) and e with a + b = s + e exactly.
__device__ __forceinline__ void two_sum2(uint64_t a, uint64_t b, uint64_t& s, uint64_t& e) {
  s = add2(a, b);
  const uint64_t bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// ---- float-float arithmetic (value = x + y, |y| <= ulp(x) / 2) -------------
// The split path's radial scans run on these: GB300 issues FP64 at about two
// FMAs per clock per SM, FP32 at 128, and the scans' results feed FP16 or
// BF16 slices, so 2^-44 (normwise) accuracy is ample.  Sums are the
// "sloppy" float-float addition: error <= 2^-44 (|a| + |b|).
__device__ __forceinline__ float2 ff_renorm(float s, float e) {  // FastTwoSum, |s| >= |e|
  const float h = s + e;
  return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  return ff_renorm(s, e + (a.y + b.y));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  return ff_renorm(p, fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p))));
}
__device__ __forceinline__ float2 ff_fma(float2 a, float2 b, float2 c) { return ff_add(ff_mul(a, b), c); }
// FP64 -> float-float (rounded head, rounded remainder): for tables made once
__device__ __forceinline__ float2 ff_from_f64(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// x * 2^e for |e| <= 252, as two exact multiplications by representable powers of two.
__device__ __forceinline__ float mul_pow2f(float x, int e) {
  e = max(-252, min(252, e));
  const int e1 = e / 2, e2 = e - e1;
  return (x * __int_as_float((127 + e1) << 23)) * __int_as_float((127 + e2) << 23);
}

// Exponent e with m * 2^e in [2^14, 2^15) for m > 0 (0 for m = 0): scales a
// row whose largest magnitude is m to the top of FP16's range.
__host__ __device__ __forceinline__ int fp16_row_exp(double m) {
  if (!(m > 0.0)) return 0;
  int e = 0;
  const double f = frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  (void)f;
  const int r = 15 - e;            // m 2^r in [2^14, 2^15)
  return r < -200 ? -200 : (r > 200 ? 200 : r);
}

// The same exponent for an FP32 m >= 0, from its bits (no FP64 instruction:
// GB300 runs those on a narrow pipe): frexp's exponent is the biased
// exponent - 126 for normal m, and -117 - clz(mantissa) for subnormal m.
__device__ __forceinline__ int fp16_row_exp_f(float m) {
  const unsigned int u = __float_as_uint(m);
  if (!(m > 0.0f)) return 0;
  const int be = (int)(u >> 23);
  const int e = be > 0 ? be - 126 : -117 - __clz(u & 0x7FFFFFu);
  const int r = 15 - e;
  return r < -200 ? -200 : (r > 200 ? 200 : r);
}

// Lane-wise FastTwoSum: s = fl(a + b), e = b - (s - a); exact (a + b = s + e)
// when |a| >= |b| or a = 0, otherwise within one rounding of b.
__device__ __forceinline__ void fast_two_sum2(uint64_t a, uint64_t b, uint64_t& s, uint64_t& e) {
  s = add2(a, b);
  e = sub2(b, sub2(s, a));
}

// Lane-wise FastTwoSum of a + v * f for a power-of-two f (v * f exact):
// s = fl(a + v f), e = v f - (s - a).
// Two floats from shared memory, kept in program order (volatile): a load
// the compiler may not hoist ahead of the TMEM loads it belongs with, so a
// fully unrolled flush does not hold every pair's factors at once.
__device__ __forceinline__ uint64_t lds_pair(const float* p) {
  uint64_t r;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(r) : "r"(smem_u32(p)));
  return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ void fast_two_sum_scaled2(uint64_t a, uint64_t v, uint64_t f, uint64_t& s, uint64_t& e) {
  const uint64_t vf = mul2(v, f);  // exact: f is a power of two
  s = add2(a, vf);
  e = sub2(vf, sub2(s, a));
}

// FP64 -> FP32 by truncation with integer operations only (GB300 runs FP64
// conversions on its narrow FP64 pipe): the head of f64_to_ff.
__device__ __forceinline__ float f64_trunc_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const unsigned int E = (hw >> 20) & 0x7FFu;  // biased FP64 exponent; FP32's normal range is 897..1150
  unsigned int m = ((E - 896u) << 23) | (((hw << 3) | (lw >> 29)) & 0x7FFFFFu);
  m = E < 897u ? 0u : (E > 1150u ? 0x7F800000u : m);  // selects, no branches
  return __uint_as_float((hw & 0x80000000u) | m);
}

// FP64 -> FP32 rounded to nearest (ties away from zero) with integer
// operations: the exponent and the top 23 mantissa bits, plus the first
// dropped bit (a carry into the exponent is the correct rounding, and 2^128
// gives infinity).  Exponents below FP32's normal range give a signed zero,
// above it an infinity, as the truncating conversions here.
__device__ __forceinline__ float f64_round_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const unsigned int E = (hw >> 20) & 0x7FFu;
  unsigned int m = (((E - 896u) << 23) | (((hw << 3) | (lw >> 29)) & 0x7FFFFFu)) + ((lw >> 28) & 1u);
  m = E < 897u ? 0u : (E > 1150u ? 0x7F800000u : m);
  return __uint_as_float((hw & 0x80000000u) | m);
}

// FP64 -> (hi, lo) FP32 pair with integer operations and one exact FP32
// subtraction: hi = the top 24 significant bits (truncated), lo = the next 23
// bits (truncated), so hi + lo keeps 47 bits.  Exponents below FP32's normal
// range give zeros; above it, an infinite hi.
__device__ __forceinline__ void f64_to_ff_fast(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126) {
    hi = lo = __int_as_float((int)sign);
    return;
  }
  if (e > 127) {
    hi = __int_as_float((int)(sign | 0x7F800000u));
    lo = 0.0f;
    return;
  }
  hi = __int_as_float((int)(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu)));
  if (e < -103) {
    lo = 0.0f;
    return;
  }
  // 1.f x 2^(e-23) minus 2^(e-23): the low mantissa bits, exactly (same exponent)
  const unsigned int eb = sign | ((unsigned int)(e - 23 + 127) << 23);
  lo = __int_as_float((int)(eb | (unsigned int)((b >> 6) & 0x7FFFFFu))) - __int_as_float((int)eb);
}

// x * f1 * f2 with the factors of pow2_pair(e): an exact power-of-two scaling.
__device__ __forceinline__ void pow2_pair(int e, float& f1, float& f2) {
  e = max(-252, min(252, e));
  const int e1 = e / 2, e2 = e - e1;
  f1 = __int_as_float((127 + e1) << 23);
  f2 = __int_as_float((127 + e2) << 23);
}

// FP64 -> (hi, lo) FP32 pair by bit manipulation (no FP64 arithmetic): hi keeps
// the top 24 significant bits (truncated), lo the next 24.  Values whose
// exponent is outside the normal FP32 range flush to zero / saturate.
__device__ __forceinline__ void f64_to_ff(double x, float& hi, float& lo) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned int sign = (unsigned int)(b >> 63) << 31;
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e < -126) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  if (e > 127) {
    hi = __int_as_float((int)(sign | 0x7F800000u));
    lo = 0.0f;
    return;
  }
  hi = __int_as_float((int)(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29)));
  unsigned int r = (unsigned int)(m & 0x1FFFFFFFull);  // 29 remaining bits, weight 2^(e-52)
  if (r == 0 || e - 52 + 29 < -126) {
    lo = 0.0f;
    return;
  }
  int lz = __clz(r) - 3;                    // leading zeros within the 29-bit field
  int top = 28 - lz;                        // index of the leading set bit
  int ee = e - 52 + top;                    // exponent of the leading bit
  unsigned int mant = (top >= 23) ? (r >> (top - 23)) : (r << (23 - top));
  if (ee < -126) {
    lo = 0.0f;
    return;
  }
  lo = __int_as_float((int)(sign | ((unsigned int)(ee + 127) << 23) | (mant & 0x7FFFFFu)));
}

// (hi, lo) -> up to three BF16 slices: v ~ s0 + s1 + s2 (each the RN BF16 of the remainder).
__device__ __forceinline__ void ff_to_bf16x3(float hi, float lo, __nv_bfloat16& s0, __nv_bfloat16& s1,
                                             __nv_bfloat16& s2) {
  s0 = __float2bfloat16_rn(hi);
  float r1 = hi - __bfloat162float(s0);  // exact
  s1 = __float2bfloat16_rn(r1);
  float r2 = (r1 - __bfloat162float(s1)) + lo;
  s2 = __float2bfloat16_rn(r2);
}

// ---- grouped launches of per-field kernels (batches) -----------------------
// A kernel body takes its block indices as a VBlock: a plain launch passes its
// own; a grouped launch runs the blocks of several problems (one per field
// of a batch) in one grid, problem k owning the flat blocks [start, start +
// gx gy gz) of GroupDims k, and hands each block its problem's indices.
struct VBlock {
  int x, y, z, gx;
};
__device__ __forceinline__ VBlock vblock_self() {
  return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x};
}
struct GroupDims {
  int gx, gy, gz, start;
};
constexpr int kMaxGroupFields = 128;  // problems per grouped launch
struct RhoList {                      // the fields of a grouped launch
  const double* p[kMaxGroupFields];
};
// The problem of flat block b (the last with start <= b) and b's indices in it.
__device__ __forceinline__ int locate_block(const GroupDims* __restrict__ dims, int n, int b, VBlock& vb) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (dims[mid].start <= b) lo = mid; else hi = mid - 1;
  }
  const GroupDims d = dims[lo];
  const int local = b - d.start;
  vb.x = local % d.gx;
  vb.y = (local / d.gx) % d.gy;
  vb.z = local / (d.gx * d.gy);
  vb.gx = d.gx;
  return lo;
}

}  // namespace tc
}  // namespace ygs
