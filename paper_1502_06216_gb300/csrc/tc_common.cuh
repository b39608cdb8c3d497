// tc_common.cuh -- shared pieces of the tensor-core kernels (internal): tile
// constants, tcgen05 / TMA / mbarrier PTX wrappers, the 128-byte-swizzled
// shared-memory layouts of the epilogue tiles, tensor-map encoding, and the
// per-handle plan of images, factors and maps.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "jko.h"
#include "jko_kernels.h"
#include "tc_gemm.h"

namespace jko {

namespace {


constexpr int BM = 128;            // UMMA M (rows of the kernel factor per tile)
constexpr int KB_BYTES = 128;      // K-block width in bytes (one 128-byte swizzle row)
constexpr int MAX_STAGES = 8;
constexpr uint32_t SMEM_BUDGET = 212 * 1024;  // operand stages + epilogue tiles per CTA
constexpr int NT = 512;            // threads per CTA: 16 warps, 4 per TMEM lane quadrant
constexpr int NWG = NT / 128;      // warps sharing one quadrant (column groups)
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier polls

enum : int { MODE_BF16 = 0, MODE_BF16X3 = 1, MODE_TF32 = 2 };

// Operand forms.  TF32: one tf32 x tf32 product.  BF16: the Gibbs factor in
// bf16, every image operand (a, b and the intermediate) as a pair x = hi + lo
// of bf16, so one product K_hi . (x_hi + x_lo); a single bf16 image rounds
// the smooth scalings the same way over whole regions and costs up to 4e-3
// of relative L1 in one pair, the pair ~2e-5.  BF16X3: also the factor as a
// pair, K_hi . (x_hi + x_lo) + K_lo . x_hi.  The image pair sits in one
// shared-memory block of 2 BN rows (hi rows, then lo rows), so K_hi . [x_hi;
// x_lo] is one MMA of width 2 BN whose accumulator halves are added in the
// epilogue.
__host__ __device__ constexpr bool img_split(int mode) { return mode != MODE_TF32; }
__host__ __device__ constexpr bool fac_split(int mode) { return mode == MODE_BF16X3; }

// Bytes of one pipeline stage: factor hi, image hi, image lo, factor lo.
__host__ __device__ constexpr uint32_t stage_bytes(int mode, int bn) {
  return ((fac_split(mode) ? 2u : 1u) * (uint32_t)BM + (img_split(mode) ? 2u : 1u) * (uint32_t)bn) *
         (uint32_t)KB_BYTES;
}
// Epilogue tiles kept beside the stages: b-update pass -> q (fp32) and the old
// b (operand type, hi [+ lo]); prox pass -> e^{-sigma w} (fp32) and the staged
// p (fp32).  Epilogue numbering as in jko_kernels.h (0 store, 1 b, 2 a).
__host__ __device__ constexpr uint32_t epi_bytes(int mode, int epi, int bn) {
  return epi == 0 ? 0u
         : epi == 1 ? (uint32_t)bn * BM * 4u +
                          (img_split(mode) ? 2u : 1u) * (uint32_t)bn * BM *
                              (mode == MODE_TF32 ? 4u : 2u)
                    : 2u * (uint32_t)bn * BM * 4u;
}
// Bytes the producer loads into the epilogue tiles (the p tile is only stored).
__host__ __device__ constexpr uint32_t epi_load_bytes(int mode, int epi, int bn) {
  return epi == 2 ? (uint32_t)bn * BM * 4u : epi_bytes(mode, epi, bn);
}
__host__ __device__ constexpr int num_stages(int mode, int epi, int bn) {
  return (SMEM_BUDGET - epi_bytes(mode, epi, bn)) / stage_bytes(mode, bn) < (uint32_t)MAX_STAGES
             ? (int)((SMEM_BUDGET - epi_bytes(mode, epi, bn)) / stage_bytes(mode, bn))
             : MAX_STAGES;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after kSpinLimit polls (the caller records a fault).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}
// Programmatic dependent launch: the next kernel of the stream may start its
// set-up once every CTA of this one has signalled; griddepcontrol.wait blocks
// until the preceding kernel has completed and its writes are visible.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
template <int MODE>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                     uint32_t idesc, uint32_t accum) {
  if (MODE == MODE_TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}
// The MMAs of one 16-byte-aligned K-step kk (0..3) of a stage: a_hi / a_lo
// are the factor halves, b the image block (hi rows then lo rows when split);
// accum = 0 starts the accumulator.  Accumulator columns: [0, BN) the hi
// product (plus K_lo . x_hi), [BN, 2 BN) the lo product.
template <int MODE, int BN>
__device__ __forceinline__ void umma_kstep(uint32_t tmem_d, uint64_t a_hi, uint64_t a_lo,
                                           uint64_t b, int kk, uint32_t accum);
template <int MODE>
__host__ __device__ constexpr uint32_t make_idesc(int M, int N);
// TMEM columns of a BN-wide tile's accumulator (a power of two >= 32).
__host__ __device__ constexpr uint32_t acc_cols(int mode, int bn) {
  return (img_split(mode) ? 2u : 1u) * (uint32_t)bn < 32u ? 32u
                                                           : (img_split(mode) ? 2u : 1u) * (uint32_t)bn;
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x,
                                             int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          (uint64_t)map),
      "r"(smem_u32(src)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// All bulk groups but the most recent one complete (their writes done).
__device__ __forceinline__ void bulk_wait_all_but_last() {
  asm volatile("cp.async.bulk.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Barrier among the first `n` threads (whole warps) of the block, id 1..15.
__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Issue-only TMEM load of 16 columns (32-bit) of this warp's 32 lanes; the
// values are valid after tmem_wait_ld() and reg_fence16().
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Issue-only TMEM load of 4 columns (32-bit) of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld4_issue(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
// Issue-only TMEM load of 8 columns (32-bit) of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void reg_fence8(uint32_t (&r)[8]) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                    "+r"(r[6]), "+r"(r[7]));
}
__device__ __forceinline__ void reg_fence4(uint32_t (&r)[4]) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// TMEM store of 16 columns (32-bit) of this warp's 32 lanes; complete for the
// issuing thread after tmem_wait_st().
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
        "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]),
        "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Ties the registers of an issued TMEM load to the point after the wait, so
// that the compiler schedules no use of them before it.
__device__ __forceinline__ void reg_fence16(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row swizzle atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);      // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor: D f32, A/B bf16 (kind::f16) or tf32, both K-major.
template <int MODE>
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | ((MODE == MODE_TF32 ? 2u : 1u) << 7) | ((MODE == MODE_TF32 ? 2u : 1u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int MODE, int BN>
__device__ __forceinline__ void umma_kstep(uint32_t tmem_d, uint64_t a_hi, uint64_t a_lo,
                                           uint64_t b, int kk, uint32_t accum) {
  const uint64_t adv = (uint64_t)(kk * 2);   // +32 bytes of K in 16-byte units
  if constexpr (!img_split(MODE)) {
    umma<MODE>(tmem_d, a_hi + adv, b + adv, make_idesc<MODE>(BM, BN), accum);
  } else {
    umma<MODE>(tmem_d, a_hi + adv, b + adv, make_idesc<MODE>(BM, 2 * BN), accum);
    if constexpr (fac_split(MODE)) umma<MODE>(tmem_d, a_lo + adv, b + adv, make_idesc<MODE>(BM, BN), 1u);
  }
}

// 16 accumulator columns c0 .. c0+15 of this warp's 32 TMEM lanes as floats:
// the hi and lo products added (split images) or the single product.
template <int MODE, int BN>
__device__ __forceinline__ void tmem_tile16(uint32_t taddr_lane, int c0, float (&v)[16]) {
  uint32_t r0[16];
  tmem_ld16_issue(taddr_lane + (uint32_t)c0, r0);
  if constexpr (img_split(MODE)) {
    uint32_t r1[16];
    tmem_ld16_issue(taddr_lane + (uint32_t)(BN + c0), r1);
    tmem_wait_ld();
    reg_fence16(r0);
    reg_fence16(r1);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
  } else {
    tmem_wait_ld();
    reg_fence16(r0);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r0[j]);
  }
}

template <int MODE> struct OpT;
template <> struct OpT<MODE_BF16> { using T = __nv_bfloat16; static constexpr int kElems = 64; };
template <> struct OpT<MODE_BF16X3> { using T = __nv_bfloat16; static constexpr int kElems = 64; };
template <> struct OpT<MODE_TF32> { using T = float; static constexpr int kElems = 32; };

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// The value an image element takes once stored as operand (tf32, or the
// bf16 pair hi + lo), as the kernels read it back.
template <int MODE>
__device__ __forceinline__ float op_value(float v) {
  if constexpr (MODE == MODE_TF32) {
    return tf32_round(v);
  } else {
    const float h = __bfloat162float(__float2bfloat16_rn(v));
    return h + __bfloat162float(__float2bfloat16_rn(v - h));
  }
}

// Operand value of one image element (hi [+ lo]) as float.
template <int MODE, typename T>
__device__ __forceinline__ float op_load(const T* hi, const T* lo, size_t i) {
  if constexpr (MODE == MODE_TF32) return hi[i];
  else return __bfloat162float(hi[i]) + __bfloat162float(lo[i]);
}
template <int MODE, typename T>
__device__ __forceinline__ void op_store(T* hi, T* lo, size_t i, float v) {
  if constexpr (MODE == MODE_TF32) {
    hi[i] = tf32_round(v);
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// 16 consecutive fp32 of one row: vector loads when the row segment is
// 16-byte aligned and complete, scalar loads of the first `cnt` otherwise.
__device__ __forceinline__ void load_f32x16(const float* src, int cnt, bool vec, float (&o)[16]) {
  if (vec && cnt == 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(src) + q);
      o[4 * q] = t.x; o[4 * q + 1] = t.y; o[4 * q + 2] = t.z; o[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = j < cnt ? src[j] : 0.0f;
  }
}
__device__ __forceinline__ void store_f32x16(float* dst, int cnt, bool vec, const float (&v)[16]) {
  if (vec && cnt == 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      reinterpret_cast<float4*>(dst)[q] =
          make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < cnt) dst[j] = v[j];
  }
}
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_bf16x2(uint32_t u) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
  return __bfloat1622float2(h);
}
// 16 operand-typed values of one row (rows padded to 16 bytes): the value is
// hi (+ lo).  Vector loads when the 16 lie inside the valid columns.
template <int MODE, typename T>
__device__ __forceinline__ void load_op16(const T* hi, const T* lo, size_t off, int cnt,
                                          float (&o)[16]) {
  if (cnt == 16) {
    if constexpr (MODE == MODE_TF32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(hi + off)[q];
        o[4 * q] = t.x; o[4 * q + 1] = t.y; o[4 * q + 2] = t.z; o[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint4 t = reinterpret_cast<const uint4*>(hi + off)[q];
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 f = unpack_bf16x2(w[k]);
          o[8 * q + 2 * k] = f.x; o[8 * q + 2 * k + 1] = f.y;
        }
      }
      if constexpr (img_split(MODE)) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint4 t = reinterpret_cast<const uint4*>(lo + off)[q];
          const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 f = unpack_bf16x2(w[k]);
            o[8 * q + 2 * k] += f.x; o[8 * q + 2 * k + 1] += f.y;
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = j < cnt ? op_load<MODE>(hi, lo, off + j) : 0.0f;
  }
}
// load_op16 through L2 only (ld.global.cg): for an image this CTA rewrites
// with TMA stores between its reads, where an L1 copy from the previous read
// would be stale.
template <int MODE, typename T>
__device__ __forceinline__ void load_op16_cg(const T* hi, const T* lo, size_t off, int cnt,
                                             float (&o)[16]) {
  if (cnt == 16) {
    if constexpr (MODE == MODE_TF32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = __ldcg(reinterpret_cast<const float4*>(hi + off) + q);
        o[4 * q] = t.x; o[4 * q + 1] = t.y; o[4 * q + 2] = t.z; o[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint4 t = __ldcg(reinterpret_cast<const uint4*>(hi + off) + q);
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 f = unpack_bf16x2(w[k]);
          o[8 * q + 2 * k] = f.x; o[8 * q + 2 * k + 1] = f.y;
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint4 t = __ldcg(reinterpret_cast<const uint4*>(lo + off) + q);
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 f = unpack_bf16x2(w[k]);
          o[8 * q + 2 * k] += f.x; o[8 * q + 2 * k + 1] += f.y;
        }
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float x = 0.0f;
      if (j < cnt) {
        if constexpr (MODE == MODE_TF32) {
          x = __ldcg(hi + off + j);
        } else {
          const unsigned short h = __ldcg(reinterpret_cast<const unsigned short*>(hi + off + j));
          const unsigned short l = __ldcg(reinterpret_cast<const unsigned short*>(lo + off + j));
          x = __uint_as_float((uint32_t)h << 16) + __uint_as_float((uint32_t)l << 16);
        }
      }
      o[j] = x;
    }
  }
}

// Writes 16 values of local row r, columns 16c .. 16c+15, into the staging
// tile in the layout of a 128-byte-swizzled TMA box of 128 rows: column block
// cb holds 128 bytes per row; the 16-byte chunk k of row r sits at k ^ (r & 7).
template <int MODE>
__device__ __forceinline__ void stage16(unsigned char* st_hi, unsigned char* st_lo, int r, int c,
                                        const float (&o)[16]) {
  constexpr uint32_t BLK = BM * 128;
  if constexpr (MODE == MODE_TF32) {
    const int cb = c >> 1, k0 = (c & 1) * 4;
    unsigned char* row = st_hi + cb * BLK + r * 128;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 u;
      u.x = __float_as_uint(tf32_round(o[4 * q]));
      u.y = __float_as_uint(tf32_round(o[4 * q + 1]));
      u.z = __float_as_uint(tf32_round(o[4 * q + 2]));
      u.w = __float_as_uint(tf32_round(o[4 * q + 3]));
      *reinterpret_cast<uint4*>(row + (((k0 + q) ^ (r & 7)) << 4)) = u;
    }
  } else {
    const int cb = c >> 2, k0 = (c & 3) * 2;
    unsigned char* row_hi = st_hi + cb * BLK + r * 128;
    unsigned char* row_lo = st_lo + cb * BLK + r * 128;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float h[8], l[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float v = o[8 * q + k];
        h[k] = __bfloat162float(__float2bfloat16_rn(v));
        l[k] = v - h[k];
      }
      uint4 u;
      u.x = pack_bf16x2(h[0], h[1]); u.y = pack_bf16x2(h[2], h[3]);
      u.z = pack_bf16x2(h[4], h[5]); u.w = pack_bf16x2(h[6], h[7]);
      *reinterpret_cast<uint4*>(row_hi + (((k0 + q) ^ (r & 7)) << 4)) = u;
      if constexpr (img_split(MODE)) {
        uint4 w;
        w.x = pack_bf16x2(l[0], l[1]); w.y = pack_bf16x2(l[2], l[3]);
        w.z = pack_bf16x2(l[4], l[5]); w.w = pack_bf16x2(l[6], l[7]);
        *reinterpret_cast<uint4*>(row_lo + (((k0 + q) ^ (r & 7)) << 4)) = w;
      }
    }
  }
}

// 16 fp32 of row r, columns 16c .. 16c+15, of a 128-byte-swizzled fp32 tile
// (column blocks of 32 floats x 128 rows, 16-byte chunk k of row r at k ^ (r & 7)).
__device__ __forceinline__ void smem_ld_f32x16(const unsigned char* reg, int r, int c,
                                               float (&o)[16]) {
  const int cb = c >> 1, k0 = (c & 1) * 4;
  const unsigned char* row = reg + cb * (BM * 128) + r * 128;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 t = *reinterpret_cast<const float4*>(row + (((k0 + q) ^ (r & 7)) << 4));
    o[4 * q] = t.x; o[4 * q + 1] = t.y; o[4 * q + 2] = t.z; o[4 * q + 3] = t.w;
  }
}
__device__ __forceinline__ void smem_st_f32x16(unsigned char* reg, int r, int c,
                                               const float (&v)[16]) {
  const int cb = c >> 1, k0 = (c & 1) * 4;
  unsigned char* row = reg + cb * (BM * 128) + r * 128;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<float4*>(row + (((k0 + q) ^ (r & 7)) << 4)) =
        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
// 16 operand values (hi [+ lo]) of row r, columns 16c .., from swizzled tiles.
template <int MODE>
__device__ __forceinline__ void smem_ld_op16(const unsigned char* hi, const unsigned char* lo,
                                             int r, int c, float (&o)[16]) {
  if constexpr (MODE == MODE_TF32) {
    smem_ld_f32x16(hi, r, c, o);
  } else {
    const int cb = c >> 2, k0 = (c & 3) * 2;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const size_t off = cb * (BM * 128) + r * 128 + (((k0 + q) ^ (r & 7)) << 4);
      const uint4 t = *reinterpret_cast<const uint4*>(hi + off);
      const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = unpack_bf16x2(w[k]);
        o[8 * q + 2 * k] = f.x; o[8 * q + 2 * k + 1] = f.y;
      }
      if constexpr (img_split(MODE)) {
        const uint4 u = *reinterpret_cast<const uint4*>(lo + off);
        const uint32_t z[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 f = unpack_bf16x2(z[k]);
          o[8 * q + 2 * k] += f.x; o[8 * q + 2 * k + 1] += f.y;
        }
      }
    }
  }
}

// Four fp32 values (columns 16c + 4g .. + 3) of row r in a swizzled fp32 tile
// (the layout of smem_ld_f32x16 / smem_st_f32x16).
__device__ __forceinline__ float4 smem_ld_f32x4(const unsigned char* reg, int r, int c, int g) {
  const unsigned char* row = reg + (c >> 1) * (BM * 128) + r * 128;
  return *reinterpret_cast<const float4*>(row + ((((c & 1) * 4 + g) ^ (r & 7)) << 4));
}
__device__ __forceinline__ void smem_st_f32x4(unsigned char* reg, int r, int c, int g, float4 v) {
  unsigned char* row = reg + (c >> 1) * (BM * 128) + r * 128;
  *reinterpret_cast<float4*>(row + ((((c & 1) * 4 + g) ^ (r & 7)) << 4)) = v;
}
// Four operand values (hi [+ lo]) of row r, columns 16c + 4g .., from swizzled
// tiles (the layout of smem_ld_op16).
template <int MODE>
__device__ __forceinline__ void smem_ld_op4(const unsigned char* hi, const unsigned char* lo, int r,
                                            int c, int g, float (&o)[4]) {
  if constexpr (MODE == MODE_TF32) {
    const float4 t = smem_ld_f32x4(hi, r, c, g);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  } else {
    const int cb = c >> 2, unit = (c & 3) * 2 + (g >> 1);
    const size_t off = cb * (BM * 128) + r * 128 + ((unit ^ (r & 7)) << 4) + (g & 1) * 8;
    const uint2 t = *reinterpret_cast<const uint2*>(hi + off);
    const float2 f0 = unpack_bf16x2(t.x), f1 = unpack_bf16x2(t.y);
    o[0] = f0.x; o[1] = f0.y; o[2] = f1.x; o[3] = f1.y;
    if constexpr (img_split(MODE)) {
      const uint2 u = *reinterpret_cast<const uint2*>(lo + off);
      const float2 h0 = unpack_bf16x2(u.x), h1 = unpack_bf16x2(u.y);
      o[0] += h0.x; o[1] += h0.y; o[2] += h1.x; o[3] += h1.y;
    }
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D tensor map of a row-major [rows][pitch] operand matrix whose first
// `cols` columns are valid; box = box_rows x (128 bytes of K).
bool make_map(CUtensorMap* map, void* base, int mode, int rows, int cols, int pitch, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const int es = mode == MODE_TF32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * es};
  cuuint32_t box[2] = {(cuuint32_t)(KB_BYTES / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, mode == MODE_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

namespace {
// Band of one 128-row tile of a 1-D factor, as the kernels walk it: K-blocks
// of KE columns starting at column x (a multiple of 128 bytes), y blocks, and
// the first and last non-zero columns z, w.  Every K=UK sub-step of every
// block is issued: skipping the sub-steps outside [z, w], which multiply
// exact zeros, measured 7 % slower (25.4 against 23.8 us per pair at 1024^2).
// Executed multiply-add flops (x2) of one tile of width bn over its band.
inline double band_tile_flops(int4 kb, int KE, int bn, double mult) {
  return 2.0 * 128.0 * (double)bn * KE * kb.y * mult;
}

// Sum of one float per thread over 16 warps (threads 0..511) in a fixed order:
// each warp's butterfly, then warp 0 over the 16 warp sums.  `sync` is the
// barrier of those 512 threads.  The result is valid in thread 0.
template <typename Sync>
__device__ __forceinline__ float tile_sum16(float v, float* scratch, Sync sync) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_f(v);
  if (lane == 0) scratch[warp] = v;
  sync();
  float t = 0.0f;
  if (warp == 0) {
    t = lane < 16 ? scratch[lane] : 0.0f;
    t = warp_sum_f(t);
  }
  return t;
}
}  // namespace

struct TcPlan {
  TcConfig cfg;
  int mode = MODE_BF16;
  int bn_x = 64, bn_y = 64;   // BN of the pass over x (N = ny) and over y (N = nx)
  int rx = 0, ry = 0;          // band radii
  int px = 0, py = 0;          // pitches (elements) of images with x / y contiguous
  // factors [axis 0 = x, 1 = y][side 0 = a (xi a), 1 = b (xi b)][hi, lo]; without
  // absorption the b side aliases the a side (the factor is symmetric)
  void* k[2][2][2] = {};
  int4* kbt[2][2] = {};        // per-tile band of each factor (see band_tile)
  float* E_abs = nullptr;      // absorbed e^{-(sigma w + beta)} (congestion kind)
  float* sw_abs = nullptr;     // absorbed sigma w + beta (entropy kinds)
  int absorbed = 0;
  void* img_a[2] = {nullptr, nullptr};   // [ny][px]
  void* img_b[2] = {nullptr, nullptr};   // [ny][px]
  void* img_t[2] = {nullptr, nullptr};   // [nx][py]
  CUtensorMap mK[2][2][2];                          // factor loads [axis][side][split]
  CUtensorMap mA[2], mB[2], mT[2];                  // image operand loads
  CUtensorMap sA[2], sB[2], sT[2];                  // epilogue stores (box 128 rows)
  CUtensorMap fQ, fE, fP;                           // fp32 fields q, e^{-sigma w}, p
  int tma_epi = 0;
  double flops[4] = {0, 0, 0, 0};
  // image operand loads with 64-row boxes (64-wide tiles: per-pass kernels and
  // the persistent loop kernel); mA/mB/mT above have boxes of the wide tile
  CUtensorMap lA[2], lB[2], lT[2];
  // persistent pair-loop kernel (tc_loop.cu): support flag, grid size and
  // executed flops of one pair
  int loop_ok = 0;
  int loop_grid = 0;
  int loop_res = 0;            // the loop kernel keeps each CTA's factor band resident
  double loop_flops_pair = 0.0;
  // log-domain form (tc_log.cu, TF32): exponent per row and 32-cell group of
  // the images a, b ([ny][gx]) and T ([nx][gy]); -sigma w log2(e) as a
  // mantissa in [1, 2) and an integer exponent; per axis the factor scaled by
  // a power of two per row and K-block, those exponents [n][gk] and its band
  int logd = 0;
  int gx = 0, gy = 0;
  int* sh_a = nullptr;
  int* sh_b = nullptr;
  int* sh_t = nullptr;
  float* lwm = nullptr;
  int* lwe = nullptr;
  void* k_log[2] = {nullptr, nullptr};
  int* sk[2] = {nullptr, nullptr};
  int gk[2] = {0, 0};
  int4* kbt_log[2] = {nullptr, nullptr};
  CUtensorMap mKl[2];          // the scaled factors as A operands
  CUtensorMap l32[3];          // a, b, T loads in 32-row boxes
};

}  // namespace jko
