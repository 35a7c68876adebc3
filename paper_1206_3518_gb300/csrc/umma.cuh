// Helpers of the 5th-generation tensor-core kernels (tc.cu, tcpair.cu): bounded mbarrier waits,
// UMMA shared-memory and instruction descriptors, the BF16 MMA issue and its commit, and the
// 128-byte swizzle of K-major tile rows.
//
// Tile format: 128-byte rows holding 32 complex K values as [Re (32 BF16) | Im (32 BF16)], rows in
// 8-row atoms of 1024 bytes with 128B swizzle (16-byte chunk c of row r stored at chunk c ^ (r & 7)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace bse {
namespace umma {

constexpr int kRow = 128;                    // bytes per tile row
constexpr int kTM = 128;                     // MMA rows (M)

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait on an mbarrier phase; false after 2 s.  Each try_wait may suspend the thread for up to
// 20 us (it resumes as soon as the phase completes), so a waiting warp takes few issue slots.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000u)
        : "memory");
    if (ok) return true;
    if (gtimer() - t0 > 2000000000ull) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// UMMA shared-memory descriptor: K-major, 128B swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)1 << 16;                           // leading-dimension byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride-dimension byte offset
  d |= (uint64_t)1 << 46;                           // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                           // 128B swizzle
  return d;
}

// Instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = n; bit 13 negates A.
__host__ __device__ constexpr uint32_t idesc_of(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}
constexpr uint32_t kNegA = 1u << 13;

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// The twelve MMAs of 16 complex K values in BF16x3 split-complex form, A and B tiles (hi, lo) at
// shared addresses ah/al, bh/bl (kk selects the K16 half of the 32-value row):
//   Re D += Re A Re B - Im A Im B,   Im D += Re A Im B + Im A Re B,   each as hi.hi + hi.lo + lo.hi.
// init != 0 starts both accumulators.
__device__ __forceinline__ void mma_cplx_k16(uint32_t d_re, uint32_t d_im, uint32_t ah, uint32_t al, uint32_t bh,
                                             uint32_t bl, int kk, uint32_t idesc, bool init) {
  const uint32_t idesc_neg = idesc | kNegA;
#pragma unroll
  for (int s = 0; s < 3; ++s) {                 // hi.hi, hi.lo, lo.hi
    const uint32_t pa = ((s == 2) ? al : ah) + kk * 32, pb = ((s == 1) ? bl : bh) + kk * 32;
    const uint32_t acc = (init && s == 0) ? 0u : 1u;
    mma_bf16(d_re, smem_desc(pa), smem_desc(pb), idesc, acc);                // Re A Re B
    mma_bf16(d_re, smem_desc(pa + 64), smem_desc(pb + 64), idesc_neg, 1u);   // - Im A Im B
    mma_bf16(d_im, smem_desc(pa), smem_desc(pb + 64), idesc, acc);           // Re A Im B
    mma_bf16(d_im, smem_desc(pa + 64), smem_desc(pb), idesc, 1u);            // Im A Re B
  }
}

// The same twelve MMAs with precomputed descriptors: da / db of the hi tiles, a_lo / b_lo the offsets (in
// 16-byte units) of the lo tiles; K16 half kk at +2, the Im half at +4 (a descriptor's start address is
// its low 14 bits, address / 16, so a byte offset o adds o / 16).
__device__ __forceinline__ void mma_cplx_k16_desc(uint32_t d_re, uint32_t d_im, uint64_t da, uint32_t a_lo, uint64_t db,
                                                  uint32_t b_lo, int kk, uint32_t idesc, bool init) {
  const uint32_t idesc_neg = idesc | kNegA;
#pragma unroll
  for (int s = 0; s < 3; ++s) {                 // hi.hi, hi.lo, lo.hi
    const uint64_t pa = da + ((s == 2) ? a_lo : 0u) + (uint32_t)kk * 2u;
    const uint64_t pb = db + ((s == 1) ? b_lo : 0u) + (uint32_t)kk * 2u;
    const uint32_t acc = (init && s == 0) ? 0u : 1u;
    mma_bf16(d_re, pa, pb, idesc, acc);                 // Re A Re B
    mma_bf16(d_re, pa + 4u, pb + 4u, idesc_neg, 1u);    // - Im A Im B
    mma_bf16(d_im, pa, pb + 4u, idesc, acc);            // Re A Im B
    mma_bf16(d_im, pa + 4u, pb, idesc, 1u);             // Im A Re B
  }
}

// A from tensor memory (column address a of lane 0), B from shared memory.
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

// The twelve MMAs of 16 complex K values with the A planes in tensor memory at columns a + 0 (Re hi),
// a + 8 (Im hi), a + 16 (Re lo), a + 24 (Im lo) (two BF16 per 32-bit column, lane = row), B in shared
// memory as for mma_cplx_k16_desc.
__device__ __forceinline__ void mma_cplx_k16_ts(uint32_t d_re, uint32_t d_im, uint32_t a, uint64_t db, uint32_t b_lo,
                                                int kk, uint32_t idesc, bool init) {
  const uint32_t idesc_neg = idesc | kNegA;
#pragma unroll
  for (int s = 0; s < 3; ++s) {                 // hi.hi, hi.lo, lo.hi
    const uint32_t ar = a + ((s == 2) ? 16u : 0u), ai = ar + 8u;
    const uint64_t pb = db + ((s == 1) ? b_lo : 0u) + (uint32_t)kk * 2u;
    const uint32_t acc = (init && s == 0) ? 0u : 1u;
    mma_bf16_ts(d_re, ar, pb, idesc, acc);              // Re A Re B
    mma_bf16_ts(d_re, ai, pb + 4u, idesc_neg, 1u);      // - Im A Im B
    mma_bf16_ts(d_im, ar, pb + 4u, idesc, acc);         // Re A Im B
    mma_bf16_ts(d_im, ai, pb, idesc, 1u);               // Im A Re B
  }
}

// 32 consecutive TMEM columns of this warp's lane quarter from registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// The twelve MMAs of 16 complex K values for conj(A) B (descriptors as mma_cplx_k16_desc):
//   Re D += Re A Re B + Im A Im B,   Im D += Re A Im B - Im A Re B.
__device__ __forceinline__ void mma_cplx_conj_k16_desc(uint32_t d_re, uint32_t d_im, uint64_t da, uint32_t a_lo,
                                                       uint64_t db, uint32_t b_lo, int kk, uint32_t idesc, bool init) {
  const uint32_t idesc_neg = idesc | kNegA;
#pragma unroll
  for (int s = 0; s < 3; ++s) {                 // hi.hi, hi.lo, lo.hi
    const uint64_t pa = da + ((s == 2) ? a_lo : 0u) + (uint32_t)kk * 2u;
    const uint64_t pb = db + ((s == 1) ? b_lo : 0u) + (uint32_t)kk * 2u;
    const uint32_t acc = (init && s == 0) ? 0u : 1u;
    mma_bf16(d_re, pa, pb, idesc, acc);                 // Re A Re B
    mma_bf16(d_re, pa + 4u, pb + 4u, idesc, 1u);        // + Im A Im B
    mma_bf16(d_im, pa, pb + 4u, idesc, acc);            // Re A Im B
    mma_bf16(d_im, pa + 4u, pb, idesc_neg, 1u);         // - Im A Re B
  }
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk copy global -> shared (16-byte aligned, size a multiple of 16), completion counted on bar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// 16-byte chunk c of row r of a swizzled K-major tile (rows of 128 bytes).
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * kRow + ((c ^ (r & 7)) << 4)); }

// x = hi + lo in BF16 (round to nearest), two values per 32-bit word (element 2i in the low half).
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 back = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - back.x, x1 - back.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// 32 consecutive TMEM columns of this warp's lane quarter into registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

}  // namespace umma
}  // namespace bse
