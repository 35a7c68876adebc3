// Mixed-precision W(q) . rho products on the 5th-generation tensor cores (step A4, BF16x3 form).
//
// The complex product X[m][n] = sum_g R[m][g] W[n][g] is a real GEMM
//   C'[m][2n + c] = sum_k A'[m][k] B'[2n + c][k],   k = 2g + {0, 1},
// with A' = R read as floats (re, im, re, im, ...), B'[2n] = (Re W, -Im W, ...) and
// B'[2n+1] = (Im W, Re W, ...), so each accumulator row is the complex64 output row.
// Every operand is split x = hi + lo in BF16 and C' = A_hi B_hi + A_hi B_lo + A_lo B_hi
// accumulates in FP32 in tensor memory (relative error ~2^-16 per product).
//
// One CTA: 128 output rows x 128 complex columns (accumulator 128 lanes x 256 FP32 columns),
// K in chunks of 64 real values.  All 256 threads convert the next chunk into a 128B-swizzled,
// K-major shared tile (canonical UMMA layout, 8-row atoms of 1 KB) while the tensor core
// consumes the previous one; one thread issues tcgen05.mma (M128 N256 K16, 3 splits x 4 steps
// per chunk) and tcgen05.commit to the chunk's mbarrier.  Every mbarrier wait is bounded by a
// 2 s %globaltimer limit; on expiry the CTA records BSE_ERR_TIMEOUT, waits once more (bounded)
// for its own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace bse {
namespace {

constexpr int kTcThreads = 256;
constexpr int TM = 128;            // output rows per CTA
constexpr int TN = 256;            // real accumulator columns per CTA (128 complex)
constexpr int TK = 64;             // real K per chunk (128 bytes of BF16 per row)
constexpr int kTileA = TM * TK * 2;          // bytes of one A split tile (16 KB)
constexpr int kTileB = TN * TK * 2;          // bytes of one B split tile (32 KB)
constexpr int kStage = 2 * kTileA + 2 * kTileB;   // A_hi, A_lo, B_hi, B_lo (96 KB)
constexpr size_t kTcSmem = 2 * kStage + 1024 + 128;  // two stages, 1 KB alignment slack, barriers

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait on an mbarrier phase; false after 2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (gtimer() - t0 > 2000000000ull) return false;
  }
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

// Instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16-byte chunk c of row r of a swizzled K-major tile (rows of 128 bytes).
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const float2 back = __bfloat1622float2(hh);
    h[i] = hh;
    l[i] = __floats2bfloat162_rn(x[2 * i] - back.x, x[2 * i + 1] - back.y);
  }
  hi = *reinterpret_cast<uint4*>(h);
  lo = *reinterpret_cast<uint4*>(l);
}

// ---------------------------------------------------------------- operand split (one pass per q chunk)
// Tile images are exactly the shared-memory images the MMA reads: A tiles 128 rows x 64 BF16 (hi 16 KB
// then lo 16 KB), B tiles 256 rows x 64 BF16 (hi 32 KB then lo 32 KB), addressed by (q, row tile, k chunk).
struct SplitGeo {
  int q_begin, mt_max, nt_max, kc_max;
  long long vbase;
  int side_c;
};

__device__ __forceinline__ size_t a_tile_off(const SplitGeo& g, int qi, int mt, int c) {
  return (((size_t)qi * g.mt_max + mt) * g.kc_max + c) * (size_t)(2 * kTileA);
}
__device__ __forceinline__ size_t b_tile_off(const SplitGeo& g, int qi, int nt, int c) {
  return (((size_t)qi * g.nt_max + nt) * g.kc_max + c) * (size_t)(2 * kTileB);
}

__global__ __launch_bounds__(kTcThreads) void split_a_kernel(DevSys d, const float2* __restrict__ rho_dir,
                                                             unsigned char* __restrict__ As, SplitGeo g) {
  const int c = blockIdx.x, mt = blockIdx.y, qi = blockIdx.z;
  const int q = g.q_begin + qi;
  const long long nblk = d.qblk_off[q + 1] - d.qblk_off[q];
  const int w = g.side_c ? d.nc * d.nc : d.nv * d.nv;
  const int M = (int)(nblk * w), NG = d.ngq[q], Kr = 2 * NG;
  if (mt * TM >= M || c * TK >= Kr) return;
  long long aoff = d.qvec_off[q] - g.vbase;
  if (g.side_c) aoff += nblk * d.nv * d.nv;
  const float* A = reinterpret_cast<const float*>(rho_dir + (size_t)aoff * d.ng_max);
  unsigned char* dst = As + a_tile_off(g, qi, mt, c);
  for (int it = threadIdx.x; it < TM * 8; it += kTcThreads) {
    const int r = it >> 3, ch = it & 7;
    const int row = mt * TM + r, kk = c * TK + 8 * ch;
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (row < M && kk + i < Kr) ? A[(size_t)row * (2 * d.ng_max) + kk + i] : 0.f;
    uint4 hi, lo;
    split8(x, hi, lo);
    *reinterpret_cast<uint4*>(dst + swz(r, ch)) = hi;
    *reinterpret_cast<uint4*>(dst + kTileA + swz(r, ch)) = lo;
  }
}

__global__ __launch_bounds__(kTcThreads) void split_b_kernel(DevSys d, const float2* __restrict__ W,
                                                             unsigned char* __restrict__ Bs, SplitGeo g) {
  const int c = blockIdx.x, nt = blockIdx.y, qi = blockIdx.z;
  const int q = g.q_begin + qi;
  const int NG = d.ngq[q];
  if (nt * (TN / 2) >= NG || c * TK >= 2 * NG) return;
  const float2* Wq = W + (size_t)q * d.ng_max * d.ng_max;
  unsigned char* bh = Bs + b_tile_off(g, qi, nt, c);
  unsigned char* bl = bh + kTileB;
  for (int it = threadIdx.x; it < (TN / 2) * 8; it += kTcThreads) {
    const int n = it >> 3, ch = it & 7;
    const int col = nt * (TN / 2) + n;
    const int g0 = (c * TK >> 1) + 4 * ch;
    float xr[8], xi[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 v = make_float2(0.f, 0.f);
      if (col < NG && g0 + i < NG) v = Wq[(size_t)col * d.ng_max + g0 + i];
      xr[2 * i] = v.x;
      xr[2 * i + 1] = -v.y;
      xi[2 * i] = v.y;
      xi[2 * i + 1] = v.x;
    }
    uint4 hr, lr, hi2, li2;
    split8(xr, hr, lr);
    split8(xi, hi2, li2);
    *reinterpret_cast<uint4*>(bh + swz(2 * n, ch)) = hr;
    *reinterpret_cast<uint4*>(bl + swz(2 * n, ch)) = lr;
    *reinterpret_cast<uint4*>(bh + swz(2 * n + 1, ch)) = hi2;
    *reinterpret_cast<uint4*>(bl + swz(2 * n + 1, ch)) = li2;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

struct TcArgs {
  const unsigned char* As;
  const unsigned char* Bs;
  float2* X;
  SplitGeo g;
  int* status;
};

// Warp-specialised GEMM on the split tiles: warp 0 streams tiles (bulk copies, transaction-counted
// mbarriers), warp 1 issues the MMAs, warps 4..7 drain the accumulator.  Two stages of 96 KB.
__global__ __launch_bounds__(kTcThreads, 1) void tc_gemm_wr(DevSys d, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + 2 * kStage);        // [2] tiles landed
  uint64_t* empty = full + 2;                           // [2] MMAs done with the stage
  uint64_t* accum = full + 4;                           // accumulator complete
  uint32_t* tmem_slot = (uint32_t*)(sm + 2 * kStage + 48);
  volatile int* fail = (volatile int*)(sm + 2 * kStage + 56);

  const SplitGeo& g = a.g;
  const int qi = blockIdx.z, q = g.q_begin + qi;
  const long long b0 = d.qblk_off[g.q_begin];
  const long long nblk = d.qblk_off[q + 1] - d.qblk_off[q];
  const int w = g.side_c ? d.nc * d.nc : d.nv * d.nv;
  const int M = (int)(nblk * w), NG = d.ngq[q];
  const int mt = blockIdx.y, nt = blockIdx.x;
  const int m0 = mt * TM, n0 = nt * (TN / 2);
  if (m0 >= M || n0 >= NG) return;
  const int nch = (2 * NG + TK - 1) / TK;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < 5; ++i) mbar_init(smem_u32(full + i), 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {                 // producer
    for (int c = 0; c < nch; ++c) {
      const int st = c & 1;
      if (c >= 2 && !mbar_wait(smem_u32(empty + st), (uint32_t)(((c - 2) >> 1) & 1))) {
        *fail = 1;
        break;
      }
      if (*fail) break;
      const uint32_t base = smem_u32(sm + st * kStage);
      mbar_expect_tx(smem_u32(full + st), (uint32_t)kStage);
      bulk_g2s(base, a.As + a_tile_off(g, qi, mt, c), 2 * kTileA, smem_u32(full + st));
      bulk_g2s(base + 2 * kTileA, a.Bs + b_tile_off(g, qi, nt, c), 2 * kTileB, smem_u32(full + st));
    }
  } else if (warp == 1 && lane == 0) {          // MMA issuer
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
      const int st = c & 1;
      if (!mbar_wait(smem_u32(full + st), (uint32_t)((c >> 1) & 1))) {
        *fail = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(sm + st * kStage);
      const uint32_t sah = sa, sal = sa + kTileA, sbh = sa + 2 * kTileA, sbl = sbh + kTileB;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const uint32_t pa = (s == 2) ? sal : sah;
        const uint32_t pb = (s == 1) ? sbl : sbh;
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk)
          mma_bf16(tmem, smem_desc(pa + kk * 32), smem_desc(pb + kk * 32), (c | s | kk) != 0 ? 1u : 0u);
      }
      mma_commit(smem_u32(empty + st));
    }
    if (ok) mma_commit(smem_u32(accum));
  } else if (warp >= 4) {                       // epilogue: TMEM lanes 32(w-4).. -> output rows
    const int ew = warp - 4;
    bool ok = mbar_wait(smem_u32(accum), 0u);
    if (!ok) {
      if (lane == 0) atomicCAS(a.status, 0, (int)BSE_ERR_TIMEOUT);
      *fail = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int r = m0 + ew * 32 + lane;
      float2* out = a.X + (size_t)((d.qblk_off[q] - b0) * w + r) * d.ng_max;
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (r < M) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int n = n0 + c0 / 2 + i;
            if (n < NG) out[n] = make_float2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

}  // namespace

size_t tc_split_bytes(const DevSys& d, long long qchunk) {
  const long long w = (d.nv * d.nv <= d.nc * d.nc) ? d.nv * d.nv : d.nc * d.nc;
  const long long mt = (d.nkpt * w + TM - 1) / TM, nt = (d.ng_max + TN / 2 - 1) / (TN / 2);
  const long long kc = (2 * d.ng_max + TK - 1) / TK;
  return (size_t)qchunk * (size_t)kc * ((size_t)mt * 2 * kTileA + (size_t)nt * 2 * kTileB);
}

// ws holds the split tiles; X is the FP32 output of the products.
int launch_gemm_wr_tc(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long vbase,
                      long long max_rows, const void* W, void* X, void* split_ws, int side_c, int* status,
                      void* stream) {
  static bool attr = false;
  if (!attr) {
    const int e = (int)cudaFuncSetAttribute((const void*)tc_gemm_wr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kTcSmem);
    if (e) return e;
    attr = true;
  }
  cudaStream_t st = (cudaStream_t)stream;
  SplitGeo g;
  g.q_begin = q_begin;
  g.vbase = vbase;
  g.side_c = side_c;
  g.mt_max = (int)((max_rows + TM - 1) / TM);
  g.nt_max = (d.ng_max + TN / 2 - 1) / (TN / 2);
  g.kc_max = (2 * d.ng_max + TK - 1) / TK;
  const int nq = q_end - q_begin;
  unsigned char* As = (unsigned char*)split_ws;
  unsigned char* Bs = As + (size_t)nq * g.mt_max * g.kc_max * 2 * kTileA;
  split_a_kernel<<<dim3(g.kc_max, g.mt_max, nq), kTcThreads, 0, st>>>(d, (const float2*)rho_dir, As, g);
  split_b_kernel<<<dim3(g.kc_max, g.nt_max, nq), kTcThreads, 0, st>>>(d, (const float2*)W, Bs, g);
  int e = (int)cudaGetLastError();
  if (e) return e;
  TcArgs a{As, Bs, (float2*)X, g, status};
  tc_gemm_wr<<<dim3(g.nt_max, g.mt_max, nq), kTcThreads, kTcSmem, st>>>(d, a);
  return (int)cudaGetLastError();
}

}  // namespace bse
