// Mixed-precision W(q) . rho products on the 5th-generation tensor cores (step A4, BF16x3 form).
//
// X[m][n] = sum_g R[m][g] W[n][g] (complex) is taken as four real products on separate real and
// imaginary planes:
//   Re X = Re R . Re W^T - Im R . Im W^T,   Im X = Re R . Im W^T + Im R . Re W^T,
// the minus sign coming from the MMA instruction's negate-A bit, so no operand is stored twice.
// Every operand is split x = hi + lo in BF16 and each real product accumulates
// hi.hi + hi.lo + lo.hi in FP32 in tensor memory (relative error ~2^-16 per product).
//
// Operands are pre-split once per q chunk into the exact shared-memory images the MMA reads:
// 128-byte rows holding 32 complex K values as [Re(32 BF16) | Im(32 BF16)], 128B-swizzled
// K-major 8-row atoms.  A tiles are 128 rows of R, B tiles N rows of W (N <= 128, a multiple of
// 16 chosen so that ceil(NG/N) tiles cover the G range with little padding).
//
// tc_gemm_wr is persistent (one CTA per SM, static round-robin over the tiles of the chunk) and
// warp-specialised: warp 0 streams tile images with bulk copies into a 3-stage ring
// (transaction-counted mbarriers), warp 1 issues M128 x N x K16 MMAs (12 per 16 complex K), and
// warps 4-7 drain the accumulator.  Two accumulators (re | im, 256 TMEM columns each) alternate
// between tiles, so the epilogue of one tile overlaps the MMAs of the next.  Every mbarrier wait
// is bounded by a 2 s %globaltimer limit; on expiry the CTA records BSE_ERR_TIMEOUT, stops
// issuing, waits (bounded) for its own copies and MMAs in flight, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "layout.cuh"
#include "umma.cuh"

namespace bse {
namespace {

constexpr int kTcThreads = 256;
constexpr int TM = 128;                      // output rows per tile
constexpr int NMAX = 128;                    // complex output columns per tile, at most
constexpr int TKC = 32;                      // complex K per stage (one 128-byte row: 32 Re | 32 Im)
constexpr int kRow = 128;                    // bytes per tile row
constexpr int kTileA = TM * kRow;            // one split of an A tile (16 KB)
constexpr int kStages = 3;
constexpr int kStage = 2 * kTileA + 2 * NMAX * kRow;   // A hi, A lo, B hi, B lo (64 KB at N = 128)
constexpr int kAccCols = 256;                // one accumulator: Re in columns [0,128), Im in [128,256)
constexpr size_t kTcSmem = (size_t)kStages * kStage + 1024 + 256;   // ring, 1 KB alignment slack, barriers

using umma::gtimer;
using umma::idesc_of;
using umma::kNegA;
using umma::mbar_arrive;
using umma::mbar_init;
using umma::mbar_wait;
using umma::mma_bf16;
using umma::mma_commit;
using umma::smem_desc;
using umma::smem_u32;
using umma::swz;

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
struct SplitGeo {
  int q_begin, nq, mt_max, nt_max, kc_max, n_tile;
  long long vbase;
  int side_c;
};

__device__ __forceinline__ size_t a_tile_off(const SplitGeo& g, int qi, int mt, int c) {
  return (((size_t)qi * g.mt_max + mt) * g.kc_max + c) * (size_t)(2 * kTileA);
}
__device__ __forceinline__ size_t b_tile_off(const SplitGeo& g, int qi, int nt, int c) {
  return (((size_t)qi * g.nt_max + nt) * g.kc_max + c) * (size_t)(2 * g.n_tile * kRow);
}

// Row r of a tile image from 8 complex values v: chunk cq holds Re, chunk 4 + cq holds Im.
__device__ __forceinline__ void put_row8(unsigned char* hi, unsigned char* lo, int r, int cq, const float2 (&v)[8]) {
  float xr[8], xi[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    xr[i] = v[i].x;
    xi[i] = v[i].y;
  }
  uint4 hr, lr, hi2, li2;
  split8(xr, hr, lr);
  split8(xi, hi2, li2);
  *reinterpret_cast<uint4*>(hi + swz(r, cq)) = hr;
  *reinterpret_cast<uint4*>(lo + swz(r, cq)) = lr;
  *reinterpret_cast<uint4*>(hi + swz(r, 4 + cq)) = hi2;
  *reinterpret_cast<uint4*>(lo + swz(r, 4 + cq)) = li2;
}

__global__ __launch_bounds__(kTcThreads) void split_a_kernel(DevSys d, const float2* __restrict__ rho_dir,
                                                             unsigned char* __restrict__ As, SplitGeo g) {
  const int c = blockIdx.x, mt = blockIdx.y, qi = blockIdx.z;
  const int q = g.q_begin + qi;
  const long long nblk = d.qblk_off[q + 1] - d.qblk_off[q];
  const int w = side_width(d, g.side_c);
  const int M = (int)(nblk * w), NG = d.ngq[q];
  if (mt * TM >= M || c * TKC >= NG) return;
  const float2* A = rho_dir + (size_t)side_rows_offset(d, q, g.side_c, g.vbase) * d.ng_max;
  unsigned char* hi = As + a_tile_off(g, qi, mt, c);
  for (int it = threadIdx.x; it < TM * 4; it += kTcThreads) {
    const int r = it >> 2, cq = it & 3;
    const int row = mt * TM + r, g0 = c * TKC + 8 * cq;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      v[i] = (row < M && g0 + i < NG) ? A[(size_t)row * d.ng_max + g0 + i] : make_float2(0.f, 0.f);
    put_row8(hi, hi + kTileA, r, cq, v);
  }
}

__global__ __launch_bounds__(kTcThreads) void split_b_kernel(DevSys d, const float2* __restrict__ W,
                                                             unsigned char* __restrict__ Bs, SplitGeo g) {
  const int c = blockIdx.x, nt = blockIdx.y, qi = blockIdx.z;
  const int q = g.q_begin + qi;
  const int NG = d.ngq[q], N = g.n_tile;
  if (nt * N >= NG || c * TKC >= NG) return;
  const float2* Wq = W + (size_t)q * d.ng_max * d.ng_max;
  unsigned char* hi = Bs + b_tile_off(g, qi, nt, c);
  for (int it = threadIdx.x; it < N * 4; it += kTcThreads) {
    const int n = it >> 2, cq = it & 3;
    const int col = nt * N + n, g0 = c * TKC + 8 * cq;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      v[i] = (col < NG && g0 + i < NG) ? Wq[(size_t)col * d.ng_max + g0 + i] : make_float2(0.f, 0.f);
    put_row8(hi, hi + N * kRow, n, cq, v);
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

// Tile t of the chunk (N tiles fastest, then row tiles, then q); false if it holds no output.
struct Tile {
  int qi, q, mt, nt, M, NG, nch;
};
__device__ __forceinline__ bool tile_of(const DevSys& d, const SplitGeo& g, int w, long long t, Tile& o) {
  o.nt = (int)(t % g.nt_max);
  const long long r = t / g.nt_max;
  o.mt = (int)(r % g.mt_max);
  o.qi = (int)(r / g.mt_max);
  o.q = g.q_begin + o.qi;
  const long long nblk = d.qblk_off[o.q + 1] - d.qblk_off[o.q];
  o.M = (int)(nblk * w);
  o.NG = d.ngq[o.q];
  o.nch = (o.NG + TKC - 1) / TKC;
  return o.mt * TM < o.M && o.nt * g.n_tile < o.NG;
}

__device__ __forceinline__ void fail_now(volatile int* fail, int* status) {
  *fail = 1;
  atomicCAS(status, 0, (int)BSE_ERR_TIMEOUT);
}

__global__ __launch_bounds__(kTcThreads, 1) void tc_gemm_wr(DevSys d, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + kStages * kStage);   // [3] stage landed
  uint64_t* empty = full + kStages;                       // [3] MMAs done with the stage
  uint64_t* tfull = empty + kStages;                      // [2] accumulator complete
  uint64_t* tempty = tfull + 2;                           // [2] accumulator drained
  uint64_t* drain = tempty + 2;                           // all MMAs of this CTA complete
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* fail = (volatile int*)(tmem_slot + 1);
  volatile unsigned* issued = (volatile unsigned*)(tmem_slot + 2);
  volatile unsigned* consumed = (volatile unsigned*)(tmem_slot + 3);

  const SplitGeo& g = a.g;
  const int N = g.n_tile;
  const int w = side_width(d, g.side_c);
  const long long b0 = d.qblk_off[g.q_begin];
  const long long ntiles = (long long)g.nq * g.mt_max * g.nt_max;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kAccCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(smem_u32(full + i), 1);
      mbar_init(smem_u32(empty + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(tfull + i), 1);
      mbar_init(smem_u32(tempty + i), 4);
    }
    mbar_init(smem_u32(drain), 1);
    *fail = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {                 // producer
    const uint32_t bbytes = (uint32_t)(2 * N * kRow);
    unsigned c = 0;
    Tile t;
    for (long long ti = blockIdx.x; ti < ntiles && !*fail; ti += gridDim.x) {
      if (!tile_of(d, g, w, ti, t)) continue;
      for (int kc = 0; kc < t.nch; ++kc, ++c) {
        const int st = (int)(c % kStages);
        if (c >= kStages && !mbar_wait(smem_u32(empty + st), ((c / kStages) - 1) & 1u)) {
          fail_now(fail, a.status);
          break;
        }
        if (*fail) break;
        const uint32_t base = smem_u32(sm + st * kStage);
        mbar_expect_tx(smem_u32(full + st), (uint32_t)(2 * kTileA) + bbytes);
        bulk_g2s(base, a.As + a_tile_off(g, t.qi, t.mt, kc), 2 * kTileA, smem_u32(full + st));
        bulk_g2s(base + 2 * kTileA, a.Bs + b_tile_off(g, t.qi, t.nt, kc), bbytes, smem_u32(full + st));
        *issued = c + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {          // MMA issuer
    const uint32_t idesc = idesc_of(N), idesc_neg = idesc | kNegA;
    unsigned c = 0, j = 0;
    Tile t;
    bool ok = true;
    for (long long ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      if (!tile_of(d, g, w, ti, t)) continue;
      const int buf = (int)(j & 1);
      if (j >= 2 && !mbar_wait(smem_u32(tempty + buf), ((j >> 1) - 1) & 1u)) {
        fail_now(fail, a.status);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d_re = tmem + (uint32_t)(buf * kAccCols), d_im = d_re + 128;
      for (int kc = 0; kc < t.nch; ++kc, ++c) {
        const int st = (int)(c % kStages);
        if (!mbar_wait(smem_u32(full + st), (c / kStages) & 1u) || *fail) {
          fail_now(fail, a.status);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sah = smem_u32(sm + st * kStage), sal = sah + kTileA;
        const uint32_t sbh = sah + 2 * kTileA, sbl = sbh + (uint32_t)(N * kRow);
        const int nkk = (t.NG - kc * TKC > 16) ? 2 : 1;   // the last chunk may need one K16 step only
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          if (kk >= nkk) break;
#pragma unroll
          for (int s = 0; s < 3; ++s) {           // hi.hi, hi.lo, lo.hi
            const uint32_t pa = ((s == 2) ? sal : sah) + kk * 32, pb = ((s == 1) ? sbl : sbh) + kk * 32;
            const uint32_t acc = (kc | kk | s) != 0 ? 1u : 0u;
            mma_bf16(d_re, smem_desc(pa), smem_desc(pb), idesc, acc);                // Re R Re W
            mma_bf16(d_re, smem_desc(pa + 64), smem_desc(pb + 64), idesc_neg, 1u);   // - Im R Im W
            mma_bf16(d_im, smem_desc(pa), smem_desc(pb + 64), idesc, acc);           // Re R Im W
            mma_bf16(d_im, smem_desc(pa + 64), smem_desc(pb), idesc, 1u);            // Im R Re W
          }
        }
        mma_commit(smem_u32(empty + st));
        *consumed = c + 1;
      }
      if (!ok) break;
      mma_commit(smem_u32(tfull + buf));
      ++j;
    }
    mma_commit(smem_u32(drain));                // tracks every MMA issued above
    if (!mbar_wait(smem_u32(drain), 0u)) fail_now(fail, a.status);
  } else if (warp >= 4) {                       // epilogue: TMEM lanes 32(w-4).. -> output rows
    const int ew = warp - 4;
    const bool even = (d.ng_max & 1) == 0;
    unsigned j = 0;
    Tile t;
    for (long long ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
      if (!tile_of(d, g, w, ti, t)) continue;
      const int buf = (int)(j & 1);
      int ok = 1;
      if (lane == 0) {
        ok = mbar_wait(smem_u32(tfull + buf), (j >> 1) & 1u) ? 1 : 0;
        if (!ok) fail_now(fail, a.status);
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = t.mt * TM, n0 = t.nt * N;
      const int r = m0 + ew * 32 + lane;
      float2* out = a.X + (size_t)((d.qblk_off[t.q] - b0) * w + r) * d.ng_max;
      const int nvalid = min(N, t.NG - n0);
#pragma unroll 1
      for (int c0 = 0; c0 < N; c0 += 32) {
        uint32_t v[32], u[32];
        const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * kAccCols + c0);
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
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
              "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
              "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]),
              "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]),
              "=r"(u[30]), "=r"(u[31])
            : "r"(taddr + 128u)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int cnt = min(32, nvalid - c0);
        if (r < t.M && cnt > 0) {
          float2* o = out + n0 + c0;
          if (even) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if (2 * i + 1 < cnt)
                *reinterpret_cast<float4*>(o + 2 * i) = make_float4(__uint_as_float(v[2 * i]), __uint_as_float(u[2 * i]),
                                                                    __uint_as_float(v[2 * i + 1]),
                                                                    __uint_as_float(u[2 * i + 1]));
              else if (2 * i < cnt)
                o[2 * i] = make_float2(__uint_as_float(v[2 * i]), __uint_as_float(u[2 * i]));
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < cnt) o[i] = make_float2(__uint_as_float(v[i]), __uint_as_float(u[i]));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(tempty + buf));
      ++j;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0) {                               // copies still in flight after a failure
    for (unsigned c = *consumed; c < *issued; ++c)
      if (!mbar_wait(smem_u32(full + c % kStages), (c / kStages) & 1u)) break;
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccCols) : "memory");
  }
}

// N tile: ceil(ng_max / ceil(ng_max / 128)) rounded up to 16.
int tc_n_tile(const DevSys& d) {
  const int nt = (d.ng_max + NMAX - 1) / NMAX;
  const int n = (d.ng_max + nt - 1) / nt;
  return (n + 15) / 16 * 16;
}

}  // namespace

size_t tc_split_bytes(const DevSys& d, long long qchunk, long long w) {
  const int N = tc_n_tile(d);
  const long long mt = (d.nkpt * w + TM - 1) / TM, nt = (d.ng_max + N - 1) / N;
  const long long kc = (d.ng_max + TKC - 1) / TKC;
  return (size_t)qchunk * (size_t)kc * ((size_t)mt * 2 * kTileA + (size_t)nt * 2 * N * kRow);
}

// ws holds the split tiles; X is the FP32 output of the products.
int launch_gemm_wr_tc(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long vbase,
                      long long max_rows, const void* W, void* X, void* split_ws, int side_c, int* status,
                      void* stream) {
  static int attr_dev = -1, num_sms = 0;
  int dev = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return e;
  if (attr_dev != dev) {
    e = (int)cudaFuncSetAttribute((const void*)tc_gemm_wr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kTcSmem);
    if (e) return e;
    e = (int)cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    attr_dev = dev;
  }
  cudaStream_t st = (cudaStream_t)stream;
  SplitGeo g;
  g.q_begin = q_begin;
  g.nq = q_end - q_begin;
  g.vbase = vbase;
  g.side_c = side_c;
  g.n_tile = tc_n_tile(d);
  g.mt_max = (int)((max_rows + TM - 1) / TM);
  g.nt_max = (d.ng_max + g.n_tile - 1) / g.n_tile;
  g.kc_max = (d.ng_max + TKC - 1) / TKC;
  unsigned char* As = (unsigned char*)split_ws;
  unsigned char* Bs = As + (size_t)g.nq * g.mt_max * g.kc_max * 2 * kTileA;
  split_a_kernel<<<dim3(g.kc_max, g.mt_max, g.nq), kTcThreads, 0, st>>>(d, (const float2*)rho_dir, As, g);
  split_b_kernel<<<dim3(g.kc_max, g.nt_max, g.nq), kTcThreads, 0, st>>>(d, (const float2*)W, Bs, g);
  e = (int)cudaGetLastError();
  if (e) return e;
  TcArgs a{As, Bs, (float2*)X, g, status};
  const long long ntiles = (long long)g.nq * g.mt_max * g.nt_max;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  if (grid <= 0) return 0;
  tc_gemm_wr<<<grid, kTcThreads, kTcSmem, st>>>(d, a);
  return (int)cudaGetLastError();
}

}  // namespace bse
