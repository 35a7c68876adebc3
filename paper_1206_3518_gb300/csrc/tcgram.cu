// Exchange part of H on the 5th-generation tensor cores (step A3 of the mixed build; Eq. V_eh):
//
//   H[S][S'] = sum_G conj(Y[S][G]) Y[S'][G] + delta_SS' (e_c + Delta - e_v),   Y[S][G] = rho_x[S][G] s(G),
//
// s(G) = sqrt(2 vbar(G) / (Omega Nk)) (zero at G = 0 and beyond the q = 0 sphere), i.e. diag + 2 K^x, on
// the 128 x 128 tiles (I <= J) of the upper triangle and the tiles (I, I - 1) just below it, which hold
// every upper block (k <= k'), also those straddling a tile boundary.
//
// Y is split x = hi + lo in BF16 once (gram_split_kernel) into the images the MMA reads: per row tile
// and chunk of 32 G, 128 rows of [Re 32 | Im 32] hi, then lo, 128B-swizzled K-major.  gram_kernel is
// persistent (one CTA per SM, static round-robin over the tiles): warp 0 brings the A (row tile I) and
// B (row tile J) images of each chunk with two bulk copies into a 3-stage ring, warp 1 issues the 12
// MMAs per 16 complex G of conj(A) B (hi.hi + hi.lo + lo.hi, FP32 accumulation in tensor memory), warps
// 4-7 drain the two alternating accumulators into H.  Every mbarrier wait is bounded (2 s); on expiry
// the CTA records BSE_ERR_TIMEOUT, stops issuing, waits (bounded) for its copies and MMAs in flight,
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "umma.cuh"

namespace bse {
namespace {

using umma::mbar_arrive;
using umma::mbar_init;
using umma::mbar_wait;
using umma::mma_commit;
using umma::smem_u32;
using umma::swz;

constexpr int kThreads = 256;
constexpr int kTM = 128;                       // rows (and columns) per tile
constexpr int kTKC = 32;                       // complex G per chunk
constexpr int kTile = kTM * umma::kRow;        // one split of a tile image (16 KB)
constexpr int kImg = 2 * kTile;                // hi then lo
constexpr int kStages = 3;
constexpr int kStage = 2 * kImg;               // A image, B image
constexpr int kAcc = 256;                      // Re in columns [0,128), Im in [128,256)
constexpr size_t kSmem = (size_t)kStages * kStage + 1024 + 256;

struct GramGeo {
  int ntr, nkc;                                 // row tiles, G chunks
  long long nupper;                             // upper tiles (I <= J)
  long long ntiles;                             // then the tiles (I, I - 1) below the diagonal
};

GramGeo geo_of(const DevSys& d) {
  GramGeo g;
  g.ntr = (d.dim + kTM - 1) / kTM;
  g.nkc = (d.ng0 + kTKC - 1) / kTKC;
  g.nupper = (long long)g.ntr * (g.ntr + 1) / 2;
  g.ntiles = g.nupper + g.ntr - 1;
  return g;
}

__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 back = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - back.x, x1 - back.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// images[tile][chunk]: rows S of the tile, 16-byte chunk cq of the row = 8 G values of Re (cq < 4) or Im.
__global__ __launch_bounds__(kThreads) void gram_split_kernel(DevSys d, const float2* __restrict__ rho_x,
                                                              unsigned char* __restrict__ img, int nkc) {
  const int c = blockIdx.x, tr = blockIdx.y;
  unsigned char* hi = img + ((size_t)tr * nkc + c) * kImg;
  unsigned char* lo = hi + kTile;
  for (int it = threadIdx.x; it < kTM * 4; it += kThreads) {
    const int r = it >> 2, cq = it & 3;
    const int S = tr * kTM + r, g0 = c * kTKC + 8 * cq;
    float xr[8], xi[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int G = g0 + i;
      float2 v = make_float2(0.f, 0.f);
      if (S < d.dim && G < d.ng0) {
        const float2 y = rho_x[(size_t)S * d.ng_max + G];
        const float sc = d.xscale[G];
        v = make_float2(y.x * sc, y.y * sc);
      }
      xr[i] = v.x;
      xi[i] = v.y;
    }
    uint4 rh, rl, ih, il;
    split_pair(xr[0], xr[1], rh.x, rl.x);
    split_pair(xr[2], xr[3], rh.y, rl.y);
    split_pair(xr[4], xr[5], rh.z, rl.z);
    split_pair(xr[6], xr[7], rh.w, rl.w);
    split_pair(xi[0], xi[1], ih.x, il.x);
    split_pair(xi[2], xi[3], ih.y, il.y);
    split_pair(xi[4], xi[5], ih.z, il.z);
    split_pair(xi[6], xi[7], ih.w, il.w);
    *reinterpret_cast<uint4*>(hi + swz(r, cq)) = rh;
    *reinterpret_cast<uint4*>(lo + swz(r, cq)) = rl;
    *reinterpret_cast<uint4*>(hi + swz(r, 4 + cq)) = ih;
    *reinterpret_cast<uint4*>(lo + swz(r, 4 + cq)) = il;
  }
}

// Tile t: the upper tiles row by row over I <= J, then (I, I - 1) for I = 1 .. n - 1 (a block of Nv Nc rows that
// straddles the row 128 I has upper entries there).
__device__ __forceinline__ long long row_start(int I, int n) { return (long long)I * n - (long long)I * (I - 1) / 2; }
__device__ __forceinline__ void tile_ij(long long t, int n, int& I, int& J) {
  const long long nup = (long long)n * (n + 1) / 2;
  if (t >= nup) {
    I = (int)(t - nup) + 1;
    J = I - 1;
    return;
  }
  const double b = 2.0 * n + 1.0;
  int i = (int)floor(0.5 * (b - sqrt(fmax(b * b - 8.0 * (double)t, 0.0))));
  i = i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
  while (i > 0 && row_start(i, n) > t) --i;
  while (i + 1 < n && row_start(i + 1, n) <= t) ++i;
  I = i;
  J = i + (int)(t - row_start(i, n));
}

__device__ __forceinline__ void fail_now(volatile int* fail, int* status) {
  *fail = 1;
  atomicCAS(status, 0, (int)BSE_ERR_TIMEOUT);
}

__global__ __launch_bounds__(kThreads, 1) void gram_kernel(DevSys d, const unsigned char* __restrict__ img,
                                                           const double* __restrict__ e, double delta,
                                                           float2* __restrict__ H, GramGeo g, int* status) {
  extern __shared__ __align__(1024) unsigned char gm_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)gm_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + kStages * kStage);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* fail = (volatile int*)(tmem_slot + 1);
  volatile unsigned* issued = (volatile unsigned*)(tmem_slot + 2);
  volatile unsigned* consumed = (volatile unsigned*)(tmem_slot + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kAcc)
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
    unsigned c = 0;
    for (long long t = blockIdx.x; t < g.ntiles && !*fail; t += gridDim.x) {
      int I, J;
      tile_ij(t, g.ntr, I, J);
      for (int kc = 0; kc < g.nkc; ++kc, ++c) {
        const int st = (int)(c % kStages);
        if (c >= kStages && !mbar_wait(smem_u32(empty + st), ((c / kStages) - 1) & 1u)) {
          fail_now(fail, status);
          break;
        }
        if (*fail) break;
        const uint32_t base = smem_u32(sm + st * kStage);
        umma::mbar_arrive_expect_tx(smem_u32(full + st), (uint32_t)(2 * kImg));
        umma::bulk_g2s(base, img + ((size_t)I * g.nkc + kc) * kImg, kImg, smem_u32(full + st));
        umma::bulk_g2s(base + kImg, img + ((size_t)J * g.nkc + kc) * kImg, kImg, smem_u32(full + st));
        *issued = c + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {          // MMA issuer
    const uint32_t idesc = umma::idesc_of(kTM);
    const uint64_t d0 = umma::smem_desc(smem_u32(sm));
    const uint32_t lo = (uint32_t)(kTile >> 4);
    unsigned c = 0, j = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < g.ntiles && ok; t += gridDim.x, ++j) {
      const int buf = (int)(j & 1);
      if (j >= 2 && !mbar_wait(smem_u32(tempty + buf), ((j >> 1) - 1) & 1u)) {
        fail_now(fail, status);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d_re = tmem + (uint32_t)(buf * kAcc), d_im = d_re + 128;
      for (int kc = 0; kc < g.nkc; ++kc, ++c) {
        const int st = (int)(c % kStages);
        if (!mbar_wait(smem_u32(full + st), (c / kStages) & 1u) || *fail) {
          fail_now(fail, status);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t da = d0 + (uint64_t)((st * kStage) >> 4), db = da + (uint64_t)(kImg >> 4);
        const int nkk = (d.ng0 - kc * kTKC > 16) ? 2 : 1;
        for (int kk = 0; kk < nkk; ++kk)
          umma::mma_cplx_conj_k16_desc(d_re, d_im, da, lo, db, lo, kk, idesc, kc == 0 && kk == 0);
        mma_commit(smem_u32(empty + st));
        *consumed = c + 1;
      }
      if (!ok) break;
      mma_commit(smem_u32(tfull + buf));
    }
    mma_commit(smem_u32(drain));                // tracks every MMA issued above
    if (!mbar_wait(smem_u32(drain), 0u)) fail_now(fail, status);
  } else if (warp >= 4) {                       // epilogue: TMEM lanes 32 (w - 4) .. -> rows of H
    const int ew = warp - 4;
    const int nvc = d.nv * d.nc;
    unsigned j = 0;
    for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x, ++j) {
      int I, J;
      tile_ij(t, g.ntr, I, J);
      const int buf = (int)(j & 1);
      int ok = 1;
      if (lane == 0) {
        ok = mbar_wait(smem_u32(tfull + buf), (j >> 1) & 1u) ? 1 : 0;
        if (!ok) fail_now(fail, status);
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int S = I * kTM + ew * 32 + lane;
      float diag = 0.f;
      if (S < d.dim) {
        const int ic = S % d.nc, iv = (S / d.nc) % d.nv, k = S / nvc;
        diag = (float)(e[(size_t)k * d.nb + d.nv + ic] + delta - e[(size_t)k * d.nb + iv]);
      }
      float2* out = H + (size_t)S * d.dim + (size_t)J * kTM;
#pragma unroll 1
      for (int c0 = 0; c0 < kTM; c0 += 32) {
        uint32_t v[32], u[32];
        const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * kAcc + c0);
        umma::tmem_ld32(taddr, v);
        umma::tmem_ld32(taddr + 128u, u);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (S < d.dim) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int S2 = J * kTM + c0 + i;
            if (S2 < d.dim) {
              float2 val = make_float2(__uint_as_float(v[i]), __uint_as_float(u[i]));
              if (S2 == S) val.x += diag;
              out[c0 + i] = val;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(tempty + buf));
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAcc) : "memory");
  }
}

}  // namespace

size_t gram_ws_bytes(const DevSys& d) {
  const GramGeo g = geo_of(d);
  return (size_t)g.ntr * g.nkc * kImg;
}

// diag + 2 K^x on the upper tiles of H with BF16x3 tensor-core products; ws holds the split images.
int launch_kernel_init_tc(const DevSys& d, const void* rho_x, const double* energies, double delta, void* H,
                          void* ws, int* status, void* stream) {
  static int attr_dev = -1, num_sms = 0;
  int dev = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return e;
  if (attr_dev != dev) {
    e = (int)cudaFuncSetAttribute((const void*)gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e) return e;
    e = (int)cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    attr_dev = dev;
  }
  const GramGeo g = geo_of(d);
  if (g.nkc < 1) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* img = (unsigned char*)ws;
  gram_split_kernel<<<dim3(g.nkc, g.ntr), kThreads, 0, st>>>(d, (const float2*)rho_x, img, g.nkc);
  if ((e = (int)cudaGetLastError())) return e;
  const int grid = (int)(g.ntiles < num_sms ? g.ntiles : num_sms);
  gram_kernel<<<grid, kThreads, kSmem, st>>>(d, img, energies, delta, (float2*)H, g, status);
  return (int)cudaGetLastError();
}

}  // namespace bse
