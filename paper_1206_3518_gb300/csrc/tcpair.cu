// Direct pair densities on the 5th-generation tensor cores (step A2 of the mixed build; Eq. pair_density
// in the plane-wave basis):
//
//   rho_nm^{kk'}(G) = sum_{G2 in S(k')} conj(c_nk(G2 - G)) c_mk'(G2),   G = g_p(q) - G0.
//
// For a fixed k the factor conj(c_nk(G2 - G)), a function of (G, G2), is the same for every block
// (k, k').  The blocks of one k whose k' lie in one region of the k' mesh (the plan's regions: a few
// neighbouring mesh points) therefore form one GEMM per band n of the set (vv' or cc'):
//
//   D[G][(k', m)] = sum_{G2 in K} A_n[G][G2] B[(k', m)][G2],
//
//   rows G     the union over the tile's blocks of the G sphere of their q (shifted by G0): the first
//              block's sphere in its sphere order, then the other points in lexicographic order;
//   K          the region's layout, the union of the spheres S(k') of its points;
//   columns    the tile's blocks times the bands m of the set.
//
// A_n is gathered into shared memory from a dense index box of S(k) (points outside S(k) read a zero
// row); B comes from packed panels of the coefficients of each region's points in its K layout (zero off
// S(k')), written once per call.  The epilogue keeps, for every block, the rows on its own sphere and writes
// them at their sphere positions, so the output is the direct set of the correlation kernels.
//
// Arithmetic (BF16x3): every operand is split x = hi + lo in BF16 and each real product accumulates
// hi.hi + hi.lo + lo.hi in FP32 in tensor memory (relative error ~2^-16 per product, as for the
// W.rho products of the mixed build).  The G = 0 overlaps of the diagonal blocks (k' = k), which
// meet the q = 0 head of W, are summed again in FP64 afterwards (tcpair_diag_kernel).
//
// tcpair_kernel is persistent (one CTA per SM) and takes tiles (k, region) from a counter, region-major.
// Warps 0-3 drain the accumulators, warp 4 issues the MMAs (12 per 16 complex K, A from tensor memory,
// B from shared memory), warps 5-12 gather the A tile of each K chunk (32 complex K values) straight into
// tensor memory (two A slots, tcgen05.st; warps 5-8 the even stages, 9-12 the odd ones), and warp 13
// brings the B rows into a ring of shared-memory stages with bulk copies (the region's panel of the chunk:
// its hi rows and its lo rows, counted on the stage's mbarrier); the columns of a region's points without
// a block in the tile are computed and dropped.
// Two accumulators (Re | Im, 2 N <= 192 TMEM columns each) alternate between passes (one band n, 128
// rows), so the epilogue of one pass overlaps the MMAs of the next.  Every mbarrier wait is bounded (2 s); on expiry the CTA
// records BSE_ERR_TIMEOUT, stops issuing, waits (bounded) for its MMAs in flight, frees its tensor
// memory and returns.
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

constexpr int kEpiWarps = 4;                   // warps 0-3: TMEM lane quarters 0-3
constexpr int kMmaWarp = 4;
constexpr int kG0 = 5;                         // first gather warp
constexpr int kGWarps = 8;
constexpr int kB0 = kG0 + kGWarps;             // the B producer warp (bulk copies)
constexpr int kMaxStages = 6;                  // B ring depth at most
constexpr int kAStages = 2;                    // A tiles in tensor memory
constexpr int kThreads = (kB0 + 1) * 32;
constexpr int kGThreads = kGWarps * 32;
constexpr int kTKC = 32;                       // complex K values per stage
constexpr int kACols = 64;                     // one A tile in TMEM: two K16 halves x (Re hi, Im hi, Re lo, Im lo) x 8
constexpr int kImgRow = 256;                   // packed image of 32 K values: hi row (128 B), lo row (128 B)
size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct TpGeo {
  int q_begin, nqc;
  long long vbase;
  int nkc;                                      // K chunks of the packed images (tc_kpad / 32)
  int stages, nmax;                             // ring depth; B rows per stage (max columns, multiple of 16)
  int stage_bytes;
  int bx, by, bz, bbox_n, bbox_c;               // difference box of S(k): dims, entries, key of G1 = 0
  int rowbox, nwords;
  int o_bar, o_bbox, o_kcoef, o_kkey, o_rows, o_bits, o_slot, o_cols, o_binfo, o_bvec, o_ptab;
  size_t smem;                                  // dynamic shared memory incl. 1 KB alignment slack
};

TpGeo tp_geo(const DevSys& d, int stages) {
  TpGeo g{};
  g.stages = stages;
  g.nkc = d.tc_kpad / kTKC;
  const int mb = d.nv > d.nc ? d.nv : d.nc;
  g.nmax = (d.tc_rsize * mb + 15) / 16 * 16;
  g.stage_bytes = 2 * g.nmax * umma::kRow;      // B hi rows, B lo rows
  const int rx = d.fwf[0] + d.fpair[0], ry = d.fwf[1] + d.fpair[1], rz = d.fwf[2] + d.fpair[2];
  g.bx = 2 * rx + 1;
  g.by = 2 * ry + 1;
  g.bz = 2 * rz + 1;
  g.bbox_n = g.bx * g.by * g.bz;
  g.bbox_c = (rx * g.by + ry) * g.bz + rz;
  g.rowbox = (2 * d.fpair[0] + 1) * (2 * d.fpair[1] + 1) * (2 * d.fpair[2] + 1);
  g.nwords = (g.rowbox + 31) / 32;
  size_t o = (size_t)stages * g.stage_bytes;
  g.o_bar = (int)o; o += align16((size_t)(2 * stages + 2 * kAStages + 5) * 8 + 8 * sizeof(int));
  g.o_bbox = (int)o; o += align16((size_t)g.bbox_n * 2);
  g.o_kcoef = (int)o; o += align16((size_t)(d.npw_max + 1) * 8);
  g.o_kkey = (int)o; o += align16((size_t)d.tc_kpad * 4);
  g.o_rows = (int)o; o += align16((size_t)g.rowbox * 4);
  g.o_bits = (int)o; o += align16((size_t)g.nwords * 4);
  g.o_slot = (int)o; o += align16((size_t)d.tc_rsize * 4);
  g.o_cols = (int)o; o += align16((size_t)d.tc_rsize * 4);
  g.o_binfo = (int)o; o += align16((size_t)d.tc_rsize * 16);
  g.o_bvec = (int)o; o += align16((size_t)d.tc_rsize * 16);
  g.o_ptab = (int)o; o += align16((size_t)128 * d.tc_rsize * 2);
  g.smem = o + 1024;
  return g;
}

__device__ __forceinline__ void fail_now(volatile int* fail, int* status) {
  *fail = 1;
  atomicCAS(status, 0, (int)BSE_ERR_TIMEOUT);
}

__device__ __forceinline__ void gather_bar() { asm volatile("barrier.sync 1, %0;" ::"n"(kGThreads) : "memory"); }

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  return (uint32_t)*reinterpret_cast<const unsigned short*>(&h);
}

// x = hi + lo in BF16 as (hi | lo << 16)
__device__ __forceinline__ uint32_t split_word(float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(h);
  return (uint32_t)*reinterpret_cast<const unsigned short*>(&h) | (bf16_bits(r) << 16);
}

// ---------------------------------------------------------------- packed coefficient panels
// Packed B panels: for each region r, set (valence bands, then conduction bands) and K chunk c, the rows
// j = slot nset + m of every k' of the region (slot: its position in the region, m: its band in the set),
// [Re 32 | Im 32] BF16 in the region's K layout (zero off S(k')), hi rows then lo rows, the 16-byte chunks of
// row j permuted by j mod 8 (128B swizzle): a stage's B tile is two bulk copies.
__device__ __forceinline__ size_t panel_off(const DevSys& d, int r, int set, int c, int nkc) {
  const size_t per_r = (size_t)nkc * 2 * umma::kRow * d.tc_rsize * (d.nv + d.nc);
  const size_t set_off = set ? (size_t)nkc * 2 * umma::kRow * d.tc_rsize * d.nv : 0;
  const int nset = set ? d.nc : d.nv;
  return (size_t)r * per_r + set_off + (size_t)c * 2 * umma::kRow * d.tc_rsize * nset;
}

__device__ __forceinline__ void region_of(const DevSys& d, int k2, int& r, int& slot) {
  const int o0 = k2 / (d.nk2 * d.nk3), o1 = (k2 / d.nk3) % d.nk2, o2 = k2 % d.nk3;
  r = ((o0 / d.tc_rg[0]) * d.tc_nr[1] + o1 / d.tc_rg[1]) * d.tc_nr[2] + o2 / d.tc_rg[2];
  slot = ((o0 % d.tc_rg[0]) * d.tc_rg[1] + o1 % d.tc_rg[1]) * d.tc_rg[2] + o2 % d.tc_rg[2];
}

__global__ void tcpair_pack_kernel(DevSys d, const float2* __restrict__ coef, unsigned char* __restrict__ bimg,
                                   int nkc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)d.nkpt * d.nb * d.npw_max;
  if (t >= total) return;
  const int i = (int)(t % d.npw_max);
  const long long kb = t / d.npw_max;           // k' * nb + band
  const int k2 = (int)(kb / d.nb), band = (int)(kb - (long long)k2 * d.nb);
  if (i >= d.npw[k2]) return;
  const int set = band < d.nv ? 0 : 1, m = set ? band - d.nv : band, nset = set ? d.nc : d.nv;
  int r, slot;
  region_of(d, k2, r, slot);
  const int l = d.tc_kpos[(size_t)k2 * d.npw_max + i];
  const float2 c = coef[t];
  const uint32_t re = split_word(c.x), im = split_word(c.y);
  const int e = l % kTKC, j = slot * nset + m, ph = j & 7;
  unsigned short* hi = reinterpret_cast<unsigned short*>(bimg + panel_off(d, r, set, l / kTKC, nkc)) + j * 64;
  unsigned short* lo = hi + d.tc_rsize * nset * 64;
  const int cr = ((e >> 3) ^ ph) * 8 + (e & 7), ci = ((4 + (e >> 3)) ^ ph) * 8 + (e & 7);
  hi[cr] = (unsigned short)(re & 0xFFFFu);
  hi[ci] = (unsigned short)(im & 0xFFFFu);
  lo[cr] = (unsigned short)(re >> 16);
  lo[ci] = (unsigned short)(im >> 16);
}

// ---------------------------------------------------------------- tile table of a q range
// blist[(k nreg + r) rsize + slot] = block (k, k') of the range with k' in region r at its slot, else -1.
__global__ void tcpair_tiles_kernel(DevSys d, int q_begin, int nqc, int* __restrict__ blist) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nqc * d.nkpt) return;
  const int q = q_begin + (int)(t / d.nkpt), k = (int)(t % d.nkpt);
  const int b = d.blkidx[(size_t)q * d.nkpt + k];
  if (b < 0) return;
  int r, s;
  region_of(d, d.blocks[b].y, r, s);
  blist[((size_t)k * d.tc_nreg + r) * d.tc_rsize + s] = b;
}

// ---------------------------------------------------------------- the GEMM tiles
__global__ __launch_bounds__(kThreads, 1) void tcpair_kernel(DevSys d, const float2* __restrict__ coef,
                                                             const unsigned char* __restrict__ bimg,
                                                             const int* __restrict__ blist, int* __restrict__ counter,
                                                             float2* __restrict__ out, TpGeo g, int* status) {
  extern __shared__ __align__(1024) unsigned char tp_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tp_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full_b = (uint64_t*)(sm + g.o_bar);   // [stages] B rows landed
  uint64_t* empty_b = full_b + g.stages;          // [stages] MMAs done with the B stage
  uint64_t* full_a = empty_b + g.stages;          // [2] A tile written to tensor memory
  uint64_t* empty_a = full_a + kAStages;          // [2] MMAs done with the A tile
  uint64_t* tfull = empty_a + kAStages;           // [2] accumulator complete
  uint64_t* tempty = tfull + 2;                    // [2] accumulator drained
  uint64_t* drain = tempty + 2;                    // every MMA of this CTA complete
  int* iv = (int*)(drain + 1);                     // tmem, fail, tile, nblk, rows, k of the box
  volatile int* fail = iv + 1;
  unsigned short* bbox = (unsigned short*)(sm + g.o_bbox);
  uint2* kcoef = (uint2*)(sm + g.o_kcoef);
  int* kkey = (int*)(sm + g.o_kkey);
  char4* rows = (char4*)(sm + g.o_rows);
  unsigned* bits = (unsigned*)(sm + g.o_bits);
  int* slot = (int*)(sm + g.o_slot);
  int* cols = (int*)(sm + g.o_cols);
  int4* binfo = (int4*)(sm + g.o_binfo);
  long long* bvec = (long long*)(sm + g.o_bvec);
  short* ptab = (short*)(sm + g.o_ptab);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = d.nkpt * d.tc_nreg, rs = d.tc_rsize;
  const int f0 = d.fwf[0], f1 = d.fwf[1], f2 = d.fwf[2];
  const int kb1 = 2 * f1 + 1, kb2 = 2 * f2 + 1;
  const int p0 = d.fpair[0], p1 = d.fpair[1], p2 = d.fpair[2];
  const int rb1 = 2 * p1 + 1, rb2 = 2 * p2 + 1;
  const int nv = d.nv, nc = d.nc;
  const uint32_t half = (uint32_t)((g.nmax + 31) & ~31);    // Re [0, half), Im [half, 2 half) of an accumulator
  const uint32_t acc_cols = 2 * half;
  const uint32_t a_col0 = 2 * acc_cols;                      // the A tiles after the two accumulators

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(iv)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < g.stages; ++i) {
      mbar_init(smem_u32(full_b + i), 1);
      mbar_init(smem_u32(empty_b + i), 1);
    }
    for (int i = 0; i < kAStages; ++i) {
      mbar_init(smem_u32(full_a + i), kGWarps / kAStages);
      mbar_init(smem_u32(empty_a + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(tfull + i), 1);
      mbar_init(smem_u32(tempty + i), kEpiWarps);
    }
    mbar_init(smem_u32(drain), 1);
    iv[1] = 0;
    iv[5] = -1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = (uint32_t)iv[0];

  unsigned sc = 0, pc = 0;                       // stages and passes issued so far (same on every role)
  while (true) {
    __syncthreads();                             // every role is done with the previous tile
    if (tid == 0) iv[2] = *fail ? ntiles : atomicAdd(counter, 1);
    __syncthreads();
    const int t_ = iv[2];
    if (t_ >= ntiles) break;
    // region-major order: the CTAs in flight share one region's packed B rows, which stay in L2
    const int r = t_ / d.nkpt, k = t_ - r * d.nkpt;
    const int tile = k * d.tc_nreg + r;
    const int kc = d.tc_kcount[r];
    const bool newk = iv[5] != k;
    // ---- tile setup: columns, K keys, difference box of S(k), rows
    if (tid < rs) slot[tid] = blist[(size_t)tile * rs + tid];
    for (int i = tid; i < g.nwords; i += kThreads) bits[i] = 0u;
    for (int i = tid; i < g.nkc * kTKC; i += kThreads) {
      int key = g.bbox_c;                        // padding: G2 = 0 (the B images are zero there)
      if (i < kc) {
        const char4 g2 = d.tc_klist[(size_t)r * d.tc_kpad + i];
        key += ((int)g2.x * g.by + (int)g2.y) * g.bz + (int)g2.z;
      }
      kkey[i] = key;
    }
    if (newk)
      for (int i = tid; i < g.bbox_n; i += kThreads) bbox[i] = (unsigned short)d.npw_max;
    __syncthreads();
    if (warp == 0) {
      int n = 0;
      for (int b0 = 0; b0 < rs; b0 += 32) {
        const int j = b0 + lane;
        const int b = j < rs ? slot[j] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, b >= 0);
        if (b >= 0) cols[n + __popc(m & ((1u << lane) - 1u))] = b;
        n += __popc(m);
      }
      if (lane == 0) iv[3] = n;
    }
    if (newk) {
      const int n1 = d.npw[k];
      for (int i = tid; i < n1; i += kThreads) {
        const char4 gg = d.gk[(size_t)k * d.npw_max + i];
        bbox[g.bbox_c + ((int)gg.x * g.by + (int)gg.y) * g.bz + (int)gg.z] = (unsigned short)i;
      }
    }
    __syncthreads();
    if (tid == 0) iv[5] = k;
    const int nblk = iv[3];
    if (nblk == 0) continue;
    for (int i = tid; i < rs; i += kThreads) {  // per slot of the region; x = -1: no block of this range
      const int b = slot[i];
      if (b < 0) {
        binfo[i] = make_int4(-1, 0, 0, 0);
        continue;
      }
      const int4 blk = d.blocks[b];
      const long long qb = d.qblk_off[blk.z], nbq = d.qblk_off[blk.z + 1] - qb;
      const long long base = d.qvec_off[blk.z] - g.vbase;
      binfo[i] = make_int4(blk.z, blk.y, blk.w, 0);
      bvec[2 * i] = base + (b - qb) * nv * nv;
      bvec[2 * i + 1] = base + nbq * nv * nv + (b - qb) * nc * nc;
    }
    for (int i = 0; i < nblk; ++i) {
      const int4 blk = d.blocks[cols[i]];
      const int gx = (blk.w & 3) - 1, gy = ((blk.w >> 2) & 3) - 1, gz = ((blk.w >> 4) & 3) - 1;
      const int ng = d.ngq[blk.z];
      for (int p = tid; p < ng; p += kThreads) {
        const char4 gp = d.gq[(size_t)blk.z * d.ng_max + p];
        const int li = ((gp.x - gx + p0) * rb1 + gp.y - gy + p1) * rb2 + gp.z - gz + p2;
        atomicOr(&bits[li >> 5], 1u << (li & 31));
      }
    }
    __syncthreads();
    int ng_ref;
    {
      const int4 b0 = d.blocks[cols[0]];
      const int4 bi = make_int4(b0.z, b0.y, b0.w, 0);
      const int gx = (bi.z & 3) - 1, gy = ((bi.z >> 2) & 3) - 1, gz = ((bi.z >> 4) & 3) - 1;
      ng_ref = d.ngq[bi.x];
      for (int p = tid; p < ng_ref; p += kThreads) {
        const char4 gp = d.gq[(size_t)bi.x * d.ng_max + p];
        const int x = gp.x - gx, y = gp.y - gy, z = gp.z - gz;
        rows[p] = make_char4((signed char)x, (signed char)y, (signed char)z, 0);
        const int li = ((x + p0) * rb1 + y + p1) * rb2 + z + p2;
        atomicAnd(&bits[li >> 5], ~(1u << (li & 31)));
      }
    }
    __syncthreads();
    if (warp == 0) {
      int n = ng_ref;
      for (int w0 = 0; w0 < g.nwords; w0 += 32) {
        const int w = w0 + lane;
        unsigned m = w < g.nwords ? bits[w] : 0u;
        const int cnt = __popc(m);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        int pos = n + incl - cnt;
        while (m) {
          const int li = w * 32 + __ffs(m) - 1;
          m &= m - 1u;
          const int z = li % rb2, y = (li / rb2) % rb1, x = li / (rb2 * rb1);
          rows[pos++] = make_char4((signed char)(x - p0), (signed char)(y - p1), (signed char)(z - p2), 0);
        }
        n += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) iv[4] = n;
    }
    __syncthreads();
    const int MT = iv[4];
    const int nmt = (MT + 127) / 128;
    const int nch = (kc + kTKC - 1) / kTKC;

    if (warp >= kG0 && warp < kB0) {             // ---- gather: A tiles into tensor memory
      // warp -> lane quarter q4 (rows 32 q4 .. 32 q4 + 31 of the M tile) and A slot sa: the four warps of
      // slot sa write every other stage, all 32 K values, in two halves (the first store overlaps the
      // second half's lookups)
      const int gt = tid - kG0 * 32, q4 = warp & 3, sa = (warp - kG0) >> 2;
      unsigned s = sc;
      for (int set = 0; set < 2; ++set) {
        const int nset = set ? nc : nv, n0 = set ? nv : 0;
        for (int nn = 0; nn < nset; ++nn) {
          gather_bar();                          // every gather warp is done with the previous band
          {
            const int n1 = d.npw[k];
            const float2* cn = coef + ((size_t)k * d.nb + n0 + nn) * d.npw_max;
            for (int i = gt; i <= d.npw_max; i += kGThreads) {
              uint2 v = make_uint2(0u, 0u);
              if (i < n1) {
                const float2 c = cn[i];
                v = make_uint2(split_word(c.x), split_word(-c.y));    // conj
              }
              kcoef[i] = v;
            }
          }
          gather_bar();
          for (int mt = 0; mt < nmt; ++mt) {
            const int row = mt * 128 + q4 * 32 + lane;
            const bool rval = row < MT;
            int rkey = 0;
            if (rval) {
              const char4 G = rows[row];
              rkey = ((int)G.x * g.by + (int)G.y) * g.bz + (int)G.z;
            }
            for (int c = 0; c < nch; ++c, ++s) {
              if ((int)(s & 1u) != sa) continue;
              int ok = 1;
              if (lane == 0) {                   // warp-uniform decision
                ok = *fail ? 0 : 1;
                if (ok && s >= (unsigned)kAStages) {
                  ok = mbar_wait(smem_u32(empty_a + sa), ((s >> 1) - 1) & 1u) ? 1 : 0;
                  if (!ok) fail_now(fail, status);
                }
              }
              ok = __shfl_sync(0xffffffffu, ok, 0);
              if (!ok) continue;
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
              for (int hk = 0; hk < 2; ++hk) {
                uint32_t v[32];
                if (rval) {
                  const int4* kp = reinterpret_cast<const int4*>(kkey + c * kTKC + hk * 16);
                  int kk16[16];
#pragma unroll
                  for (int q = 0; q < 4; ++q) {
                    const int4 t = kp[q];
                    kk16[4 * q] = t.x;
                    kk16[4 * q + 1] = t.y;
                    kk16[4 * q + 2] = t.z;
                    kk16[4 * q + 3] = t.w;
                  }
                  uint2 x[16];
#pragma unroll
                  for (int e = 0; e < 16; ++e) x[e] = kcoef[bbox[kk16[e] - rkey]];
#pragma unroll
                  for (int j = 0; j < 8; ++j) {
                    v[j] = __byte_perm(x[2 * j].x, x[2 * j + 1].x, 0x5410);        // Re hi
                    v[8 + j] = __byte_perm(x[2 * j].y, x[2 * j + 1].y, 0x5410);    // Im hi
                    v[16 + j] = __byte_perm(x[2 * j].x, x[2 * j + 1].x, 0x7632);   // Re lo
                    v[24 + j] = __byte_perm(x[2 * j].y, x[2 * j + 1].y, 0x7632);   // Im lo
                  }
                } else {
#pragma unroll
                  for (int j = 0; j < 32; ++j) v[j] = 0u;
                }
                umma::tmem_st32(tmem + ((uint32_t)(q4 * 32) << 16) + a_col0 + (uint32_t)(sa * kACols + hk * 32), v);
              }
              asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
              asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(full_a + sa));
            }
          }
        }
      }
    } else if (warp == kB0) {                    // ---- B producer: the region's panel, two bulk copies per stage
      unsigned s = sc;
      for (int set = 0; set < 2; ++set) {
        const int nset = set ? nc : nv;
        const uint32_t half_bytes = (uint32_t)(rs * nset) * umma::kRow;
        for (int nn = 0; nn < nset; ++nn)
          for (int mt = 0; mt < nmt; ++mt)
            for (int c = 0; c < nch; ++c, ++s) {
              if (lane != 0) continue;
              const int st = (int)(s % (unsigned)g.stages);
              if (*fail) continue;
              if (s >= (unsigned)g.stages && !mbar_wait(smem_u32(empty_b + st), ((s / g.stages) - 1) & 1u)) {
                fail_now(fail, status);
                continue;
              }
              umma::mbar_arrive_expect_tx(smem_u32(full_b + st), 2 * half_bytes);
              const uint32_t bh = smem_u32(sm + (size_t)st * g.stage_bytes);
              const unsigned char* p = bimg + panel_off(d, r, set, c, g.nkc);
              umma::bulk_g2s(bh, p, half_bytes, smem_u32(full_b + st));
              umma::bulk_g2s(bh + (uint32_t)(g.nmax * umma::kRow), p + half_bytes, half_bytes, smem_u32(full_b + st));
            }
      }
    } else if (warp == kMmaWarp) {               // ---- MMA issue
      if (lane == 0) {
        unsigned s = sc, p = pc;
        bool ok = !*fail;
        const uint64_t dstage0 = umma::smem_desc(smem_u32(sm));     // B stage st: + st stage_bytes / 16
        const uint32_t blo = (uint32_t)((g.nmax * umma::kRow) >> 4);
        for (int set = 0; set < 2; ++set) {
          const int nset = set ? nc : nv;
          const int N = (rs * nset + 15) & ~15;
          const uint32_t idesc = umma::idesc_of(N);
          for (int nn = 0; nn < nset; ++nn)
            for (int mt = 0; mt < nmt; ++mt, ++p) {
              const int buf = (int)(p & 1u);
              if (ok && p >= 2 && !mbar_wait(smem_u32(tempty + buf), ((p >> 1) - 1) & 1u)) {
                fail_now(fail, status);
                ok = false;
              }
              if (ok) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t d_re = tmem + (uint32_t)buf * acc_cols, d_im = d_re + half;
              for (int c = 0; c < nch; ++c, ++s) {
                if (!ok || *fail) {
                  ok = false;
                  continue;
                }
                const int st = (int)(s % (unsigned)g.stages), sa = (int)(s & 1u);
                if (!mbar_wait(smem_u32(full_a + sa), (s >> 1) & 1u) ||
                    !mbar_wait(smem_u32(full_b + st), (s / g.stages) & 1u) || *fail) {
                  fail_now(fail, status);
                  ok = false;
                  continue;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t db = dstage0 + (uint64_t)((st * g.stage_bytes) >> 4);
                const uint32_t a = tmem + a_col0 + (uint32_t)(sa * kACols);
                const int nkk = (kc - c * kTKC > 16) ? 2 : 1;
                for (int kk = 0; kk < nkk; ++kk)
                  umma::mma_cplx_k16_ts(d_re, d_im, a + (uint32_t)(kk * 32), db, blo, kk, idesc, c == 0 && kk == 0);
                mma_commit(smem_u32(empty_a + sa));
                mma_commit(smem_u32(empty_b + st));
              }
              if (ok) mma_commit(smem_u32(tfull + buf));
            }
        }
      }
    } else {                                     // ---- epilogue: TMEM lanes 32 warp .. -> rows
      unsigned p = pc;
      const size_t pq = (size_t)(2 * f0 + 1) * kb1 * kb2;
      short* pt = ptab + (size_t)(warp * 32 + lane) * rs;
      for (int set = 0; set < 2; ++set) {
        const int nset = set ? nc : nv;
        const int ncols = rs * nset;
        for (int nn = 0; nn < nset; ++nn)
          for (int mt = 0; mt < nmt; ++mt, ++p) {
            const int buf = (int)(p & 1u);
            const int row = mt * 128 + warp * 32 + lane;
            const bool valid = row < MT;
            // sphere positions of this row on every block of the tile (independent loads, before the wait)
            if (valid) {
              const char4 G = rows[row];
#pragma unroll 4
              for (int b = 0; b < rs; ++b) {
                const int4 bi = binfo[b];
                const int x = G.x + (bi.z & 3) - 1, y = G.y + ((bi.z >> 2) & 3) - 1, z = G.z + ((bi.z >> 4) & 3) - 1;
                short pb = -1;
                if (bi.x >= 0 && x >= -f0 && x <= f0 && y >= -f1 && y <= f1 && z >= -f2 && z <= f2)
                  pb = d.tc_pmap[(size_t)bi.x * pq + ((size_t)(x + f0) * kb1 + y + f1) * kb2 + z + f2];
                pt[b] = pb;
              }
            }
            int ok = 1;
            if (lane == 0) {
              ok = (!*fail && mbar_wait(smem_u32(tfull + buf), (p >> 1) & 1u)) ? 1 : 0;
              if (!ok) fail_now(fail, status);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) continue;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c0 = 0; c0 < ncols; c0 += 32) {
              uint32_t v[32], u[32];
              const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)buf * acc_cols + (uint32_t)c0;
              umma::tmem_ld32(taddr, v);
              umma::tmem_ld32(taddr + half, u);
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
              if (!valid) continue;
              int b = c0 / nset, m = c0 - b * nset;
              int pb = pt[b];
              long long vec0 = bvec[2 * b + set] + (long long)nn * nset;
#pragma unroll
              for (int jj = 0; jj < 32; ++jj) {
                if (c0 + jj < ncols && pb >= 0)
                  out[(size_t)(vec0 + m) * d.ng_max + pb] = make_float2(__uint_as_float(v[jj]), __uint_as_float(u[jj]));
                if (++m == nset) {
                  m = 0;
                  ++b;
                  if (c0 + jj + 1 < ncols) {
                    pb = pt[b];
                    vec0 = bvec[2 * b + set] + (long long)nn * nset;
                  }
                }
              }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(tempty + buf));
          }
      }
    }
    sc += (unsigned)((nv + nc) * nmt * nch);
    pc += (unsigned)((nv + nc) * nmt);
  }
  if (warp == kMmaWarp && lane == 0) {          // tracks every MMA issued above
    mma_commit(smem_u32(drain));
    if (!mbar_wait(smem_u32(drain), 0u)) fail_now(fail, status);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ---------------------------------------------------------------- FP64 G = 0 overlaps of the diagonal blocks
// rho_nm^{kk}(0) = sum_G1 conj(c_nk(G1)) c_mk(G1), one warp per band product; q = 0 must be in the range.
__global__ void tcpair_diag_kernel(DevSys d, const float2* __restrict__ coef, float2* __restrict__ out,
                                   long long vbase) {
  const int k = blockIdx.x;
  const int b = d.blkidx[k];                     // q = 0 row of the table: the block (k, k)
  if (b < 0) return;
  const long long qb = d.qblk_off[0], nbq = d.qblk_off[1] - qb;
  const long long base = d.qvec_off[0] - vbase;
  const int nv = d.nv, nc = d.nc, n1 = d.npw[k];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = w; t < nv * nv + nc * nc; t += nw) {
    int a, bb;
    long long vec;
    if (t < nv * nv) {
      a = t / nv;
      bb = t % nv;
      vec = base + (b - qb) * nv * nv + t;
    } else {
      const int u = t - nv * nv;
      a = nv + u / nc;
      bb = nv + u % nc;
      vec = base + nbq * nv * nv + (b - qb) * nc * nc + u;
    }
    const float2* x = coef + ((size_t)k * d.nb + a) * d.npw_max;
    const float2* y = coef + ((size_t)k * d.nb + bb) * d.npw_max;
    double sr = 0.0, si = 0.0;
    for (int i = lane; i < n1; i += 32) {
      const float2 xv = x[i], yv = y[i];
      sr += (double)xv.x * yv.x + (double)xv.y * yv.y;      // conj(x) y
      si += (double)xv.x * yv.y - (double)xv.y * yv.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) out[(size_t)vec * d.ng_max] = make_float2((float)sr, (float)si);
  }
}

int stages_of(const DevSys& d) {
  for (int st = kMaxStages; st >= 2; --st)
    if (tp_geo(d, st).smem <= 227 * 1024) return st;
  return 0;
}

struct TpWs {
  size_t bimg, blist, counter, total;
};

TpWs tp_ws(const DevSys& d) {
  TpWs w;
  size_t o = 0;
  w.bimg = o; o += ((size_t)d.nkpt * d.nb * (d.tc_kpad / kTKC) * kImgRow + 255) & ~(size_t)255;
  w.blist = o; o += ((size_t)d.nkpt * d.tc_nreg * d.tc_rsize * sizeof(int) + 255) & ~(size_t)255;
  w.counter = o; o += 256;
  w.total = o;
  return w;
}

}  // namespace

// The tensor-core route needs a region of at most one N tile of columns and its tiles in shared memory.
int tcpair_valid(const DevSys& d) {
  if (d.tc_kpad < kTKC || d.tc_rsize < 1 || d.tc_rsize * (d.nv > d.nc ? d.nv : d.nc) > 96) return 0;
  if (d.tc_rsize > kThreads) return 0;
  return stages_of(d) > 0 ? 1 : 0;
}

size_t tcpair_ws_bytes(const DevSys& d) { return tcpair_valid(d) ? tp_ws(d).total : 0; }

// coef: the coefficient copy of the pair workspace; ws: the tensor-route area (tcpair_ws_bytes).
int launch_tcpair(const DevSys& d, const void* coef, void* ws, void* rho_dir, int q_begin, int q_end,
                  long long vbase, int* status, void* stream) {
  if (!tcpair_valid(d)) return (int)cudaErrorInvalidValue;
  static int attr_dev = -1, num_sms = 0;
  static size_t attr_smem = 0;
  const int stages = stages_of(d);
  TpGeo g = tp_geo(d, stages);
  int dev = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return e;
  if (attr_dev != dev || attr_smem < g.smem) {
    e = (int)cudaFuncSetAttribute((const void*)tcpair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(227 * 1024));
    if (e) return e;
    e = (int)cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    attr_dev = dev;
    attr_smem = 227 * 1024;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const TpWs w = tp_ws(d);
  unsigned char* base = (unsigned char*)ws;
  unsigned char* bimg = base + w.bimg;
  int* blist = (int*)(base + w.blist);
  int* counter = (int*)(base + w.counter);
  g.q_begin = q_begin;
  g.nqc = q_end - q_begin;
  g.vbase = vbase;
  if ((e = (int)cudaMemsetAsync(bimg, 0, w.blist - w.bimg, st))) return e;
  const long long npk = (long long)d.nkpt * d.nb * d.npw_max;
  tcpair_pack_kernel<<<(unsigned)((npk + 255) / 256), 256, 0, st>>>(d, (const float2*)coef, bimg, g.nkc);
  if ((e = (int)cudaGetLastError())) return e;
  if ((e = (int)cudaMemsetAsync(blist, 0xFF, w.counter - w.blist, st))) return e;
  const long long nt = (long long)g.nqc * d.nkpt;
  tcpair_tiles_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(d, q_begin, g.nqc, blist);
  if ((e = (int)cudaGetLastError())) return e;
  if ((e = (int)cudaMemsetAsync(counter, 0, sizeof(int), st))) return e;
  const int ntiles = d.nkpt * d.tc_nreg;
  const int grid = ntiles < num_sms ? ntiles : num_sms;
  tcpair_kernel<<<grid, kThreads, g.smem, st>>>(d, (const float2*)coef, bimg, blist, counter, (float2*)rho_dir, g,
                                                status);
  if ((e = (int)cudaGetLastError())) return e;
  if (q_begin == 0) {
    tcpair_diag_kernel<<<d.nkpt, 256, 0, st>>>(d, (const float2*)coef, (float2*)rho_dir, vbase);
    e = (int)cudaGetLastError();
  }
  return e;
}

}  // namespace bse
