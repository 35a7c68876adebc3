// Job decoding of the pair-density kernels (step A2): which (k, k') block, q, G0, bands and output
// vectors a CTA works on, and where each band product goes.  Shared by the pruned-FFT kernel and the
// plane-wave correlation kernel so that both write one layout.
#pragma once

#include "internal.h"

namespace bse {
namespace pj {

// Jobs are laid out over the (q, k) cells of a q chunk in tiles of kTQ x kTK so that
// CTAs running together share wavefunction slabs in L2.
constexpr int kTQ = 8, kTK = 16;

struct Job {
  int k, k2, a0, na, b0, nb, q, g0x, g0y, g0z;
  int mode;             // 0 (v x c) products, 1 vv', 2 cc', 3 vv' then cc';
                        // coupling: 5 vc' then cv', 6 vc', 7 cv'
  float2* out_v;        // first output vector of the vv' (exchange, vc') products
  float2* out_c;        // first output vector of the cc' (cv') products
};

__device__ __forceinline__ int nprod(const DevSys& d, int mode) {
  switch (mode) {
    case 0: case 6: case 7: return d.nv * d.nc;
    case 1: return d.nv * d.nv;
    case 2: return d.nc * d.nc;
    case 5: return 2 * d.nv * d.nc;
    default: return d.nv * d.nv + d.nc * d.nc;
  }
}

__device__ __forceinline__ bool decode_job(const DevSys& d, int mode, bool merged, int q0, int nqc, long long vbase,
                                           float2* out, Job& j) {
  if (mode == 4) {                         // v at k, c at k' = fold(k + q), k + q = k' + G0 (all k)
    const int qi = (int)(blockIdx.x / d.nkpt), k = (int)(blockIdx.x - (long long)qi * d.nkpt);
    const int q = q0 + qi;
    const int k1 = k / (d.nk2 * d.nk3), k2 = (k / d.nk3) % d.nk2, k3 = k % d.nk3;
    const int q1 = q / (d.nk2 * d.nk3), q2 = (q / d.nk3) % d.nk2, q3 = q % d.nk3;
    const int s1 = k1 + q1, s2 = k2 + q2, s3 = k3 + q3;
    const int f1 = s1 % d.nk1, f2 = s2 % d.nk2, f3 = s3 % d.nk3;
    j.k = k;
    j.k2 = (f1 * d.nk2 + f2) * d.nk3 + f3;
    j.q = q;
    j.g0x = -(s1 / d.nk1);                 // sampled at G - g0 = G + G0
    j.g0y = -(s2 / d.nk2);
    j.g0z = -(s3 / d.nk3);
    j.a0 = 0;
    j.na = d.nv;
    j.b0 = d.nv;
    j.nb = d.nc;
    j.mode = 0;
    j.out_v = out + ((size_t)qi * d.nkpt + k) * d.nv * d.nc * d.ng_max;
    j.out_c = nullptr;
    return true;
  }
  if (mode == 0) {
    j.k = j.k2 = blockIdx.x;
    j.a0 = 0;
    j.na = d.nv;
    j.b0 = d.nv;
    j.nb = d.nc;
    j.q = 0;
    j.g0x = j.g0y = j.g0z = 0;
    j.mode = 0;
    j.out_v = out + (size_t)blockIdx.x * d.nv * d.nc * d.ng_max;
    j.out_c = nullptr;
    return true;
  }
  long long cell = blockIdx.x;
  int group = 0;
  if (!merged) {
    group = (int)(cell & 1);
    cell >>= 1;
  }
  const int ntk = (d.nkpt + kTK - 1) / kTK;
  const long long tile = cell / (kTQ * kTK);
  const int u = (int)(cell - tile * (kTQ * kTK));
  const int tq = (int)(tile / ntk), tk = (int)(tile - (long long)tq * ntk);
  const int q = q0 + tq * kTQ + u / kTK;
  const int k = tk * kTK + u % kTK;
  if (q >= q0 + nqc || k >= d.nkpt) return false;
  const int b = d.blkidx[(size_t)q * d.nkpt + k];
  if (b < 0) return false;
  const int4 blk = d.blocks[b];
  j.k = blk.x;
  j.k2 = blk.y;
  j.q = blk.z;
  j.g0x = (blk.w & 3) - 1;
  j.g0y = ((blk.w >> 2) & 3) - 1;
  j.g0z = ((blk.w >> 4) & 3) - 1;
  const long long qb = d.qblk_off[q];
  const long long nblk = d.qblk_off[q + 1] - qb;
  const long long local = b - qb;
  if (mode == 5) {                         // coupling densities: per q [nblk][Nv Nc] vc', then [nblk][Nc Nv] cv'
    const long long w = (long long)d.nv * d.nc;
    const long long cbase = 2 * w * qb - vbase;
    j.out_v = out + (size_t)(cbase + local * w) * d.ng_max;
    j.out_c = out + (size_t)(cbase + nblk * w + local * w) * d.ng_max;
    if (merged) {
      j.mode = 5;
      j.a0 = j.b0 = 0;
      j.na = j.nb = d.nb;
    } else if (group == 0) {               // v at k, c at k'
      j.mode = 6;
      j.a0 = 0;
      j.na = d.nv;
      j.b0 = d.nv;
      j.nb = d.nc;
    } else {                               // c at k, v at k'
      j.mode = 7;
      j.a0 = d.nv;
      j.na = d.nc;
      j.b0 = 0;
      j.nb = d.nv;
    }
    return true;
  }
  const long long base = d.qvec_off[q] - vbase;
  j.out_v = out + (size_t)(base + local * d.nv * d.nv) * d.ng_max;
  j.out_c = out + (size_t)(base + nblk * d.nv * d.nv + local * d.nc * d.nc) * d.ng_max;
  if (merged) {
    j.mode = 3;
    j.a0 = j.b0 = 0;
    j.na = j.nb = d.nb;
  } else if (group == 0) {
    j.mode = 1;
    j.a0 = j.b0 = 0;
    j.na = j.nb = d.nv;
  } else {
    j.mode = 2;
    j.a0 = j.b0 = d.nv;
    j.na = j.nb = d.nc;
  }
  return true;
}

// product p -> (slab of the n band, slab of the m band, output vector)
__device__ __forceinline__ void product_of(const DevSys& d, const Job& j, int p, int& sa, int& sb, float2*& dst) {
  const int nv = d.nv, nc = d.nc;
  if (j.mode == 0) {                       // (v, c) at k = k'
    sa = p / nc;
    sb = j.na + p % nc;
    dst = j.out_v + (size_t)p * d.ng_max;
  } else if (j.mode == 1) {                // (v, v')
    sa = p / nv;
    sb = j.na + p % nv;
    dst = j.out_v + (size_t)p * d.ng_max;
  } else if (j.mode == 2) {                // (c, c')
    sa = p / nc;
    sb = j.na + p % nc;
    dst = j.out_c + (size_t)p * d.ng_max;
  } else if (j.mode == 5) {                // merged coupling: (v, c') then (c, v'); slabs hold all nb bands
    if (p < nv * nc) {
      sa = p / nc;
      sb = j.na + nv + p % nc;
      dst = j.out_v + (size_t)p * d.ng_max;
    } else {
      const int t = p - nv * nc;
      sa = nv + t / nv;
      sb = j.na + t % nv;
      dst = j.out_c + (size_t)t * d.ng_max;
    }
  } else if (j.mode == 6) {                // (v at k, c' at k')
    sa = p / nc;
    sb = j.na + p % nc;
    dst = j.out_v + (size_t)p * d.ng_max;
  } else if (j.mode == 7) {                // (c at k, v' at k')
    sa = p / nv;
    sb = j.na + p % nv;
    dst = j.out_c + (size_t)p * d.ng_max;
  } else if (p < nv * nv) {                // merged: (v, v') then (c, c'); slabs hold all nb bands
    sa = p / nv;
    sb = j.na + p % nv;
    dst = j.out_v + (size_t)p * d.ng_max;
  } else {
    const int t = p - nv * nv;
    sa = nv + t / nc;
    sb = j.na + nv + t % nc;
    dst = j.out_c + (size_t)t * d.ng_max;
  }
}

}  // namespace pj
}  // namespace bse
