// Pair densities by direct plane-wave correlation (step A2; Eq. pair_density in the plane-wave basis).
//
//   rho_nm^{kk'}(G) = sum_{G2 in S(k')} conj(c_nk(G2 - G)) c_mk'(G2),   G = g_p(q) - G0,
//
// c_nk(G1) = 0 outside the sphere S(k).  This is the same quantity as the pruned-FFT route of
// pair.cu (the FFT of conj(u_nk) u_mk' evaluated on the sphere of q), computed without the real-space
// grid: on these workloads a sphere holds ~1% of the FFT box (fcc 8x8x8: ~300 of 32^3 points), so
// the correlation takes ~4x fewer multiply-adds per band product than the FFT kernel spends, needs no
// grid, and has no aliasing condition.
//
// One CTA per job (decode_job of pairjob.cuh: the blocks of the direct and coupling sets, the
// exchange set, or the (k, k+q) set of the screening), one thread per sphere point p of q.
// Shared memory holds the job's coefficients at k (packed per G1, plus a zero row), those at k'
// (packed per G2 for broadcast loads), and a dense index box of S(k) over the key range
// G2 - G (per axis |.| <= fwf + fpair), whose entries outside the sphere point at the zero row.  The
// inner loop runs over G2: one box lookup, a
// gather of the k bands (one packed row, 128-bit loads), a broadcast of the k' bands, then every band
// product of the job as FP32 complex multiply-adds.  The G = 0 overlaps of the diagonal blocks are
// summed again in FP64.
#include <cuda_runtime.h>

#include "internal.h"
#include "pairjob.cuh"

namespace bse {
namespace {

using namespace pj;

constexpr int kGcMaxThreads = 576;      // one thread per sphere point up to 576 points (fcc 12x12x12: 531); 113 registers

// KIND 0: v x c at (k, k') (exchange and screening sets), 1: vv' then cc' (direct set),
// 2: vc' then cv' (coupling set).
template <int NV, int NC, int KIND>
struct Shape {
  static constexpr int NB = NV + NC;
  static constexpr int NA = KIND == 0 ? NV : NB;      // bands at k
  static constexpr int NK = KIND == 0 ? NC : NB;      // bands at k'
  static constexpr int NKP = (NK + 1) & ~1;           // packed row of k' bands (float4 loads)
  // packed row of k bands: even, and an odd number of 16-byte units so that rows gathered by
  // different lanes spread over the shared-memory banks
  static constexpr int RS = (((NA + 1) & ~1) / 2) % 2 == 1 ? ((NA + 1) & ~1) : ((NA + 1) & ~1) + 2;
  static constexpr int P = KIND == 0 ? NV * NC : (KIND == 1 ? NV * NV + NC * NC : 2 * NV * NC);
  // band at k, band at k', output (0: out_v, 1: out_c), index within that output
  static constexpr int a(int p) {
    return KIND == 0 ? p / NC : KIND == 1 ? (p < NV * NV ? p / NV : NV + (p - NV * NV) / NC)
                                          : (p < NV * NC ? p / NC : NV + (p - NV * NC) / NV);
  }
  static constexpr int b(int p) {
    return KIND == 0 ? p % NC : KIND == 1 ? (p < NV * NV ? p % NV : NV + (p - NV * NV) % NC)
                                          : (p < NV * NC ? NV + p % NC : (p - NV * NC) % NV);
  }
  static constexpr int o(int p) { return KIND == 0 ? 0 : KIND == 1 ? (p < NV * NV ? 0 : 1) : (p < NV * NC ? 0 : 1); }
  static constexpr int t(int p) {
    return KIND == 0 ? p : KIND == 1 ? (p < NV * NV ? p : p - NV * NV) : (p < NV * NC ? p : p - NV * NC);
  }
};

// Direct set split over two CTAs per block (vv' or cc'): NBG bands at k and at k', all NBG^2 products to
// the output of group GROUP (0: out_v, 1: out_c).  Half the accumulators of the merged shape, so two
// CTAs share an SM.
template <int NBG, int GROUP>
struct SplitShape {
  static constexpr int NA = NBG;
  static constexpr int NK = NBG;
  static constexpr int NKP = (NK + 1) & ~1;
  static constexpr int RS = (((NA + 1) & ~1) / 2) % 2 == 1 ? ((NA + 1) & ~1) : ((NA + 1) & ~1) + 2;
  static constexpr int P = NBG * NBG;
  static constexpr int a(int p) { return p / NBG; }
  static constexpr int b(int p) { return p % NBG; }
  static constexpr int o(int) { return GROUP; }
  static constexpr int t(int p) { return p; }
};

struct Box {
  int rx, ry, rz, dy, dz, n;   // key (g1, g2, g3) -> ((g1 + rx) dy + g2 + ry) dz + g3 + rz
};

template <class S>
size_t shape_smem_bytes(const DevSys& d, const Box& bx) {
  const size_t ca = (size_t)S::RS * (d.npw_max + 1) * sizeof(float2);
  const size_t cb = (size_t)d.npw_max * S::NKP * sizeof(float2);
  const size_t lin = (size_t)d.npw_max * sizeof(int);
  const size_t box = ((size_t)bx.n * sizeof(unsigned short) + 15) & ~(size_t)15;
  return ((ca + 15) & ~(size_t)15) + cb + lin + box;
}

template <int NV, int NC, int KIND>
size_t smem_bytes(const DevSys& d, const Box& bx) {
  return shape_smem_bytes<Shape<NV, NC, KIND>>(d, bx);
}

template <int NV, int NC>
size_t split_smem_bytes(const DevSys& d, const Box& bx) {
  return NV >= NC ? shape_smem_bytes<SplitShape<NV, 0>>(d, bx) : shape_smem_bytes<SplitShape<NC, 1>>(d, bx);
}

// Diagonal blocks (k = k', q = 0, G0 = 0): the first sphere point is G = 0, where the overlaps
// rho_nm^{kk}(0) are delta_nm (0 for the coupling set) up to rounding and meet the q = 0 head of W
// (~1e4 Ha bohr^3 for the slab workloads).  One warp sums them again with FP64 accumulation.
template <class S>
__device__ __noinline__ void g0_overlaps(const float2* ca, const float2* cb2, int n2, const Job& jb, int ng_max) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < S::P; ++q) {
    double sr = 0.0, si = 0.0;
    for (int i = lane; i < n2; i += 32) {
      const float2 x = ca[i * S::RS + S::a(q)], y = cb2[i * S::NKP + S::b(q)];
      sr += (double)x.x * y.x + (double)x.y * y.y;        // conj(x) y
      si += (double)x.x * y.y - (double)x.y * y.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      float2* dst = (S::o(q) == 0 ? jb.out_v : jb.out_c) + (size_t)S::t(q) * ng_max;
      dst[0] = make_float2((float)sr, (float)si);
    }
  }
}

// One job: shared-memory setup, then every sphere point of q over the sphere of k' (see top of file).
template <class S, int PF, bool OVERLAPS>
__device__ __forceinline__ void corr_body(const DevSys& d, const float2* __restrict__ coef, const Job& jb,
                                          const Box& bx) {
  constexpr int NA = S::NA, NK = S::NK, NKP = S::NKP, P = S::P;
  extern __shared__ __align__(16) float4 smv[];
  constexpr int RS = S::RS;
  float2* ca = reinterpret_cast<float2*>(smv);         // [npw_max + 1][RS]: k bands per G1; row npw_max is zero
  const size_t ca_bytes = (((size_t)RS * (d.npw_max + 1) * sizeof(float2)) + 15) & ~(size_t)15;
  float4* cb = reinterpret_cast<float4*>(reinterpret_cast<char*>(smv) + ca_bytes);   // [npw_max][NKP/2]
  int* lin2 = reinterpret_cast<int*>(cb + (size_t)d.npw_max * (NKP / 2));
  unsigned short* box = reinterpret_cast<unsigned short*>(lin2 + d.npw_max);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int zrow = d.npw_max;
  const int n1 = d.npw[jb.k], n2 = d.npw[jb.k2];

  for (int i = tid; i < bx.n; i += nt) box[i] = (unsigned short)zrow;
  for (int i = tid; i < RS * (d.npw_max + 1); i += nt) {
    const int g = i / RS, n = i - g * RS;
    ca[i] = (n < NA && g < n1) ? coef[((size_t)jb.k * d.nb + jb.a0 + n) * d.npw_max + g] : make_float2(0.f, 0.f);
  }
  float2* cb2 = reinterpret_cast<float2*>(cb);
  for (int i = tid; i < n2 * NKP; i += nt) {
    const int g = i / NKP, m = i - g * NKP;
    cb2[i] = m < NK ? coef[((size_t)jb.k2 * d.nb + jb.b0 + m) * d.npw_max + g] : make_float2(0.f, 0.f);
  }
  for (int i = tid; i < n2; i += nt) {
    const char4 g = d.gk[(size_t)jb.k2 * d.npw_max + i];
    lin2[i] = ((int)g.x * bx.dy + (int)g.y) * bx.dz + (int)g.z;
  }
  __syncthreads();
  for (int i = tid; i < n1; i += nt) {
    const char4 g = d.gk[(size_t)jb.k * d.npw_max + i];
    box[(((int)g.x + bx.rx) * bx.dy + (int)g.y + bx.ry) * bx.dz + (int)g.z + bx.rz] = (unsigned short)i;
  }
  __syncthreads();

  const int NG = d.ngq[jb.q];
  for (int p0 = 0; p0 < NG; p0 += nt) {
    const int p = p0 + tid;
    const bool act = p < NG;
    const char4 gp = d.gq[(size_t)jb.q * d.ng_max + (act ? p : 0)];
    // key of G1 = G2 - G with G = g_p - G0
    const int base = ((-(int)gp.x + jb.g0x + bx.rx) * bx.dy + (-(int)gp.y + jb.g0y + bx.ry)) * bx.dz +
                     (-(int)gp.z + jb.g0z + bx.rz);
    float acc[2 * P];
#pragma unroll
    for (int i = 0; i < 2 * P; ++i) acc[i] = 0.f;
    constexpr int NAP = (NA + 1) & ~1;
    if (PF) {
      // Software pipeline: the k bands of G2 index i + 1 (box lookup, then the gathered row) are loaded
      // while the products of index i run, so the two dependent shared-memory loads overlap the FMA block.
      const float4* ca4 = reinterpret_cast<const float4*>(ca);
      float4 a4[NAP / 2];
      {
        const int idx0 = n2 > 0 ? box[base + lin2[0]] : zrow;
#pragma unroll
        for (int n = 0; n < NAP / 2; ++n) a4[n] = ca4[idx0 * (RS / 2) + n];
      }
      for (int i = 0; i < n2; ++i) {
        const int idx_next = i + 1 < n2 ? box[base + lin2[i + 1]] : zrow;
        float4 an4[NAP / 2];
#pragma unroll
        for (int n = 0; n < NAP / 2; ++n) an4[n] = ca4[idx_next * (RS / 2) + n];
        float2 a[NAP];
#pragma unroll
        for (int n = 0; n < NAP / 2; ++n) {
          a[2 * n] = make_float2(a4[n].x, a4[n].y);
          a[2 * n + 1] = make_float2(a4[n].z, a4[n].w);
        }
        float2 bv[NKP];
#pragma unroll
        for (int m = 0; m < NKP / 2; ++m) {
          const float4 v = cb[i * (NKP / 2) + m];
          bv[2 * m] = make_float2(v.x, v.y);
          bv[2 * m + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const float2 x = a[S::a(q)], y = bv[S::b(q)];
          acc[2 * q] = fmaf(x.x, y.x, fmaf(x.y, y.y, acc[2 * q]));          // conj(x) y
          acc[2 * q + 1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, acc[2 * q + 1]));
        }
#pragma unroll
        for (int n = 0; n < NAP / 2; ++n) a4[n] = an4[n];
      }
    } else {
      int idx = n2 > 0 ? box[base + lin2[0]] : zrow;
      for (int i = 0; i < n2; ++i) {
        const int idx_next = i + 1 < n2 ? box[base + lin2[i + 1]] : zrow;   // next lookup overlaps this FMA block
        float2 a[NAP];
        const float4* row = reinterpret_cast<const float4*>(ca + (size_t)idx * RS);
#pragma unroll
        for (int n = 0; n < NAP / 2; ++n) {
          const float4 v = row[n];
          a[2 * n] = make_float2(v.x, v.y);
          a[2 * n + 1] = make_float2(v.z, v.w);
        }
        float2 bv[NKP];
#pragma unroll
        for (int m = 0; m < NKP / 2; ++m) {
          const float4 v = cb[(size_t)i * (NKP / 2) + m];
          bv[2 * m] = make_float2(v.x, v.y);
          bv[2 * m + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const float2 x = a[S::a(q)], y = bv[S::b(q)];
          acc[2 * q] = fmaf(x.x, y.x, fmaf(x.y, y.y, acc[2 * q]));          // conj(x) y
          acc[2 * q + 1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, acc[2 * q + 1]));
        }
        idx = idx_next;
      }
    }
    if (act) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        float2* dst = (S::o(q) == 0 ? jb.out_v : jb.out_c) + (size_t)S::t(q) * d.ng_max;
        dst[p] = make_float2(acc[2 * q], acc[2 * q + 1]);
      }
    }
    if (OVERLAPS && p0 == 0 && tid < 32 && jb.k == jb.k2) {
      const char4 g = d.gq[(size_t)jb.q * d.ng_max];
      if (g.x == 0 && g.y == 0 && g.z == 0 && jb.g0x == 0 && jb.g0y == 0 && jb.g0z == 0) {
        __syncwarp();
        g0_overlaps<S>(ca, cb2, n2, jb, d.ng_max);
      }
    }
  }
}

template <int NV, int NC, int KIND, int PF>
__global__ __launch_bounds__(kGcMaxThreads) void gcorr_kernel(DevSys d, const float2* __restrict__ coef,
                                                              float2* __restrict__ out, int mode, int q0, int nqc,
                                                              long long vbase, Box bx) {
  Job jb;
  if (!decode_job(d, mode, true, q0, nqc, vbase, out, jb)) return;
  corr_body<Shape<NV, NC, KIND>, PF, KIND != 0>(d, coef, jb, bx);
}

// Direct set with the vv' and cc' products of a block in separate CTAs (two CTAs per SM).
template <int NV, int NC>
__global__ __launch_bounds__(kGcMaxThreads, 2) void gcorr_split_kernel(DevSys d, const float2* __restrict__ coef,
                                                                      float2* __restrict__ out, int mode, int q0,
                                                                      int nqc, long long vbase, Box bx) {
  Job jb;
  if (!decode_job(d, mode, false, q0, nqc, vbase, out, jb)) return;
  if (jb.mode == 1)
    corr_body<SplitShape<NV, 0>, 0, true>(d, coef, jb, bx);
  else
    corr_body<SplitShape<NC, 1>, 0, true>(d, coef, jb, bx);
}

typedef void (*GcFn)(DevSys, const float2*, float2*, int, int, int, long long, Box);

// fn[kind][pf]: pf = 1 is the software-pipelined gather; split: the direct set in two CTAs per block
struct GcEntry {
  int nv, nc;
  GcFn fn[3][2];
  size_t (*smem[3])(const DevSys&, const Box&);
  GcFn split;
  size_t (*split_smem)(const DevSys&, const Box&);
};

#define BSE_GC(NV, NC)                                                                                   \
  GcEntry {                                                                                              \
    NV, NC,                                                                                              \
        {{gcorr_kernel<NV, NC, 0, 0>, gcorr_kernel<NV, NC, 0, 1>},                                       \
         {gcorr_kernel<NV, NC, 1, 0>, gcorr_kernel<NV, NC, 1, 1>},                                       \
         {gcorr_kernel<NV, NC, 2, 0>, gcorr_kernel<NV, NC, 2, 1>}},                                      \
        {smem_bytes<NV, NC, 0>, smem_bytes<NV, NC, 1>, smem_bytes<NV, NC, 2>}, gcorr_split_kernel<NV, NC>,  \
        split_smem_bytes<NV, NC>                                                                         \
  }

// band counts compiled: the fcc workloads (3v3c, 3v4c, 4v4c, the 2v2c test cell) and every
// hexagonal sheet of the batch (1-3 valence x 1-3 conduction)
const GcEntry kGc[] = {
    BSE_GC(3, 4), BSE_GC(3, 3), BSE_GC(4, 4), BSE_GC(2, 2), BSE_GC(1, 1), BSE_GC(1, 2),
    BSE_GC(1, 3), BSE_GC(2, 1), BSE_GC(2, 3), BSE_GC(3, 1), BSE_GC(3, 2),
};

const GcEntry* find(const DevSys& d) {
  for (const GcEntry& e : kGc)
    if (e.nv == d.nv && e.nc == d.nc) return &e;
  return nullptr;
}

Box box_of(const DevSys& d) {
  Box b;
  b.rx = d.fwf[0] + d.fpair[0];
  b.ry = d.fwf[1] + d.fpair[1];
  b.rz = d.fwf[2] + d.fpair[2];
  b.dy = 2 * b.ry + 1;
  b.dz = 2 * b.rz + 1;
  b.n = (2 * b.rx + 1) * b.dy * b.dz;
  return b;
}

int threads_of(const DevSys& d) {
  int t = (d.ng_max + 31) / 32 * 32;
  return t < kGcMaxThreads ? t : kGcMaxThreads;
}

}  // namespace

// Valid when the band counts are compiled, the sphere index fits 16 bits and shared memory suffices.
int gcorr_valid(const DevSys& d) {
  const GcEntry* e = find(d);
  if (!e || d.npw_max >= 65535) return 0;
  const Box bx = box_of(d);
  for (int k = 0; k < 3; ++k)
    if (e->smem[k](d, bx) > 227 * 1024) return 0;
  return 1;
}

// The split direct-set kernel fits two CTAs per SM when its shared memory does.
int gcorr_split_valid(const DevSys& d) {
  const GcEntry* e = find(d);
  if (!e || !gcorr_valid(d)) return 0;
  return e->split_smem(d, box_of(d)) <= 113 * 1024 ? 1 : 0;
}

int gcorr_threads(const DevSys& d) { return threads_of(d); }

// kind 0: exchange / screening sets, 1: direct set, 2: coupling set, 3: direct set split over two CTAs per
// block (cells must count both); cells = CTAs of the launch; pf = 1: the software-pipelined gather.
int launch_gcorr(const DevSys& d, const void* coef, void* out, int kind, int mode, int q0, int nqc, long long vbase,
                 long long cells, int pf, void* stream) {
  const GcEntry* e = find(d);
  if (!e || kind < 0 || kind > 3) return (int)cudaErrorInvalidValue;
  if (cells <= 0) return 0;
  if (cells >= (1LL << 31)) return (int)cudaErrorInvalidValue;
  const Box bx = box_of(d);
  const size_t sm = kind == 3 ? e->split_smem(d, bx) : e->smem[kind](d, bx);
  const GcFn fn = kind == 3 ? e->split : e->fn[kind][pf ? 1 : 0];
  int err = (int)cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (err) return err;
  fn<<<(unsigned)cells, threads_of(d), sm, (cudaStream_t)stream>>>(d, (const float2*)coef, (float2*)out,
                                                                          mode, q0, nqc, vbase, bx);
  return (int)cudaGetLastError();
}

}  // namespace bse
