// Pair densities by batched, pruned 3D FFTs (steps A1, A2) and the k.p dipole (A6).
//
// Eq. pair_density: rho_nm^{kk'}(G) = <psi_nk| exp(-i(q+G).r) |psi_mk'> with k' = k + q
// unfolded; with psi = Omega^{-1/2} exp(ik.r) u and u(r) = sum_G c(G) exp(iG.r) this is
// (1/N_r) sum_r conj(u_nk(r)) u_mk'(r) exp(-iG.r) on an alias-free grid.
//
// A1 (realspace_kernel): one CTA per (k, n).  The sphere is scattered into a small
// box of the kept frequencies, then three passes of register FFTs (x, y, z) expand
// it onto the N1 x N2 x N3 grid; only lines that carry nonzero data are transformed.
//
// A2 (pair_kernel): one CTA per job = (k, k', band set n, band set m).  The grid is
// streamed in x-slabs, ROWS z-lines at a time, for every band of the job (each
// u_nk line read once per job and reused by all |m| products): one 2D tensor copy
// (TMA) per band and chunk into a double buffer, completion counted on an mbarrier
// per buffer.  The copy box is N3 + 2 wide so that the two out-of-bounds columns
// (filled with zeros) pad the shared rows for conflict-free float4 reads.  Per slab:
//   stage 1: each thread forms conj(u_n) u_m along one z-line and FFTs it in
//            registers, keeping |f3| <= F3;
//   stage 2: y-line FFTs of the kept planes, keeping |f2| <= F2;
//   stage 3: the x direction is a direct DFT accumulated over slabs, evaluated
//            only at the sphere points (register accumulators; each thread owns
//            sphere points and accumulates every product there).
// Work therefore scales with the kept windows rather than with N^3 log N in the
// last two passes.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>

#include "fft.cuh"
#include "pairjob.cuh"
#include "internal.h"

namespace bse {
namespace {

__constant__ float2 c_tw[fft::kTwN];

using fft::cadd;
using fft::cconj;
using fft::cmul;

constexpr int kThreads = 256;

// ---------------------------------------------------------------- A1
template <int N1, int N2, int N3, int F1, int F2, int F3>
struct RsCfg {
  static constexpr int M1 = 2 * F1 + 1, M2 = 2 * F2 + 1, M3 = 2 * F3 + 1;
  static constexpr int GS = (N1 % 16 == 0) ? 16 : ((N1 % 12 == 0) ? 12 : ((N1 % 8 == 0) ? 8 : N1));
  static constexpr size_t smem = sizeof(float2) * ((size_t)M1 * M2 * M3 + (size_t)N1 * M2 * M3 + (size_t)GS * N2 * M3);
};

template <int N1, int N2, int N3, int F1, int F2, int F3>
__global__ __launch_bounds__(kThreads) void realspace_kernel(DevSys d, const float2* __restrict__ coef,
                                                             float2* __restrict__ u) {
  using C = RsCfg<N1, N2, N3, F1, F2, F3>;
  constexpr int M1 = C::M1, M2 = C::M2, M3 = C::M3, GS = C::GS;
  extern __shared__ float4 sm4[];
  float2* box = reinterpret_cast<float2*>(sm4);
  float2* T1 = box + M1 * M2 * M3;
  float2* T2 = T1 + N1 * M2 * M3;
  const int tid = threadIdx.x;
  const int k = blockIdx.x / d.nb, n = blockIdx.x % d.nb;
  for (int i = tid; i < M1 * M2 * M3; i += kThreads) box[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int npw = d.npw[k];
  for (int t = tid; t < npw; t += kThreads) {
    const char4 g = d.gk[(size_t)k * d.npw_max + t];
    box[((g.x + F1) * M2 + (g.y + F2)) * M3 + (g.z + F3)] = coef[((size_t)k * d.nb + n) * d.npw_max + t];
  }
  __syncthreads();
  for (int it = tid; it < M2 * M3; it += kThreads) {          // x pass, nonzero (f2, f3) lines
    float2 x[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) x[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int f = -F1; f <= F1; ++f) x[(f + N1) % N1] = box[(f + F1) * M2 * M3 + it];
    fft::line<N1, false>(x);
#pragma unroll
    for (int j = 0; j < N1; ++j) T1[j * M2 * M3 + it] = x[j];
  }
  __syncthreads();
  float2* dst0 = u + ((size_t)k * d.nb + n) * ((size_t)N1 * N2 * N3);
  for (int s0 = 0; s0 < N1; s0 += GS) {
    for (int it = tid; it < GS * M3; it += kThreads) {        // y pass on GS slabs
      const int jj = it / M3, m3 = it % M3;
      float2 y[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) y[j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int f = -F2; f <= F2; ++f) y[(f + N2) % N2] = T1[((s0 + jj) * M2 + (f + F2)) * M3 + m3];
      fft::line<N2, false>(y);
#pragma unroll
      for (int j = 0; j < N2; ++j) T2[(jj * N2 + j) * M3 + m3] = y[j];
    }
    __syncthreads();
    for (int it = tid; it < GS * N2; it += kThreads) {        // z pass, full lines written out
      const int jj = it / N2, j2 = it % N2;
      float2 z[N3];
#pragma unroll
      for (int j = 0; j < N3; ++j) z[j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int f = -F3; f <= F3; ++f) z[(f + N3) % N3] = T2[(jj * N2 + j2) * M3 + (f + F3)];
      fft::line<N3, false>(z);
      float4* dst = reinterpret_cast<float4*>(dst0 + ((size_t)(s0 + jj) * N2 + j2) * N3);
#pragma unroll
      for (int j = 0; j < N3 / 2; ++j) dst[j] = make_float4(z[2 * j].x, z[2 * j].y, z[2 * j + 1].x, z[2 * j + 1].y);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- A2
// Template parameters: grid N1 x N2 x N3; kept windows |f2| <= F2, |f3| <= F3; PMAX band
// products and BMAX band slabs per CTA; ROWS z-lines per pipelined chunk; PPT sphere points
// per thread in stage 3; THREADS per CTA; MERGED = one CTA computes both the vv' and the cc'
// products of a block (else one CTA per block and group); SINGLE = whole x-slabs (ROWS = N2) in
// one buffer whose refill is issued after stage 1 and lands during stages 2 and 3 (else two
// buffers of ROWS-line chunks, the next chunk loading while the current one is transformed).
template <int N1, int N2, int N3, int F2, int F3, int PMAX, int BMAX, int ROWS, int PPT, int THREADS, bool MERGED,
          bool SINGLE>
struct PairCfg {
  static constexpr int M2 = 2 * F2 + 1, M3 = 2 * F3 + 1;
  static constexpr int LD = N3 + 2;    // z-line stride in shared memory: 16-B aligned rows, float4 reads conflict-free
  static constexpr int NCH = N1 * (N2 / ROWS);
  static_assert(N2 % ROWS == 0, "ROWS must divide N2");
  static_assert(BMAX <= THREADS, "one band copy per thread and chunk");
  static_assert(!SINGLE || ROWS == N2, "a single buffer holds whole slabs");
  static constexpr int NBUF = SINGLE ? 1 : 2;
  static_assert(((N3 + 2) * 8) % 16 == 0, "copy box rows are 16-byte multiples");
  static constexpr int S1P = (N2 + 1) * M3;   // product stride of S1 (one padding row: spreads banks)
  static constexpr int BSTR = (ROWS * LD * 8 + 127) / 128 * 16;   // band stride in float2: 128-byte multiple
  static size_t smem(int ng_max) {
    return 24 + sizeof(float2) * ((size_t)NBUF * BMAX * BSTR + (size_t)PMAX * S1P + (size_t)PMAX * M2 * M3 + N1) +
           sizeof(int2) * (size_t)ng_max;
  }
};

using namespace pj;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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

template <int N1, int N2, int N3, int F2, int F3, int PMAX, int BMAX, int ROWS, int PPT, int THREADS, bool MERGED,
          bool SINGLE>
__global__ __launch_bounds__(THREADS, 1) void pair_kernel(DevSys d, const float2* __restrict__ u,
                                                          float2* __restrict__ out, int mode, int q0, int nqc,
                                                          long long vbase, int* status,
                                                          const __grid_constant__ CUtensorMap tm) {
  using C = PairCfg<N1, N2, N3, F2, F3, PMAX, BMAX, ROWS, PPT, THREADS, MERGED, SINGLE>;
  constexpr int M2 = C::M2, M3 = C::M3, LD = C::LD, NCH = C::NCH, S1P = C::S1P, BSTR = C::BSTR;
  constexpr int CPR = N2 / ROWS;            // chunks per slab
  extern __shared__ __align__(128) float4 sm4[];
  float2* ub = reinterpret_cast<float2*>(sm4);          // [NBUF][BMAX][BSTR]: ROWS rows of LD per band
  float2* S1 = ub + C::NBUF * BMAX * BSTR;              // [PMAX][N2 (+1 pad)][M3]
  float2* S2 = S1 + PMAX * S1P;                         // [PMAX][M2][M3]
  float2* tw1 = S2 + PMAX * M2 * M3;                    // [N1] exp(-2 pi i g j1/N1) of the current slab
  uint64_t* bars = reinterpret_cast<uint64_t*>(tw1 + N1);   // [2] chunk landed (one per buffer)
  volatile int& s_fail = *reinterpret_cast<volatile int*>(bars + 2);
  int2* sg = reinterpret_cast<int2*>(bars + 3);

  Job jb;
  if (!decode_job(d, mode, MERGED, q0, nqc, vbase, out, jb)) return;
  const int tid = threadIdx.x;
  if (smem_u32(sm4) & 127u) {               // box copies need 128-byte aligned destinations
    if (tid == 0) atomicCAS(status, 0, (int)BSE_ERR_CUDA);
    return;
  }
  const uint32_t bar0 = smem_u32(bars);
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int P = nprod(d, jb.mode);
  const int NG = d.ngq[jb.q];
  for (int t = tid; t < NG; t += THREADS) {
    const char4 g = d.gq[(size_t)jb.q * d.ng_max + t];
    const int G1 = g.x - jb.g0x, G2 = g.y - jb.g0y, G3 = g.z - jb.g0z;   // G = g_p - G0
    sg[t] = make_int2(((G1 % N1) + N1) % N1, (G2 + F2) * M3 + (G3 + F3));
  }
  float2 acc[PPT * PMAX];
#pragma unroll
  for (int a = 0; a < PPT * PMAX; ++a) acc[a] = make_float2(0.f, 0.f);

  // loads: thread tid < nbands copies band tid's ROWS z-lines of each chunk as one 2D box (LD x ROWS;
  // the two columns past N3 are out of bounds and arrive as zeros)
  const int nbands = jb.na + jb.nb;
  long long lbase = 0;
  if (tid < nbands)
    lbase = (tid < jb.na) ? ((long long)jb.k * d.nb + jb.a0 + tid) * (N1 * N2)
                          : ((long long)jb.k2 * d.nb + jb.b0 + tid - jb.na) * (N1 * N2);
  constexpr uint32_t kBox = ROWS * LD * sizeof(float2), kBand = BSTR * sizeof(float2), kBuf = BMAX * kBand;
  const uint32_t chunk_bytes = (uint32_t)nbands * kBox;
  const uint32_t ldst = smem_u32(ub) + (uint32_t)tid * kBand;
  __syncthreads();                          // barriers initialised, sphere table filled

  bool alive = true;                        // false once one of this thread's waits gave up
  // chunk c lands in buffer bufi(c), counted on mbarrier bufi(c) in phase phase(c)
  auto bufi = [](int c) { return SINGLE ? 0 : (c & 1); };
  auto phase = [](int c) { return (uint32_t)(SINGLE ? c : (c >> 1)) & 1u; };
  auto issue = [&](int c) {
    if (!alive) return;
    const int j1 = c / CPR, r0 = (c - j1 * CPR) * ROWS;
    const uint32_t bar = bar0 + 8u * (uint32_t)bufi(c);
    if (tid == 0) mbar_expect_tx(bar, chunk_bytes);
    if (tid < nbands) {
      const int y = (int)(lbase + j1 * N2 + r0);
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
          ::"r"(ldst + (uint32_t)bufi(c) * kBuf), "l"(reinterpret_cast<uint64_t>(&tm)), "r"(0), "r"(y), "r"(bar)
          : "memory");
    }
  };

  // stage-1 items of this thread (fixed for every chunk): line it = tid + k THREADS
  constexpr int K1 = (PMAX * ROWS + THREADS - 1) / THREADS;
  int it1[K1], p1[K1], sa1[K1], sb1[K1];
#pragma unroll
  for (int k1 = 0; k1 < K1; ++k1) {
    it1[k1] = tid + k1 * THREADS;
    p1[k1] = it1[k1] / ROWS;
    float2* dst_unused;
    if (it1[k1] < P * ROWS) product_of(d, jb, p1[k1], sa1[k1], sb1[k1], dst_unused);
  }

  // Barriers: a chunk that does not end a slab ends with one (its buffer is refilled next);
  // a slab-end chunk has one before stage 2 and one before stage 3, which also order every
  // thread's wait on a buffer's mbarrier before the next expect_tx on it.  With a single
  // buffer the next slab is issued after the barrier that ends stage 1.
  issue(0);
  for (int c = 0; c < NCH; ++c) {
    if (!SINGLE && c + 1 < NCH) issue(c + 1);
    if (alive && !mbar_wait(bar0 + 8u * (uint32_t)bufi(c), phase(c))) {
      alive = false;                        // a copy never landed: stop waiting and issuing, report below
      s_fail = 1;
    }
    const int j1 = c / CPR, r0 = (c - j1 * CPR) * ROWS;
    const float2* buf = ub + (size_t)bufi(c) * BMAX * BSTR;
#pragma unroll
    for (int k1 = 0; k1 < K1; ++k1) {                           // stage 1: product + z FFT
      if (it1[k1] >= P * ROWS) continue;
      const int p = p1[k1], row = it1[k1] - p * ROWS;
      const int sa = sa1[k1], sb = sb1[k1];
      const float4* xa = reinterpret_cast<const float4*>(buf + (size_t)sa * BSTR + (size_t)row * LD);
      const float4* xb = reinterpret_cast<const float4*>(buf + (size_t)sb * BSTR + (size_t)row * LD);
      float2 x[N3];
#pragma unroll
      for (int h = 0; h < N3 / 2; ++h) {
        const float4 va = xa[h], vb = xb[h];
        x[2 * h] = make_float2(va.x * vb.x + va.y * vb.y, va.x * vb.y - va.y * vb.x);          // conj(a) b
        x[2 * h + 1] = make_float2(va.z * vb.z + va.w * vb.w, va.z * vb.w - va.w * vb.z);
      }
      fft::line<N3, true>(x);
      float2* s1 = S1 + (size_t)p * S1P + (size_t)(r0 + row) * M3;
#pragma unroll
      for (int f = -F3; f <= F3; ++f) s1[f + F3] = x[(f + N3) % N3];
    }
    if (r0 + ROWS == N2) {                                       // slab complete
      __syncthreads();
      if (SINGLE && c + 1 < NCH) issue(c + 1);                  // lands during stages 2 and 3
      for (int it = tid; it < P * M3; it += THREADS) {          // stage 2: y FFT of kept planes
        const int p = it / M3, m3 = it - p * M3;
        float2 y[N2];
#pragma unroll
        for (int j = 0; j < N2; ++j) y[j] = S1[(size_t)p * S1P + (size_t)j * M3 + m3];
        fft::line<N2, true>(y);
#pragma unroll
        for (int f = -F2; f <= F2; ++f) S2[((size_t)p * M2 + (f + F2)) * M3 + m3] = y[(f + N2) % N2];
      }
      for (int g = tid; g < N1; g += THREADS) tw1[g] = fft::tw<N1, true>(c_tw, g * j1);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < PPT; ++i) {                            // stage 3: x DFT at this thread's sphere points
        const int t = tid + i * THREADS;
        if (t < NG) {
          const int2 g = sg[t];
          const float2 w = tw1[g.x];
          const float2* s2 = S2 + g.y;
#pragma unroll
          for (int p = 0; p < PMAX; ++p)
            if (p < P) acc[i * PMAX + p] = cadd(acc[i * PMAX + p], cmul(s2[p * M2 * M3], w));
        }
      }
    } else {
      __syncthreads();
    }
  }
  __syncthreads();
  if (s_fail) {                             // bounded wait for copies still in flight, then report
    if (tid == 0) {
      if (!SINGLE && NCH >= 2) mbar_wait(bar0 + 8u * (uint32_t)bufi(NCH - 2), phase(NCH - 2));
      mbar_wait(bar0 + 8u * (uint32_t)bufi(NCH - 1), phase(NCH - 1));
      atomicCAS(status, 0, (int)BSE_ERR_TIMEOUT);
    }
    return;
  }
  const float inv = 1.0f / (float)(N1 * N2 * N3);
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int t = tid + i * THREADS;
    if (t >= NG) continue;
#pragma unroll
    for (int p = 0; p < PMAX; ++p) {
      if (p < P) {
        int sa, sb;
        float2* dst;
        product_of(d, jb, p, sa, sb, dst);
        dst[t] = make_float2(acc[i * PMAX + p].x * inv, acc[i * PMAX + p].y * inv);
      }
    }
  }
}

// ---------------------------------------------------------------- A6
__global__ void dipole_kernel(DevSys d, const float2* __restrict__ coef, const double* __restrict__ e,
                              double gap_floor, double2* __restrict__ P) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= d.dim) return;
  const int ic = warp % d.nc, iv = (warp / d.nc) % d.nv, k = warp / (d.nv * d.nc);
  const float2* cv = coef + ((size_t)k * d.nb + iv) * d.npw_max;
  const float2* cc = coef + ((size_t)k * d.nb + d.nv + ic) * d.npw_max;
  const double* kg = d.kgq + (size_t)k * d.npw_max;
  double re = 0.0, im = 0.0;
  for (int t = lane; t < d.npw[k]; t += 32) {
    const double2 a = make_double2(cv[t].x, cv[t].y), b = make_double2(cc[t].x, cc[t].y);
    // conj(a) * b * (qhat.(k+G))
    re += kg[t] * (a.x * b.x + a.y * b.y);
    im += kg[t] * (a.x * b.y - a.y * b.x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    const double de = fmax(e[(size_t)k * d.nb + d.nv + ic] - e[(size_t)k * d.nb + iv], gap_floor);
    P[warp] = make_double2(re / de, -im / de);     // conj(sum) / de
  }
}

// ---------------------------------------------------------------- dispatch
typedef void (*RsFn)(DevSys, const float2*, float2*);
typedef void (*PairFn)(DevSys, const float2*, float2*, int, int, int, long long, int*, CUtensorMap);

struct Variant {
  int n1, n2, n3, f1, f2, f3, pmax, bmax, threads, ppt, rows;
  bool merged;
  RsFn rs;
  size_t rs_smem;
  PairFn pair;
  size_t (*pair_smem)(int);
};

#define BSE_VARIANT(N1, N2, N3, F1, F2, F3, PMAX, BMAX, ROWS, PPT, THREADS, MERGED, SINGLE)                      \
  Variant {                                                                                                      \
    N1, N2, N3, F1, F2, F3, PMAX, BMAX, THREADS, PPT, ROWS, MERGED, realspace_kernel<N1, N2, N3, F1, F2, F3>,    \
        RsCfg<N1, N2, N3, F1, F2, F3>::smem,                                                                     \
        pair_kernel<N1, N2, N3, F2, F3, PMAX, BMAX, ROWS, PPT, THREADS, MERGED, SINGLE>,                         \
        PairCfg<N1, N2, N3, F2, F3, PMAX, BMAX, ROWS, PPT, THREADS, MERGED, SINGLE>::smem                        \
  }

// Candidate tile shapes per grid; the planner takes the first valid one unless a variant was chosen
// (by the autotuner or the caller).  The hexagonal-sheet grid has variants sized for 2-5, 8-10 and
// 18 band products, the fcc 8x8x8 grid three chunk heights (whole slabs measured fastest).
const Variant kVariants[] = {
    BSE_VARIANT(8, 8, 8, 2, 2, 2, 18, 12, 8, 1, 128, true, false),         // small test cells
    BSE_VARIANT(24, 24, 24, 3, 3, 3, 18, 12, 24, 1, 448, true, false),     // fcc 4x4x4, 3v3c
    BSE_VARIANT(32, 32, 32, 5, 5, 5, 25, 14, 32, 1, 416, true, true),      // fcc 8x8x8, 3v4c: whole slabs
    BSE_VARIANT(32, 32, 32, 5, 5, 5, 25, 14, 16, 1, 416, true, false),     //   half slabs, two buffers
    BSE_VARIANT(32, 32, 32, 5, 5, 5, 25, 14, 8, 2, 224, true, false),      //   half-height chunks
    BSE_VARIANT(48, 48, 48, 6, 6, 6, 16, 8, 16, 3, 256, false, false),     // fcc 12x12x12, 4v4c
    BSE_VARIANT(12, 12, 48, 2, 2, 10, 18, 12, 12, 1, 224, true, false),    // hexagonal sheets, <= 3v3c
    BSE_VARIANT(12, 12, 48, 2, 2, 10, 10, 8, 12, 1, 128, true, false),     //   <= 10 products, <= 4 bands
    BSE_VARIANT(12, 12, 48, 2, 2, 10, 5, 6, 12, 2, 64, true, false),       //   1v2c, 2v1c, 1v1c
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

bool valid_for(const Variant& v, const DevSys& d) {
  if (v.n1 != d.n1 || v.n2 != d.n2 || v.n3 != d.n3) return false;
  const int vmax = d.nv > d.nc ? d.nv : d.nc;
  const int f[3] = {v.f1, v.f2, v.f3};
  bool ok = true;
  for (int j = 0; j < 3; ++j) ok = ok && d.fwf[j] <= f[j] && d.fpair[j] <= f[j];
  const int pd = v.merged ? d.nv * d.nv + d.nc * d.nc : vmax * vmax;
  const int bd = v.merged ? 2 * d.nb : 2 * vmax;
  const int px = d.nv * d.nc;
  const int pm = pd > px ? pd : px;
  return ok && pm <= v.pmax && bd <= v.bmax && d.nb <= v.bmax && d.ng_max <= v.ppt * v.threads;
}

// FFT variant for the real-space stage and for pair launches when no correlation variant is in use.
const Variant* pick(const DevSys& d) {
  if (d.pair_variant >= 0 && d.pair_variant < kNumVariants && valid_for(kVariants[d.pair_variant], d))
    return &kVariants[d.pair_variant];
  for (const Variant& v : kVariants)
    if (valid_for(v, d)) return &v;
  return nullptr;
}

// The plane-wave correlation kernel (gcorr.cu) is variant kGcorrIndex; it is the default wherever it
// is compiled for the system's band counts, and the FFT variants stay selectable.
// Variant kGcorrPfIndex is the same kernel with the gather of the next G2 row software-pipelined;
// kGcorrSplitIndex runs the direct set with the vv' and cc' products of a block in separate CTAs
// (the other sets as kGcorrIndex).
constexpr int kGcorrIndex = 64, kGcorrPfIndex = 65, kGcorrSplitIndex = 66;
constexpr int kGcorrDefaultPf = 0;
bool use_gcorr(const DevSys& d) {
  if (!gcorr_valid(d)) return false;
  return d.pair_variant == -1 || d.pair_variant == kGcorrIndex || d.pair_variant == kGcorrPfIndex ||
         (d.pair_variant == kGcorrSplitIndex && gcorr_split_valid(d));
}
bool gcorr_split(const DevSys& d) { return d.pair_variant == kGcorrSplitIndex && gcorr_split_valid(d); }
int gcorr_pf(const DevSys& d) {
  return d.pair_variant == kGcorrPfIndex ? 1 : d.pair_variant == kGcorrIndex ? 0 : kGcorrDefaultPf;
}

// Coefficients c_nk(G) are kept after u_nk(r) in the pair workspace (the correlation kernel reads them).
size_t u_bytes(const DevSys& d) { return ((size_t)d.nkpt * d.nb * d.n1 * d.n2 * d.n3 * 8 + 255) & ~(size_t)255; }
const void* coef_copy(const DevSys& d, const void* ws) { return (const char*)ws + u_bytes(d); }

// Tensor map of the u(r) workspace as a 2D array of z-lines ([Nk Nb N1 N2] lines x N3 complex,
// 8-byte elements); boxes of (N3 + 2) x ROWS, out-of-bounds elements read as zero.
static int make_tmap(const DevSys& d, const Variant* v, const void* u, CUtensorMap* tm) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q) != cudaSuccess || !fp)
      return (int)cudaErrorUnknown;
    enc = (PFN_cuTensorMapEncodeTiled_v12000)fp;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)d.n3, (cuuint64_t)d.nkpt * d.nb * d.n1 * d.n2};
  cuuint64_t gstr[1] = {(cuuint64_t)d.n3 * 8};
  cuuint32_t box[2] = {(cuuint32_t)(d.n3 + 2), (cuuint32_t)v->rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(u), gdim, gstr, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}
}  // namespace

int upload_twiddles() {
  float2 h[fft::kTwN];
  for (int t = 0; t < fft::kTwN; ++t)
    h[t] = make_float2((float)std::cos(2.0 * kPi * t / fft::kTwN), (float)std::sin(2.0 * kPi * t / fft::kTwN));
  return (int)cudaMemcpyToSymbol(c_tw, h, sizeof(h));
}

int pair_supported(const DevSys& d) { return pick(d) != nullptr; }

static size_t pair_base_bytes(const DevSys& d) {
  return (u_bytes(d) + (size_t)d.nkpt * d.nb * d.npw_max * 8 + 255) & ~(size_t)255;
}

// u(r), the coefficient copy, then the tensor route's packed images and tile table (when valid).
size_t pair_ws_bytes(const DevSys& d) { return pair_base_bytes(d) + tcpair_ws_bytes(d); }

int launch_pair_direct_tensor(const DevSys& d, void* ws, void* rho_dir, int q_begin, int q_end, long long vbase,
                              int* status, void* stream) {
  return launch_tcpair(d, coef_copy(d, ws), (char*)ws + pair_base_bytes(d), rho_dir, q_begin, q_end, vbase, status,
                       stream);
}

int pair_variants(const DevSys& d, int* out, int cap) {
  int n = 0;
  if (gcorr_valid(d)) {                      // rows = 0 marks the plane-wave correlation kernel
    const int order[3] = {kGcorrDefaultPf ? kGcorrPfIndex : kGcorrIndex, kGcorrDefaultPf ? kGcorrIndex : kGcorrPfIndex,
                          kGcorrSplitIndex};
    for (int idx : order) {
      if (idx == kGcorrSplitIndex && !gcorr_split_valid(d)) continue;
      if (out && n < cap) {
        int* o = out + 7 * n;
        o[0] = idx;
        o[1] = gcorr_threads(d);
        o[2] = 0;
        const int pd = idx == kGcorrSplitIndex ? (d.nv > d.nc ? d.nv * d.nv : d.nc * d.nc)
                                               : d.nv * d.nv + d.nc * d.nc;     // direct-set products per CTA
        o[3] = 2 * d.nv * d.nc > pd ? 2 * d.nv * d.nc : pd;
        o[4] = 2 * d.nb;
        o[5] = 1;
        o[6] = 1;
      }
      ++n;
    }
  }
  for (int i = 0; i < kNumVariants; ++i) {
    const Variant& v = kVariants[i];
    if (!valid_for(v, d)) continue;
    if (out && n < cap) {
      int* o = out + 7 * n;
      o[0] = i;
      o[1] = v.threads;
      o[2] = v.rows;
      o[3] = v.pmax;
      o[4] = v.bmax;
      o[5] = v.ppt;
      o[6] = v.merged ? 1 : 0;
    }
    ++n;
  }
  return n;
}

int pair_variant_current(const DevSys& d) {
  if (use_gcorr(d)) return gcorr_split(d) ? kGcorrSplitIndex : gcorr_pf(d) ? kGcorrPfIndex : kGcorrIndex;
  const Variant* v = pick(d);
  return v ? (int)(v - kVariants) : -1;
}

int launch_realspace(const DevSys& d, const void* coef, void* u, void* stream) {
  const Variant* v = pick(d);
  if (!v) return (int)cudaErrorInvalidValue;
  cudaFuncSetAttribute((const void*)v->rs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->rs_smem);
  v->rs<<<d.nkpt * d.nb, kThreads, v->rs_smem, (cudaStream_t)stream>>>(d, (const float2*)coef, (float2*)u);
  if (int e = (int)cudaGetLastError()) return e;
  return (int)cudaMemcpyAsync((char*)u + u_bytes(d), coef, (size_t)d.nkpt * d.nb * d.npw_max * 8,
                              cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
}

int launch_pair_exchange(const DevSys& d, const void* u, void* rho_x, int* status, void* stream) {
  if (use_gcorr(d)) return launch_gcorr(d, coef_copy(d, u), rho_x, 0, 0, 0, 0, 0, d.nkpt, gcorr_pf(d), stream);
  const Variant* v = pick(d);
  if (!v) return (int)cudaErrorInvalidValue;
  const size_t sm = v->pair_smem(d.ng_max);
  cudaFuncSetAttribute((const void*)v->pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  CUtensorMap tm;
  if (int e = make_tmap(d, v, u, &tm)) return e;
  v->pair<<<d.nkpt, v->threads, sm, (cudaStream_t)stream>>>(d, (const float2*)u, (float2*)rho_x, 0, 0, 0, 0, status, tm);
  return (int)cudaGetLastError();
}

static long long job_cells(const DevSys& d, int nqc, bool merged) {
  const long long ntk = (d.nkpt + kTK - 1) / kTK, ntq = (nqc + kTQ - 1) / kTQ;
  return ntq * ntk * kTQ * kTK * (merged ? 1 : 2);
}

int launch_pair_direct(const DevSys& d, const void* u, void* rho_dir, int q_begin, int q_end, long long vbase,
                       int* status, void* stream) {
  if (use_gcorr(d))
    return gcorr_split(d)
               ? launch_gcorr(d, coef_copy(d, u), rho_dir, 3, 1, q_begin, q_end - q_begin, vbase,
                              job_cells(d, q_end - q_begin, false), 0, stream)
               : launch_gcorr(d, coef_copy(d, u), rho_dir, 1, 1, q_begin, q_end - q_begin, vbase,
                              job_cells(d, q_end - q_begin, true), gcorr_pf(d), stream);
  const Variant* v = pick(d);
  if (!v) return (int)cudaErrorInvalidValue;
  const size_t sm = v->pair_smem(d.ng_max);
  cudaFuncSetAttribute((const void*)v->pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int nqc = q_end - q_begin;
  const long long ntk = (d.nkpt + kTK - 1) / kTK, ntq = (nqc + kTQ - 1) / kTQ;
  const long long cells = ntq * ntk * kTQ * kTK * (v->merged ? 1 : 2);
  if (cells >= (1LL << 31)) return (int)cudaErrorInvalidValue;
  CUtensorMap tm;
  if (int e = make_tmap(d, v, u, &tm)) return e;
  v->pair<<<(unsigned)cells, v->threads, sm, (cudaStream_t)stream>>>(d, (const float2*)u, (float2*)rho_dir, 1,
                                                                     q_begin, nqc, vbase, status, tm);
  return (int)cudaGetLastError();
}

// Coupling densities rho_vc'^{kk'} and rho_cv'^{kk'} of the upper blocks of [q_begin, q_end) (same
// job tiling as the direct set; nv^2 + nc^2 >= 2 nv nc, so every variant valid there fits these).
int launch_pair_coupling(const DevSys& d, const void* u, void* rho_cpl, int q_begin, int q_end, long long vbase,
                         int* status, void* stream) {
  if (use_gcorr(d))
    return launch_gcorr(d, coef_copy(d, u), rho_cpl, 2, 5, q_begin, q_end - q_begin, vbase,
                        job_cells(d, q_end - q_begin, true), gcorr_pf(d), stream);
  const Variant* v = pick(d);
  if (!v) return (int)cudaErrorInvalidValue;
  const size_t sm = v->pair_smem(d.ng_max);
  cudaFuncSetAttribute((const void*)v->pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int nqc = q_end - q_begin;
  const long long ntk = (d.nkpt + kTK - 1) / kTK, ntq = (nqc + kTQ - 1) / kTQ;
  const long long cells = ntq * ntk * kTQ * kTK * (v->merged ? 1 : 2);
  if (cells >= (1LL << 31)) return (int)cudaErrorInvalidValue;
  CUtensorMap tm;
  if (int e = make_tmap(d, v, u, &tm)) return e;
  v->pair<<<(unsigned)cells, v->threads, sm, (cudaStream_t)stream>>>(d, (const float2*)u, (float2*)rho_cpl, 5,
                                                                     q_begin, nqc, vbase, status, tm);
  return (int)cudaGetLastError();
}

// rho_vc^{k,k+q}(G) for every k and q in [q_begin, q_end): rows ((q - q_begin) Nk + k) Nv Nc + v Nc + c.
int launch_pair_chi0(const DevSys& d, const void* u, void* rho, int q_begin, int q_end, int* status, void* stream) {
  if (use_gcorr(d))
    return launch_gcorr(d, coef_copy(d, u), rho, 0, 4, q_begin, q_end - q_begin, 0,
                        (long long)(q_end - q_begin) * d.nkpt, gcorr_pf(d), stream);
  const Variant* v = pick(d);
  if (!v) return (int)cudaErrorInvalidValue;
  const size_t sm = v->pair_smem(d.ng_max);
  cudaFuncSetAttribute((const void*)v->pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const long long cells = (long long)(q_end - q_begin) * d.nkpt;
  if (cells >= (1LL << 31)) return (int)cudaErrorInvalidValue;
  CUtensorMap tm;
  if (int e = make_tmap(d, v, u, &tm)) return e;
  v->pair<<<(unsigned)cells, v->threads, sm, (cudaStream_t)stream>>>(d, (const float2*)u, (float2*)rho, 4, q_begin,
                                                                     q_end - q_begin, 0, status, tm);
  return (int)cudaGetLastError();
}

int launch_dipole(const DevSys& d, const void* coef, const double* energies, double gap_floor, void* P,
                  void* stream) {
  const int threads = 256;
  const long long blocks = ((long long)d.dim * 32 + threads - 1) / threads;
  dipole_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(d, (const float2*)coef, energies, gap_floor,
                                                                       (double2*)P);
  return (int)cudaGetLastError();
}

}  // namespace bse
