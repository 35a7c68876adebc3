// Haydock recursion and continued fraction (steps A7, A8), and Y = H X.
//
// The spectrum (Eq. epsilon_chi_bar in the TDA, Appendix A) is
//   eps_2(w) = -C Im[P^H (z - H)^{-1} P] = -C |P|^2 Im g(z),  z = w + i eta,
// with g the continued fraction of the Lanczos coefficients of H started at
// P/|P|.  Lanczos with classical Gram-Schmidt against the whole basis applied
// twice per step (FP64 basis and recurrence); the matrix-vector product reads
// H in FP32, multiplies in FP32 and combines 16-element partial sums in FP64.
//
// GB300's FP64 pipes are narrow, so the O(j dim) work of each step (projections and
// updates against the basis) runs in double-float arithmetic on the FP32 pipes: the basis
// is stored split (hi, lo) per component, products are made error-free with FMA and sums
// carried with TwoSum (about 46 significant bits, orthogonality ~1e-13), and the
// matrix-vector product keeps compensated FP32 partial sums.  Only O(dim) per step and
// the coefficient reductions use native FP64.
//
// One persistent cooperative launch runs every step.  Each CTA owns a
// contiguous slice of rows for the product, the projections and the updates,
// so the only global exchanges are the projection coefficients and two norms
// per step (bounded grid barriers; a wait that exceeds 2 s sets
// BSE_ERR_TIMEOUT in the plan status word and the kernel returns).
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace bse {
namespace {

constexpr int kThreads = 512, kWarps = kThreads / 32;
constexpr int kMaxGrid = 1024;
// Breakdown when b_{j+1} <= kBreakdownRel |H v_j|: the product reads the FP32 copy of v_j with FP32
// matrix entries, so a Krylov space that closes in exact arithmetic leaves a residual at the FP32
// rounding level (~1e-7 |H v_j|); genuine steps couple at O(0.1) of |H v_j|.
constexpr double kBreakdownRel = 1e-6;
constexpr int kXTile = 8192;          // columns of v_j staged in shared memory per pass (64 KB)
constexpr size_t kDynMax = 150 * 1024;   // dynamic shared memory budget: the rest stays L1 for the H stream

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Limit of one grid-barrier wait (ns); settable per device for failure-injection tests.
__device__ unsigned long long g_wait_limit_ns = 2000000000ull;

// Barrier over the gsize CTAs of one system's group, on a (count, generation) pair: arrivals are
// acquire-release atomics, the last arrival resets the count and releases the generation, the
// others poll it with acquire loads.  False if the wait timed out or another CTA already
// reported an error.
__device__ bool grid_barrier(unsigned* bar, int* status, unsigned gsize) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* gen = bar + 1;
    const unsigned g = ld_acquire(gen);
    const unsigned arrived = atom_add_acq_rel(bar, 1u);
    int good = 1;
    if (arrived == gsize - 1) {
      atomicExch(bar, 0u);
      red_add_release(gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      unsigned it = 0;
      while (ld_acquire(gen) == g) {
        if ((it++ & 31u) == 0) {             // the first poll and every 32nd: a zero limit expires at once
          if (*(volatile int*)status != 0) {
            good = 0;
            break;
          }
          if (globaltimer() - t0 >= g_wait_limit_ns) {
            atomicCAS(status, 0, (int)BSE_ERR_TIMEOUT);
            good = 0;
            break;
          }
        }
        __nanosleep(32);
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// x loaders of bse_apply_H: the FP64 inputs are read-only and rounded to FP32 on the fly.
__device__ __forceinline__ float4 load_x2(const double2* x, int i) {
  const double2 a = __ldg(x + 2 * i), b = __ldg(x + 2 * i + 1);
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}
__device__ __forceinline__ float2 load_x1(const double2* x, int i) {
  const double2 a = __ldg(x + i);
  return make_float2((float)a.x, (float)a.y);
}

// ---------------------------------------------------------------- double-float helpers
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// acc (hi, lo) += a * b with a, b given as (hi, lo); the error of the leading product is exact (FMA).
__device__ __forceinline__ void df_mac(float2& acc, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  float s, t;
  two_sum(acc.x, p, s, t);
  acc.x = s;
  acc.y += t + e;
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void df_add(float2& acc, float2 a) {
  float s, t;
  two_sum(acc.x, a.x, s, t);
  acc.x = s;
  acc.y += t + a.y;
}
__device__ __forceinline__ float2 df_norm(float2 a) {   // renormalise so |lo| <= ulp(hi)/2
  const float s = a.x + a.y;
  return make_float2(s, a.y - (s - a.x));
}
__device__ __forceinline__ float2 df_split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
// complex double-float element: (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ float4 cdf_split(double2 z) {
  const float2 r = df_split(z.x), i = df_split(z.y);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ double2 cdf_val(float4 z) {
  return make_double2(df_val(make_float2(z.x, z.y)), df_val(make_float2(z.z, z.w)));
}
__device__ __forceinline__ float4 df_shfl_xor(float4 v, int o) {
  return make_float4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
                     __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o));
}
__device__ __forceinline__ float4 cdf_warp_sum(float4 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float4 u = df_shfl_xor(v, o);
    float2 re = make_float2(v.x, v.y), im = make_float2(v.z, v.w);
    df_add(re, make_float2(u.x, u.y));
    df_add(im, make_float2(u.z, u.w));
    re = df_norm(re);
    im = df_norm(im);
    v = make_float4(re.x, re.y, im.x, im.y);
  }
  return v;
}

// Row dot  sum_c H[r][c] x[c]: FP32 products over 16 elements per lane, then carried
// in a compensated (hi, lo) FP32 sum; one FP64 combine per row.
template <typename XT>
__device__ __forceinline__ double2 row_dot(const float2* __restrict__ Hr, const XT* x, int dim, int lane) {
  float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
  auto carry = [&](float2 s) {
    df_add(ar, make_float2(s.x, 0.f));
    df_add(ai, make_float2(s.y, 0.f));
  };
  if ((dim & 1) == 0) {
    const float4* h4 = reinterpret_cast<const float4*>(Hr);
    const int n4 = dim >> 1;
    int i = lane;
    for (; i + 32 * 7 < n4; i += 32 * 8) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 h = __ldg(h4 + i + 32 * u);
        const float4 v = load_x2(x, i + 32 * u);
        s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
        s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
        s.x = fmaf(h.z, v.z, fmaf(-h.w, v.w, s.x));
        s.y = fmaf(h.z, v.w, fmaf(h.w, v.z, s.y));
      }
      carry(s);
    }
    float2 s = make_float2(0.f, 0.f);
    for (; i < n4; i += 32) {
      const float4 h = __ldg(h4 + i);
      const float4 v = load_x2(x, i);
      s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
      s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
      s.x = fmaf(h.z, v.z, fmaf(-h.w, v.w, s.x));
      s.y = fmaf(h.z, v.w, fmaf(h.w, v.z, s.y));
    }
    carry(s);
  } else {
    int i = lane;
    for (; i + 32 * 15 < dim; i += 32 * 16) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float2 h = __ldg(Hr + i + 32 * u);
        const float2 v = load_x1(x, i + 32 * u);
        s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
        s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
      }
      carry(s);
    }
    float2 s = make_float2(0.f, 0.f);
    for (; i < dim; i += 32) {
      const float2 h = __ldg(Hr + i);
      const float2 v = load_x1(x, i);
      s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
      s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
    }
    carry(s);
  }
  const float4 t = cdf_warp_sum(make_float4(ar.x, ar.y, ai.x, ai.y));
  return cdf_val(t);
}

// Segment dot over cols columns starting at Hr (row pointer already offset), x in shared memory.
// Returns the lane's compensated (re, im) partial (not warp-reduced).
__device__ __forceinline__ void seg_dot(const float2* __restrict__ Hr, const float2* xs, int cols, int lane,
                                        float2& ar, float2& ai) {
  auto carry = [&](float2 s) {
    df_add(ar, make_float2(s.x, 0.f));
    df_add(ai, make_float2(s.y, 0.f));
  };
  if ((reinterpret_cast<uintptr_t>(Hr) & 15) == 0) {      // float4 pairs, odd tail by lane 0
    const float4* h4 = reinterpret_cast<const float4*>(Hr);
    const float4* x4 = reinterpret_cast<const float4*>(xs);
    const int n4 = cols >> 1;
    int i = lane;
    for (; i + 32 * 15 < n4; i += 32 * 16) {
      float4 h[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) h[u] = __ldcs(h4 + i + 32 * u);
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float4 v = x4[i + 32 * u];
        s.x = fmaf(h[u].x, v.x, fmaf(-h[u].y, v.y, s.x));
        s.y = fmaf(h[u].x, v.y, fmaf(h[u].y, v.x, s.y));
        s.x = fmaf(h[u].z, v.z, fmaf(-h[u].w, v.w, s.x));
        s.y = fmaf(h[u].z, v.w, fmaf(h[u].w, v.z, s.y));
        if ((u & 7) == 7) {
          carry(s);
          s = make_float2(0.f, 0.f);
        }
      }
    }
    float2 s = make_float2(0.f, 0.f);
    int cnt = 0;
    for (; i < n4; i += 32) {
      const float4 h = __ldcs(h4 + i);
      const float4 v = x4[i];
      s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
      s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
      s.x = fmaf(h.z, v.z, fmaf(-h.w, v.w, s.x));
      s.y = fmaf(h.z, v.w, fmaf(h.w, v.z, s.y));
      if (++cnt == 8) {
        carry(s);
        s = make_float2(0.f, 0.f);
        cnt = 0;
      }
    }
    carry(s);
    if ((cols & 1) && lane == 0) {          // odd tail element
      const float2 h = __ldcs(Hr + cols - 1), v = xs[cols - 1];
      carry(make_float2(h.x * v.x - h.y * v.y, h.x * v.y + h.y * v.x));
    }
  } else {
    float2 s = make_float2(0.f, 0.f);
    int cnt = 0;
    for (int i = lane; i < cols; i += 32) {
      const float2 h = __ldcs(Hr + i), v = xs[i];
      s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
      s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
      if (++cnt == 16) {
        carry(s);
        s = make_float2(0.f, 0.f);
        cnt = 0;
      }
    }
    carry(s);
  }
}

struct HayArgs {
  int dim;
  double prefactor;
  int cta0, ncta;   // this system's CTA group inside the launch
  int grank, gsize; // filled per CTA: rank in the group, group size
  const float2* H;
  const double2* P;
  int nsteps;
  const double* omega;
  int nw;
  double eta;
  double* eps2;
  double* ab;
  int* steps_done;
  float4* V;        // [nsteps][dim] basis, double-float split (re.hi, re.lo, im.hi, im.lo)
  float2* vf;       // [dim] FP32 copy of the current basis vector
  double2* hpart;   // [grid][nsteps] per-CTA projection partials
  double2* h1;      // [nsteps]
  double2* h2;      // [nsteps]
  double* npart;    // [grid][2]
  unsigned* bar;    // [2]
  int* status;
};

// hpart[cta][i] = sum over own rows conj(V[i][r]) w[r], i in [0, n) (double-float products).
// One thread per basis vector walks the CTA's rows with independent, unrolled loads (the rows of
// V owned by a CTA are written and read by that CTA only, so plain cached loads are coherent).
// This CTA's rows of basis vector i: the shared copy for i < vsk (row stride vrows), else global.
struct BasisRows {
  const float4* sm;     // [vsk][vrows]
  const float4* gl;     // V + row0, row stride dim
  int vsk, vrows, dim;
  __device__ __forceinline__ const float4* row(int i) const {
    return i < vsk ? sm + (size_t)i * vrows : gl + (size_t)i * dim;
  }
};

__device__ void project_partial(const HayArgs& A, const BasisRows& Vb, const float4* wsm, int nrows, int n) {
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const float4* Vi = Vb.row(i);
    float2 sr[4], si[4];                    // four independent chains (rows mod 4) hide the add latency
#pragma unroll
    for (int u = 0; u < 4; ++u) sr[u] = si[u] = make_float2(0.f, 0.f);
    auto mac = [&](float2& ar, float2& ai, float4 v, float4 w) {
      const float2 vr = make_float2(v.x, v.y), vi = make_float2(v.z, v.w);
      const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
      // conj(v) w = (vr wr + vi wi) + i (vr wi - vi wr)
      df_mac(ar, vr, wr);
      df_mac(ar, vi, wi);
      df_mac(ai, vr, wi);
      df_mac(ai, df_neg(vi), wr);
    };
    int r = 0;
    for (; r + 4 <= nrows; r += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = Vi[r + u];
#pragma unroll
      for (int u = 0; u < 4; ++u) mac(sr[u], si[u], v[u], wsm[r + u]);
    }
    for (; r < nrows; ++r) mac(sr[0], si[0], Vi[r], wsm[r]);
#pragma unroll
    for (int u = 1; u < 4; ++u) {
      df_add(sr[0], sr[u]);
      df_add(si[0], si[u]);
    }
    A.hpart[(size_t)A.grank * A.nsteps + i] = cdf_val(make_float4(sr[0].x, sr[0].y, si[0].x, si[0].y));
  }
}

// h[i] = sum_cta hpart[cta][i] for the i owned by this CTA (deterministic order, FP64).
__device__ void reduce_coeffs(const HayArgs& A, double2* h, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = A.grank + A.gsize * warp; i < n; i += A.gsize * kWarps) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = lane; c < A.gsize; c += 32) {
      const double2 v = __ldcg(A.hpart + (size_t)c * A.nsteps + i);
      s.x += v.x;
      s.y += v.y;
    }
    s = warp_sum(s);
    if (lane == 0) h[i] = s;
  }
}

// w[r] -= sum_i V[i][r] h[i] over own rows.  Threads are (vector group, row) with rows fastest:
// each sums every ng-th basis vector for its row with independent, unrolled loads, then the
// ng partials of a row are added in a fixed order.  h is staged split (hi, lo) in hs.
__device__ void subtract_projection(const BasisRows& Vb, float4* wsm, float4* red, float4* hs, const double2* h,
                                    int nrows, int n) {
  for (int i = threadIdx.x; i < n; i += kThreads) hs[i] = cdf_split(__ldcg(h + i));
  __syncthreads();
  for (int rb = 0; rb < nrows; rb += kThreads) {
    const int nr = min(nrows - rb, kThreads);
    const int ng = kThreads / nr;
    const int r = threadIdx.x % nr, ig = threadIdx.x / nr;
    if (ig < ng) {
      float2 sr[4], si[4];                  // four independent chains
#pragma unroll
      for (int u = 0; u < 4; ++u) sr[u] = si[u] = make_float2(0.f, 0.f);
      auto mac = [&](float2& ar, float2& ai, float4 v, float4 c) {
        const float2 vr = make_float2(v.x, v.y), vi = make_float2(v.z, v.w);
        const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
        // v c = (vr cr - vi ci) + i (vr ci + vi cr)
        df_mac(ar, vr, cr);
        df_mac(ar, df_neg(vi), ci);
        df_mac(ai, vr, ci);
        df_mac(ai, vi, cr);
      };
      const int rr = rb + r;
      int i = ig;
      for (; i + 3 * ng < n; i += 4 * ng) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = Vb.row(i + u * ng)[rr];
#pragma unroll
        for (int u = 0; u < 4; ++u) mac(sr[u], si[u], v[u], hs[i + u * ng]);
      }
      for (; i < n; i += ng) mac(sr[0], si[0], Vb.row(i)[rr], hs[i]);
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        df_add(sr[0], sr[u]);
        df_add(si[0], si[u]);
      }
      red[ig * nr + r] = make_float4(sr[0].x, sr[0].y, si[0].x, si[0].y);
    }
    __syncthreads();
    if (threadIdx.x < nr) {
      float2 tr = make_float2(0.f, 0.f), ti = make_float2(0.f, 0.f);
      for (int q = 0; q < ng; ++q) {
        const float4 t = red[q * nr + threadIdx.x];
        df_add(tr, make_float2(t.x, t.y));
        df_add(ti, make_float2(t.z, t.w));
      }
      const float4 w = wsm[rb + threadIdx.x];
      float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
      df_add(wr, df_neg(tr));
      df_add(wi, df_neg(ti));
      wr = df_norm(wr);
      wi = df_norm(wi);
      wsm[rb + threadIdx.x] = make_float4(wr.x, wr.y, wi.x, wi.y);
    }
    __syncthreads();
  }
}

__device__ double block_sum(double v, double* red1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red1[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kWarps; ++q) t += red1[q];
  return t;    // valid in thread 0
}

// sum over CTAs of npart[c][which], identical order in every CTA.
__device__ double all_cta_sum(const HayArgs& A, int which, double* red1) {
  double v = 0.0;
  for (int c = threadIdx.x; c < A.gsize; c += kThreads) v += __ldcg(A.npart + 2 * c + which);
  double t = block_sum(v, red1);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = t;
  __syncthreads();
  return bc;
}

// both sums of npart[c][0] and npart[c][1] in one pass by warp 0 (identical order in every CTA)
__device__ double2 all_cta_sum2(const HayArgs& A, double2* red2) {
  if (threadIdx.x < 32) {
    double2 v = make_double2(0.0, 0.0);
    for (int c = threadIdx.x; c < A.gsize; c += 32) {
      const double2 p = __ldcg(reinterpret_cast<const double2*>(A.npart) + c);
      v.x += p.x;
      v.y += p.y;
    }
    v = warp_sum(v);
    if (threadIdx.x == 0) red2[0] = v;
  }
  __syncthreads();
  const double2 t = red2[0];
  __syncthreads();
  return t;
}

constexpr int kMaxBatch = 24;

// One system of a batched launch (pointers into that system's workspace).
struct HaySys {
  int dim, cta0, ncta;
  double prefactor;
  const float2* H;
  const double2* P;
  double* eps2;
  double* ab;
  int* steps_done;
  float4* V;
  float2* vf;
  double2* hpart;
  double2* h1;
  double2* h2;
  double* npart;
  unsigned* bar;
};

struct HayBatch {
  int nsys, nsteps, nw, rows_max;   // rows_max: largest rows-per-CTA over the systems
  int xtile;                        // columns of v_j staged per pass
  int vsk;                          // basis vectors whose own rows are kept in shared memory
  double eta;
  const double* omega;
  int* status;
  HaySys s[kMaxBatch];
};

// The CTA's rows of the first B.vsk basis vectors also live in shared memory (they are read only by
// this CTA), so most projections and updates read shared memory; the global copy serves the rest
// and the adjoint.
__global__ __launch_bounds__(kThreads, 1) void haydock_kernel(const __grid_constant__ HayBatch B) {
  int g = 0;
  while (g + 1 < B.nsys && (int)blockIdx.x >= B.s[g + 1].cta0) ++g;
  const HaySys& S = B.s[g];
  HayArgs A;
  A.dim = S.dim;
  A.prefactor = S.prefactor;
  A.cta0 = S.cta0;
  A.ncta = S.ncta;
  A.grank = (int)blockIdx.x - S.cta0;
  A.gsize = S.ncta;
  A.H = S.H;
  A.P = S.P;
  A.nsteps = B.nsteps;
  A.omega = B.omega;
  A.nw = B.nw;
  A.eta = B.eta;
  A.eps2 = S.eps2;
  A.ab = S.ab;
  A.steps_done = S.steps_done;
  A.V = S.V;
  A.vf = S.vf;
  A.hpart = S.hpart;
  A.h1 = S.h1;
  A.h2 = S.h2;
  A.npart = S.npart;
  A.bar = S.bar;
  A.status = B.status;
  extern __shared__ float4 dyn[];
  float4* wsm = dyn;                                // own rows of w (double-float)
  float4* hs = dyn + B.rows_max;                    // projection coefficients (double-float)
  float2* xs = reinterpret_cast<float2*>(hs + B.nsteps);   // column tile of v_j (FP32)
  float4* vsm = reinterpret_cast<float4*>(xs + B.xtile);   // [vsk][rows_max] own rows of the first basis vectors
  if (B.vsk > 0 && (reinterpret_cast<uintptr_t>(vsm) & 15) != 0) {   // float4 rows must be 16-byte aligned
    if (threadIdx.x == 0) atomicCAS(B.status, 0, (int)BSE_ERR_CUDA);
    return;
  }
  __shared__ float4 red[kThreads];
  __shared__ double red1[kWarps];
  const int dim = A.dim;
  const int rows_per = (dim + A.gsize - 1) / A.gsize;
  const int row0 = min(dim, A.grank * rows_per);
  const int nrows = min(dim, row0 + rows_per) - row0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // v_0 = P / |P|
  double pp = 0.0;
  for (int r = threadIdx.x; r < nrows; r += kThreads) {
    const double2 p = A.P[row0 + r];
    pp += p.x * p.x + p.y * p.y;
  }
  pp = block_sum(pp, red1);
  if (threadIdx.x == 0) A.npart[2 * A.grank] = pp;
  if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
  const double pn2 = all_cta_sum(A, 0, red1);
  const double pinv = 1.0 / sqrt(pn2);
  for (int r = threadIdx.x; r < nrows; r += kThreads) {
    const double2 p = A.P[row0 + r];
    const double2 v = make_double2(p.x * pinv, p.y * pinv);
    A.V[row0 + r] = cdf_split(v);
    if (B.vsk > 0) vsm[r] = cdf_split(v);
    A.vf[row0 + r] = make_float2((float)v.x, (float)v.y);
  }
  const BasisRows Vb{vsm, A.V + row0, B.vsk, B.rows_max, dim};
  if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;

  int done = A.nsteps;
  float vscale = 1.0f;                      // vf holds v_j / vscale: w_j unnormalised, scaled when staged
  for (int j = 0; j < A.nsteps; ++j) {
    // w = H v_j on own rows: v_j staged in shared memory in column tiles, H streamed once
    for (int r = threadIdx.x; r < nrows; r += kThreads) wsm[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int col0 = 0; col0 < dim; col0 += B.xtile) {
      const int cols = min(B.xtile, dim - col0);
      __syncthreads();
      for (int c = threadIdx.x; c < cols; c += kThreads) {
        const float2 x = __ldcg(A.vf + col0 + c);
        xs[c] = make_float2(x.x * vscale, x.y * vscale);
      }
      __syncthreads();
      for (int r = warp; r < nrows; r += kWarps) {
        float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
        seg_dot(A.H + (size_t)(row0 + r) * dim + col0, xs, cols, lane, ar, ai);
        const float4 t = cdf_warp_sum(make_float4(ar.x, ar.y, ai.x, ai.y));
        if (lane == 0) {
          const float4 o = wsm[r];
          float2 re = make_float2(o.x, o.y), im = make_float2(o.z, o.w);
          df_add(re, make_float2(t.x, t.y));
          df_add(im, make_float2(t.z, t.w));
          re = df_norm(re);
          im = df_norm(im);
          wsm[r] = make_float4(re.x, re.y, im.x, im.y);
        }
      }
    }
    __syncthreads();
    if (warp == 0) {                        // |H v_j|^2 only sets the breakdown threshold: FP32, one warp
      float hv2 = 0.f;
      for (int r = lane; r < nrows; r += 32) {
        const float4 w = wsm[r];
        hv2 += w.x * w.x + w.z * w.z;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hv2 += __shfl_xor_sync(0xffffffffu, hv2, o);
      if (lane == 0) A.npart[2 * A.grank + 1] = hv2;
    }
    project_partial(A, Vb, wsm, nrows, j + 1);
    if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
    reduce_coeffs(A, A.h1, j + 1);
    if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
    subtract_projection(Vb, wsm, red, hs, A.h1, nrows, j + 1);
    project_partial(A, Vb, wsm, nrows, j + 1);
    if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
    reduce_coeffs(A, A.h2, j + 1);
    if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
    subtract_projection(Vb, wsm, red, hs, A.h2, nrows, j + 1);
    for (int r = threadIdx.x; r < nrows; r += kThreads) {     // published unnormalised
      const float4 w = wsm[r];
      A.vf[row0 + r] = make_float2(w.x + w.y, w.z + w.w);
    }
    if (warp == 0) {                        // |w|^2 of own rows in FP64 by one warp (FP64 issues slowly)
      double ww = 0.0;
      for (int r = lane; r < nrows; r += 32) {
        const double2 w = cdf_val(wsm[r]);
        ww += w.x * w.x + w.y * w.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ww += __shfl_xor_sync(0xffffffffu, ww, o);
      if (lane == 0) A.npart[2 * A.grank] = ww;
    }
    if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
    const double2 sums = all_cta_sum2(A, reinterpret_cast<double2*>(red));
    const double bn2 = sums.x, sc2 = sums.y;
    const double2 c1 = __ldcg(A.h1 + j), c2 = __ldcg(A.h2 + j);
    const double aj = c1.x + c2.x;
    const double bn = sqrt(bn2);
    const bool last = (j + 1 == A.nsteps);
    const bool brk = !last && !(bn > kBreakdownRel * sqrt(sc2));
    if (A.grank == 0 && threadIdx.x == 0) {
      A.ab[j] = aj;
      if (j == 0) A.ab[A.nsteps] = 0.0;
      if (!last) A.ab[A.nsteps + j + 1] = brk ? 0.0 : bn;
    }
    if (last) break;
    if (brk) {
      done = j + 1;
      break;
    }
    const double binv = 1.0 / bn;
    float4* Vn = A.V + (size_t)(j + 1) * dim + row0;   // own rows only: no grid barrier needed
    for (int r = threadIdx.x; r < nrows; r += kThreads) {
      const double2 w = cdf_val(wsm[r]);
      const float4 v = cdf_split(make_double2(w.x * binv, w.y * binv));
      Vn[r] = v;
      if (j + 1 < B.vsk) vsm[(size_t)(j + 1) * B.rows_max + r] = v;
    }
    vscale = (float)binv;
  }
  if (!grid_barrier(A.bar, A.status, (unsigned)A.gsize)) return;
  if (A.grank == 0 && threadIdx.x == 0) *A.steps_done = done;
  // continued fraction from the bottom: g = 1/(z - a_j - b_{j+1}^2 g)
  const double C = A.prefactor * pn2;
  for (int wi = A.grank * kThreads + threadIdx.x; wi < A.nw; wi += A.gsize * kThreads) {
    const double zr = A.omega[wi], zi = A.eta;
    double gr = 0.0, gi = 0.0;
    for (int jj = done - 1; jj >= 0; --jj) {
      const double a = __ldcg(A.ab + jj);
      double dr = zr - a, di = zi;
      if (jj + 1 < done) {
        const double b = __ldcg(A.ab + A.nsteps + jj + 1);
        dr -= b * b * gr;
        di -= b * b * gi;
      }
      const double den = dr * dr + di * di;
      gr = dr / den;
      gi = -di / den;
    }
    A.eps2[wi] = -C * gi;
  }
}

// Y[v] = H X[v]: warp per (row, vector); FP32 products, FP64 combine.
__global__ void apply_h_kernel(DevSys d, const float2* __restrict__ H, const double2* __restrict__ X,
                               double2* __restrict__ Y, int nvec) {
  const int dim = d.dim;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)dim * nvec) return;
  const int v = (int)(warp / dim), r = (int)(warp % dim);
  const double2 s = row_dot(H + (size_t)r * dim, X + (size_t)v * dim, dim, lane);
  if (lane == 0) Y[(size_t)v * dim + r] = s;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SpecLayout {
  size_t V, vf, hpart, h1, h2, npart, bar, total;
};

SpecLayout spec_layout(const DevSys& d, long long nsteps) {
  SpecLayout L;
  size_t o = 0;
  L.V = o; o = align256(o + (size_t)nsteps * d.dim * sizeof(double2));
  L.vf = o; o = align256(o + (size_t)d.dim * sizeof(float2));
  L.hpart = o; o = align256(o + (size_t)kMaxGrid * nsteps * sizeof(double2));
  L.h1 = o; o = align256(o + (size_t)nsteps * sizeof(double2));
  L.h2 = o; o = align256(o + (size_t)nsteps * sizeof(double2));
  L.npart = o; o = align256(o + (size_t)kMaxGrid * 2 * sizeof(double));
  L.bar = o; o = align256(o + 2 * sizeof(unsigned));
  L.total = o;
  return L;
}

}  // namespace

size_t spectrum_ws_bytes(const DevSys& d, long long nsteps) { return spec_layout(d, nsteps).total; }

// Launch the recursion for n systems in one cooperative grid of one CTA per SM; each system
// gets a CTA group sized by its H bytes (at least one CTA) and its own workspace.
int run_haydock_batch(const HayJob* jobs, int n, int nsteps, const double* omega, int nw, double eta, int* status,
                      void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (n < 1 || n > kMaxBatch) return -2;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = sms < kMaxGrid ? sms : kMaxGrid;
  if (n > grid) return -2;
  double tot = 0.0;
  for (int i = 0; i < n; ++i) tot += (double)jobs[i].d->dim * jobs[i].d->dim;
  int ncta[kMaxBatch];
  int used = 0, big = 0;
  for (int i = 0; i < n; ++i) {
    const double share = (double)jobs[i].d->dim * jobs[i].d->dim / tot;
    ncta[i] = 1 + (int)(share * (grid - n));
    used += ncta[i];
    if (jobs[i].d->dim > jobs[big].d->dim) big = i;
  }
  ncta[big] += grid - used;
  HayBatch B;
  B.nsys = n;
  B.nsteps = nsteps;
  B.nw = nw;
  B.eta = eta;
  B.omega = omega;
  B.status = status;
  B.rows_max = 0;
  int cta = 0;
  for (int i = 0; i < n; ++i) {
    const DevSys& d = *jobs[i].d;
    const SpecLayout L = spec_layout(d, nsteps);
    char* base = (char*)jobs[i].ws;
    HaySys& S = B.s[i];
    S.dim = d.dim;
    S.prefactor = d.prefactor;
    S.cta0 = cta;
    S.ncta = ncta[i];
    cta += ncta[i];
    S.H = (const float2*)jobs[i].H;
    S.P = (const double2*)jobs[i].P;
    S.eps2 = jobs[i].eps2;
    S.ab = jobs[i].ab;
    S.steps_done = jobs[i].steps_done;
    S.V = (float4*)(base + L.V);
    S.vf = (float2*)(base + L.vf);
    S.hpart = (double2*)(base + L.hpart);
    S.h1 = (double2*)(base + L.h1);
    S.h2 = (double2*)(base + L.h2);
    S.npart = (double*)(base + L.npart);
    S.bar = (unsigned*)(base + L.bar);
    const int rows = (d.dim + ncta[i] - 1) / ncta[i];
    if (rows > B.rows_max) B.rows_max = rows;
    const int e = (int)cudaMemsetAsync(S.bar, 0, 2 * sizeof(unsigned), st);
    if (e) return e;
  }
  // x tile of up to 8192 columns, then as many basis vectors' own rows in shared memory as fit
  int dim_max = 0;
  for (int i = 0; i < n; ++i) dim_max = jobs[i].d->dim > dim_max ? jobs[i].d->dim : dim_max;
  B.xtile = dim_max < kXTile ? (dim_max + 1) / 2 * 2 : kXTile;   // even: the basis rows after it stay 16-byte aligned
  const size_t fixed = ((size_t)B.rows_max + (size_t)nsteps) * sizeof(float4) + (size_t)B.xtile * sizeof(float2);
  if (fixed > kDynMax || fixed % sizeof(float4) != 0) return -1;
  const size_t per_vec = (size_t)B.rows_max * sizeof(float4);
  const size_t fit = (kDynMax - fixed) / per_vec;
  B.vsk = (int)(fit < (size_t)nsteps ? fit : (size_t)nsteps);
  const size_t dyn = fixed + (size_t)B.vsk * per_vec;
  cudaFuncSetAttribute((const void*)haydock_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, haydock_kernel, kThreads, dyn);
  if (occ < 1) return -1;
  void* args[] = {&B};
  return (int)cudaLaunchCooperativeKernel((const void*)haydock_kernel, dim3(grid), dim3(kThreads), args, dyn, st);
}

int set_wait_limit(unsigned long long ns) { return (int)cudaMemcpyToSymbol(g_wait_limit_ns, &ns, sizeof(ns)); }

// Shared with the adjoint: one system into a caller-laid-out workspace.
int run_haydock(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw, double eta,
                double* eps2, double* ab, int* steps_done, void* ws, int* status, void* stream, float4** V_out) {
  HayJob j{&d, H, P, eps2, ab, steps_done, ws};
  if (V_out) *V_out = (float4*)((char*)ws + spec_layout(d, nsteps).V);
  return run_haydock_batch(&j, 1, nsteps, omega, nw, eta, status, stream);
}

int launch_spectrum(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw,
                    double eta, double* eps2, double* ab, int* steps_done, void* ws, int* status, void* stream) {
  return run_haydock(d, H, P, nsteps, omega, nw, eta, eps2, ab, steps_done, ws, status, stream, nullptr);
}

// ---------------------------------------------------------------------------
// Spectrum with library-owned scratch, for callers that cannot allocate device
// memory themselves.  The scratch is one file-scope device array of fixed size;
// every device that loads this library holds it until the process exits.  Host
// code may not pass the array's name to a kernel (in host code it is only a
// stand-in for the symbol), so its device address is looked up with
// cudaGetSymbolAddress on every call made outside stream capture (a module
// reloaded after cudaDeviceReset gets a fresh address) and cached per device for
// calls made while the stream is being captured.  All calls share the array:
// calls that overlap on the GPU race on it.
namespace {
constexpr size_t kStaticScratchBytes = size_t(48) << 20;
static __device__ __align__(256) unsigned char g_spectrum_scratch[kStaticScratchBytes];
constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;
}  // namespace

size_t spectrum_static_capacity() { return kStaticScratchBytes; }

int launch_spectrum_static(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw,
                           double eta, double* eps2, double* ab, int* steps_done, int* status, void* stream) {
  int dev = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  e = (int)cudaStreamIsCapturing((cudaStream_t)stream, &capture);
  if (e) return e;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (capture == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
      void* p = nullptr;
      e = (int)cudaGetSymbolAddress(&p, g_spectrum_scratch);
      if (e) return e;
      g_scratch_addr[dev] = p;
    }
    ws = g_scratch_addr[dev];
  }
  // The barrier words are cleared by run_haydock before the launch; every other
  // scratch word is written before it is read.
  return run_haydock(d, H, P, nsteps, omega, nw, eta, eps2, ab, steps_done, ws, status, stream, nullptr);
}

int launch_apply_h(const DevSys& d, const void* H, const void* X, void* Y, int nvec, void* stream) {
  const long long warps = (long long)d.dim * nvec;
  apply_h_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d, (const float2*)H, (const double2*)X, (double2*)Y, nvec);
  return (int)cudaGetLastError();
}

}  // namespace bse
