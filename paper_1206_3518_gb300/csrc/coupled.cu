// Spectrum of the BSE with e-h / h-e coupling (Appendix A, beyond the Tamm-Dancoff approximation).
//
// In the basis (e-h, h-e) the two-particle Hamiltonian is H2 = [[A, B], [-conj B, -conj A]]; with
// F = diag(1, -1), M = F H2 = [[A, B], [conj B, conj A]] is Hermitian and, for a stable system,
// positive definite, and H2 is self-adjoint in <x, y>_M = x^H M y.  Eqs. Dyson_eh_rearrange and
// epsilon_chi_bar give
//     eps_2(w) = -C Im[Pt^H (z - H2)^{-1} F Pt],  Pt = (P, -conj P),  z = w + i eta.
// With s = F Pt = (P, conj P), Pt^H F Pt = 0 turns the M-inner-product resolvent of s into
// <s, (z - H2)^{-1} s>_M = z Pt^H (z - H2)^{-1} F Pt, so eps_2 = -C |s|_M^2 Im[g(z)/z] where g is the
// continued fraction of a Lanczos recursion on H2 in the M inner product started from s.
//
// The antiunitary swap Sigma(x, y) = (conj y, conj x) anticommutes with H2 and fixes s.  The Lanczos
// vectors are therefore Sigma-even and Sigma-odd in turn, q_j = (x_j, sigma_j conj x_j) with
// sigma_j = (-1)^j, every diagonal coefficient a_j vanishes, and H2 q_j = (t_j, -sigma_j conj t_j) with
// t_j = A x_j + sigma_j B conj(x_j).  Only the top halves x_j are stored and iterated:
//     |q|_M^2 = 2 Re(x^H t),   <q_i, w>_M = d + sigma_i sigma conj(d),  d = p_i^H y  (p_i = t_i / b_i),
// i.e. 2 Re d for q_i of the parity of w and 2i Im d for the other parity; either correction
// w -= <q_i, w>_M q_i keeps the parity of w.  Each new residual is reorthogonalised (classical
// Gram-Schmidt, twice) against every stored vector: the overlaps with the other parity vanish in exact
// arithmetic but not in rounding.
//
// One step j = one read of A and B:
//   mv      t = A fl32(w_j) + sigma_j B conj(fl32(w_j)); partial sums of 2 Re(w_j^H t) per CTA
//   update  beta_j^2 (each CTA sums the partials in the same order), breakdown test, b_j = beta_j,
//           q_j = w_j / b_j, p_j = t / b_j, w_{j+1} = p_j - b_j q_{j-1}; partial projections of
//           w_{j+1} on every p_i, i <= j, per CTA range
//   reduce  the partials of all CTAs into <q_i, w>_M (one warp per i)
//   reorth  w -= sum_i c_i q_i and the second partial projections; reduce; w -= sum_i c'_i q_i, fl32(w)
// No kernel waits for another CTA: the kernels of a step are ordered by the stream, so the whole
// recursion is capturable in a CUDA graph.  q_j, w, b_j and the cross-CTA sums are FP64; the stored basis
// (q_i, p_i), the matrix-vector product and the per-CTA projection sums (corrections of rounding size)
// are FP32.
#include <cuda_runtime.h>

#include "internal.h"

namespace bse {
namespace {

constexpr int kMvThreads = 256, kNseg = 4, kMaxRows = 64, kMaxMv = 1024;
constexpr int kVecThreads = 256, kVecWarps = kVecThreads / 32, kMaxL = 256, kMaxVec = 1024;
constexpr double kBreakdownRel = 1e-6;     // |w_j|_M <= 1e-6 |H2 q_{j-1}|_M (FP32 product rounding ~1e-7)

struct CplWs {
  float2* Q32;      // [nsteps][dim] fl32(q_j)
  float2* P32;      // [nsteps][dim] fl32(p_j), p_j = top half of H2 q_j
  double2* w;       // [dim] residual / next vector (FP64)
  double2* qd;      // [2][dim] q_j, q_{j-1} (FP64)
  float2* t;        // [dim] product of the current step
  float2* x32;      // [dim] fl32(w), the product's input
  double* mvpart;   // [kMaxMv] partial 2 Re(w^H t) per product CTA
  float2* ppart;    // [nsteps][kMaxVec] partial p_i^H w per vector CTA
  double2* c;       // [2][nsteps] M-inner products <q_i, w>_M of pass 1 and pass 2
  int* ctl;         // [0] done, [1] steps
};

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

CplWs carve(void* base, int dim, int nsteps) {
  char* p = (char*)base;
  CplWs w;
  size_t o = 0;
  w.Q32 = (float2*)(p + o); o = al256(o + (size_t)nsteps * dim * sizeof(float2));
  w.P32 = (float2*)(p + o); o = al256(o + (size_t)nsteps * dim * sizeof(float2));
  w.w = (double2*)(p + o); o = al256(o + (size_t)dim * sizeof(double2));
  w.qd = (double2*)(p + o); o = al256(o + 2 * (size_t)dim * sizeof(double2));
  w.t = (float2*)(p + o); o = al256(o + (size_t)dim * sizeof(float2));
  w.x32 = (float2*)(p + o); o = al256(o + (size_t)dim * sizeof(float2));
  w.mvpart = (double*)(p + o); o = al256(o + kMaxMv * sizeof(double));
  w.ppart = (float2*)(p + o); o = al256(o + (size_t)kMaxVec * nsteps * sizeof(float2));
  w.c = (double2*)(p + o); o = al256(o + 2 * (size_t)nsteps * sizeof(double2));
  w.ctl = (int*)(p + o); o = al256(o + 4 * sizeof(int));
  return w;
}

size_t carve_bytes(int dim, int nsteps) {
  size_t o = 0;
  o = al256(o + (size_t)nsteps * dim * sizeof(float2));
  o = al256(o + (size_t)nsteps * dim * sizeof(float2));
  o = al256(o + (size_t)dim * sizeof(double2));
  o = al256(o + 2 * (size_t)dim * sizeof(double2));
  o = al256(o + (size_t)dim * sizeof(float2));
  o = al256(o + (size_t)dim * sizeof(float2));
  o = al256(o + kMaxMv * sizeof(double));
  o = al256(o + (size_t)kMaxVec * nsteps * sizeof(float2));
  o = al256(o + 2 * (size_t)nsteps * sizeof(double2));
  o = al256(o + 4 * sizeof(int));
  return o;
}

__device__ __forceinline__ bool finished(const CplWs& ws) { return *(volatile const int*)ws.ctl != 0; }

__device__ __forceinline__ void range_of(int dim, int& r0, int& r1) {
  r0 = (int)((long long)blockIdx.x * dim / gridDim.x);
  r1 = (int)((long long)(blockIdx.x + 1) * dim / gridDim.x);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc += a x + s b conj(x)
__device__ __forceinline__ void mac2(float2& acc, float ax, float ay, float bx, float by, float xx, float xy, float s) {
  acc.x = fmaf(ax, xx, fmaf(-ay, xy, acc.x));
  acc.y = fmaf(ax, xy, fmaf(ay, xx, acc.y));
  acc.x = fmaf(s * bx, xx, fmaf(s * by, xy, acc.x));
  acc.y = fmaf(s * by, xx, fmaf(-s * bx, xy, acc.y));
}

__global__ void start_kernel(int dim, const double2* __restrict__ P, CplWs ws, double* __restrict__ b, int nsteps) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += stride) {
    const double2 p = P[r];
    ws.w[r] = p;
    ws.x32[r] = make_float2((float)p.x, (float)p.y);
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsteps; j += stride) b[j] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ws.ctl[0] = 0;
    ws.ctl[1] = nsteps;
  }
}

// t = A x + s B conj(x) over this CTA's rows; rows in pairs, columns in kNseg segments, one warp per
// (pair, segment) unit; A and B are streamed once (evict-first loads), x is read through L1.
template <bool VEC>
__global__ __launch_bounds__(kMvThreads) void mv_kernel(int dim, const float2* __restrict__ A,
                                                        const float2* __restrict__ Bm, float s, CplWs ws) {
  if (finished(ws)) return;
  __shared__ float2 red[kMaxRows][kNseg];
  __shared__ double wsum[kMvThreads / 32];
  int r0, r1;
  range_of(dim, r0, r1);
  const int nr = r1 - r0, np = (nr + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int E = VEC ? 2 : 1;
  const int nvec = dim / E;
  for (int u = warp; u < np * kNseg; u += kMvThreads / 32) {
    const int pr = u / kNseg, seg = u - pr * kNseg;
    const int ra = r0 + 2 * pr;
    const bool hb = ra + 1 < r1;
    const int rb = hb ? ra + 1 : ra;
    const int v0 = (int)((long long)seg * nvec / kNseg), v1 = (int)((long long)(seg + 1) * nvec / kNseg);
    float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
    if (VEC) {
      const float4* Aa = reinterpret_cast<const float4*>(A + (size_t)ra * dim);
      const float4* Ab = reinterpret_cast<const float4*>(A + (size_t)rb * dim);
      const float4* Ba = reinterpret_cast<const float4*>(Bm + (size_t)ra * dim);
      const float4* Bb = reinterpret_cast<const float4*>(Bm + (size_t)rb * dim);
      const float4* X = reinterpret_cast<const float4*>(ws.x32);
#pragma unroll 4
      for (int v = v0 + lane; v < v1; v += 32) {
        const float4 aa = __ldcs(Aa + v), ab = __ldcs(Ab + v), ba = __ldcs(Ba + v), bb = __ldcs(Bb + v);
        const float4 x = __ldg(X + v);
        mac2(sa, aa.x, aa.y, ba.x, ba.y, x.x, x.y, s);
        mac2(sa, aa.z, aa.w, ba.z, ba.w, x.z, x.w, s);
        mac2(sb, ab.x, ab.y, bb.x, bb.y, x.x, x.y, s);
        mac2(sb, ab.z, ab.w, bb.z, bb.w, x.z, x.w, s);
      }
    } else {
      const float2* Aa = A + (size_t)ra * dim;
      const float2* Ab = A + (size_t)rb * dim;
      const float2* Ba = Bm + (size_t)ra * dim;
      const float2* Bb = Bm + (size_t)rb * dim;
#pragma unroll 4
      for (int v = v0 + lane; v < v1; v += 32) {
        const float2 aa = __ldcs(Aa + v), ab = __ldcs(Ab + v), ba = __ldcs(Ba + v), bb = __ldcs(Bb + v);
        const float2 x = __ldg(ws.x32 + v);
        mac2(sa, aa.x, aa.y, ba.x, ba.y, x.x, x.y, s);
        mac2(sb, ab.x, ab.y, bb.x, bb.y, x.x, x.y, s);
      }
    }
    sa.x = warp_sumf(sa.x);
    sa.y = warp_sumf(sa.y);
    sb.x = warp_sumf(sb.x);
    sb.y = warp_sumf(sb.y);
    if (lane == 0) {
      red[2 * pr][seg] = sa;
      if (hb) red[2 * pr + 1][seg] = sb;
    }
  }
  __syncthreads();
  double part = 0.0;
  for (int i = threadIdx.x; i < nr; i += kMvThreads) {
    float2 tv = red[i][0];
#pragma unroll
    for (int g = 1; g < kNseg; ++g) {
      tv.x += red[i][g].x;
      tv.y += red[i][g].y;
    }
    ws.t[r0 + i] = tv;
    const double2 wv = ws.w[r0 + i];
    part += 2.0 * (wv.x * (double)tv.x + wv.y * (double)tv.y);
  }
  part = warp_sum(part);
  if (lane == 0) wsum[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kMvThreads / 32; ++w) tot += wsum[w];
    ws.mvpart[blockIdx.x] = tot;
  }
}

// Partial p_i^H w over this CTA's range for every i < nset (one thread per i, FP32 products and sums: the
// coefficients are corrections of rounding size); ppart[i][cta].
__device__ __forceinline__ void project_partials(const CplWs& ws, int dim, int nset, int r0, int L,
                                                 const float2* s_wf) {
  for (int i = threadIdx.x; i < nset; i += kVecThreads) {
    const float2* Pi = ws.P32 + (size_t)i * dim + r0;
    float ax = 0.f, ay = 0.f;
#pragma unroll 8
    for (int r = 0; r < L; ++r) {
      const float2 pv = Pi[r], wv = s_wf[r];
      ax = fmaf(pv.x, wv.x, fmaf(pv.y, wv.y, ax));      // conj(p) w
      ay = fmaf(pv.x, wv.y, fmaf(-pv.y, wv.x, ay));
    }
    ws.ppart[(size_t)i * kMaxVec + blockIdx.x] = make_float2(ax, ay);
  }
}

__global__ __launch_bounds__(kVecThreads) void update_kernel(int dim, int j, int nsteps, int nmv, CplWs ws,
                                                             double* __restrict__ b, int* __restrict__ status) {
  if (finished(ws)) return;
  __shared__ double s_beta2;
  __shared__ float2 s_wf[kMaxL];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    double v = 0.0;
    for (int i = lane; i < nmv; i += 32) v += __ldcg(ws.mvpart + i);
    v = warp_sum(v);
    if (lane == 0) s_beta2 = v;
  }
  __syncthreads();
  const double beta2 = s_beta2;
  const double bprev = j >= 2 ? b[j - 1] : 0.0;
  const double thr = kBreakdownRel * kBreakdownRel * (bprev * bprev + fabs(beta2));
  const bool stop = (j == 0) ? !(beta2 > 0.0) : (beta2 <= thr);
  if (stop) {                       // every CTA sees the same sums and stops here
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ws.ctl[1] = j;
      ws.ctl[0] = 1;
      if (j == 0 || beta2 < -thr) atomicCAS(status, 0, (int)BSE_ERR_INDEFINITE);
    }
    return;
  }
  const double bj = sqrt(beta2), inv = 1.0 / bj;
  if (blockIdx.x == 0 && threadIdx.x == 0) b[j] = bj;
  int r0, r1;
  range_of(dim, r0, r1);
  const int L = r1 - r0;
  const bool more = j + 1 < nsteps;
  double2* qcur = ws.qd + (size_t)(j & 1) * dim;
  const double2* qprev = ws.qd + (size_t)((j + 1) & 1) * dim;
  for (int i = threadIdx.x; i < L; i += kVecThreads) {
    const int r = r0 + i;
    const double2 wv = ws.w[r];
    const double2 q = make_double2(wv.x * inv, wv.y * inv);
    const float2 tv = ws.t[r];
    const double2 p = make_double2((double)tv.x * inv, (double)tv.y * inv);
    qcur[r] = q;
    ws.Q32[(size_t)j * dim + r] = make_float2((float)q.x, (float)q.y);
    ws.P32[(size_t)j * dim + r] = make_float2((float)p.x, (float)p.y);
    if (more) {
      double2 wn = p;
      if (j >= 1) {
        const double2 qp = qprev[r];
        wn.x -= bj * qp.x;
        wn.y -= bj * qp.y;
      }
      ws.w[r] = wn;
      s_wf[i] = make_float2((float)wn.x, (float)wn.y);
    }
  }
  if (!more) return;
  __syncthreads();
  project_partials(ws, dim, j + 1, r0, L, s_wf);
}

// c[i] = <q_i, w_{j+1}>_M from the partials of all vector CTAs (one warp per i, FP64 sums in CTA order):
// 2 Re d for i of the parity of j + 1, 2i Im d otherwise.
__global__ __launch_bounds__(kVecThreads) void reduce_kernel(int j, int nvec_ctas, int pass, int nsteps, CplWs ws) {
  if (finished(ws)) return;
  const int i = blockIdx.x * kVecWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i > j) return;
  double ax = 0.0, ay = 0.0;
  for (int c = lane; c < nvec_ctas; c += 32) {
    const float2 v = ws.ppart[(size_t)i * kMaxVec + c];
    ax += (double)v.x;
    ay += (double)v.y;
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  if (lane == 0)
    ws.c[(size_t)(pass - 1) * nsteps + i] =
        (((i ^ (j + 1)) & 1) == 0) ? make_double2(2.0 * ax, 0.0) : make_double2(0.0, 2.0 * ay);
}

// w -= sum_{i <= j} <q_i, w>_M q_i (pass 1: then the partials of the second projections; pass 2: then
// fl32(w) for the product).  Threads take (element, group of i) so that many loads are in flight.
__global__ __launch_bounds__(kVecThreads) void reorth_kernel(int dim, int j, int nsteps, int pass, CplWs ws) {
  if (finished(ws)) return;
  __shared__ float2 part[kVecThreads];
  __shared__ float2 s_wf[kMaxL];
  const int nset = j + 1;
  const double2* c = ws.c + (size_t)(pass - 1) * nsteps;
  int r0, r1;
  range_of(dim, r0, r1);
  const int L = r1 - r0;
  const int ngrp = L > 0 ? (kVecThreads / L > 0 ? kVecThreads / L : 1) : 1;
  const int t = threadIdx.x, rr = L > 0 ? t % L : 0, grp = L > 0 ? t / L : kVecThreads;
  if (grp < ngrp) {
    float ax = 0.f, ay = 0.f;
    const float2* Qr = ws.Q32 + r0 + rr;
#pragma unroll 4
    for (int i = grp; i < nset; i += ngrp) {
      const double2 cd = __ldg(c + i);
      const float cx = (float)cd.x, cy = (float)cd.y;
      const float2 qv = Qr[(size_t)i * dim];
      ax = fmaf(cx, qv.x, fmaf(-cy, qv.y, ax));
      ay = fmaf(cx, qv.y, fmaf(cy, qv.x, ay));
    }
    part[grp * L + rr] = make_float2(ax, ay);
  }
  __syncthreads();
  for (int i = t; i < L; i += kVecThreads) {
    float sx = 0.f, sy = 0.f;
    for (int g = 0; g < ngrp; ++g) {
      sx += part[g * L + i].x;
      sy += part[g * L + i].y;
    }
    double2 wv = ws.w[r0 + i];
    wv.x -= (double)sx;
    wv.y -= (double)sy;
    ws.w[r0 + i] = wv;
    const float2 wf = make_float2((float)wv.x, (float)wv.y);
    s_wf[i] = wf;
    if (pass == 2) ws.x32[r0 + i] = wf;
  }
  if (pass == 2) return;
  __syncthreads();
  project_partials(ws, dim, nset, r0, L, s_wf);
}

__device__ __forceinline__ double2 cdivd(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// eps_2(w) = -C b_0^2 Im[g(z)/z], g = 1/(z - b_1^2/(z - b_2^2/(... (z - b_{n-1}^2/z)))), z = w + i eta.
__global__ void eps2_kernel(const double* __restrict__ omega, int nw, double eta, double C,
                            const double* __restrict__ b, CplWs ws, int nsteps, double* __restrict__ eps2,
                            int* __restrict__ steps_done) {
  const int n = ws.ctl[0] ? ws.ctl[1] : nsteps;
  if (blockIdx.x == 0 && threadIdx.x == 0) *steps_done = n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
    if (n == 0) {
      eps2[i] = 0.0;
      continue;
    }
    const double2 z = make_double2(omega[i], eta);
    double2 g = cdivd(make_double2(1.0, 0.0), z);
    for (int jj = n - 1; jj >= 1; --jj) {
      const double b2 = b[jj] * b[jj];
      g = cdivd(make_double2(1.0, 0.0), make_double2(z.x - b2 * g.x, z.y - b2 * g.y));
    }
    const double2 h = cdivd(g, z);
    eps2[i] = -C * b[0] * b[0] * h.y;
  }
}

}  // namespace

size_t coupled_ws_bytes(const DevSys& d, long long nsteps) { return carve_bytes(d.dim, (int)nsteps); }

// Returns -2 when the system is larger than the kernels' fixed tables (dim > 65536).
int launch_spectrum_coupled(const DevSys& d, const void* A, const void* Bm, const void* P, int nsteps,
                            const double* omega, int nw, double eta, double* eps2, double* b, int* steps_done,
                            void* ws_base, int* status, void* stream) {
  static int nsm_dev = -1, nsm = 0;
  int dev = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return e;
  if (nsm_dev != dev) {
    if ((e = (int)cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    nsm_dev = dev;
  }
  const int dim = d.dim;
  if (dim > 65536) return -2;
  int g1 = 3 * nsm;                      // three product CTAs per SM (the register limit)
  g1 = g1 > (dim + kMaxRows - 1) / kMaxRows ? g1 : (dim + kMaxRows - 1) / kMaxRows;
  g1 = g1 < (dim + 1) / 2 ? g1 : (dim + 1) / 2;
  g1 = g1 < kMaxMv ? g1 : kMaxMv;
  int g2 = nsm < (dim + 31) / 32 ? nsm : (dim + 31) / 32;
  g2 = g2 > (dim + kMaxL - 1) / kMaxL ? g2 : (dim + kMaxL - 1) / kMaxL;
  g2 = g2 < kMaxVec ? g2 : kMaxVec;
  if (g1 < 1) g1 = 1;
  if (g2 < 1) g2 = 1;
  CplWs ws = carve(ws_base, dim, nsteps);
  cudaStream_t st = (cudaStream_t)stream;
  const bool vec = (dim % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bm)) % 16 == 0);
  start_kernel<<<g2, kVecThreads, 0, st>>>(dim, (const double2*)P, ws, b, nsteps);
  for (int j = 0; j < nsteps; ++j) {
    const float sg = (j & 1) ? -1.f : 1.f;
    if (vec)
      mv_kernel<true><<<g1, kMvThreads, 0, st>>>(dim, (const float2*)A, (const float2*)Bm, sg, ws);
    else
      mv_kernel<false><<<g1, kMvThreads, 0, st>>>(dim, (const float2*)A, (const float2*)Bm, sg, ws);
    update_kernel<<<g2, kVecThreads, 0, st>>>(dim, j, nsteps, g1, ws, b, status);
    if (j + 1 < nsteps) {
      const int gr = (j + 1 + kVecWarps - 1) / kVecWarps;
      reduce_kernel<<<gr, kVecThreads, 0, st>>>(j, g2, 1, nsteps, ws);
      reorth_kernel<<<g2, kVecThreads, 0, st>>>(dim, j, nsteps, 1, ws);
      reduce_kernel<<<gr, kVecThreads, 0, st>>>(j, g2, 2, nsteps, ws);
      reorth_kernel<<<g2, kVecThreads, 0, st>>>(dim, j, nsteps, 2, ws);
    }
  }
  eps2_kernel<<<(nw + 255) / 256 > 0 ? (nw + 255) / 256 : 1, 256, 0, st>>>(omega, nw, eta, d.prefactor, b, ws, nsteps,
                                                                          eps2, steps_done);
  return (int)cudaGetLastError();
}

}  // namespace bse
