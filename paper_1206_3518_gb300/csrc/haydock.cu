// Haydock recursion and continued fraction (steps A7, A8), and Y = H X.
//
// The spectrum (Eq. epsilon_chi_bar in the TDA, Appendix A) is
//   eps_2(w) = -C Im[P^H (z - H)^{-1} P] = -C |P|^2 Im g(z),  z = w + i eta,
// with g the continued fraction of the Lanczos coefficients of H started at
// P/|P|.  Lanczos with classical Gram-Schmidt against the whole basis applied
// twice per step (FP64 basis and recurrence); the matrix-vector product reads
// H in FP32, multiplies in FP32 and combines 16-element partial sums in FP64.
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
constexpr double kBreakdownRel = 1e-10;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier over a (count, generation) pair; false if the wait timed out or
// another CTA already reported an error.
__device__ bool grid_barrier(unsigned* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      while (*gen == g) {
        if (*(volatile int*)status != 0) {
          good = 0;
          break;
        }
        if (globaltimer() - t0 > 2000000000ull) {
          atomicCAS(status, 0, (int)BSE_ERR_TIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
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

// x loaders: FP32 vectors written by other CTAs inside the kernel bypass L1 (ld.cg);
// FP64 inputs of bse_apply_H are read-only and rounded to FP32 on the fly.
__device__ __forceinline__ float4 load_x2(const float2* x, int i) {
  return __ldcg(reinterpret_cast<const float4*>(x) + i);
}
__device__ __forceinline__ float4 load_x2(const double2* x, int i) {
  const double2 a = __ldg(x + 2 * i), b = __ldg(x + 2 * i + 1);
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}
__device__ __forceinline__ float2 load_x1(const float2* x, int i) { return __ldcg(x + i); }
__device__ __forceinline__ float2 load_x1(const double2* x, int i) {
  const double2 a = __ldg(x + i);
  return make_float2((float)a.x, (float)a.y);
}

// Row dot  sum_c H[r][c] x[c]: FP32 products accumulated over 16 elements per lane,
// then combined in FP64 (vector loads of H when dim is even).
template <typename XT>
__device__ __forceinline__ double2 row_dot(const float2* __restrict__ Hr, const XT* x, int dim, int lane) {
  double2 acc = make_double2(0.0, 0.0);
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
      acc.x += s.x;
      acc.y += s.y;
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
    acc.x += s.x;
    acc.y += s.y;
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
      acc.x += s.x;
      acc.y += s.y;
    }
    float2 s = make_float2(0.f, 0.f);
    for (; i < dim; i += 32) {
      const float2 h = __ldg(Hr + i);
      const float2 v = load_x1(x, i);
      s.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, s.x));
      s.y = fmaf(h.x, v.y, fmaf(h.y, v.x, s.y));
    }
    acc.x += s.x;
    acc.y += s.y;
  }
  return warp_sum(acc);
}

struct HayArgs {
  DevSys d;
  const float2* H;
  const double2* P;
  int nsteps;
  const double* omega;
  int nw;
  double eta;
  double* eps2;
  double* ab;
  int* steps_done;
  double2* V;       // [nsteps][dim]
  float2* vf;       // [dim]
  double2* hpart;   // [grid][nsteps]
  double2* h1;      // [nsteps]
  double2* h2;      // [nsteps]
  double* npart;    // [grid][2]
  unsigned* bar;    // [2]
  int* status;
};

// hpart[cta][i] = sum over own rows conj(V[i][r]) w[r], i in [0, n).
__device__ void project_partial(const HayArgs& A, const double2* wsm, int row0, int nrows, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dim = A.d.dim;
  for (int i = warp; i < n; i += kWarps) {
    const double2* Vi = A.V + (size_t)i * dim + row0;
    double2 s = make_double2(0.0, 0.0);
    for (int r = lane; r < nrows; r += 32) {
      const double2 v = __ldcg(Vi + r), w = wsm[r];
      s.x += v.x * w.x + v.y * w.y;
      s.y += v.x * w.y - v.y * w.x;
    }
    s = warp_sum(s);
    if (lane == 0) A.hpart[(size_t)blockIdx.x * A.nsteps + i] = s;
  }
}

// h[i] = sum_cta hpart[cta][i] for the i owned by this CTA (deterministic order).
__device__ void reduce_coeffs(const HayArgs& A, double2* h, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = blockIdx.x + gridDim.x * warp; i < n; i += gridDim.x * kWarps) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = lane; c < (int)gridDim.x; c += 32) {
      const double2 v = __ldcg(A.hpart + (size_t)c * A.nsteps + i);
      s.x += v.x;
      s.y += v.y;
    }
    s = warp_sum(s);
    if (lane == 0) h[i] = s;
  }
}

// w[r] -= sum_i V[i][r] h[i] over own rows; warps split i, lanes split rows.
__device__ void subtract_projection(const HayArgs& A, double2* wsm, double2 (*red)[32], const double2* h, int row0,
                                    int nrows, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dim = A.d.dim;
  for (int r0 = 0; r0 < nrows; r0 += 32) {
    const int r = r0 + lane;
    double2 s = make_double2(0.0, 0.0);
    if (r < nrows) {
      for (int i = warp; i < n; i += kWarps) {
        const double2 v = __ldcg(A.V + (size_t)i * dim + row0 + r);
        const double2 c = __ldcg(h + i);
        s.x += v.x * c.x - v.y * c.y;
        s.y += v.x * c.y + v.y * c.x;
      }
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && r < nrows) {
      double2 t = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kWarps; ++q) {
        t.x += red[q][lane].x;
        t.y += red[q][lane].y;
      }
      wsm[r].x -= t.x;
      wsm[r].y -= t.y;
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
  for (int c = threadIdx.x; c < (int)gridDim.x; c += kThreads) v += __ldcg(A.npart + 2 * c + which);
  double t = block_sum(v, red1);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = t;
  __syncthreads();
  return bc;
}

__global__ __launch_bounds__(kThreads, 1) void haydock_kernel(HayArgs A) {
  extern __shared__ double2 wsm[];                 // own rows of w
  __shared__ double2 red[kWarps][32];
  __shared__ double red1[kWarps];
  const int dim = A.d.dim;
  const int rows_per = (dim + gridDim.x - 1) / gridDim.x;
  const int row0 = min(dim, (int)blockIdx.x * rows_per);
  const int nrows = min(dim, row0 + rows_per) - row0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // v_0 = P / |P|
  double pp = 0.0;
  for (int r = threadIdx.x; r < nrows; r += kThreads) {
    const double2 p = A.P[row0 + r];
    pp += p.x * p.x + p.y * p.y;
  }
  pp = block_sum(pp, red1);
  if (threadIdx.x == 0) A.npart[2 * blockIdx.x] = pp;
  if (!grid_barrier(A.bar, A.status)) return;
  const double pn2 = all_cta_sum(A, 0, red1);
  const double pinv = 1.0 / sqrt(pn2);
  for (int r = threadIdx.x; r < nrows; r += kThreads) {
    const double2 p = A.P[row0 + r];
    const double2 v = make_double2(p.x * pinv, p.y * pinv);
    A.V[row0 + r] = v;
    A.vf[row0 + r] = make_float2((float)v.x, (float)v.y);
  }
  if (!grid_barrier(A.bar, A.status)) return;

  int done = A.nsteps;
  for (int j = 0; j < A.nsteps; ++j) {
    // w = H v_j on own rows, |H v_j|^2 partial
    double hv2 = 0.0;
    for (int r = warp; r < nrows; r += kWarps) {
      const double2 s = row_dot(A.H + (size_t)(row0 + r) * dim, A.vf, dim, lane);
      if (lane == 0) {
        wsm[r] = s;
        hv2 += s.x * s.x + s.y * s.y;
      }
    }
    hv2 = block_sum(hv2, red1);
    if (threadIdx.x == 0) A.npart[2 * blockIdx.x + 1] = hv2;
    __syncthreads();
    project_partial(A, wsm, row0, nrows, j + 1);
    if (!grid_barrier(A.bar, A.status)) return;
    reduce_coeffs(A, A.h1, j + 1);
    if (!grid_barrier(A.bar, A.status)) return;
    subtract_projection(A, wsm, red, A.h1, row0, nrows, j + 1);
    project_partial(A, wsm, row0, nrows, j + 1);
    if (!grid_barrier(A.bar, A.status)) return;
    reduce_coeffs(A, A.h2, j + 1);
    if (!grid_barrier(A.bar, A.status)) return;
    subtract_projection(A, wsm, red, A.h2, row0, nrows, j + 1);
    double ww = 0.0;
    for (int r = threadIdx.x; r < nrows; r += kThreads) ww += wsm[r].x * wsm[r].x + wsm[r].y * wsm[r].y;
    ww = block_sum(ww, red1);
    if (threadIdx.x == 0) A.npart[2 * blockIdx.x] = ww;
    if (!grid_barrier(A.bar, A.status)) return;
    const double bn2 = all_cta_sum(A, 0, red1);
    const double sc2 = all_cta_sum(A, 1, red1);
    const double2 c1 = __ldcg(A.h1 + j), c2 = __ldcg(A.h2 + j);
    const double aj = c1.x + c2.x;
    const double bn = sqrt(bn2);
    const bool last = (j + 1 == A.nsteps);
    const bool brk = !last && !(bn > kBreakdownRel * sqrt(sc2));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
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
    double2* Vn = A.V + (size_t)(j + 1) * dim + row0;
    for (int r = threadIdx.x; r < nrows; r += kThreads) {
      const double2 v = make_double2(wsm[r].x * binv, wsm[r].y * binv);
      Vn[r] = v;
      A.vf[row0 + r] = make_float2((float)v.x, (float)v.y);
    }
    if (!grid_barrier(A.bar, A.status)) return;
  }
  if (!grid_barrier(A.bar, A.status)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.steps_done = done;
  // continued fraction from the bottom: g = 1/(z - a_j - b_{j+1}^2 g)
  const double C = A.d.prefactor * pn2;
  for (int wi = blockIdx.x * kThreads + threadIdx.x; wi < A.nw; wi += gridDim.x * kThreads) {
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

// Shared with the adjoint: runs the recursion into a caller-laid-out workspace.
int run_haydock(const DevSys& d, const void* H, const void* P, int nsteps, const double* omega, int nw, double eta,
                double* eps2, double* ab, int* steps_done, void* ws, int* status, void* stream, double2** V_out) {
  cudaStream_t st = (cudaStream_t)stream;
  const SpecLayout L = spec_layout(d, nsteps);
  char* base = (char*)ws;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rows_per_max = (d.dim + sms - 1) / sms;
  const size_t dyn = (size_t)rows_per_max * sizeof(double2);
  if (dyn > 160 * 1024) return -1;
  cudaFuncSetAttribute((const void*)haydock_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, haydock_kernel, kThreads, dyn);
  if (occ < 1) return -1;
  int grid = sms;                       // one CTA per SM: every CTA streams its own rows of H
  if (grid > kMaxGrid) grid = kMaxGrid;
  HayArgs A;
  A.d = d;
  A.H = (const float2*)H;
  A.P = (const double2*)P;
  A.nsteps = nsteps;
  A.omega = omega;
  A.nw = nw;
  A.eta = eta;
  A.eps2 = eps2;
  A.ab = ab;
  A.steps_done = steps_done;
  A.V = (double2*)(base + L.V);
  A.vf = (float2*)(base + L.vf);
  A.hpart = (double2*)(base + L.hpart);
  A.h1 = (double2*)(base + L.h1);
  A.h2 = (double2*)(base + L.h2);
  A.npart = (double*)(base + L.npart);
  A.bar = (unsigned*)(base + L.bar);
  A.status = status;
  if (V_out) *V_out = A.V;
  int e = (int)cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), st);
  if (e) return e;
  void* args[] = {&A};
  e = (int)cudaLaunchCooperativeKernel((const void*)haydock_kernel, dim3(grid), dim3(kThreads), args, dyn, st);
  return e;
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
// stand-in for the symbol), so its device address is looked up once per device
// with cudaGetSymbolAddress and cached.  All calls share the array: calls that
// overlap on the GPU race on it.
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
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
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
