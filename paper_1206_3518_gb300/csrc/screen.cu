// Static RPA screening from the system's own states (Sec. II A-B, Eqs. chi0_GG, epsilon_-1;
// the W_GG'(q) form of Sec. III A).  Not on the spectrum path: it produces the W that step A4
// otherwise takes as input.
//
//   a_S(G)  = sqrt(|w_S|) v^1/2(q+G) rho_vc^{k,k+q}(G),  w_S = 4/(Omega Nk)/(e_vk - e_c,k+q) < 0
//             (q = 0: a_S(0) = sqrt(|w_S|) sqrt(4 pi) conj(P_S), the k.p optical limit)
//   eps(q)  = I + sum_S a_S a_S^H            (= 1 - v^1/2 chi0 v^1/2, Hermitian, eigenvalues >= 1)
//   eps^-1  by Newton-Schulz: X <- X (2 I - eps X) from X_0 = 2/(1 + R) I, R a Gershgorin bound of
//           the largest eigenvalue, so |I - eps X_k| <= ((R - 1)/(R + 1))^(2^k)
//   W(q)    = v^1/2 eps^-1 v^1/2; at q = 0 the head is the mini-zone average [eps^-1]_00 12 pi/q_c^2
//             and the wings are zero.
//
// Everything is batched over the q points of a range: one launch per stage.
#include <cuda_runtime.h>

#include "gemm_tile.cuh"
#include "internal.h"

namespace bse {
namespace {

using gemm::BM;
using gemm::BN;
constexpr int kT = gemm::kThreads;

// In place: rho rows -> a rows (q-range layout [q][k][v][c][ng_max]).
__global__ void scale_kernel(DevSys d, float2* __restrict__ a, const double* __restrict__ e,
                             const double2* __restrict__ P, int q_begin, double gap_floor) {
  const long long row = blockIdx.x;                  // ((qi Nk + k) Nv + v) Nc + c
  const int nvc = d.nv * d.nc;
  const int qi = (int)(row / ((long long)d.nkpt * nvc));
  const int rem = (int)(row - (long long)qi * d.nkpt * nvc);
  const int k = rem / nvc, iv = (rem / d.nc) % d.nv, ic = rem % d.nc;
  const int q = q_begin + qi;
  const int k1 = k / (d.nk2 * d.nk3), k2 = (k / d.nk3) % d.nk2, k3 = k % d.nk3;
  const int q1 = q / (d.nk2 * d.nk3), q2 = (q / d.nk3) % d.nk2, q3 = q % d.nk3;
  const int kp = (((k1 + q1) % d.nk1) * d.nk2 + (k2 + q2) % d.nk2) * d.nk3 + (k3 + q3) % d.nk3;
  const double de = fmax(e[(size_t)kp * d.nb + d.nv + ic] - e[(size_t)k * d.nb + iv], gap_floor);
  const float sw = (float)sqrt(4.0 / (d.omega_cell * d.nkpt * de));
  const int NG = d.ngq[q];
  float2* r = a + (size_t)row * d.ng_max;
  const float* vs = d.vsq + (size_t)q * d.ng_max;
  for (int g = threadIdx.x; g < d.ng_max; g += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (g < NG) {
      if (q == 0 && g == 0) {
        const double2 p = P[rem];                    // conj(P_S) sqrt(4 pi)
        const double f = 3.5449077018110320546 * (double)sw;
        v = make_float2((float)(p.x * f), (float)(-p.y * f));
      } else {
        const float2 x = r[g];
        const float f = sw * vs[g];
        v = make_float2(x.x * f, x.y * f);
      }
    }
    r[g] = v;
  }
}

// eps(q) = I + A^T conj(A) with A = a rows of q (K = Nk Nv Nc); one 64 x 64 tile per CTA.
__global__ __launch_bounds__(kT) void eps_kernel(DevSys d, const float2* __restrict__ a, float2* __restrict__ eps,
                                                 int q_begin) {
  const int qi = blockIdx.z, q = q_begin + qi;
  const int NG = d.ngq[q];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= NG || n0 >= NG) return;
  const long long K = (long long)d.nkpt * d.nv * d.nc;
  const float2* A = a + (size_t)qi * K * d.ng_max;
  __shared__ gemm::Smem sm;
  float2 acc[4][4];
  // C[m][n] = sum_s A[s][m] conj(A[s][n]): operands stored [k][m]
  gemm::tile<false, false, false, true>(A, d.ng_max, NG, A, d.ng_max, NG, (int)K, m0, n0, sm, acc);
  float2* E = eps + (size_t)qi * d.ng_max * d.ng_max;
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + tm * 4 + i;
    if (r >= NG) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tn * 4 + j;
      if (c >= NG) continue;
      float2 v = acc[i][j];
      if (r == c) v.x += 1.f;
      E[(size_t)r * d.ng_max + c] = v;
    }
  }
}

// X = 2/(1 + R) I with R = max row sum of |eps| (Gershgorin bound of the largest eigenvalue).
__global__ void ns_init_kernel(DevSys d, const float2* __restrict__ eps, float2* __restrict__ X, int q_begin) {
  const int qi = blockIdx.x, q = q_begin + qi;
  const int NG = d.ngq[q];
  const float2* E = eps + (size_t)qi * d.ng_max * d.ng_max;
  float2* Xq = X + (size_t)qi * d.ng_max * d.ng_max;
  __shared__ float red[32];
  float rmax = 0.f;
  for (int r = threadIdx.x; r < NG; r += blockDim.x) {
    float srow = 0.f;
    for (int c = 0; c < NG; ++c) {
      const float2 v = E[(size_t)r * d.ng_max + c];
      srow += sqrtf(v.x * v.x + v.y * v.y);
    }
    rmax = fmaxf(rmax, srow);
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
  __syncthreads();
  if (threadIdx.x < 32) {
    float m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const float x0 = 2.f / (1.f + red[0]);
  for (long long i = threadIdx.x; i < (long long)d.ng_max * d.ng_max; i += blockDim.x) {
    const int r = (int)(i / d.ng_max), c = (int)(i % d.ng_max);
    Xq[i] = make_float2((r == c && r < NG) ? x0 : 0.f, 0.f);
  }
}

// C = alpha I + beta A B for every q of the range (NG x NG, row-major with stride ng_max).
__global__ __launch_bounds__(kT) void axpb_kernel(DevSys d, const float2* __restrict__ A, const float2* __restrict__ B,
                                                  float2* __restrict__ C, float alpha, float beta, int q_begin) {
  const int qi = blockIdx.z, q = q_begin + qi;
  const int NG = d.ngq[q];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= NG || n0 >= NG) return;
  const size_t off = (size_t)qi * d.ng_max * d.ng_max;
  __shared__ gemm::Smem sm;
  float2 acc[4][4];
  gemm::tile<true, false, false, false>(A + off, d.ng_max, NG, B + off, d.ng_max, NG, NG, m0, n0, sm, acc);
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + tm * 4 + i;
    if (r >= NG) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tn * 4 + j;
      if (c >= NG) continue;
      float2 v = make_float2(beta * acc[i][j].x, beta * acc[i][j].y);
      if (r == c) v.x += alpha;
      C[off + (size_t)r * d.ng_max + c] = v;
    }
  }
}

// residual[q] = max |I - eps X| (from T = eps X).
__global__ void residual_kernel(DevSys d, const float2* __restrict__ T, float* __restrict__ res, int q_begin) {
  const int qi = blockIdx.x, q = q_begin + qi;
  const int NG = d.ngq[q];
  const float2* Tq = T + (size_t)qi * d.ng_max * d.ng_max;
  float m = 0.f;
  for (long long i = threadIdx.x; i < (long long)NG * NG; i += blockDim.x) {
    const int r = (int)(i / NG), c = (int)(i % NG);
    float2 v = Tq[(size_t)r * d.ng_max + c];
    if (r == c) v.x -= 1.f;
    m = fmaxf(m, sqrtf(v.x * v.x + v.y * v.y));
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    res[qi] = t;
  }
}

// W(q) = v^1/2 eps^-1 v^1/2 (head at q = 0: mini-zone average, wings zero); zero padding to ng_max.
__global__ void w_kernel(DevSys d, const float2* __restrict__ X, float2* __restrict__ W, int q_begin, float head) {
  const int qi = blockIdx.y, q = q_begin + qi;
  const int NG = d.ngq[q];
  const float2* Xq = X + (size_t)qi * d.ng_max * d.ng_max;
  float2* Wq = W + (size_t)q * d.ng_max * d.ng_max;
  const float* vs = d.vsq + (size_t)q * d.ng_max;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)d.ng_max * d.ng_max;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / d.ng_max), c = (int)(i % d.ng_max);
    float2 v = make_float2(0.f, 0.f);
    if (r < NG && c < NG) {
      const float2 x = Xq[i];
      if (q == 0 && (r == 0 || c == 0)) {
        if (r == 0 && c == 0) v = make_float2(x.x * head, x.y * head);
      } else {
        const float f = vs[r] * vs[c];
        v = make_float2(x.x * f, x.y * f);
      }
    }
    Wq[i] = v;
  }
}

}  // namespace

size_t screen_ws_bytes(const DevSys& d, long long qchunk) {
  return (size_t)4 * qchunk * d.ng_max * d.ng_max * sizeof(float2);
}

// ws: eps, X, Y, T (each [nq][ng_max][ng_max] complex64).
int launch_screening(const DevSys& d, void* rho_chi, const double* energies, const void* P, int q_begin, int q_end,
                     int iterations, void* W, float* residual, void* ws, double gap_floor, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int nq = q_end - q_begin;
  const long long rows = (long long)nq * d.nkpt * d.nv * d.nc;
  scale_kernel<<<(unsigned)rows, 128, 0, st>>>(d, (float2*)rho_chi, energies, (const double2*)P, q_begin, gap_floor);
  const size_t mat = (size_t)d.ng_max * d.ng_max;
  float2* E = (float2*)ws;
  float2* X = E + (size_t)nq * mat;
  float2* Y = X + (size_t)nq * mat;
  float2* T = Y + (size_t)nq * mat;
  dim3 grid((d.ng_max + BN - 1) / BN, (d.ng_max + BM - 1) / BM, nq);
  eps_kernel<<<grid, kT, 0, st>>>(d, (const float2*)rho_chi, E, q_begin);
  ns_init_kernel<<<nq, 256, 0, st>>>(d, E, X, q_begin);
  for (int it = 0; it < iterations; ++it) {
    axpb_kernel<<<grid, kT, 0, st>>>(d, E, X, T, 2.f, -1.f, q_begin);     // T = 2 I - eps X
    axpb_kernel<<<grid, kT, 0, st>>>(d, X, T, Y, 0.f, 1.f, q_begin);      // Y = X T
    float2* t = X;
    X = Y;
    Y = t;
  }
  if (residual) {
    axpb_kernel<<<grid, kT, 0, st>>>(d, E, X, T, 0.f, 1.f, q_begin);      // T = eps X
    residual_kernel<<<nq, 256, 0, st>>>(d, T, residual, q_begin);
  }
  const double qc = cbrt(6.0 * kPi * kPi / (d.omega_cell * d.nkpt));
  const float head = (float)(12.0 * kPi / (qc * qc));
  w_kernel<<<dim3(64, nq), 256, 0, st>>>(d, X, (float2*)W, q_begin, head);
  return (int)cudaGetLastError();
}

}  // namespace bse
