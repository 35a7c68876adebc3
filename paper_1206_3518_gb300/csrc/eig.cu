// Exciton states (Eq. bse_eig): eigenpairs H A_l = E_l A_l of the Tamm-Dancoff Hamiltonian.
//
// A Lanczos tridiagonalisation of Krylov dimension n started from a caller vector: the recursion of
// steps A7 (FP32 products with H, classical Gram-Schmidt applied twice against the whole basis in
// double-float, FP64 coefficients) stores the orthonormal basis v_0 .. v_{n-1}; T = V^H H V is
// tridiagonal.  The eigenvalues of T come from bisection on Sturm counts and its eigenvectors y_l from
// inverse iteration (ritz.cu); A_l = sum_j y_l(j) v_j.  With n = dim and a start vector that overlaps
// every eigenvector (a random one), T is similar to H and the pairs are all eigenpairs of H - the
// eigensolver of the paper's route; with n < dim they are Ritz pairs (the extreme and isolated states
// converge first).  Eigenvalues that coincide to rounding are returned once (a Krylov space holds one
// vector of a degenerate eigenspace), and inverse iteration does not re-orthogonalise eigenvectors of
// clusters closer than ~1e-10 of |H|.
//
// The back-transformation is a tiled FP32 product (64 x 64 outputs of A per CTA, 16 basis vectors per
// shared-memory stage): Y [n][n] (FP64 eigenvectors of T, rounded to FP32) times V [n][dim] (the
// double-float basis, hi + lo rounded to FP32), written as complex64 rows of A.
#include <cuda_runtime.h>

#include "internal.h"

namespace bse {
namespace {

constexpr int kT = 64, kKC = 16;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// A[l][x] = sum_j Y[l][j] V[j][x], l < n, x < dim (V: complex double-float (re.hi, re.lo, im.hi, im.lo))
__global__ void __launch_bounds__(256) backtransform_kernel(int n, int dim, const double* __restrict__ Y,
                                                            const float4* __restrict__ V, float2* __restrict__ A) {
  __shared__ float sy[kT][kKC + 1];
  __shared__ float2 sv[kKC][kT];
  const int l0 = blockIdx.y * kT, x0 = blockIdx.x * kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < n; k0 += kKC) {
    for (int t = threadIdx.x; t < kT * kKC; t += 256) {
      const int i = t / kKC, kk = t - i * kKC;
      sy[i][kk] = (l0 + i < n && k0 + kk < n) ? (float)Y[(size_t)(l0 + i) * n + k0 + kk] : 0.f;
      const int kb = t / kT, c = t - kb * kT;
      float2 v = make_float2(0.f, 0.f);
      if (k0 + kb < n && x0 + c < dim) {
        const float4 z = V[(size_t)(k0 + kb) * dim + x0 + c];
        v = make_float2(z.x + z.y, z.z + z.w);
      }
      sv[kb][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKC; ++kk) {
      float y[4];
      float2 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) y[i] = sy[ty * 4 + i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = sv[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(y[i], v[j].x, acc[i][j].x);
          acc[i][j].y = fmaf(y[i], v[j].y, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + ty * 4 + i, x = x0 + tx * 4 + j;
      if (l < n && x < dim) A[(size_t)l * dim + x] = acc[i][j];
    }
}

struct StatesLayout {
  size_t spec, ritz, Y, weight, total;
};

StatesLayout states_layout(const DevSys& d, long long n) {
  StatesLayout L;
  size_t o = 0;
  L.spec = o; o = align256(o + spectrum_ws_bytes(d, n));
  L.ritz = o; o = align256(o + ritz_ws_bytes(n));
  L.Y = o; o = align256(o + (size_t)n * n * sizeof(double));
  L.weight = o; o = align256(o + (size_t)n * sizeof(double));
  L.total = o;
  return L;
}

}  // namespace

size_t states_ws_bytes(const DevSys& d, long long n) { return states_layout(d, n).total; }

int launch_exciton_states(const DevSys& d, const void* H, const void* X0, int n, double* theta, void* A, double* ab,
                          int* steps_done, void* ws, int* status, void* stream) {
  const StatesLayout L = states_layout(d, n);
  char* base = (char*)ws;
  float4* V = nullptr;
  int e = run_haydock(d, H, X0, n, nullptr, 0, 1.0, nullptr, ab, steps_done, base + L.spec, status, stream, &V);
  if (e) return e;
  double* Y = (double*)(base + L.Y);
  e = launch_ritz_vectors(ab, steps_done, n, theta, (double*)(base + L.weight), base + L.ritz, Y, stream);
  if (e || !A) return e;
  dim3 grid((d.dim + kT - 1) / kT, (n + kT - 1) / kT);
  backtransform_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, d.dim, Y, V, (float2*)A);
  return (int)cudaGetLastError();
}

}  // namespace bse
