// Exciton energies and oscillator strengths from the Haydock recursion (steps A7-A8).
//
// The continued fraction g(z) = e_0^T (z - T)^{-1} e_0 of the Lanczos tridiagonal T (diagonal a_j,
// off-diagonal b_j) is the pole sum g(z) = sum_i w_i / (z - theta_i), theta_i the eigenvalues of T and
// w_i the squared first components of its normalised eigenvectors.  Converged Ritz pairs are
// eigenpairs of H: exciton energies E_l and normalised oscillator strengths |P^H A_l|^2 / |P|^2 (the
// spectral representation behind Eq. resolvent and Eq. epsilon_chi_bar).
//
// One thread per Ritz value, FP64: the i-th smallest eigenvalue by bisection on Sturm counts within
// the Gershgorin interval, then two steps of inverse iteration with (T - theta I) factorised by
// Gaussian elimination with partial pivoting (per-thread scratch in the caller's workspace).
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace bse {
namespace {

constexpr int kRitzThreads = 128;

// number of eigenvalues of T smaller than x
__device__ int sturm_count(const double* a, const double* b, int n, double x, double tiny) {
  int c = 0;
  double q = a[0] - x;
  if (q < 0.0) ++c;
  for (int j = 1; j < n; ++j) {
    if (fabs(q) < tiny) q = q < 0.0 ? -tiny : tiny;
    q = (a[j] - x) - b[j] * b[j] / q;
    if (q < 0.0) ++c;
  }
  return c;
}

// Solve (T - s I) x = r in place of r, given the factorisation in d, u, u2, m, pv (see below).
__device__ void lu_solve(const double* d, const double* u, const double* u2, const double* m, const double* pv,
                         double* r, int n) {
  for (int j = 0; j + 1 < n; ++j) {
    if (pv[j] != 0.0) {
      const double t = r[j];
      r[j] = r[j + 1];
      r[j + 1] = t;
    }
    r[j + 1] -= m[j] * r[j];
  }
  r[n - 1] /= d[n - 1];
  if (n >= 2) r[n - 2] = (r[n - 2] - u[n - 2] * r[n - 1]) / d[n - 2];
  for (int j = n - 3; j >= 0; --j) r[j] = (r[j] - u[j] * r[j + 1] - u2[j] * r[j + 2]) / d[j];
}

// vecs (optional) [nsteps][nsteps]: row i receives the normalised eigenvector of T for theta_i (zero
// past the recursion's length and for rows i >= steps done).
__global__ __launch_bounds__(kRitzThreads) void ritz_kernel(const double* __restrict__ ab,
                                                           const int* __restrict__ steps_done, int nsteps,
                                                           double* __restrict__ theta, double* __restrict__ weight,
                                                           double* __restrict__ ws, double* __restrict__ vecs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsteps) return;
  int n = *steps_done;
  n = n < nsteps ? n : nsteps;
  double* vrow = vecs ? vecs + (size_t)i * nsteps : nullptr;
  if (i >= n || n < 1) {
    theta[i] = 0.0;
    weight[i] = 0.0;
    if (vrow)
      for (int j = 0; j < nsteps; ++j) vrow[j] = 0.0;
    return;
  }
  const double* a = ab;
  const double* b = ab + nsteps;          // b[j] couples j - 1 and j; b[0] unused
  if (n == 1) {
    theta[i] = a[0];
    weight[i] = 1.0;
    if (vrow)
      for (int j = 0; j < nsteps; ++j) vrow[j] = j == 0 ? 1.0 : 0.0;
    return;
  }
  double lo = DBL_MAX, hi = -DBL_MAX, scale = 0.0;
  for (int j = 0; j < n; ++j) {
    const double r = (j > 0 ? fabs(b[j]) : 0.0) + (j + 1 < n ? fabs(b[j + 1]) : 0.0);
    lo = fmin(lo, a[j] - r);
    hi = fmax(hi, a[j] + r);
    scale = fmax(scale, fabs(a[j]) + r);
  }
  const double tiny = DBL_MIN / DBL_EPSILON + 1e-300 * scale;
  lo -= 1e-12 * scale;
  hi += 1e-12 * scale;
  for (int it = 0; it < 200 && hi - lo > 2.0 * DBL_EPSILON * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, n, mid, tiny) > i) hi = mid; else lo = mid;
  }
  const double th = 0.5 * (lo + hi);
  theta[i] = th;

  // (T - th I) = P L U with partial pivoting: u2 is the second superdiagonal created by row swaps
  double* d = ws + (size_t)i * 6 * nsteps;
  double* u = d + nsteps;
  double* u2 = u + nsteps;
  double* m = u2 + nsteps;
  double* pv = m + nsteps;
  double* x = pv + nsteps;
  const double floor = DBL_EPSILON * scale + tiny;
  for (int j = 0; j < n; ++j) {
    d[j] = a[j] - th;
    u[j] = j + 1 < n ? b[j + 1] : 0.0;
    u2[j] = 0.0;
    x[j] = 1.0;
  }
  for (int j = 0; j + 1 < n; ++j) {
    const double l = b[j + 1];            // subdiagonal entry of row j + 1
    if (fabs(d[j]) >= fabs(l)) {
      pv[j] = 0.0;
      if (fabs(d[j]) < floor) d[j] = d[j] < 0.0 ? -floor : floor;
      m[j] = l / d[j];
      d[j + 1] -= m[j] * u[j];
    } else {                              // swap rows j and j + 1
      pv[j] = 1.0;
      m[j] = d[j] / l;
      d[j] = l;
      const double t = d[j + 1];
      d[j + 1] = u[j] - m[j] * t;
      if (j + 2 < n) {
        u2[j] = u[j + 1];
        u[j + 1] = -m[j] * u2[j];
      }
      u[j] = t;
    }
  }
  if (fabs(d[n - 1]) < floor) d[n - 1] = d[n - 1] < 0.0 ? -floor : floor;
  for (int pass = 0; pass < 2; ++pass) {
    lu_solve(d, u, u2, m, pv, x, n);
    double nrm = 0.0;
    for (int j = 0; j < n; ++j) nrm = fmax(nrm, fabs(x[j]));
    for (int j = 0; j < n; ++j) x[j] /= nrm;
  }
  double s2 = 0.0;
  for (int j = 0; j < n; ++j) s2 += x[j] * x[j];
  weight[i] = x[0] * x[0] / s2;
  if (vrow) {
    const double inv = 1.0 / sqrt(s2);
    for (int j = 0; j < nsteps; ++j) vrow[j] = j < n ? x[j] * inv : 0.0;
  }
}

}  // namespace

size_t ritz_ws_bytes(long long nsteps) { return (size_t)6 * nsteps * nsteps * sizeof(double); }

int launch_ritz(const double* ab, const int* steps_done, int nsteps, double* theta, double* weight, void* ws,
                void* stream) {
  return launch_ritz_vectors(ab, steps_done, nsteps, theta, weight, ws, nullptr, stream);
}

int launch_ritz_vectors(const double* ab, const int* steps_done, int nsteps, double* theta, double* weight, void* ws,
                        double* vecs, void* stream) {
  const int blocks = (nsteps + kRitzThreads - 1) / kRitzThreads;
  ritz_kernel<<<blocks, kRitzThreads, 0, (cudaStream_t)stream>>>(ab, steps_done, nsteps, theta, weight, (double*)ws,
                                                                vecs);
  return (int)cudaGetLastError();
}

}  // namespace bse
