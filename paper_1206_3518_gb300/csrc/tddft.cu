// Macroscopic dielectric function from TDDFT with local fields (Sec. II A-B: Eqs. chi0_GG, Dyson_GG,
// epsilon_-1, epsilon_M) in the optical limit q -> 0, on the q = 0 sphere of the system.
//
//   chi~0_GG'(w) = 2/(Omega Nk) sum_S [ a_S(G) conj a_S(G') / (w - de_S + i eta)
//                                      - abar_S(G) conj abar_S(G') / (w + de_S + i eta) ]
//   a_S(G) = v^1/2(G) rho_vc^{kk}(G),  abar_S(G) = v^1/2(G) conj(rho_vc^{kk}(-G))   (G != 0)
//   a_S(0) = sqrt(4 pi) conj(P_S),     abar_S(0) = -sqrt(4 pi) P_S                   (k.p limit)
//   eps^-1 = I + (I - chi~0 (I + F))^-1 chi~0,   eps_M = 1/[eps^-1]_00
//
// F = v^-1/2 f_xc v^-1/2 is zero for the RPA and the adiabatic local-density kernel otherwise:
// f_xc(r) = d^2(n eps_xc)/dn^2 at the density n(r) = 2/(Omega Nk) sum_{k,v} |u_vk(r)|^2 (Slater
// exchange + Perdew-Zunger correlation), F_GG' = |G| f_xc(G - G') |G'|/(4 pi).
//
// Kernels: a_S, abar_S and de_S from rho_x, P and the energies; chi~0(w) as a weighted complex Gram
// product per frequency (64 x 64 output tiles, 16 transitions per shared-memory stage, FP32); the
// density, f_xc(r) and its transform onto the difference box of the sphere (three separable direct
// DFT passes in FP64); the batched Dyson solve: M = I - chi~0 (I + F) augmented with chi~0 e_0, Gaussian
// elimination with partial pivoting and back substitution, one CTA per frequency (FP32 matrix, FP64
// result).  No device-side waits; capturable.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace bse {
namespace {

constexpr int kT = 64;            // output tile (G x G')
constexpr int kKC = 16;           // transitions per shared-memory stage

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// a, abar [dim][ng0] and de [dim]
__global__ void optical_pairs_kernel(DevSys d, const float2* __restrict__ rho_x, const double2* __restrict__ P,
                                     const double* __restrict__ e, double delta, float2* __restrict__ a,
                                     float2* __restrict__ ab, double* __restrict__ de) {
  const long long n = (long long)d.dim * d.ng0;
  const float s4pi = 3.5449077018110318f;   // sqrt(4 pi)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int S = (int)(i / d.ng0), g = (int)(i - (long long)S * d.ng0);
    float2 x, y;
    if (g == 0) {
      const double2 p = P[S];
      x = make_float2(s4pi * (float)p.x, -s4pi * (float)p.y);
      y = make_float2(-s4pi * (float)p.x, -s4pi * (float)p.y);
    } else {
      const float vs = d.vsq[g];                                   // q = 0 row: sqrt(4 pi)/|G|
      const float2 r = rho_x[(size_t)S * d.ng_max + g];
      const float2 rm = rho_x[(size_t)S * d.ng_max + d.gminus0[g]];
      x = make_float2(vs * r.x, vs * r.y);
      y = make_float2(vs * rm.x, -vs * rm.y);
    }
    a[i] = x;
    ab[i] = y;
    if (g == 0) {
      const int nvc = d.nv * d.nc, k = S / nvc, v = (S / d.nc) % d.nv, c = S % d.nc;
      de[S] = e[(size_t)k * d.nb + d.nv + c] + delta - e[(size_t)k * d.nb + v];
    }
  }
}

// chi[w][G][G'] for the frequencies of the launch (blockIdx.z); 256 threads, 4 x 4 outputs each
__global__ void __launch_bounds__(256) chi0_kernel(int dim, int ng, const float2* __restrict__ a,
                                                   const float2* __restrict__ ab, const double* __restrict__ de,
                                                   const double* __restrict__ omega, double eta, double pref,
                                                   float2* __restrict__ chi) {
  __shared__ float2 sa[kKC][kT], sap[kKC][kT], sb[kKC][kT], sbp[kKC][kT];
  __shared__ float2 r[kKC], rb[kKC];
  const int w = blockIdx.z;
  const int g0 = blockIdx.y * kT, h0 = blockIdx.x * kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double om = omega[w];
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int s0 = 0; s0 < dim; s0 += kKC) {
    for (int t = threadIdx.x; t < kKC * kT; t += 256) {
      const int kk = t / kT, c = t - kk * kT, S = s0 + kk;
      const bool sv = S < dim;
      sa[kk][c] = (sv && g0 + c < ng) ? a[(size_t)S * ng + g0 + c] : make_float2(0.f, 0.f);
      sb[kk][c] = (sv && g0 + c < ng) ? ab[(size_t)S * ng + g0 + c] : make_float2(0.f, 0.f);
      sap[kk][c] = (sv && h0 + c < ng) ? a[(size_t)S * ng + h0 + c] : make_float2(0.f, 0.f);
      sbp[kk][c] = (sv && h0 + c < ng) ? ab[(size_t)S * ng + h0 + c] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < kKC) {
      const int S = s0 + threadIdx.x;
      float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
      if (S < dim) {
        const double u = om - de[S], v = om + de[S];
        const double du = u * u + eta * eta, dv = v * v + eta * eta;
        x = make_float2((float)(u / du), (float)(-eta / du));          // 1/(w - de + i eta)
        y = make_float2((float)(-v / dv), (float)(eta / dv));          // -1/(w + de + i eta)
      }
      r[threadIdx.x] = x;
      rb[threadIdx.x] = y;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKC; ++kk) {
      float2 x[4], xb[4], y[4], yb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        x[i] = cmul(sa[kk][ty * 4 + i], r[kk]);
        xb[i] = cmul(sb[kk][ty * 4 + i], rb[kk]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        y[j] = sap[kk][tx * 4 + j];
        yb[j] = sbp[kk][tx * 4 + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {                                  // x conj(y) + xb conj(yb)
          acc[i][j].x += x[i].x * y[j].x + x[i].y * y[j].y + xb[i].x * yb[j].x + xb[i].y * yb[j].y;
          acc[i][j].y += x[i].y * y[j].x - x[i].x * y[j].y + xb[i].y * yb[j].x - xb[i].x * yb[j].y;
        }
    }
    __syncthreads();
  }
  const float p = (float)pref;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int g = g0 + ty * 4 + i, h = h0 + tx * 4 + j;
      if (g < ng && h < ng) chi[((size_t)w * ng + g) * ng + h] = make_float2(p * acc[i][j].x, p * acc[i][j].y);
    }
}

// C[w] = A[w] B for n x n complex matrices (B shared), 64 x 64 tiles
__global__ void __launch_bounds__(256) batched_gemm_kernel(int n, const float2* __restrict__ A,
                                                           const float2* __restrict__ B, float2* __restrict__ C) {
  __shared__ float2 sa[kT][kKC + 1], sb[kKC][kT];
  const int w = blockIdx.z;
  const int r0 = blockIdx.y * kT, c0 = blockIdx.x * kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float2* Aw = A + (size_t)w * n * n;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < n; k0 += kKC) {
    for (int t = threadIdx.x; t < kT * kKC; t += 256) {
      const int i = t / kKC, kk = t - i * kKC;
      sa[i][kk] = (r0 + i < n && k0 + kk < n) ? Aw[(size_t)(r0 + i) * n + k0 + kk] : make_float2(0.f, 0.f);
      const int kb = t / kT, j = t - kb * kT;
      sb[kb][j] = (k0 + kb < n && c0 + j < n) ? B[(size_t)(k0 + kb) * n + c0 + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKC; ++kk) {
      float2 x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = sa[ty * 4 + i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) y[j] = sb[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x += x[i].x * y[j].x - x[i].y * y[j].y;
          acc[i][j].y += x[i].x * y[j].y + x[i].y * y[j].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = r0 + ty * 4 + i, cc = c0 + tx * 4 + j;
      if (rr < n && cc < n) C[((size_t)w * n + rr) * n + cc] = acc[i][j];
    }
}

// Augmented systems [M | b] (row stride n + 1): M = I - (chi~0 + P), b = chi~0 e_0; P = chi~0 F or absent.
__global__ void augment_kernel(int n, int nw, const float2* __restrict__ chi, const float2* __restrict__ prod,
                               float2* __restrict__ aug) {
  const long long total = (long long)nw * n * (n + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t / ((long long)n * (n + 1)));
    const long long rem = t - (long long)w * n * (n + 1);
    const int i = (int)(rem / (n + 1)), j = (int)(rem - (long long)i * (n + 1));
    const float2* cw = chi + (size_t)w * n * n;
    float2 v;
    if (j == n) {
      v = cw[(size_t)i * n];
    } else {
      float2 c = cw[(size_t)i * n + j];
      if (prod) {
        const float2 p = prod[((size_t)w * n + i) * n + j];
        c.x += p.x;
        c.y += p.y;
      }
      v = make_float2((i == j ? 1.f : 0.f) - c.x, -c.y);
    }
    aug[t] = v;
  }
}

// One CTA per frequency: Gaussian elimination with partial pivoting on [M | b], back substitution
// for x, eps_M = 1/(1 + x_0).
__global__ void __launch_bounds__(1024) dyson_solve_kernel(int n, float2* __restrict__ aug,
                                                           double2* __restrict__ eps_m, float2* __restrict__ xbuf) {
  const int w = blockIdx.x, ld = n + 1, tid = threadIdx.x, nt = blockDim.x;
  float2* M = aug + (size_t)w * n * ld;
  float2* x = xbuf + (size_t)w * n;
  __shared__ float red_v[32];
  __shared__ int red_i[32];
  __shared__ int piv;
  __shared__ float2 pivrow_inv;
  extern __shared__ float2 lmul[];                                  // [n] multipliers of the current column
  for (int k = 0; k < n; ++k) {
    // pivot: largest |M[i][k]|, i >= k
    float best = -1.f;
    int bi = k;
    for (int i = k + tid; i < n; i += nt) {
      const float2 v = M[(size_t)i * ld + k];
      const float m = v.x * v.x + v.y * v.y;
      if (m > best) { best = m; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid < 32) {
      best = tid < (nt >> 5) ? red_v[tid] : -1.f;
      bi = tid < (nt >> 5) ? red_i[tid] : k;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) piv = bi;
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = k + tid; j <= n; j += nt) {
        const float2 t0 = M[(size_t)k * ld + j];
        M[(size_t)k * ld + j] = M[(size_t)p * ld + j];
        M[(size_t)p * ld + j] = t0;
      }
    __syncthreads();
    if (tid == 0) {
      const float2 d = M[(size_t)k * ld + k];
      const float m = d.x * d.x + d.y * d.y;
      pivrow_inv = make_float2(d.x / m, -d.y / m);
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < n; i += nt) lmul[i] = cmul(M[(size_t)i * ld + k], pivrow_inv);
    __syncthreads();
    const int cols = n - k;                                         // columns k + 1 .. n
    const long long cnt = (long long)(n - k - 1) * cols;
    for (long long t = tid; t < cnt; t += nt) {
      const int i = k + 1 + (int)(t / cols), j = k + 1 + (int)(t - (long long)(i - k - 1) * cols);
      const float2 l = lmul[i], u = M[(size_t)k * ld + j];
      float2 v = M[(size_t)i * ld + j];
      v.x -= l.x * u.x - l.y * u.y;
      v.y -= l.x * u.y + l.y * u.x;
      M[(size_t)i * ld + j] = v;
    }
    __syncthreads();
  }
  // back substitution, one row at a time from the bottom (block reduction of the row's dot product)
  for (int i = n - 1; i >= 0; --i) {
    float sr = 0.f, si = 0.f;
    for (int j = i + 1 + tid; j < n; j += nt) {
      const float2 m = M[(size_t)i * ld + j], xv = x[j];
      sr += m.x * xv.x - m.y * xv.y;
      si += m.x * xv.y + m.y * xv.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = sr; reinterpret_cast<float*>(red_i)[tid >> 5] = si; }
    __syncthreads();
    if (tid == 0) {
      float tr = 0.f, ti = 0.f;
      for (int u = 0; u < (nt >> 5); ++u) { tr += red_v[u]; ti += reinterpret_cast<float*>(red_i)[u]; }
      const float2 b = M[(size_t)i * ld + n], d = M[(size_t)i * ld + i];
      const float2 num = make_float2(b.x - tr, b.y - ti);
      const float m = d.x * d.x + d.y * d.y;
      x[i] = make_float2((num.x * d.x + num.y * d.y) / m, (num.y * d.x - num.x * d.y) / m);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double re = 1.0 + (double)x[0].x, im = (double)x[0].y;
    const double m = re * re + im * im;
    eps_m[w] = make_double2(re / m, -im / m);
  }
}

// ---------------------------------------------------------------------------- ALDA

__device__ __forceinline__ double lda_fxc(double n) {
  const double kPiD = 3.141592653589793;
  const double fx = -(1.0 / 3.0) * cbrt(3.0 / kPiD) * pow(n, -2.0 / 3.0);
  const double rs = cbrt(3.0 / (4.0 * kPiD * n));
  double d1, d2;
  if (rs >= 1.0) {                               // Perdew-Zunger, gamma / (1 + beta1 sqrt(rs) + beta2 rs)
    const double g = -0.1423, b1 = 1.0529, b2 = 0.3334, sq = sqrt(rs);
    const double D = 1.0 + b1 * sq + b2 * rs, D1 = b1 / (2.0 * sq) + b2, D2 = -b1 / (4.0 * rs * sq);
    d1 = -g * D1 / (D * D);
    d2 = -g * (D2 / (D * D) - 2.0 * D1 * D1 / (D * D * D));
  } else {                                       // A ln rs + B + C rs ln rs + D rs
    const double A = 0.0311, C = 0.0020, Dd = -0.0116;
    d1 = A / rs + C * (log(rs) + 1.0) + Dd;
    d2 = -A / (rs * rs) + C / rs;
  }
  const double fc = -(rs / (3.0 * n)) * ((2.0 / 3.0) * d1 - (rs / 3.0) * d2);
  return fx + fc;
}

// f_xc(r) at every grid point from the valence bands of u(r) in the pair workspace
__global__ void alda_fxc_kernel(DevSys d, const float2* __restrict__ u, double* __restrict__ f, double norm2) {
  const long long nr = (long long)d.n1 * d.n2 * d.n3;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr; r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < d.nkpt; ++k)
      for (int v = 0; v < d.nv; ++v) {
        const float2 x = u[((size_t)k * d.nb + v) * nr + r];
        s += (double)x.x * x.x + (double)x.y * x.y;
      }
    const double n = fmax(norm2 * s, 1e-6);
    f[r] = lda_fxc(n);
  }
}

// One separable DFT pass along axis `ax` of a box whose other two extents are (e1, e2):
// out[j][i1][i2] = sum_x in[x][i1][i2] exp(-2 pi i (j - m) x / N), j = 0 .. 2m, in/out indexed with the
// transformed axis first.  Input real (pass 1) or complex.
__global__ void dft_pass_kernel(const double2* __restrict__ in, double2* __restrict__ out, int N, int m, int e1, int e2,
                                int in_stride_ax, int in_stride_1, int in_stride_2, int out_stride_ax,
                                int out_stride_1, int out_stride_2) {
  const long long total = (long long)(2 * m + 1) * e1 * e2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / ((long long)e1 * e2));
    const int rem = (int)(t - (long long)j * e1 * e2);
    const int i1 = rem / e2, i2 = rem - i1 * e2;
    const int fq = j - m;
    double sr = 0.0, si = 0.0;
    for (int x = 0; x < N; ++x) {
      const double2 v = in[(size_t)x * in_stride_ax + (size_t)i1 * in_stride_1 + (size_t)i2 * in_stride_2];
      double sn, cs;
      sincospi(-2.0 * (double)(((long long)fq * x) % N) / (double)N, &sn, &cs);
      sr += v.x * cs - v.y * sn;
      si += v.x * sn + v.y * cs;
    }
    out[(size_t)j * out_stride_ax + (size_t)i1 * out_stride_1 + (size_t)i2 * out_stride_2] = make_double2(sr, si);
  }
}

__global__ void real_to_complex_kernel(const double* __restrict__ f, double2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2(f[i], 0.0);
}

// F[G][G'] = |G| fhat(G - G') |G'| / (4 pi); fhat on the box [-m1..m1] x [-m2..m2] x [-m3..m3]
__global__ void fxc_matrix_kernel(DevSys d, const double2* __restrict__ fhat, int m1, int m2, int m3, double inv_nr,
                                  float2* __restrict__ F) {
  const int ng = d.ng0;
  const long long total = (long long)ng * ng;
  const double s4pi = 3.5449077018110318;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t / ng), h = (int)(t - (long long)g * ng);
    const char4 a = d.gq[g], b = d.gq[h];
    const int dx = (int)a.x - (int)b.x + m1, dy = (int)a.y - (int)b.y + m2, dz = (int)a.z - (int)b.z + m3;
    const double2 v = fhat[((size_t)dx * (2 * m2 + 1) + dy) * (2 * m3 + 1) + dz];
    const float va = d.vsq[g], vb = d.vsq[h];
    float2 out = make_float2(0.f, 0.f);
    if (va > 0.f && vb > 0.f) {
      const double la = s4pi / va, lb = s4pi / vb;                // |G|, |G'|
      const double s = la * lb * inv_nr / (4.0 * 3.141592653589793);
      out = make_float2((float)(s * v.x), (float)(s * v.y));
    }
    F[t] = out;
  }
}

unsigned blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t chi0_ws_bytes(const DevSys& d) {
  return 2 * align256((size_t)d.dim * d.ng0 * sizeof(float2)) + align256((size_t)d.dim * sizeof(double));
}

int launch_chi0_optical(const DevSys& d, const void* rho_x, const void* P, const double* energies, double delta,
                        const double* omega, int nw, double eta, void* chi0, void* ws, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  float2* a = (float2*)base;
  float2* ab = (float2*)(base + align256((size_t)d.dim * d.ng0 * sizeof(float2)));
  double* de = (double*)(base + 2 * align256((size_t)d.dim * d.ng0 * sizeof(float2)));
  optical_pairs_kernel<<<blocks_for((long long)d.dim * d.ng0, 256), 256, 0, st>>>(
      d, (const float2*)rho_x, (const double2*)P, energies, delta, a, ab, de);
  if (int e = (int)cudaGetLastError()) return e;
  if (nw <= 0) return 0;
  const int nt = (d.ng0 + kT - 1) / kT;
  for (int w0 = 0; w0 < nw; w0 += 65535) {
    const int nwc = nw - w0 < 65535 ? nw - w0 : 65535;
    dim3 grid(nt, nt, nwc);
    chi0_kernel<<<grid, 256, 0, st>>>(d.dim, d.ng0, a, ab, de, omega + w0, eta, 2.0 * d.norm,
                                      (float2*)chi0 + (size_t)w0 * d.ng0 * d.ng0);
    if (int e = (int)cudaGetLastError()) return e;
  }
  return 0;
}

size_t alda_ws_bytes(const DevSys& d) {
  const size_t nr = (size_t)d.n1 * d.n2 * d.n3;
  // f(r) (doubles), then two complex double buffers for the DFT passes (the first holds f as complex)
  return align256(nr * sizeof(double)) + 2 * align256(nr * sizeof(double2));
}

int launch_alda_kernel(const DevSys& d, const void* pair_ws, const int* m, void* F, void* ws, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const long long nr = (long long)d.n1 * d.n2 * d.n3;
  char* base = (char*)ws;
  double* f = (double*)base;
  double2* b0 = (double2*)(base + align256(nr * sizeof(double)));
  double2* b1 = (double2*)(base + align256(nr * sizeof(double)) + align256(nr * sizeof(double2)));
  alda_fxc_kernel<<<blocks_for(nr, 256), 256, 0, st>>>(d, (const float2*)pair_ws, f, 2.0 * d.norm);
  if (int e = (int)cudaGetLastError()) return e;
  real_to_complex_kernel<<<blocks_for(nr, 256), 256, 0, st>>>(f, b0, nr);
  if (int e = (int)cudaGetLastError()) return e;
  const int m1 = m[0], m2 = m[1], m3 = m[2];
  const int w1 = 2 * m1 + 1, w2 = 2 * m2 + 1, w3 = 2 * m3 + 1;
  // pass 1, x: b0 [x][y][z] -> b1 [j1][y][z]
  dft_pass_kernel<<<blocks_for((long long)w1 * d.n2 * d.n3, 128), 128, 0, st>>>(
      b0, b1, d.n1, m1, d.n2, d.n3, d.n2 * d.n3, d.n3, 1, d.n2 * d.n3, d.n3, 1);
  if (int e = (int)cudaGetLastError()) return e;
  // pass 2, y: b1 [j1][y][z] -> b0 [j1][j2][z]   (transformed axis y; other axes j1 (e1), z (e2))
  dft_pass_kernel<<<blocks_for((long long)w2 * w1 * d.n3, 128), 128, 0, st>>>(
      b1, b0, d.n2, m2, w1, d.n3, d.n3, d.n2 * d.n3, 1, d.n3, w2 * d.n3, 1);
  if (int e = (int)cudaGetLastError()) return e;
  // pass 3, z: b0 [j1][j2][z] -> b1 [j1][j2][j3]
  dft_pass_kernel<<<blocks_for((long long)w3 * w1 * w2, 128), 128, 0, st>>>(
      b0, b1, d.n3, m3, w1, w2, 1, w2 * d.n3, d.n3, 1, w2 * w3, w3);
  if (int e = (int)cudaGetLastError()) return e;
  fxc_matrix_kernel<<<blocks_for((long long)d.ng0 * d.ng0, 256), 256, 0, st>>>(d, b1, m1, m2, m3, 1.0 / (double)nr,
                                                                             (float2*)F);
  return (int)cudaGetLastError();
}

size_t epsm_ws_bytes(const DevSys& d, long long nw) {
  const size_t n = d.ng0;
  return align256((size_t)nw * n * (n + 1) * sizeof(float2)) + align256((size_t)nw * n * n * sizeof(float2)) +
         align256((size_t)nw * n * sizeof(float2));
}

int launch_epsilon_macro(const DevSys& d, const void* chi0, const void* F, int nw, void* eps_m, void* ws,
                         void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int n = d.ng0;
  char* base = (char*)ws;
  float2* aug = (float2*)base;
  float2* prod = (float2*)(base + align256((size_t)nw * n * (n + 1) * sizeof(float2)));
  float2* xb = (float2*)(base + align256((size_t)nw * n * (n + 1) * sizeof(float2)) +
                         align256((size_t)nw * n * n * sizeof(float2)));
  if (F) {
    const int nt = (n + kT - 1) / kT;
    for (int w0 = 0; w0 < nw; w0 += 65535) {
      const int nwc = nw - w0 < 65535 ? nw - w0 : 65535;
      batched_gemm_kernel<<<dim3(nt, nt, nwc), 256, 0, st>>>(n, (const float2*)chi0 + (size_t)w0 * n * n,
                                                             (const float2*)F, prod + (size_t)w0 * n * n);
      if (int e = (int)cudaGetLastError()) return e;
    }
  }
  augment_kernel<<<blocks_for((long long)nw * n * (n + 1), 256), 256, 0, st>>>(n, nw, (const float2*)chi0,
                                                                              F ? prod : nullptr, aug);
  if (int e = (int)cudaGetLastError()) return e;
  const size_t sm = (size_t)n * sizeof(float2);
  if (sm > 48 * 1024) {
    if (int e = (int)cudaFuncSetAttribute((const void*)dyson_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm))
      return e;
  }
  dyson_solve_kernel<<<nw, 1024, sm, st>>>(n, aug, (double2*)eps_m, xb);
  return (int)cudaGetLastError();
}

}  // namespace bse
