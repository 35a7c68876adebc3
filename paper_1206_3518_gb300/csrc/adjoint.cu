// Adjoint of a spectral loss (step A9).
//
// eps_2(w) = -C Im[P^H R(z) P], R(z) = (z - H)^{-1}, z = w + i eta (Eq. epsilon_chi_bar in
// the TDA, Appendix A resolvent).  For g(w) = dL/deps_2(w) and any perturbation dH,
// dL = Re sum_ij conj(G_ij) dH_ij with G = -C sum_w g(w) i xt(w) x(w)^H, x = R(z)P,
// xt = R(conj z)P.  The Lanczos basis V (rows v_j) is recomputed, H V^T ~ V^T T, and
// R(z)P ~ |P| V^T y(z) with y(z) = (z - T)^{-1} e_0, so xt = |P| V^T conj(y).  The
// Hermitian part of G, the gradient for Hermitian perturbations of H, is then
//   G_h = V^T M_h conj(V),  M_h[j][l] = -C |P|^2 sum_w g(w) Im(y_j(w) y_l(w))   (real symmetric),
// and dL/dDelta = Re tr G = tr M_h (orthonormal basis).  y(z) is obtained stably from the
// tail continued fractions t_j = 1/(z - a_j - b_{j+1}^2 t_{j+1}): y_0 = t_0, y_j = b_j t_j y_{j-1}.
//
// Chain to the kernel inputs (H = diag + 2K^x - K^d, upper blocks k <= k' mirrored; the
// effective gradient of an upper block is 2 G_h for k < k' and G_h for k = k'):
//   dL/drho_x[S][G]   = 4 vbar(G)/(Omega Nk) sum_S' G_h[S'][S] rho_x[S'][G]
//   per upper block, Gm[vv'][cc'] = block gradient at ((k,v,c),(k',v',c')):
//   dL/drho_cc'[cc'] = -(1/(Omega Nk)) sum_vv' Gm[vv'][cc'] (W rho_vv')
//   dL/drho_vv'[vv'] = -(1/(Omega Nk)) sum_cc' conj(Gm[vv'][cc']) (W rho_cc')
//   dL/dW_q          = -(1/(Omega Nk)) sum_blocks sum_cc' Y[cc'] rho_cc'^H,  Y[cc'] = sum_vv' Gm rho_vv'
// every stored entry of rho and W taken as a free variable.
#include <cuda_runtime.h>

#include <algorithm>

#include "gemm_tile.cuh"
#include "internal.h"

namespace bse {
namespace {

constexpr int kNwChunk = 256;       // frequencies per resolvent chunk
constexpr int kQChunk = 32;         // q points per direct-term chunk

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BwdLayout {
  size_t spec, eps2, ab, done, scal, Y, Mh, Mf, Vf, Zf, Gh, Xv, Xc, Yd, total;
  long long rows_v, rows_c;
};

BwdLayout bwd_layout(const DevSys& d, long long nsteps) {
  BwdLayout L;
  const long long qc = kQChunk < d.nq ? kQChunk : d.nq;
  long long nb = qc * d.nkpt;
  if (nb > d.nblocks) nb = d.nblocks;
  L.rows_v = nb * d.nv * d.nv;
  L.rows_c = nb * d.nc * d.nc;
  size_t o = 0;
  L.spec = o; o = a256(o + spectrum_ws_bytes(d, nsteps));
  L.eps2 = o; o = a256(o + 8 * (size_t)kNwChunk);
  L.ab = o; o = a256(o + 16 * (size_t)nsteps);
  L.done = o; o = a256(o + 16);
  L.scal = o; o = a256(o + 64);
  L.Y = o; o = a256(o + 16 * (size_t)kNwChunk * nsteps);
  L.Mh = o; o = a256(o + 8 * (size_t)nsteps * nsteps);
  L.Mf = o; o = a256(o + 8 * (size_t)nsteps * nsteps);
  L.Vf = o; o = a256(o + 8 * (size_t)nsteps * d.dim);
  L.Zf = o; o = a256(o + 8 * (size_t)nsteps * d.dim);
  L.Gh = o; o = a256(o + 8 * (size_t)d.dim * d.dim);
  L.Xv = o; o = a256(o + 8 * (size_t)L.rows_v * d.ng_max);
  L.Xc = o; o = a256(o + 8 * (size_t)L.rows_c * d.ng_max);
  L.Yd = o; o = a256(o + 8 * (size_t)L.rows_c * d.ng_max);
  L.total = o;
  return L;
}

__global__ void norm2_kernel(const double2* __restrict__ P, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += P[i].x * P[i].x + P[i].y * P[i].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[0] = t;
  }
}

// y(w) = (z - T)^{-1} e_0 for the frequencies of one chunk; Y[w][j], j < n.
__global__ void resolvent_kernel(const double* __restrict__ ab, int nsteps, const int* __restrict__ done,
                                 const double* __restrict__ omega, int w0, int nwc, double eta,
                                 double2* __restrict__ Y) {
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= nwc) return;
  const int n = *done;
  const double zr = omega[w0 + wi], zi = eta;
  double2* y = Y + (size_t)wi * nsteps;
  double tr = 0.0, ti = 0.0;
  for (int j = n - 1; j >= 0; --j) {                 // tail fractions t_j
    double dr = zr - ab[j], di = zi;
    if (j + 1 < n) {
      const double b2 = ab[nsteps + j + 1] * ab[nsteps + j + 1];
      dr -= b2 * tr;
      di -= b2 * ti;
    }
    const double den = dr * dr + di * di;
    tr = dr / den;
    ti = -di / den;
    y[j] = make_double2(tr, ti);
  }
  double2 prev = y[0];                                // y_0 = t_0
  for (int j = 1; j < n; ++j) {
    const double b = ab[nsteps + j];
    const double2 t = y[j];
    const double2 cur = make_double2(b * (t.x * prev.x - t.y * prev.y), b * (t.x * prev.y + t.y * prev.x));
    y[j] = cur;
    prev = cur;
  }
}

// Mh[j][l] += -C |P|^2 sum_{w in chunk} g(w) Im(y_j y_l)  (j <= l, mirrored).
__global__ void mh_kernel(const double2* __restrict__ Y, int nsteps, const int* __restrict__ done,
                          const double* __restrict__ g, int w0, int nwc, const double* __restrict__ scal, double cpref,
                          double* __restrict__ Mh) {
  const int n = *done;
  const int j = blockIdx.y * 16 + threadIdx.y, l = blockIdx.x * 16 + threadIdx.x;
  if (j >= n || l >= n || j > l) return;
  double s = 0.0;
  for (int w = 0; w < nwc; ++w) {
    const double2 a = Y[(size_t)w * nsteps + j], b = Y[(size_t)w * nsteps + l];
    s += g[w0 + w] * (a.x * b.y + a.y * b.x);
  }
  const double v = -cpref * scal[0] * s;
  Mh[(size_t)j * nsteps + l] += v;
  if (j != l) Mh[(size_t)l * nsteps + j] += v;
}

// dL/dDelta = tr Mh; Mf = (complex64) Mh; Vf = (complex64) V.
__global__ void finish_m_kernel(const double* __restrict__ Mh, int nsteps, const int* __restrict__ done,
                                double* __restrict__ d_delta, float2* __restrict__ Mf) {
  const int n = *done;
  __shared__ double red[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += Mh[(size_t)j * nsteps + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  for (int i = threadIdx.x; i < nsteps * nsteps; i += blockDim.x) {
    const int j = i / nsteps, l = i % nsteps;
    Mf[i] = make_float2((j < n && l < n) ? (float)Mh[i] : 0.f, 0.f);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *d_delta = t;
  }
}

// Vf = FP32 basis (the hi parts of the double-float split), zero beyond the steps done.
__global__ void v_to_float_kernel(const float4* __restrict__ V, long long n, const int* __restrict__ done, int dim,
                                  float2* __restrict__ Vf) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = (int)(i / dim);
  const float4 v = V[i];
  Vf[i] = (j < *done) ? make_float2(v.x + v.y, v.z + v.w) : make_float2(0.f, 0.f);
}

// Generic grouped product C = opA(A) opB(B)^T with per-column epilogue scale (dense, one group).
template <bool A_KC, bool B_KC, bool CA, bool CB>
__global__ __launch_bounds__(gemm::kThreads) void gemm_kernel(const float2* __restrict__ A, long long lda, int M,
                                                             const float2* __restrict__ B, long long ldb, int N, int K,
                                                             float2* __restrict__ C, long long ldc, float alpha,
                                                             const float* __restrict__ colscale2) {
  const int m0 = blockIdx.y * gemm::BM, n0 = blockIdx.x * gemm::BN;
  if (m0 >= M || n0 >= N) return;
  __shared__ gemm::Smem sm;
  float2 acc[4][4];
  gemm::tile<A_KC, B_KC, CA, CB>(A, lda, M, B, ldb, N, K, m0, n0, sm, acc);
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + tm * 4 + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tn * 4 + j;
      if (c >= N) continue;
      float sc = alpha;
      if (colscale2) sc *= colscale2[c] * colscale2[c];
      C[(size_t)r * ldc + c] = make_float2(sc * acc[i][j].x, sc * acc[i][j].y);
    }
  }
}

// dW_q[G][G'] = -norm sum_k Y_q[k][G] conj(Rc_q[k][G'])  grouped over the q chunk.
__global__ __launch_bounds__(gemm::kThreads) void gemm_dw_kernel(DevSys d, const float2* __restrict__ Yd,
                                                                const float2* __restrict__ rho_dir,
                                                                float2* __restrict__ dW, int q_begin) {
  const int q = q_begin + blockIdx.z;
  const long long b0 = d.qblk_off[q_begin];
  const long long nblk = d.qblk_off[q + 1] - d.qblk_off[q];
  const int nc2 = d.nc * d.nc, NG = d.ngq[q];
  const int K = (int)(nblk * nc2);
  const int m0 = blockIdx.y * gemm::BM, n0 = blockIdx.x * gemm::BN;
  if (m0 >= NG || n0 >= NG || K == 0) return;
  const float2* A = Yd + (size_t)((d.qblk_off[q] - b0) * nc2) * d.ng_max;
  const float2* B = rho_dir + (size_t)(d.qvec_off[q] + nblk * d.nv * d.nv) * d.ng_max;
  __shared__ gemm::Smem sm;
  float2 acc[4][4];
  gemm::tile<false, false, false, true>(A, d.ng_max, NG, B, d.ng_max, NG, K, m0, n0, sm, acc);
  float2* C = dW + (size_t)q * d.ng_max * d.ng_max;
  const float nrm = -(float)d.norm;
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + tm * 4 + i;
    if (r >= NG) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tn * 4 + j;
      if (c < NG) C[(size_t)r * d.ng_max + c] = make_float2(nrm * acc[i][j].x, nrm * acc[i][j].y);
    }
  }
}

// Per upper block of the chunk: block gradient Gm, dL/drho_vv', dL/drho_cc' and Y = Gm-weighted rho_vv'.
__global__ __launch_bounds__(256) void block_grad_kernel(DevSys d, const float2* __restrict__ Gh,
                                                         const float2* __restrict__ rho_dir,
                                                         const float2* __restrict__ Xv, const float2* __restrict__ Xc,
                                                         float2* __restrict__ drho_dir, float2* __restrict__ Yd,
                                                         int q_begin) {
  __shared__ float2 Gm[16][16];
  const long long b0 = d.qblk_off[q_begin];
  const long long b = b0 + blockIdx.x;
  const int4 blk = d.blocks[b];
  const int k = blk.x, k2 = blk.y, q = blk.z;
  const long long qb = d.qblk_off[q];
  const long long nblk = d.qblk_off[q + 1] - qb;
  const long long local = b - qb;
  const int nv = d.nv, nc = d.nc, nv2 = nv * nv, nc2 = nc * nc, nvc = nv * nc;
  const float fac = (k == k2) ? 1.f : 2.f;
  for (int t = threadIdx.x; t < nv2 * nc2; t += blockDim.x) {
    const int a = t / nc2, c = t % nc2;
    const int v = a / nv, vp = a % nv, cc = c / nc, cp = c % nc;
    const float2 g = Gh[(size_t)(k * nvc + v * nc + cc) * d.dim + (size_t)k2 * nvc + vp * nc + cp];
    Gm[a][c] = make_float2(fac * g.x, fac * g.y);
  }
  __syncthreads();
  const long long vq = d.qvec_off[q];
  const float2* Rv = rho_dir + (size_t)(vq + local * nv2) * d.ng_max;
  float2* dRv = drho_dir ? drho_dir + (size_t)(vq + local * nv2) * d.ng_max : nullptr;
  float2* dRc = drho_dir ? drho_dir + (size_t)(vq + nblk * nv2 + local * nc2) * d.ng_max : nullptr;
  const float2* xv = Xv + (size_t)((qb - b0 + local) * nv2) * d.ng_max;
  const float2* xc = Xc + (size_t)((qb - b0 + local) * nc2) * d.ng_max;
  float2* y = Yd + (size_t)((qb - b0 + local) * nc2) * d.ng_max;
  const int NG = d.ngq[q];
  const float nrm = (float)d.norm;
  for (int G = threadIdx.x; G < NG; G += blockDim.x) {
    float2 rv[16], xvv[16], xcc[16];
    for (int a = 0; a < nv2; ++a) {
      rv[a] = Rv[(size_t)a * d.ng_max + G];
      xvv[a] = xv[(size_t)a * d.ng_max + G];
    }
    for (int c = 0; c < nc2; ++c) xcc[c] = xc[(size_t)c * d.ng_max + G];
    for (int c = 0; c < nc2; ++c) {
      float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
      for (int a = 0; a < nv2; ++a) {
        const float2 g = Gm[a][c];
        s1.x += g.x * xvv[a].x - g.y * xvv[a].y;
        s1.y += g.x * xvv[a].y + g.y * xvv[a].x;
        s2.x += g.x * rv[a].x - g.y * rv[a].y;
        s2.y += g.x * rv[a].y + g.y * rv[a].x;
      }
      if (dRc) dRc[(size_t)c * d.ng_max + G] = make_float2(-nrm * s1.x, -nrm * s1.y);
      y[(size_t)c * d.ng_max + G] = s2;
    }
    if (dRv) {
      for (int a = 0; a < nv2; ++a) {
        float2 s = make_float2(0.f, 0.f);
        for (int c = 0; c < nc2; ++c) {
          const float2 g = Gm[a][c];            // conj(g) * xc
          s.x += g.x * xcc[c].x + g.y * xcc[c].y;
          s.y += g.x * xcc[c].y - g.y * xcc[c].x;
        }
        dRv[(size_t)a * d.ng_max + G] = make_float2(-nrm * s.x, -nrm * s.y);
      }
    }
  }
}

}  // namespace

size_t backward_ws_bytes(const DevSys& d, long long nsteps) { return bwd_layout(d, nsteps).total; }



int launch_backward(const DevSys& d, const long long* h_qblk_off, const long long* h_qvec_off, const void* H,
                    const void* P, int nsteps, const double* omega, int nw, double eta, const double* dL,
                    const void* rho_x, const void* rho_dir, const void* W, double* d_delta, void* dH, void* drho_x,
                    void* drho_dir, void* dW, void* ws, int* status, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const BwdLayout L = bwd_layout(d, nsteps);
  char* base = (char*)ws;
  double* ab = (double*)(base + L.ab);
  int* done = (int*)(base + L.done);
  double* scal = (double*)(base + L.scal);
  double2* Y = (double2*)(base + L.Y);
  double* Mh = (double*)(base + L.Mh);
  float2* Mf = (float2*)(base + L.Mf);
  float2* Vf = (float2*)(base + L.Vf);
  float2* Zf = (float2*)(base + L.Zf);
  float2* Gh = dH ? (float2*)dH : (float2*)(base + L.Gh);
  float4* V = nullptr;
  // 1. Lanczos recomputed (the spectrum it evaluates on the first frequencies is not used).
  int e = run_haydock(d, H, P, nsteps, omega, nw < kNwChunk ? nw : kNwChunk, eta, (double*)(base + L.eps2), ab, done,
                      base + L.spec, status, stream, &V);
  if (e) return e;
  norm2_kernel<<<1, 1024, 0, st>>>((const double2*)P, d.dim, scal);
  // 2. M_h from the Krylov resolvent, chunked over frequencies.
  if ((e = (int)cudaMemsetAsync(Mh, 0, 8 * (size_t)nsteps * nsteps, st))) return e;
  for (int w0 = 0; w0 < nw; w0 += kNwChunk) {
    const int nwc = (nw - w0) < kNwChunk ? (nw - w0) : kNwChunk;
    resolvent_kernel<<<(nwc + 127) / 128, 128, 0, st>>>(ab, nsteps, done, omega, w0, nwc, eta, Y);
    dim3 g16((nsteps + 15) / 16, (nsteps + 15) / 16);
    mh_kernel<<<g16, dim3(16, 16), 0, st>>>(Y, nsteps, done, dL, w0, nwc, scal, d.prefactor, Mh);
  }
  finish_m_kernel<<<1, 1024, 0, st>>>(Mh, nsteps, done, d_delta, Mf);
  const long long nv_el = (long long)nsteps * d.dim;
  v_to_float_kernel<<<(unsigned)((nv_el + 255) / 256), 256, 0, st>>>(V, nv_el, done, d.dim, Vf);
  if ((e = (int)cudaGetLastError())) return e;
  // 3. Z = M_h conj(V) (n x dim), G_h = V^T Z (dim x dim), FP32 products.
  {
    dim3 gz((d.dim + 63) / 64, (nsteps + 63) / 64);
    gemm_kernel<true, false, false, true><<<gz, gemm::kThreads, 0, st>>>(Mf, nsteps, nsteps, Vf, d.dim, d.dim, nsteps,
                                                                        Zf, d.dim, 1.f, nullptr);
    dim3 gg((d.dim + 63) / 64, (d.dim + 63) / 64);
    gemm_kernel<false, false, false, false><<<gg, gemm::kThreads, 0, st>>>(Vf, d.dim, d.dim, Zf, d.dim, d.dim, nsteps,
                                                                          Gh, d.dim, 1.f, nullptr);
    if ((e = (int)cudaGetLastError())) return e;
  }
  // 4. exchange: dL/drho_x[S][G] = 2 xscale(G)^2 sum_S' conj(G_h[S][S']) rho_x[S'][G]
  if (drho_x) {
    if ((e = (int)cudaMemsetAsync(drho_x, 0, 8 * (size_t)d.dim * d.ng_max, st))) return e;
    dim3 gx((d.ng0 + 63) / 64, (d.dim + 63) / 64);
    gemm_kernel<true, false, true, false><<<gx, gemm::kThreads, 0, st>>>(
        Gh, d.dim, d.dim, (const float2*)rho_x, d.ng_max, d.ng0, d.dim, (float2*)drho_x, d.ng_max, 2.f, d.xscale);
    if ((e = (int)cudaGetLastError())) return e;
  }
  // 5. direct term, q chunks
  if (drho_dir || dW) {
    if (drho_dir && (e = (int)cudaMemsetAsync(drho_dir, 0, 8 * (size_t)h_qvec_off[d.nq] * d.ng_max, st))) return e;
    if (dW && (e = (int)cudaMemsetAsync(dW, 0, 8 * (size_t)d.nq * d.ng_max * d.ng_max, st))) return e;
    float2* Xv = (float2*)(base + L.Xv);
    float2* Xc = (float2*)(base + L.Xc);
    float2* Yd = (float2*)(base + L.Yd);
    for (int q0 = 0; q0 < d.nq; q0 += kQChunk) {
      const int q1 = (q0 + kQChunk) < d.nq ? q0 + kQChunk : d.nq;
      long long maxb = 0;
      for (int q = q0; q < q1; ++q) maxb = std::max(maxb, h_qblk_off[q + 1] - h_qblk_off[q]);
      if ((e = launch_gemm_wr(d, rho_dir, q0, q1, 0, maxb * d.nv * d.nv, W, Xv, 0, stream))) return e;
      if ((e = launch_gemm_wr(d, rho_dir, q0, q1, 0, maxb * d.nc * d.nc, W, Xc, 1, stream))) return e;
      const long long nb = h_qblk_off[q1] - h_qblk_off[q0];
      if (nb > 0)
        block_grad_kernel<<<(unsigned)nb, 256, 0, st>>>(d, Gh, (const float2*)rho_dir, Xv, Xc, (float2*)drho_dir, Yd,
                                                        q0);
      if (dW) {
        dim3 gw((d.ng_max + 63) / 64, (d.ng_max + 63) / 64, q1 - q0);
        gemm_dw_kernel<<<gw, gemm::kThreads, 0, st>>>(d, Yd, (const float2*)rho_dir, (float2*)dW, q0);
      }
      if ((e = (int)cudaGetLastError())) return e;
    }
  }
  return 0;
}

}  // namespace bse
