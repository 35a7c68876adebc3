// Kernel contractions and Hamiltonian assembly, CUDA-core FP32 form (steps A3-A5).
//
// Eq. kernel (TDA, singlet):  H = diag(e_c + Delta - e_v) + 2 K^x - K^d
//   K^x_SS' = (1/(Omega Nk)) sum_{G != 0} conj(rho_vc^{kk}(G)) vbar(G) rho_v'c'^{k'k'}(G)   (Eq. V_eh)
//   K^d_SS' = (1/(Omega Nk)) sum_{G,G'} conj(rho_vv'^{kk'}(G)) W_GG'(q) rho_cc'^{kk'}(G')  (Eq. W_SS)
//
// init_kernel   : 2K^x + diag on every tile that touches the upper block triangle; the
//                 exchange scale sqrt(2 vbar/(Omega Nk)) is applied to both operands.
// gemm_wr       : per q, X = W(q) R for the smaller band side (grouped over the q chunk),
//                 stored as X^T rows [col][G] (G contiguous); its own register-blocked tile.
// block_kernel  : per upper block (k <= k'), M = X^H R of the other side (K = NG_q),
//                 H_kk' = H_kk' - M/(Omega Nk) and the mirror H_k'k = H_kk'^H;
//                 diagonal blocks become (B + B^H)/2.
// init_kernel uses the tiled FP32 complex "NT" core of gemm_tile.cuh: C[m][n] =
// sum_k opA(A[m][k]) B[n][k] with both operands K-contiguous.
#include <cuda_runtime.h>

#include "gemm_tile.cuh"
#include "internal.h"
#include "layout.cuh"

namespace bse {
namespace {

using gemm::BM;
using gemm::BN;
constexpr int kGemmThreads = gemm::kThreads;

__device__ __forceinline__ int kpt_of_pair(const DevSys& d, int S) { return S / (d.nv * d.nc); }

// H[S][S'] = 2 K^x + delta_SS' (e_c + Delta - e_v) on tiles touching k(S) <= k(S').
__global__ __launch_bounds__(kGemmThreads) void init_kernel(DevSys d, const float2* __restrict__ rho_x,
                                                            const double* __restrict__ e, double delta,
                                                            float2* __restrict__ H) {
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= d.dim || n0 >= d.dim) return;
  if (kpt_of_pair(d, m0) > kpt_of_pair(d, min(n0 + BN, d.dim) - 1)) return;   // strictly lower block triangle
  __shared__ gemm::Smem sm;
  float2 acc[4][4];
  gemm::tile<true, true, true, false, true>(rho_x, d.ng_max, d.dim, rho_x, d.ng_max, d.dim, d.ng0, m0, n0, sm, acc,
                                            d.xscale);
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int S = m0 + tm * 4 + i;
    if (S >= d.dim) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int S2 = n0 + tn * 4 + j;
      if (S2 >= d.dim) continue;
      float2 v = acc[i][j];
      if (S == S2) {
        const int ic = S % d.nc, iv = (S / d.nc) % d.nv, k = S / (d.nv * d.nc);
        v.x += (float)(e[(size_t)k * d.nb + d.nv + ic] + delta - e[(size_t)k * d.nb + iv]);
      }
      H[(size_t)S * d.dim + S2] = v;
    }
  }
}

// Grouped over the q chunk: X_q^T[col][G] = sum_G' R_q[col][G'] W_q[G][G']  (W Hermitian).
// Tile 128 rows x 64 columns, K in steps of 16 complex; 256 threads, each 8 rows x 4 columns.
// Operands are staged transposed ([k][row]) in shared memory so that a thread reads its 8
// A values and 4 B values of one k with float4 loads; the next K step is prefetched into
// registers while the current one is consumed (two shared buffers, one barrier per step).
namespace wr {
constexpr int TM = 128, TN = 64, TK = 16, kThreads = 256;
struct Smem {                   // 48 KB: two K steps of both operands
  float2 a[2][TK][TM];
  float2 b[2][TK][TN];
};
}  // namespace wr

__global__ __launch_bounds__(wr::kThreads, 2) void gemm_wr(DevSys d, const float2* __restrict__ rho_dir,
                                                          const float2* __restrict__ W, float2* __restrict__ X,
                                                          int q_begin, long long vbase, int side_c) {
  using namespace wr;
  const int q = q_begin + blockIdx.z;
  const long long b0 = d.qblk_off[q_begin];
  const long long nblk = d.qblk_off[q + 1] - d.qblk_off[q];
  const int w = side_width(d, side_c);
  const int M = (int)(nblk * w), NG = d.ngq[q];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (m0 >= M || n0 >= NG) return;
  const float2* A = rho_dir + (size_t)side_rows_offset(d, q, side_c, vbase) * d.ng_max;
  const float2* B = W + (size_t)q * d.ng_max * d.ng_max;
  float2* C = X + (size_t)((d.qblk_off[q] - b0) * w) * d.ng_max;
  __shared__ __align__(16) Smem sm;
  const int t = threadIdx.x;
  const int tm = t / 16, tn = t % 16;
  // staging assignment: A row t/2, K half t%2 (8 values); B row t/4, K quarter t%4 (4 values)
  const int ar = t >> 1, ah = (t & 1) * 8, br = t >> 2, bq = (t & 3) * 4;
  const bool a_in = m0 + ar < M, b_in = n0 + br < NG;
  const float2* Ap = A + (size_t)(m0 + ar) * d.ng_max;
  const float2* Bp = B + (size_t)(n0 + br) * d.ng_max;
  float2 ra[8], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + ah + i;
      ra[i] = (a_in && k < NG) ? Ap[k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + bq + i;
      rb[i] = (b_in && k < NG) ? Bp[k] : make_float2(0.f, 0.f);
    }
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.a[buf][ah + i][ar] = ra[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) sm.b[buf][bq + i][br] = rb[i];
  };
  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  fetch(0);
  put(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < NG; k0 += TK) {
    const bool more = k0 + TK < NG;
    if (more) fetch(k0 + TK);
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      float2 av[8], bv[4];
      const float4* pa = reinterpret_cast<const float4*>(&sm.a[buf][k][tm * 8]);
      const float4* pb = reinterpret_cast<const float4*>(&sm.b[buf][k][tn * 4]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = pa[i];
        av[2 * i] = make_float2(v.x, v.y);
        av[2 * i + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float4 v = pb[j];
        bv[2 * j] = make_float2(v.x, v.y);
        bv[2 * j + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, acc[i][j].y));
        }
    }
    if (more) {
      put(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + tm * 8 + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tn * 4 + j;
      if (c < NG) C[(size_t)r * d.ng_max + c] = acc[i][j];
    }
  }
}

constexpr int kBlkThreads = 256, KC = 32;
constexpr int kBlkPerCta = 4, kBlkT = kBlkThreads / kBlkPerCta;   // block_kernel: 64 threads per block

// Per upper block: M[a][c] = sum_G conj(L[a][G]) Rr[c][G], a = (v,v'), c = (c,c');
// side V: L = X (= W R_v), Rr = R_c;  side C: L = R_v, Rr = X (= W R_c).
// Four blocks per CTA, 64 threads per block, each thread a 2 x 2 patch of the (at most 16 x 16) product:
// four shared-memory loads per four complex multiply-adds, sixteen global loads per thread in flight
// per K step.
__global__ __launch_bounds__(kBlkThreads) void block_kernel(DevSys d, const float2* __restrict__ rho_dir,
                                                           const float2* __restrict__ X, float2* __restrict__ H,
                                                           int q_begin, long long vbase, int side_c, long long b_count) {
  __shared__ float2 Ls[kBlkPerCta][16][KC + 1];
  __shared__ float2 Rs[kBlkPerCta][16][KC + 1];
  __shared__ float2 Bs[kBlkPerCta][16][17];
  __shared__ int ngs[kBlkPerCta];
  const int grp = threadIdx.x / kBlkT, t = threadIdx.x % kBlkT;
  const long long bi = (long long)blockIdx.x * kBlkPerCta + grp;
  const bool live = bi < b_count;
  const long long b0 = d.qblk_off[q_begin];
  const long long b = b0 + (live ? bi : 0);
  const int4 blk = d.blocks[b];
  const int k = blk.x, k2 = blk.y, q = blk.z;
  const long long qb = d.qblk_off[q];
  const long long nblk = d.qblk_off[q + 1] - qb;
  const long long local = b - qb;
  const int nv2 = d.nv * d.nv, nc2 = d.nc * d.nc;
  const long long vbase_q = d.qvec_off[q] - vbase;
  const float2* Rv = rho_dir + (size_t)(vbase_q + local * nv2) * d.ng_max;
  const float2* Rc = rho_dir + (size_t)(vbase_q + nblk * nv2 + local * nc2) * d.ng_max;
  const int w = side_c ? nc2 : nv2;
  const float2* Xb = X + (size_t)((qb - b0 + local) * w) * d.ng_max;
  const float2* L = side_c ? Rv : Xb;
  const float2* R = side_c ? Xb : Rc;
  const int NG = live ? d.ngq[q] : 0;
  if (t == 0) ngs[grp] = NG;
  __syncthreads();
  int ngmax = 0;
#pragma unroll
  for (int i = 0; i < kBlkPerCta; ++i) ngmax = max(ngmax, ngs[i]);
  const int i2 = t >> 3, j2 = t & 7;                 // rows a = 2 i2, 2 i2 + 1; columns c = 2 j2, 2 j2 + 1
  float2 acc[2][2];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) acc[x][y] = make_float2(0.f, 0.f);
  for (int g0 = 0; g0 < ngmax; g0 += KC) {
    for (int i = t; i < 16 * KC; i += kBlkT) {
      const int r = i / KC, g = i % KC;
      const bool in = (g0 + g) < NG;
      Ls[grp][r][g] = (r < nv2 && in) ? L[(size_t)r * d.ng_max + g0 + g] : make_float2(0.f, 0.f);
      Rs[grp][r][g] = (r < nc2 && in) ? R[(size_t)r * d.ng_max + g0 + g] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int g = 0; g < KC; ++g) {
      const float2 l0 = Ls[grp][2 * i2][g], l1 = Ls[grp][2 * i2 + 1][g];
      const float2 r0 = Rs[grp][2 * j2][g], r1 = Rs[grp][2 * j2 + 1][g];
      const float2 lv[2] = {l0, l1}, rv[2] = {r0, r1};
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          acc[x][y].x = fmaf(lv[x].x, rv[y].x, fmaf(lv[x].y, rv[y].y, acc[x][y].x));     // conj(l) r
          acc[x][y].y = fmaf(lv[x].x, rv[y].y, fmaf(-lv[x].y, rv[y].x, acc[x][y].y));
        }
    }
    __syncthreads();
  }
  const int nv = d.nv, nc = d.nc, nvc = nv * nc;
  const float nrm = (float)d.norm;
  int rows[2][2], colsv[2][2];
  float2 vals[2][2];
  bool act[2][2];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int a = 2 * i2 + x, c = 2 * j2 + y;
      act[x][y] = live && a < nv2 && c < nc2;
      rows[x][y] = colsv[x][y] = 0;
      vals[x][y] = make_float2(0.f, 0.f);
      if (!act[x][y]) continue;
      const int v = a / nv, vp = a % nv, cc = c / nc, cp = c % nc;
      const int row = v * nc + cc;                 // (k, v, c) local
      const int col = vp * nc + cp;                // (k', v', c') local
      rows[x][y] = row;
      colsv[x][y] = col;
      const size_t hij = (size_t)(k * nvc + row) * d.dim + (size_t)k2 * nvc + col;
      const float2 h = H[hij];
      const float2 val = make_float2(h.x - nrm * acc[x][y].x, h.y - nrm * acc[x][y].y);
      vals[x][y] = val;
      if (k != k2) {
        H[hij] = val;
        H[(size_t)(k2 * nvc + col) * d.dim + (size_t)k * nvc + row] = make_float2(val.x, -val.y);
      } else {
        Bs[grp][row][col] = val;
      }
    }
  __syncthreads();
  if (k == k2) {
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        if (!act[x][y]) continue;
        const int row = rows[x][y], col = colsv[x][y];
        const float2 o = Bs[grp][col][row];
        H[(size_t)(k * nvc + row) * d.dim + (size_t)k * nvc + col] =
            make_float2(0.5f * (vals[x][y].x + o.x), 0.5f * (vals[x][y].y - o.y));
      }
  }
}

// Lower blocks from the upper ones, H_k'k = H_kk'^H, and diagonal blocks (B + B^H)/2 (for a build
// without the direct term, which otherwise does this in its epilogue).
__global__ void mirror_kernel(DevSys d, float2* __restrict__ H) {
  const long long n = (long long)d.dim * d.dim;
  const int nvc = d.nv * d.nc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int S = (int)(i / d.dim), S2 = (int)(i - (long long)S * d.dim);
    const int k = S / nvc, k2 = S2 / nvc;
    if (k > k2) {
      const float2 u = H[(size_t)S2 * d.dim + S];
      H[i] = make_float2(u.x, -u.y);
    } else if (k == k2 && S < S2) {
      const float2 a = H[i], b = H[(size_t)S2 * d.dim + S];
      const float2 m = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
      H[i] = m;
      H[(size_t)S2 * d.dim + S] = make_float2(m.x, -m.y);
    } else if (S == S2) {
      H[i].y = 0.f;
    }
  }
}

// ---------------------------------------------------------------- coupling block B (Appendix A)
//
// B_SS' = 2 Bx_SS' - Bd_SS' couples the e-h pair S = (k, v, c) with the h-e pair (k', c' -> v'):
//   Bx_SS' = (1/(Omega Nk)) sum_{G != 0} conj(rho_vc^{kk}(G)) vbar(G) conj(rho_v'c'^{k'k'}(-G))
//   Bd_SS' = (1/(Omega Nk)) sum_{G,G'} conj(rho_vc'^{kk'}(G)) W_GG'(q) rho_cv'^{kk'}(G')
// B is symmetric: the upper blocks k <= k' are built and mirrored as B_k'k = B_kk'^T.

// rhot[S][G] = conj(rho_x[S][-G]) on the q = 0 sphere (the h-e pair density).
__global__ void minus_g_kernel(DevSys d, const float2* __restrict__ rho_x, float2* __restrict__ rhot) {
  const long long n = (long long)d.dim * d.ng0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int S = (int)(i / d.ng0), t = (int)(i - (long long)S * d.ng0);
    const int m = d.gminus0[t];
    const float2 v = m >= 0 ? rho_x[(size_t)S * d.ng_max + m] : make_float2(0.f, 0.f);
    rhot[(size_t)S * d.ng_max + t] = make_float2(v.x, -v.y);
  }
}

// B = 2 Bx on tiles touching k(S) <= k(S') (the exchange scale sqrt(2 vbar/(Omega Nk)) on both operands).
__global__ __launch_bounds__(kGemmThreads) void cpl_init_kernel(DevSys d, const float2* __restrict__ rho_x,
                                                                const float2* __restrict__ rhot,
                                                                float2* __restrict__ Bm) {
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= d.dim || n0 >= d.dim) return;
  if (kpt_of_pair(d, m0) > kpt_of_pair(d, min(n0 + BN, d.dim) - 1)) return;
  __shared__ gemm::Smem sm;
  float2 acc[4][4];
  gemm::tile<true, true, true, false, true>(rho_x, d.ng_max, d.dim, rhot, d.ng_max, d.dim, d.ng0, m0, n0, sm, acc,
                                            d.xscale);
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int S = m0 + tm * 4 + i;
    if (S >= d.dim) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int S2 = n0 + tn * 4 + j;
      if (S2 < d.dim) Bm[(size_t)S * d.dim + S2] = acc[i][j];
    }
  }
}

// Per upper block: M[a][c] = sum_G conj(Lv[a][G]) X[c][G], a = (v, c'), c = (c, v'), X = W rho_cv';
// B[(k,v,c)][(k',v',c')] -= M/(Omega Nk), mirror B_k'k = B_kk'^T, diagonal blocks (B + B^T)/2.
__global__ __launch_bounds__(kBlkThreads) void cpl_block_kernel(DevSys d, const float2* __restrict__ rho_cpl,
                                                               const float2* __restrict__ X, float2* __restrict__ Bm,
                                                               int q_begin, long long vbase) {
  __shared__ float2 Ls[16][KC + 1];
  __shared__ float2 Rs[16][KC + 1];
  __shared__ float2 Bs[16][17];
  const long long b0 = d.qblk_off[q_begin];
  const long long b = b0 + blockIdx.x;
  const int4 blk = d.blocks[b];
  const int k = blk.x, k2 = blk.y, q = blk.z;
  const long long qb = d.qblk_off[q];
  const long long local = b - qb;
  const int nv = d.nv, nc = d.nc, w = nv * nc;
  const float2* L = rho_cpl + (size_t)(2LL * w * qb - vbase + local * w) * d.ng_max;
  const float2* R = X + (size_t)((qb - b0 + local) * w) * d.ng_max;
  const int NG = d.ngq[q];
  const int t = threadIdx.x;
  const int a = t / w, c = t % w;
  const bool active = t < w * w;
  float2 acc = make_float2(0.f, 0.f);
  for (int g0 = 0; g0 < NG; g0 += KC) {
    for (int i = t; i < 16 * KC; i += kBlkThreads) {
      const int r = i / KC, g = i % KC;
      const bool in = r < w && (g0 + g) < NG;
      Ls[r][g] = in ? L[(size_t)r * d.ng_max + g0 + g] : make_float2(0.f, 0.f);
      Rs[r][g] = in ? R[(size_t)r * d.ng_max + g0 + g] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (active) {
#pragma unroll 8
      for (int g = 0; g < KC; ++g) {
        const float2 l = Ls[a][g], r = Rs[c][g];
        acc.x = fmaf(l.x, r.x, fmaf(l.y, r.y, acc.x));     // conj(l) r
        acc.y = fmaf(l.x, r.y, fmaf(-l.y, r.x, acc.y));
      }
    }
    __syncthreads();
  }
  const float nrm = (float)d.norm;
  int row = 0, col = 0;
  float2 val = make_float2(0.f, 0.f);
  if (active) {
    const int v = a / nc, cp = a % nc, cc = c / nv, vp = c % nv;
    row = v * nc + cc;                 // (k, v, c) local
    col = vp * nc + cp;                // (k', v', c') local
    const size_t bij = (size_t)(k * w + row) * d.dim + (size_t)k2 * w + col;
    const float2 h = Bm[bij];
    val = make_float2(h.x - nrm * acc.x, h.y - nrm * acc.y);
    if (k != k2) {
      Bm[bij] = val;
      Bm[(size_t)(k2 * w + col) * d.dim + (size_t)k * w + row] = val;
    } else {
      Bs[row][col] = val;
    }
  }
  if (k == k2) {
    __syncthreads();
    if (active) {
      const float2 o = Bs[col][row];
      Bm[(size_t)(k * w + row) * d.dim + (size_t)k * w + col] = make_float2(0.5f * (val.x + o.x), 0.5f * (val.y + o.y));
    }
  }
}

// Lower blocks B_k'k = B_kk'^T and diagonal blocks (B + B^T)/2 for a build without the direct term.
__global__ void cpl_mirror_kernel(DevSys d, float2* __restrict__ Bm) {
  const long long n = (long long)d.dim * d.dim;
  const int nvc = d.nv * d.nc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int S = (int)(i / d.dim), S2 = (int)(i - (long long)S * d.dim);
    const int k = S / nvc, k2 = S2 / nvc;
    if (k > k2) {
      Bm[i] = Bm[(size_t)S2 * d.dim + S];
    } else if (k == k2 && S < S2) {
      const float2 a = Bm[i], b = Bm[(size_t)S2 * d.dim + S];
      const float2 m = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
      Bm[i] = m;
      Bm[(size_t)S2 * d.dim + S] = m;
    }
  }
}

// k-point symmetry: block (ik, ik2) = representative block (or its conjugate transpose), and the mirror
// H_{ik2, ik} = H_{ik, ik2}^H; one CTA per listed block, one thread per element.
__global__ void symfill_kernel(DevSys d, float2* __restrict__ H) {
  const int4 f = d.fill[blockIdx.x];
  const int nvc = d.nv * d.nc;
  const bool mirrored = f.w < 0;
  const int ra = f.z, rb = mirrored ? -f.w - 1 : f.w;
  for (int t = threadIdx.x; t < nvc * nvc; t += blockDim.x) {
    const int i = t / nvc, j = t - i * nvc;
    float2 v;
    if (mirrored) {
      const float2 u = H[(size_t)(ra * nvc + j) * d.dim + rb * nvc + i];
      v = make_float2(u.x, -u.y);
    } else {
      v = H[(size_t)(ra * nvc + i) * d.dim + rb * nvc + j];
    }
    H[(size_t)(f.x * nvc + i) * d.dim + f.y * nvc + j] = v;
    if (f.x != f.y) H[(size_t)(f.y * nvc + j) * d.dim + f.x * nvc + i] = make_float2(v.x, -v.y);
  }
}
}  // namespace

int launch_symfill(const DevSys& d, void* H, void* stream) {
  if (d.nfill <= 0) return 0;
  if (d.nfill >= (1LL << 31)) return (int)cudaErrorInvalidValue;
  const int nvc = d.nv * d.nc;
  symfill_kernel<<<(unsigned)d.nfill, nvc * nvc < 256 ? (nvc * nvc + 31) / 32 * 32 : 256, 0, (cudaStream_t)stream>>>(
      d, (float2*)H);
  return (int)cudaGetLastError();
}

int launch_mirror(const DevSys& d, void* H, void* stream) {
  mirror_kernel<<<1216, 256, 0, (cudaStream_t)stream>>>(d, (float2*)H);
  return (int)cudaGetLastError();
}

// FP32 W.rho rows of a q chunk (w rows per block), then (for BSE_PREC_BF16X3) the split BF16 tile images.
static size_t x_bytes(const DevSys& d, long long qchunk, long long w) {
  long long nb = qchunk * d.nkpt;
  if (nb > d.nblocks) nb = d.nblocks;
  return (((size_t)(nb * w) * d.ng_max * sizeof(float2)) + 255) & ~(size_t)255;
}

static long long direct_width(const DevSys& d) {
  return (d.nv * d.nv <= d.nc * d.nc) ? d.nv * d.nv : d.nc * d.nc;
}

// The direct stage's W.rho rows and split images of a q chunk; at least the exchange stage's split images of
// rho_x (BSE_BK_INIT with BSE_PREC_BF16X3).
size_t kernel_ws_bytes(const DevSys& d, long long qchunk) {
  const long long w = direct_width(d);
  const size_t direct = x_bytes(d, qchunk, w) + tc_split_bytes(d, qchunk, w);
  const size_t init = gram_ws_bytes(d);
  return direct > init ? direct : init;
}

// Coupling build: W.rho_cv' rows and split images of a q chunk, or (init) conj(rho_x(-G)) rows.
size_t coupling_ws_bytes(const DevSys& d, long long qchunk) {
  const long long w = (long long)d.nv * d.nc;
  const size_t direct = qchunk > 0 ? x_bytes(d, qchunk, w) + tc_split_bytes(d, qchunk, w) : 0;
  const size_t init = (((size_t)d.dim * d.ng_max * sizeof(float2)) + 255) & ~(size_t)255;
  return direct > init ? direct : init;
}

int launch_kernel_init(const DevSys& d, const void* rho_x, const double* energies, double delta, void* H,
                       void* stream) {
  dim3 grid((d.dim + BN - 1) / BN, (d.dim + BM - 1) / BM);
  init_kernel<<<grid, kGemmThreads, 0, (cudaStream_t)stream>>>(d, (const float2*)rho_x, energies, delta, (float2*)H);
  return (int)cudaGetLastError();
}

int launch_gemm_wr(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long vbase, long long max_rows,
                   const void* W, void* X, int side_c, void* stream) {
  dim3 grid((d.ng_max + wr::TN - 1) / wr::TN, (unsigned)((max_rows + wr::TM - 1) / wr::TM), q_end - q_begin);
  gemm_wr<<<grid, wr::kThreads, 0, (cudaStream_t)stream>>>(d, (const float2*)rho_dir, (const float2*)W, (float2*)X,
                                                          q_begin, vbase, side_c);
  return (int)cudaGetLastError();
}

int launch_kernel_direct_range(const DevSys& d, const void* rho_dir, int q_begin, int q_end, long long b_begin,
                               long long b_count, long long vbase, long long max_rows, const void* W, int prec,
                               void* H, void* ws, int* status, void* stream) {
  const int side_c = (d.nc * d.nc < d.nv * d.nv) ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  int e;
  if (prec != BSE_PREC_BF16X3 && prec != BSE_PREC_FP32) return -1;
  if (b_count <= 0 || max_rows <= 0) return 0;     // no block in the range (k-point symmetry can leave q empty)
  if (prec == BSE_PREC_BF16X3) {
    void* split_ws = (char*)ws + x_bytes(d, q_end - q_begin, direct_width(d));
    e = launch_gemm_wr_tc(d, rho_dir, q_begin, q_end, vbase, max_rows, W, ws, split_ws, side_c, status, stream);
  } else if (prec == BSE_PREC_FP32) {
    dim3 grid((d.ng_max + wr::TN - 1) / wr::TN, (unsigned)((max_rows + wr::TM - 1) / wr::TM), q_end - q_begin);
    gemm_wr<<<grid, wr::kThreads, 0, st>>>(d, (const float2*)rho_dir, (const float2*)W, (float2*)ws, q_begin, vbase,
                                           side_c);
    e = (int)cudaGetLastError();
  } else {
    return -1;
  }
  if (e) return e;
  if (b_count > 0)
    block_kernel<<<(unsigned)((b_count + kBlkPerCta - 1) / kBlkPerCta), kBlkThreads, 0, st>>>(
        d, (const float2*)rho_dir, (const float2*)ws, (float2*)H, q_begin, vbase, side_c, b_count);
  return (int)cudaGetLastError();
}

int launch_coupling_init(const DevSys& d, const void* rho_x, void* Bm, void* ws, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  minus_g_kernel<<<1216, 256, 0, st>>>(d, (const float2*)rho_x, (float2*)ws);
  dim3 grid((d.dim + BN - 1) / BN, (d.dim + BM - 1) / BM);
  cpl_init_kernel<<<grid, kGemmThreads, 0, st>>>(d, (const float2*)rho_x, (const float2*)ws, (float2*)Bm);
  return (int)cudaGetLastError();
}

int launch_coupling_mirror(const DevSys& d, void* Bm, void* stream) {
  cpl_mirror_kernel<<<1216, 256, 0, (cudaStream_t)stream>>>(d, (float2*)Bm);
  return (int)cudaGetLastError();
}

int launch_coupling_direct_range(const DevSys& d, const void* rho_cpl, int q_begin, int q_end, long long b_count,
                                 long long vbase, long long max_rows, const void* W, int prec, void* Bm, void* ws,
                                 int* status, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const long long w = (long long)d.nv * d.nc;
  int e;
  if (prec == BSE_PREC_BF16X3) {
    void* split_ws = (char*)ws + x_bytes(d, q_end - q_begin, w);
    e = launch_gemm_wr_tc(d, rho_cpl, q_begin, q_end, vbase, max_rows, W, ws, split_ws, 2, status, stream);
  } else if (prec == BSE_PREC_FP32) {
    dim3 grid((d.ng_max + wr::TN - 1) / wr::TN, (unsigned)((max_rows + wr::TM - 1) / wr::TM), q_end - q_begin);
    gemm_wr<<<grid, wr::kThreads, 0, st>>>(d, (const float2*)rho_cpl, (const float2*)W, (float2*)ws, q_begin, vbase,
                                           2);
    e = (int)cudaGetLastError();
  } else {
    return -1;
  }
  if (e) return e;
  if (b_count > 0)
    cpl_block_kernel<<<(unsigned)b_count, kBlkThreads, 0, st>>>(d, (const float2*)rho_cpl, (const float2*)ws,
                                                                (float2*)Bm, q_begin, vbase);
  return (int)cudaGetLastError();
}

}  // namespace bse
