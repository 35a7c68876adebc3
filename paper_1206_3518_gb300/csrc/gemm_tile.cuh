// One 64x64 tile of a complex FP32 product C = opA(A) opB(B)^T accumulated in registers.
//
// A(m, k) is read from A[m*lda + k] (A_KC: K contiguous) or A[k*lda + m]; B(n, k) likewise.
// CONJ_A / CONJ_B conjugate the operand.  256 threads, 4x4 outputs per thread
// (rows tm*4.., cols tn*4..), K staged in shared memory 16 at a time; out-of-range
// elements read as zero.  Loads are coalesced for either layout.
#pragma once

#include <vector_types.h>

namespace bse {
namespace gemm {

constexpr int BM = 64, BN = 64, BK = 16, kThreads = 256;

struct Smem {
  float2 a[BK][BM + 1];
  float2 b[BK][BN + 1];
};

template <bool KC, bool CONJ, bool SCALE>
__device__ __forceinline__ void stage(const float2* __restrict__ X, long long ld, int R, int K, int r0, int k0,
                                      const float* __restrict__ ks, float2 (*S)[BM + 1]) {
  const int t = threadIdx.x;
  if (KC) {                      // rows of X are K-contiguous: threads run along k
    const int lk = t % BK, lr = t / BK;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = lr + 16 * i, kk = k0 + lk;
      float2 v = make_float2(0.f, 0.f);
      if (kk < K && r0 + r < R) v = X[(long long)(r0 + r) * ld + kk];
      if (CONJ) v.y = -v.y;
      if (SCALE && kk < K) {
        const float sc = ks[kk];
        v.x *= sc;
        v.y *= sc;
      }
      S[lk][r] = v;
    }
  } else {                       // X[k][r]: threads run along r
    const int lr = t % BM, lk = t / BM;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kk = k0 + lk + 4 * i;
      float2 v = make_float2(0.f, 0.f);
      if (kk < K && r0 + lr < R) v = X[(long long)kk * ld + r0 + lr];
      if (CONJ) v.y = -v.y;
      if (SCALE && kk < K) {
        const float sc = ks[kk];
        v.x *= sc;
        v.y *= sc;
      }
      S[lk + 4 * i][lr] = v;
    }
  }
}

// SCALE multiplies both operands by ks[k] (e.g. sqrt of a diagonal metric between them).
template <bool A_KC, bool B_KC, bool CONJ_A, bool CONJ_B, bool SCALE = false>
__device__ __forceinline__ void tile(const float2* __restrict__ A, long long lda, int M, const float2* __restrict__ B,
                                     long long ldb, int N, int K, int m0, int n0, Smem& sm, float2 (&acc)[4][4],
                                     const float* __restrict__ ks = nullptr) {
  const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += BK) {
    stage<A_KC, CONJ_A, SCALE>(A, lda, M, K, m0, k0, ks, sm.a);
    stage<B_KC, CONJ_B, SCALE>(B, ldb, N, K, n0, k0, ks, sm.b);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float2 av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sm.a[k][tm * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sm.b[k][tn * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
}

}  // namespace gemm
}  // namespace bse
