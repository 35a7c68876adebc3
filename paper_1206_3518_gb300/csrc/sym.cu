// W on the full q mesh from W on the irreducible q points (Sec. III A):
//   q = s R q_IBZ + G0  =>  W_GG'(q) = W_{s R^-1 (G + G0), s R^-1 (G' + G0)}(q_IBZ), conjugated when s = -1.
// The planner supplies, per q, the irreducible index, the time-reversal flag and the sphere map
// p -> perm[p] (position of s R^-1 (g_p + G0) on the sphere of q_IBZ).
#include <cuda_runtime.h>

#include "internal.h"

namespace bse {
namespace {

__global__ void unfold_w_kernel(DevSys d, const float2* __restrict__ W_ibz, float2* __restrict__ W, int q_begin) {
  const int q = q_begin + blockIdx.y;
  const int ng = d.ngq[q], ld = d.ng_max;
  const int2 sym = d.qsym[q];
  const float2* src = W_ibz + (size_t)sym.x * ld * ld;
  float2* dst = W + (size_t)q * ld * ld;
  const int* perm = d.qperm + (size_t)q * ld;
  const long long n = (long long)ld * ld;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / ld), c = (int)(i - (long long)r * ld);
    float2 v = make_float2(0.f, 0.f);
    if (r < ng && c < ng) {
      v = src[(size_t)perm[r] * ld + perm[c]];
      if (sym.y) v.y = -v.y;
    }
    dst[i] = v;
  }
}

}  // namespace

int launch_unfold_w(const DevSys& d, const void* W_ibz, void* W, int q_begin, int q_end, void* stream) {
  const long long n = (long long)d.ng_max * d.ng_max;
  const int bx = (int)((n + 255) / 256 < 64 ? (n + 255) / 256 : 64);
  dim3 grid(bx > 0 ? bx : 1, q_end - q_begin);
  unfold_w_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d, (const float2*)W_ibz, (float2*)W, q_begin);
  return (int)cudaGetLastError();
}

}  // namespace bse
