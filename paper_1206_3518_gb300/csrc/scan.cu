// Input scans for non-finite values.  Every compute entry point passes its caller-supplied
// floating-point inputs through one streaming pass here before its own kernels; a NaN or an
// infinity anywhere sets BSE_ERR_NONFINITE in the plan's device status word (first error wins),
// which bse_status_read returns.  The pass reads each input once at HBM speed (loads marked
// evict-first) and writes nothing but the status word.
#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"

namespace bse {
namespace {

// IEEE-754: exponent bits all set <=> infinity or NaN.
__device__ __forceinline__ bool bad32(unsigned u) { return (u & 0x7f800000u) == 0x7f800000u; }
__device__ __forceinline__ bool bad64hi(unsigned hi) { return (hi & 0x7ff00000u) == 0x7ff00000u; }

template <int E>
__device__ __forceinline__ bool bad_vec(uint4 u) {
  if (E == 4) return bad32(u.x) | bad32(u.y) | bad32(u.z) | bad32(u.w);
  return bad64hi(u.y) | bad64hi(u.w);   // little endian: the high word follows the low word
}

template <int E>
__device__ __forceinline__ bool bad_elem(const unsigned char* p) {
  if (E == 4) return bad32(*(const unsigned*)p);
  return bad64hi(*(const unsigned*)(p + 4));
}

// n elements of E bytes at p (p aligned to E).  The 16-byte-aligned body is read as uint4, the
// at most 15 bytes before it and after it element by element.
template <int E>
__global__ void __launch_bounds__(256) nonfinite_kernel(const unsigned char* p, long long n, int* status) {
  const uintptr_t a = (uintptr_t)p;
  long long head = (long long)((16 - (a & 15u)) & 15u) / E;
  if (head > n) head = n;
  const long long nvec = (n - head) * E / 16;
  const long long tail0 = head + nvec * (16 / E);
  const uint4* body = (const uint4*)(p + head * E);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  for (long long j = i0; j < nvec; j += stride) bad |= bad_vec<E>(__ldcs(body + j));
  for (long long j = i0; j < head; j += stride) bad |= bad_elem<E>(p + j * E);
  for (long long j = tail0 + i0; j < n; j += stride) bad |= bad_elem<E>(p + j * E);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, (int)BSE_ERR_NONFINITE);
}

}  // namespace

int launch_nonfinite_scan(const void* p, long long n, int elem_bytes, int* status, void* stream) {
  if (!p || n <= 0) return 0;
  if (elem_bytes != 4 && elem_bytes != 8) return (int)cudaErrorInvalidValue;
  if (((uintptr_t)p) % (uintptr_t)elem_bytes) return (int)cudaErrorMisalignedAddress;
  int dev = 0, sms = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return e;
  e = (int)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return e;
  const long long words = n * elem_bytes / 16 + 1;
  long long blocks = (words + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (elem_bytes == 4)
    nonfinite_kernel<4><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>((const unsigned char*)p, n, status);
  else
    nonfinite_kernel<8><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>((const unsigned char*)p, n, status);
  return (int)cudaGetLastError();
}

}  // namespace bse
