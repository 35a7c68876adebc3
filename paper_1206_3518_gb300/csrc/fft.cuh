// Register-resident mixed-radix (4, 2, 3) Stockham FFT for one line per thread.
//
// Every index is a compile-time constant after unrolling, so the line lives in
// registers and the twiddles become constant-bank operands.  Stage s with
// radix R and current sub-transform length Ns maps input j + r*N/R to output
// (j/Ns)*Ns*R + (j mod Ns) + r*Ns after twiddling by exp(-+2 pi i r (j mod Ns)/(Ns R))
// (self-sorting Stockham form; no bit reversal).  FWD = exp(-i...), !FWD = exp(+i...),
// both unnormalised.  Host-callable as well, so the factorisation is unit-tested on CPU.
#pragma once

#include <vector_types.h>

#ifndef BSE_HD
#define BSE_HD __host__ __device__ __forceinline__
#endif

namespace bse {
namespace fft {

constexpr int kTwN = 192;   // table length: multiple of every supported N (2^a 3^b <= 64)

struct Twiddles {
  const float2* t;          // t[k] = (cos(2 pi k/192), sin(2 pi k/192))
};

BSE_HD float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
BSE_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
BSE_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
BSE_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

template <int N, bool FWD>
BSE_HD float2 tw(const float2* table, int t) {
  const float2 w = table[((t % N + N) % N) * (kTwN / N)];
  return FWD ? make_float2(w.x, -w.y) : w;
}

template <int R, bool FWD>
BSE_HD void dft(float2 (&v)[R]);

template <>
BSE_HD void dft<2, true>(float2 (&v)[2]) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
BSE_HD void dft<2, false>(float2 (&v)[2]) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool FWD>
BSE_HD void dft4(float2 (&v)[4]) {
  const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  const float2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  // FWD: X1 = t1 - i t3, X3 = t1 + i t3 ; INV: signs swapped
  const float2 it3 = FWD ? make_float2(t3.y, -t3.x) : make_float2(-t3.y, t3.x);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, it3);
  v[3] = csub(t1, it3);
}
template <>
BSE_HD void dft<4, true>(float2 (&v)[4]) { dft4<true>(v); }
template <>
BSE_HD void dft<4, false>(float2 (&v)[4]) { dft4<false>(v); }

template <bool FWD>
BSE_HD void dft3(float2 (&v)[3]) {
  const float c = -0.5f;
  const float s = FWD ? -0.86602540378443864676f : 0.86602540378443864676f;   // -+ sin(2 pi/3)
  const float2 sum = cadd(v[1], v[2]), dif = csub(v[1], v[2]);
  const float2 m = make_float2(v[0].x + c * sum.x, v[0].y + c * sum.y);
  const float2 r = make_float2(-s * dif.y, s * dif.x);                       // i s dif
  v[0] = cadd(v[0], sum);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}
template <>
BSE_HD void dft<3, true>(float2 (&v)[3]) { dft3<true>(v); }
template <>
BSE_HD void dft<3, false>(float2 (&v)[3]) { dft3<false>(v); }

template <int N, int Ns, bool FWD>
struct Stockham {
  static BSE_HD void run(const float2* table, float2 (&x)[N]) {
    if constexpr (Ns < N) {
      constexpr int Rm = N / Ns;
      constexpr int R = (Rm % 4 == 0) ? 4 : ((Rm % 2 == 0) ? 2 : 3);
      float2 y[N];
#pragma unroll
      for (int j = 0; j < N / R; ++j) {
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[j + r * (N / R)];
        const int jm = j % Ns;
#pragma unroll
        for (int r = 1; r < R; ++r)
          if (jm != 0) v[r] = cmul(v[r], tw<N, FWD>(table, r * jm * (N / (Ns * R))));
        dft<R, FWD>(v);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) y[base + r * Ns] = v[r];
      }
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = y[i];
      Stockham<N, Ns * R, FWD>::run(table, x);
    }
  }
};

// In-place N-point DFT of one register line: FWD -> X_f = sum_j x_j exp(-2 pi i f j/N).
template <int N, bool FWD>
BSE_HD void line(const float2* table, float2 (&x)[N]) {
  Stockham<N, 1, FWD>::run(table, x);
}

}  // namespace fft
}  // namespace bse
