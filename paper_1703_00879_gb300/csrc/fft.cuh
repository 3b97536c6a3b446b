// Shared-memory Stockham FFT building blocks for sm_103a.
//
// A tile of TW independent columns of length L (power of two) lives in shared
// memory as buf[n * PITCH + c] (float2, c = column, n = element).  Each stage is
// one radix-R Stockham autosort pass (Govindaraju et al., SC'08 formulation):
// every butterfly j loads elements j + r L/R, applies twiddles w^(r (j mod Ns)),
// does an in-register radix-R DFT and stores at (j/Ns) Ns R + (j mod Ns) + r Ns.
// The output is in natural order.  Consecutive threads handle consecutive
// columns, so every shared-memory access of a half warp is bank-conflict free
// for PITCH = TW (column tiles) or TW + 1 (row tiles).
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / T) of the tile's transform
// table length T (host-computed in double precision, rounded to float); a
// length-L transform reads it with stride T / L.  INV selects exp(+...) (the
// unnormalised inverse).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cola {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by +i
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot_q(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = rot_q<INV>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float r = 0.70710678118654752440f;
  // o1 *= w8, o2 *= w8^2, o3 *= w8^3 with w8 = exp(-/+ i pi/4)
  o1 = INV ? make_float2((o1.x - o1.y) * r, (o1.x + o1.y) * r)
           : make_float2((o1.x + o1.y) * r, (o1.y - o1.x) * r);
  o2 = rot_q<INV>(o2);
  o3 = INV ? make_float2((-o3.x - o3.y) * r, (o3.x - o3.y) * r)
           : make_float2((o3.y - o3.x) * r, (-o3.x - o3.y) * r);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 2) {
    dft2<INV>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else {
    static_assert(R == 8, "radix");
    dft8<INV>(v);
  }
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Radix of stage s for a length-L transform: radix 8 first, one radix 2 or 4 last.
template <int L, int S>
struct StageRadix {
  static constexpr int p = ilog2(L);
  static constexpr int n8 = p / 3;
  static constexpr int rem = p % 3;
  static constexpr int value = (S < n8) ? 8 : (rem == 1 ? 2 : 4);
  static constexpr int nstages = n8 + (rem ? 1 : 0);
};

// One Stockham stage on a TW x L shared-memory tile.
template <int L, int R, int NS, int TW, int PITCH, int NT, bool INV, int TWS>
__device__ __forceinline__ void fft_stage(float2* __restrict__ buf, const float2* __restrict__ tw) {
  constexpr int NB = L / R;           // butterflies per column
  constexpr int TOT = NB * TW;
  constexpr int PER = (TOT + NT - 1) / NT;
  const int tid = threadIdx.x;
  float2 v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = tid + i * NT;
    if ((TOT % NT) == 0 || b < TOT) {
      const int c = b % TW, j = b / TW;
      const int k = j & (NS - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = buf[(j + r * NB) * PITCH + c];
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r * k * (L / (NS * R))) * TWS];
          if (INV) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      dftR<R, INV>(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = tid + i * NT;
    if ((TOT % NT) == 0 || b < TOT) {
      const int c = b % TW, j = b / TW;
      const int k = j & (NS - 1);
      const int idxD = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(idxD + r * NS) * PITCH + c] = v[i][r];
    }
  }
  __syncthreads();
}

template <int L, int S, int NS, int TW, int PITCH, int NT, bool INV, int TWS>
__device__ __forceinline__ void fft_stages(float2* buf, const float2* tw) {
  if constexpr (S < StageRadix<L, 0>::nstages) {
    constexpr int R = StageRadix<L, S>::value;
    fft_stage<L, R, NS, TW, PITCH, NT, INV, TWS>(buf, tw);
    fft_stages<L, S + 1, NS * R, TW, PITCH, NT, INV, TWS>(buf, tw);
  }
}

// Full length-L transform of all TW columns (caller synchronises before the call).
// tw is a table of length L * TWS.
template <int L, int TW, int PITCH, int NT, bool INV, int TWS = 1>
__device__ __forceinline__ void fft_tile(float2* buf, const float2* tw) {
  fft_stages<L, 0, 1, TW, PITCH, NT, INV, TWS>(buf, tw);
}

// Signed frequency index of position n in a length-N transform.
__device__ __forceinline__ int freq_index(int n, int N) { return n < (N >> 1) ? n : n - N; }

}  // namespace cola
