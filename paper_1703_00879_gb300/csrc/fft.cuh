// Shared-memory FFT building blocks for sm_103a.
//
// A tile of TW independent columns of length L (power of two) lives in shared
// memory as buf[n * PITCH + c] (float2, c = column, n = element).  A transform
// is two in-register DFT passes of radix R1, R2 <= 32 (L = R1 R2, the
// "four-step" factorisation) with one twiddle multiplication between them, so
// each element makes two round trips through shared memory.  Consecutive
// threads handle consecutive columns.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / T) of the tile's transform
// table length T (host-computed in double precision, rounded to float); a
// length-L transform reads it with stride T / L.  INV selects exp(+...) (the
// unnormalised inverse).
//
// The in-register DFTs are radix-2 decimation in time (inputs in bit-reversed
// positions, placed there at compile time by the loads; outputs in natural
// order): a twiddled butterfly a +- w b is two fused multiply-adds per component
// for a + w b and one for 2a - (a + w b), issued as paired (two-component)
// FMAs; the decimation-in-frequency form (subtract, then multiply by w) takes
// more.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cola {

// Additions, subtractions and scalings of complex values use the paired
// single-precision instructions of this architecture (two components per
// instruction, each rounded exactly as the scalar operation).  The complex
// multiply stays scalar: its paired form (a multiply and an FMA on swapped
// operands) measured no faster.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
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

// cos(2 pi m / 32) for m = 0..8 (standard values; sin(2 pi m/32) = cos32(8 - m)).
__host__ __device__ constexpr float cos32(int m) {
  return m == 0 ? 1.0f
       : m == 1 ? 0.98078528040323044913f
       : m == 2 ? 0.92387953251128675613f
       : m == 3 ? 0.83146961230254523708f
       : m == 4 ? 0.70710678118654752440f
       : m == 5 ? 0.55557023301960222474f
       : m == 6 ? 0.38268343236508977173f
       : m == 7 ? 0.19509032201612826785f
       : 0.0f;
}

// a * exp(-/+ 2 pi i m / 32), m in [0, 16) a compile-time constant after unrolling.
template <bool INV>
__device__ __forceinline__ float2 w32mul(float2 a, int m) {
  if (m == 0) return a;
  if (m == 8) return rot_q<INV>(a);
  const float c = m <= 8 ? cos32(m) : -cos32(16 - m);
  const float s = m <= 8 ? cos32(8 - m) : cos32(m - 8);
  return INV ? make_float2(a.x * c - a.y * s, a.y * c + a.x * s)
             : make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
}

// Decimation-in-time butterfly (a, b) <- (a + w b, a - w b) with
// w = exp(-/+ 2 pi i m / 32), m in [0, 16) a compile-time constant after
// unrolling: m = 0 and 8 are additions, the others two paired FMAs for a + w b
// and one for 2a - (a + w b) (the same per-component FMAs as the scalar form).
template <bool INV>
__device__ __forceinline__ void bfly_tw(float2& a, float2& b, int m) {
  if (m == 0) {
    dft2<INV>(a, b);
    return;
  }
  if (m == 8) {
    const float2 wb = rot_q<INV>(b), t = a;
    a = cadd(t, wb);
    b = csub(t, wb);
    return;
  }
  const float c = m <= 8 ? cos32(m) : -cos32(16 - m);
  const float s = m <= 8 ? cos32(8 - m) : cos32(m - 8);  // sin(2 pi m / 32) >= 0
  // forward w b = (c br + s bi, c bi - s br); inverse (c br - s bi, c bi + s br)
  const float sg = INV ? -s : s;
  // x = (c br + (sg bi + ar), c bi + (-sg br + ai)), b <- 2a - x: paired FMAs
  const float2 t = __ffma2_rn(make_float2(sg, -sg), make_float2(b.y, b.x), a);
  const float2 x = __ffma2_rn(make_float2(c, c), b, t);
  b = __ffma2_rn(make_float2(2.f, 2.f), a, make_float2(-x.x, -x.y));
  a = x;
}

// 8-point DFT, natural order in and out: two 4-point DFTs of the even and odd
// inputs and one decimation-in-time layer.
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  bfly_tw<INV>(e0, o0, 0);
  bfly_tw<INV>(e1, o1, 4);
  bfly_tw<INV>(e2, o2, 8);
  bfly_tw<INV>(e3, o3, 12);
  v[0] = e0;
  v[1] = e1;
  v[2] = e2;
  v[3] = e3;
  v[4] = o0;
  v[5] = o1;
  v[6] = o2;
  v[7] = o3;
}

// In-register DFT of R = 2..32 points on the strided view v[0], v[S], ...,
// v[(R-1)S], in place.  R <= 8: natural order.  R = 16, 32: radix-2
// decimation in time, so input n must sit at position pos_of<R>(n) (placed
// there at compile time by the caller) and output k ends at position k.
template <int R>
__host__ __device__ constexpr int pos_of(int n) {
  if constexpr (R <= 8) {
    return n;
  } else {
    return (n % 2 == 0) ? pos_of<R / 2>(n / 2) : R / 2 + pos_of<R / 2>((n - 1) / 2);
  }
}

template <bool INV, int S>
__device__ __forceinline__ void dft8s(float2* v) {
  float2 t[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) t[i] = v[i * S];
  dft8<INV>(t);
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i * S] = t[i];
}

template <int R, bool INV, int S = 1>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(v[0], v[S]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[S], v[2 * S], v[3 * S]);
  } else if constexpr (R == 8) {
    dft8s<INV, S>(v);
  } else {
    static_assert(R == 16 || R == 32, "radix");
    // even inputs in the first half, odd in the second (pos_of), each half a
    // DFT of R / 2 points in natural order, then one butterfly layer
    dftR<R / 2, INV, S>(v);
    dftR<R / 2, INV, S>(v + (R / 2) * S);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) bfly_tw<INV>(v[k * S], v[(k + R / 2) * S], k * (32 / R));
  }
}

// 32-point DFT shared by a thread pair (lanes l and l ^ 16 of a full warp):
// the thread with half = 0 holds x[0..15] in v, its partner x[16..31].  One
// radix-2 decimation-in-frequency step exchanges the halves by shuffle (half 0
// forms a[n] = x[n] + x[n + 16], half 1 b[n] = (x[n] - x[n + 16]) w32^n), then
// each runs a 16-point DFT: half h ends with X[2k + h] at v[k].
template <bool INV>
__device__ __forceinline__ void dft32_pair(float2 (&v)[16], int half) {
  const float sg = half ? -1.f : 1.f;
  float2 u[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    const float ox = __shfl_xor_sync(0xffffffffu, v[n].x, 16);
    const float oy = __shfl_xor_sync(0xffffffffu, v[n].y, 16);
    const float2 t = make_float2(fmaf(sg, v[n].x, ox), fmaf(sg, v[n].y, oy));
    const float2 tw = w32mul<INV>(t, n);
    u[pos_of<16>(n)] = half ? tw : t;
  }
  dftR<16, INV>(u);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = u[k];
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// L = R1 R2 with R1 <= R2 <= 32.
template <int L>
struct Split {
  static constexpr int p = ilog2(L);
  static constexpr int R1 = 1 << (p / 2);
  static constexpr int R2 = L / R1;
  static_assert(R2 <= 32 && R1 * R2 == L, "transform length");
};

// Rows of shared memory a length-L column-tile transform needs: L, plus R2
// padding rows for the intermediate.
template <int L>
__host__ __device__ constexpr int fft_rows() {
  return L + Split<L>::R2;
}

// Length-L transform of the TW columns of a shared-memory tile (four-step):
// step 1: for each n2 < R2, DFT_R1 over x[R2 n1 + n2], times w_L^(n2 k1);
// step 2: for each k1 < R1, DFT_R2 over n2 gives X[k1 + R1 k2].
// The intermediate Y[n2][k1] goes to row n2 (R1 + 1) + k1, one padding row
// per R1 (the tile needs fft_rows<L>() rows): with a row pitch that is a
// multiple of 8 the 16 lanes of a half-warp hit 16 different bank pairs, and
// every address is a per-thread base plus a compile-time offset.  tw has
// L * TWS entries; the caller synchronises before the call; returns after a
// barrier.
//
// Hooks (defaults: the tile itself): step 1 reads element n of column c as
// ld(buf, n, c, at) and step 2 writes X[n] as st(X[n], n, c, at), at = n PITCH
// + c, so a k-space operation fuses into the first load or the last store
// (reading or writing another array at the same offset); st.ready() runs in
// every thread before the barrier between the steps.  A store hook with
// kSmem = false writes the outputs itself (e.g. straight to HBM) and the tile
// is left holding the intermediate.
struct TileLoad {
  __device__ __forceinline__ float2 operator()(const float2* buf, int, int, int at) const { return buf[at]; }
};
struct TileStore {
  static constexpr bool kSmem = true;
  __device__ __forceinline__ float2 operator()(float2 v, int, int, int) const { return v; }
  __device__ __forceinline__ void ready() const {}
};

template <int L, int TW, int PITCH, int NT, bool INV, int TWS = 1, class Load = TileLoad,
          class Store = TileStore>
__device__ __forceinline__ void fft_tile(float2* __restrict__ buf, const float2* __restrict__ tw,
                                         Load ld = Load(), Store st = Store()) {
  constexpr int R1 = Split<L>::R1, R2 = Split<L>::R2;
  constexpr int U1 = TW * R2, P1 = (U1 + NT - 1) / NT;
  constexpr int U2 = TW * R1, P2 = (U2 + NT - 1) / NT;
  static_assert(PITCH % 8 == 0, "column tiles: row pitch a multiple of 8");
  const int tid = threadIdx.x;
  {
    float2 v[P1][R1];
#pragma unroll
    for (int i = 0; i < P1; ++i) {
      const int u = tid + i * NT;
      if ((U1 % NT) == 0 || u < U1) {
        const int c = u % TW, n2 = u / TW;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
          v[i][pos_of<R1>(n1)] = ld(buf, R2 * n1 + n2, c, (R2 * n1 + n2) * PITCH + c);
        dftR<R1, INV>(v[i]);
        if (n2 > 0) {
#pragma unroll
          for (int k1 = 1; k1 < R1; ++k1) {
            float2 w = tw[n2 * k1 * TWS];
            if (INV) w.y = -w.y;
            v[i][k1] = cmul(v[i][k1], w);
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P1; ++i) {
      const int u = tid + i * NT;
      if ((U1 % NT) == 0 || u < U1) {
        const int c = u % TW, n2 = u / TW;
        float2* y = buf + n2 * (R1 + 1) * PITCH + c;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) y[k1 * PITCH] = v[i][k1];
      }
    }
  }
  st.ready();
  __syncthreads();
  {
    float2 y[P2][R2];
#pragma unroll
    for (int i = 0; i < P2; ++i) {
      const int u = tid + i * NT;
      if ((U2 % NT) == 0 || u < U2) {
        const int c = u % TW, k1 = u / TW;
        const float2* yr = buf + k1 * PITCH + c;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) y[i][pos_of<R2>(n2)] = yr[n2 * (R1 + 1) * PITCH];
        dftR<R2, INV>(y[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P2; ++i) {
      const int u = tid + i * NT;
      if ((U2 % NT) == 0 || u < U2) {
        const int c = u % TW, k1 = u / TW;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int n = k1 + R1 * k2;
          const float2 o = st(y[i][k2], n, c, n * PITCH + c);
          if constexpr (Store::kSmem) buf[n * PITCH + c] = o;
        }
      }
    }
  }
  __syncthreads();
}

// Row pitch (complex values) of a row-major tile transformed in place by
// fft_rowtile<L>: at least L + R2 - 1 (room for the padded intermediate) and
// 8 mod 16, so that the half-warps of both steps hit distinct bank pairs.
template <int L>
__host__ __device__ constexpr int rowtile_pitch() {
  return ((L + Split<L>::R2 - 1 - 8 + 15) / 16) * 16 + 8;
}

// Load hook of fft_rowtile's first step: element n of row c as pre(x, c, n).
struct NoPre {
  __device__ __forceinline__ float2 operator()(float2 v, int, int) const { return v; }
};

// Length-L transforms of the TW rows of a row-major shared-memory tile, in
// place: row c holds x[n] at buf[c * CW + n] (CW = rowtile_pitch<L>()).  Same
// four-step factorisation as fft_tile, with the element index as the fast
// thread index (consecutive lanes touch consecutive elements of one row):
// step 1 (thread = (c, n2)): DFT_R1 over x[R2 n1 + n2] (each value passed
// through pre() as it is loaded), times w_L^(n2 k1), intermediate at
// n2 (R1 + 1) + k1; step 2 (thread = (c, k1)): DFT_R2 gives X[k1 + R1 k2].
// PAIR32: for L = 16 x 32 with half as many step-2 items as threads, step 2
// runs on thread pairs (dft32_pair), halving its registers per thread.
// The caller synchronises before the call; returns after a barrier.
// Store hook of fft_rowtile's last step: output k of row c as st(X[k], c, k);
// with kSmem = false the hook writes the output itself and the tile keeps the
// intermediate.
struct RowStore {
  static constexpr bool kSmem = true;
  __device__ __forceinline__ float2 operator()(float2 v, int, int) const { return v; }
};

template <int L, int TW, int CW, int NT, bool INV, int TWS = 1, class Pre = NoPre, bool PAIR32 = false,
          class Store = RowStore>
__device__ __forceinline__ void fft_rowtile(float2* __restrict__ buf, const float2* __restrict__ tw,
                                            Pre pre = Pre(), Store st = Store()) {
  constexpr int R1 = Split<L>::R1, R2 = Split<L>::R2;
  constexpr int U1 = TW * R2, P1 = (U1 + NT - 1) / NT;
  constexpr int U2 = TW * R1, P2 = (U2 + NT - 1) / NT;
  static_assert(CW >= L + R2 - 1, "row pitch too small for the intermediate");
  const int tid = threadIdx.x;
  {
    float2 v[P1][R1];
#pragma unroll
    for (int i = 0; i < P1; ++i) {
      const int u = tid + i * NT;
      if ((U1 % NT) == 0 || u < U1) {
        const int c = u / R2, n2 = u % R2;
        const float2* x = buf + c * CW + n2;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[i][pos_of<R1>(n1)] = pre(x[R2 * n1], c, R2 * n1 + n2);
        dftR<R1, INV>(v[i]);
        if (n2 > 0) {
#pragma unroll
          for (int k1 = 1; k1 < R1; ++k1) {
            float2 w = tw[n2 * k1 * TWS];
            if (INV) w.y = -w.y;
            v[i][k1] = cmul(v[i][k1], w);
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P1; ++i) {
      const int u = tid + i * NT;
      if ((U1 % NT) == 0 || u < U1) {
        const int c = u / R2, n2 = u % R2;
        float2* y = buf + c * CW + n2 * (R1 + 1);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) y[k1] = v[i][k1];
      }
    }
  }
  __syncthreads();
  if constexpr (PAIR32 && R1 == 16 && R2 == 32 && 2 * U2 == NT) {
    // step 2 on thread pairs (dft32_pair): U2 items would leave half the threads
    // idle; half the registers per thread
    const int half = (tid >> 4) & 1, u = (tid >> 5) * 16 + (tid & 15);
    const int c = u / R1, k1 = u % R1;
    float2 y[16];
    const float2* yr = buf + c * CW + k1 + 16 * half * (R1 + 1);
#pragma unroll
    for (int j = 0; j < 16; ++j) y[j] = yr[j * (R1 + 1)];
    dft32_pair<INV>(y, half);
    __syncthreads();
    float2* X = buf + c * CW + k1 + R1 * half;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 o = st(y[k], c, k1 + R1 * (2 * k + half));
      if constexpr (Store::kSmem) X[2 * R1 * k] = o;
    }
  } else {
    float2 y[P2][R2];
#pragma unroll
    for (int i = 0; i < P2; ++i) {
      const int u = tid + i * NT;
      if ((U2 % NT) == 0 || u < U2) {
        const int c = u / R1, k1 = u % R1;
        const float2* yr = buf + c * CW + k1;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) y[i][pos_of<R2>(n2)] = yr[n2 * (R1 + 1)];
        dftR<R2, INV>(y[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < P2; ++i) {
      const int u = tid + i * NT;
      if ((U2 % NT) == 0 || u < U2) {
        const int c = u / R1, k1 = u % R1;
        float2* X = buf + c * CW + k1;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const float2 o = st(y[i][k2], c, k1 + R1 * k2);
          if constexpr (Store::kSmem) X[R1 * k2] = o;
        }
      }
    }
  }
  __syncthreads();
}

template <int L, int TW, int CW, int NT, bool INV, int TWS = 1, class Pre = NoPre, bool PAIR32 = false,
          class Store = RowStore>
__device__ __noinline__ void fft_rowtile_call(float2* buf, const float2* tw, Pre pre = Pre(),
                                              Store st = Store()) {
  fft_rowtile<L, TW, CW, NT, INV, TWS, Pre, PAIR32, Store>(buf, tw, pre, st);
}

// Out-of-line copy for kernels that run several transforms per tile: each
// call gets its own register allocation instead of one inlined body per call.
template <int L, int TW, int PITCH, int NT, bool INV, int TWS = 1, class Load = TileLoad,
          class Store = TileStore>
__device__ __noinline__ void fft_tile_call(float2* buf, const float2* tw, Load ld = Load(),
                                           Store st = Store()) {
  fft_tile<L, TW, PITCH, NT, INV, TWS, Load, Store>(buf, tw, ld, st);
}

// Signed frequency index of position n in a length-N transform.
__device__ __forceinline__ int freq_index(int n, int N) { return n < (N >> 1) ? n : n - N; }

}  // namespace cola
