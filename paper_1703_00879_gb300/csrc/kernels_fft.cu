// FFT passes of the PM step, with the k-space operations of the method fused
// into the passes that already hold the data in shared memory.
//
// A 3-D real transform is three passes over HBM: rows along x (contiguous,
// real <-> half spectrum by the two-for-one packing z = x[2j] + i x[2j+1]),
// then columns along y and along z (tiles of TW adjacent kx columns, so every
// row segment of a tile is one or more whole 32-byte sectors).  Fusions:
//   * the z pass of a forward transform also applies the Green's function
//     (and G_eff, screening coupling, gradient) and runs the inverse z pass of
//     each output before writing it back (Poisson solve, App. B);
//   * the y inverse pass can emit the y derivative as a second output;
//   * the x inverse pass can apply the x derivative on load;
//   * the screening source S = delta * eps is formed between an inverse and a
//     forward x pass in one kernel (Sec. 6.1, Sec. 6.2);
//   * the LPT reweight by the per-k growth tables (Sec. 4.1, App. A) happens
//     on load of the z inverse pass.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cola_internal.h"
#include "fft.cuh"

namespace cola {
namespace {

constexpr int NT = 256;

template <int N>
struct Tiles {
  static constexpr int col1 = N <= 512 ? 16 : 8;                                  // 1 buffer
  static constexpr int col2 = N <= 256 ? 16 : (N == 512 ? 8 : 4);                 // 2 buffers
  static constexpr int col4 = N <= 128 ? 16 : (N == 256 ? 8 : (N == 512 ? 4 : 2));  // 4 buffers
  static constexpr int rows = N <= 512 ? 16 : 8;                                  // x pass rows
};

template <class K>
cudaError_t prep_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  return cudaSuccess;
}

__device__ __forceinline__ void load_tw(float2* tw, const float2* __restrict__ twg, int n) {
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
}

// ---------------------------------------------------------------- column tiles
// Tile element (n, c) of sub-block `sub` lives at buf[n * TP + sub * TW + c];
// global element at g[base + n * sn + c], valid for c0 + c < nvalid.
template <int N, int TW, int TP>
__device__ __forceinline__ void col_load(float2* buf, int sub, const float2* __restrict__ g,
                                         int64_t base, int64_t sn, int c0, int nvalid) {
#pragma unroll 4
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    float2 v = make_float2(0.f, 0.f);
    if (c0 + c < nvalid) v = g[base + (int64_t)n * sn + c];
    buf[n * TP + sub * TW + c] = v;
  }
}

template <int N, int TW, int TP>
__device__ __forceinline__ void col_store(const float2* buf, int sub, float2* __restrict__ g,
                                          int64_t base, int64_t sn, int c0, int nvalid) {
#pragma unroll 4
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    if (c0 + c < nvalid) g[base + (int64_t)n * sn + c] = buf[n * TP + sub * TW + c];
  }
}

// 16-bit seed loads: one 32-bit word holds (re, im).
template <int PREC>
__device__ __forceinline__ float2 seed_value(const void* __restrict__ g, int64_t i, float scale) {
  if constexpr (PREC == 0) {
    return static_cast<const float2*>(g)[i];
  } else {
    const uint32_t w = static_cast<const uint32_t*>(g)[i];
    float re, im;
    if constexpr (PREC == 1) {
      re = __uint_as_float(w << 16);
      im = __uint_as_float(w & 0xFFFF0000u);
    } else {
      re = __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu)));
      im = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    }
    return make_float2(re * scale, im * scale);
  }
}

template <int N, int TW, int TP, int PREC>
__device__ __forceinline__ void col_load_seed(float2* buf, int sub, const void* __restrict__ g,
                                              int64_t base, int64_t sn, int c0, int nvalid,
                                              float scale) {
#pragma unroll 4
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    float2 v = make_float2(0.f, 0.f);
    if (c0 + c < nvalid) v = seed_value<PREC>(g, base + (int64_t)n * sn + c, scale);
    buf[n * TP + sub * TW + c] = v;
  }
}

// ---------------------------------------------------------------- plain column pass
template <int N, int TW, bool INV>
__global__ void __launch_bounds__(NT) k_col(float2* __restrict__ data, int64_t sn, int64_t so,
                                            const float2* __restrict__ twg) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int c0 = blockIdx.x * TW;
  const int64_t base = (int64_t)blockIdx.y * so + c0;
  col_load<N, TW, TW>(buf, 0, data, base, sn, c0, N / 2 + 1);
  __syncthreads();
  fft_tile<N, TW, TW, NT, INV>(buf, tw);
  col_store<N, TW, TW>(buf, 0, data, base, sn, c0, N / 2 + 1);
}

// ---------------------------------------------------------------- y inverse, two outputs
template <int N, int TW>
__global__ void __launch_bounds__(NT) k_yinv2(const float2* __restrict__ in,
                                              float2* __restrict__ outp,
                                              float2* __restrict__ outd, int64_t P, float kfs,
                                              const float2* __restrict__ twg) {
  constexpr int TP = 2 * TW;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int c0 = blockIdx.x * TW;
  const int64_t base = (int64_t)blockIdx.y * N * P + c0;
  col_load<N, TW, TP>(buf, 0, in, base, P, c0, N / 2 + 1);
  __syncthreads();
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    const float f = (n == N / 2) ? 0.f : kfs * (float)freq_index(n, N);
    buf[n * TP + TW + c] = cscale(cmul_i(buf[n * TP + c]), f);
  }
  __syncthreads();
  fft_tile<N, TP, TP, NT, true>(buf, tw);
  col_store<N, TW, TP>(buf, 0, outp, base, P, c0, N / 2 + 1);
  col_store<N, TW, TP>(buf, 1, outd, base, P, c0, N / 2 + 1);
}

__device__ __forceinline__ float kk2(int ix, int iy, int iz, int N, float kf) {
  const float fx = (float)ix, fy = (float)freq_index(iy, N), fz = (float)freq_index(iz, N);
  return kf * kf * (fx * fx + fy * fy + fz * fz);
}

// ---------------------------------------------------------------- screening field (z pass)
template <int N, int TW, int MODEL>
__global__ void __launch_bounds__(NT) k_z_screen_field(const float2* __restrict__ in,
                                                       float2* __restrict__ dk_out,
                                                       float2* __restrict__ w_out, int64_t P,
                                                       ForceParams fp,
                                                       const float2* __restrict__ twg) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int c0 = blockIdx.x * TW;
  const int iy = blockIdx.y;
  const int64_t base = (int64_t)iy * P + c0;
  const int64_t sn = (int64_t)N * P;
  col_load<N, TW, TW>(buf, 0, in, base, sn, c0, N / 2 + 1);
  __syncthreads();
  fft_tile<N, TW, TW, NT, false>(buf, tw);
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    const float2 v = buf[n * TW + c];
    if (c0 + c < N / 2 + 1) dk_out[base + (int64_t)n * sn + c] = v;
    const float k2 = kk2(c0 + c, iy, n, N, fp.kf);
    float m = 0.f;
    if (k2 > 0.f) {
      if (MODEL == 1) m = -fp.kappa_norm / k2;
      else m = __expf(-k2 * fp.R2half) * fp.norm;
    }
    buf[n * TW + c] = cscale(v, m);
  }
  __syncthreads();
  fft_tile<N, TW, TW, NT, true>(buf, tw);
  col_store<N, TW, TW>(buf, 0, w_out, base, sn, c0, N / 2 + 1);
}

// ---------------------------------------------------------------- force (z pass)
template <int N, int TW, bool SCREENED, bool KEEP>
__global__ void __launch_bounds__(NT) k_z_force(const float2* __restrict__ in,
                                                const float2* __restrict__ dk,
                                                float2* __restrict__ phi_out,
                                                float2* __restrict__ phiz_out,
                                                float2* __restrict__ dk_keep, int64_t P,
                                                ForceParams fp, const float2* __restrict__ twg) {
  constexpr int TP = 2 * TW;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int c0 = blockIdx.x * TW;
  const int iy = blockIdx.y;
  const int64_t base = (int64_t)iy * P + c0;
  const int64_t sn = (int64_t)N * P;
  col_load<N, TW, TP>(buf, 0, in, base, sn, c0, N / 2 + 1);
  if (SCREENED) col_load<N, TW, TP>(buf, 1, dk, base, sn, c0, N / 2 + 1);
  __syncthreads();
  fft_tile<N, TW, TP, NT, false>(buf, tw);
  if (KEEP) col_store<N, TW, TP>(buf, 0, dk_keep, base, sn, c0, N / 2 + 1);
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    const float k2 = kk2(c0 + c, iy, n, N, fp.kf);
    float2 phi = make_float2(0.f, 0.f);
    if (k2 > 0.f) {
      const float yuk = k2 / (k2 + fp.a2m2);
      const float g = -fp.kappa_norm / k2;
      const float2 src = buf[n * TP + c];
      if (SCREENED) {
        const float2 d = buf[n * TP + TW + c];
        phi = cscale(cadd(d, cscale(src, fp.C * yuk)), g);
      } else {
        phi = cscale(src, g * (1.f + fp.C * yuk));
      }
    }
    const float kzs = (n == N / 2) ? 0.f : -fp.kf * (float)freq_index(n, N);
    buf[n * TP + c] = phi;
    buf[n * TP + TW + c] = cscale(cmul_i(phi), kzs);
  }
  __syncthreads();
  fft_tile<N, TP, TP, NT, true>(buf, tw);
  col_store<N, TW, TP>(buf, 0, phi_out, base, sn, c0, N / 2 + 1);
  col_store<N, TW, TP>(buf, 1, phiz_out, base, sn, c0, N / 2 + 1);
}

// ---------------------------------------------------------------- LPT reweight (z pass)
template <int N, int TW, int PREC>
__global__ void __launch_bounds__(NT) k_lpt_z(const void* __restrict__ phi1,
                                              const void* __restrict__ phi2,
                                              float2* __restrict__ o0, float2* __restrict__ o1,
                                              float2* __restrict__ o2, float2* __restrict__ o3,
                                              int64_t P, LptParams lp,
                                              const float2* __restrict__ twg) {
  constexpr int TP = 4 * TW;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int c0 = blockIdx.x * TW;
  const int iy = blockIdx.y;
  const int64_t base = (int64_t)iy * P + c0;
  const int64_t sn = (int64_t)N * P;
  col_load_seed<N, TW, TP, PREC>(buf, 0, phi1, base, sn, c0, N / 2 + 1, lp.seed_scale1);
  col_load_seed<N, TW, TP, PREC>(buf, 1, phi2, base, sn, c0, N / 2 + 1, lp.seed_scale2);
  __syncthreads();
  for (int e = threadIdx.x; e < N * TW; e += NT) {
    const int c = e % TW, n = e / TW;
    const float k2 = kk2(c0 + c, iy, n, N, lp.kf);
    float2 d = make_float2(0.f, 0.f), A = make_float2(0.f, 0.f);
    if (k2 > 0.f) {
      const float u = (0.5f * __logf(k2) - lp.lnk0) * lp.inv_dlnk;
      int i = (int)floorf(u);
      i = min(max(i, 0), lp.nk - 2);
      const float f = u - (float)i;
      const float4 t0 = lp.tab[i], t1 = lp.tab[i + 1];
      const float c1 = t0.x * (1.f - f) + t1.x * f;
      const float c2 = t0.y * (1.f - f) + t1.y * f;
      const float e1 = t0.z * (1.f - f) + t1.z * f;
      const float e2 = t0.w * (1.f - f) + t1.w * f;
      const float2 p1 = buf[n * TP + c], p2 = buf[n * TP + TW + c];
      d = cscale(cadd(cscale(p1, c1), cscale(p2, c2)), lp.norm);
      A = cscale(cadd(cscale(p1, e1), cscale(p2, e2)), lp.norm);
    }
    const float kz = (n == N / 2) ? 0.f : lp.kf * (float)freq_index(n, N);
    buf[n * TP + c] = d;
    buf[n * TP + TW + c] = cscale(cmul_i(d), kz);
    buf[n * TP + 2 * TW + c] = A;
    buf[n * TP + 3 * TW + c] = cscale(cmul_i(A), kz);
  }
  __syncthreads();
  fft_tile<N, TP, TP, NT, true>(buf, tw);
  col_store<N, TW, TP>(buf, 0, o0, base, sn, c0, N / 2 + 1);
  col_store<N, TW, TP>(buf, 1, o1, base, sn, c0, N / 2 + 1);
  col_store<N, TW, TP>(buf, 2, o2, base, sn, c0, N / 2 + 1);
  col_store<N, TW, TP>(buf, 3, o3, base, sn, c0, N / 2 + 1);
}

// ---------------------------------------------------------------- x passes (rows)
// r2c post-processing: X[k] = (Z[k] + conj Z[M-k])/2 - i/2 w^k (Z[k] - conj Z[M-k]).
template <int N, int TWX, int PITCH>
__device__ __forceinline__ void row_r2c_store(const float2* buf, const float2* tw,
                                              float2* __restrict__ out, int64_t row0,
                                              int64_t P) {
  constexpr int M = N / 2;
#pragma unroll 2
  for (int e = threadIdx.x; e < TWX * (M + 1); e += NT) {
    const int r = e / (M + 1), k = e - r * (M + 1);
    const float2 a = buf[(k & (M - 1)) * PITCH + r];
    const float2 b = cconj(buf[((M - k) & (M - 1)) * PITCH + r]);
    const float2 E = cscale(cadd(a, b), 0.5f);
    const float2 D = csub(a, b);
    const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // (-i/2) D
    out[(row0 + r) * P + k] = cadd(E, cmul(tw[k], O));
  }
}

// c2r pre-processing (unnormalised inverse, 2x folded in):
// E = X[k] + conj X[M-k], O = w^-k (X[k] - conj X[M-k]), Z[k] = E + i O,
// Z[M-k] = conj E + i conj O.  Imaginary parts of X[0], X[M] are dropped.
template <int N, int TWX, int PITCH>
__device__ __forceinline__ void row_c2r_load(float2* buf, const float2* tw,
                                             const float2* __restrict__ in, int64_t row0,
                                             int64_t P, float kfs) {
  constexpr int M = N / 2;
#pragma unroll 2
  for (int e = threadIdx.x; e < TWX * (M + 1); e += NT) {
    const int r = e / (M + 1), k = e - r * (M + 1);
    float2 v = in[(row0 + r) * P + k];
    if (kfs != 0.f) v = (k == M) ? make_float2(0.f, 0.f) : cscale(cmul_i(v), kfs * (float)k);
    if (k == 0 || k == M) v.y = 0.f;
    buf[k * PITCH + r] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TWX * (M / 2 + 1); e += NT) {
    const int r = e / (M / 2 + 1), k = e - r * (M / 2 + 1);
    const float2 a = buf[k * PITCH + r];
    const float2 b = cconj(buf[(M - k) * PITCH + r]);
    const float2 E = cadd(a, b);
    const float2 O = cmul(cconj(tw[k]), csub(a, b));
    const float2 Z = cadd(E, cmul_i(O));
    buf[k * PITCH + r] = Z;
    if (k != 0 && k != M - k) buf[(M - k) * PITCH + r] = cadd(cconj(E), cmul_i(cconj(O)));
  }
  __syncthreads();
}

template <int N, int TWX>
__global__ void __launch_bounds__(NT) k_xr2c(const float* __restrict__ in,
                                             float2* __restrict__ out, int64_t P, float scale,
                                             float offset, const float2* __restrict__ twg) {
  constexpr int M = N / 2, PITCH = TWX + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int64_t row0 = (int64_t)blockIdx.x * TWX;
#pragma unroll 4
  for (int e = threadIdx.x; e < TWX * M; e += NT) {
    const int r = e / M, j = e % M;
    float2 v = reinterpret_cast<const float2*>(in + (row0 + r) * N)[j];
    v.x = v.x * scale + offset;
    v.y = v.y * scale + offset;
    buf[j * PITCH + r] = v;
  }
  __syncthreads();
  fft_tile<M, TWX, PITCH, NT, false, 2>(buf, tw);
  row_r2c_store<N, TWX, PITCH>(buf, tw, out, row0, P);
}

template <int N, int TWX>
__global__ void __launch_bounds__(NT) k_xc2r(const float2* __restrict__ in,
                                             float* __restrict__ out, int64_t P, float kfs,
                                             const float2* __restrict__ twg) {
  constexpr int M = N / 2, PITCH = TWX + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int64_t row0 = (int64_t)blockIdx.x * TWX;
  __syncthreads();
  row_c2r_load<N, TWX, PITCH>(buf, tw, in, row0, P, kfs);
  fft_tile<M, TWX, PITCH, NT, true, 2>(buf, tw);
#pragma unroll 4
  for (int e = threadIdx.x; e < TWX * M; e += NT) {
    const int r = e / M, j = e % M;
    reinterpret_cast<float2*>(out + (row0 + r) * N)[j] = buf[j * PITCH + r];
  }
}

template <int MODEL>
__device__ __forceinline__ float screen_eps(float w, const ForceParams& fp) {
  if (MODEL == 1) {
    const float aw = fabsf(w);
    return aw > fp.fr_thr ? fp.fr_thr / aw : 1.f;
  } else {
    const float x = fp.dgp_coef * fmaxf(1.f + w, 0.f);
    return 2.f / (sqrtf(1.f + x) + 1.f);
  }
}

template <int N, int TWX, int MODEL>
__global__ void __launch_bounds__(NT) k_x_screen(const float2* __restrict__ w_in,
                                                 const float* __restrict__ rho,
                                                 float2* __restrict__ s_out, int64_t P,
                                                 ForceParams fp,
                                                 const float2* __restrict__ twg) {
  constexpr int M = N / 2, PITCH = TWX + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_tw(tw, twg, N);
  const int64_t row0 = (int64_t)blockIdx.x * TWX;
  __syncthreads();
  row_c2r_load<N, TWX, PITCH>(buf, tw, w_in, row0, P, 0.f);
  fft_tile<M, TWX, PITCH, NT, true, 2>(buf, tw);
#pragma unroll 4
  for (int e = threadIdx.x; e < TWX * M; e += NT) {
    const int r = e / M, j = e % M;
    const float2 w = buf[j * PITCH + r];
    const float2 rr = reinterpret_cast<const float2*>(rho + (row0 + r) * N)[j];
    const float d0 = rr.x * fp.inv_rhobar - 1.f, d1 = rr.y * fp.inv_rhobar - 1.f;
    buf[j * PITCH + r] = make_float2(d0 * screen_eps<MODEL>(w.x, fp), d1 * screen_eps<MODEL>(w.y, fp));
  }
  __syncthreads();
  fft_tile<M, TWX, PITCH, NT, false, 2>(buf, tw);
  row_r2c_store<N, TWX, PITCH>(buf, tw, s_out, row0, P);
}

}  // namespace

#define COLA_SWITCH_N(NVAL, ...)                 \
  switch (NVAL) {                                \
    case 32: { constexpr int N = 32; __VA_ARGS__; } break;     \
    case 64: { constexpr int N = 64; __VA_ARGS__; } break;     \
    case 128: { constexpr int N = 128; __VA_ARGS__; } break;   \
    case 256: { constexpr int N = 256; __VA_ARGS__; } break;   \
    case 512: { constexpr int N = 512; __VA_ARGS__; } break;   \
    case 1024: { constexpr int N = 1024; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;       \
  }

template <int N>
static cudaError_t launch_xr2c(const float* in, float2* out, float scale, float offset,
                               const float2* tw, cudaStream_t s) {
  constexpr int TWX = Tiles<N>::rows;
  const size_t sm = (N + (N / 2) * (TWX + 1)) * sizeof(float2);
  auto k = k_xr2c<N, TWX>;
  cudaError_t e = prep_smem(k, sm);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)((int64_t)N * N / TWX), NT, sm, s>>>(in, out, half_pitch(N), scale, offset, tw);
  return cudaGetLastError();
}

cudaError_t fft_xr2c(int Nv, const float* in, float2* out, float scale, float offset,
                     const float2* tw, cudaStream_t s) {
  COLA_SWITCH_N(Nv, return launch_xr2c<N>(in, out, scale, offset, tw, s));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_xc2r(const float2* in, float* out, float kfs, const float2* tw,
                               cudaStream_t s) {
  constexpr int TWX = Tiles<N>::rows;
  const size_t sm = (N + (N / 2 + 1) * (TWX + 1)) * sizeof(float2);
  auto k = k_xc2r<N, TWX>;
  cudaError_t e = prep_smem(k, sm);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)((int64_t)N * N / TWX), NT, sm, s>>>(in, out, half_pitch(N), kfs, tw);
  return cudaGetLastError();
}

cudaError_t fft_xc2r(int Nv, const float2* in, float* out, float kfs, const float2* tw,
                     cudaStream_t s) {
  COLA_SWITCH_N(Nv, return launch_xc2r<N>(in, out, kfs, tw, s));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_col(float2* data, int axis, bool inv, const float2* tw,
                              cudaStream_t s) {
  constexpr int TW = Tiles<N>::col1;
  const int64_t P = half_pitch(N);
  const int64_t sn = axis == 1 ? P : (int64_t)N * P;
  const int64_t so = axis == 1 ? (int64_t)N * P : P;
  const size_t sm = (N + (size_t)N * TW) * sizeof(float2);
  dim3 grid((N / 2) / TW + 1, N);
  if (inv) {
    auto k = k_col<N, TW, true>;
    cudaError_t e = prep_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(data, sn, so, tw);
  } else {
    auto k = k_col<N, TW, false>;
    cudaError_t e = prep_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(data, sn, so, tw);
  }
  return cudaGetLastError();
}

cudaError_t fft_col(int Nv, float2* data, int axis, bool inv, const float2* tw, cudaStream_t s) {
  COLA_SWITCH_N(Nv, return launch_col<N>(data, axis, inv, tw, s));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_yinv2(const float2* in, float2* outp, float2* outd, float kfs,
                                const float2* tw, cudaStream_t s) {
  constexpr int TW = Tiles<N>::col2;
  const size_t sm = (N + (size_t)N * 2 * TW) * sizeof(float2);
  auto k = k_yinv2<N, TW>;
  cudaError_t e = prep_smem(k, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((N / 2) / TW + 1, N);
  k<<<grid, NT, sm, s>>>(in, outp, outd, half_pitch(N), kfs, tw);
  return cudaGetLastError();
}

cudaError_t fft_yinv2(int Nv, const float2* in, float2* outp, float2* outd, float kfs,
                      const float2* tw, cudaStream_t s) {
  COLA_SWITCH_N(Nv, return launch_yinv2<N>(in, outp, outd, kfs, tw, s));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_zsf(const float2* in, float2* dk_out, float2* w_out,
                              const ForceParams& fp, const float2* tw, cudaStream_t s) {
  constexpr int TW = Tiles<N>::col1;
  const size_t sm = (N + (size_t)N * TW) * sizeof(float2);
  dim3 grid((N / 2) / TW + 1, N);
  if (fp.model == 1) {
    auto k = k_z_screen_field<N, TW, 1>;
    cudaError_t e = prep_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(in, dk_out, w_out, half_pitch(N), fp, tw);
  } else {
    auto k = k_z_screen_field<N, TW, 2>;
    cudaError_t e = prep_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(in, dk_out, w_out, half_pitch(N), fp, tw);
  }
  return cudaGetLastError();
}

cudaError_t mesh_z_screen_field(int Nv, const float2* in, float2* dk_out, float2* w_out,
                                const ForceParams& fp, const float2* tw, cudaStream_t s) {
  if (fp.model != 1 && fp.model != 2) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_zsf<N>(in, dk_out, w_out, fp, tw, s));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_xscreen(const float2* w_in, const float* rho, float2* s_out,
                                  const ForceParams& fp, const float2* tw, cudaStream_t s) {
  constexpr int TWX = Tiles<N>::rows;
  const size_t sm = (N + (N / 2 + 1) * (TWX + 1)) * sizeof(float2);
  const unsigned grid = (unsigned)((int64_t)N * N / TWX);
  if (fp.model == 1) {
    auto k = k_x_screen<N, TWX, 1>;
    cudaError_t e = prep_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(w_in, rho, s_out, half_pitch(N), fp, tw);
  } else {
    auto k = k_x_screen<N, TWX, 2>;
    cudaError_t e = prep_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(w_in, rho, s_out, half_pitch(N), fp, tw);
  }
  return cudaGetLastError();
}

cudaError_t mesh_x_screen_source(int Nv, const float2* w_in, const float* rho, float2* s_out,
                                 const ForceParams& fp, const float2* tw, cudaStream_t s) {
  if (fp.model != 1 && fp.model != 2) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_xscreen<N>(w_in, rho, s_out, fp, tw, s));
  return cudaSuccess;
}

template <int N, bool SCR, bool KEEP>
static cudaError_t launch_zforce_t(const float2* in, const float2* dk, float2* phi,
                                   float2* phiz, float2* keep, const ForceParams& fp,
                                   const float2* tw, cudaStream_t s) {
  constexpr int TW = Tiles<N>::col2;
  const size_t sm = (N + (size_t)N * 2 * TW) * sizeof(float2);
  auto k = k_z_force<N, TW, SCR, KEEP>;
  cudaError_t e = prep_smem(k, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((N / 2) / TW + 1, N);
  k<<<grid, NT, sm, s>>>(in, dk, phi, phiz, keep, half_pitch(N), fp, tw);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_zforce(const float2* in, const float2* dk, float2* phi, float2* phiz,
                                 float2* keep, const ForceParams& fp, const float2* tw,
                                 cudaStream_t s) {
  if (fp.screened) return launch_zforce_t<N, true, false>(in, dk, phi, phiz, keep, fp, tw, s);
  if (keep) return launch_zforce_t<N, false, true>(in, dk, phi, phiz, keep, fp, tw, s);
  return launch_zforce_t<N, false, false>(in, dk, phi, phiz, keep, fp, tw, s);
}

cudaError_t mesh_z_force(int Nv, const float2* in, const float2* dk, float2* phi_out,
                         float2* phiz_out, float2* dk_keep, const ForceParams& fp,
                         const float2* tw, cudaStream_t s) {
  if (fp.screened && dk == nullptr) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_zforce<N>(in, dk, phi_out, phiz_out, dk_keep, fp, tw, s));
  return cudaSuccess;
}

template <int N, int PREC>
static cudaError_t launch_lpt_t(const void* p1, const void* p2, float2* o0, float2* o1,
                                float2* o2, float2* o3, const LptParams& lp, const float2* tw,
                                cudaStream_t s) {
  constexpr int TW = Tiles<N>::col4;
  const size_t sm = (N + (size_t)N * 4 * TW) * sizeof(float2);
  auto k = k_lpt_z<N, TW, PREC>;
  cudaError_t e = prep_smem(k, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((N / 2) / TW + 1, N);
  k<<<grid, NT, sm, s>>>(p1, p2, o0, o1, o2, o3, half_pitch(N), lp, tw);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_lpt(const void* p1, const void* p2, float2* o0, float2* o1, float2* o2,
                              float2* o3, const LptParams& lp, const float2* tw,
                              cudaStream_t s) {
  if (lp.seed_prec == 1) return launch_lpt_t<N, 1>(p1, p2, o0, o1, o2, o3, lp, tw, s);
  if (lp.seed_prec == 2) return launch_lpt_t<N, 2>(p1, p2, o0, o1, o2, o3, lp, tw, s);
  return launch_lpt_t<N, 0>(p1, p2, o0, o1, o2, o3, lp, tw, s);
}

cudaError_t lpt_z(int Nv, const void* phi1, const void* phi2, float2* o0, float2* o1, float2* o2,
                  float2* o3, const LptParams& lp, const float2* tw, cudaStream_t s) {
  COLA_SWITCH_N(Nv, return launch_lpt<N>(phi1, phi2, o0, o1, o2, o3, lp, tw, s));
  return cudaSuccess;
}

}  // namespace cola
