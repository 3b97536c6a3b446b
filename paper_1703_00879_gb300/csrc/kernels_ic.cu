// Initial-condition kernels (run once per simulation, not on the step path):
// Philox white noise, the Gaussian delta(k), phi1 = delta/k^2 (Sec. 3.1), the
// Hessian of phi1 and the 2LPT source of Eq. lcdm2lpt (Sec. 3.2), phi2, the
// initial particle state, layout packing and reduced-precision seed storage.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "cola_internal.h"

namespace cola {
namespace {

constexpr int NTI = 256;

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + NTI - 1) / NTI); }

// Philox-4x32-10 (Salmon et al., SC'11): ten rounds of the multiply-xor
// bijection with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments
// 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Unit Gaussian per lattice point: counter (idx lo, idx hi, 0, 0), key = seed,
// u_i = (w_i + 1/2) / 2^32, g = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller) in
// single precision: ln u1 from u1 itself below 1/2 and as ln(1 - v) with
// v = (2^32 - 1 - w_1 + 1/2) / 2^32 above, so that every u1 keeps its relative
// precision; the result is within a few ulp of the double-precision formula
// rounded to float (this GPU's double-precision rate made the double version
// 15 ms for 512^3 points).
// Multi-simulation kernels take the simulation from blockIdx.y and move every
// buffer pointer by its shift; per-simulation values come from the header.
__global__ void k_noise(int64_t n, uint32_t k0, uint32_t k1, float* __restrict__ out,
                        const SimHeader* __restrict__ hdr, Multi mm) {
  const int64_t i = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (i >= n) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  out = moved(out, by);
  if (hdr) {
    const unsigned long long sd = moved(hdr, by)->seed;
    k0 = (uint32_t)sd;
    k1 = (uint32_t)(sd >> 32);
  }
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0u), k0, k1);
  const float lu = r.x < 0x80000000u ? logf(((float)r.x + 0.5f) * 0x1p-32f)
                                      : log1pf(-((float)(0xFFFFFFFFu - r.x) + 0.5f) * 0x1p-32f);
  out[i] = sqrtf(-2.f * lu) * cospif(((float)r.y + 0.5f) * 0x1p-31f);  // cos(pi * 2 u2)
}

struct Mode {
  int ix, fy, fz;
  bool nyx, nyy, nyz;
};

// Mode of element m of a half spectrum (layout of cola_internal.h); padding
// elements (kx > N/2) are not valid.
__device__ __forceinline__ Mode mode_of(int64_t m, int N, int64_t P, bool& valid) {
  Mode md;
  const int64_t pr = m / (2 * P);            // (z >> 1) N + y
  const int w = (int)(m - pr * 2 * P);       // position in the interleaved row pair
  const int ix = (w >> 4) * 8 + (w & 7);
  const int iy = (int)(pr % N), iz = (int)(pr / N) * 2 + ((w >> 3) & 1);
  valid = ix <= N / 2;
  md.ix = ix;
  md.fy = iy < N / 2 ? iy : iy - N;
  md.fz = iz < N / 2 ? iz : iz - N;
  md.nyx = ix == N / 2;
  md.nyy = iy == N / 2;
  md.nyz = iz == N / 2;
  return md;
}

// Eisenstein & Hu (1998) no-wiggle transfer function, k in h/Mpc.
__device__ double eh_T(const EHDev& e, double k) {
  const double kmpc = k * e.h;
  const double x = 0.43 * kmpc * e.s;
  const double x2 = x * x;
  const double gamma = e.Omh * (e.alpha + (1.0 - e.alpha) / (1.0 + x2 * x2));
  const double q = k * e.theta2 / gamma;
  const double L0 = log(2.0 * 2.718281828459045235 + 1.8 * q);
  const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return L0 / (L0 + C0 * q * q);
}

// The factor of phi1(k) = f(|n|^2) delta(k) (Sec. 3.1), f = sqrt(P(k) N^3 / L^3) / k^2
// with k = kf |n|, depends on the integer |n|^2 only: one double-precision
// evaluation per value 0 .. 3 (N/2)^2 into tab (each simulation its own table)
// instead of one per mode.
__global__ void k_ic_amp(int N, double* __restrict__ tab, float kf, EHDev eh,
                         const SimHeader* __restrict__ hdr, Multi mm) {
  const int64_t q = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (q > 3LL * (N / 2) * (N / 2)) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  tab = moved(tab, by);
  if (hdr) eh = moved(hdr, by)->eh;
  if (q == 0) {
    tab[0] = 0.0;
    return;
  }
  const double k = (double)kf * sqrt((double)q);
  const double T = eh_T(eh, k);
  const double pk = eh.amp * pow(k, eh.ns) * T * T;
  tab[q] = sqrt(pk * eh.N3_over_L3) / (k * k);
}

__global__ void k_ic_phi1(int N, int64_t P, float2* __restrict__ c, const double* __restrict__ tab,
                          Multi mm) {
  const int64_t m = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (m >= (int64_t)N * N * P) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  c = moved(c, by);
  tab = moved(tab, by);
  bool valid;
  const Mode md = mode_of(m, N, P, valid);
  if (!valid) return;
  const double f = tab[md.ix * md.ix + md.fy * md.fy + md.fz * md.fz];  // 0 at k = 0
  const float2 v = c[m];
  c[m] = make_float2((float)(v.x * f), (float)(v.y * f));
}

__global__ void k_ic_hessian(int N, int64_t P, const float2* __restrict__ phi1,
                             float2* __restrict__ out, int i, int j, float kf, float norm, Multi mm) {
  const int64_t m = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (m >= (int64_t)N * N * P) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  phi1 = moved(phi1, by);
  out = moved(out, by);
  bool valid;
  const Mode md = mode_of(m, N, P, valid);
  if (!valid) return;
  const float kv[3] = {kf * md.ix, kf * md.fy, kf * md.fz};
  const bool ny[3] = {md.nyx, md.nyy, md.nyz};
  float f = -kv[i] * kv[j] * norm;
  if (i != j && (ny[i] || ny[j])) f = 0.f;
  const float2 v = phi1[m];
  out[m] = make_float2(v.x * f, v.y * f);
}

// sum_{i<j} (phi_ii phi_jj - phi_ij^2) = 1/2 [(lap phi)^2 - (phi_ij)^2]
__global__ void k_ic_source(int64_t n, const float* __restrict__ hxx,
                            const float* __restrict__ hyy, const float* __restrict__ hzz,
                            const float* __restrict__ hxy, const float* __restrict__ hxz,
                            const float* __restrict__ hyz, float* __restrict__ src, Multi mm) {
  const int64_t i = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (i >= n) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  hxx = moved(hxx, by);
  hyy = moved(hyy, by);
  hzz = moved(hzz, by);
  hxy = moved(hxy, by);
  hxz = moved(hxz, by);
  hyz = moved(hyz, by);
  src = moved(src, by);
  const float a = hxx[i], b = hyy[i], c = hzz[i], d = hxy[i], e = hxz[i], f = hyz[i];
  src[i] = (a * b - d * d) + (a * c - e * e) + (b * c - f * f);
}

__global__ void k_ic_phi2(int N, int64_t P, float2* __restrict__ c, float kf, Multi mm) {
  const int64_t m = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (m >= (int64_t)N * N * P) return;
  c = moved(c, shift_of(mm, blockIdx.y));
  bool valid;
  const Mode md = mode_of(m, N, P, valid);
  if (!valid) return;
  const float k2 = kf * kf * ((float)md.ix * md.ix + (float)md.fy * md.fy + (float)md.fz * md.fz);
  const float2 v = c[m];
  c[m] = k2 > 0.f ? make_float2(-v.x / k2, -v.y / k2) : make_float2(0.f, 0.f);
}

__global__ void k_ic_particles(int64_t P, const float* __restrict__ px,
                               const float* __restrict__ py, const float* __restrict__ pz,
                               float* __restrict__ sx, float* __restrict__ sy,
                               float* __restrict__ sz, float* __restrict__ vx,
                               float* __restrict__ vy, float* __restrict__ vz, Multi mm,
                               LptMix mix) {
  const int64_t i = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (i >= P) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  px = moved(px, by);
  py = moved(py, by);
  pz = moved(pz, by);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  vx = moved(vx, by);
  vy = moved(vy, by);
  vz = moved(vz, by);
  if (mix.on) {  // s = D1 Psi1 + D2 Psi2 at a_ini
    const float4 cf = mix_coeffs(mix, by);
    sx[i] = cf.x * px[i] + cf.y * moved(mix.q2[0], by)[i];
    sy[i] = cf.x * py[i] + cf.y * moved(mix.q2[1], by)[i];
    sz[i] = cf.x * pz[i] + cf.y * moved(mix.q2[2], by)[i];
  } else {
    sx[i] = px[i];
    sy[i] = py[i];
    sz[i] = pz[i];
  }
  vx[i] = 0.f;
  vy[i] = 0.f;
  vz[i] = 0.f;
}

__global__ void k_half_pack(int N, int64_t P, const float2* __restrict__ dense,
                            float2* __restrict__ padded, bool to_padded) {
  const int64_t W = N / 2 + 1;
  const int64_t m = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (m >= (int64_t)N * N * W) return;
  const int64_t row = m / W;  // z N + y of the dense [z][y][kx] array
  const int64_t at = hidx((int)(row / N), (int)(row % N), (int)(m % W), N, P);
  if (to_padded) padded[at] = dense[m];
  else const_cast<float2*>(dense)[m] = padded[at];
}

__global__ void k_absmax(int64_t n, int N, int64_t P, const float2* __restrict__ src,
                         unsigned int* __restrict__ out, Multi mm) {
  const int64_t by = shift_of(mm, blockIdx.y);
  src = moved(src, by);
  out = moved(out, by);
  float mx = 0.f;
  for (int64_t m = (int64_t)blockIdx.x * NTI + threadIdx.x; m < n;
       m += (int64_t)gridDim.x * NTI) {
    const int w = (int)(m % (2 * P));
    if ((w >> 4) * 8 + (w & 7) > N / 2) continue;  // padding (kx > N/2)
    const float2 v = src[m];
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

__global__ void k_seed_scale(SimHeader* hdr, const float* __restrict__ absmax, int f, Multi mm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= mm.nb) return;
  const int64_t by = shift_of(mm, b);
  SimHeader* h = moved(hdr, by);
  const float amax = *moved(absmax, by);
  h->seed_scale[f] = amax > 0.f ? amax / h->seed_target : 1.f;
}

__global__ void k_quantise(int64_t n, const float2* __restrict__ src, uint32_t* __restrict__ dst,
                           int prec, const SimHeader* __restrict__ hdr, int f, Multi mm) {
  const int64_t m = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (m >= n) return;
  const int64_t by = shift_of(mm, blockIdx.y);
  src = moved(src, by);
  dst = moved(dst, by);
  const float inv_scale = 1.f / moved(hdr, by)->seed_scale[f];
  const float2 v = src[m];
  uint32_t lo, hi;
  if (prec == 1) {
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(v.x * inv_scale));
    hi = __bfloat16_as_ushort(__float2bfloat16_rn(v.y * inv_scale));
  } else {
    lo = __half_as_ushort(__float2half_rn(v.x * inv_scale));
    hi = __half_as_ushort(__float2half_rn(v.y * inv_scale));
  }
  dst[m] = lo | (hi << 16);
}

}  // namespace

cudaError_t ic_noise(int N, uint64_t seed, float* out, cudaStream_t s, Multi m, const SimHeader* hdr) {
  const int64_t n = (int64_t)N * N * N;
  k_noise<<<dim3(blocks_for(n), m.nb), NTI, 0, s>>>(n, (uint32_t)seed, (uint32_t)(seed >> 32), out, hdr, m);
  return cudaGetLastError();
}

cudaError_t ic_phi1(int N, float2* c, float kf, const EHDev& eh, double* work, cudaStream_t s, Multi m,
                    const SimHeader* hdr) {
  const int64_t nq = 3LL * (N / 2) * (N / 2) + 1;
  k_ic_amp<<<dim3(blocks_for(nq), m.nb), NTI, 0, s>>>(N, work, kf, eh, hdr, m);
  const int64_t n = half_elems(N);
  k_ic_phi1<<<dim3(blocks_for(n), m.nb), NTI, 0, s>>>(N, half_pitch(N), c, work, m);
  return cudaGetLastError();
}

cudaError_t ic_hessian(int N, const float2* phi1, float2* out, int i, int j, float kf,
                       cudaStream_t s, Multi m) {
  const int64_t n = half_elems(N);
  const float norm = (float)(1.0 / ((double)N * N * N));
  k_ic_hessian<<<dim3(blocks_for(n), m.nb), NTI, 0, s>>>(N, half_pitch(N), phi1, out, i, j, kf, norm, m);
  return cudaGetLastError();
}

cudaError_t ic_source(int64_t n, const float* hxx, const float* hyy, const float* hzz,
                      const float* hxy, const float* hxz, const float* hyz, float* src,
                      cudaStream_t s, Multi m) {
  k_ic_source<<<dim3(blocks_for(n), m.nb), NTI, 0, s>>>(n, hxx, hyy, hzz, hxy, hxz, hyz, src, m);
  return cudaGetLastError();
}

cudaError_t ic_phi2(int N, float2* c, float kf, cudaStream_t s, Multi m) {
  const int64_t n = half_elems(N);
  k_ic_phi2<<<dim3(blocks_for(n), m.nb), NTI, 0, s>>>(N, half_pitch(N), c, kf, m);
  return cudaGetLastError();
}

cudaError_t ic_particles(int64_t P, const float* px, const float* py, const float* pz, float* sx,
                         float* sy, float* sz, float* vx, float* vy, float* vz,
                         cudaStream_t s, Multi m, LptMix mix) {
  k_ic_particles<<<dim3(blocks_for(P), m.nb), NTI, 0, s>>>(P, px, py, pz, sx, sy, sz, vx, vy, vz, m,
                                                           mix);
  return cudaGetLastError();
}

namespace {
__global__ void k_lpt_mix(int64_t P, const float* __restrict__ p0, const float* __restrict__ p1,
                          const float* __restrict__ p2, LptMix mix, int acc, float* __restrict__ o0,
                          float* __restrict__ o1, float* __restrict__ o2) {
  const int64_t i = (int64_t)blockIdx.x * NTI + threadIdx.x;
  if (i >= P) return;
  const float4 cf = mix_coeffs(mix, 0);
  const float a = acc ? cf.z : cf.x, b = acc ? cf.w : cf.y;
  o0[i] = a * p0[i] + b * mix.q2[0][i];
  o1[i] = a * p1[i] + b * mix.q2[1][i];
  o2[i] = a * p2[i] + b * mix.q2[2][i];
}
}  // namespace

cudaError_t lpt_mix(int64_t P, const float* const* psi1, const LptMix& mix, int acc, float* const* out,
                    cudaStream_t s) {
  k_lpt_mix<<<blocks_for(P), NTI, 0, s>>>(P, psi1[0], psi1[1], psi1[2], mix, acc, out[0], out[1], out[2]);
  return cudaGetLastError();
}

cudaError_t half_pack(int N, const float2* dense, float2* padded, cudaStream_t s) {
  const int64_t n = (int64_t)N * N * (N / 2 + 1);
  k_half_pack<<<blocks_for(n), NTI, 0, s>>>(N, half_pitch(N), dense, padded, true);
  return cudaGetLastError();
}

cudaError_t half_unpack(int N, const float2* padded, float2* dense, cudaStream_t s) {
  const int64_t n = (int64_t)N * N * (N / 2 + 1);
  k_half_pack<<<blocks_for(n), NTI, 0, s>>>(N, half_pitch(N), dense, const_cast<float2*>(padded),
                                            false);
  return cudaGetLastError();
}

cudaError_t seed_absmax(int N, const float2* src, float* out_absmax, cudaStream_t s, Multi m) {
  const int64_t n = half_elems(N);
  cudaError_t e = zero_f32(out_absmax, 4, s, m);  // the float and its 16-byte group
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n + NTI - 1) / NTI, 152 * 16 / std::min(m.nb, 16)));
  k_absmax<<<dim3(grid, m.nb), NTI, 0, s>>>(n, N, half_pitch(N), src,
                                            reinterpret_cast<unsigned int*>(out_absmax), m);
  return cudaGetLastError();
}

cudaError_t seed_scale_set(SimHeader* hdr, const float* absmax, int f, cudaStream_t s, Multi m) {
  k_seed_scale<<<(m.nb + 127) / 128, 128, 0, s>>>(hdr, absmax, f, m);
  return cudaGetLastError();
}

cudaError_t seed_quantise(int N, const float2* src, void* dst, int prec, const SimHeader* hdr, int f,
                          cudaStream_t s, Multi m) {
  const int64_t n = half_elems(N);
  k_quantise<<<dim3(blocks_for(n), m.nb), NTI, 0, s>>>(n, src, static_cast<uint32_t*>(dst), prec, hdr,
                                                       f, m);
  return cudaGetLastError();
}

}  // namespace cola
