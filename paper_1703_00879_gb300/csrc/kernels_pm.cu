// Particle kernels of the COLA step: drift with cloud-in-cell deposit, CIC
// gather with kick, snapshot, and the P(k) binning.
//
// Particles stay in Lagrangian order (p = (z Np + y) Np + x), so the lattice
// point q is implicit and the LPT fields are read at index p (App. A: each
// particle needs the displacement field at its original lattice point).  The
// displacement s = x - q is stored instead of x, and the mesh coordinate is
// formed as integer + fraction (q's cell split exactly, then s Nm/L added to the
// fractional part), so float positions keep ~1e-6 cell resolution at any box size.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "cola_internal.h"

namespace cola {
namespace {

constexpr int NTP = 256;

// Value of a 16-bit field entry (prec 1 bf16, 2 fp16), before its field scale.
__device__ __forceinline__ float lq_value(unsigned short u, int prec) {
  return prec == 1 ? __bfloat162float(__ushort_as_bfloat16(u)) : __half2float(__ushort_as_half(u));
}

struct Cic {
  int i0[3], i1[3];
  float f[3];
};

// Cell indices and CIC fractions of the particle at lattice (ix, iy, iz) with displacement s.
__device__ __forceinline__ Cic cic_setup(const PartParams& pp, int ix, int iy, int iz, float sx,
                                        float sy, float sz) {
  Cic c;
  const int li[3] = {ix, iy, iz};
  const float sv[3] = {sx, sy, sz};
  const int mask = pp.Nm - 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int num = li[d] * pp.Nm;  // q in cells = num / Np
    const int base = num >> pp.lgNp;
    // (num mod Np) / Np, exact: the division by Np = 2^lgNp is a multiplication
    // by the float with exponent field 127 - lgNp (lgNp <= 12)
    const float qf = (float)(num - (base << pp.lgNp)) * __int_as_float((127 - pp.lgNp) << 23);
    const float u = qf + sv[d] * pp.cellscale;
    const float fl = floorf(u);
    c.f[d] = u - fl;
    c.i0[d] = (base + (int)fl) & mask;
    c.i1[d] = (c.i0[d] + 1) & mask;
  }
  return c;
}

// Non-returning global reductions.  atomicAdd on a float4 returns the old
// value, and those returns cost as much crossbar traffic as the additions
// themselves (ncu: as many xbar-to-L1 sectors as L1-to-xbar sectors); the
// deposit never reads them.
__device__ __forceinline__ void red_add4(float* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// Adds a0 at row[i0] and a1 at row[i1] (i1 = i0 + 1, or 0 when i0 ends the
// row).  One vector reduction (red.global.add.v4.f32, zeros in the other lanes)
// covers the 16-byte group of i0 and, unless i0 is the group's last cell, i1;
// otherwise (q = 3, which includes the wrap: Nm is a multiple of 4) a scalar
// reduction adds a1.  Every lane issues the vector reduction, so a warp runs two
// reduction instructions per call rather than three on divergent paths.
__device__ __forceinline__ void row_add(float* __restrict__ row, int i0, int i1, float a0, float a1) {
  const int q = i0 & 3;
  const float4 v = make_float4(q == 0 ? a0 : 0.f, q == 1 ? a0 : (q == 0 ? a1 : 0.f),
                               q == 2 ? a0 : (q == 1 ? a1 : 0.f), q == 3 ? a0 : (q == 2 ? a1 : 0.f));
  red_add4(row + (i0 - q), v);
  if (q == 3) red_add(row + i1, a1);
}

__device__ __forceinline__ void cic_deposit(float* __restrict__ rho, int Nm, const Cic& c) {
  const float wx0 = 1.f - c.f[0], wx1 = c.f[0];
  const float wy0 = 1.f - c.f[1], wy1 = c.f[1];
  const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
  const int64_t z0 = (int64_t)c.i0[2] * Nm, z1 = (int64_t)c.i1[2] * Nm;
  const int64_t r00 = (z0 + c.i0[1]) * Nm, r01 = (z0 + c.i1[1]) * Nm;
  const int64_t r10 = (z1 + c.i0[1]) * Nm, r11 = (z1 + c.i1[1]) * Nm;
  const float w00 = wz0 * wy0, w01 = wz0 * wy1, w10 = wz1 * wy0, w11 = wz1 * wy1;
  row_add(rho + r00, c.i0[0], c.i1[0], w00 * wx0, w00 * wx1);
  row_add(rho + r01, c.i0[0], c.i1[0], w01 * wx0, w01 * wx1);
  row_add(rho + r10, c.i0[0], c.i1[0], w10 * wx0, w10 * wx1);
  row_add(rho + r11, c.i0[0], c.i1[0], w11 * wx0, w11 * wx1);
}

// CIC deposit from a whole warp (every lane calls it; `valid` marks real
// particles).  Particles of the warp with the same base cell reach the same
// eight cells: their weights are summed on the lowest such lane, which alone
// issues the atomics.  Clustered particles then cost shuffles instead of
// atomics on the same addresses.
__device__ __forceinline__ void cic_deposit_merged(float* __restrict__ rho, int Nm, const Cic& c, bool valid) {
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const float wx0 = 1.f - c.f[0], wx1 = c.f[0];
  const float wy0 = 1.f - c.f[1], wy1 = c.f[1];
  const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
  float w[8] = {wz0 * wy0 * wx0, wz0 * wy0 * wx1, wz0 * wy1 * wx0, wz0 * wy1 * wx1,
                wz1 * wy0 * wx0, wz1 * wy0 * wx1, wz1 * wy1 * wx0, wz1 * wy1 * wx1};
  const uint32_t key = ((uint32_t)c.i0[2] * (uint32_t)Nm + (uint32_t)c.i0[1]) * (uint32_t)Nm + (uint32_t)c.i0[0];
  const unsigned peers = __match_any_sync(act, key);
  const int lane = (int)(threadIdx.x & 31), leader = __ffs(peers) - 1;
  for (unsigned todo = __ballot_sync(act, lane != leader); todo; todo &= todo - 1) {  // warp-uniform
    const int j = __ffs(todo) - 1;
    const bool take = lane == leader && ((peers >> j) & 1u);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float v = __shfl_sync(act, w[q], j);
      if (take) w[q] += v;
    }
  }
  if (lane != leader) return;
  const int64_t z0 = (int64_t)c.i0[2] * Nm, z1 = (int64_t)c.i1[2] * Nm;
  row_add(rho + (z0 + c.i0[1]) * Nm, c.i0[0], c.i1[0], w[0], w[1]);
  row_add(rho + (z0 + c.i1[1]) * Nm, c.i0[0], c.i1[0], w[2], w[3]);
  row_add(rho + (z1 + c.i0[1]) * Nm, c.i0[0], c.i1[0], w[4], w[5]);
  row_add(rho + (z1 + c.i1[1]) * Nm, c.i0[0], c.i1[0], w[6], w[7]);
}

__device__ __forceinline__ float cic_interp(const float* __restrict__ F, int Nm, const Cic& c) {
  const float wx0 = 1.f - c.f[0], wx1 = c.f[0];
  const float wy0 = 1.f - c.f[1], wy1 = c.f[1];
  const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
  const int64_t z0 = (int64_t)c.i0[2] * Nm, z1 = (int64_t)c.i1[2] * Nm;
  const int64_t r00 = (z0 + c.i0[1]) * Nm, r01 = (z0 + c.i1[1]) * Nm;
  const int64_t r10 = (z1 + c.i0[1]) * Nm, r11 = (z1 + c.i1[1]) * Nm;
  const float a00 = wx0 * __ldg(F + r00 + c.i0[0]) + wx1 * __ldg(F + r00 + c.i1[0]);
  const float a01 = wx0 * __ldg(F + r01 + c.i0[0]) + wx1 * __ldg(F + r01 + c.i1[0]);
  const float a10 = wx0 * __ldg(F + r10 + c.i0[0]) + wx1 * __ldg(F + r10 + c.i1[0]);
  const float a11 = wx0 * __ldg(F + r11 + c.i0[0]) + wx1 * __ldg(F + r11 + c.i1[0]);
  return wz0 * (wy0 * a00 + wy1 * a01) + wz1 * (wy0 * a10 + wy1 * a11);
}

// (F_x, F_y) at the particle from the interleaved pair mesh Fxy (one float2 per
// cell): the same weights and operation order as cic_interp per component, one
// 8-byte load per corner instead of two 4-byte loads.
__device__ __forceinline__ float2 cic_interp2(const float2* __restrict__ F, int Nm, const Cic& c) {
  const float wx0 = 1.f - c.f[0], wx1 = c.f[0];
  const float wy0 = 1.f - c.f[1], wy1 = c.f[1];
  const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
  const int64_t z0 = (int64_t)c.i0[2] * Nm, z1 = (int64_t)c.i1[2] * Nm;
  const int64_t r00 = (z0 + c.i0[1]) * Nm, r01 = (z0 + c.i1[1]) * Nm;
  const int64_t r10 = (z1 + c.i0[1]) * Nm, r11 = (z1 + c.i1[1]) * Nm;
  auto row = [&](int64_t r) {
    const float2 a = __ldg(F + r + c.i0[0]), b = __ldg(F + r + c.i1[0]);
    return make_float2(wx0 * a.x + wx1 * b.x, wx0 * a.y + wx1 * b.y);
  };
  const float2 a00 = row(r00), a01 = row(r01), a10 = row(r10), a11 = row(r11);
  return make_float2(wz0 * (wy0 * a00.x + wy1 * a01.x) + wz1 * (wy0 * a10.x + wy1 * a11.x),
                     wz0 * (wy0 * a00.y + wy1 * a01.y) + wz1 * (wy0 * a10.y + wy1 * a11.y));
}

__global__ void __launch_bounds__(NTP) k_split_pairs(const float2* __restrict__ fxy, float* __restrict__ x,
                                                     float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * NTP + threadIdx.x; i < n; i += (int64_t)gridDim.x * NTP) {
    const float2 v = fxy[i];
    if (x) x[i] = v.x;
    if (y) y[i] = v.y;
  }
}

__device__ __forceinline__ void lattice(const PartParams& pp, int64_t p, int& ix, int& iy, int& iz) {
  const int m = pp.Np - 1;
  ix = (int)(p & m);
  iy = (int)((p >> pp.lgNp) & m);
  iz = (int)(p >> (2 * pp.lgNp));
}

// Multi-simulation kernels take the simulation from blockIdx.y and move every
// buffer pointer by its shift.
__global__ void __launch_bounds__(NTP) k_deposit(PartParams pp, const float* __restrict__ sx,
                                                 const float* __restrict__ sy,
                                                 const float* __restrict__ sz,
                                                 float* __restrict__ rho, int64_t P, Multi m) {
  const int64_t p = (int64_t)blockIdx.x * NTP + threadIdx.x;
  if (p >= P) return;
  const int64_t by = shift_of(m, blockIdx.y);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  rho = moved(rho, by);
  int ix, iy, iz;
  lattice(pp, p, ix, iy, iz);
  cic_deposit(rho, pp.Nm, cic_setup(pp, ix, iy, iz, sx[p], sy[p], sz[p]));
}

// Particle of work item i of the gather: a warp takes an 8 x 4 patch of the
// Lagrangian lattice (8 along x, 4 along y) instead of 32 along x.  Loads of
// per-particle arrays still fill whole 32-byte sectors, and once the particles
// have clustered a compact patch touches fewer mesh sectors than a line (the
// last step's gather 9.95 -> 6.9 ms at 512^3 / 1024^3).  The deposit keeps
// lines: its atomics from a patch collide more (4.0 -> 4.5 ms at the first step).
__device__ __forceinline__ int64_t patch84(const PartParams& pp, int64_t i) {
  const int lane = (int)(i & 31);
  const int64_t w = i >> 5;
  const int xw = pp.lgNp - 3;                      // warps along x per 4-row band
  const int64_t xh = w & ((1 << xw) - 1), band = w >> xw;  // band = z Np/4 + y/4
  const int64_t x = (xh << 3) | (lane & 7);
  const int64_t yz = (band << 2) | (lane >> 3);    // y + z Np (4 | Np)
  return (yz << pp.lgNp) | x;
}

// Sec. 2 drift in the LPT frame: delta_v += acc dtk (closing the previous
// half kick), s += delta_v dtd + dPsi_LPT(q); then CIC deposit of x = q + s.
__global__ void __launch_bounds__(NTP) k_drift_deposit(
    PartParams pp, float* __restrict__ sx, float* __restrict__ sy, float* __restrict__ sz,
    float* __restrict__ vx, float* __restrict__ vy, float* __restrict__ vz,
    const float* __restrict__ ax, const float* __restrict__ ay, const float* __restrict__ az,
    const float* __restrict__ dpx, const float* __restrict__ dpy,
    const float* __restrict__ dpz, float* __restrict__ rho, StepDt dt, int64_t P, Multi m,
    LptMix mix) {
  const int64_t p = (int64_t)blockIdx.x * NTP + threadIdx.x;
  const bool valid = p < P;
  const int64_t by = shift_of(m, blockIdx.y);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  vx = moved(vx, by);
  vy = moved(vy, by);
  vz = moved(vz, by);
  ax = moved(ax, by);
  ay = moved(ay, by);
  az = moved(az, by);
  dpx = moved(dpx, by);
  dpy = moved(dpy, by);
  dpz = moved(dpz, by);
  rho = moved(rho, by);
  float dtk = dt.dtk, dtd = dt.dtd;
  if (dt.hdr) {
    const SimHeader* h = moved(dt.hdr, by);
    dtk = h->ddt[3 * h->step];
    dtd = h->ddt[3 * h->step + 1];
  }
  Cic c{};
  if (valid) {
    float lx, ly, lz;
    if (dt.lq) {  // 16-bit drift fields, one scale per field
      const SimHeader* h = moved(dt.hdr, by);
      lx = lq_value(reinterpret_cast<const unsigned short*>(dpx)[p], dt.lq) * h->lq_used[0];
      ly = lq_value(reinterpret_cast<const unsigned short*>(dpy)[p], dt.lq) * h->lq_used[1];
      lz = lq_value(reinterpret_cast<const unsigned short*>(dpz)[p], dt.lq) * h->lq_used[2];
    } else {
      lx = dpx[p];
      ly = dpy[p];
      lz = dpz[p];
    }
    if (mix.on) {  // Delta Psi = c1 Psi1 + c2 Psi2
      const float4 cf = mix_coeffs(mix, by);
      lx = cf.x * lx + cf.y * moved(mix.q2[0], by)[p];
      ly = cf.x * ly + cf.y * moved(mix.q2[1], by)[p];
      lz = cf.x * lz + cf.y * moved(mix.q2[2], by)[p];
    }
    const float ux = vx[p] + ax[p] * dtk;
    const float uy = vy[p] + ay[p] * dtk;
    const float uz = vz[p] + az[p] * dtk;
    const float nx = sx[p] + ux * dtd + lx;
    const float ny = sy[p] + uy * dtd + ly;
    const float nz = sz[p] + uz * dtd + lz;
    vx[p] = ux;
    vy[p] = uy;
    vz[p] = uz;
    sx[p] = nx;
    sy[p] = ny;
    sz[p] = nz;
    int ix, iy, iz;
    lattice(pp, p, ix, iy, iz);
    c = cic_setup(pp, ix, iy, iz, nx, ny, nz);
  }
  cic_deposit_merged(rho, pp.Nm, c, valid);
}

// Sec. 2 kick: acc = g(x) - A_LPT(q), delta_v += acc dtk.  Each thread handles
// PPT particles (p, p + NTP, ...) of its block so that the dependent chains
// (displacement load -> cell index -> 24 mesh loads) of different particles overlap.
constexpr int PPT = 2;

template <bool XY>
__global__ void __launch_bounds__(NTP) k_gather_kick(
    PartParams pp, const float* __restrict__ sx, const float* __restrict__ sy,
    const float* __restrict__ sz, float* __restrict__ vx, float* __restrict__ vy,
    float* __restrict__ vz, float* __restrict__ ax, float* __restrict__ ay,
    float* __restrict__ az, const float* __restrict__ Ax, const float* __restrict__ Ay,
    const float* __restrict__ Az, const float* __restrict__ F0, const float* __restrict__ F1,
    const float* __restrict__ Fz, StepDt dt, int64_t P, Multi m, LptMix mix) {
  const int64_t p0 = (int64_t)blockIdx.x * NTP * PPT + threadIdx.x;
  const int64_t by = shift_of(m, blockIdx.y);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  vx = moved(vx, by);
  vy = moved(vy, by);
  vz = moved(vz, by);
  ax = moved(ax, by);
  ay = moved(ay, by);
  az = moved(az, by);
  Ax = moved(Ax, by);
  Ay = moved(Ay, by);
  Az = moved(Az, by);
  F0 = moved(F0, by);
  F1 = moved(F1, by);
  Fz = moved(Fz, by);
  float dtk = dt.dtk;
  if (dt.hdr) {
    const SimHeader* h = moved(dt.hdr, by);
    dtk = h->ddt[3 * h->step + 2];
  }
  float px[PPT], py[PPT], pz[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int64_t p = patch84(pp, p0 + u * NTP);
    if (p0 + u * NTP < P) {
      px[u] = sx[p];
      py[u] = sy[p];
      pz[u] = sz[p];
    }
  }
  float gx[PPT], gy[PPT], gz[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int64_t p = patch84(pp, p0 + u * NTP);
    if (p0 + u * NTP < P) {
      int ix, iy, iz;
      lattice(pp, p, ix, iy, iz);
      const Cic c = cic_setup(pp, ix, iy, iz, px[u], py[u], pz[u]);
      if constexpr (XY) {  // (F_x, F_y) pairs in F0
        const float2 gxy = cic_interp2(reinterpret_cast<const float2*>(F0), pp.Nm, c);
        gx[u] = gxy.x;
        gy[u] = gxy.y;
      } else {
        gx[u] = cic_interp(F0, pp.Nm, c);
        gy[u] = cic_interp(F1, pp.Nm, c);
      }
      gz[u] = cic_interp(Fz, pp.Nm, c);
    }
  }
  float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
  if (mix.on) cf = mix_coeffs(mix, by);
  float qs[3] = {1.f, 1.f, 1.f};
  if (dt.lq) {
    const SimHeader* h = moved(dt.hdr, by);
    for (int d = 0; d < 3; ++d) qs[d] = h->lq_used[3 + d];
  }
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int64_t p = patch84(pp, p0 + u * NTP);
    if (p0 + u * NTP < P) {
      float lx, ly, lz;
      if (dt.lq) {  // 16-bit kick fields, one scale per field
        lx = lq_value(reinterpret_cast<const unsigned short*>(Ax)[p], dt.lq) * qs[0];
        ly = lq_value(reinterpret_cast<const unsigned short*>(Ay)[p], dt.lq) * qs[1];
        lz = lq_value(reinterpret_cast<const unsigned short*>(Az)[p], dt.lq) * qs[2];
      } else {
        lx = Ax[p];
        ly = Ay[p];
        lz = Az[p];
      }
      if (mix.on) {  // A_LPT = e1 Psi1 + e2 Psi2
        lx = cf.z * lx + cf.w * moved(mix.q2[0], by)[p];
        ly = cf.z * ly + cf.w * moved(mix.q2[1], by)[p];
        lz = cf.z * lz + cf.w * moved(mix.q2[2], by)[p];
      }
      const float ex = gx[u] - lx, ey = gy[u] - ly, ez = gz[u] - lz;
      ax[p] = ex;
      ay[p] = ey;
      az[p] = ez;
      vx[p] += ex * dtk;
      vy[p] += ey * dtk;
      vz[p] += ez * dtk;
    }
  }
}

// The end of step n and the start of step n + 1 in one pass over the particles
// (Sec. 2), for consecutive steps of one simulation: the kick of step n,
// acc = g(x) - A_n(q) and delta_v += acc dtk2_n, then the closing half kick of
// step n + 1, delta_v += acc dtk1_{n+1}, the drift s += delta_v dtd_{n+1} +
// dPsi_{n+1}(q) and the CIC deposit of the new x.  The arithmetic and its order
// are those of k_gather_kick followed by k_drift_deposit, so the particle state
// is the same bit for bit; acc is not stored (the next gather forms it again)
// and delta_v and s are read and written once instead of twice.  hdr->step = n.
// Particles as in the gather (8 x 4 lattice patches per warp, PPT per thread).
template <int Q, int MINB, bool XY>
__global__ void __launch_bounds__(NTP, MINB) k_kick_drift_deposit(
    PartParams pp, float* __restrict__ sx, float* __restrict__ sy, float* __restrict__ sz,
    float* __restrict__ vx, float* __restrict__ vy, float* __restrict__ vz,
    const float* __restrict__ Ax, const float* __restrict__ Ay, const float* __restrict__ Az,
    const float* __restrict__ dpx, const float* __restrict__ dpy, const float* __restrict__ dpz,
    const float* __restrict__ F0, const float* __restrict__ F1, const float* __restrict__ Fz,
    float* __restrict__ rho, const SimHeader* __restrict__ hdr, int64_t P, Multi m) {
  const int64_t p0 = (int64_t)blockIdx.x * NTP * Q + threadIdx.x;
  const int64_t by = shift_of(m, blockIdx.y);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  vx = moved(vx, by);
  vy = moved(vy, by);
  vz = moved(vz, by);
  Ax = moved(Ax, by);
  Ay = moved(Ay, by);
  Az = moved(Az, by);
  dpx = moved(dpx, by);
  dpy = moved(dpy, by);
  dpz = moved(dpz, by);
  F0 = moved(F0, by);
  F1 = moved(F1, by);
  Fz = moved(Fz, by);
  rho = moved(rho, by);
  const SimHeader* h = moved(hdr, by);
  const int n = h->step;
  const float dtk2 = h->ddt[3 * n + 2], dtk1 = h->ddt[3 * (n + 1)], dtd = h->ddt[3 * (n + 1) + 1];
  float px[Q], py[Q], pz[Q];
#pragma unroll
  for (int u = 0; u < Q; ++u) {
    const int64_t p = patch84(pp, p0 + u * NTP);
    if (p0 + u * NTP < P) {
      px[u] = sx[p];
      py[u] = sy[p];
      pz[u] = sz[p];
    }
  }
  float gx[Q], gy[Q], gz[Q];
#pragma unroll
  for (int u = 0; u < Q; ++u) {
    const int64_t p = patch84(pp, p0 + u * NTP);
    if (p0 + u * NTP < P) {
      int ix, iy, iz;
      lattice(pp, p, ix, iy, iz);
      const Cic c = cic_setup(pp, ix, iy, iz, px[u], py[u], pz[u]);
      if constexpr (XY) {  // (F_x, F_y) pairs in F0
        const float2 gxy = cic_interp2(reinterpret_cast<const float2*>(F0), pp.Nm, c);
        gx[u] = gxy.x;
        gy[u] = gxy.y;
      } else {
        gx[u] = cic_interp(F0, pp.Nm, c);
        gy[u] = cic_interp(F1, pp.Nm, c);
      }
      gz[u] = cic_interp(Fz, pp.Nm, c);
    }
  }
#pragma unroll
  for (int u = 0; u < Q; ++u) {
    const int64_t p = patch84(pp, p0 + u * NTP);
    const bool valid = p0 + u * NTP < P;
    Cic c{};
    if (valid) {
      const float ex = gx[u] - Ax[p], ey = gy[u] - Ay[p], ez = gz[u] - Az[p];
      float ux = vx[p], uy = vy[p], uz = vz[p];
      ux += ex * dtk2;  // the kick of step n
      uy += ey * dtk2;
      uz += ez * dtk2;
      ux = ux + ex * dtk1;  // the closing half kick of step n + 1
      uy = uy + ey * dtk1;
      uz = uz + ez * dtk1;
      const float nx = px[u] + ux * dtd + dpx[p];
      const float ny = py[u] + uy * dtd + dpy[p];
      const float nz = pz[u] + uz * dtd + dpz[p];
      vx[p] = ux;
      vy[p] = uy;
      vz[p] = uz;
      sx[p] = nx;
      sy[p] = ny;
      sz[p] = nz;
      int ix, iy, iz;
      lattice(pp, p, ix, iy, iz);
      c = cic_setup(pp, ix, iy, iz, nx, ny, nz);
    }
    cic_deposit_merged(rho, pp.Nm, c, valid);
  }
}

// ---------------------------------------------------------------- shared-memory boxes
// Alternative drift + deposit and gather + kick kernels, chosen per batch by
// the batch autotuner (cola_batch_plan deposit_box / gather_box).  Each CTA
// takes an 8 x 8 x 8 block of the Lagrangian lattice (two particles per
// thread); particles that start together stay close for much of a run, so the
// block's CIC stencils cover a compact box of mesh cells, found by a block
// reduction (rows aligned to 16 bytes).  Deposit: the weights are summed into
// the box in shared memory and leave with one 16-byte vector atomic per four
// cells (zero groups skipped).  Gather: the three force components of the box
// are copied into shared memory with 16-byte cp.async pieces and every
// particle interpolates there.  A block whose box exceeds the capacity falls
// back to the direct global atomics or loads.  Results equal the direct
// kernels' (the same weights and values; only the order of float additions in
// the deposit differs).  On the 512^3 / 1024^3 step both measured slower than
// the direct kernels (deposit 5.4 -> 9.0 ms against 4.0 -> 5.8 ms over 30
// steps; gather 8.0 -> 10.7 ms against 4.1 -> 7.1 ms), so the single-run path
// keeps the direct ones.
constexpr int LB = 8;                    // lattice block side
constexpr int LBP = LB * LB * LB;        // particles per CTA (2 per thread)
constexpr int kMaxDepositBox = 16384;    // cells (64 KB)
constexpr int kMaxGatherBox = 8192;      // cells x 3 components (96 KB)
static_assert(LBP == 2 * NTP, "two particles per thread");

// CIC base cell without the periodic wrap (so that a block's cells form one
// box) and the fractions; the arithmetic of cic_setup.
struct CicU {
  int i0[3];
  float f[3];
};

__device__ __forceinline__ CicU cic_unwrapped(const PartParams& pp, int ix, int iy, int iz, float sx, float sy,
                                             float sz) {
  CicU c;
  const int li[3] = {ix, iy, iz};
  const float sv[3] = {sx, sy, sz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int num = li[d] * pp.Nm;
    const int base = num >> pp.lgNp;
    const float qf = (float)(num - (base << pp.lgNp)) * __int_as_float((127 - pp.lgNp) << 23);
    const float u = qf + sv[d] * pp.cellscale;
    const float fl = floorf(u);
    c.f[d] = u - fl;
    c.i0[d] = base + (int)fl;
  }
  return c;
}

__device__ __forceinline__ Cic wrap(const CicU& u, int Nm) {
  Cic c;
  const int mask = Nm - 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c.i0[d] = u.i0[d] & mask;
    c.i1[d] = (c.i0[d] + 1) & mask;
    c.f[d] = u.f[d];
  }
  return c;
}

// Lattice point of particle k (0, 1) of this thread in the CTA's block, and its index.
struct BlockLattice {
  int ox, oy, oz;
  __device__ __forceinline__ explicit BlockLattice(const PartParams& pp) {
    const int lg = pp.lgNp - 3, m = (1 << lg) - 1;
    const uint32_t b = blockIdx.x;
    ox = (int)(b & m) << 3;
    oy = (int)((b >> lg) & m) << 3;
    oz = (int)(b >> (2 * lg)) << 3;
  }
  __device__ __forceinline__ int64_t at(const PartParams& pp, int k, int& ix, int& iy, int& iz) const {
    const int l = threadIdx.x + k * NTP;
    ix = ox + (l & 7);
    iy = oy + ((l >> 3) & 7);
    iz = oz + (l >> 6);
    return ((((int64_t)iz << pp.lgNp) + iy) << pp.lgNp) + ix;
  }
};

// The block's box: lo = smallest base cell per axis, ex = cells per axis (the
// largest base cell + 2 - lo).  Every thread gets the result.
struct Box {
  int lo[3], ex[3];
};

__device__ __forceinline__ Box block_box(const CicU (&c)[2], int (*red)[6]) {
  int v[6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    v[d] = min(c[0].i0[d], c[1].i0[d]);
    v[3 + d] = -max(c[0].i0[d], c[1].i0[d]);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 6; ++q) v[q] = __reduce_min_sync(0xffffffffu, v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) red[w][q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    int r = red[0][q];
#pragma unroll
    for (int j = 1; j < NTP / 32; ++j) r = min(r, red[j][q]);
    v[q] = r;
  }
  Box b;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = v[d];
    b.ex[d] = -v[3 + d] + 2 - v[d];
  }
  return b;
}

// Rows (y, z) of a box with `len` entries along x, walked by the CTA: each warp
// takes 32 / len rows at a time when a row fits in a warp, else one row whose
// entries its lanes stride through.  f(e, r, yy, zz) for entry e of row r.
template <class F>
__device__ __forceinline__ void for_box_rows(int len, int ey, int ez, F f) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrow = ey * ez;
  if (len <= 32) {
    const int rpw = 32 / len, sub = lane / len, e = lane - sub * len;
    if (sub >= rpw) return;
    for (int r = w * rpw + sub; r < nrow; r += (NTP / 32) * rpw) {
      const int zz = r / ey, yy = r - zz * ey;
      f(e, r, yy, zz);
    }
  } else {
    for (int r = w; r < nrow; r += NTP / 32) {
      const int zz = r / ey, yy = r - zz * ey;
      for (int e = lane; e < len; e += 32) f(e, r, yy, zz);
    }
  }
}

// CIC interpolation from a shared box (strides 1, sy, sz; q = the base cell), in
// the operation order of cic_interp.
__device__ __forceinline__ float box_interp(const float* __restrict__ q, int sy, int sz, const CicU& c) {
  const float wx0 = 1.f - c.f[0], wx1 = c.f[0];
  const float wy0 = 1.f - c.f[1], wy1 = c.f[1];
  const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
  const float a00 = wx0 * q[0] + wx1 * q[1];
  const float a01 = wx0 * q[sy] + wx1 * q[sy + 1];
  const float a10 = wx0 * q[sz] + wx1 * q[sz + 1];
  const float a11 = wx0 * q[sz + sy] + wx1 * q[sz + sy + 1];
  return wz0 * (wy0 * a00 + wy1 * a01) + wz1 * (wy0 * a10 + wy1 * a11);
}

// The same for the (x, y) pairs of the interleaved box (one float2 per cell).
__device__ __forceinline__ float2 box_interp2(const float2* __restrict__ q, int sy, int sz, const CicU& c) {
  const float wx0 = 1.f - c.f[0], wx1 = c.f[0];
  const float wy0 = 1.f - c.f[1], wy1 = c.f[1];
  const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
  auto row = [&](int o) {
    const float2 a = q[o], b = q[o + 1];
    return make_float2(wx0 * a.x + wx1 * b.x, wx0 * a.y + wx1 * b.y);
  };
  const float2 a00 = row(0), a01 = row(sy), a10 = row(sz), a11 = row(sz + sy);
  return make_float2(wz0 * (wy0 * a00.x + wy1 * a01.x) + wz1 * (wy0 * a10.x + wy1 * a11.x),
                     wz0 * (wy0 * a00.y + wy1 * a01.y) + wz1 * (wy0 * a10.y + wy1 * a11.y));
}

__device__ __forceinline__ void cp_async16_pm(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Box of the CTA's particles with 16-byte aligned rows: x from x0 (a multiple
// of 4), ex cells per row (a multiple of 4).
__device__ __forceinline__ void aligned_rows(const Box& b, int& x0, int& ex) {
  x0 = b.lo[0] & ~3;
  ex = ((b.lo[0] + b.ex[0] - x0) + 3) & ~3;
}

// Drift (as k_drift_deposit) and the CIC deposit binned in a shared box of at
// most `cap` cells.
__global__ void __launch_bounds__(NTP, 3) k_drift_deposit_box(
    PartParams pp, float* __restrict__ sx, float* __restrict__ sy, float* __restrict__ sz,
    float* __restrict__ vx, float* __restrict__ vy, float* __restrict__ vz,
    const float* __restrict__ ax, const float* __restrict__ ay, const float* __restrict__ az,
    const float* __restrict__ dpx, const float* __restrict__ dpy,
    const float* __restrict__ dpz, float* __restrict__ rho, StepDt dt, Multi m, LptMix mix, int cap) {
  extern __shared__ __align__(16) float sbox[];
  __shared__ int red[NTP / 32][6];
  const int64_t by = shift_of(m, blockIdx.y);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  vx = moved(vx, by);
  vy = moved(vy, by);
  vz = moved(vz, by);
  ax = moved(ax, by);
  ay = moved(ay, by);
  az = moved(az, by);
  dpx = moved(dpx, by);
  dpy = moved(dpy, by);
  dpz = moved(dpz, by);
  rho = moved(rho, by);
  float dtk = dt.dtk, dtd = dt.dtd;
  float qs[3] = {1.f, 1.f, 1.f};
  if (dt.hdr) {
    const SimHeader* h = moved(dt.hdr, by);
    dtk = h->ddt[3 * h->step];
    dtd = h->ddt[3 * h->step + 1];
    if (dt.lq)
      for (int d = 0; d < 3; ++d) qs[d] = h->lq_used[d];
  }
  float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
  if (mix.on) cf = mix_coeffs(mix, by);
  const BlockLattice bl(pp);
  CicU c[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    int ix, iy, iz;
    const int64_t p = bl.at(pp, k, ix, iy, iz);
    float lx, ly, lz;
    if (dt.lq) {  // 16-bit drift fields, one scale per field
      lx = lq_value(reinterpret_cast<const unsigned short*>(dpx)[p], dt.lq) * qs[0];
      ly = lq_value(reinterpret_cast<const unsigned short*>(dpy)[p], dt.lq) * qs[1];
      lz = lq_value(reinterpret_cast<const unsigned short*>(dpz)[p], dt.lq) * qs[2];
    } else {
      lx = dpx[p];
      ly = dpy[p];
      lz = dpz[p];
    }
    if (mix.on) {  // Delta Psi = c1 Psi1 + c2 Psi2
      lx = cf.x * lx + cf.y * moved(mix.q2[0], by)[p];
      ly = cf.x * ly + cf.y * moved(mix.q2[1], by)[p];
      lz = cf.x * lz + cf.y * moved(mix.q2[2], by)[p];
    }
    const float ux = vx[p] + ax[p] * dtk;
    const float uy = vy[p] + ay[p] * dtk;
    const float uz = vz[p] + az[p] * dtk;
    const float nx = sx[p] + ux * dtd + lx;
    const float ny = sy[p] + uy * dtd + ly;
    const float nz = sz[p] + uz * dtd + lz;
    vx[p] = ux;
    vy[p] = uy;
    vz[p] = uz;
    sx[p] = nx;
    sy[p] = ny;
    sz[p] = nz;
    c[k] = cic_unwrapped(pp, ix, iy, iz, nx, ny, nz);
  }
  const Box b = block_box(c, red);
  int x0, ex;
  aligned_rows(b, x0, ex);
  const int64_t ncell = (int64_t)ex * b.ex[1] * b.ex[2];
  const int Nm = pp.Nm;
  if (ncell > cap) {
#pragma unroll
    for (int k = 0; k < 2; ++k) cic_deposit_merged(rho, Nm, wrap(c[k], Nm), true);
    return;
  }
  float4* s4 = reinterpret_cast<float4*>(sbox);
  const int n4 = (int)ncell >> 2;
  for (int i = threadIdx.x; i < n4; i += NTP) s4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const int syb = ex, szb = ex * b.ex[1];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float wx0 = 1.f - c[k].f[0], wx1 = c[k].f[0];
    const float wy0 = 1.f - c[k].f[1], wy1 = c[k].f[1];
    const float wz0 = 1.f - c[k].f[2], wz1 = c[k].f[2];
    float* q = sbox + (c[k].i0[2] - b.lo[2]) * szb + (c[k].i0[1] - b.lo[1]) * syb + (c[k].i0[0] - x0);
    atomicAdd(q, wz0 * wy0 * wx0);
    atomicAdd(q + 1, wz0 * wy0 * wx1);
    atomicAdd(q + syb, wz0 * wy1 * wx0);
    atomicAdd(q + syb + 1, wz0 * wy1 * wx1);
    atomicAdd(q + szb, wz1 * wy0 * wx0);
    atomicAdd(q + szb + 1, wz1 * wy0 * wx1);
    atomicAdd(q + szb + syb, wz1 * wy1 * wx0);
    atomicAdd(q + szb + syb + 1, wz1 * wy1 * wx1);
  }
  __syncthreads();
  const int mask = Nm - 1;
  for_box_rows(ex >> 2, b.ex[1], b.ex[2], [&](int g, int r, int yy, int zz) {
    const float4 v = s4[r * (ex >> 2) + g];
    if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
      const int64_t row = ((int64_t)((b.lo[2] + zz) & mask) * Nm + ((b.lo[1] + yy) & mask)) * Nm;
      red_add4(rho + row + ((x0 + 4 * g) & mask), v);
    }
  });
}

// Gather (three force components staged in a shared box of at most `cap`
// cells) and kick, as k_gather_kick.
template <bool XY>
__global__ void __launch_bounds__(NTP, 2) k_gather_kick_box(
    PartParams pp, const float* __restrict__ sx, const float* __restrict__ sy,
    const float* __restrict__ sz, float* __restrict__ vx, float* __restrict__ vy,
    float* __restrict__ vz, float* __restrict__ ax, float* __restrict__ ay,
    float* __restrict__ az, const float* __restrict__ Ax, const float* __restrict__ Ay,
    const float* __restrict__ Az, const float* __restrict__ F0, const float* __restrict__ F1,
    const float* __restrict__ Fz, StepDt dt, Multi m, LptMix mix, int cap) {
  extern __shared__ __align__(16) float sbox[];
  __shared__ int red[NTP / 32][6];
  const int64_t by = shift_of(m, blockIdx.y);
  sx = moved(sx, by);
  sy = moved(sy, by);
  sz = moved(sz, by);
  vx = moved(vx, by);
  vy = moved(vy, by);
  vz = moved(vz, by);
  ax = moved(ax, by);
  ay = moved(ay, by);
  az = moved(az, by);
  Ax = moved(Ax, by);
  Ay = moved(Ay, by);
  Az = moved(Az, by);
  F0 = moved(F0, by);
  F1 = moved(F1, by);
  Fz = moved(Fz, by);
  float dtk = dt.dtk;
  float qs[3] = {1.f, 1.f, 1.f};
  if (dt.hdr) {
    const SimHeader* h = moved(dt.hdr, by);
    dtk = h->ddt[3 * h->step + 2];
    if (dt.lq)
      for (int d = 0; d < 3; ++d) qs[d] = h->lq_used[3 + d];
  }
  const BlockLattice bl(pp);
  int64_t p[2];
  CicU c[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    int ix, iy, iz;
    p[k] = bl.at(pp, k, ix, iy, iz);
    c[k] = cic_unwrapped(pp, ix, iy, iz, sx[p[k]], sy[p[k]], sz[p[k]]);
  }
  const Box b = block_box(c, red);
  int x0, ex;
  aligned_rows(b, x0, ex);
  const int64_t ncell = (int64_t)ex * b.ex[1] * b.ex[2];
  float g[2][3];
  if (ncell <= cap) {
    const int Nm = pp.Nm, mask = Nm - 1;
    for_box_rows(ex >> 2, b.ex[1], b.ex[2], [&](int e, int r, int yy, int zz) {
      const int64_t gi = ((int64_t)((b.lo[2] + zz) & mask) * Nm + ((b.lo[1] + yy) & mask)) * Nm +
                         ((x0 + 4 * e) & mask);
      const int cell = r * ex + 4 * e;
      if constexpr (XY) {  // (x, y) pairs: 2 cap floats, then z
        float2* sxy = reinterpret_cast<float2*>(sbox);
        const float2* F2 = reinterpret_cast<const float2*>(F0);
        cp_async16_pm(sxy + cell, F2 + gi);
        cp_async16_pm(sxy + cell + 2, F2 + gi + 2);
      } else {
        cp_async16_pm(sbox + cell, F0 + gi);
        cp_async16_pm(sbox + cap + cell, F1 + gi);
      }
      cp_async16_pm(sbox + 2 * cap + cell, Fz + gi);
    });
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    const int syb = ex, szb = ex * b.ex[1];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int o = (c[k].i0[2] - b.lo[2]) * szb + (c[k].i0[1] - b.lo[1]) * syb + (c[k].i0[0] - x0);
      if constexpr (XY) {
        const float2 gxy = box_interp2(reinterpret_cast<const float2*>(sbox) + o, syb, szb, c[k]);
        g[k][0] = gxy.x;
        g[k][1] = gxy.y;
      } else {
        g[k][0] = box_interp(sbox + o, syb, szb, c[k]);
        g[k][1] = box_interp(sbox + cap + o, syb, szb, c[k]);
      }
      g[k][2] = box_interp(sbox + 2 * cap + o, syb, szb, c[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const Cic cw = wrap(c[k], pp.Nm);
      if constexpr (XY) {
        const float2 gxy = cic_interp2(reinterpret_cast<const float2*>(F0), pp.Nm, cw);
        g[k][0] = gxy.x;
        g[k][1] = gxy.y;
      } else {
        g[k][0] = cic_interp(F0, pp.Nm, cw);
        g[k][1] = cic_interp(F1, pp.Nm, cw);
      }
      g[k][2] = cic_interp(Fz, pp.Nm, cw);
    }
  }
  float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
  if (mix.on) cf = mix_coeffs(mix, by);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int64_t q = p[k];
    float lx, ly, lz;
    if (dt.lq) {  // 16-bit kick fields, one scale per field
      lx = lq_value(reinterpret_cast<const unsigned short*>(Ax)[q], dt.lq) * qs[0];
      ly = lq_value(reinterpret_cast<const unsigned short*>(Ay)[q], dt.lq) * qs[1];
      lz = lq_value(reinterpret_cast<const unsigned short*>(Az)[q], dt.lq) * qs[2];
    } else {
      lx = Ax[q];
      ly = Ay[q];
      lz = Az[q];
    }
    if (mix.on) {  // A_LPT = e1 Psi1 + e2 Psi2
      lx = cf.z * lx + cf.w * moved(mix.q2[0], by)[q];
      ly = cf.z * ly + cf.w * moved(mix.q2[1], by)[q];
      lz = cf.z * lz + cf.w * moved(mix.q2[2], by)[q];
    }
    const float ex_ = g[k][0] - lx, ey = g[k][1] - ly, ez = g[k][2] - lz;
    ax[q] = ex_;
    ay[q] = ey;
    az[q] = ez;
    vx[q] += ex_ * dtk;
    vy[q] += ey * dtk;
    vz[q] += ez * dtk;
  }
}

// The [P][3] outputs leave through shared memory as whole 16-byte pieces (a CTA's
// 256 particles are 3 KB of each array): the outputs may be page-locked host
// memory written across the chip-to-host link, where partial lines cost most.
__global__ void __launch_bounds__(NTP) k_snapshot(
    PartParams pp, const float* __restrict__ sx, const float* __restrict__ sy,
    const float* __restrict__ sz, const float* __restrict__ vx, const float* __restrict__ vy,
    const float* __restrict__ vz, const float* __restrict__ lx, const float* __restrict__ ly,
    const float* __restrict__ lz, float vscale, float* __restrict__ pos,
    float* __restrict__ vel, int64_t P, LptMix mix, double dq, double invL) {
  __shared__ __align__(16) float st[2][3 * NTP];
  const int64_t base = (int64_t)blockIdx.x * NTP, p = base + threadIdx.x;
  if (p < P) {
    int li[3];
    lattice(pp, p, li[0], li[1], li[2]);
    const float sv[3] = {sx[p], sy[p], sz[p]};
    if (pos) {
      // x = q + s wrapped into [0, L) in double precision; dq = L / Np and 1/L come from
      // the host (no double division per particle: this GPU's double rate is low)
      const double L = pp.L;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double x = (double)li[d] * dq + (double)sv[d];
        x -= L * floor(x * invL);
        if (x < 0.0) x += L;
        if (x >= L) x -= L;
        st[0][3 * threadIdx.x + d] = (float)x;
      }
    }
    if (vel) {
      float l[3] = {lx[p], ly[p], lz[p]};
      if (mix.on) {  // dPsi/dtau = dD1 Psi1 + dD2 Psi2
        const float4 cf = mix_coeffs(mix, 0);
#pragma unroll
        for (int d = 0; d < 3; ++d) l[d] = cf.x * l[d] + cf.y * mix.q2[d][p];
      }
      st[1][3 * threadIdx.x + 0] = (vx[p] + l[0]) * vscale;
      st[1][3 * threadIdx.x + 1] = (vy[p] + l[1]) * vscale;
      st[1][3 * threadIdx.x + 2] = (vz[p] + l[2]) * vscale;
    }
  }
  __syncthreads();
  const int n = (int)(3 * (P - base < NTP ? P - base : NTP));  // floats of this CTA per output
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float* o = k ? vel : pos;
    if (!o) continue;
    o += 3 * base;
    if (n == 3 * NTP && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
      for (int i = threadIdx.x; i < 3 * NTP / 4; i += NTP)
        reinterpret_cast<float4*>(o)[i] = reinterpret_cast<const float4*>(st[k])[i];
    } else {
      for (int i = threadIdx.x; i < n; i += NTP) o[i] = st[k][i];
    }
  }
}

__global__ void __launch_bounds__(NTP) k_pos_deposit(int Nm, float cellscale,
                                                     const float* __restrict__ pos, int64_t n,
                                                     float* __restrict__ rho) {
  const int64_t p = (int64_t)blockIdx.x * NTP + threadIdx.x;
  if (p >= n) return;
  Cic c;
  const int mask = Nm - 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float u = pos[p * 3 + d] * cellscale;
    const float fl = floorf(u);
    c.f[d] = u - fl;
    const int64_t ii = (int64_t)fl;
    c.i0[d] = (int)(ii & mask);
    c.i1[d] = (c.i0[d] + 1) & mask;
  }
  cic_deposit(rho, Nm, c);
}

// P(k) estimator: per mode of the half spectrum, bin b = floor(|n| - 1/2),
// weight 1 on the kx = 0, N/2 planes and 2 elsewhere, |delta|^2 norm / W_CIC^2 with
// W_CIC = prod sinc^2(pi n_i/N) (the window in single precision, a relative error
// ~1e-7 of P).  acc holds [count | sum P | sum |k| in units of k_F] per bin, in
// double precision.
//
// One warp per (z, y) row; lane l takes the run kx = l K .. l K + K - 1
// (K = ceil((N/2 + 1) / 32)).  Along a run |n|^2 = kx^2 + ny^2 + nz^2 only grows,
// so the bins are non-decreasing: a lane sums its modes in registers and adds to
// the block's shared-memory bins once per bin it meets (and stops at the first
// mode beyond the last bin).  The bin is decided exactly by integer comparisons,
// 4 |n|^2 against (2b + 1)^2 and (2b + 3)^2.  |n| = s + r / (2 s) with s = sqrtf(|n|^2)
// and r = |n|^2 - s^2 from one FMA (exact).  Double precision stays out of the
// per-mode work (this GPU's double rate is low, and a double atomic on shared
// memory is a compare-and-swap loop): within a run the weights are an integer,
// s an exact 64-bit integer count of 2^-23 (s >= 1 is a multiple of it), the
// corrections r / (2 s) (below 2^-15 each) and the powers single precision; the
// block's bins take them as 64-bit integer and float atomics once per bin met
// (the power as a float pair: the sum and the exact rounding error of each
// addition, recovered from the value the atomic returns), and the launch's bins
// in double at the end: |k| with a relative error ~1e-15.
__global__ void __launch_bounds__(NTP) k_pk_bin(const float2* __restrict__ dk, int N,
                                                int64_t P, int nbins,
                                                double* __restrict__ acc, double norm, Multi m,
                                                int64_t acc_stride) {
  // block bins: power (double), count and sum of s 2^23 (64-bit integers), sum of
  // the corrections (float); then the CIC window per kx
  extern __shared__ __align__(16) unsigned char pk_sh[];
  unsigned long long* bw = reinterpret_cast<unsigned long long*>(pk_sh);
  unsigned long long* bs = bw + nbins;
  float* bp = reinterpret_cast<float*>(bs + nbins);  // power: value and rounding error
  float* bq = bp + nbins;
  float* bc = bq + nbins;
  float* wx = bc + nbins;
  const int64_t by = shift_of(m, blockIdx.y);
  dk = moved(dk, by);
  acc = acc_stride > 0 ? acc + blockIdx.y * acc_stride : moved(acc, by);
  const int H = N / 2 + 1, K = (H + 31) / 32;
  const float pi = 3.14159265358979f;
  auto win = [&](int n) {
    if (n == 0) return 1.f;
    const float t = (float)n / (float)N;
    const float sc = sinpif(t) / (pi * t);
    return sc * sc;
  };
  for (int i = threadIdx.x; i < nbins; i += NTP) {
    bw[i] = bs[i] = 0ull;
    bp[i] = bq[i] = bc[i] = 0.f;
  }
  for (int i = threadIdx.x; i < H; i += NTP) wx[i] = win(i);
  __syncthreads();
  const int lane = threadIdx.x & 31, wpb = NTP / 32;
  for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < N * N; row += gridDim.x * wpb) {
    const int iz = row / N, iy = row - iz * N;
    const int ny = iy < N / 2 ? iy : iy - N, nz = iz < N / 2 ? iz : iz - N;
    const int c = ny * ny + nz * nz;
    const float wyz = win(ny) * win(nz);
    int cur = -1;
    int sw = 0;
    float sp = 0.f, snc = 0.f;
    long long sni = 0;
    auto flush = [&]() {
      if (cur >= 0) {
        // power: the float bin and, from the value the atomic replaced, the exact
        // rounding error of that addition into a second float (two-sum)
        const float old = atomicAdd(&bp[cur], sp), sum = old + sp;
        const float bv = sum - old;
        atomicAdd(&bq[cur], (old - (sum - bv)) + (sp - bv));
        atomicAdd(&bw[cur], (unsigned long long)sw);
        atomicAdd(&bs[cur], (unsigned long long)sni);
        atomicAdd(&bc[cur], snc);
      }
    };
    const int x0 = lane * K, x1 = min(x0 + K, H);
    for (int ix = x0; ix < x1; ++ix) {
      const int q = ix * ix + c;  // |n|^2 < 2^24 for N <= 4096
      if (q == 0) continue;       // the k = 0 mode is in no bin
      int b = (int)(sqrtf((float)q) - 0.5f);
      while (b > 0 && (2 * b + 1) * (2 * b + 1) > 4 * q) --b;
      while ((2 * b + 3) * (2 * b + 3) <= 4 * q) ++b;
      if (b >= nbins) break;  // every later mode of the run is beyond the last bin too
      if (b != cur) {
        flush();
        cur = b;
        sw = 0;
        sp = snc = 0.f;
        sni = 0;
      }
      const float qf = (float)q;
      const float s = sqrtf(qf);
      const float r = fmaf(-s, s, qf);
      const int wi = (ix == 0 || ix == N / 2) ? 1 : 2;
      const float wt = (float)wi;
      const float2 v = dk[hidx(iz, iy, ix, N, P)];
      const float wf = wx[ix] * wyz;
      sw += wi;
      sp += wt * (v.x * v.x + v.y * v.y) / (wf * wf);
      sni += (long long)wi * __float2ll_rn(s * 8388608.f);  // s 2^23, an integer
      snc += wt * __fdividef(r, 2.f * s);
    }
    flush();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += NTP)
    if (bw[i] != 0ull) {
      atomicAdd(&acc[i], (double)bw[i]);
      atomicAdd(&acc[nbins + i], ((double)bp[i] + (double)bq[i]) * norm);
      atomicAdd(&acc[2 * nbins + i], (double)bs[i] * 0x1p-23 + (double)bc[i]);
    }
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + NTP - 1) / NTP); }

__global__ void k_step_advance(SimHeader* hdr, Multi m) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < m.nb) moved(hdr, shift_of(m, b))->step += 1;
}

// Writes the header; the seed scales are written only on the device (by the
// initial conditions) and keep their values.
__global__ void k_set_header(SimHeader* hdr, SimHeader v) {
  v.seed_scale[0] = hdr->seed_scale[0];
  v.seed_scale[1] = hdr->seed_scale[1];
  for (int f = 0; f < 6; ++f) {
    v.lq_scale[f] = hdr->lq_scale[f];
    v.lq_used[f] = hdr->lq_used[f];
    v.lq_amax[f] = hdr->lq_amax[f];
  }
  *hdr = v;
}

__device__ __forceinline__ float lq_target(int prec) { return prec == 2 ? 1024.f : 1.f; }

// Growth of field f's coefficient from table row r0 to r1 (1 when unknown).
__device__ __forceinline__ float lq_growth(const SimHeader* h, int f, int r0, int r1) {
  if (!h->lqg) return 1.f;
  const float2 g0 = h->lqg[r0], g1 = h->lqg[r1];
  const float a = f < 3 ? g0.x : g0.y, b = f < 3 ? g1.x : g1.y;
  return a > 0.f && b > 0.f ? b / a : 1.f;
}

__global__ void k_lq_update(SimHeader* hdr, int prec, int nsteps, Multi m) {
  const int b = blockIdx.x, f = threadIdx.x;
  if (f >= 6) return;
  SimHeader* h = moved(hdr, shift_of(m, b));
  h->lq_used[f] = h->lq_scale[f];
  const float a = h->lq_amax[f];
  const int r = h->step + 1;  // the row just written; the next pass writes r + 1
  if (a > 0.f) h->lq_scale[f] = a * (r + 1 <= nsteps ? lq_growth(h, f, r, r + 1) : 1.f) / lq_target(prec);
  h->lq_amax[f] = 0.f;
}

// Largest |value| of field blockIdx.z (of six) into lq_amax (values >= 0: the
// float bit patterns order like the ints).
__global__ void __launch_bounds__(NTP) k_lq_absmax(SimHeader* hdr, const float* __restrict__ f0,
                                                   const float* __restrict__ f1, const float* __restrict__ f2,
                                                   const float* __restrict__ f3, const float* __restrict__ f4,
                                                   const float* __restrict__ f5, int64_t P, Multi m) {
  const int64_t by = shift_of(m, blockIdx.y);
  const int f = blockIdx.z;
  const float* src = moved(f == 0 ? f0 : f == 1 ? f1 : f == 2 ? f2 : f == 3 ? f3 : f == 4 ? f4 : f5, by);
  float a = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * NTP + threadIdx.x; i < P; i += (int64_t)gridDim.x * NTP)
    a = fmaxf(a, fabsf(src[i]));
  const unsigned ua = __reduce_max_sync(0xffffffffu, __float_as_uint(a));
  if ((threadIdx.x & 31) == 0 && ua != 0u) atomicMax(reinterpret_cast<unsigned*>(&moved(hdr, by)->lq_amax[f]), ua);
}

__global__ void k_lq_init(SimHeader* hdr, int prec, Multi m) {
  const int b = blockIdx.x, f = threadIdx.x;
  if (f >= 6) return;
  SimHeader* h = moved(hdr, shift_of(m, b));
  const float a = h->lq_amax[f];
  h->lq_scale[f] = h->lq_used[f] = a > 0.f ? a * lq_growth(h, f, 0, 1) / lq_target(prec) : 1.f;
  h->lq_amax[f] = 0.f;
}

__global__ void k_lq_zero_amax(SimHeader* hdr, Multi m) {
  SimHeader* h = moved(hdr, shift_of(m, blockIdx.x));
  if (threadIdx.x < 6) h->lq_amax[threadIdx.x] = 0.f;
}

__global__ void __launch_bounds__(NTP) k_lq_dequant(const unsigned short* __restrict__ src, float* __restrict__ dst,
                                                    int64_t P, int prec, const SimHeader* hdr, int f) {
  const float sc = hdr->lq_used[f];
  for (int64_t i = (int64_t)blockIdx.x * NTP + threadIdx.x; i < P; i += (int64_t)gridDim.x * NTP)
    dst[i] = lq_value(src[i], prec) * sc;
}

// Up to kParamWords int64 values carried in the launch parameters (a host to
// device copy that neither synchronises nor needs pinned memory).
constexpr int kParamWords = 480;
struct ParamWords {
  int64_t v[kParamWords];
};
__global__ void k_write_words(int64_t* __restrict__ dst, int n, const __grid_constant__ ParamWords w) {
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i < n) dst[i] = w.v[i];
}

__global__ void __launch_bounds__(NTP) k_zero(float4* __restrict__ p, int64_t n4, Multi m) {
  p = moved(p, shift_of(m, blockIdx.y));
  for (int64_t i = (int64_t)blockIdx.x * NTP + threadIdx.x; i < n4; i += (int64_t)gridDim.x * NTP)
    p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

cudaError_t part_deposit(const PartParams& pp, const float* sx, const float* sy, const float* sz,
                         float* rho, int64_t P, cudaStream_t s, Multi m) {
  k_deposit<<<dim3(blocks_for(P), m.nb), NTP, 0, s>>>(pp, sx, sy, sz, rho, P, m);
  return cudaGetLastError();
}

namespace {
thread_local int g_dep_box = 0, g_gk_box = 0;  // see set_particle_plan

// Dynamic shared memory of a box kernel, raised once to its largest box.
template <class K>
cudaError_t box_smem_attr(K kernel, size_t max_bytes, bool& done) {
  if (done) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes);
  if (e == cudaSuccess) done = true;
  return e;
}
bool g_dep_attr = false, g_gk_attr = false, g_gk_attr_xy = false;
}  // namespace

void set_particle_plan(int deposit_box, int gather_box) {
  g_dep_box = std::max(0, std::min(deposit_box, kMaxDepositBox)) & ~3;
  g_gk_box = std::max(0, std::min(gather_box, kMaxGatherBox)) & ~3;
}

cudaError_t part_drift_deposit(const PartParams& pp, float* sx, float* sy, float* sz, float* vx,
                               float* vy, float* vz, const float* ax, const float* ay,
                               const float* az, const float* dpx, const float* dpy,
                               const float* dpz, float* rho, StepDt dt, int64_t P,
                               cudaStream_t s, Multi m, LptMix mix) {
  if (g_dep_box > 0 && P == (int64_t)pp.Np * pp.Np * pp.Np && pp.Np >= LB) {
    cudaError_t e = box_smem_attr(k_drift_deposit_box, kMaxDepositBox * sizeof(float), g_dep_attr);
    if (e != cudaSuccess) return e;
    k_drift_deposit_box<<<dim3((unsigned)(P / LBP), m.nb), NTP, (size_t)g_dep_box * sizeof(float), s>>>(
        pp, sx, sy, sz, vx, vy, vz, ax, ay, az, dpx, dpy, dpz, rho, dt, m, mix, g_dep_box);
    return cudaGetLastError();
  }
  k_drift_deposit<<<dim3(blocks_for(P), m.nb), NTP, 0, s>>>(pp, sx, sy, sz, vx, vy, vz, ax, ay, az,
                                                            dpx, dpy, dpz, rho, dt, P, m, mix);
  return cudaGetLastError();
}

cudaError_t part_gather_kick(const PartParams& pp, const float* sx, const float* sy,
                             const float* sz, float* vx, float* vy, float* vz, float* ax,
                             float* ay, float* az, const float* Ax, const float* Ay,
                             const float* Az, const float* F0, const float* F1, const float* Fz, bool pairs,
                             StepDt dt, int64_t P, cudaStream_t s, Multi m, LptMix mix) {
  if (g_gk_box > 0 && P == (int64_t)pp.Np * pp.Np * pp.Np && pp.Np >= LB) {
    auto k = pairs ? k_gather_kick_box<true> : k_gather_kick_box<false>;
    cudaError_t e = box_smem_attr(k, 3 * kMaxGatherBox * sizeof(float), pairs ? g_gk_attr_xy : g_gk_attr);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)(P / LBP), m.nb), NTP, 3 * (size_t)g_gk_box * sizeof(float), s>>>(
        pp, sx, sy, sz, vx, vy, vz, ax, ay, az, Ax, Ay, Az, F0, F1, Fz, dt, m, mix, g_gk_box);
    return cudaGetLastError();
  }
  auto k = pairs ? k_gather_kick<true> : k_gather_kick<false>;
  k<<<dim3((unsigned)((P + NTP * PPT - 1) / (NTP * PPT)), m.nb), NTP, 0, s>>>(
      pp, sx, sy, sz, vx, vy, vz, ax, ay, az, Ax, Ay, Az, F0, F1, Fz, dt, P, m, mix);
  return cudaGetLastError();
}

cudaError_t split_pairs(const float2* fxy, float* x, float* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + NTP - 1) / NTP, 152 * 8));
  k_split_pairs<<<grid, NTP, 0, s>>>(fxy, x, y, n);
  return cudaGetLastError();
}

cudaError_t part_kick_drift_deposit(const PartParams& pp, float* sx, float* sy, float* sz, float* vx,
                                    float* vy, float* vz, const float* Ax, const float* Ay,
                                    const float* Az, const float* dpx, const float* dpy,
                                    const float* dpz, const float* F0, const float* F1, const float* Fz,
                                    bool pairs, float* rho, const SimHeader* hdr, int64_t P, cudaStream_t s,
                                    Multi m) {
  // two particles per thread at four CTAs per SM (64 registers); measured on the 512^3 / 1024^3
  // run (ms per launch): 8.9 against 9.5 at 76 registers, 10.4 at 119, 9.4 with one particle
  constexpr int Q = 2;
  auto k = pairs ? k_kick_drift_deposit<Q, 4, true> : k_kick_drift_deposit<Q, 4, false>;
  k<<<dim3((unsigned)((P + NTP * Q - 1) / (NTP * Q)), m.nb), NTP, 0, s>>>(
      pp, sx, sy, sz, vx, vy, vz, Ax, Ay, Az, dpx, dpy, dpz, F0, F1, Fz, rho, hdr, P, m);
  return cudaGetLastError();
}

cudaError_t part_snapshot(const PartParams& pp, const float* sx, const float* sy, const float* sz,
                          const float* vx, const float* vy, const float* vz, const float* lx,
                          const float* ly, const float* lz, float vscale, float* pos, float* vel,
                          int64_t P, cudaStream_t s, LptMix mix) {
  const double L = pp.L;
  k_snapshot<<<blocks_for(P), NTP, 0, s>>>(pp, sx, sy, sz, vx, vy, vz, lx, ly, lz, vscale, pos,
                                           vel, P, mix, L / pp.Np, 1.0 / L);
  return cudaGetLastError();
}

cudaError_t lq_update(SimHeader* hdr, int prec, int nsteps, cudaStream_t s, Multi m) {
  k_lq_update<<<m.nb, 32, 0, s>>>(hdr, prec, nsteps, m);
  return cudaGetLastError();
}

cudaError_t lq_init(SimHeader* hdr, const float* const* fields, int64_t P, int prec, cudaStream_t s, Multi m) {
  k_lq_zero_amax<<<m.nb, 32, 0, s>>>(hdr, m);
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((P + NTP - 1) / NTP, 152 * 4));
  k_lq_absmax<<<dim3(gx, m.nb, 6), NTP, 0, s>>>(hdr, fields[0], fields[1], fields[2], fields[3], fields[4],
                                                fields[5], P, m);
  k_lq_init<<<m.nb, 32, 0, s>>>(hdr, prec, m);
  return cudaGetLastError();
}

cudaError_t lq_dequant(const void* src, float* dst, int64_t P, int prec, const SimHeader* hdr, int f,
                       cudaStream_t s) {
  if (prec != 1 && prec != 2) return cudaErrorInvalidValue;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((P + NTP - 1) / NTP, 152 * 8));
  k_lq_dequant<<<gx, NTP, 0, s>>>(static_cast<const unsigned short*>(src), dst, P, prec, hdr, f);
  return cudaGetLastError();
}

// Non-finite values (NaN, +-Inf) among nf arrays of n floats each, added into *out.
struct NineArrays {
  const float* f[9];
};
__global__ void __launch_bounds__(NTP) k_count_nonfinite(const __grid_constant__ NineArrays a, int nf, int64_t n,
                                                         unsigned long long* __restrict__ out) {
  unsigned cnt = 0;
  for (int j = 0; j < nf; ++j)
    for (int64_t i = (int64_t)blockIdx.x * NTP + threadIdx.x; i < n; i += (int64_t)gridDim.x * NTP)
      cnt += isfinite(a.f[j][i]) ? 0u : 1u;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, (unsigned long long)cnt);
}

cudaError_t count_nonfinite(const float* const* f, int nf, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (nf < 1 || nf > 9) return cudaErrorInvalidValue;
  NineArrays a{};
  for (int j = 0; j < nf; ++j) a.f[j] = f[j];
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + NTP - 1) / NTP, 152 * 8));
  k_count_nonfinite<<<gx, NTP, 0, s>>>(a, nf, n, out);
  return cudaGetLastError();
}

cudaError_t step_advance(SimHeader* hdr, cudaStream_t s, Multi m) {
  k_step_advance<<<(m.nb + 127) / 128, 128, 0, s>>>(hdr, m);
  return cudaGetLastError();
}

cudaError_t set_header(SimHeader* hdr, const SimHeader& v, cudaStream_t s) {
  k_set_header<<<1, 1, 0, s>>>(hdr, v);
  return cudaGetLastError();
}

cudaError_t write_words(int64_t* dst, const int64_t* src, int64_t n, cudaStream_t s) {
  for (int64_t o = 0; o < n; o += kParamWords) {
    ParamWords w;
    const int c = (int)std::min<int64_t>(kParamWords, n - o);
    for (int i = 0; i < c; ++i) w.v[i] = src[o + i];
    k_write_words<<<(c + 127) / 128, 128, 0, s>>>(dst + o, c, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t zero_f32(float* p, int64_t n, cudaStream_t s, Multi m) {
  if (m.nb == 1 && !m.shift) return cudaMemsetAsync(p, 0, n * sizeof(float), s);
  if (n % 4 != 0 || (reinterpret_cast<uintptr_t>(p) & 15)) return cudaErrorInvalidValue;
  const int64_t n4 = n / 4;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n4 + NTP - 1) / NTP, 1024));
  k_zero<<<dim3(gx, m.nb), NTP, 0, s>>>(reinterpret_cast<float4*>(p), n4, m);
  return cudaGetLastError();
}

cudaError_t pos_deposit(int Nm, float cellscale, const float* pos, int64_t n, float* rho,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_pos_deposit<<<blocks_for(n), NTP, 0, s>>>(Nm, cellscale, pos, n, rho);
  return cudaGetLastError();
}

cudaError_t pk_bin(int N, const float2* dk, int nbins, double* acc, double norm,
                   cudaStream_t s, Multi m, int64_t acc_stride) {
  // bins (two 64-bit integers, three floats) and the window per kx
  const size_t sm = (size_t)nbins * 28 + (size_t)(N / 2 + 1) * sizeof(float);
  if (N > 4096 || sm > 200 * 1024) return cudaErrorInvalidValue;  // |n|^2 in 24 bits
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_pk_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t rows = (int64_t)N * N, wpb = NTP / 32;
  unsigned grid = (unsigned)std::min<int64_t>((rows + wpb - 1) / wpb, 152 * 8);
  if (m.nb > 1) grid = std::max<unsigned>(1, grid / (unsigned)std::min(m.nb, 8));
  k_pk_bin<<<dim3(grid, m.nb), NTP, sm, s>>>(dk, N, half_pitch(N), nbins, acc, norm, m, acc_stride);
  return cudaGetLastError();
}

}  // namespace cola
