// FFT passes of the PM step, with the k-space operations of the method fused
// into the passes that already hold the data in shared memory.
//
// A 3-D real transform is three passes over HBM: rows along x (contiguous,
// real <-> half spectrum by the two-for-one packing z = x[2j] + i x[2j+1]),
// then columns along y and along z (tiles of TW >= 4 adjacent kx columns, so
// every row segment of a tile is at least one whole 32-byte sector).
//
// Every pass is a persistent kernel (grid = SMs x resident CTAs) that walks
// its tiles in a software pipeline: the next tile is staged with cp.async into
// a second shared-memory buffer while the current tile is transformed.  The
// half spectra use the plane-pair interleaved layout of cola_internal.h.
//
// Most k-space operations and output stores run inside the tile transforms,
// through their load hook (first step) and store hook (last step), so a tile
// makes one round trip through shared memory per transform step and outputs
// leave for HBM from registers.
//
// Fusions:
//   * the z pass of a forward transform also applies the Green's function
//     (and G_eff, screening coupling, gradient) and runs the inverse z pass of
//     each output before writing it back (Poisson solve, App. B);
//   * the y inverse pass can emit the y derivative as a second output;
//   * the x inverse pass can apply the x derivative on load, and transforms up
//     to six independent arrays in one launch;
//   * the screening source S = delta * eps is formed between an inverse and a
//     forward x pass in one kernel (Sec. 6.1, Sec. 6.2);
//   * the LPT reweight by the per-k growth tables (Sec. 4.1, App. A) happens
//     on load of the z inverse pass.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "cola_internal.h"
#include "fft.cuh"

namespace cola {
namespace {

constexpr int NT = 256;

// Column tile width: about 4096 complex values per buffer, between 4 and 16
// columns; 8 columns (64-byte row segments) for single-array 1024-point columns.
constexpr int col_tw(int N, int NBUF) {
  return (N == 1024 && NBUF == 1) ? 8
         : (4096 / (N * NBUF)) < 4 ? 4 : ((4096 / (N * NBUF)) > 16 ? 16 : 4096 / (N * NBUF));
}
// Rows per x-pass tile: about 8192 staged values per tile (~64 KB in flight
// per CTA pair), 8..64 rows.
constexpr int row_tw(int N) { return 8192 / N < 8 ? 8 : (8192 / N > 64 ? 64 : 8192 / N); }

// Resident CTAs per SM that the shared memory of a kernel allows (1..3); used
// as the register bound of __launch_bounds__ so registers never limit occupancy
// below it.  Transforms of 512 points and more, and the force-side z passes
// (two transforms per tile), would spill at 3 and take at most 2.
constexpr int blocks_for_smem(size_t bytes, int N) {
  return bytes > 112 * 1024 ? 1 : (bytes > 72 * 1024 || N >= 512 ? 2 : 3);
}
// Stage buffer of a column tile: fft_rows rows (the transform's padding rows
// follow the N data rows) of NBUF arrays x TW columns.
constexpr int col_rows(int N) { return N + (1 << (ilog2(N) - ilog2(N) / 2)); }
constexpr size_t col_smem_c(int N, int NBUF) {
  return (N + 2 * (size_t)col_rows(N) * NBUF * col_tw(N, NBUF)) * 8;
}
// the same for an explicit tile width
constexpr size_t col_smem_tw(int N, int TW) { return (N + 2 * (size_t)col_rows(N) * TW) * 8; }
// Tile width of the fused force-side z passes: 128-byte tile rows at N = 512
// (the z stride is N P 8 bytes; longer contiguous rows per DRAM page), the
// column default elsewhere.
constexpr int ztw(int N) { return N == 512 ? 16 : col_tw(N, 1); }

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

thread_local int g_grid_cap = 0;  // 0: no cap (see set_grid_cap)

struct KernelInfo {
  const void* fn;
  size_t smem;
  int per_sm;
};
std::mutex g_kinfo_mu;
std::vector<KernelInfo> g_kinfo;

// Sets the shared-memory limit of a kernel once and caches its resident CTAs per SM.
template <class K>
cudaError_t resident_ctas(K kernel, size_t smem, int& per_sm) {
  std::lock_guard<std::mutex> lk(g_kinfo_mu);
  for (const KernelInfo& k : g_kinfo)
    if (k.fn == (const void*)kernel && k.smem == smem) {
      per_sm = k.per_sm;
      return cudaSuccess;
    }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem);
  if (e != cudaSuccess) return e;
  g_kinfo.push_back({(const void*)kernel, smem, per_sm});
  return cudaSuccess;
}

// Persistent grid: resident CTAs x SMs, at most one CTA per tile, at most the
// calling thread's grid cap (used when many small simulations run concurrently).
template <class K>
cudaError_t prep(K kernel, size_t smem, int64_t ntiles, unsigned& grid) {
  if (ntiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;  // tile indices are 32-bit
  int per_sm = 0;
  cudaError_t e = resident_ctas(kernel, smem, per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t g = std::min<int64_t>(ntiles, (int64_t)per_sm * sm_count());
  if (g_grid_cap > 0) g = std::min<int64_t>(g, g_grid_cap);
  grid = (unsigned)std::max<int64_t>(g, 1);
  return cudaSuccess;
}

__device__ __forceinline__ void load_tw(float2* tw, const float2* __restrict__ twg, int n) {
  for (int i = threadIdx.x; i < n; i += NT) tw[i] = twg[i];
}

// ---------------------------------------------------------------- cp.async helpers
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;  // 0: zero-fill, nothing read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// ---------------------------------------------------------------- column tiles
// Tile element (n, c) of sub-block `sub` lives at buf[n * TP + sub * TW + c];
// global element at g[base + row(n) + hcol(c)] with row(n) = (n >> 1) ra +
// (n & 1) rb (the half-spectrum layout of cola_internal.h); only columns
// c0 + c < N/2 + 1 exist.  Each thread keeps one 16-byte piece (or one column)
// and walks rows n0, n0 + step, ... (step even, so n & 1 stays fixed).
template <int N, int TW, int TP>
__device__ __forceinline__ void col_issue(float2* buf, int sub, const float2* __restrict__ g,
                                          int64_t base, int64_t ra, int64_t rb, int c0) {
  constexpr int CH = TW / 2;  // 16-byte pieces per row segment
  constexpr int STEP = NT / CH;
  static_assert(STEP % 2 == 0, "row step must be even");
  const int j = threadIdx.x % CH, n0 = threadIdx.x / CH;
  const bool v = c0 + 2 * j < N / 2 + 1;
  const float2* src = g + base + (n0 >> 1) * ra + (n0 & 1) * rb + hcol(2 * j);
  float2* dst = buf + n0 * TP + sub * TW + 2 * j;
#pragma unroll 4
  for (int n = n0; n < N; n += STEP) {
    cp_async16(dst, v ? (const void*)src : (const void*)g, v);
    src += (STEP / 2) * ra;
    dst += STEP * TP;
  }
}

// 16-bit seeds: 4 complex values (uint32 each) per 16-byte chunk.  Field f of
// row n is staged raw in the sub-block 2/3 area of that row:
// raw(f, n, c) = ((uint32*)buf)[8 n TW + 4 TW + f TW + c]  (TP = 4 TW).
template <int N, int TW>
__device__ __forceinline__ void col_issue_raw(uint32_t* rb_, int f, const uint32_t* __restrict__ g,
                                              int64_t base, int64_t ra, int64_t rb, int c0) {
  constexpr int CH = TW / 4;
  constexpr int STEP = NT / CH;
  static_assert(STEP % 2 == 0, "row step must be even");
  const int j = threadIdx.x % CH, n0 = threadIdx.x / CH;
  const bool v = c0 + 4 * j < N / 2 + 1;
  const uint32_t* src = g + base + (n0 >> 1) * ra + (n0 & 1) * rb + hcol(4 * j);
  uint32_t* dst = rb_ + 8 * n0 * TW + 4 * TW + f * TW + 4 * j;
#pragma unroll 4
  for (int n = n0; n < N; n += STEP) {
    cp_async16(dst, v ? (const void*)src : (const void*)g, v);
    src += (STEP / 2) * ra;
    dst += 8 * STEP * TW;
  }
}

template <int N, int TW, int TP>
__device__ __forceinline__ void col_store(const float2* buf, int sub, float2* __restrict__ g,
                                          int64_t base, int64_t ra, int64_t rb, int c0) {
  constexpr int STEP = NT / TW;
  static_assert(STEP % 2 == 0, "row step must be even");
  const int c = threadIdx.x % TW, n0 = threadIdx.x / TW;
  if (c0 + c >= N / 2 + 1) return;
  float2* dst = g + base + (n0 >> 1) * ra + (n0 & 1) * rb + hcol(c);
  const float2* src = buf + n0 * TP + sub * TW + c;
#pragma unroll 4
  for (int n = n0; n < N; n += STEP) {
    *dst = *src;
    dst += (STEP / 2) * ra;
    src += STEP * TP;
  }
}

// The elements of an N x TW column tile that a thread owns: column c = tid mod
// TW and rows n = n0 + i STEP, i < E (STEP = NT / TW, n0 = tid / TW).  |n|^2
// of element (kx, ky, n) is sxy + fz(n)^2 with sxy = kx^2 + ky^2 kept per
// thread; the integer sum is exact, so k^2 = kf^2 |n|^2 rounds once.
template <int N, int TW>
struct TileLane {
  static constexpr int STEP = NT / TW, E = N * TW / NT;
  int c, n0, sxy;
  __device__ __forceinline__ TileLane(int c0, int iy) {
    c = threadIdx.x % TW;
    n0 = threadIdx.x / TW;
    const int fx = c0 + c, fy = freq_index(iy, N);
    sxy = fx * fx + fy * fy;
  }
  __device__ __forceinline__ int row(int i) const { return n0 + i * STEP; }
  __device__ __forceinline__ float k2(int n, float kf2) const {
    const int fz = freq_index(n, N);
    return kf2 * (float)(sxy + fz * fz);
  }
};

// Store hook of a column transform that writes element (n, c) straight to
// g[(n >> 1) ra + (n & 1) rb + hcol(c)] (g = the tile's base, columns c < live
// exist) instead of through the tile and col_store: a warp's stores cover whole
// 128-byte chunk pairs.
struct ColOut {
  static constexpr bool kSmem = false;
  float2* g;
  int64_t ra, rb;
  int live;
  __device__ __forceinline__ float2 operator()(float2 v, int n, int c, int) const {
    if (c < live) g[(n >> 1) * ra + (n & 1) * rb + hcol(c)] = v;
    return v;
  }
  __device__ __forceinline__ void ready() const {}
};

// Column geometry: tile t -> (simulation b, outer index o, column block c0);
// base = the element offset of (o, row 0, c0) and `by` = the byte shift of
// simulation b's buffers.  Outer index o sits at (o >> 1) oa + (o & 1) ob and
// tile row n at (n >> 1) ra + (n & 1) rb.  With pair_tiles, consecutive tiles
// take o = 2i and 2i + 1 of the same column block (the two halves of each
// 128-byte chunk pair of the y pass are read by neighbouring CTAs together).
template <int N, int TW>
struct ColGeo {
  static constexpr int ntx = (N / 2) / TW + 1;
  static constexpr int64_t tps = (int64_t)N * ntx;  // tiles per simulation
  int64_t oa, ob, ra, rb;
  int pair_tiles;
  int zaxis;  // 1: tiles run along z (o = y), 0: along y (o = z)
  Multi m;
  // t < 2^31 (prep checks the tile count); divisions by compile-time constants
  __device__ __forceinline__ void tile(int64_t t64, int& o, int& c0, int64_t& base, int64_t& by) const {
    uint32_t t = (uint32_t)t64;
    const uint32_t b = t / (uint32_t)tps;
    t -= b * (uint32_t)tps;
    by = shift_of(m, (int)b);
    if (pair_tiles) {
      const uint32_t q = t / (2 * ntx), r = t - q * (2 * ntx);
      o = (int)(q * 2 + (r & 1));
      c0 = (int)(r >> 1) * TW;
    } else {
      const uint32_t q = t / ntx;
      o = (int)q;
      c0 = (int)(t - q * ntx) * TW;
    }
    base = (o >> 1) * oa + (o & 1) * ob + hcol(c0);
  }
};

// Software pipeline over the tiles of one launch.  Op supplies
//   issue(buf, t): cp.async the inputs of tile t into buf (no commit)
//   issue_side(t): cp.async of a second input of tile t into op.extra (no commit;
//     may do nothing); its group is committed BEFORE the next tile's prefetch,
//     so process() can wait for it with cp_async_wait<1>() while the prefetch
//     of tile t + grid stays in flight
//   process(buf, tw, t): transform + store (leaves buf free after a final barrier)
template <int N, int BUFELEMS, class Op>
__device__ __forceinline__ void col_pipeline(Op op, const float2* __restrict__ twg,
                                             int64_t ntiles) {
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + N;
  float2* b1 = b0 + BUFELEMS;
  op.extra = b1 + BUFELEMS;  // optional per-op scratch after the two stage buffers
  load_tw(tw, twg, N);
  int64_t t = blockIdx.x;
  if (t < ntiles) op.issue(b0, t);
  cp_async_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    op.issue_side(t);  // op.extra is free: the previous tile ended with a barrier
    cp_async_commit();
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) op.issue(cur ? b0 : b1, tn);
    cp_async_commit();
    cp_async_wait<2>();  // tile t's main input has landed
    __syncthreads();
    op.process(cur ? b1 : b0, tw, t);
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- TMA tile loads
// Single-simulation launches of the long column passes stage their tiles with
// the tensor-memory accelerator: thread 0 issues a few cp.async.bulk.tensor
// copies per tile, completion is tracked by an mbarrier per stage buffer, and
// the transform warps issue no load instructions.  The half spectrum is seen
// as a 5-D array of 8-byte elements (column within a 64-byte half chunk, plane
// parity, chunk, y, plane pair), byte strides 8, 64, 128, 2P*8, 2NP*8: the
// interleaved layout of cola_internal.h.  A z tile (TW <= 8 columns of one y)
// is boxes of {TW, 2, 1, 1, <= 256 pairs}, landing as rows n = 2j + parity of
// TW values; a y tile (one z) boxes of {TW, 1, 1, <= 256 rows, 1}.
__device__ unsigned int g_tile_load_failures;  // waits that ran out (host: tile_load_failures)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of b to complete, for limit_ns (one second) at most.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity,
                                         uint64_t limit_ns = 1000000000ull) {
  if (bar_try(b, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!bar_try(b, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// orders this CTA's earlier generic-proxy accesses to shared memory before
// later async-proxy (TMA) writes
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void fence_bar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load5(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5, %6}], [%7];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// 1-D bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global memory into shared memory, completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Zero fill by bulk stores from a zeroed shared-memory region (thread 0): `bytes`
// (a multiple of 16) at dst, in pieces of at most ZB bytes, one bulk group; at
// most eight groups stay outstanding (the region is never written again, so
// only the count is bounded).
__device__ __forceinline__ void bulk_zero(char* dst, int64_t bytes, const void* zeros, uint32_t ZB) {
  for (int64_t o = 0; o < bytes; o += ZB) {
    const uint32_t len = (uint32_t)(bytes - o < (int64_t)ZB ? bytes - o : (int64_t)ZB);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst + o),
                 "r"(smem_u32(zeros)), "r"(len)
                 : "memory");
  }
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 8;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_store_drain() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Issue the loads of column tile t of `geo` into buf (thread 0; buf 128-byte aligned).
template <int N, int TW>
__device__ __forceinline__ void tma_tile(const ColGeo<N, TW>& geo, const CUtensorMap* map, float2* buf,
                                         int64_t t, uint64_t* bar) {
  static_assert(TW <= 8 && TW % 2 == 0, "TMA tiles: at most one 64-byte half chunk");
  int o, c0;
  int64_t base, by;
  geo.tile(t, o, c0, base, by);
  bar_expect(bar, (uint32_t)(N * TW * sizeof(float2)));
  if (geo.zaxis) {
    constexpr int B = N / 2 < 256 ? N / 2 : 256;
#pragma unroll
    for (int k = 0; k < N / 2; k += B) tma_load5(buf + 2 * k * TW, map, c0 & 7, 0, c0 >> 3, o, k, bar);
  } else {
    constexpr int B = N < 256 ? N : 256;
#pragma unroll
    for (int k = 0; k < N; k += B) tma_load5(buf + k * TW, map, c0 & 7, o & 1, c0 >> 3, k, o >> 1, bar);
  }
}

// col_pipeline with TMA staging (one simulation).  Op supplies geo, process()
// and, for a side input (kSide), the members sbar / spar that its process()
// waits on through tma_side_wait; map1 is the side input's tensor map.
// Barriers: bars[0], bars[1] for the two stage buffers, bars[2] for the side
// input (landing in op.extra, N x TW).  A wait that runs out stops the CTA
// (counted in g_tile_load_failures) after a bounded wait for its copies.
struct TmaSide {
  uint64_t* bar = nullptr;
  uint32_t parity = 0;
  int* fail = nullptr;
  // thread 0 waits; the caller's next barrier publishes the data
  __device__ __forceinline__ void wait() const {
    if (bar && threadIdx.x == 0 && !bar_wait(bar, parity)) *fail = 1;
  }
};

// Shared memory: twiddles (N), two stage buffers, EXTRA float2 of op.extra,
// then the three barriers and the failure flag.
template <int N, int BUFELEMS, int EXTRA>
constexpr size_t tma_smem() {
  return ((size_t)N + 2 * (size_t)BUFELEMS + EXTRA) * sizeof(float2) + 4 * sizeof(uint64_t);
}

template <int N, int BUFELEMS, bool SIDE, int EXTRA, class Op>
__device__ __forceinline__ void col_pipeline_tma(Op op, const float2* __restrict__ twg, int64_t ntiles,
                                                 const CUtensorMap* map0, const CUtensorMap* map1) {
  static_assert((N * sizeof(float2)) % 128 == 0 && (BUFELEMS * sizeof(float2)) % 128 == 0,
                "TMA destinations 128-byte aligned");
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + N;
  float2* b1 = b0 + BUFELEMS;
  op.extra = b1 + BUFELEMS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(op.extra + EXTRA);
  int& fail = *reinterpret_cast<int*>(bars + 3);
  const bool lead = threadIdx.x == 0;
  if (lead) {
    bar_init(&bars[0]);
    bar_init(&bars[1]);
    bar_init(&bars[2]);
    fence_bar_init();
    fail = (smem_u32(sm) & 127) ? 1 : 0;  // no copy goes into a misaligned buffer
  }
  load_tw(tw, twg, N);
  __syncthreads();
  if (fail) {
    if (lead) atomicAdd(&g_tile_load_failures, 1u);
    return;
  }
  // thread 0: parity of each barrier's next phase (bit i) and copies issued but
  // not yet waited for (bit i)
  uint32_t par = 0, pend = 0;
  int64_t t = blockIdx.x;
  if (lead && t < ntiles) {
    tma_tile(op.geo, map0, b0, t, &bars[0]);
    pend |= 1u;
  }
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    if (lead) {
      fence_async_smem();  // the previous tile's accesses to the buffers and to extra are done
      if (SIDE) {
        tma_tile(op.geo, map1, op.extra, t, &bars[2]);
        pend |= 4u;
      }
      const int64_t tn = t + gridDim.x;
      if (tn < ntiles) {
        tma_tile(op.geo, map0, cur ? b0 : b1, tn, &bars[cur ^ 1]);
        pend |= 1u << (cur ^ 1);
      }
      if (bar_wait(&bars[cur], (par >> cur) & 1u)) {
        par ^= 1u << cur;
        pend &= ~(1u << cur);
      } else {
        fail = 1;
      }
    }
    __syncthreads();
    if (fail) break;
    if constexpr (SIDE) op.side = TmaSide{&bars[2], (par >> 2) & 1u, &fail};
    op.process(cur ? b1 : b0, tw, t);
    __syncthreads();
    if (fail) break;
    if (SIDE && lead) {
      par ^= 4u;
      pend &= ~4u;
    }
    cur ^= 1;
  }
  if (lead && fail) {
    atomicAdd(&g_tile_load_failures, 1u);
    for (int i = 0; i < 3; ++i)
      if ((pend >> i) & 1u) bar_wait(&bars[i], (par >> i) & 1u);  // bounded: copies in flight land before exit
  }
}

// Self-test of the bounded wait: one thread arms a barrier phase for 16 bytes
// that no copy will deliver and waits on it with bar_wait; g_wait_probe = 1 when
// the wait gave up after limit_ns, 0 if the phase completed.
__device__ int g_wait_probe;
__global__ void k_wait_probe(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  bar_init(&bar);
  fence_bar_init();
  bar_expect(&bar, 16);
  g_wait_probe = bar_wait(&bar, 0, limit_ns) ? 0 : 1;
}

// ---------------------------------------------------------------- plain column pass
// out = transform of in along the tile axis; out may alias in.
template <int N, int TW, bool INV>
struct OpCol {
  ColGeo<N, TW> geo;
  const float2* in;
  float2* out;
  float2* extra = nullptr;  // scratch after the stage buffers (set by col_pipeline)
  __device__ __forceinline__ void issue_side(int64_t) const {}
  __device__ __forceinline__ void issue(float2* buf, int64_t t) const {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    col_issue<N, TW, TW>(buf, 0, moved(in, by), base, geo.ra, geo.rb, c0);
  }
  // outputs go to HBM from the last step's registers (ColOut)
  __device__ __forceinline__ void process(float2* buf, const float2* tw, int64_t t) const {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    fft_tile<N, TW, TW, NT, INV, 1, TileLoad, ColOut>(
        buf, tw, TileLoad{}, ColOut{moved(out, by) + base, geo.ra, geo.rb, N / 2 + 1 - c0});
  }
};

template <int N, int TW, bool INV, bool TMA>
__global__ void __launch_bounds__(NT, blocks_for_smem(col_smem_c(N, 1), N)) k_col(OpCol<N, TW, INV> op, const float2* __restrict__ twg,
                                            int64_t ntiles, const __grid_constant__ CUtensorMap map) {
  if constexpr (TMA) col_pipeline_tma<N, fft_rows<N>() * TW, false, 0>(op, twg, ntiles, &map, nullptr);
  else col_pipeline<N, fft_rows<N>() * TW>(op, twg, ntiles);
}

// ---------------------------------------------------------------- y inverse, two outputs
template <int N, int TW>
struct OpYinv2 {
  // Load hook of the two-array transform: columns c < TW are the staged input,
  // columns TW + c its y derivative i kfs f_n (zero on the Nyquist row), formed
  // from column c as the first step loads it.
  struct PairLoad {
    float kfs;
    __device__ __forceinline__ float2 operator()(const float2* buf, int n, int c, int at) const {
      const bool d = c >= TW;
      const float2 v = buf[d ? at - TW : at];
      const float f = (n == N / 2) ? 0.f : kfs * (float)freq_index(n, N);
      const float a = d ? 0.f : 1.f, b = d ? f : 0.f;  // v (a + i b)
      return make_float2(a * v.x - b * v.y, a * v.y + b * v.x);
    }
  };
  // Store hook: columns c < TW to the plain output, TW + c to the derivative,
  // straight from the last step's registers.
  struct PairOut {
    static constexpr bool kSmem = false;
    float2 *gp, *gd;
    int64_t ra, rb;
    int live;
    __device__ __forceinline__ float2 operator()(float2 v, int n, int c, int) const {
      const bool d = c >= TW;
      const int cc = d ? c - TW : c;
      if (cc < live) (d ? gd : gp)[(n >> 1) * ra + (n & 1) * rb + hcol(cc)] = v;
      return v;
    }
    __device__ __forceinline__ void ready() const {}
  };
  ColGeo<N, TW> geo;
  const float2* in;
  float2 *outp, *outd;
  float kfs;
  float2* extra = nullptr;  // scratch after the stage buffers (set by col_pipeline)
  __device__ __forceinline__ void issue_side(int64_t) const {}
  __device__ __forceinline__ void issue(float2* buf, int64_t t) const {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    col_issue<N, TW, 2 * TW>(buf, 0, moved(in, by), base, geo.ra, geo.rb, c0);
  }
  __device__ __forceinline__ void process(float2* buf, const float2* tw, int64_t t) const {
    constexpr int TP = 2 * TW;
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    fft_tile<N, TP, TP, NT, true, 1, PairLoad, PairOut>(
        buf, tw, PairLoad{kfs},
        PairOut{moved(outp, by) + base, moved(outd, by) + base, geo.ra, geo.rb, N / 2 + 1 - c0});
  }
};

template <int N, int TW>
__global__ void __launch_bounds__(NT, blocks_for_smem(col_smem_c(N, 2), N)) k_yinv2(OpYinv2<N, TW> op, const float2* __restrict__ twg,
                                              int64_t ntiles) {
  col_pipeline<N, fft_rows<N>() * 2 * TW>(op, twg, ntiles);
}

// y inverse with the y derivative as a second output, for long columns (512
// and 1024 points) where a two-array tile would need 32-byte rows: three tile
// buffers of TW columns rotate between the input (transformed in place for the
// plain output), the derivative and the prefetch of the next input, so the
// input is read from HBM once with TW-column (64-byte) rows.  Given input
// buffer I, the derivative goes to (I + 1) mod 3 and the prefetch to (I + 2)
// mod 3, which holds the next tile's input.
// Load hook: i kfs f_n times element (n, c) of another tile (zero on the Nyquist row).
template <int N>
struct DerivLoad {
  const float2* src;
  float kfs;
  __device__ __forceinline__ float2 operator()(const float2*, int n, int, int at) const {
    const float f = (n == N / 2) ? 0.f : kfs * (float)freq_index(n, N);
    return cscale(cmul_i(src[at]), f);
  }
};

template <int N, int TW>
constexpr size_t yinv2r_smem() {
  return (N + 3 * (size_t)fft_rows<N>() * TW) * sizeof(float2);
}
template <int N, int TW>
struct Yinv2rCfg {
  static constexpr bool ONE_CTA = blocks_for_smem(yinv2r_smem<N, TW>(), N) < 2;
};

// Both transforms of tile t from input buffer bi (the derivative into bd).
template <int N, int TW>
__device__ __forceinline__ void yinv2r_tile(const ColGeo<N, TW>& geo, float2* bi, float2* bd,
                                            const float2* tw, float2* __restrict__ outp,
                                            float2* __restrict__ outd, float kfs, int64_t t) {
  int o, c0;
  int64_t base, by;
  geo.tile(t, o, c0, base, by);
  const ColOut out{nullptr, geo.ra, geo.rb, N / 2 + 1 - c0};
  ColOut od = out, op = out;
  od.g = moved(outd, by) + base;
  op.g = moved(outp, by) + base;
  if constexpr (Yinv2rCfg<N, TW>::ONE_CTA) {
    // one CTA per SM: the derivative transform runs first, its first step
    // reading the input (times i kfs f_n) from bi, which the plain transform
    // then overwrites; both store straight to HBM
    fft_tile_call<N, TW, TW, NT, true, 1, DerivLoad<N>, ColOut>(bd, tw, DerivLoad<N>{bi, kfs}, od);
    fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(bi, tw, TileLoad{}, op);
  } else {
    // two CTAs per SM (128 registers, where the load hook spills): a pass over the tile
    const DerivLoad<N> dl{bi, kfs};
    for (int e = threadIdx.x; e < N * TW; e += NT) bd[e] = dl(bd, e / TW, 0, e);
    __syncthreads();
    fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(bd, tw, TileLoad{}, od);
    fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(bi, tw, TileLoad{}, op);
  }
}

// TMA: buffer i's copies complete on barrier i (after the three buffers; the
// failure flag follows), as in col_pipeline_tma.
template <int N, int TW, bool TMA>
__global__ void __launch_bounds__(NT, blocks_for_smem(yinv2r_smem<N, TW>(), N)) k_yinv2r(
    ColGeo<N, TW> geo, const float2* __restrict__ in, float2* __restrict__ outp,
    float2* __restrict__ outd, float kfs, const float2* __restrict__ twg, int64_t ntiles,
    const __grid_constant__ CUtensorMap map) {
  constexpr int B = fft_rows<N>() * TW;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  auto buf = [&](int i) { return sm + N + i * B; };
  if constexpr (TMA) {
    static_assert((N * sizeof(float2)) % 128 == 0 && (B * sizeof(float2)) % 128 == 0,
                  "TMA destinations 128-byte aligned");
    uint64_t* bars = reinterpret_cast<uint64_t*>(buf(3));
    int& fail = *reinterpret_cast<int*>(bars + 3);
    const bool lead = threadIdx.x == 0;
    if (lead) {
      bar_init(&bars[0]);
      bar_init(&bars[1]);
      bar_init(&bars[2]);
      fence_bar_init();
      fail = (smem_u32(sm) & 127) ? 1 : 0;
    }
    load_tw(tw, twg, N);
    __syncthreads();
    if (fail) {
      if (lead) atomicAdd(&g_tile_load_failures, 1u);
      return;
    }
    uint32_t par = 0, pend = 0;  // thread 0: next phase parity and pending copies, bit i = barrier i
    int64_t t = blockIdx.x;
    if (lead && t < ntiles) {
      tma_tile(geo, &map, buf(0), t, &bars[0]);
      pend |= 1u;
    }
    int I = 0;
    for (; t < ntiles; t += gridDim.x) {
      const int D = I == 2 ? 0 : I + 1, F = I == 0 ? 2 : I - 1;
      if (lead) {
        fence_async_smem();
        const int64_t tn = t + gridDim.x;
        if (tn < ntiles) {
          tma_tile(geo, &map, buf(F), tn, &bars[F]);
          pend |= 1u << F;
        }
        if (bar_wait(&bars[I], (par >> I) & 1u)) {
          par ^= 1u << I;
          pend &= ~(1u << I);
        } else {
          fail = 1;
        }
      }
      __syncthreads();
      if (fail) break;
      yinv2r_tile<N, TW>(geo, buf(I), buf(D), tw, outp, outd, kfs, t);
      __syncthreads();  // both buffers are free for later prefetches
      I = F;
    }
    if (lead && fail) {
      atomicAdd(&g_tile_load_failures, 1u);
      for (int i = 0; i < 3; ++i)
        if ((pend >> i) & 1u) bar_wait(&bars[i], (par >> i) & 1u);
    }
  } else {
    load_tw(tw, twg, N);
    int64_t t = blockIdx.x;
    if (t < ntiles) {
      int o, c0;
      int64_t base, by;
      geo.tile(t, o, c0, base, by);
      col_issue<N, TW, TW>(buf(0), 0, moved(in, by), base, geo.ra, geo.rb, c0);
    }
    cp_async_commit();
    int I = 0;
    for (; t < ntiles; t += gridDim.x) {
      const int D = I == 2 ? 0 : I + 1, F = I == 0 ? 2 : I - 1;
      const int64_t tn = t + gridDim.x;
      if (tn < ntiles) {
        int o, c0;
        int64_t base, by;
        geo.tile(tn, o, c0, base, by);
        col_issue<N, TW, TW>(buf(F), 0, moved(in, by), base, geo.ra, geo.rb, c0);
      }
      cp_async_commit();
      cp_async_wait<1>();  // tile t's input has landed
      __syncthreads();
      yinv2r_tile<N, TW>(geo, buf(I), buf(D), tw, outp, outd, kfs, t);
      __syncthreads();  // both buffers are free for later prefetches
      I = F;
    }
    cp_async_wait<0>();
  }
}

// ---------------------------------------------------------------- screening field (z pass)
// Smoothing window of the Vainshtein density (App. B) at h = k^2 R^2 / 2:
// 0 Gaussian exp(-h); 1 top-hat 3 (sin x - x cos x) / x^3 with x^2 = 2h, by its
// Taylor series below x = 1/2 where the closed form cancels; 2 sharp-k, 1 for
// kR <= 1 (h <= 1/2) and 0 beyond.
__device__ __forceinline__ float smoothing_window(float h, int filter) {
  if (filter == 0) return __expf(-h);
  if (filter == 2) return h <= 0.5f ? 1.f : 0.f;
  const float x2 = 2.f * h;
  if (x2 < 0.25f)
    return fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 1330560.f, -1.f / 15120.f), 1.f / 280.f), -0.1f), 1.f);
  const float x = sqrtf(x2);
  float s, c;
  sincospif(x * 0.318309886f, &s, &c);  // argument reduction exact in units of pi
  return 3.f * (s - x * c) / (x * x2);
}

// MODEL: 1 the Newtonian potential (chameleon-type screening); 2 the density
// smoothed by the Gaussian window; 3 the density smoothed by the top-hat or
// sharp-k window (fp.filter).  The Gaussian keeps a kernel of its own: a
// per-element switch over the windows slows the pass by a third.
template <int N, int TW, int MODEL>
struct OpZScreenField {
  // Store hook of the forward transform: delta(k) out to HBM, the field's
  // multiplier (-kappa/k^2, or the smoothing window) applied in place.
  struct Field {
    static constexpr bool kSmem = true;
    float2* dk;  // delta(k) of the tile: element (n, c) at dk[(n >> 1) ra + (n & 1) rb + hcol(c)]
    int64_t ra, rb;
    int c0, fy2;
    float kf2, kappa_norm, R2half, norm;
    int filter;
    __device__ __forceinline__ float2 operator()(float2 v, int n, int c, int) const {
      if (c0 + c < N / 2 + 1) dk[(n >> 1) * ra + (n & 1) * rb + hcol(c)] = v;
      const int fx = c0 + c, fz = freq_index(n, N);
      const float k2 = kf2 * (float)(fx * fx + fy2 + fz * fz);
      float m = 0.f;
      if (k2 > 0.f) {
        if (MODEL == 1) m = __fdividef(-kappa_norm, k2);
        else if (MODEL == 2) m = __expf(-k2 * R2half) * norm;
        else m = smoothing_window(k2 * R2half, filter) * norm;
      }
      return cscale(v, m);
    }
    __device__ __forceinline__ void ready() const {}
  };
  ColGeo<N, TW> geo;
  const float2* in;
  float2 *dk_out, *w_out;
  ForceParams fp;
  float2* extra = nullptr;  // scratch after the stage buffers (set by col_pipeline)
  __device__ __forceinline__ void issue_side(int64_t) const {}
  __device__ __forceinline__ void issue(float2* buf, int64_t t) const {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    col_issue<N, TW, TW>(buf, 0, moved(in, by), base, geo.ra, geo.rb, c0);
  }
  __device__ __forceinline__ void process(float2* buf, const float2* tw, int64_t t) const {
    int iy, c0;
    int64_t base, by;
    geo.tile(t, iy, c0, base, by);
    ForceParams fp = this->fp;
    resolve(fp, by);
    const int fy = freq_index(iy, N);
    const Field f{moved(dk_out, by) + base, geo.ra, geo.rb, c0, fy * fy, fp.kf * fp.kf, fp.kappa_norm,
                  fp.R2half, fp.norm, fp.filter};
    fft_tile_call<N, TW, TW, NT, false, 1, TileLoad, Field>(buf, tw, TileLoad{}, f);
    fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(
        buf, tw, TileLoad{}, ColOut{moved(w_out, by) + base, geo.ra, geo.rb, N / 2 + 1 - c0});
  }
};

template <int N, int TW, int MODEL, bool TMA>
__global__ void __launch_bounds__(NT, blocks_for_smem(col_smem_tw(N, TW), N) < 2 ? 1 : 2) k_z_screen_field(OpZScreenField<N, TW, MODEL> op,
                                                       const float2* __restrict__ twg,
                                                       int64_t ntiles, const __grid_constant__ CUtensorMap map) {
  if (!op.geo.m.shift) resolve(op.fp, 0);  // one simulation: once per launch
  if constexpr (TMA) col_pipeline_tma<N, fft_rows<N>() * TW, false, 0>(op, twg, ntiles, &map, nullptr);
  else col_pipeline<N, fft_rows<N>() * TW>(op, twg, ntiles);
}

// ---------------------------------------------------------------- force (z pass)
// Per tile: the source (S, or delta when unscreened) is staged and transformed
// forward while delta(k) lands in a second shared-memory tile (screened runs);
// Phi_tot(k) is formed from both and kept in that second tile, and the two
// outputs (Phi and -i kz Phi) are inverse transformed one after the other in
// the staging buffer and stored to HBM.
template <int N, int TW, bool SCREENED>
struct OpZForce {
  // One CTA per SM (N >= 512, up to 255 registers): Phi_tot(k) is formed in the
  // forward transform's last store; with two CTAs (128 registers) that spills,
  // and a separate pass over the tile forms it instead.
  static constexpr bool FUSED = blocks_for_smem(col_smem_tw(N, TW) + (size_t)N * TW * 8, N) < 2;
  // Store hook of the forward transform of S: Phi_tot(k) (App. B), written to
  // the buffer for the Phi inverse and to `ph` (which held delta(k)) for the
  // gradient; ready() waits for this tile's delta(k) between the two steps.
  struct Combine {
    static constexpr bool kSmem = true;
    float2* ph;
    int c0, fy2;
    float kf2, a2m2, kappa_norm, C;
    __device__ __forceinline__ float2 operator()(float2 src, int n, int c, int at) const {
      const int fx = c0 + c, fz = freq_index(n, N);
      const float k2 = kf2 * (float)(fx * fx + fy2 + fz * fz);
      float2 phi = make_float2(0.f, 0.f);
      if (k2 > 0.f) {
        const float yuk = __fdividef(k2, k2 + a2m2);
        const float g = __fdividef(-kappa_norm, k2);
        if (SCREENED) phi = cscale(cadd(ph[at], cscale(src, C * yuk)), g);
        else phi = cscale(src, g * (1.f + C * yuk));
      }
      ph[at] = phi;
      return phi;
    }
    TmaSide side;  // TMA staging: the barrier of delta(k)'s copy
    __device__ __forceinline__ void ready() const {
      if (!SCREENED) return;
      if (side.bar) side.wait();  // thread 0; the transform's next barrier publishes the tile
      else cp_async_wait<1>();    // delta(k); the next tile's prefetch may stay in flight
    }
  };
  // Load hook of the gradient transform: -i kz Phi_tot(k), zero on the Nyquist row.
  struct GradZ {
    const float2* ph;
    float mkf;
    __device__ __forceinline__ float2 operator()(const float2*, int n, int, int at) const {
      const float kzs = (n == N / 2) ? 0.f : mkf * (float)freq_index(n, N);
      return cscale(cmul_i(ph[at]), kzs);
    }
  };
  ColGeo<N, TW> geo;
  const float2 *in, *dk;
  float2 *phi_out, *phiz_out;
  ForceParams fp;
  float2* extra = nullptr;  // scratch after the stage buffers (set by col_pipeline)
  TmaSide side;             // set per tile by col_pipeline_tma
  __device__ __forceinline__ void issue(float2* buf, int64_t t) const {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    col_issue<N, TW, TW>(buf, 0, moved(in, by), base, geo.ra, geo.rb, c0);
  }
  // delta(k) of the tile into extra; lands while S is transformed
  __device__ __forceinline__ void issue_side(int64_t t) const {
    if (SCREENED) {
      int o, c0;
      int64_t base, by;
      geo.tile(t, o, c0, base, by);
      col_issue<N, TW, TW>(extra, 0, moved(dk, by), base, geo.ra, geo.rb, c0);
    }
  }
  __device__ __forceinline__ void process(float2* buf, const float2* tw, int64_t t) const {
    int iy, c0;
    int64_t base, by;
    geo.tile(t, iy, c0, base, by);
    ForceParams fp = this->fp;
    resolve(fp, by);
    float2* ph = extra;  // delta(k) of the tile, then Phi_tot(k), N x TW
    const int fy = freq_index(iy, N);
    const Combine cmb{ph, c0, fy * fy, fp.kf * fp.kf, fp.a2m2, fp.kappa_norm, fp.C, side};
    if constexpr (FUSED) {
      fft_tile_call<N, TW, TW, NT, false, 1, TileLoad, Combine>(buf, tw, TileLoad{}, cmb);
    } else {
      fft_tile_call<N, TW, TW, NT, false>(buf, tw);
      cmb.ready();
      __syncthreads();
      const TileLane<N, TW> ln(c0, iy);
#pragma unroll 4
      for (int i = 0; i < ln.E; ++i) {
        const int n = ln.row(i), at = n * TW + ln.c;
        buf[at] = cmb(buf[at], n, ln.c, at);
      }
      __syncthreads();
    }
    const GradZ grad{ph, -fp.kf};
    if constexpr (FUSED) {
      // both inverse transforms store straight to HBM; the gradient transform
      // reads ph, not the tile
      const ColOut o{nullptr, geo.ra, geo.rb, N / 2 + 1 - c0};
      ColOut op = o, oz = o;
      op.g = moved(phi_out, by) + base;
      oz.g = moved(phiz_out, by) + base;
      fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(buf, tw, TileLoad{}, op);
      fft_tile_call<N, TW, TW, NT, true, 1, GradZ, ColOut>(buf, tw, grad, oz);
    } else {
      const ColOut o{nullptr, geo.ra, geo.rb, N / 2 + 1 - c0};
      ColOut op = o, oz = o;
      op.g = moved(phi_out, by) + base;
      oz.g = moved(phiz_out, by) + base;
      fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(buf, tw, TileLoad{}, op);
      const TileLane<N, TW> ln(c0, iy);
#pragma unroll 4
      for (int i = 0; i < ln.E; ++i) {
        const int n = ln.row(i), at = n * TW + ln.c;
        buf[at] = grad(buf, n, ln.c, at);
      }
      __syncthreads();
      fft_tile_call<N, TW, TW, NT, true, 1, TileLoad, ColOut>(buf, tw, TileLoad{}, oz);
    }
  }
};

template <int N, int TW, bool SCREENED, bool TMA>
__global__ void __launch_bounds__(NT, blocks_for_smem(col_smem_tw(N, TW) + (size_t)N * TW * 8, N) < 2 ? 1 : 2) k_z_force(
    OpZForce<N, TW, SCREENED> op, const float2* __restrict__ twg, int64_t ntiles,
    const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap) {
  if (!op.geo.m.shift) resolve(op.fp, 0);  // one simulation: once per launch
  if constexpr (TMA) col_pipeline_tma<N, fft_rows<N>() * TW, SCREENED, N * TW>(op, twg, ntiles, &map, &dmap);
  else col_pipeline<N, fft_rows<N>() * TW>(op, twg, ntiles);
}

// ---------------------------------------------------------------- LPT reweight (z pass)
template <int PREC>
__device__ __forceinline__ float2 dequant(uint32_t w, float scale) {
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

template <int N, int TW, int PREC>
struct OpLptZ {
  ColGeo<N, TW> geo;
  const void *phi1, *phi2;
  float2 *o0, *o1, *o2, *o3;
  LptParams lp;
  int tab_smem;             // 1: the (single) table row is staged in extra once per CTA
  // zero fill riding on this issue-bound pass: each tile clears its share (zchunk bytes)
  // of zdst (zbytes per simulation, moved by the simulation's shift), by bulk stores
  // from a zeroed 16 KB region after the table row; nullptr: none
  char* zdst = nullptr;
  int64_t zbytes = 0, zchunk = 0;
  float2* extra = nullptr;  // scratch after the stage buffers (set by col_pipeline)
  static constexpr uint32_t kZero = 16384;
  __device__ __forceinline__ void issue_side(int64_t) const {}
  __device__ __forceinline__ void issue(float2* buf, int64_t t) const {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    if constexpr (PREC == 0) {
      col_issue<N, TW, 4 * TW>(buf, 0, moved(static_cast<const float2*>(phi1), by), base, geo.ra, geo.rb, c0);
      col_issue<N, TW, 4 * TW>(buf, 1, moved(static_cast<const float2*>(phi2), by), base, geo.ra, geo.rb, c0);
    } else {
      // raw 16-bit pairs staged in the (still unused) output sub-blocks 2 and 3
      uint32_t* rb = reinterpret_cast<uint32_t*>(buf);
      col_issue_raw<N, TW>(rb, 0, moved(static_cast<const uint32_t*>(phi1), by), base, geo.ra, geo.rb, c0);
      col_issue_raw<N, TW>(rb, 1, moved(static_cast<const uint32_t*>(phi2), by), base, geo.ra, geo.rb, c0);
    }
  }
  __device__ __forceinline__ void process(float2* buf, const float2* tw, int64_t t) const {
    constexpr int TP = 4 * TW;
    int iy, c0;
    int64_t base, by;
    geo.tile(t, iy, c0, base, by);
    LptParams lp = this->lp;
    resolve(lp, by);  // no-op when resolved once for the launch
    const float4* tab = lp.row;
    if (tab_smem) {
      float4* st = reinterpret_cast<float4*>(extra);
      if (t == blockIdx.x) {  // this CTA's first tile: stage the row
        for (int i = threadIdx.x; i < lp.nk; i += NT) st[i] = tab[i];
        __syncthreads();
      }
      tab = st;
    }
    if (zdst) {
      float4* zr = reinterpret_cast<float4*>(extra) + (tab_smem ? lp.nk : 0);
      if (t == blockIdx.x) {  // first tile: zero the region for the async proxy
        for (int i = threadIdx.x; i < (int)(kZero / 16); i += NT) zr[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        fence_async_smem();
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        const int64_t tps = ColGeo<N, TW>::tps, tl = t % tps;
        const int64_t a = tl * zchunk, b = a + zchunk < zbytes ? a + zchunk : zbytes;
        if (a < b) bulk_zero(moved(zdst, by) + a, b - a, zr, kZero);
      }
    }
    if constexpr (PREC != 0) {
      const uint32_t* rb = reinterpret_cast<const uint32_t*>(buf);
      const float sc1 = lp.scale[0], sc2 = lp.scale[1];
      for (int e = threadIdx.x; e < N * TW; e += NT) {
        const int c = e % TW, n = e / TW;
        const float2 a = dequant<PREC>(rb[8 * n * TW + 4 * TW + c], sc1);
        const float2 b = dequant<PREC>(rb[8 * n * TW + 5 * TW + c], sc2);
        buf[n * TP + c] = a;
        buf[n * TP + TW + c] = b;
      }
      __syncthreads();  // the raw staging (sub-blocks 2, 3) is consumed
    }
    const TileLane<N, TW> ln(c0, iy);
    const float kf2 = lp.kf * lp.kf;
    const int c = ln.c;
#pragma unroll 2
    for (int i = 0; i < ln.E; ++i) {
      const int n = ln.row(i);
      const float k2 = ln.k2(n, kf2);
      float2 d = make_float2(0.f, 0.f), A = make_float2(0.f, 0.f);
      if (k2 > 0.f) {
        const float u = (0.5f * __logf(k2) - lp.lnk0) * lp.inv_dlnk;
        int i0 = (int)floorf(u);
        i0 = min(max(i0, 0), lp.nk - 2);
        const float f = u - (float)i0;
        const float4 t0 = tab[i0], t1 = tab[i0 + 1];
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
    col_store<N, TW, TP>(buf, 0, moved(o0, by), base, geo.ra, geo.rb, c0);
    col_store<N, TW, TP>(buf, 1, moved(o1, by), base, geo.ra, geo.rb, c0);
    col_store<N, TW, TP>(buf, 2, moved(o2, by), base, geo.ra, geo.rb, c0);
    col_store<N, TW, TP>(buf, 3, moved(o3, by), base, geo.ra, geo.rb, c0);
  }
};

template <int N, int TW, int PREC>
__global__ void __launch_bounds__(NT, blocks_for_smem(col_smem_c(N, 4), N)) k_lpt_z(OpLptZ<N, TW, PREC> op,
                                              const float2* __restrict__ twg, int64_t ntiles) {
  if (!op.geo.m.shift) resolve(op.lp, 0);  // one simulation: once per launch
  col_pipeline<N, fft_rows<N>() * 4 * TW>(op, twg, ntiles);
  if (op.zdst && threadIdx.x == 0) bulk_store_drain();  // the zero fill completes with the kernel
}

// The LPT z pass with 8-column tiles (N = 256, 512), where four 4-column
// output arrays would otherwise fill shared memory: an 8-column tile reads and
// writes whole 128-byte plane-pair pieces of the interleaved layout (4-column
// tiles move 32-byte halves of them).  Shared memory: two input buffers
// (phi1 in columns 0..7, phi2 in 8..15; double-buffered) and one work buffer
// that first holds (d, i kz d) and then (A, i kz A), each pair inverse
// transformed as one 16-column tile whose outputs leave for HBM from the last
// step's registers.  The table row is read through L1.  16-bit seeds are
// staged raw (phi1 words 0..7, phi2 words 8..15 of each 32-word row) and
// dequantised as the work pairs are formed.
template <int N, int PREC>
struct LptZ8 {
  static constexpr int TW = 8, TP = 16, ROWS = fft_rows<N>(), BUF = ROWS * TP;
  static constexpr size_t smem = (N + 3 * (size_t)BUF) * sizeof(float2);
};

// Store hook: columns c < 8 to ga, 8..15 to gb (columns c0 + c < N/2 + 1 exist).
struct PairColOut {
  static constexpr bool kSmem = false;
  float2 *ga, *gb;
  int64_t ra, rb;
  int live;
  __device__ __forceinline__ float2 operator()(float2 v, int n, int c, int) const {
    const bool b = c >= 8;
    const int cc = b ? c - 8 : c;
    if (cc < live) (b ? gb : ga)[(n >> 1) * ra + (n & 1) * rb + hcol(cc)] = v;
    return v;
  }
  __device__ __forceinline__ void ready() const {}
};

// 16-bit seeds of one field, raw, into words f*8 .. f*8+7 of each 32-word staged row.
template <int N>
__device__ __forceinline__ void col_issue_raw8(uint32_t* sb, int f, const uint32_t* __restrict__ g, int64_t base,
                                               int64_t ra, int64_t rb, int c0) {
  constexpr int STEP = NT / 2;  // two 16-byte pieces (8 words) per row and field
  const int j = threadIdx.x & 1, n0 = threadIdx.x >> 1;
  const bool v = c0 + 4 * j < N / 2 + 1;
  const uint32_t* src = g + base + (n0 >> 1) * ra + (n0 & 1) * rb + hcol(4 * j);
  uint32_t* dst = sb + n0 * 32 + f * 8 + 4 * j;
#pragma unroll 4
  for (int n = n0; n < N; n += STEP) {
    cp_async16(dst, v ? (const void*)src : (const void*)g, v);
    src += (STEP / 2) * ra;
    dst += STEP * 32;
  }
}

template <int N, int PREC>
__global__ void __launch_bounds__(NT, 1) k_lpt_z8(ColGeo<N, 8> geo, const void* __restrict__ phi1,
                                                   const void* __restrict__ phi2, float2* __restrict__ o0,
                                                   float2* __restrict__ o1, float2* __restrict__ o2,
                                                   float2* __restrict__ o3, LptParams lp0,
                                                   const float2* __restrict__ twg, int64_t ntiles) {
  using C = LptZ8<N, PREC>;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* const S0 = sm + N;
  float2* const S1 = sm + N + C::BUF;
  float2* const W = sm + N + 2 * C::BUF;
  load_tw(tw, twg, N);
  auto issue = [&](float2* buf, int64_t t) {
    int o, c0;
    int64_t base, by;
    geo.tile(t, o, c0, base, by);
    if constexpr (PREC == 0) {
      col_issue<N, 8, 16>(buf, 0, moved(static_cast<const float2*>(phi1), by), base, geo.ra, geo.rb, c0);
      col_issue<N, 8, 16>(buf, 1, moved(static_cast<const float2*>(phi2), by), base, geo.ra, geo.rb, c0);
    } else {
      uint32_t* sb = reinterpret_cast<uint32_t*>(buf);
      col_issue_raw8<N>(sb, 0, moved(static_cast<const uint32_t*>(phi1), by), base, geo.ra, geo.rb, c0);
      col_issue_raw8<N>(sb, 1, moved(static_cast<const uint32_t*>(phi2), by), base, geo.ra, geo.rb, c0);
    }
  };
  if (!geo.m.shift) resolve(lp0, 0);  // one simulation: once per launch
  int64_t t = blockIdx.x;
  if (t < ntiles) issue(S0, t);
  cp_async_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) issue(cur ? S0 : S1, tn);
    cp_async_commit();
    cp_async_wait<1>();  // tile t's seeds have landed
    __syncthreads();
    int iy, c0;
    int64_t base, by;
    geo.tile(t, iy, c0, base, by);
    LptParams lp = lp0;
    resolve(lp, by);
    const float4* __restrict__ tab = lp.row;
    const float2* sb = cur ? S1 : S0;
    const TileLane<N, 8> ln(c0, iy);
    const float kf2 = lp.kf * lp.kf;
    const int c = ln.c;
    // pass 0: (d, i kz d) with (c1, c2); pass 1: (A, i kz A) with (e1, e2)
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 2
      for (int i = 0; i < ln.E; ++i) {
        const int n = ln.row(i);
        const float k2 = ln.k2(n, kf2);
        float2 v = make_float2(0.f, 0.f);
        if (k2 > 0.f) {
          const float u = (0.5f * __logf(k2) - lp.lnk0) * lp.inv_dlnk;
          int i0 = (int)floorf(u);
          i0 = min(max(i0, 0), lp.nk - 2);
          const float f = u - (float)i0;
          const float4 t0 = __ldg(tab + i0), t1 = __ldg(tab + i0 + 1);
          const float a = pass == 0 ? t0.x * (1.f - f) + t1.x * f : t0.z * (1.f - f) + t1.z * f;
          const float b = pass == 0 ? t0.y * (1.f - f) + t1.y * f : t0.w * (1.f - f) + t1.w * f;
          float2 p1, p2;
          if constexpr (PREC == 0) {
            p1 = sb[n * 16 + c];
            p2 = sb[n * 16 + 8 + c];
          } else {
            const uint32_t* rb = reinterpret_cast<const uint32_t*>(sb);
            p1 = dequant<PREC>(rb[n * 32 + c], lp.scale[0]);
            p2 = dequant<PREC>(rb[n * 32 + 8 + c], lp.scale[1]);
          }
          v = cscale(cadd(cscale(p1, a), cscale(p2, b)), lp.norm);
        }
        const float kz = (n == N / 2) ? 0.f : lp.kf * (float)freq_index(n, N);
        W[n * 16 + c] = v;
        W[n * 16 + 8 + c] = cscale(cmul_i(v), kz);
      }
      __syncthreads();
      const PairColOut out{moved(pass == 0 ? o0 : o2, by) + base, moved(pass == 0 ? o1 : o3, by) + base, geo.ra,
                           geo.rb, N / 2 + 1 - c0};
      fft_tile_call<N, 16, 16, NT, true, 1, TileLoad, PairColOut>(W, tw, TileLoad{}, out);
    }
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- x passes (rows)
// A row tile holds TWX rows of the half-length complex transform (M = N/2)
// row-major in shared memory, row r at st[r * CW + k] (CW = rowtile_pitch<M>),
// exactly as cp.async staged them; the transform runs in place
// (fft_rowtile).  Tiles are double-buffered: the next tile is staged into the
// other buffer while the current one is transformed.
template <int N, int TWX>
struct RowCfg {
  static constexpr int M = N / 2;
  static constexpr int CW = rowtile_pitch<M>();    // complex values per staged row (>= M + 2)
  static constexpr size_t stage = (size_t)TWX * CW;  // float2 per buffer
  static constexpr size_t smem = (N + 2 * stage) * sizeof(float2);
};

// The rows of a row tile (first pair-major row q0, TWX even) are the pairs
// (z, y) and (z + 1, y) of TWX/2 consecutive y: in the half spectrum one
// contiguous block of TWX/2 interleaved row pairs (2P complex values each), in
// real space two blocks of TWX/2 consecutive rows (even tile rows from real row
// real_row_q(q0), odd ones from real_row_q(q0 + 1)).  Tile row r is staged at
// st[r * CW ...].
//
// Walk over the NPAIR row pairs of a tile in memory order, LEN positions per
// pair: warps take whole pairs, or split each pair into NW / NPAIR segments
// when there are fewer pairs than warps; f(pair, p0, p1) visits p = p0, p0 +
// 32, ... < p1 with p0 = segment start + lane (segment starts are multiples of
// 32, so each warp reads or writes whole lines).
template <int NPAIR, int LEN, class F>
__device__ __forceinline__ void for_pairs(F f) {
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (NPAIR >= NW) {
    for (int pr = warp; pr < NPAIR; pr += NW) f(pr, lane, LEN);
  } else {
    constexpr int S = NW / NPAIR;
    constexpr int SEG = (LEN + 32 * S - 1) / (32 * S) * 32;
    const int s = warp % S;
    f(warp / S, s * SEG + lane, (s + 1) * SEG < LEN ? (s + 1) * SEG : LEN);
  }
}

// Complex half rows (M + 1 values, staged as M + 2 to keep 16-byte pieces).
// Piece p of a row pair holds values 2p, 2p + 1 of the pair: row (p >> 2) & 1,
// columns k = (p >> 3) 8 + 2 (p & 3), k + 1; p + 32 is the same row, k + 32.
template <int N, int TWX>
__device__ __forceinline__ void stage_complex_rows(float2* st, const float2* __restrict__ in,
                                                   int64_t q0) {
  using C = RowCfg<N, TWX>;
  constexpr int P = (int)half_pitch(N);  // 16-byte pieces per row pair
  const float2* src = in + hrow_q(q0, P);
  for_pairs<TWX / 2, P>([&](int pr, int p0, int p1) {
    int k = (p0 >> 3) * 8 + 2 * (p0 & 3);
    float2* d = st + (2 * pr + ((p0 >> 2) & 1)) * C::CW + k;
    const float2* g = src + (int64_t)pr * 2 * P + 2 * p0;
    for (int p = p0; p < p1; p += 32, k += 32, d += 32, g += 64)
      if (k < C::M + 2) cp_async16(d, g, true);
  });
}

// A pair tile: TWX/4 row pairs of a and the same row pairs of b (first pair-major
// row q0), row pair i of a at tile rows 4i (plane z) and 4i + 2 (plane z + 1), of b
// at 4i + 1 and 4i + 3, so that tile rows 2w and 2w + 1 are the same real row of a
// and of b.
template <int N, int TWX>
__device__ __forceinline__ void stage_complex_rows_pair(float2* st, const float2* __restrict__ a,
                                                        const float2* __restrict__ b, int64_t q0) {
  using C = RowCfg<N, TWX>;
  constexpr int P = (int)half_pitch(N);
  const float2* srca = a + hrow_q(q0, P);
  const float2* srcb = b + hrow_q(q0, P);
  for_pairs<TWX / 2, P>([&](int pr, int p0, int p1) {
    const int job = pr & 1, i = pr >> 1;
    int k = (p0 >> 3) * 8 + 2 * (p0 & 3);
    float2* d = st + (4 * i + 2 * ((p0 >> 2) & 1) + job) * C::CW + k;
    const float2* g = (job ? srcb : srca) + (int64_t)i * 2 * P + 2 * p0;
    for (int p = p0; p < p1; p += 32, k += 32, d += 32, g += 64)
      if (k < C::M + 2) cp_async16(d, g, true);
  });
}

// real rows of N floats: row r at floats [pitch r, pitch r + N), i.e. the M
// complex values z[j] = x[2j] + i x[2j+1] at st[r * CW + j] when pitch = 2 CW
template <int N, int TWX>
__device__ __forceinline__ void stage_real_rows(float* st, const float* __restrict__ in, int64_t q0,
                                                int pitch_floats) {
  constexpr int CH = N / 4;           // 16-byte pieces per row
  constexpr int HALF = TWX / 2 * CH;  // pieces per block of one parity
  static_assert(HALF % NT == 0, "a parity block is whole iterations");
  const float* src0 = in + real_row_q(q0, N) * N;
  const float* src1 = in + real_row_q(q0 + 1, N) * N;
#pragma unroll
  for (int i = 0; i < 2 * HALF / NT; ++i) {
    const int h = i * NT / HALF;  // constant per iteration
    const int e2 = threadIdx.x + i * NT - h * HALF;
    cp_async16(st + (2 * (e2 / CH) + h) * pitch_floats + 4 * (e2 % CH), (h ? src1 : src0) + 4 * e2, true);
  }
}

// r2c post-processing: X[k] = (Z[k] + conj Z[M-k])/2 - i/2 w^k (Z[k] - conj Z[M-k]),
// written in memory order; position w of a row pair is row (w >> 3) & 1,
// column k = (w >> 4) 8 + (w & 7); w + 32 is the same row, k + 16.  Padding
// columns k > M are not written.
template <int N, int TWX>
__device__ __forceinline__ void row_r2c_store(const float2* buf, const float2* tw,
                                              float2* __restrict__ out, int64_t q0) {
  using C = RowCfg<N, TWX>;
  constexpr int M = N / 2;
  constexpr int P = (int)half_pitch(N);
  float2* dst = out + hrow_q(q0, P);
  for_pairs<TWX / 2, 2 * P>([&](int pr, int w0, int w1) {
    int k = (w0 >> 4) * 8 + (w0 & 7);
    const float2* z = buf + (2 * pr + ((w0 >> 3) & 1)) * C::CW;
    float2* o = dst + (int64_t)pr * 2 * P + w0;
#pragma unroll 2
    for (int w = w0; w < w1; w += 32, k += 16, o += 32) {
      if (k > M) continue;
      const float2 a = z[k & (M - 1)];
      const float2 b = cconj(z[(M - k) & (M - 1)]);
      const float2 E = cscale(cadd(a, b), 0.5f);
      const float2 D = csub(a, b);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // (-i/2) D
      *o = cadd(E, cmul(tw[k], O));
    }
  });
}

// The c2r input convention on a staged spectrum value X[k] (k = 0..M): the
// optional derivative i kfs k (zero at the Nyquist k = M), and the imaginary
// parts of X[0], X[M] dropped.
template <int M>
__device__ __forceinline__ float2 c2r_in(float2 x, int k, float kfs) {
  if (kfs != 0.f) x = (k == M) ? make_float2(0.f, 0.f) : cscale(cmul_i(x), kfs * (float)k);
  if (k == 0 || k == M) x.y = 0.f;
  return x;
}

// c2r pre-processing (unnormalised inverse, 2x folded in) as the first step of
// the inverse row transform loads element n of tile row r: with E = X[n] +
// conj X[M-n] and O = w^-n (X[n] - conj X[M-n]), Z[n] = E + i O.  The partner
// M - n is read from the staged row itself, which no thread overwrites before
// every load of that step is done (no separate pass over the tile).  Pitch CW.
template <int N, int CW>
struct C2rCombine {
  const float2* buf;
  const float2* tw;
  float kfs;
  __device__ __forceinline__ float2 operator()(float2 zn, int r, int n) const {
    constexpr int M = N / 2;
    const float2 a = c2r_in<M>(zn, n, kfs);
    const float2 b = cconj(c2r_in<M>(buf[r * CW + M - n], M - n, kfs));
    const float2 E = cadd(a, b);
    const float2 O = cmul(cconj(tw[n]), csub(a, b));
    return cadd(E, cmul_i(O));
  }
};

// Resident CTAs per SM for the plain row passes: 3 when three tiles fit in
// shared memory and the transform is short enough (<= 256 points) to stay in
// 85 registers, else 2.
template <int N, int TWX>
constexpr int row_blocks() {
  return (N <= 512 && RowCfg<N, TWX>::smem <= 74 * 1024) ? 3 : 2;
}

struct ScaleOffset {
  float scale, offset;
  __device__ __forceinline__ float2 operator()(float2 v, int, int) const {
    return make_float2(fmaf(v.x, scale, offset), fmaf(v.y, scale, offset));
  }
};

// Row tile t of a multi-simulation launch: simulation t / tps, first row (t mod tps) TWX
// in the pair-major row order q of the half-spectrum layout (TWX even).
struct RowTile {
  int64_t row0, by;
};
template <int N, int TWX>
__device__ __forceinline__ RowTile row_tile(int64_t t64, const Multi& m) {
  constexpr uint32_t TPS = (uint32_t)N * N / TWX;  // tiles per simulation
  const uint32_t t = (uint32_t)t64, b = t / TPS;     // t < 2^31 (checked by prep)
  return RowTile{(int64_t)(t - b * TPS) * TWX, shift_of(m, (int)b)};
}

// The real rows of row tile q0 into st by 1-D bulk copies (thread 0): tile row r
// (r even from real_row_q(q0), odd from real_row_q(q0 + 1)) at st + r * pitch floats.
template <int N, int TWX>
__device__ __forceinline__ void bulk_real_rows(float* st, const float* __restrict__ in, int64_t q0,
                                               int pitch_floats, uint64_t* bar) {
  bar_expect(bar, (uint32_t)(TWX * N * sizeof(float)));
  const float* src0 = in + real_row_q(q0, N) * N;
  const float* src1 = in + real_row_q(q0 + 1, N) * N;
#pragma unroll
  for (int r = 0; r < TWX; ++r)
    bulk_load(st + r * pitch_floats, ((r & 1) ? src1 : src0) + (r >> 1) * N, N * sizeof(float), bar);
}

template <int N, int TWX, bool BULK>
__global__ void __launch_bounds__(NT, row_blocks<N, TWX>()) k_xr2c(const float* __restrict__ in, float2* __restrict__ out,
                                                float scale, float offset,
                                                const float2* __restrict__ twg, int64_t ntiles,
                                                Multi m) {
  using C = RowCfg<N, TWX>;
  constexpr int M = N / 2;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* st0 = sm + N;
  float2* st1 = st0 + C::stage;
  if constexpr (BULK) {
    // one simulation: bulk-copy staging, one barrier per stage buffer (after the two buffers)
    uint64_t* bars = reinterpret_cast<uint64_t*>(st1 + C::stage);
    int& fail = *reinterpret_cast<int*>(bars + 2);
    const bool lead = threadIdx.x == 0;
    if (lead) {
      bar_init(&bars[0]);
      bar_init(&bars[1]);
      fence_bar_init();
      fail = 0;
    }
    load_tw(tw, twg, N);
    __syncthreads();
    uint32_t par = 0, pend = 0;
    int64_t t = blockIdx.x;
    if (lead && t < ntiles) {
      bulk_real_rows<N, TWX>(reinterpret_cast<float*>(st0), in, row_tile<N, TWX>(t, m).row0, 2 * C::CW, &bars[0]);
      pend |= 1u;
    }
    int cur = 0;
    for (; t < ntiles; t += gridDim.x) {
      if (lead) {
        fence_async_smem();
        const int64_t tn = t + gridDim.x;
        if (tn < ntiles) {
          bulk_real_rows<N, TWX>(reinterpret_cast<float*>(cur ? st0 : st1), in, row_tile<N, TWX>(tn, m).row0,
                                 2 * C::CW, &bars[cur ^ 1]);
          pend |= 1u << (cur ^ 1);
        }
        if (bar_wait(&bars[cur], (par >> cur) & 1u)) {
          par ^= 1u << cur;
          pend &= ~(1u << cur);
        } else {
          fail = 1;
        }
      }
      __syncthreads();
      if (fail) break;
      float2* buf = cur ? st1 : st0;
      fft_rowtile<M, TWX, C::CW, NT, false, 2>(buf, tw, ScaleOffset{scale, offset});
      row_r2c_store<N, TWX>(buf, tw, out, row_tile<N, TWX>(t, m).row0);
      __syncthreads();
      cur ^= 1;
    }
    if (lead && fail) {
      atomicAdd(&g_tile_load_failures, 1u);
      for (int i = 0; i < 2; ++i)
        if ((pend >> i) & 1u) bar_wait(&bars[i], (par >> i) & 1u);
    }
    return;
  }
  load_tw(tw, twg, N);
  int64_t t = blockIdx.x;
  if (t < ntiles) {
    const RowTile r = row_tile<N, TWX>(t, m);
    stage_real_rows<N, TWX>(reinterpret_cast<float*>(st0), moved(in, r.by), r.row0, 2 * C::CW);
  }
  cp_async_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) {
      const RowTile r = row_tile<N, TWX>(tn, m);
      stage_real_rows<N, TWX>(reinterpret_cast<float*>(cur ? st0 : st1), moved(in, r.by), r.row0, 2 * C::CW);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    float2* buf = cur ? st1 : st0;
    fft_rowtile<M, TWX, C::CW, NT, false, 2>(buf, tw, ScaleOffset{scale, offset});
    const RowTile r = row_tile<N, TWX>(t, m);
    row_r2c_store<N, TWX>(buf, tw, moved(out, r.by), r.row0);
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// Up to six independent row transforms per launch (job = tile / tiles_per_job).
struct RowJobs {
  const void* in[6];
  void* out[6];
  float kfs[6];
  int njobs;
  uint32_t jmul, jshift;  // q / njobs = (umulhi(q, jmul) + q) >> jshift for q < 2^31
  const SimHeader* hdr;   // 16-bit outputs: scales and absmax of each job (moved per simulation)
};

// Division by an invariant integer d >= 1 through a multiply-high (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI 1994):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (umulhi(n, m) + n) >> l,
// exact for every n < 2^31.
inline void fast_div_magic(uint32_t d, uint32_t& mul, uint32_t& shift) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  mul = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  shift = l;
}
__device__ __forceinline__ uint32_t fast_div(uint32_t n, uint32_t mul, uint32_t shift) {
  return (__umulhi(n, mul) + n) >> shift;
}

// Tile t of a multi-job, multi-simulation c2r launch: simulation, job, first row.
struct JobTile {
  int job;
  int64_t row0, by;
  uint32_t q;  // simulation * njobs + job
};
template <int N, int TWX>
__device__ __forceinline__ JobTile job_tile(int64_t t64, const RowJobs& jobs, const Multi& m) {
  constexpr uint32_t TPJ = (uint32_t)N * N / TWX;  // tiles per job
  const uint32_t t = (uint32_t)t64, q = t / TPJ;     // q = simulation * njobs + job
  const uint32_t b = fast_div(q, jobs.jmul, jobs.jshift);
  return JobTile{(int)(q - b * (uint32_t)jobs.njobs), (int64_t)(t - q * TPJ) * TWX, shift_of(m, (int)b), q};
}

// Store hook of the c2r row transform: tile row r's M complex outputs (2M
// reals) to real row r / 2 of the even (o0) or odd (o1) block.
template <int M>
struct RealRowOut {
  static constexpr bool kSmem = false;
  float2 *o0, *o1;
  __device__ __forceinline__ float2 operator()(float2 v, int r, int k) const {
    ((r & 1) ? o1 : o0)[(r >> 1) * M + k] = v;
    return v;
  }
};

// The same with 16-bit outputs (variant a.S1, the six per-step LPT fields):
// value / scale as bf16 (OUT 1) or fp16 (OUT 2, saturated at the largest
// finite value), two reals per 32-bit word; the largest |value| is kept in *amax.
template <int M, int OUT>
struct RealRowOut16 {
  static constexpr bool kSmem = false;
  uint32_t *o0, *o1;
  float inv;
  float* amax;
  __device__ __forceinline__ float2 operator()(float2 v, int r, int k) const {
    *amax = fmaxf(*amax, fmaxf(fabsf(v.x), fabsf(v.y)));
    float a = v.x * inv, b = v.y * inv;
    uint32_t w;
    if constexpr (OUT == 1) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      w = *reinterpret_cast<const uint32_t*>(&h);
    } else {
      a = fminf(fmaxf(a, -65504.f), 65504.f);
      b = fminf(fmaxf(b, -65504.f), 65504.f);
      const __half2 h = __floats2half2_rn(a, b);
      w = *reinterpret_cast<const uint32_t*>(&h);
    }
    ((r & 1) ? o1 : o0)[(r >> 1) * M + k] = w;
    return v;
  }
};

// Largest |value| of a job's tiles into hdr->lq_amax[job] (one atomic per warp).
__device__ __forceinline__ void amax_flush(const SimHeader* h, int job, float a) {
  const unsigned ua = __reduce_max_sync(0xffffffffu, __float_as_uint(a));
  if ((threadIdx.x & 31) == 0 && ua != 0u && h)
    atomicMax(reinterpret_cast<unsigned*>(const_cast<float*>(&h->lq_amax[job])), ua);
}

template <int N, int TWX, int OUT = 0>
__global__ void __launch_bounds__(NT, row_blocks<N, TWX>()) k_xc2r(const __grid_constant__ RowJobs jobs,
                                                const float2* __restrict__ twg, int64_t tiles_per_job,
                                                Multi m) {
  using C = RowCfg<N, TWX>;
  constexpr int M = N / 2;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* st0 = sm + N;
  float2* st1 = st0 + C::stage;
  load_tw(tw, twg, N);
  const int64_t ntiles = tiles_per_job * jobs.njobs * m.nb;
  int64_t t = blockIdx.x;
  if (t < ntiles) {
    const JobTile j = job_tile<N, TWX>(t, jobs, m);
    stage_complex_rows<N, TWX>(st0, moved(static_cast<const float2*>(jobs.in[j.job]), j.by), j.row0);
  }
  cp_async_commit();
  int cur = 0;
  // 16-bit outputs: running |value| maximum of the current (simulation, job)
  float run_max = 0.f;
  uint32_t run_q = 0xffffffffu;
  const SimHeader* run_h = nullptr;
  int run_job = 0;
  for (; t < ntiles; t += gridDim.x) {
    const JobTile j = job_tile<N, TWX>(t, jobs, m);
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) {
      const JobTile jn = job_tile<N, TWX>(tn, jobs, m);
      stage_complex_rows<N, TWX>(cur ? st0 : st1, moved(static_cast<const float2*>(jobs.in[jn.job]), jn.by),
                                 jn.row0);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    float2* buf = cur ? st1 : st0;
    // the c2r pre-processing rides on the transform's first loads
    using Pre = C2rCombine<N, C::CW>;
    const Pre pre{buf, tw, jobs.kfs[j.job]};
    // even tile rows go to one block of consecutive real rows, odd ones to
    // another, straight from the transform's last step
    if constexpr (OUT == 0) {
      float* out = moved(static_cast<float*>(jobs.out[j.job]), j.by);
      const RealRowOut<M> o{reinterpret_cast<float2*>(out + real_row_q(j.row0, N) * N),
                            reinterpret_cast<float2*>(out + real_row_q(j.row0 + 1, N) * N)};
      fft_rowtile<M, TWX, C::CW, NT, true, 2, Pre, false, RealRowOut<M>>(buf, tw, pre, o);
    } else {
      const SimHeader* h = moved(jobs.hdr, j.by);
      if (j.q != run_q) {  // the same for every thread of the CTA
        amax_flush(run_h, run_job, run_max);
        run_max = 0.f;
        run_q = j.q;
        run_h = h;
        run_job = j.job;
      }
      uint32_t* out = moved(static_cast<uint32_t*>(jobs.out[j.job]), j.by);
      float tile_max = 0.f;
      const RealRowOut16<M, OUT> o{out + real_row_q(j.row0, N) * M, out + real_row_q(j.row0 + 1, N) * M,
                                   1.f / h->lq_scale[j.job], &tile_max};
      fft_rowtile<M, TWX, C::CW, NT, true, 2, Pre, false, RealRowOut16<M, OUT>>(buf, tw, pre, o);
      run_max = fmaxf(run_max, tile_max);
    }
    __syncthreads();
    cur ^= 1;
  }
  if constexpr (OUT != 0) amax_flush(run_h, run_job, run_max);
  cp_async_wait<0>();
}

// C2rCombine with the x-derivative factor of even tile rows (kfs) and of odd
// ones (kfs1): a pair tile's rows of a and of b.
template <int N, int CW>
struct C2rCombine2 {
  const float2* buf;
  const float2* tw;
  float kfs, kfs1;
  __device__ __forceinline__ float2 operator()(float2 zn, int r, int n) const {
    return C2rCombine<N, CW>{buf, tw, (r & 1) ? kfs1 : kfs}(zn, r, n);
  }
};

// Store hook of a pair tile's c2r: the last transform step leaves output k of
// tile rows 2w (a) and 2w + 1 (b) in lanes l and l ^ R1 of one warp (R1 = the
// first-step radix, the outputs per row and lane group of that step); one
// shuffle gives lane l (a) the pair (a, b) of real 2k and lane l ^ R1 (b) that
// of real 2k + 1, and each writes one 8-byte pair, so a warp's stores cover
// consecutive cells.  o0 / o1: cell 0 of the first real row of planes z / z + 1.
template <int N, int R1>
struct PairRowOut {
  static constexpr bool kSmem = false;
  float2 *o0, *o1;
  __device__ __forceinline__ float2 operator()(float2 v, int r, int k) const {
    const int isb = r & 1;
    const float recv = __shfl_xor_sync(0xffffffffu, isb ? v.x : v.y, R1);
    float2* row = (((r >> 1) & 1) ? o1 : o0) + (int64_t)(r >> 2) * N;
    // one store instruction for the warp: cell 2k (a lanes) or 2k + 1 (b lanes)
    row[2 * k + isb] = isb ? make_float2(recv, v.y) : make_float2(v.x, recv);
    return v;
  }
};

// c2r of the rows of a (x derivative i kfs kx on load) and of b into the (x, y)
// pairs of one interleaved real field (App. B: F_x and F_y of the force mesh),
// pair tiles of TWX/4 row pairs of each.
template <int N, int TWX>
__global__ void __launch_bounds__(NT, row_blocks<N, TWX>()) k_xc2r_pair(
    const float2* __restrict__ a, const float2* __restrict__ b, float2* __restrict__ out, float kfs,
    const float2* __restrict__ twg, int64_t tiles_per_sim, Multi m) {
  using C = RowCfg<N, TWX>;
  constexpr int M = N / 2, R1 = Split<M>::R1;
  static_assert(R1 < 32 && TWX * R1 % 32 == 0, "pair lanes within whole warps");
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* st0 = sm + N;
  float2* st1 = st0 + C::stage;
  load_tw(tw, twg, N);
  const int64_t ntiles = tiles_per_sim * m.nb;
  auto tile = [&](int64_t t, int64_t& q0, int64_t& by) {
    const int64_t s = t / tiles_per_sim;
    q0 = (t - s * tiles_per_sim) * (TWX / 2);
    by = shift_of(m, (int)s);
  };
  int64_t t = blockIdx.x;
  if (t < ntiles) {
    int64_t q0, by;
    tile(t, q0, by);
    stage_complex_rows_pair<N, TWX>(st0, moved(a, by), moved(b, by), q0);
  }
  cp_async_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    int64_t q0, by;
    tile(t, q0, by);
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) {
      int64_t qn, bn;
      tile(tn, qn, bn);
      stage_complex_rows_pair<N, TWX>(cur ? st0 : st1, moved(a, bn), moved(b, bn), qn);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    float2* buf = cur ? st1 : st0;
    float2* o = moved(out, by);
    const PairRowOut<N, R1> st{o + real_row_q(q0, N) * N, o + real_row_q(q0 + 1, N) * N};
    fft_rowtile<M, TWX, C::CW, NT, true, 2, C2rCombine2<N, C::CW>, false, PairRowOut<N, R1>>(
        buf, tw, C2rCombine2<N, C::CW>{buf, tw, kfs, 0.f}, st);
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// Screening factor eps(w) (Sec. 6.1, Sec. 6.2).  The divisions and the square
// root use the fast intrinsics (a few ulp), well below the FP32 rounding of
// the transforms the factor feeds.
// p: f(R) the threshold fr_thr on |Phi_N|; nDGP the coefficient dgp_coef.
template <int MODEL>
__device__ __forceinline__ float screen_eps(float w, float p) {
  if (MODEL == 1) {
    const float aw = fabsf(w);
    return aw > p ? __fdividef(p, aw) : 1.f;
  } else {
    const float u = 1.f + p * fmaxf(1.f + w, 0.f);  // >= 1
    return __fdividef(2.f, u * rsqrtf(u) + 1.f);
  }
}

// Load hook of the forward transform of a screening pass: element j of tile row
// r is S = delta eps(w), w the screening field (the tile value) and delta =
// rho / rho_bar - 1 from consecutive density rows in global memory (M float2
// per row, read-only path); used by the plane pass.
template <int M, int MODEL>
struct ScreenSource {
  const float2* rho;
  float inv_rhobar, p;
  __device__ __forceinline__ float2 operator()(float2 w, int r, int j) const {
    const float2 rv = __ldg(rho + r * M + j);
    const float d0 = rv.x * inv_rhobar - 1.f, d1 = rv.y * inv_rhobar - 1.f;
    return make_float2(d0 * screen_eps<MODEL>(w.x, p), d1 * screen_eps<MODEL>(w.y, p));
  }
};

// The same for an x-pass row tile, whose even rows are consecutive density rows
// from `even` and odd rows from `odd`: each warp's loads of one transform step
// cover 32 consecutive values of a row.
template <int M, int MODEL>
struct ScreenSourceRows {
  const float2* even;
  const float2* odd;
  float inv_rhobar, p;
  __device__ __forceinline__ float2 operator()(float2 w, int r, int j) const {
    const float2 rv = __ldg((r & 1 ? odd : even) + (r >> 1) * M + j);
    const float d0 = rv.x * inv_rhobar - 1.f, d1 = rv.y * inv_rhobar - 1.f;
    return make_float2(d0 * screen_eps<MODEL>(w.x, p), d1 * screen_eps<MODEL>(w.y, p));
  }
};

// Screening source S = delta eps: c2r of the screening field rows, eps from the
// field and delta from rho (read from global memory by the forward transform's
// loads), r2c.  Shared memory: twiddles, two row tiles (double-buffered field rows).
template <int N, int TWX>
constexpr size_t xscreen_smem() {
  return RowCfg<N, TWX>::smem;
}

template <int N, int TWX, int MODEL>
__global__ void __launch_bounds__(NT, 2) k_x_screen(const float2* __restrict__ w_in,
                                                    const float* __restrict__ rho,
                                                    float2* __restrict__ s_out,
                                                    ForceParams fp0, const float2* __restrict__ twg,
                                                    int64_t ntiles, Multi m) {
  if (!m.shift) resolve(fp0, 0);  // one simulation: once per launch
  using C = RowCfg<N, TWX>;
  constexpr int M = N / 2;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* st0 = sm + N;
  float2* st1 = st0 + C::stage;
  load_tw(tw, twg, N);
  int64_t t = blockIdx.x;
  if (t < ntiles) {
    const RowTile r = row_tile<N, TWX>(t, m);
    stage_complex_rows<N, TWX>(st0, moved(w_in, r.by), r.row0);
  }
  cp_async_commit();
  int cur = 0;
  for (; t < ntiles; t += gridDim.x) {
    const RowTile r = row_tile<N, TWX>(t, m);
    const int64_t row0 = r.row0;
    ForceParams fp = fp0;
    resolve(fp, r.by);
    const int64_t tn = t + gridDim.x;
    float2* buf = cur ? st1 : st0;
    cp_async_wait<0>();  // w rows of this tile (the only group in flight)
    __syncthreads();
    // the next tile's w rows into the other buffer land while this tile is transformed
    if (tn < ntiles) {
      const RowTile rn = row_tile<N, TWX>(tn, m);
      stage_complex_rows<N, TWX>(cur ? st0 : st1, moved(w_in, rn.by), rn.row0);
    }
    cp_async_commit();
    fft_rowtile_call<M, TWX, C::CW, NT, true, 2, C2rCombine<N, C::CW>, true>(buf, tw,
                                                                           C2rCombine<N, C::CW>{buf, tw, 0.f});
    // S = delta eps(w) is formed as the forward transform loads it
    const float* rho_t = moved(rho, r.by);
    const ScreenSourceRows<M, MODEL> src{reinterpret_cast<const float2*>(rho_t + real_row_q(row0, N) * N),
                                         reinterpret_cast<const float2*>(rho_t + real_row_q(row0 + 1, N) * N),
                                         fp.inv_rhobar, MODEL == 1 ? fp.fr_thr : fp.dgp_coef};
    fft_rowtile_call<M, TWX, C::CW, NT, false, 2, ScreenSourceRows<M, MODEL>, true>(buf, tw, src);
    row_r2c_store<N, TWX>(buf, tw, moved(s_out, r.by), row0);
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- plane passes (N <= 128)
// Up to 128 points a whole z-plane of the half spectrum (N rows of M + 1 = N/2 + 1
// values) fits in one CTA's shared memory, so the x and y steps of a 3-D
// transform run as one pass over HBM: one CTA per plane (and simulation) stages
// the plane, transforms its rows and then its columns in place, and writes it
// back; the intermediate between the x and y steps never leaves the SM.  The
// plane's rows have the row-transform pitch CW (>= M + R2 - 1, 8 mod 16, so the
// row steps are conflict-free) and the column transforms run on chunks of
// TWCOL columns at that pitch, with the padding rows of their intermediate
// below the plane.
template <int N>
struct PlaneCfg {
  static constexpr int M = N / 2;
  static constexpr int CW = rowtile_pitch<M>();
  static constexpr int ROWS = fft_rows<N>();
  static constexpr int TWCOL = N == 128 ? 24 : CW;  // column chunk (a multiple of 8, CW = 3 x 24 at N = 128)
  static constexpr size_t buf = (size_t)ROWS * CW;   // float2
  static constexpr size_t smem = ((size_t)N + buf) * sizeof(float2);
  static_assert(CW >= M + 1 && CW % 8 == 0 && CW % TWCOL == 0 && TWCOL % 8 == 0, "plane pitch");
};

// The N real rows of a plane (N floats each) as M complex values per row at pitch CW.
template <int N>
__device__ __forceinline__ void stage_real_plane(float2* buf, const float* __restrict__ src) {
  constexpr int CH = N / 4, CW = PlaneCfg<N>::CW;  // 16-byte pieces per row
  for (int e = threadIdx.x; e < N * CH; e += NT) {
    const int y = e / CH, p = e - y * CH;
    cp_async16(reinterpret_cast<float*>(buf + y * CW) + 4 * p, src + (int64_t)y * N + 4 * p, true);
  }
}

// r2c split of every plane row in place (the split of row_r2c_store): from the
// packed transform Z of row r, X[k] = (Z[k] + conj Z[M-k])/2 - i/2 w^k (Z[k] - conj Z[M-k])
// for k = 0..M; a thread takes the pair (k, M - k) (k = 0: X[0] and X[M] from Z[0]).
template <int N>
__device__ __forceinline__ void plane_r2c_split(float2* buf, const float2* tw) {
  constexpr int M = N / 2, CW = PlaneCfg<N>::CW, H = M / 2 + 1;
  auto X = [&](float2 a, float2 bz, float2 w) {
    const float2 b = cconj(bz);
    const float2 E = cscale(cadd(a, b), 0.5f), D = csub(a, b);
    return cadd(E, cmul(w, make_float2(0.5f * D.y, -0.5f * D.x)));
  };
  for (int e = threadIdx.x; e < N * H; e += NT) {
    const int r = e / H, k = e - r * H;
    float2* z = buf + r * CW;
    const float2 zk = z[k], zm = z[(M - k) & (M - 1)];
    const float2 xk = X(zk, zm, tw[k]), xm = X(zm, zk, tw[M - k]);
    z[k] = xk;
    if (k != M - k) z[M - k] = xm;
  }
  __syncthreads();
}

// Forward x (r2c, input scaled then offset) and y transforms of plane blockIdx.x of a
// real N^3 field into the interleaved half spectrum (the z pass follows separately).
template <int N>
__global__ void __launch_bounds__(NT) k_plane_r2c(const float* __restrict__ in, float2* __restrict__ out,
                                                  float scale, float offset, const float2* __restrict__ twg,
                                                  Multi m) {
  using C = PlaneCfg<N>;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  const int z = blockIdx.x;
  const int64_t by = shift_of(m, blockIdx.y);
  load_tw(tw, twg, N);
  stage_real_plane<N>(buf, moved(in, by) + (int64_t)z * N * N);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  fft_rowtile<C::M, N, C::CW, NT, false, 2>(buf, tw, ScaleOffset{scale, offset});
  plane_r2c_split<N>(buf, tw);
  constexpr int64_t P = half_pitch(N);
  float2* g = moved(out, by) + hrow(z, 0, N, P);
#pragma unroll 1
  for (int c0 = 0; c0 < C::CW; c0 += C::TWCOL)
    fft_tile<N, C::TWCOL, C::CW, NT, false, 1, TileLoad, ColOut>(
        buf + c0, tw, TileLoad{}, ColOut{g + hcol(c0), 4 * P, 2 * P, C::M + 1 - c0});
}

// Store hook of a plane's row transforms: real row r (M float2 = N reals) to g + r M.
template <int M>
struct PlaneRowOut {
  static constexpr bool kSmem = false;
  float2* g;
  __device__ __forceinline__ float2 operator()(float2 v, int r, int k) const {
    g[r * M + k] = v;
    return v;
  }
};

// The N complex rows (ky) of plane z of an interleaved half spectrum into buf (pitch CW).
template <int N>
__device__ __forceinline__ void stage_complex_plane(float2* buf, const float2* __restrict__ g, int z) {
  constexpr int M = N / 2, CW = PlaneCfg<N>::CW;
  constexpr int64_t P = half_pitch(N);
  constexpr int CH = (M + 2) / 2;  // 16-byte pieces per row (kx = 0..M, staged as M + 2)
  const float2* src = g + hrow(z, 0, N, P);
  for (int e = threadIdx.x; e < N * CH; e += NT) {
    const int y = e / CH, p = e - y * CH, kx = 2 * p;
    cp_async16(buf + y * CW + kx, src + (int64_t)y * 2 * P + hcol(kx), true);
  }
}

// y inverse of every column chunk of plane a, in place.
template <int N>
__device__ __forceinline__ void plane_yinv(float2* a, const float2* tw) {
  using C = PlaneCfg<N>;
#pragma unroll 1
  for (int c0 = 0; c0 < C::CW; c0 += C::TWCOL) fft_tile<N, C::TWCOL, C::CW, NT, true>(a + c0, tw);
}

// c2r of the N rows of plane buffer a (x derivative i kfs kx applied on load when
// kfs != 0) to the real plane at g (N x N floats).
template <int N>
__device__ __forceinline__ void plane_xc2r(float2* a, const float2* tw, float kfs, float* g) {
  using C = PlaneCfg<N>;
  fft_rowtile<C::M, N, C::CW, NT, true, 2, C2rCombine<N, C::CW>, false, PlaneRowOut<C::M>>(
      a, tw, C2rCombine<N, C::CW>{a, tw, kfs}, PlaneRowOut<C::M>{reinterpret_cast<float2*>(g)});
}

// i kfs f_y times every value of plane buffer a (f_y the signed frequency of row y;
// zero on the Nyquist row), in place.
template <int N>
__device__ __forceinline__ void plane_deriv_y(float2* a, float kfs) {
  using C = PlaneCfg<N>;
  for (int e = threadIdx.x; e < N * C::CW; e += NT) {
    const int y = e / C::CW;
    const float f = (y == N / 2) ? 0.f : kfs * (float)freq_index(y, N);
    a[e] = cscale(cmul_i(a[e]), f);
  }
  __syncthreads();
}

// Gradient components from spectra after their z inverse, one (plane, component)
// per CTA: component q is c2r(yinv(in[q] times i kfs ky when bit q of dy)) with
// i kfs kx applied on load when bit q of dx.  The CTAs of one plane are
// consecutive (x = plane * n + q), so components that share an input spectrum
// run side by side and the repeated reads of its plane come from L2.
struct PlaneJobs {
  const float2* in[6];
  float* out[6];
  int n, dx, dy;
  float kfs;
  float* zdst = nullptr;  // optional: zdst[0, zfloats) of each simulation is cleared, zchunk
  int64_t zfloats = 0;    // floats (a multiple of 4) per CTA, by 16-byte stores
  int64_t zchunk = 0;
};

template <int N>
__global__ void __launch_bounds__(NT) k_plane_grad(PlaneJobs jobs, const float2* __restrict__ twg, Multi m) {
  using C = PlaneCfg<N>;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* a = sm + N;
  const int z = blockIdx.x / jobs.n, q = blockIdx.x - z * jobs.n;
  const int64_t by = shift_of(m, blockIdx.y), off = (int64_t)z * N * N;
  const float2* in = jobs.in[0];
  float* out = jobs.out[0];
#pragma unroll
  for (int i = 1; i < 6; ++i)  // selects, not an indexed copy of the parameters
    if (i == q) {
      in = jobs.in[i];
      out = jobs.out[i];
    }
  load_tw(tw, twg, N);
  stage_complex_plane<N>(a, moved(in, by), z);
  cp_async_commit();
  if (jobs.zdst) {  // this CTA's share of the zero fill while its plane lands
    const int64_t lo = (int64_t)blockIdx.x * jobs.zchunk, hi = min(lo + jobs.zchunk, jobs.zfloats);
    float4* d = reinterpret_cast<float4*>(moved(jobs.zdst, by));
    for (int64_t i = lo / 4 + threadIdx.x; i < hi / 4; i += NT) d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_async_wait<0>();
  __syncthreads();
  if ((jobs.dy >> q) & 1) plane_deriv_y<N>(a, jobs.kfs);
  plane_yinv<N>(a, tw);
  plane_xc2r<N>(a, tw, ((jobs.dx >> q) & 1) ? jobs.kfs : 0.f, moved(out, by) + off);
}

// Screening source of plane blockIdx.x in one pass (Sec. 6.1, Sec. 6.2): the
// screening field's plane after its z inverse is transformed back along y and x
// (c2r), S = delta eps(w) is formed as the forward x transform loads it (delta
// read from the density plane in global memory), and the forward x (r2c) and y
// steps write S's plane of the interleaved half spectrum; the z pass follows.
template <int N, int MODEL>
__global__ void __launch_bounds__(NT) k_plane_screen(const float2* __restrict__ w_in,
                                                     const float* __restrict__ rho,
                                                     float2* __restrict__ s_out, ForceParams fp,
                                                     const float2* __restrict__ twg, Multi m) {
  using C = PlaneCfg<N>;
  constexpr int M = C::M;
  extern __shared__ __align__(128) float2 sm[];
  float2* tw = sm;
  float2* a = sm + N;
  const int z = blockIdx.x;
  const int64_t by = shift_of(m, blockIdx.y);
  resolve(fp, by);
  load_tw(tw, twg, N);
  stage_complex_plane<N>(a, moved(w_in, by), z);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  plane_yinv<N>(a, tw);
  fft_rowtile<M, N, C::CW, NT, true, 2, C2rCombine<N, C::CW>>(a, tw, C2rCombine<N, C::CW>{a, tw, 0.f});
  const ScreenSource<M, MODEL> src{reinterpret_cast<const float2*>(moved(rho, by) + (int64_t)z * N * N),
                                         fp.inv_rhobar, MODEL == 1 ? fp.fr_thr : fp.dgp_coef};
  fft_rowtile<M, N, C::CW, NT, false, 2, ScreenSource<M, MODEL>>(a, tw, src);
  plane_r2c_split<N>(a, tw);
  constexpr int64_t P = half_pitch(N);
  float2* g = moved(s_out, by) + hrow(z, 0, N, P);
#pragma unroll 1
  for (int c0 = 0; c0 < C::CW; c0 += C::TWCOL)
    fft_tile<N, C::TWCOL, C::CW, NT, false, 1, TileLoad, ColOut>(
        a + c0, tw, TileLoad{}, ColOut{g + hcol(c0), 4 * P, 2 * P, C::M + 1 - c0});
}

// ---------------------------------------------------------------- launch helpers
template <int N, int NBUF>
constexpr size_t col_smem() {
  static_assert(col_rows(N) == fft_rows<N>(), "column stage rows");
  return col_smem_c(N, NBUF);
}

template <int N>
constexpr size_t row_smem() {
  return RowCfg<N, row_tw(N)>::smem;
}

// Along y: o = z, n = y.  Along z: o = y, n = z (rows of a plane pair 8 elements apart).
template <int N, int TW>
ColGeo<N, TW> geo_y(Multi m) {
  const int64_t P = half_pitch(N);
  return ColGeo<N, TW>{2 * N * P, 8, 4 * P, 2 * P, 1, 0, m};
}
template <int N, int TW>
ColGeo<N, TW> geo_z(Multi m) {
  const int64_t P = half_pitch(N);
  return ColGeo<N, TW>{4 * P, 2 * P, 2 * N * P, 8, 0, 1, m};
}
template <int N, int TW>
constexpr int64_t col_tiles() {
  return (int64_t)N * ((N / 2) / TW + 1);
}

}  // namespace

void set_grid_cap(int max_ctas) { g_grid_cap = max_ctas > 0 ? max_ctas : 0; }

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
                               const float2* tw, cudaStream_t s, Multi m) {
  constexpr int TWX = row_tw(N);
  const int64_t tps = (int64_t)N * N / TWX;
  const int64_t ntiles = tps * m.nb;
  auto go = [&](auto bulk_c) {
    constexpr bool BULK = decltype(bulk_c)::value;
    const size_t sm = row_smem<N>() + (BULK ? 2 * sizeof(uint64_t) + 16 : 0);
    auto k = k_xr2c<N, TWX, BULK>;
    unsigned grid;
    cudaError_t e = prep(k, sm, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(in, out, scale, offset, tw, ntiles, m);
    return cudaGetLastError();
  };
  // one 1024-point simulation: 1-D bulk copies stage the real rows (1.93 -> 1.90 ms at 1024^3)
  if constexpr (N >= 1024) {
    if (!m.shift && (reinterpret_cast<uintptr_t>(in) & 15) == 0) return go(std::true_type{});
  }
  return go(std::false_type{});
}

cudaError_t fft_xr2c(int Nv, const float* in, float2* out, float scale, float offset,
                     const float2* tw, cudaStream_t s, Multi m) {
  COLA_SWITCH_N(Nv, return launch_xr2c<N>(in, out, scale, offset, tw, s, m));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_xc2r_multi(int njobs, const float2* const* in, float* const* out,
                                     const float* kfs, const float2* tw, cudaStream_t s, Multi m) {
  constexpr int TWX = row_tw(N);
  const size_t sm = row_smem<N>();
  RowJobs jobs{};
  jobs.njobs = njobs;
  fast_div_magic((uint32_t)njobs, jobs.jmul, jobs.jshift);
  for (int i = 0; i < njobs; ++i) {
    jobs.in[i] = in[i];
    jobs.out[i] = out[i];
    jobs.kfs[i] = kfs[i];
  }
  const int64_t tpj = (int64_t)N * N / TWX;
  auto k = k_xc2r<N, TWX>;
  unsigned grid;
  cudaError_t e = prep(k, sm, tpj * njobs * m.nb, grid);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, sm, s>>>(jobs, tw, tpj, m);
  return cudaGetLastError();
}

cudaError_t fft_xc2r_multi(int Nv, int njobs, const float2* const* in, float* const* out,
                           const float* kfs, const float2* tw, cudaStream_t s, Multi m) {
  if (njobs < 1 || njobs > 6) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_xc2r_multi<N>(njobs, in, out, kfs, tw, s, m));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_xc2r_pair(const float2* a, const float2* b, float* xy, float kfs, const float2* tw,
                                   cudaStream_t s, Multi m) {
  if constexpr (N < 256) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int TWX = row_tw(N);
    const size_t sm = row_smem<N>();
    const int64_t tps = (int64_t)N * N / (TWX / 2);
    auto k = k_xc2r_pair<N, TWX>;
    unsigned grid;
    cudaError_t e = prep(k, sm, tps * m.nb, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(a, b, reinterpret_cast<float2*>(xy), kfs, tw, tps, m);
    return cudaGetLastError();
  }
}

cudaError_t fft_xc2r_pair(int Nv, const float2* a, const float2* b, float* xy, float kfs, const float2* tw,
                          cudaStream_t s, Multi m) {
  COLA_SWITCH_N(Nv, return launch_xc2r_pair<N>(a, b, xy, kfs, tw, s, m));
  return cudaSuccess;
}

template <int N, int OUT>
static cudaError_t launch_xc2r_multi16(int njobs, const float2* const* in, void* const* out, const float* kfs,
                                       const SimHeader* hdr, const float2* tw, cudaStream_t s, Multi m) {
  constexpr int TWX = row_tw(N);
  const size_t sm = row_smem<N>();
  RowJobs jobs{};
  jobs.njobs = njobs;
  jobs.hdr = hdr;
  fast_div_magic((uint32_t)njobs, jobs.jmul, jobs.jshift);
  for (int i = 0; i < njobs; ++i) {
    jobs.in[i] = in[i];
    jobs.out[i] = out[i];
    jobs.kfs[i] = kfs[i];
  }
  const int64_t tpj = (int64_t)N * N / TWX;
  auto k = k_xc2r<N, TWX, OUT>;
  unsigned grid;
  cudaError_t e = prep(k, sm, tpj * njobs * m.nb, grid);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, sm, s>>>(jobs, tw, tpj, m);
  return cudaGetLastError();
}

cudaError_t fft_xc2r_multi16(int Nv, int njobs, const float2* const* in, void* const* out, const float* kfs,
                             int prec, const SimHeader* hdr, const float2* tw, cudaStream_t s, Multi m) {
  if (njobs < 1 || njobs > 6 || !hdr || (prec != 1 && prec != 2)) return cudaErrorInvalidValue;
#define COLA_C2R16(NN)                                                                                    \
  case NN:                                                                                               \
    return prec == 1 ? launch_xc2r_multi16<NN, 1>(njobs, in, out, kfs, hdr, tw, s, m)                    \
                     : launch_xc2r_multi16<NN, 2>(njobs, in, out, kfs, hdr, tw, s, m);
  switch (Nv) {
    COLA_C2R16(32)
    COLA_C2R16(64)
    COLA_C2R16(128)
    COLA_C2R16(256)
    COLA_C2R16(512)
    default:
      return cudaErrorInvalidValue;
  }
#undef COLA_C2R16
}

cudaError_t fft_xc2r(int Nv, const float2* in, float* out, float kfs, const float2* tw,
                     cudaStream_t s, Multi m) {
  return fft_xc2r_multi(Nv, 1, &in, &out, &kfs, tw, s, m);
}

// Tensor map of a half spectrum for the TMA tile loads of a column pass along
// z (zaxis) or y, TW columns per tile (the 5-D view described above
// tma_tile).  False when the driver's encoder is unavailable or refuses the
// map: the launch then stages its tiles with cp.async.
static bool spectrum_map(CUtensorMap& map, const float2* base, int N, int TW, bool zaxis) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  if (!encode || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t P = (cuuint64_t)half_pitch(N), n = (cuuint64_t)N;
  const cuuint64_t dims[5] = {8, 2, P / 8, n, n / 2};
  const cuuint64_t strides[4] = {64, 128, 2 * P * 8, 2 * P * n * 8};
  const cuuint32_t box[5] = {(cuuint32_t)TW, zaxis ? 2u : 1u, 1u, zaxis ? 1u : (cuuint32_t)std::min(N, 256),
                             zaxis ? (cuuint32_t)std::min(N / 2, 256) : 1u};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<float2*>(base), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA staging applies to single-simulation launches of 1024-point columns
// (tiles of at most one 64-byte half chunk).  Measured on GB300 (ms per launch
// against cp.async staging): z force pass 5.09 -> 4.57, screening-field z pass
// 3.24 -> 3.05, y passes 1-2 % faster; at N = 512 the plain y pass runs two
// CTAs per SM at 128 registers and lost (0.187 -> 0.222).
template <int N, int TW>
constexpr bool tma_shape() {
  return N >= 1024 && TW <= 8 && TW % 2 == 0;
}

template <int N>
static cudaError_t launch_col(float2* data, int axis, bool inv, const float2* tw,
                              cudaStream_t s, Multi m) {
  constexpr int TW = col_tw(N, 1);
  constexpr size_t sm = col_smem<N, 1>();
  const int64_t ntiles = col_tiles<N, TW>() * m.nb;
  const ColGeo<N, TW> geo = axis == 1 ? geo_y<N, TW>(m) : geo_z<N, TW>(m);
  CUtensorMap map{};
  const bool tma = tma_shape<N, TW>() && !m.shift && spectrum_map(map, data, N, TW, axis != 1);
  auto go = [&](auto inv_c, auto tma_c) {
    constexpr bool INV = decltype(inv_c)::value, TMA = decltype(tma_c)::value;
    constexpr size_t smk = TMA ? tma_smem<N, fft_rows<N>() * TW, 0>() : sm;
    auto k = k_col<N, TW, INV, TMA>;
    unsigned grid;
    cudaError_t e = prep(k, smk, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smk, s>>>(OpCol<N, TW, INV>{geo, data, data}, tw, ntiles, map);
    return cudaGetLastError();
  };
  using T = std::true_type;
  using F = std::false_type;
  if constexpr (tma_shape<N, TW>()) {
    if (tma) return inv ? go(T{}, T{}) : go(F{}, T{});
  }
  return inv ? go(T{}, F{}) : go(F{}, F{});
}

cudaError_t fft_col(int Nv, float2* data, int axis, bool inv, const float2* tw, cudaStream_t s,
                    Multi m) {
  COLA_SWITCH_N(Nv, return launch_col<N>(data, axis, inv, tw, s, m));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_yinv2(const float2* in, float2* outp, float2* outd, float kfs,
                                const float2* tw, cudaStream_t s, Multi m) {
  if constexpr (N >= 512) {
    // one pass with three rotating single-array tile buffers (k_yinv2r)
    constexpr int TW = col_tw(N, 1);
    const int64_t ntiles = col_tiles<N, TW>() * m.nb;
    CUtensorMap map{};
    const bool tma = tma_shape<N, TW>() && !m.shift && spectrum_map(map, in, N, TW, false);
    auto go = [&](auto tma_c) {
      constexpr bool TMA = decltype(tma_c)::value;
      constexpr size_t sm = yinv2r_smem<N, TW>() + (TMA ? 4 * sizeof(uint64_t) : 0);
      auto k = k_yinv2r<N, TW, TMA>;
      unsigned grid;
      cudaError_t e = prep(k, sm, ntiles, grid);
      if (e != cudaSuccess) return e;
      k<<<grid, NT, sm, s>>>(geo_y<N, TW>(m), in, outp, outd, kfs, tw, ntiles, map);
      return cudaGetLastError();
    };
    if constexpr (tma_shape<N, TW>()) {
      if (tma) return go(std::true_type{});
    }
    return go(std::false_type{});
  } else {
    constexpr int TW = col_tw(N, 2);
    constexpr size_t sm = col_smem<N, 2>();
    const int64_t ntiles = col_tiles<N, TW>() * m.nb;
    auto k = k_yinv2<N, TW>;
    unsigned grid;
    cudaError_t e = prep(k, sm, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(OpYinv2<N, TW>{geo_y<N, TW>(m), in, outp, outd, kfs}, tw, ntiles);
    return cudaGetLastError();
  }
}

cudaError_t fft_yinv2(int Nv, const float2* in, float2* outp, float2* outd, float kfs,
                      const float2* tw, cudaStream_t s, Multi m) {
  COLA_SWITCH_N(Nv, return launch_yinv2<N>(in, outp, outd, kfs, tw, s, m));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_zsf(const float2* in, float2* dk_out, float2* w_out,
                              const ForceParams& fp, const float2* tw, cudaStream_t s, Multi m) {
  constexpr int TW = ztw(N);
  constexpr size_t sm = col_smem_tw(N, TW);
  const int64_t ntiles = col_tiles<N, TW>() * m.nb;
  CUtensorMap map{};
  const bool tma = tma_shape<N, TW>() && !m.shift && spectrum_map(map, in, N, TW, true);
  auto go = [&](auto model, auto tma_c) {
    constexpr int MODEL = decltype(model)::value;
    constexpr bool TMA = decltype(tma_c)::value;
    constexpr size_t smk = TMA ? tma_smem<N, fft_rows<N>() * TW, 0>() : sm;
    auto k = k_z_screen_field<N, TW, MODEL, TMA>;
    unsigned grid;
    cudaError_t e = prep(k, smk, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smk, s>>>(OpZScreenField<N, TW, MODEL>{geo_z<N, TW>(m), in, dk_out, w_out, fp}, tw, ntiles,
                            map);
    return cudaGetLastError();
  };
  auto pick = [&](auto tma_c) {
    if (fp.model == 1) return go(std::integral_constant<int, 1>{}, tma_c);
    if (fp.filter == 0) return go(std::integral_constant<int, 2>{}, tma_c);
    return go(std::integral_constant<int, 3>{}, tma_c);
  };
  if constexpr (tma_shape<N, TW>()) {
    if (tma) return pick(std::true_type{});
  }
  return pick(std::false_type{});
}

cudaError_t mesh_z_screen_field(int Nv, const float2* in, float2* dk_out, float2* w_out,
                                const ForceParams& fp, const float2* tw, cudaStream_t s, Multi m) {
  if (fp.model != 1 && fp.model != 2) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_zsf<N>(in, dk_out, w_out, fp, tw, s, m));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_xscreen(const float2* w_in, const float* rho, float2* s_out,
                                  const ForceParams& fp, const float2* tw, cudaStream_t s, Multi m) {
  constexpr int TWX = row_tw(N);
  constexpr size_t sm = xscreen_smem<N, TWX>();
  const int64_t tps = (int64_t)N * N / TWX;
  const int64_t ntiles = tps * m.nb;
  unsigned grid;
  if (fp.model == 1) {
    auto k = k_x_screen<N, TWX, 1>;
    cudaError_t e = prep(k, sm, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(w_in, rho, s_out, fp, tw, ntiles, m);
  } else {
    auto k = k_x_screen<N, TWX, 2>;
    cudaError_t e = prep(k, sm, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, sm, s>>>(w_in, rho, s_out, fp, tw, ntiles, m);
  }
  return cudaGetLastError();
}

cudaError_t mesh_x_screen_source(int Nv, const float2* w_in, const float* rho, float2* s_out,
                                 const ForceParams& fp, const float2* tw, cudaStream_t s, Multi m) {
  if (fp.model != 1 && fp.model != 2) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_xscreen<N>(w_in, rho, s_out, fp, tw, s, m));
  return cudaSuccess;
}

template <int N, bool SCR>
static cudaError_t launch_zforce_t(const float2* in, const float2* dk, float2* phi,
                                   float2* phiz, const ForceParams& fp,
                                   const float2* tw, cudaStream_t s, Multi m) {
  constexpr int TW = ztw(N);
  constexpr size_t sm = col_smem_tw(N, TW) + (size_t)N * TW * sizeof(float2);
  const int64_t ntiles = col_tiles<N, TW>() * m.nb;
  CUtensorMap map{}, dmap{};
  const bool tma = tma_shape<N, TW>() && !m.shift && spectrum_map(map, in, N, TW, true) &&
                   (!SCR || spectrum_map(dmap, dk, N, TW, true));
  auto go = [&](auto tma_c) {
    constexpr bool TMA = decltype(tma_c)::value;
    constexpr size_t smk = TMA ? tma_smem<N, fft_rows<N>() * TW, N * TW>() : sm;
    auto k = k_z_force<N, TW, SCR, TMA>;
    unsigned grid;
    cudaError_t e = prep(k, smk, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smk, s>>>(OpZForce<N, TW, SCR>{geo_z<N, TW>(m), in, dk, phi, phiz, fp}, tw, ntiles, map,
                            dmap);
    return cudaGetLastError();
  };
  if constexpr (tma_shape<N, TW>()) {
    if (tma) return go(std::true_type{});
  }
  return go(std::false_type{});
}

cudaError_t mesh_z_force(int Nv, const float2* in, const float2* dk, float2* phi_out,
                         float2* phiz_out, const ForceParams& fp, const float2* tw, cudaStream_t s,
                         Multi m) {
  if (fp.screened && dk == nullptr) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return fp.screened ? launch_zforce_t<N, true>(in, dk, phi_out, phiz_out, fp, tw, s, m)
                                       : launch_zforce_t<N, false>(in, dk, phi_out, phiz_out, fp, tw, s, m));
  return cudaSuccess;
}

template <int N, int PREC>
static cudaError_t launch_lpt_t(const void* p1, const void* p2, float2* o0, float2* o1,
                                float2* o2, float2* o3, const LptParams& lp, const float2* tw,
                                cudaStream_t s, Multi m, float* zero_dst, int64_t zero_floats,
                                bool* zeroed) {
  constexpr int TW = col_tw(N, 4);
  // one simulation at N >= 512 (one CTA per SM either way): the table row also
  // goes to shared memory
  const int tab_smem = (N >= 512 && !m.shift) ? 1 : 0;
  // the zero fill rides along where the pass runs one CTA per SM (N >= 512: room for the
  // 16 KB zero region) on 16-byte aligned memory
  const bool zf = zero_dst && zero_floats > 0 && N >= 512 && (zero_floats % 4) == 0 &&
                  (reinterpret_cast<uintptr_t>(zero_dst) & 15) == 0;
  using Op = OpLptZ<N, TW, PREC>;
  const size_t sm = col_smem<N, 4>() + (tab_smem ? (size_t)lp.nk * sizeof(float4) : 0) + (zf ? Op::kZero : 0);
  const int64_t ntiles = col_tiles<N, TW>() * m.nb;
  auto k = k_lpt_z<N, TW, PREC>;
  unsigned grid;
  cudaError_t e = prep(k, sm, ntiles, grid);
  if (e != cudaSuccess) return e;
  Op op{geo_z<N, TW>(m), p1, p2, o0, o1, o2, o3, lp, tab_smem};
  if (zf) {
    op.zdst = reinterpret_cast<char*>(zero_dst);
    op.zbytes = zero_floats * (int64_t)sizeof(float);
    const int64_t tps = col_tiles<N, TW>();
    op.zchunk = ((op.zbytes + tps - 1) / tps + 15) / 16 * 16;
  }
  k<<<grid, NT, sm, s>>>(op, tw, ntiles);
  e = cudaGetLastError();
  if (e == cudaSuccess && zeroed) *zeroed = zf;
  return e;
}

template <int N, int PREC>
static cudaError_t launch_lpt8(const void* p1, const void* p2, float2* o0, float2* o1, float2* o2, float2* o3,
                               const LptParams& lp, const float2* tw, cudaStream_t s, Multi m) {
  const size_t sm = LptZ8<N, PREC>::smem;
  const int64_t ntiles = col_tiles<N, 8>() * m.nb;
  auto k = k_lpt_z8<N, PREC>;
  unsigned grid;
  cudaError_t e = prep(k, sm, ntiles, grid);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, sm, s>>>(geo_z<N, 8>(m), p1, p2, o0, o1, o2, o3, lp, tw, ntiles);
  return cudaGetLastError();
}
template <int N>
static cudaError_t launch_lpt(const void* p1, const void* p2, float2* o0, float2* o1, float2* o2,
                              float2* o3, const LptParams& lp, const float2* tw,
                              cudaStream_t s, Multi m, float* zd, int64_t zn, bool* zeroed) {
  // measured on GB300 (ms per launch, 4-column -> 8-column tiles): N = 256 FP32 0.154 -> 0.144,
  // FP16 0.180 -> 0.143; N = 512 FP32 1.40 -> 1.46 (kept on 4 columns), FP16 1.55 -> 1.44
  if constexpr (N == 256 || N == 512) {
    if (lp.seed_prec == 1) return launch_lpt8<N, 1>(p1, p2, o0, o1, o2, o3, lp, tw, s, m);
    if (lp.seed_prec == 2) return launch_lpt8<N, 2>(p1, p2, o0, o1, o2, o3, lp, tw, s, m);
    if constexpr (N == 256) return launch_lpt8<N, 0>(p1, p2, o0, o1, o2, o3, lp, tw, s, m);
  }
  if (lp.seed_prec == 1) return launch_lpt_t<N, 1>(p1, p2, o0, o1, o2, o3, lp, tw, s, m, zd, zn, zeroed);
  if (lp.seed_prec == 2) return launch_lpt_t<N, 2>(p1, p2, o0, o1, o2, o3, lp, tw, s, m, zd, zn, zeroed);
  return launch_lpt_t<N, 0>(p1, p2, o0, o1, o2, o3, lp, tw, s, m, zd, zn, zeroed);
}

cudaError_t lpt_z(int Nv, const void* phi1, const void* phi2, float2* o0, float2* o1, float2* o2,
                  float2* o3, const LptParams& lp, const float2* tw, cudaStream_t s, Multi m,
                  float* zero_dst, int64_t zero_floats, bool* zeroed) {
  if (zeroed) *zeroed = false;
  if (Nv > 512) return cudaErrorInvalidValue;  // four double-buffered 4-column tiles exceed shared memory
  COLA_SWITCH_N(Nv, return launch_lpt<N>(phi1, phi2, o0, o1, o2, o3, lp, tw, s, m, zero_dst, zero_floats, zeroed));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_plane_r2c(const float* in, float2* out, float scale, float offset,
                                    const float2* tw, cudaStream_t s, Multi m) {
  if constexpr (N > 128) {
    return cudaErrorInvalidValue;
  } else {
    constexpr size_t sm = PlaneCfg<N>::smem;
    auto k = k_plane_r2c<N>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k<<<dim3(N, m.nb), NT, sm, s>>>(in, out, scale, offset, tw, m);
    return cudaGetLastError();
  }
}

cudaError_t fft_plane_r2c(int Nv, const float* in, float2* out, float scale, float offset, const float2* tw,
                          cudaStream_t s, Multi m) {
  COLA_SWITCH_N(Nv, return launch_plane_r2c<N>(in, out, scale, offset, tw, s, m));
  return cudaSuccess;
}

template <int N>
static cudaError_t launch_plane_grad(const PlaneJobs& jobs, const float2* tw, cudaStream_t s, Multi m) {
  if constexpr (N > 128) {
    return cudaErrorInvalidValue;
  } else {
    constexpr size_t sm = PlaneCfg<N>::smem;
    auto k = k_plane_grad<N>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k<<<dim3(jobs.n * N, m.nb), NT, sm, s>>>(jobs, tw, m);
    return cudaGetLastError();
  }
}

static cudaError_t plane_grad(int Nv, const PlaneJobs& jobs, const float2* tw, cudaStream_t s, Multi m) {
  if (jobs.n < 1 || jobs.n > 6) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_plane_grad<N>(jobs, tw, s, m));
  return cudaSuccess;
}

cudaError_t fft_plane_force(int Nv, const float2* phi, const float2* phiz, float* fx, float* fy, float* fz,
                            float kfs, const float2* tw, cudaStream_t s, Multi m) {
  const PlaneJobs jobs{{phi, phi, phiz}, {fx, fy, fz}, 3, 1, 2, kfs};
  return plane_grad(Nv, jobs, tw, s, m);
}

cudaError_t fft_plane_lpt(int Nv, const float2* const* lc, float* const* out, float kfs, const float2* tw,
                          cudaStream_t s, Multi m, float* zero_dst, int64_t zero_floats, bool* zeroed) {
  PlaneJobs jobs{{lc[0], lc[0], lc[1], lc[2], lc[2], lc[3]},
                 {out[0], out[1], out[2], out[3], out[4], out[5]},
                 6,
                 0b001001,
                 0b010010,
                 kfs};
  const bool zf = zero_dst && zero_floats > 0 && (zero_floats % 4) == 0 &&
                  (reinterpret_cast<uintptr_t>(zero_dst) & 15) == 0;
  if (zf) {
    const int64_t ctas = (int64_t)jobs.n * Nv;
    jobs.zdst = zero_dst;
    jobs.zfloats = zero_floats;
    jobs.zchunk = (zero_floats + 4 * ctas - 1) / (4 * ctas) * 4;
  }
  const cudaError_t e = plane_grad(Nv, jobs, tw, s, m);
  if (e == cudaSuccess && zeroed) *zeroed = zf;
  return e;
}

template <int N>
static cudaError_t launch_plane_screen(const float2* w_in, const float* rho, float2* s_out,
                                       const ForceParams& fp, const float2* tw, cudaStream_t s, Multi m) {
  if constexpr (N > 128) {
    return cudaErrorInvalidValue;
  } else {
    constexpr size_t sm = PlaneCfg<N>::smem;
    auto k = fp.model == 1 ? k_plane_screen<N, 1> : k_plane_screen<N, 2>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k<<<dim3(N, m.nb), NT, sm, s>>>(w_in, rho, s_out, fp, tw, m);
    return cudaGetLastError();
  }
}

cudaError_t fft_plane_screen(int Nv, const float2* w_in, const float* rho, float2* s_out, const ForceParams& fp,
                             const float2* tw, cudaStream_t s, Multi m) {
  if (fp.model != 1 && fp.model != 2) return cudaErrorInvalidValue;
  COLA_SWITCH_N(Nv, return launch_plane_screen<N>(w_in, rho, s_out, fp, tw, s, m));
  return cudaSuccess;
}

cudaError_t wait_probe(double seconds, int* timed_out) {
  if (!(seconds > 0) || seconds > 10) return cudaErrorInvalidValue;
  k_wait_probe<<<1, 32, 0, cudaStreamPerThread>>>((uint64_t)(seconds * 1e9));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbolAsync(timed_out, g_wait_probe, sizeof(int), 0, cudaMemcpyDeviceToHost,
                                  cudaStreamPerThread);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
  return e;
}

cudaError_t tile_load_failures(unsigned* dst, cudaStream_t s) {
  return cudaMemcpyFromSymbolAsync(dst, g_tile_load_failures, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
}

}  // namespace cola
