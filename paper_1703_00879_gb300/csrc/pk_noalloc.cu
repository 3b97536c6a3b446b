// Matter power spectrum of caller-given particle positions with no device
// allocation at all.
//
// Who needs this: callers that cannot call cudaMalloc/cudaFree at the moment
// they want a P(k).  cudaFree (and cudaMalloc when the pool must grow)
// synchronises the whole device, which stalls every other stream of a
// latency-bound serving loop; a process whose device memory is owned by
// another allocator (for example a framework's caching allocator holding a
// fixed pool) may not be able to obtain fresh memory at all; and diagnostics
// run in the middle of a long simulation must not be able to fail on an
// allocation.  Such callers pass their own input and output buffers and the
// scratch comes from a file-scope device array that the library reserves on
// every GPU that loads it.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; each call clears what must start at zero.  Calls whose
// device work overlaps (on different streams, or from different host threads
// without ordering) race on the array and must not be issued.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "cola.h"
#include "cola_internal.h"

namespace {

constexpr int kMaxMesh = COLA_PK_NOALLOC_MAX_NMESH;
constexpr int kMaxBinsNA = 2000;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kTwBytes = align256((size_t)kMaxMesh * 8);                     // twiddles
constexpr size_t kAccBytes = align256((size_t)3 * kMaxBinsNA * 8);              // bin sums (double)
constexpr size_t kRhoBytes = align256((size_t)kMaxMesh * kMaxMesh * kMaxMesh * 4);
constexpr size_t kHalfBytes =
    align256((size_t)kMaxMesh * kMaxMesh * (((kMaxMesh / 2 + 1 + 15) / 16) * 16) * 8);
constexpr size_t kScratchBytes = kTwBytes + kAccBytes + kRhoBytes + kHalfBytes;

// The scratch: on the host this name is only a stand-in for the symbol; its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_pk_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<char> g_reserved;  // per device: the scratch's module has been loaded

int na_fail(int code, const std::string& m) {
  cola::set_context_free_error(m);  // reported by cola_last_error(NULL)
  return code;
}

// The device address of the scratch on the current device.  Asked for on every
// call (cheap once the module is loaded), so no address outlives a device reset.
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_pk_scratch);
  if (e != cudaSuccess || !p)
    return na_fail(COLA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = static_cast<unsigned char*>(p);
  return COLA_OK;
}

}  // namespace

// Set-up, once per device with that device current (cola_init calls it): with
// lazy module loading the scratch is reserved only when its module loads, so
// this loads it now, at a known time, rather than at the first cola_pk_noalloc.
int cola::pk_noalloc_reserve() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(COLA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_reserved.size() <= dev) g_reserved.resize(dev + 1, 0);
  if (g_reserved[dev]) return COLA_OK;
  unsigned char* p = nullptr;
  const int rc = scratch_address(&p);
  if (rc != COLA_OK) return rc;
  g_reserved[dev] = 1;
  return COLA_OK;
}

extern "C" int cola_pk_noalloc(const float* pos, int64_t n, int32_t nmesh, double Lbox,
                               int32_t nbins, double* k, double* pk, int64_t* nmodes,
                               void* stream) {
  cola::set_context_free_error("");
  if (nmesh < 32 || nmesh > kMaxMesh || (nmesh & (nmesh - 1)) != 0)
    return na_fail(COLA_EINVAL, "cola_pk_noalloc: nmesh must be a power of two in 32.." +
                                    std::to_string(kMaxMesh) + " (the static scratch holds at most " +
                                    std::to_string(kMaxMesh) + "^3 cells)");
  if (n <= 0 || !pos) return na_fail(COLA_EINVAL, "cola_pk_noalloc: need n > 0 positions");
  if (!(Lbox > 0)) return na_fail(COLA_EINVAL, "cola_pk_noalloc: Lbox must be > 0");
  if (nbins < 1 || nbins > kMaxBinsNA) return na_fail(COLA_EINVAL, "cola_pk_noalloc: nbins out of range 1..2000");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != COLA_OK) return rc;
  float2* tw = reinterpret_cast<float2*>(base);
  double* acc = reinterpret_cast<double*>(base + kTwBytes);
  float* rho = reinterpret_cast<float*>(base + kTwBytes + kAccBytes);
  float2* half = reinterpret_cast<float2*>(base + kTwBytes + kAccBytes + kRhoBytes);
  const int N = nmesh;
  const double pi = 3.14159265358979323846;
  std::vector<float2> htw(N);
  for (int m = 0; m < N; ++m)
    htw[m] = make_float2((float)std::cos(-2.0 * pi * m / N), (float)std::sin(-2.0 * pi * m / N));
  const double N3 = (double)N * N * N;
#define NA_CK(expr)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return na_fail(COLA_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  NA_CK(cudaMemcpyAsync(tw, htw.data(), N * sizeof(float2), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemsetAsync(rho, 0, (size_t)N * N * N * sizeof(float), st));
  NA_CK(cudaMemsetAsync(acc, 0, (size_t)3 * nbins * sizeof(double), st));
  NA_CK(cola::pos_deposit(N, (float)(N / Lbox), pos, n, rho, st));
  NA_CK(cola::fft_xr2c(N, rho, half, (float)(N3 / (double)n), -1.f, tw, st));
  NA_CK(cola::fft_col(N, half, 1, false, tw, st));
  NA_CK(cola::fft_col(N, half, 2, false, tw, st));
  NA_CK(cola::pk_bin(N, half, nbins, acc, Lbox * Lbox * Lbox / (N3 * N3), st));
  std::vector<double> h(3 * nbins);
  NA_CK(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
  const double kf = 2.0 * pi / Lbox;
  for (int b = 0; b < nbins; ++b) {
    const double cnt = h[b];
    if (k) k[b] = cnt > 0 ? h[2 * nbins + b] / cnt * kf : NAN;
    if (pk) pk[b] = cnt > 0 ? h[nbins + b] / cnt : NAN;
    if (nmodes) nmodes[b] = (int64_t)llround(cnt);
  }
  return COLA_OK;
}
