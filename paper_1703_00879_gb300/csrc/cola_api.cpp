// C ABI of libcola: context, buffers, and the orchestration of the COLA step
// (Sec. 2, Sec. 4, Sec. 6, App. A, App. B) on one CUDA stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "cola.h"
#include "cola_internal.h"
#include "host_cosmo.h"

using namespace cola;

namespace {
thread_local std::string g_err;
}

void cola::set_context_free_error(const std::string& msg) { g_err = msg; }

struct cola_ctx {
  cola_config cfg{};
  cola_model model{};  // its table pointers are cleared: the tables live in hm
  HModel hm;            // the model as the host solvers take it
  bool model_set = false, ic_done = false, have_force = false, have_lpt = false;
  // scale-independent LPT fast path: lr[0..2] hold Psi1 and lr[3..5] Psi2 from
  // the ICs on, and the per-step LPT transforms are skipped
  bool lpt_fast = false;
  cudaStream_t st = nullptr;
  cola_alloc_fn alloc = nullptr;
  cola_free_fn freef = nullptr;
  void* user = nullptr;
  std::string err;
  std::vector<void*> allocs;
  cudaEvent_t ev_order = nullptr;  // orders the context's stream with cola_step_many's stream
  double wait_limit_s = 0;         // > 0: host waits give up after this long (COLA_ETIMEOUT)
  cudaEvent_t ev_wait = nullptr;   // recorded by bounded host waits
  double* pk_host = nullptr;       // pinned [3 * kMaxBins] (cola_pk_async)
  cudaEvent_t pk_event = nullptr;
  int pk_nbins = 0;                // bins of the pending cola_pk_async, 0: none
  int Np = 0, Nm = 0, lgNp = 0, nk = 0;
  double L = 0;
  int64_t P = 0, M = 0;
  std::vector<double> a, dtk1, dtd, dtk2;
  int step = 0;
  double lnk0 = 0, dlnk = 0;
  // particles (SoA)
  float* s[3] = {};
  float* v[3] = {};
  float* acc[3] = {};
  // seeds
  float2* phi[2] = {};
  void* seedq[2] = {};
  // LPT work
  float2* lc[6] = {};
  float* lr[6] = {};
  // second slot of the kick fields (FP32 runs): multi-step cola_step computes step n+1's
  // LPT fields before step n's kick, so the two kick fields alternate; kslot = the slot
  // holding the last step's (0: lr[3..5], 1: lrk)
  float* lrk[3] = {};
  int kslot = 0;
  // reduced-precision variant: the per-step drift (0..2) and kick (3..5) LPT
  // fields as 16-bit values with one FP32 scale per field (SimHeader lq_*)
  uint16_t* lq[6] = {};
  // mesh
  float* rho = nullptr;
  float2 *Cd = nullptr, *Ck = nullptr, *Cw = nullptr, *Cphi = nullptr, *Cphz = nullptr;
  // force mesh: F_x, F_y, F_z in F[0], F[1] = F[0] + M, F[2]; with fpairs (meshes
  // above 128 points) F[0] holds the (F_x, F_y) pairs instead (2 floats per cell
  // over F[0] and F[1]'s storage, read by the gather as one 8-byte load per corner)
  float* F[3] = {};
  bool fpairs = false;
  float2 *tw_np = nullptr, *tw_nm = nullptr;
  char* tables = nullptr;      // tab, vtab, dfp, ddt: this context's copy of its key's tables
  size_t tables_bytes = 0;
  float4 *tab = nullptr, *vtab = nullptr;
  double* pk_acc = nullptr;
  float* scratch = nullptr;
  EHParams eh{};
  double Dratio = 1.0;
  // device-resident step state: current step and per-step parameters, so the
  // launch sequence of a step does not depend on which step it is
  SimHeader* hdr = nullptr;    // device header (in the context's allocation)
  SimHeader hh{};              // host copy of what was last written to it
  ForceParams* dfp = nullptr;  // [nsteps]: force parameters at a_{n+1}
  float* ddt = nullptr;        // [nsteps][3]: half kick, drift, half kick
  // per-stage event timing
  bool prof = false;
  struct Stage {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double ms = 0;
    int64_t launches = 0;
    double bytes = 0;
  };
  std::vector<Stage> stages;
  std::vector<cudaEvent_t> event_pool;
};

// A batch of contexts advanced together, one CUDA graph launch per step.
struct cola_batch {
  std::vector<cola_ctx*> ctx;
  bool uniform = false;                    // one shape: multi-simulation launches possible
  cudaStream_t st = nullptr;               // caller's stream (may be the legacy stream)
  cudaStream_t cap_st = nullptr;           // owned: graphs are captured and launched here
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaStream_t> chain_st;      // forked capture streams (owned, created on demand)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;           // one per chain stream (owned)
  cola_batch_plan plan{1, 1, 0, 0, 0};
  int step = 0;
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    void* shifts = nullptr;                // device shift arrays the graph's launches read
                                           // (through the first context's allocator, on cap_st)
  };
  std::map<std::tuple<int, int, int, int, int, int>, Graph> graphs;  // (plan, launch sequence) -> graph
                                                                     // serving every step
  double* pk_acc = nullptr;                // [n][3 * kMaxBins] + n shifts (batch P(k)), through
                                           // the first context's allocator, on st
  std::string err;
};

namespace {

constexpr int kMaxBins = 2000;

enum Stage {
  ST_LPT_Z, ST_LPT_Y, ST_LPT_X, ST_RHO_ZERO, ST_DRIFT_DEPOSIT, ST_MESH_XR2C, ST_MESH_Y,
  ST_Z_SCREEN_FIELD, ST_X_SCREEN_SOURCE, ST_Z_FORCE, ST_MESH_YINV, ST_MESH_XC2R, ST_GATHER_KICK,
  ST_KICK_DRIFT_DEPOSIT, ST_COUNT
};
const char* const kStageNames[ST_COUNT] = {
    "lpt_z_reweight", "lpt_y_inverse", "lpt_x_c2r", "rho_zero", "drift_deposit", "mesh_x_r2c",
    "mesh_y_forward", "z_screen_field", "x_screen_source", "z_force", "mesh_y_inverse",
    "mesh_x_c2r", "gather_kick", "kick_drift_deposit"};

cudaEvent_t take_event(cola_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records the start of a launch group; returns the event (null when not
// profiling).  Every stage is also an NVTX range (a no-op without a tool
// attached), so a timeline profiler shows the step's stages by name.
cudaEvent_t prof_begin(cola_ctx* c, int stage) {
  nvtxRangePushA(kStageNames[stage]);
  if (!c->prof) return nullptr;
  cudaEvent_t e = take_event(c);
  if (e) cudaEventRecord(e, c->st);
  return e;
}

// Closes a launch group of `launches` kernels that moves `bytes` algorithmic
// bytes in total.
void prof_end(cola_ctx* c, int stage, cudaEvent_t start, int launches, double bytes) {
  nvtxRangePop();
  if (!c->prof || !start) return;
  cudaEvent_t e = take_event(c);
  if (!e) return;
  cudaEventRecord(e, c->st);
  auto& s = c->stages[stage];
  s.pending.emplace_back(start, e);
  s.launches += launches;
  s.bytes += bytes;
}

int fail(cola_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_err = msg;
  return code;
}

#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, COLA_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define CHECK_RC(expr)          \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != COLA_OK) return rc_; \
  } while (0)

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Device memory through the context's callbacks, for use on stream st (NULL
// callbacks: the stream-ordered cudaMallocAsync / cudaFreeAsync).
void* dev_alloc_on(cola_ctx* c, size_t bytes, cudaStream_t st) {
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, (void*)st, c->user);
  } else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dev_free_on(cola_ctx* c, void* p, cudaStream_t st) {
  if (!p) return;
  if (c->freef) c->freef(p, (void*)st, c->user);
  else if (!c->alloc) cudaFreeAsync(p, st);
}

void* dev_alloc(cola_ctx* c, size_t bytes) { return dev_alloc_on(c, bytes, c->st); }
void dev_free(cola_ctx* c, void* p) { dev_free_on(c, p, c->st); }

template <class T>
int alloc_buf(cola_ctx* c, T** out, size_t count) {
  void* p = dev_alloc(c, count * sizeof(T));
  if (!p) return fail(c, COLA_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
  c->allocs.push_back(p);
  *out = static_cast<T*>(p);
  return COLA_OK;
}

// Temporary device buffer, released by the destructor in stream order (the
// free callback, like cudaFreeAsync, lets only later work on the stream reuse it).
struct Temp {
  cola_ctx* c;
  void* p = nullptr;
  Temp(cola_ctx* cc, size_t bytes) : c(cc) {
    if (bytes) p = dev_alloc(c, bytes);
  }
  ~Temp() { dev_free(c, p); }
};

// Waits on the host for the work queued so far on the context's stream; with a
// wait limit set, gives up after that long with COLA_ETIMEOUT (the work stays
// queued and completes later; the context stays usable).
int host_wait(cola_ctx* ctx) {
  if (!(ctx->wait_limit_s > 0)) {
    CK(cudaStreamSynchronize(ctx->st));
    return COLA_OK;
  }
  if (!ctx->ev_wait) CK(cudaEventCreateWithFlags(&ctx->ev_wait, cudaEventDisableTiming));
  CK(cudaEventRecord(ctx->ev_wait, ctx->st));
  const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(ctx->wait_limit_s);
  for (;;) {
    const cudaError_t e = cudaEventQuery(ctx->ev_wait);
    if (e == cudaSuccess) return COLA_OK;
    if (e != cudaErrorNotReady) return fail(ctx, COLA_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(e));
    if (std::chrono::steady_clock::now() >= t_end)
      return fail(ctx, COLA_ETIMEOUT, "the device work did not complete within the wait limit");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int validate_cfg(const cola_config* cfg, cola_ctx* c) {
  if (!cfg) return fail(c, COLA_EINVAL, "cfg is NULL");
  if (!pow2_in(cfg->Np, 32, 512)) return fail(c, COLA_EINVAL, "Np must be a power of two in 32..512");
  if (!pow2_in(cfg->Nmesh, 32, 1024)) return fail(c, COLA_EINVAL, "Nmesh must be a power of two in 32..1024");
  if (cfg->nsteps < 1) return fail(c, COLA_EINVAL, "nsteps must be >= 1");
  if (!(cfg->Lbox > 0)) return fail(c, COLA_EINVAL, "Lbox must be > 0");
  if (!(cfg->Omega_m > 0 && cfg->Omega_m <= 1) || !(cfg->Omega_b >= 0 && cfg->Omega_b < cfg->Omega_m) ||
      !(cfg->h > 0) || !(cfg->sigma8 > 0))
    return fail(c, COLA_EINVAL, "cosmological parameters out of range");
  if (!(cfg->z_ini > cfg->z_final) || !(cfg->z_final >= 0))
    return fail(c, COLA_EINVAL, "need z_ini > z_final >= 0");
  if (cfg->nk_table < 16 || cfg->nk_table > (1 << 20)) return fail(c, COLA_EINVAL, "nk_table out of range");
  if (cfg->seed_precision < 0 || cfg->seed_precision > 2) return fail(c, COLA_EINVAL, "seed_precision must be 0, 1 or 2");
  return COLA_OK;
}

int validate_model(const cola_model* m, cola_ctx* c) {
  if (!m) return fail(c, COLA_EINVAL, "model is NULL");
  if (m->kind < 0 || m->kind > 4) return fail(c, COLA_EINVAL, "unknown model kind");
  if (m->kind == COLA_MB) {
    if (m->mb_n < 2 || m->mb_n > 4096) return fail(c, COLA_EINVAL, "mb_n must be in [2, 4096]");
    if (!m->mb_a || !m->mb_beta || !m->mb_m) return fail(c, COLA_EINVAL, "mb tables are NULL");
    for (int i = 0; i < m->mb_n; ++i) {
      if (!(m->mb_a[i] > 0) || (i > 0 && !(m->mb_a[i] > m->mb_a[i - 1])) || !std::isfinite(m->mb_a[i]))
        return fail(c, COLA_EINVAL, "mb_a must be positive and strictly ascending");
      if (!(m->mb_beta[i] >= 0) || !std::isfinite(m->mb_beta[i]))
        return fail(c, COLA_EINVAL, "mb_beta must be finite and >= 0");
      if (!(m->mb_m[i] > 0) || !std::isfinite(m->mb_m[i])) return fail(c, COLA_EINVAL, "mb_m must be finite and > 0");
    }
    if (!(m->mb_phicrit0 >= 0)) return fail(c, COLA_EINVAL, "mb_phicrit0 must be >= 0");
  }
  if (m->kind == COLA_SYMM && !(m->beta_star > 0 && m->m_star > 0 && m->a_star > 0 && m->a_star <= 1))
    return fail(c, COLA_EINVAL, "symmetron needs beta_star > 0, m_star > 0 and 0 < a_star <= 1");
  if (m->kind == COLA_FOFR && !(m->fR0 > 0)) return fail(c, COLA_EINVAL, "f(R) needs fR0 > 0");
  if (m->kind == COLA_NDGP && !(m->rcH0 > 0)) return fail(c, COLA_EINVAL, "nDGP needs rcH0 > 0");
  if (m->kind == COLA_NDGP && m->screening && !(m->R_smooth > 0))
    return fail(c, COLA_EINVAL, "Vainshtein screening needs R_smooth > 0");
  if (m->filter < 0 || m->filter > 2)
    return fail(c, COLA_EINVAL, "filter: 0 Gaussian, 1 top-hat, 2 sharp-k");
  return COLA_OK;
}

// A tabulated {m, beta} model must cover the run's scale factors.
int validate_model_range(const cola_config& cfg, const cola_model& m, cola_ctx* c) {
  if (m.kind != COLA_MB) return COLA_OK;
  const double ai = 1.0 / (1.0 + cfg.z_ini), af = 1.0 / (1.0 + cfg.z_final);
  if (m.mb_a[0] > ai || m.mb_a[m.mb_n - 1] < af)
    return fail(c, COLA_EINVAL, "mb_a must cover [a_ini, a_final] of the run");
  return COLA_OK;
}

bool chameleon_kind(int kind) { return kind == COLA_FOFR || kind == COLA_SYMM || kind == COLA_MB; }

std::vector<double> a_nodes(const cola_config& cfg) {
  const double ai = 1.0 / (1.0 + cfg.z_ini), af = 1.0 / (1.0 + cfg.z_final);
  std::vector<double> a(cfg.nsteps + 1);
  for (int i = 0; i <= cfg.nsteps; ++i) a[i] = ai + i * (af - ai) / cfg.nsteps;
  a[cfg.nsteps] = af;
  return a;
}

void k_nodes(const cola_config& cfg, double& lnk0, double& dlnk, std::vector<double>& k) {
  const double kF = 2.0 * kPi / cfg.Lbox;
  const double kmin = 0.5 * kF, kmax = 1.01 * std::sqrt(3.0) * kPi * cfg.Np / cfg.Lbox;
  lnk0 = std::log(kmin);
  dlnk = (std::log(kmax) - lnk0) / (cfg.nk_table - 1);
  k.resize(cfg.nk_table);
  for (int j = 0; j < cfg.nk_table; ++j) k[j] = std::exp(lnk0 + dlnk * j);
}

HModel hmodel(const cola_model& m) {
  HModel h;
  h.kind = m.kind;
  h.beta_star = m.beta_star;
  h.m_star = m.m_star;
  h.a_star = m.a_star;
  h.fR0 = m.fR0;
  h.rcH0 = m.rcH0;
  h.R_smooth = m.R_smooth;
  h.screening = m.screening;
  h.scale_dependent = m.scale_dependent;
  if (m.kind == COLA_MB) {
    h.ta.assign(m.mb_a, m.mb_a + m.mb_n);
    h.tbeta.assign(m.mb_beta, m.mb_beta + m.mb_n);
    h.tM2.resize(m.mb_n);
    for (int i = 0; i < m.mb_n; ++i) h.tM2[i] = m.mb_m[i] * m.mb_m[i];
    h.phicrit0 = m.mb_phicrit0;
    mb_prepare(h);
  }
  return h;
}

// Growth tables depend only on (Omega_m, box, Np, time grid, nk, model): solved
// once per distinct key and shared by every context of the process.
std::mutex g_growth_mu;
std::map<std::vector<double>, Growth> g_growth_cache;

void growth_for(const cola_config& cfg, const HModel& m, Growth& g, std::vector<double>* kout,
                double* lnk0_out, double* dlnk_out) {
  double lnk0, dlnk;
  std::vector<double> k;
  k_nodes(cfg, lnk0, dlnk, k);
  const bool lcdm = (m.kind == COLA_LCDM) || !m.scale_dependent;
  std::vector<double> key = {cfg.Omega_m, cfg.Lbox, (double)cfg.Np, cfg.z_ini, cfg.z_final,
                             (double)cfg.nsteps, (double)cfg.nk_table, (double)m.kind,
                             lcdm ? 0.0 : m.fR0, lcdm ? 0.0 : m.rcH0, lcdm ? 1.0 : 0.0,
                             lcdm ? 0.0 : m.beta_star, lcdm ? 0.0 : m.m_star, lcdm ? 0.0 : m.a_star};
  if (!lcdm)
    for (const auto* v : {&m.ta, &m.tbeta, &m.tM2}) key.insert(key.end(), v->begin(), v->end());
  {
    std::lock_guard<std::mutex> lk(g_growth_mu);
    auto it = g_growth_cache.find(key);
    if (it != g_growth_cache.end()) {
      g = it->second;
      if (kout) *kout = k;
      if (lnk0_out) *lnk0_out = lnk0;
      if (dlnk_out) *dlnk_out = dlnk;
      return;
    }
  }
  solve_growth(m, cfg.Omega_m, a_nodes(cfg), k, lcdm, g);
  {
    std::lock_guard<std::mutex> lk(g_growth_mu);
    if (g_growth_cache.size() > 4096) g_growth_cache.clear();
    g_growth_cache.emplace(key, g);
  }
  if (kout) *kout = k;
  if (lnk0_out) *lnk0_out = lnk0;
  if (dlnk_out) *dlnk_out = dlnk;
}

// ---------------------------------------------------------------- host tables and uploads
// Read-only data that depends only on a key (the growth tables, per-step force
// parameters and time integrals of a (configuration without the seed, model)
// pair) is computed on the host once per key and kept in a bounded host cache;
// every context holds its own device copy inside its single allocation, so all
// device memory comes through the caller's allocator and goes in cola_free.
constexpr size_t kMaxHostTableBytes = (size_t)256 << 20;
std::mutex g_host_mu;
std::map<std::vector<double>, std::shared_ptr<const std::vector<char>>> g_host_tables;
std::deque<std::vector<double>> g_host_order;  // insertion order, for eviction
size_t g_host_bytes = 0;

std::shared_ptr<const std::vector<char>> host_table(const std::vector<double>& key, size_t bytes,
                                                    const std::function<void(char*)>& fill) {
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    auto it = g_host_tables.find(key);
    if (it != g_host_tables.end()) return it->second;
  }
  auto v = std::make_shared<std::vector<char>>(bytes);
  fill(v->data());
  std::lock_guard<std::mutex> lk(g_host_mu);
  // oldest entries out until the new one fits (contexts hold no reference: their
  // device copies were made at upload)
  while (!g_host_order.empty() && g_host_bytes + bytes > kMaxHostTableBytes) {
    auto it = g_host_tables.find(g_host_order.front());
    if (it != g_host_tables.end()) {
      g_host_bytes -= it->second->size();
      g_host_tables.erase(it);
    }
    g_host_order.pop_front();
  }
  if (g_host_tables.emplace(key, v).second) {
    g_host_order.push_back(key);
    g_host_bytes += bytes;
  }
  return v;
}

// Host-to-device uploads are staged through one pinned ring (allocated once per
// process) and copied asynchronously on the caller's stream, so an upload never
// waits for other work on that stream and never synchronises the device.  A
// ring region is reused once the copy that last read it has completed; that
// copy was issued a whole ring earlier.
#define CHECK_CUDA_RET(x)                   \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)
class UploadRing {
 public:
  cudaError_t copy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(mu_);
    if (!buf_) {
      cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&buf_), kCap, cudaHostAllocPortable);
      if (e != cudaSuccess) {
        buf_ = nullptr;
        return e;
      }
    }
    const char* in = static_cast<const char*>(src);
    char* out = static_cast<char*>(dst);
    for (size_t done = 0; done < bytes;) {
      const size_t len = std::min(bytes - done, kCap / 4);
      if (head_ + len > kCap) {
        // the tail past head_ is skipped: its copies, a lap old, must be done
        while (!live_.empty() && live_.front().off >= head_) CHECK_CUDA_RET(retire());
        head_ = 0;
      }
      while (!live_.empty() && live_.front().off < head_ + len && head_ < live_.front().off + live_.front().len)
        CHECK_CUDA_RET(retire());
      std::memcpy(buf_ + head_, in + done, len);
      cudaError_t e = cudaMemcpyAsync(out + done, buf_ + head_, len, cudaMemcpyHostToDevice, st);
      cudaEvent_t ev = nullptr;
      if (e == cudaSuccess) e = take(&ev);
      if (e == cudaSuccess) e = cudaEventRecord(ev, st);
      if (e != cudaSuccess) {
        // the copy may be in flight: wait for it before the region can be reused
        cudaStreamSynchronize(st);
        if (ev) spare_.push_back(ev);
        return e;
      }
      live_.push_back({head_, len, ev});
      head_ += len;
      done += len;
    }
    return cudaSuccess;
  }

 private:
  static constexpr size_t kCap = 64u << 20;
  struct Span {
    size_t off, len;
    cudaEvent_t ev;
  };
  cudaError_t retire() {
    Span s = live_.front();
    live_.pop_front();
    cudaError_t e = cudaEventSynchronize(s.ev);
    spare_.push_back(s.ev);
    return e;
  }
  cudaError_t take(cudaEvent_t* ev) {
    if (!spare_.empty()) {
      *ev = spare_.back();
      spare_.pop_back();
      return cudaSuccess;
    }
    return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  }
  std::mutex mu_;
  char* buf_ = nullptr;
  size_t head_ = 0;
  std::deque<Span> live_;
  std::vector<cudaEvent_t> spare_;
};
#undef CHECK_CUDA_RET

// One ring per device: a ring's events belong to the device current when they
// were created, and are recorded on that device's streams.
std::mutex g_ring_mu;
std::map<int, std::unique_ptr<UploadRing>> g_rings;

UploadRing* ring_of_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_ring_mu);
  auto& r = g_rings[dev];
  if (!r) r = std::make_unique<UploadRing>();
  return r.get();
}

// Large device-to-host copies into caller-owned pageable memory.  A plain
// cudaMemcpy of that kind runs at the speed of one host thread first-touching
// the destination pages (about 8 GB/s on the Grace host, against about 190
// GB/s for the device-to-pinned copy).  Here the data goes in chunks into two
// pinned slots (per device) while the previous chunk is copied out by several
// host threads at once.
class DownloadRing {
 public:
  cudaError_t copy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(mu_);
    if (!buf_[0]) {
      for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&buf_[i]), kChunk, cudaHostAllocPortable);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
      }
    }
    const char* in = static_cast<const char*>(src);
    char* out = static_cast<char*>(dst);
    const size_t n = (bytes + kChunk - 1) / kChunk;
    auto issue = [&](size_t i) {
      const size_t len = std::min(kChunk, bytes - i * kChunk);
      cudaError_t e = cudaMemcpyAsync(buf_[i & 1], in + i * kChunk, len, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaEventRecord(ev_[i & 1], st);
      return e;
    };
    cudaError_t e = issue(0);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
      if (i + 1 < n) e = issue(i + 1);  // its slot's previous chunk was copied out last iteration
      if (e == cudaSuccess) e = cudaEventSynchronize(ev_[i & 1]);
      if (e == cudaSuccess) parallel_copy(out + i * kChunk, buf_[i & 1], std::min(kChunk, bytes - i * kChunk));
    }
    if (e != cudaSuccess) cudaStreamSynchronize(st);  // no copy may still target a slot
    return e;
  }

 private:
  static constexpr size_t kChunk = (size_t)128 << 20;
  static void parallel_copy(char* dst, const char* src, size_t len) {
    const size_t kPart = (size_t)8 << 20;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t T = std::min<size_t>(std::min<size_t>(hw, 16), std::max<size_t>(1, len / kPart));
    std::vector<std::thread> th;
    const size_t per = (len + T - 1) / T;
    for (size_t t = 1; t < T; ++t) {
      const size_t a = t * per, b = std::min(len, a + per);
      if (a < b) th.emplace_back([=] { std::memcpy(dst + a, src + a, b - a); });
    }
    std::memcpy(dst, src, std::min(len, per));
    for (auto& x : th) x.join();
  }
  std::mutex mu_;
  char* buf_[2] = {nullptr, nullptr};
  cudaEvent_t ev_[2] = {nullptr, nullptr};
};

std::mutex g_down_mu;
std::map<int, std::unique_ptr<DownloadRing>> g_downs;

DownloadRing* download_ring() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_down_mu);
  auto& r = g_downs[dev];
  if (!r) r = std::make_unique<DownloadRing>();
  return r.get();
}

// Pinned host buffers of cola_pk_async results ([3 * kMaxBins] doubles each),
// recycled across contexts and never released: page-locked allocations and
// releases can synchronise the device, which a serving loop must not see.
class PinnedSlots {
 public:
  double* get() {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.empty()) {
      constexpr int kChunk = 32;
      const size_t each = 3 * (size_t)kMaxBins;
      double* p = nullptr;
      if (cudaHostAlloc(reinterpret_cast<void**>(&p), kChunk * each * sizeof(double), cudaHostAllocPortable) !=
          cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      for (int i = 0; i < kChunk; ++i) free_.push_back(p + i * each);
    }
    double* p = free_.back();
    free_.pop_back();
    return p;
  }
  void put(double* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    free_.push_back(p);
  }

 private:
  std::mutex mu_;
  std::vector<double*> free_;
};

PinnedSlots g_pk_slots;

int upload(cola_ctx* ctx, void* dst, const void* src, size_t bytes) {
  UploadRing* ring = ring_of_current_device();
  if (!ring) return fail(ctx, COLA_ECUDA, "upload: no current device");
  CK(ring->copy(dst, src, bytes, ctx->st));
  return COLA_OK;
}

// Twiddle table e^{-2 pi i m/N}, m = 0..N-1, computed in FP64.
int upload_twiddles(cola_ctx* ctx, int N, float2* dst) {
  std::vector<float2> t(N);
  for (int m = 0; m < N; ++m) {
    const double ang = -2.0 * kPi * m / N;
    t[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  return upload(ctx, dst, t.data(), t.size() * sizeof(float2));
}

// ---------------------------------------------------------------- context memory
// Every per-context device buffer lives in one allocation (one call of the
// allocator per context); each buffer starts on a 256-byte boundary.
struct Layout {
  struct Item {
    void** dst;
    size_t off;
  };
  std::vector<Item> items;
  size_t size = 0;
  template <class T>
  void add(T** p, size_t count) {
    items.push_back({reinterpret_cast<void**>(p), size});
    size += (count * sizeof(T) + 255) / 256 * 256;
  }
  void place(char* base) const {
    for (const auto& it : items) *it.dst = base + it.off;
  }
};

// Byte layout of a context's tables: [tab | vtab] float4 rows 0..nsteps+1 (rows
// as documented on SimHeader, plus row nsteps+1 = (1, 0, 0, 1), the Psi1 / Psi2
// pass of the scale-independent fast path), the per-step force parameters and
// the per-step time integrals.
struct TableLayout {
  size_t tab_b, fp_off, dt_off, g_off, bytes;
  explicit TableLayout(const cola_config& cfg) {
    const size_t ns = (size_t)cfg.nsteps, nk = (size_t)cfg.nk_table;
    tab_b = (ns + 2) * nk * sizeof(float4);
    fp_off = 2 * tab_b;
    dt_off = fp_off + (ns * sizeof(ForceParams) + 255) / 256 * 256;
    g_off = dt_off + (3 * ns * sizeof(float) + 255) / 256 * 256;  // [ns + 2] float2 row growth
    bytes = g_off + (ns + 2) * sizeof(float2);
  }
};

void context_layout(cola_ctx* c, const cola_config& cfg, Layout& L) {
  const int64_t P = (int64_t)cfg.Np * cfg.Np * cfg.Np, M = (int64_t)cfg.Nmesh * cfg.Nmesh * cfg.Nmesh;
  const int64_t hp = half_elems(cfg.Np), hm = half_elems(cfg.Nmesh);
  for (int d = 0; d < 3; ++d) {
    L.add(&c->s[d], P);
    L.add(&c->v[d], P);
    L.add(&c->acc[d], P);
  }
  for (int f = 0; f < 2; ++f) {
    L.add(&c->phi[f], hp);
    if (cfg.seed_precision) L.add(reinterpret_cast<uint32_t**>(&c->seedq[f]), hp);
  }
  for (int i = 0; i < 6; ++i) {
    L.add(&c->lc[i], hp);
    L.add(&c->lr[i], P);
    if (cfg.seed_precision) L.add(&c->lq[i], P);
  }
  if (!cfg.seed_precision)
    for (int d = 0; d < 3; ++d) L.add(&c->lrk[d], P);
  L.add(&c->rho, M);
  L.add(&c->Cd, hm);
  L.add(&c->Ck, hm);
  L.add(&c->Cw, hm);
  L.add(&c->Cphi, hm);
  L.add(&c->Cphz, hm);
  L.add(&c->F[0], 2 * M);
  L.add(&c->F[2], M);
  L.add(&c->pk_acc, 3 * kMaxBins);
  L.add(&c->hdr, 1);
  L.add(&c->scratch, 64);
  L.add(&c->tw_np, cfg.Np);
  L.add(&c->tw_nm, cfg.Nmesh);
  c->tables_bytes = TableLayout(cfg).bytes;
  L.add(&c->tables, c->tables_bytes);
}

ForceParams force_params(const cola_ctx* c, double a) {
  ForceParams fp{};
  const double Om = c->cfg.Omega_m;
  const double N3 = (double)c->Nm * c->Nm * c->Nm;
  fp.kf = (float)(2.0 * kPi / c->L);
  fp.kappa_norm = (float)(1.5 * Om * a / N3);
  fp.norm = (float)(1.0 / N3);
  fp.inv_rhobar = (float)(N3 / ((double)c->Np * c->Np * c->Np));
  fp.model = chameleon_kind(c->model.kind) ? COLA_FOFR : c->model.kind;  // screening family
  fp.screened = 0;
  if (c->model.kind == COLA_FOFR) {
    fp.C = (float)(1.0 / 3.0);
    fp.a2m2 = (float)(a * a * fr_m2(a, Om, c->model.fR0));
    fp.fr_thr = (float)(1.5 * fr_fR(a, Om, c->model.fR0) * a * a * kCLight * kCLight);
    fp.screened = c->model.screening ? 1 : 0;
  } else if (c->model.kind == COLA_SYMM) {
    // App. C: C = 2 beta^2(a), range 1/m(a), Phi_crit from the App. C integral (0 before a_*)
    const double u = symm_u(a, c->model.a_star);
    fp.C = (float)(2.0 * c->model.beta_star * c->model.beta_star * u);
    fp.a2m2 = (float)(a * a * c->model.m_star * c->model.m_star * u * kH0OverC * kH0OverC);
    fp.fr_thr = (float)(symm_phi_crit(a, Om, c->model.m_star, c->model.a_star) * a * a * kCLight * kCLight);
    fp.screened = c->model.screening ? 1 : 0;
  } else if (c->model.kind == COLA_MB) {
    // App. C with tabulated beta(a), m(a): C = 2 beta^2, range 1/m, Phi_crit from the integral
    double beta, M2, dM2;
    mb_eval(c->hm, a, beta, M2, dM2);
    fp.C = (float)(2.0 * beta * beta);
    fp.a2m2 = (float)(a * a * M2 * kH0OverC * kH0OverC);
    fp.fr_thr = (float)(mb_phi_crit(c->hm, a, Om) * a * a * kCLight * kCLight);
    fp.screened = c->model.screening ? 1 : 0;
  } else if (c->model.kind == COLA_NDGP) {
    const double b = dgp_beta(a, Om, c->model.rcH0);
    fp.C = (float)(1.0 / (3.0 * b));
    fp.a2m2 = 0.f;
    fp.dgp_coef = (float)(8.0 * c->model.rcH0 * c->model.rcH0 * Om / (9.0 * b * b));
    fp.R2half = (float)(0.5 * c->model.R_smooth * c->model.R_smooth);
    fp.filter = c->model.filter;
    fp.screened = c->model.screening ? 1 : 0;
  }
  return fp;
}

// 3-D transforms on the internal half-spectrum layout (plane pairs interleaved
// in 64-byte chunks, cola_internal.h).
int r2c3(cola_ctx* ctx, int N, const float* in, float2* out, const float2* tw, float scale,
         float offset, Multi m = {}) {
  CK(fft_xr2c(N, in, out, scale, offset, tw, ctx->st, m));
  CK(fft_col(N, out, 1, false, tw, ctx->st, m));
  CK(fft_col(N, out, 2, false, tw, ctx->st, m));
  return COLA_OK;
}

int c2r3(cola_ctx* ctx, int N, float2* in, float* out, const float2* tw, Multi m = {}) {
  CK(fft_col(N, in, 2, true, tw, ctx->st, m));
  CK(fft_col(N, in, 1, true, tw, ctx->st, m));
  CK(fft_xc2r(N, in, out, 0.f, tw, ctx->st, m));
  return COLA_OK;
}

// Sec. 4.1 / App. A: LPT fields at the lattice from the k-space seeds and one
// row of table `vel` (0 displacement/acceleration, 1 velocity): row0, plus the
// device step counter when add_step; over m's simulations (ctx is the first).
int run_lpt(cola_ctx* ctx, int vel, int row0, bool add_step, Multi m = {}, float* zero_dst = nullptr,
            int64_t zero_floats = 0, bool* zeroed = nullptr, int kslot = 0) {
  LptParams lp{};
  lp.hdr = ctx->hdr;
  lp.vel = vel;
  lp.row0 = row0;
  lp.add_step = add_step ? 1 : 0;
  lp.lnk0 = (float)ctx->lnk0;
  lp.inv_dlnk = (float)(1.0 / ctx->dlnk);
  lp.nk = ctx->nk;
  lp.kf = (float)(2.0 * kPi / ctx->L);
  lp.norm = (float)(1.0 / ((double)ctx->Np * ctx->Np * ctx->Np));
  lp.seed_prec = ctx->cfg.seed_precision;
  const void* p1 = lp.seed_prec ? ctx->seedq[0] : (const void*)ctx->phi[0];
  const void* p2 = lp.seed_prec ? ctx->seedq[1] : (const void*)ctx->phi[1];
  const int N = ctx->Np;
  const float kf = lp.kf;
  auto st = ctx->st;
  const double H = (double)N * N * (N / 2 + 1) * 8.0, R = (double)N * N * N * 4.0;
  const double seedH = H * (lp.seed_prec ? 0.5 : 1.0);
  cudaEvent_t e = prof_begin(ctx, ST_LPT_Z);
  bool zd = false;
  CK(lpt_z(N, p1, p2, ctx->lc[0], ctx->lc[1], ctx->lc[2], ctx->lc[3], lp, ctx->tw_np, st, m, zero_dst,
           zero_floats, &zd));
  if (zeroed) *zeroed = zd;
  prof_end(ctx, ST_LPT_Z, e, 1, m.nb * (2 * seedH + 4 * H + (zd ? 4.0 * (double)zero_floats : 0.0)));
  // variant a.S1: the per-step drift and kick fields leave the x pass as 16-bit
  // values (one FP32 scale per field, delayed scaling)
  const bool q16 = lp.seed_prec != 0 && vel == 0 && add_step;
  if (N <= 128 && !q16) {
    // y and x steps of the six outputs in one pass per (plane, field)
    e = prof_begin(ctx, ST_LPT_X);
    float* const* ko = kslot ? ctx->lrk : ctx->lr + 3;
    const float2* in4[4] = {ctx->lc[0], ctx->lc[1], ctx->lc[2], ctx->lc[3]};
    float* out6[6] = {ctx->lr[0], ctx->lr[1], ctx->lr[2], ko[0], ko[1], ko[2]};
    bool zp = false;
    CK(fft_plane_lpt(N, in4, out6, kf, ctx->tw_np, st, m, zd ? nullptr : zero_dst, zero_floats, &zp));
    if (zeroed) *zeroed = zd || zp;
    prof_end(ctx, ST_LPT_X, e, 1, m.nb * (4 * H + 6 * R + (zp ? 4.0 * (double)zero_floats : 0.0)));
    ctx->have_lpt = true;
    return COLA_OK;
  }
  e = prof_begin(ctx, ST_LPT_Y);
  CK(fft_yinv2(N, ctx->lc[0], ctx->lc[0], ctx->lc[4], kf, ctx->tw_np, st, m));
  CK(fft_col(N, ctx->lc[1], 1, true, ctx->tw_np, st, m));
  CK(fft_yinv2(N, ctx->lc[2], ctx->lc[2], ctx->lc[5], kf, ctx->tw_np, st, m));
  CK(fft_col(N, ctx->lc[3], 1, true, ctx->tw_np, st, m));
  prof_end(ctx, ST_LPT_Y, e, 4, m.nb * 10.0 * H);
  e = prof_begin(ctx, ST_LPT_X);
  {
    const float2* in6[6] = {ctx->lc[0], ctx->lc[4], ctx->lc[1], ctx->lc[2], ctx->lc[5], ctx->lc[3]};
    const float kfs6[6] = {kf, 0.f, 0.f, kf, 0.f, 0.f};
    if (q16) {
      void* out6[6] = {ctx->lq[0], ctx->lq[1], ctx->lq[2], ctx->lq[3], ctx->lq[4], ctx->lq[5]};
      CK(fft_xc2r_multi16(N, 6, in6, out6, kfs6, lp.seed_prec, ctx->hdr, ctx->tw_np, st, m));
      CK(lq_update(ctx->hdr, lp.seed_prec, ctx->cfg.nsteps, st, m));
    } else {
      float* const* ko = kslot ? ctx->lrk : ctx->lr + 3;
      float* out6[6] = {ctx->lr[0], ctx->lr[1], ctx->lr[2], ko[0], ko[1], ko[2]};
      CK(fft_xc2r_multi(N, 6, in6, out6, kfs6, ctx->tw_np, st, m));
    }
  }
  prof_end(ctx, ST_LPT_X, e, q16 ? 2 : 1, m.nb * 6 * (H + (q16 ? 0.5 : 1.0) * R));
  ctx->have_lpt = true;
  return COLA_OK;
}

// Simulations advanced by one launch sequence: `all` moves the pointers of
// `lead` to every one of them; the model-dependent force stages run over the
// subsets (each with its own first context and shifts).
struct Group {
  struct Sub {
    cola_ctx* lead = nullptr;
    Multi m;
  };
  cola_ctx* lead = nullptr;
  Multi all;
  Sub unscreened, fr_screened, dgp_screened, screened;
};

Group single_group(cola_ctx* ctx) {
  Group g;
  g.lead = ctx;
  const Group::Sub me{ctx, Multi{}};
  const bool scr = ctx->model.kind != COLA_LCDM && ctx->model.screening;
  if (!scr) g.unscreened = me;
  else if (chameleon_kind(ctx->model.kind)) g.fr_screened = g.screened = me;
  else g.dgp_screened = g.screened = me;
  return g;
}

// App. B: mesh force -grad(Phi_N + phi) at scale factor a from the density in
// rho, for every simulation of g.  device_params: each simulation's values
// come from its header, those of its current step or (ini) those at a_ini (a
// is then only used for the model flags); otherwise the values at a (single
// simulation).
int force_group(const Group& g, double a, bool device_params, bool ini = false) {
  cola_ctx* ctx = g.lead;
  const Multi all = g.all;
  auto fp_of = [&](cola_ctx* c) {
    ForceParams fp = force_params(c, a);
    if (device_params) {
      fp.hdr = c->hdr;
      fp.ini = ini ? 1 : 0;
    }
    return fp;
  };
  const ForceParams fp = fp_of(ctx);
  const int N = ctx->Nm;
  auto st = ctx->st;
  const float2* tw = ctx->tw_nm;
  const double H = (double)N * N * (N / 2 + 1) * 8.0, R = (double)N * N * N * 4.0;
  // up to 128 points the x and y steps of each transform run plane by plane in one pass
  const bool plane = N <= 128;
  cudaEvent_t e = prof_begin(ctx, ST_MESH_XR2C);
  if (plane) {
    CK(fft_plane_r2c(N, ctx->rho, ctx->Cd, fp.inv_rhobar, -1.f, tw, st, all));
  } else {
    CK(fft_xr2c(N, ctx->rho, ctx->Cd, fp.inv_rhobar, -1.f, tw, st, all));
  }
  prof_end(ctx, ST_MESH_XR2C, e, 1, all.nb * (R + H));
  if (!plane) {
    e = prof_begin(ctx, ST_MESH_Y);
    CK(fft_col(N, ctx->Cd, 1, false, tw, st, all));
    prof_end(ctx, ST_MESH_Y, e, 1, all.nb * 2 * H);
  }
  if (const Group::Sub& sc = g.screened; sc.lead) {
    e = prof_begin(ctx, ST_Z_SCREEN_FIELD);
    for (const Group::Sub* sub : {&g.fr_screened, &g.dgp_screened})
      if (sub->lead)
        CK(mesh_z_screen_field(N, sub->lead->Cd, sub->lead->Ck, sub->lead->Cw, fp_of(sub->lead), tw, st,
                               sub->m));
    prof_end(ctx, ST_Z_SCREEN_FIELD, e, (g.fr_screened.lead ? 1 : 0) + (g.dgp_screened.lead ? 1 : 0),
             sc.m.nb * 3 * H);
    if (plane) {
      // y inverse, x c2r, S = delta eps, x r2c and y forward in one pass per plane
      e = prof_begin(ctx, ST_X_SCREEN_SOURCE);
      for (const Group::Sub* sub : {&g.fr_screened, &g.dgp_screened})
        if (sub->lead)
          CK(fft_plane_screen(N, sub->lead->Cw, sub->lead->rho, sub->lead->Cd, fp_of(sub->lead), tw, st,
                              sub->m));
      prof_end(ctx, ST_X_SCREEN_SOURCE, e, (g.fr_screened.lead ? 1 : 0) + (g.dgp_screened.lead ? 1 : 0),
               sc.m.nb * (2 * H + R));
    } else {
      e = prof_begin(ctx, ST_MESH_YINV);
      CK(fft_col(N, sc.lead->Cw, 1, true, tw, st, sc.m));
      prof_end(ctx, ST_MESH_YINV, e, 1, sc.m.nb * 2 * H);
      e = prof_begin(ctx, ST_X_SCREEN_SOURCE);
      for (const Group::Sub* sub : {&g.fr_screened, &g.dgp_screened})
        if (sub->lead)
          CK(mesh_x_screen_source(N, sub->lead->Cw, sub->lead->rho, sub->lead->Cd, fp_of(sub->lead), tw,
                                  st, sub->m));
      prof_end(ctx, ST_X_SCREEN_SOURCE, e, (g.fr_screened.lead ? 1 : 0) + (g.dgp_screened.lead ? 1 : 0),
               sc.m.nb * (2 * H + R));
      e = prof_begin(ctx, ST_MESH_Y);
      CK(fft_col(N, sc.lead->Cd, 1, false, tw, st, sc.m));
      prof_end(ctx, ST_MESH_Y, e, 1, sc.m.nb * 2 * H);
    }
    e = prof_begin(ctx, ST_Z_FORCE);
    CK(mesh_z_force(N, sc.lead->Cd, sc.lead->Ck, sc.lead->Cphi, sc.lead->Cphz, fp_of(sc.lead), tw, st,
                    sc.m));
    prof_end(ctx, ST_Z_FORCE, e, 1, sc.m.nb * 4 * H);
  }
  if (const Group::Sub& un = g.unscreened; un.lead) {
    e = prof_begin(ctx, ST_Z_FORCE);
    CK(mesh_z_force(N, un.lead->Cd, nullptr, un.lead->Cphi, un.lead->Cphz, fp_of(un.lead), tw, st,
                    un.m));
    prof_end(ctx, ST_Z_FORCE, e, 1, un.m.nb * 3 * H);
  }
  if (plane) {
    e = prof_begin(ctx, ST_MESH_XC2R);
    CK(fft_plane_force(N, ctx->Cphi, ctx->Cphz, ctx->F[0], ctx->F[1], ctx->F[2], -fp.kf, tw, st, all));
    prof_end(ctx, ST_MESH_XC2R, e, 1, all.nb * (2 * H + 3 * R));
  } else {
    e = prof_begin(ctx, ST_MESH_YINV);
    CK(fft_yinv2(N, ctx->Cphi, ctx->Cphi, ctx->Cw, -fp.kf, tw, st, all));
    CK(fft_col(N, ctx->Cphz, 1, true, tw, st, all));
    prof_end(ctx, ST_MESH_YINV, e, 2, all.nb * 5.0 * H);
    e = prof_begin(ctx, ST_MESH_XC2R);
    const float2* in3[3] = {ctx->Cphi, ctx->Cw, ctx->Cphz};
    if (ctx->fpairs) {
      // F_x and F_y as the (x, y) pairs of the interleaved mesh in F[0]
      CK(fft_xc2r_pair(N, ctx->Cphi, ctx->Cw, ctx->F[0], -fp.kf, tw, st, all));
      const float kfs_z = 0.f;
      CK(fft_xc2r_multi(N, 1, in3 + 2, ctx->F + 2, &kfs_z, tw, st, all));
    } else {
      float* out3[3] = {ctx->F[0], ctx->F[1], ctx->F[2]};
      const float kfs3[3] = {-fp.kf, 0.f, 0.f};
      CK(fft_xc2r_multi(N, 3, in3, out3, kfs3, tw, st, all));
    }
    prof_end(ctx, ST_MESH_XC2R, e, ctx->fpairs ? 2 : 1, all.nb * 3 * (H + R));
  }
  ctx->have_force = true;
  return COLA_OK;
}

int run_force(cola_ctx* ctx, double a, bool device_params = false) {
  return force_group(single_group(ctx), a, device_params);
}

PartParams part_params(const cola_ctx* c) {
  PartParams pp;
  pp.Np = c->Np;
  pp.Nm = c->Nm;
  pp.lgNp = c->lgNp;
  pp.cellscale = (float)(c->Nm / c->L);
  pp.L = (float)c->L;
  return pp;
}

// The spectrum of the initial conditions in device form.
EHDev eh_dev(const cola_ctx* ctx) {
  const int N = ctx->Np;
  EHDev eh;
  eh.theta2 = ctx->eh.theta2;
  eh.s = ctx->eh.s;
  eh.alpha = ctx->eh.alpha;
  eh.Omh = ctx->eh.Omh;
  eh.h = ctx->eh.h;
  eh.ns = ctx->eh.ns;
  eh.amp = ctx->eh.amp * ctx->Dratio * ctx->Dratio;
  eh.N3_over_L3 = (double)N * N * N / (ctx->L * ctx->L * ctx->L);
  return eh;
}

// LPT mixing parameters of the fast path: coefficients from row row0 (+ the
// device step when add_step) of the table (vtab when vel); Psi2 in lr[3..5].
LptMix lpt_mix_of(const cola_ctx* ctx, int row0, int add_step, bool vel) {
  LptMix x{};
  x.hdr = ctx->hdr;
  for (int d = 0; d < 3; ++d) x.q2[d] = ctx->lr[3 + d];
  x.on = 1;
  x.vel = vel ? 1 : 0;
  x.row0 = row0;
  x.add_step = add_step;
  x.nk = ctx->nk;
  return x;
}

// Initial conditions (Sec. 3, Sec. 4.1, App. A) of every simulation of g on
// g.lead->st: white noise from each one's seed, phi1 = delta/k^2, the 2LPT phi2
// (skipped when `potentials`: phi1 and phi2 are already in place), the
// reduced-precision seeds, the particles on the LPT trajectory at a_ini, and the
// initial force and residual acceleration.  Per-simulation values (seed,
// spectrum, force parameters at a_ini, seed scales) live in the headers, which
// must hold step 0 before this runs.
int ic_group(const Group& g, bool potentials) {
  cola_ctx* ctx = g.lead;
  const Multi m = g.all;
  const int N = ctx->Np;
  auto st = ctx->st;
  const float kf = (float)(2.0 * kPi / ctx->L);
  if (!potentials) {
    CK(ic_noise(N, ctx->cfg.seed, ctx->lr[0], st, m, ctx->hdr));
    CHECK_RC(r2c3(ctx, N, ctx->lr[0], ctx->phi[0], ctx->tw_np, 1.f, 0.f, m));
    // lr[1] is free until the Hessians: the per-|n|^2 factor table
    CK(ic_phi1(N, ctx->phi[0], kf, eh_dev(ctx), reinterpret_cast<double*>(ctx->lr[1]), st, m, ctx->hdr));
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int h = 0; h < 6; ++h) {
      CK(ic_hessian(N, ctx->phi[0], ctx->lc[0], ij[h][0], ij[h][1], kf, st, m));
      CHECK_RC(c2r3(ctx, N, ctx->lc[0], ctx->lr[h], ctx->tw_np, m));
    }
    float* src = reinterpret_cast<float*>(ctx->lc[1]);
    CK(ic_source(ctx->P, ctx->lr[0], ctx->lr[1], ctx->lr[2], ctx->lr[3], ctx->lr[4], ctx->lr[5], src, st,
                 m));
    CHECK_RC(r2c3(ctx, N, src, ctx->phi[1], ctx->tw_np, 1.f, 0.f, m));
    CK(ic_phi2(N, ctx->phi[1], kf, st, m));
  }
  if (ctx->cfg.seed_precision) {
    for (int f = 0; f < 2; ++f) {
      CK(seed_absmax(N, ctx->phi[f], ctx->scratch, st, m));
      CK(seed_scale_set(ctx->hdr, ctx->scratch, f, st, m));
      CK(seed_quantise(N, ctx->phi[f], ctx->seedq[f], ctx->cfg.seed_precision, ctx->hdr, f, st, m));
    }
  }
  const PartParams pp = part_params(ctx);
  if (ctx->lpt_fast) {
    // Psi1, Psi2 once (table row nsteps+1), then the particles and A_LPT at a_ini
    // as combinations with row 0's coefficients
    CHECK_RC(run_lpt(ctx, 0, ctx->cfg.nsteps + 1, false, m));
    const LptMix mix = lpt_mix_of(ctx, 0, 0, false);
    CK(ic_particles(ctx->P, ctx->lr[0], ctx->lr[1], ctx->lr[2], ctx->s[0], ctx->s[1], ctx->s[2],
                    ctx->v[0], ctx->v[1], ctx->v[2], st, m, mix));
    CK(zero_f32(ctx->rho, ctx->M, st, m));
    CK(part_deposit(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->rho, ctx->P, st, m));
    CHECK_RC(force_group(g, ctx->a[0], true, true));
    CK(part_gather_kick(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                        ctx->acc[0], ctx->acc[1], ctx->acc[2], ctx->lr[0], ctx->lr[1], ctx->lr[2],
                        ctx->F[0], ctx->F[1], ctx->F[2], ctx->fpairs, StepDt{nullptr, 0.f, 0.f}, ctx->P, st, m,
                        mix));
    return COLA_OK;
  }
  CHECK_RC(run_lpt(ctx, 0, 0, false, m));
  if (ctx->cfg.seed_precision) {
    // first scales of the 16-bit per-step fields: the drift and kick fields at a_ini
    const float* f6[6] = {ctx->lr[0], ctx->lr[1], ctx->lr[2], ctx->lr[3], ctx->lr[4], ctx->lr[5]};
    CK(lq_init(ctx->hdr, f6, ctx->P, ctx->cfg.seed_precision, st, m));
  }
  CK(ic_particles(ctx->P, ctx->lr[0], ctx->lr[1], ctx->lr[2], ctx->s[0], ctx->s[1], ctx->s[2],
                  ctx->v[0], ctx->v[1], ctx->v[2], st, m));
  CK(zero_f32(ctx->rho, ctx->M, st, m));
  CK(part_deposit(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->rho, ctx->P, st, m));
  CHECK_RC(force_group(g, ctx->a[0], true, true));
  CK(part_gather_kick(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                      ctx->acc[0], ctx->acc[1], ctx->acc[2], ctx->lr[3], ctx->lr[4], ctx->lr[5],
                      ctx->F[0], ctx->F[1], ctx->F[2], ctx->fpairs, StepDt{nullptr, 0.f, 0.f}, ctx->P, st,
                      m));
  return COLA_OK;
}

// One context's initial conditions on its own stream.
int finish_ic(cola_ctx* ctx, bool potentials) {
  ctx->hh.step = 0;
  CK(set_header(ctx->hdr, ctx->hh, ctx->st));
  CHECK_RC(ic_group(single_group(ctx), potentials));
  ctx->step = 0;
  ctx->ic_done = true;
  return COLA_OK;
}

// The device address of page-locked host memory at p (registered or allocated by
// cudaHostAlloc and mapped, as every such allocation is with unified addressing),
// or nullptr for other memory.
void* mapped_host(void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Device-to-host copy into caller memory, synchronous for the caller: large
// copies without a wait limit go through the download ring, the rest through
// cudaMemcpyAsync and a (bounded) wait.
int copy_to_host(cola_ctx* ctx, void* dst, const void* src, size_t bytes) {
  // page-locked destinations take the copy engine straight; large pageable ones go
  // through the pinned download ring
  cudaPointerAttributes at{};
  const bool pinned = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost;
  if (!pinned) cudaGetLastError();
  if (!pinned && bytes >= ((size_t)64 << 20) && !(ctx->wait_limit_s > 0)) {
    DownloadRing* r = download_ring();
    if (!r) return fail(ctx, COLA_ECUDA, "no current device");
    CK(r->copy(dst, src, bytes, ctx->st));
    return COLA_OK;
  }
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->st));
  return host_wait(ctx);
}

int copy_out(cola_ctx* ctx, void* dst, const void* src, size_t bytes, int where) {
  if (where == COLA_HOST) return copy_to_host(ctx, dst, src, bytes);
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->st));
  return COLA_OK;
}

// The force mesh as three component arrays of M floats at d (F_x, F_y, F_z), host
// or device; pairs are split on the device (straight into device destinations,
// through the free complex work buffers for host ones).
int export_force(cola_ctx* ctx, char* d, int where) {
  const size_t mb = (size_t)ctx->M * sizeof(float);
  if (!ctx->fpairs) {
    for (int c = 0; c < 3; ++c) CHECK_RC(copy_out(ctx, d + c * mb, ctx->F[c], mb, where));
    return COLA_OK;
  }
  const float2* fxy = reinterpret_cast<const float2*>(ctx->F[0]);
  if (where == COLA_DEVICE) {
    CK(split_pairs(fxy, reinterpret_cast<float*>(d), reinterpret_cast<float*>(d + mb), ctx->M, ctx->st));
  } else {
    float* x = reinterpret_cast<float*>(ctx->Cphi);
    float* y = reinterpret_cast<float*>(ctx->Cphz);
    CK(split_pairs(fxy, x, y, ctx->M, ctx->st));
    CHECK_RC(copy_out(ctx, d, x, mb, where));
    CHECK_RC(copy_out(ctx, d + mb, y, mb, where));
  }
  return copy_out(ctx, d + 2 * mb, ctx->F[2], mb, where);
}

int copy_in(cola_ctx* ctx, void* dst, const void* src, size_t bytes, int where) {
  CK(cudaMemcpyAsync(dst, src, bytes, where == COLA_HOST ? cudaMemcpyHostToDevice
                                                         : cudaMemcpyDeviceToDevice, ctx->st));
  if (where == COLA_HOST) return host_wait(ctx);
  return COLA_OK;
}

// Dense [N][N][N/2+1] complex copy of a padded half spectrum (tmp: device dense buffer).
int export_half(cola_ctx* ctx, int N, const float2* padded, float2* tmp, void* dst, int where) {
  const size_t bytes = (size_t)N * N * (N / 2 + 1) * sizeof(float2);
  if (where == COLA_DEVICE) {
    CK(half_unpack(N, padded, static_cast<float2*>(dst), ctx->st));
    return COLA_OK;
  }
  CK(half_unpack(N, padded, tmp, ctx->st));
  return copy_out(ctx, dst, tmp, bytes, where);
}

// Enqueues the next step (Sec. 2, a_n -> a_{n+1}) of every simulation of g on
// g.lead->st without touching the host step counters.  The step index comes
// from each simulation's device header, so the launch sequence is the same for
// every step.  n is the host's step index, used only for the model flags.
int enqueue_group_tail(const Group& g, int kslot);

int enqueue_group_step(const Group& g, int n, bool head_only = false) {
  cola_ctx* ctx = g.lead;
  const Multi m = g.all;
  const PartParams pp = part_params(ctx);
  const double Pb = (double)ctx->P, Mb = (double)ctx->M;
  const StepDt dt0{ctx->hdr, 0.f, 0.f};
  // fast path: the step's LPT fields are combinations of Psi1, Psi2 formed in
  // the particle kernels (row 1 + step), no LPT transforms
  const bool fast = ctx->lpt_fast;
  const LptMix mix = fast ? lpt_mix_of(ctx, 1, 1, false) : LptMix{};
  // the density zero fill rides on the LPT z pass where that pass can take it
  bool rho_zeroed = false;
  if (!fast) CHECK_RC(run_lpt(ctx, 0, 1, true, m, ctx->rho, ctx->M, &rho_zeroed));
  // variant a.S1: the drift and kick read the 16-bit fields
  const int lq = (!fast && ctx->cfg.seed_precision) ? ctx->cfg.seed_precision : 0;
  StepDt dt = dt0;
  dt.lq = lq;
  const float* ld[3] = {ctx->lr[0], ctx->lr[1], ctx->lr[2]};
  const float* lk[3] = {ctx->lr[3], ctx->lr[4], ctx->lr[5]};
  if (lq)
    for (int d = 0; d < 3; ++d) {
      ld[d] = reinterpret_cast<const float*>(ctx->lq[d]);
      lk[d] = reinterpret_cast<const float*>(ctx->lq[3 + d]);
    }
  cudaEvent_t e = nullptr;
  if (!rho_zeroed) {
    e = prof_begin(ctx, ST_RHO_ZERO);
    CK(zero_f32(ctx->rho, ctx->M, ctx->st, m));
    prof_end(ctx, ST_RHO_ZERO, e, 1, m.nb * 4.0 * Mb);
  }
  e = prof_begin(ctx, ST_DRIFT_DEPOSIT);
  CK(part_drift_deposit(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                        ctx->acc[0], ctx->acc[1], ctx->acc[2], ld[0], ld[1], ld[2], ctx->rho, dt,
                        ctx->P, ctx->st, m, mix));
  prof_end(ctx, ST_DRIFT_DEPOSIT, e, 1, m.nb * ((fast ? 84.0 : lq ? 66.0 : 72.0) * Pb + 8.0 * Mb));
  CHECK_RC(force_group(g, ctx->a[n + 1], true));
  if (head_only) return COLA_OK;
  return enqueue_group_tail(g, 0);
}

// The kick that ends a step (the force of the step is in F) and the device step
// advance; the step's kick fields are in slot kslot (see cola_ctx::lrk).
int enqueue_group_tail(const Group& g, int kslot) {
  cola_ctx* ctx = g.lead;
  const Multi m = g.all;
  const PartParams pp = part_params(ctx);
  const double Pb = (double)ctx->P, Mb = (double)ctx->M;
  const bool fast = ctx->lpt_fast;
  const LptMix mix = fast ? lpt_mix_of(ctx, 1, 1, false) : LptMix{};
  const int lq = (!fast && ctx->cfg.seed_precision) ? ctx->cfg.seed_precision : 0;
  StepDt dt{ctx->hdr, 0.f, 0.f};
  dt.lq = lq;
  const float* lk[3] = {ctx->lr[3], ctx->lr[4], ctx->lr[5]};
  if (kslot)
    for (int d = 0; d < 3; ++d) lk[d] = ctx->lrk[d];
  if (lq)
    for (int d = 0; d < 3; ++d) lk[d] = reinterpret_cast<const float*>(ctx->lq[3 + d]);
  cudaEvent_t e = prof_begin(ctx, ST_GATHER_KICK);
  if (fast)  // A_LPT: Psi1 (lr[0..2]) mixed with Psi2
    for (int d = 0; d < 3; ++d) lk[d] = ctx->lr[d];
  CK(part_gather_kick(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                      ctx->acc[0], ctx->acc[1], ctx->acc[2], lk[0], lk[1], lk[2], ctx->F[0],
                      ctx->F[1], ctx->F[2], ctx->fpairs, dt, ctx->P, ctx->st, m, mix));
  prof_end(ctx, ST_GATHER_KICK, e, 1, m.nb * ((fast ? 72.0 : lq ? 54.0 : 60.0) * Pb + 12.0 * Mb));
  CK(step_advance(ctx->hdr, ctx->st, m));
  ctx->kslot = kslot;  // multi-simulation groups use slot 0 (their callers reset every member)
  return COLA_OK;
}

int enqueue_step(cola_ctx* ctx, int n) { return enqueue_group_step(single_group(ctx), n); }

// K >= 2 consecutive steps of one simulation (Sec. 2) with the kick of each step
// but the last and the drift + deposit of the next in one pass
// (k_kick_drift_deposit): step n+1's LPT fields are formed before step n's kick,
// its kick fields into the other slot.  The particle state after the K steps is
// the one K separate steps leave.  FP32 fields, per-k LPT path.
bool fused_steps_ok(const cola_ctx* ctx, int K) {
  return K >= 2 && !ctx->lpt_fast && !ctx->cfg.seed_precision && ctx->lrk[0] != nullptr;
}

// The boundary between step n and step n + 1 of every simulation of g in the
// fused form: step n+1's LPT fields (table row 2 + device step n; drift fields
// into lr[0..2], kick fields into slot 1 - cur), the kick of step n (its kick
// fields in slot cur) with the drift + deposit of step n + 1 in one pass, the
// device step advance and the force of step n + 1.
int enqueue_group_mid(const Group& g, int n, int cur) {
  cola_ctx* ctx = g.lead;
  const Multi m = g.all;
  const PartParams pp = part_params(ctx);
  const double Pb = (double)ctx->P, Mb = (double)ctx->M;
  bool zeroed = false;
  CHECK_RC(run_lpt(ctx, 0, 2, true, m, ctx->rho, ctx->M, &zeroed, 1 - cur));
  if (!zeroed) {
    cudaEvent_t e = prof_begin(ctx, ST_RHO_ZERO);
    CK(zero_f32(ctx->rho, ctx->M, ctx->st, m));
    prof_end(ctx, ST_RHO_ZERO, e, 1, m.nb * 4.0 * Mb);
  }
  const float* const* ka = cur ? ctx->lrk : ctx->lr + 3;
  cudaEvent_t e = prof_begin(ctx, ST_KICK_DRIFT_DEPOSIT);
  CK(part_kick_drift_deposit(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2], ka[0], ka[1],
                             ka[2], ctx->lr[0], ctx->lr[1], ctx->lr[2], ctx->F[0], ctx->F[1], ctx->F[2],
                             ctx->fpairs, ctx->rho,
                             ctx->hdr, ctx->P, ctx->st, m));
  prof_end(ctx, ST_KICK_DRIFT_DEPOSIT, e, 1, m.nb * (72.0 * Pb + 20.0 * Mb));
  CK(step_advance(ctx->hdr, ctx->st, m));
  return force_group(g, ctx->a[n + 2], true);
}

int enqueue_steps_fused(cola_ctx* ctx, int K) {
  const Group g = single_group(ctx);
  CHECK_RC(enqueue_group_step(g, ctx->step, true));  // LPT, drift + deposit, force of the first step
  int cur = 0;
  for (int i = 1; i < K; ++i) {
    CHECK_RC(enqueue_group_mid(g, ctx->step, cur));
    ctx->step += 1;
    cur = 1 - cur;
  }
  CHECK_RC(enqueue_group_tail(g, cur));
  ctx->step += 1;
  return COLA_OK;
}

// Launch sequences a batch graph holds: a whole step, or the pieces of a run of
// fused steps (the first step's head; a boundary with the kick fields of the
// ending step in slot 0 or 1; the last step's tail from slot 0 or 1).
enum BatchKind { BK_STEP, BK_HEAD, BK_MID0, BK_MID1, BK_TAIL0, BK_TAIL1 };

int enqueue_kind(const Group& g, int n, int kind) {
  switch (kind) {
    case BK_STEP: return enqueue_group_step(g, n);
    case BK_HEAD: return enqueue_group_step(g, n, true);
    case BK_MID0: case BK_MID1: return enqueue_group_mid(g, n, kind - BK_MID0);
    default: return enqueue_group_tail(g, kind - BK_TAIL0);
  }
}

}  // namespace

extern "C" {

int cola_init(const cola_config* cfg, cola_alloc_fn alloc, cola_free_fn free_fn, void* user,
              void* stream, cola_ctx** out) {
  if (!out) return fail(nullptr, COLA_EINVAL, "out is NULL");
  *out = nullptr;
  {
    int rc = validate_cfg(cfg, nullptr);
    if (rc) return rc;
  }
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, COLA_EINVAL, "give both alloc and free callbacks or neither");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, COLA_ECUDA, "no CUDA device available");
  }
  {
    // the allocation-free P(k) scratch is reserved on this device now (see cola_pk_noalloc)
    int rc = pk_noalloc_reserve();
    if (rc) return rc;
  }
  cola_ctx* ctx = new cola_ctx();
  ctx->cfg = *cfg;
  ctx->st = static_cast<cudaStream_t>(stream);
  ctx->alloc = alloc;
  ctx->freef = free_fn;
  ctx->user = user;
  ctx->Np = cfg->Np;
  ctx->Nm = cfg->Nmesh;
  ctx->lgNp = ilog2i(cfg->Np);
  ctx->L = cfg->Lbox;
  ctx->nk = cfg->nk_table;
  ctx->P = (int64_t)cfg->Np * cfg->Np * cfg->Np;
  ctx->M = (int64_t)cfg->Nmesh * cfg->Nmesh * cfg->Nmesh;
  ctx->a = a_nodes(*cfg);
  const double Om = cfg->Omega_m;
  {
    // the time integrals depend only on (Omega_m, z_ini, z_final, nsteps): computed once per key
    static std::mutex mu;
    static std::map<std::vector<double>, std::vector<double>> cache;
    const std::vector<double> key = {Om, cfg->z_ini, cfg->z_final, (double)cfg->nsteps};
    std::vector<double> tau;
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(key);
      if (it != cache.end()) tau = it->second;
    }
    if (tau.empty()) {
      for (int n = 0; n < cfg->nsteps; ++n) {
        const double a0 = ctx->a[n], a1 = ctx->a[n + 1], am = 0.5 * (a0 + a1);
        tau.push_back(hdtau(a0, am, Om));
        tau.push_back(hdtau(a0, a1, Om));
        tau.push_back(hdtau(am, a1, Om));
      }
      std::lock_guard<std::mutex> lk(mu);
      if (cache.size() > 4096) cache.clear();
      cache.emplace(key, tau);
    }
    for (int n = 0; n < cfg->nsteps; ++n) {
      ctx->dtk1.push_back(tau[3 * n]);
      ctx->dtd.push_back(tau[3 * n + 1]);
      ctx->dtk2.push_back(tau[3 * n + 2]);
    }
  }
  std::vector<double> kdummy;
  k_nodes(*cfg, ctx->lnk0, ctx->dlnk, kdummy);
  int rc = COLA_OK;
  {
    Layout lay;
    context_layout(ctx, *cfg, lay);
    void* slab = dev_alloc(ctx, lay.size);
    if (!slab) {
      rc = fail(ctx, COLA_ENOMEM, "device allocation of " + std::to_string(lay.size) + " bytes failed");
    } else if (reinterpret_cast<uintptr_t>(slab) & 255) {
      // the kernels' 16-byte vector accesses, bulk copies and tensor maps rely on
      // every buffer starting on a 256-byte boundary (the slab's offsets keep it)
      dev_free(ctx, slab);
      rc = fail(ctx, COLA_EINVAL, "the allocator returned a block not aligned to 256 bytes");
    } else {
      ctx->allocs.push_back(slab);
      lay.place(static_cast<char*>(slab));
      ctx->F[1] = ctx->F[0] + ctx->M;
      ctx->fpairs = ctx->Nm > 128;  // the plane passes (N <= 128) write plain components
    }
  }
  if (!rc) rc = upload_twiddles(ctx, ctx->Np, ctx->tw_np);
  if (!rc) rc = upload_twiddles(ctx, ctx->Nm, ctx->tw_nm);
  if (rc) {
    g_err = ctx->err;
    cola_free(ctx);
    return rc;
  }
  // spectrum normalisation and LCDM growth ratio depend only on the cosmology
  // and a_ini: computed once per distinct key and shared by every context
  {
    static std::mutex mu;
    static std::map<std::vector<double>, std::pair<EHParams, double>> cache;
    const std::vector<double> key = {cfg->Omega_m, cfg->Omega_b, cfg->h, cfg->n_s, cfg->sigma8, ctx->a[0]};
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
      HModel lc;
      Growth g;
      std::vector<double> nodes = {ctx->a[0], 1.0};
      solve_growth(lc, Om, nodes, std::vector<double>{1.0}, true, g);
      if (cache.size() > 64) cache.clear();
      it = cache.emplace(key, std::make_pair(eh_params(cfg->Omega_m, cfg->Omega_b, cfg->h, cfg->n_s,
                                                       cfg->sigma8), 1.0 / g.D1[1])).first;
    }
    ctx->eh = it->second.first;
    ctx->Dratio = it->second.second;
  }
  *out = ctx;
  return COLA_OK;
}

int cola_set_model(cola_ctx* ctx, const cola_model* model) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  CHECK_RC(validate_model(model, ctx));
  if (ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_set_model after cola_ic");
  CHECK_RC(validate_model_range(ctx->cfg, *model, ctx));
  ctx->hm = hmodel(*model);
  ctx->model = *model;
  ctx->model.mb_a = ctx->model.mb_beta = ctx->model.mb_m = nullptr;
  ctx->model_set = true;  // force_params reads the model
  const cola_config& cfg = ctx->cfg;
  const int nk = ctx->nk, ns = cfg.nsteps;
  const TableLayout tl(cfg);
  const size_t tab_b = tl.tab_b, fp_off = tl.fp_off, dt_off = tl.dt_off, g_off = tl.g_off, bytes = tl.bytes;
  // kind 1: (every configuration field but the seed and the seed precision, the model)
  std::vector<double> key = {1.0, (double)cfg.Np, (double)cfg.Nmesh, cfg.Lbox, (double)ns,
                             cfg.z_ini, cfg.z_final, cfg.Omega_m, cfg.Omega_b, cfg.h, cfg.n_s,
                             cfg.sigma8, (double)nk, (double)model->kind, model->fR0, model->rcH0,
                             model->R_smooth, (double)model->screening,
                             (double)model->scale_dependent, (double)model->filter,
                             model->beta_star, model->m_star, model->a_star, ctx->hm.phicrit0};
  for (const auto* v : {&ctx->hm.ta, &ctx->hm.tbeta, &ctx->hm.tM2}) key.insert(key.end(), v->begin(), v->end());
  const auto host = host_table(key, bytes, [&](char* h) {
    Growth g;
    growth_for(cfg, ctx->hm, g, nullptr, nullptr, nullptr);
    float4* tab = reinterpret_cast<float4*>(h);
    float4* vtab = reinterpret_cast<float4*>(h + tab_b);
    for (int n = 0; n <= ns; ++n) {
      for (int j = 0; j < nk; ++j) {
        const size_t i = (size_t)n * nk + j;
        if (n == 0) {
          tab[i] = make_float4((float)g.D1[i], (float)g.D2[i], (float)g.ddD1[i], (float)g.ddD2[i]);
        } else {
          const size_t q = (size_t)(n - 1) * nk + j;
          tab[i] = make_float4((float)(g.D1[i] - g.D1[q]), (float)(g.D2[i] - g.D2[q]),
                               (float)g.ddD1[i], (float)g.ddD2[i]);
        }
        vtab[i] = make_float4((float)g.dD1[i], (float)g.dD2[i], 0.f, 0.f);
      }
    }
    for (int j = 0; j < nk; ++j) {
      tab[(size_t)(ns + 1) * nk + j] = make_float4(1.f, 0.f, 0.f, 1.f);
      vtab[(size_t)(ns + 1) * nk + j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ForceParams* fp = reinterpret_cast<ForceParams*>(h + fp_off);
    float* dt = reinterpret_cast<float*>(h + dt_off);
    for (int n = 0; n < ns; ++n) {
      fp[n] = force_params(ctx, ctx->a[n + 1]);
      dt[3 * n + 0] = (float)ctx->dtk1[n];
      dt[3 * n + 1] = (float)ctx->dtd[n];
      dt[3 * n + 2] = (float)ctx->dtk2[n];
    }
    // per row: the largest Psi1 coefficient of the drift (c1) and kick (e1) fields
    float2* rg = reinterpret_cast<float2*>(h + g_off);
    for (int n = 0; n < ns + 2; ++n) {
      float c = 0.f, e = 0.f;
      for (int j = 0; j < nk; ++j) {
        c = std::max(c, std::abs(tab[(size_t)n * nk + j].x));
        e = std::max(e, std::abs(tab[(size_t)n * nk + j].z));
      }
      rg[n] = make_float2(c, e);
    }
  });
  CHECK_RC(upload(ctx, ctx->tables, host->data(), bytes));
  char* base = ctx->tables;
  ctx->tab = reinterpret_cast<float4*>(base);
  ctx->vtab = reinterpret_cast<float4*>(base + tab_b);
  ctx->dfp = reinterpret_cast<ForceParams*>(base + fp_off);
  ctx->ddt = reinterpret_cast<float*>(base + dt_off);
  ctx->hh.dfp = ctx->dfp;
  ctx->hh.ddt = ctx->ddt;
  ctx->hh.tab = ctx->tab;
  ctx->hh.vtab = ctx->vtab;
  ctx->hh.lqg = reinterpret_cast<const float2*>(base + g_off);
  ctx->hh.fp_ini = force_params(ctx, ctx->a[0]);
  ctx->hh.seed = ctx->cfg.seed;
  // bf16: unit scale of the largest value; fp16: the largest value at 2^15
  ctx->hh.seed_target = ctx->cfg.seed_precision == COLA_SEED_FP16 ? 32768.f : 1.f;
  ctx->hh.eh = eh_dev(ctx);
  CK(set_header(ctx->hdr, ctx->hh, ctx->st));
  return COLA_OK;
}

int cola_set_lpt_fast(cola_ctx* ctx, int32_t on) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->model_set) return fail(ctx, COLA_ESTATE, "cola_set_lpt_fast before cola_set_model");
  if (ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_set_lpt_fast after cola_ic");
  if (on) {
    // only for growth that does not depend on k: every table column equal
    Growth g;
    growth_for(ctx->cfg, ctx->hm, g, nullptr, nullptr, nullptr);
    const std::vector<double>* cols[6] = {&g.D1, &g.dD1, &g.ddD1, &g.D2, &g.dD2, &g.ddD2};
    for (const auto* c : cols)
      for (int n = 0; n < g.na; ++n) {
        const double ref = (*c)[(size_t)n * g.nk];
        for (int j = 1; j < g.nk; ++j)
          if (std::abs((*c)[(size_t)n * g.nk + j] - ref) > 1e-12 * std::max(1.0, std::abs(ref)))
            return fail(ctx, COLA_EINVAL, "cola_set_lpt_fast: the growth of this model depends on k");
      }
  }
  ctx->lpt_fast = on != 0;
  return COLA_OK;
}

int cola_ic(cola_ctx* ctx) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->model_set) return fail(ctx, COLA_ESTATE, "cola_ic before cola_set_model");
  return finish_ic(ctx, false);
}

int cola_ic_from_potentials(cola_ctx* ctx, const float* phi1, const float* phi2, int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!phi1 || !phi2) return fail(ctx, COLA_EINVAL, "phi1/phi2 is NULL");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  if (!ctx->model_set) return fail(ctx, COLA_ESTATE, "cola_ic_from_potentials before cola_set_model");
  const int N = ctx->Np;
  const size_t bytes = (size_t)N * N * (N / 2 + 1) * sizeof(float2);
  const float* src[2] = {phi1, phi2};
  for (int f = 0; f < 2; ++f) {
    const float2* dense = reinterpret_cast<const float2*>(src[f]);
    if (where == COLA_HOST) {
      CHECK_RC(copy_in(ctx, ctx->lc[0], src[f], bytes, where));
      dense = ctx->lc[0];
    }
    CK(half_pack(N, dense, ctx->phi[f], ctx->st));
    CHECK_RC(host_wait(ctx));
  }
  return finish_ic(ctx, true);
}

int cola_step(cola_ctx* ctx, int32_t nsteps) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_step before cola_ic");
  if (nsteps < 0) nsteps = ctx->cfg.nsteps - ctx->step;
  if (ctx->step + nsteps > ctx->cfg.nsteps) return fail(ctx, COLA_EINVAL, "past the last step");
  if (fused_steps_ok(ctx, nsteps)) return enqueue_steps_fused(ctx, nsteps);
  for (int it = 0; it < nsteps; ++it) {
    CHECK_RC(enqueue_step(ctx, ctx->step));
    ctx->step += 1;
  }
  return COLA_OK;
}

int cola_snapshot(cola_ctx* ctx, float* pos, float* vel, int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_snapshot before cola_ic");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  if (!pos && !vel) return COLA_OK;
  const size_t bytes = (size_t)ctx->P * 3 * sizeof(float);
  // LPT velocity dPsi/dtau at a_step: the velocity-table transform, or on the
  // fast path dD1 Psi1 + dD2 Psi2 formed in the snapshot kernel
  const LptMix mix = ctx->lpt_fast ? lpt_mix_of(ctx, ctx->step, 0, true) : LptMix{};
  if (vel && !ctx->lpt_fast) CHECK_RC(run_lpt(ctx, 1, ctx->step, false));
  const PartParams pp = part_params(ctx);
  const float vscale = (float)(100.0 / ctx->a[ctx->step]);
  if (where == COLA_DEVICE) {
    CK(part_snapshot(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                     ctx->lr[0], ctx->lr[1], ctx->lr[2], vscale, pos, vel, ctx->P, ctx->st, mix));
    return COLA_OK;
  }
  // host: page-locked caller buffers the device can address are written by the
  // snapshot kernel itself; the others are staged on the device and copied
  float* mp = pos ? static_cast<float*>(mapped_host(pos)) : nullptr;
  float* mv = vel ? static_cast<float*>(mapped_host(vel)) : nullptr;
  Temp tp(ctx, pos && !mp ? bytes : 0), tv(ctx, vel && !mv ? bytes : 0);
  if ((pos && !mp && !tp.p) || (vel && !mv && !tv.p))
    return fail(ctx, COLA_ENOMEM, "snapshot staging allocation failed");
  CK(part_snapshot(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                   ctx->lr[0], ctx->lr[1], ctx->lr[2], vscale, pos ? (mp ? mp : static_cast<float*>(tp.p)) : nullptr,
                   vel ? (mv ? mv : static_cast<float*>(tv.p)) : nullptr, ctx->P, ctx->st, mix));
  if (pos && !mp) CHECK_RC(copy_to_host(ctx, pos, tp.p, bytes));
  if (vel && !mv) CHECK_RC(copy_to_host(ctx, vel, tv.p, bytes));
  const bool copied = (pos && !mp) || (vel && !mv);  // a copy above already waited for the kernel
  return copied ? COLA_OK : host_wait(ctx);
}

// Deposit, forward transform and binning of the current particles into
// ctx->pk_acc (Sec. 7 estimator), enqueued on ctx->st.
static int enqueue_pk(cola_ctx* ctx, int32_t nbins) {
  const int N = ctx->Nm;
  const PartParams pp = part_params(ctx);
  const ForceParams fp = force_params(ctx, ctx->a[ctx->step]);
  CK(cudaMemsetAsync(ctx->rho, 0, ctx->M * sizeof(float), ctx->st));
  CK(part_deposit(pp, ctx->s[0], ctx->s[1], ctx->s[2], ctx->rho, ctx->P, ctx->st));
  CHECK_RC(r2c3(ctx, N, ctx->rho, ctx->Cw, ctx->tw_nm, fp.inv_rhobar, -1.f));
  CK(cudaMemsetAsync(ctx->pk_acc, 0, 3 * nbins * sizeof(double), ctx->st));
  const double L = ctx->L, N3 = (double)N * N * N;
  CK(pk_bin(N, ctx->Cw, nbins, ctx->pk_acc, L * L * L / (N3 * N3), ctx->st));
  return COLA_OK;
}

// Bin sums [count | sum P | sum |k|/k_F] -> mean k, mean P, mode counts.
static void finish_pk(const cola_ctx* ctx, const double* h, int32_t nbins, double* k, double* pk,
                      int64_t* nmodes) {
  const double kf = 2.0 * kPi / ctx->L;
  for (int b = 0; b < nbins; ++b) {
    const double cnt = h[b];
    if (k) k[b] = cnt > 0 ? h[2 * nbins + b] / cnt * kf : NAN;
    if (pk) pk[b] = cnt > 0 ? h[nbins + b] / cnt : NAN;
    if (nmodes) nmodes[b] = (int64_t)llround(cnt);
  }
}

int cola_pk(cola_ctx* ctx, int32_t nbins, double* k, double* pk, int64_t* nmodes) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_pk before cola_ic");
  if (nbins < 1 || nbins > kMaxBins) return fail(ctx, COLA_EINVAL, "nbins out of range 1..2000");
  if (ctx->pk_nbins) return fail(ctx, COLA_ESTATE, "a cola_pk_async result is still pending");
  CHECK_RC(enqueue_pk(ctx, nbins));
  // the sums land in a pinned slot, so a wait that times out leaves no copy into freed memory
  if (!ctx->pk_host && !(ctx->pk_host = g_pk_slots.get()))
    return fail(ctx, COLA_ENOMEM, "cola_pk: pinned host buffer allocation failed");
  CK(cudaMemcpyAsync(ctx->pk_host, ctx->pk_acc, 3 * (size_t)nbins * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->st));
  CHECK_RC(host_wait(ctx));
  finish_pk(ctx, ctx->pk_host, nbins, k, pk, nmodes);
  return COLA_OK;
}

int cola_pk_async(cola_ctx* ctx, int32_t nbins) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_pk_async before cola_ic");
  if (nbins < 1 || nbins > kMaxBins) return fail(ctx, COLA_EINVAL, "nbins out of range 1..2000");
  if (ctx->pk_nbins) return fail(ctx, COLA_ESTATE, "a cola_pk_async result is still pending");
  if (!ctx->pk_host && !(ctx->pk_host = g_pk_slots.get()))
    return fail(ctx, COLA_ENOMEM, "cola_pk_async: pinned host buffer allocation failed");
  if (!ctx->pk_event) CK(cudaEventCreateWithFlags(&ctx->pk_event, cudaEventDisableTiming));
  CHECK_RC(enqueue_pk(ctx, nbins));
  CK(cudaMemcpyAsync(ctx->pk_host, ctx->pk_acc, 3 * (size_t)nbins * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaEventRecord(ctx->pk_event, ctx->st));
  ctx->pk_nbins = nbins;
  return COLA_OK;
}

int cola_pk_ready(cola_ctx* ctx) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->pk_nbins) return fail(ctx, COLA_ESTATE, "no cola_pk_async pending");
  const cudaError_t e = cudaEventQuery(ctx->pk_event);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return fail(ctx, COLA_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(e));
}

int cola_pk_result(cola_ctx* ctx, double* k, double* pk, int64_t* nmodes) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->pk_nbins) return fail(ctx, COLA_ESTATE, "no cola_pk_async pending");
  if (ctx->wait_limit_s > 0) {
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(ctx->wait_limit_s);
    for (;;) {
      const cudaError_t e = cudaEventQuery(ctx->pk_event);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return fail(ctx, COLA_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(e));
      if (std::chrono::steady_clock::now() >= t_end)
        return fail(ctx, COLA_ETIMEOUT, "the P(k) did not complete within the wait limit");
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  } else {
    CK(cudaEventSynchronize(ctx->pk_event));
  }
  finish_pk(ctx, ctx->pk_host, ctx->pk_nbins, k, pk, nmodes);
  ctx->pk_nbins = 0;
  return COLA_OK;
}

int cola_check_state(cola_ctx* ctx, int64_t* nonfinite) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!nonfinite) return fail(ctx, COLA_EINVAL, "nonfinite is NULL");
  if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_check_state before cola_ic");
  const float* f[9] = {ctx->s[0], ctx->s[1], ctx->s[2], ctx->v[0], ctx->v[1], ctx->v[2],
                       ctx->acc[0], ctx->acc[1], ctx->acc[2]};
  unsigned long long* d = reinterpret_cast<unsigned long long*>(ctx->scratch);
  CK(count_nonfinite(f, 9, ctx->P, d, ctx->st));
  // the count lands in a pinned slot, so a wait that times out leaves no copy into freed memory
  if (!ctx->pk_host && !(ctx->pk_host = g_pk_slots.get()))
    return fail(ctx, COLA_ENOMEM, "cola_check_state: pinned host buffer allocation failed");
  if (ctx->pk_nbins) return fail(ctx, COLA_ESTATE, "a cola_pk_async result is still pending");
  CK(cudaMemcpyAsync(ctx->pk_host, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->st));
  CK(tile_load_failures(reinterpret_cast<unsigned*>(ctx->pk_host + 1), ctx->st));
  CHECK_RC(host_wait(ctx));
  unsigned long long v = 0;
  unsigned lost = 0;
  std::memcpy(&v, ctx->pk_host, sizeof(v));
  std::memcpy(&lost, ctx->pk_host + 1, sizeof(lost));
  *nonfinite = (int64_t)v;
  if (lost)
    return fail(ctx, COLA_ECUDA,
                "a transform's tile load on this device did not complete within its one-second wait; "
                "results computed since are invalid");
  return COLA_OK;
}

int cola_set_wait_limit(cola_ctx* ctx, double seconds) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!(seconds >= 0) || !std::isfinite(seconds)) return fail(ctx, COLA_EINVAL, "wait limit must be finite and >= 0");
  ctx->wait_limit_s = seconds;
  return COLA_OK;
}

int cola_wait(cola_ctx* ctx) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  return host_wait(ctx);
}

int cola_selftest_wait(double seconds, int* timed_out) {
  if (!timed_out) return fail(nullptr, COLA_EINVAL, "timed_out is NULL");
  if (!(seconds > 0) || seconds > 10) return fail(nullptr, COLA_EINVAL, "limit out of range (0, 10] s");
  const cudaError_t e = wait_probe(seconds, timed_out);
  if (e != cudaSuccess) return fail(nullptr, COLA_ECUDA, std::string("cola_selftest_wait: ") + cudaGetErrorString(e));
  return COLA_OK;
}

int cola_set_stream(cola_ctx* ctx, void* stream) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (st == ctx->st) return COLA_OK;
  // work already queued on the old stream precedes later work on the new one
  if (!ctx->ev_order) CK(cudaEventCreateWithFlags(&ctx->ev_order, cudaEventDisableTiming));
  CK(cudaEventRecord(ctx->ev_order, ctx->st));
  CK(cudaStreamWaitEvent(st, ctx->ev_order, 0));
  ctx->st = st;
  return COLA_OK;
}

double cola_scale_factor(const cola_ctx* ctx) { return ctx ? ctx->a[ctx->step] : NAN; }

int32_t cola_steps_done(const cola_ctx* ctx) { return ctx ? ctx->step : -1; }

const char* cola_last_error(const cola_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

void cola_free(cola_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  for (auto& stg : ctx->stages)
    for (auto& pr : stg.pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->ev_order) cudaEventDestroy(ctx->ev_order);
  if (ctx->pk_event) cudaEventDestroy(ctx->pk_event);
  if (ctx->ev_wait) cudaEventDestroy(ctx->ev_wait);
  g_pk_slots.put(ctx->pk_host);
  for (void* p : ctx->allocs) dev_free(ctx, p);
  if (!ctx->alloc) cudaStreamSynchronize(ctx->st);
  cudaGetLastError();
  delete ctx;
}

int cola_export(cola_ctx* ctx, int32_t which, void* dst, int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!dst) return fail(ctx, COLA_EINVAL, "dst is NULL");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  const size_t pb = (size_t)ctx->P * sizeof(float), mb = (size_t)ctx->M * sizeof(float);
  char* d = static_cast<char*>(dst);
  switch (which) {
    case COLA_F_DISP:
    case COLA_F_DV:
    case COLA_F_ACC: {
      if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "no particle state before cola_ic");
      float* const* arr = which == COLA_F_DISP ? ctx->s : which == COLA_F_DV ? ctx->v : ctx->acc;
      for (int c = 0; c < 3; ++c) CHECK_RC(copy_out(ctx, d + c * pb, arr[c], pb, where));
      return COLA_OK;
    }
    case COLA_F_RHO:
      if (!ctx->have_force) return fail(ctx, COLA_ESTATE, "no deposit yet");
      return copy_out(ctx, dst, ctx->rho, mb, where);
    case COLA_F_DELTAK: {
      if (!ctx->have_force) return fail(ctx, COLA_ESTATE, "no deposit yet");
      const ForceParams fp = force_params(ctx, ctx->a[ctx->step]);
      CHECK_RC(r2c3(ctx, ctx->Nm, ctx->rho, ctx->Cw, ctx->tw_nm, fp.inv_rhobar, -1.f));
      return export_half(ctx, ctx->Nm, ctx->Cw, ctx->Cphi, dst, where);
    }
    case COLA_F_FORCE:
      if (!ctx->have_force) return fail(ctx, COLA_ESTATE, "no force yet");
      return export_force(ctx, d, where);
    case COLA_F_PHI1:
    case COLA_F_PHI2:
      if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "no seeds before cola_ic");
      return export_half(ctx, ctx->Np, ctx->phi[which - COLA_F_PHI1], ctx->lc[5], dst, where);
    case COLA_F_LPT_DISP:
    case COLA_F_LPT_ACC: {
      if (!ctx->have_lpt) return fail(ctx, COLA_ESTATE, "no LPT fields yet");
      const int o = which == COLA_F_LPT_DISP ? 0 : 3;
      if (ctx->lpt_fast) {
        // the fields of the last step (row `step`; row 0 before the first step),
        // formed from Psi1, Psi2 into the idle LPT spectrum buffers
        float* tmp[3] = {reinterpret_cast<float*>(ctx->lc[0]), reinterpret_cast<float*>(ctx->lc[1]),
                         reinterpret_cast<float*>(ctx->lc[2])};
        const float* psi1[3] = {ctx->lr[0], ctx->lr[1], ctx->lr[2]};
        CK(lpt_mix(ctx->P, psi1, lpt_mix_of(ctx, ctx->step, 0, false), o == 3 ? 1 : 0, tmp, ctx->st));
        for (int c = 0; c < 3; ++c) CHECK_RC(copy_out(ctx, d + c * pb, tmp[c], pb, where));
        return COLA_OK;
      }
      if (ctx->cfg.seed_precision && ctx->step > 0) {
        // variant a.S1: the last step's fields are the 16-bit ones, dequantised
        float* tmp = reinterpret_cast<float*>(ctx->lc[0]);
        for (int c = 0; c < 3; ++c) {
          CK(lq_dequant(ctx->lq[o + c], tmp, ctx->P, ctx->cfg.seed_precision, ctx->hdr, o + c, ctx->st));
          CHECK_RC(copy_out(ctx, d + c * pb, tmp, pb, where));
        }
        return COLA_OK;
      }
      for (int c = 0; c < 3; ++c)
        CHECK_RC(copy_out(ctx, d + c * pb, (o == 3 && ctx->kslot) ? ctx->lrk[c] : ctx->lr[o + c], pb, where));
      return COLA_OK;
    }
    default:
      return fail(ctx, COLA_EINVAL, "unknown array id");
  }
}

int cola_import_state(cola_ctx* ctx, const float* disp, const float* dv, const float* acc,
                      int32_t steps_done, int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!ctx->ic_done) return fail(ctx, COLA_ESTATE, "cola_import_state before cola_ic");
  if (!disp || !dv || !acc) return fail(ctx, COLA_EINVAL, "NULL state array");
  if (steps_done < 0 || steps_done > ctx->cfg.nsteps) return fail(ctx, COLA_EINVAL, "steps_done out of range");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  const size_t pb = (size_t)ctx->P * sizeof(float);
  const float* src[3] = {disp, dv, acc};
  float* const* dstv[3] = {ctx->s, ctx->v, ctx->acc};
  for (int q = 0; q < 3; ++q)
    for (int c = 0; c < 3; ++c)
      CHECK_RC(copy_in(ctx, dstv[q][c], reinterpret_cast<const char*>(src[q]) + c * pb, pb, where));
  ctx->hh.step = steps_done;
  CK(set_header(ctx->hdr, ctx->hh, ctx->st));
  ctx->step = steps_done;
  return COLA_OK;
}

int cola_fft(cola_ctx* ctx, int32_t dir, const void* in, void* out, int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!in || !out) return fail(ctx, COLA_EINVAL, "NULL buffer");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  const int N = ctx->Nm;
  const size_t rb = (size_t)ctx->M * sizeof(float);
  const size_t cb = (size_t)N * N * (N / 2 + 1) * sizeof(float2);
  if (dir == 1) {
    const float* src = static_cast<const float*>(in);
    if (where == COLA_HOST) {
      CHECK_RC(copy_in(ctx, ctx->F[0], in, rb, where));
      src = ctx->F[0];
    }
    CHECK_RC(r2c3(ctx, N, src, ctx->Cw, ctx->tw_nm, 1.f, 0.f));
    return export_half(ctx, N, ctx->Cw, ctx->Cphi, out, where);
  }
  if (dir == -1) {
    const float2* dense = static_cast<const float2*>(in);
    if (where == COLA_HOST) {
      CHECK_RC(copy_in(ctx, ctx->Cphi, in, cb, where));
      dense = ctx->Cphi;
    }
    CK(half_pack(N, dense, ctx->Cw, ctx->st));
    float* dst = where == COLA_DEVICE ? static_cast<float*>(out) : ctx->F[0];
    CHECK_RC(c2r3(ctx, N, ctx->Cw, dst, ctx->tw_nm));
    if (where == COLA_HOST) return copy_out(ctx, out, ctx->F[0], rb, where);
    return COLA_OK;
  }
  return fail(ctx, COLA_EINVAL, "dir must be +1 or -1");
}

int cola_cic_deposit(cola_ctx* ctx, const float* pos, int64_t n, float* rho, int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if ((!pos && n > 0) || !rho || n < 0) return fail(ctx, COLA_EINVAL, "bad buffers");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  const float* dpos = pos;
  Temp t(ctx, where == COLA_HOST && n > 0 ? (size_t)n * 3 * sizeof(float) : 0);
  if (where == COLA_HOST && n > 0) {
    if (!t.p) return fail(ctx, COLA_ENOMEM, "staging allocation failed");
    CHECK_RC(copy_in(ctx, t.p, pos, (size_t)n * 3 * sizeof(float), where));
    dpos = static_cast<const float*>(t.p);
  }
  CK(cudaMemsetAsync(ctx->rho, 0, ctx->M * sizeof(float), ctx->st));
  CK(pos_deposit(ctx->Nm, (float)(ctx->Nm / ctx->L), dpos, n, ctx->rho, ctx->st));
  return copy_out(ctx, rho, ctx->rho, (size_t)ctx->M * sizeof(float), where);
}

int cola_force_from_density(cola_ctx* ctx, const float* rho, double a, float* force,
                            int32_t where) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  if (!rho || !force) return fail(ctx, COLA_EINVAL, "NULL buffer");
  if (!ctx->model_set) return fail(ctx, COLA_ESTATE, "no model set");
  if (!(a > 0)) return fail(ctx, COLA_EINVAL, "a must be > 0");
  if (where != COLA_HOST && where != COLA_DEVICE) return fail(ctx, COLA_EINVAL, "bad where");
  const size_t mb = (size_t)ctx->M * sizeof(float);
  CHECK_RC(copy_in(ctx, ctx->rho, rho, mb, where));
  CHECK_RC(run_force(ctx, a));
  return export_force(ctx, reinterpret_cast<char*>(force), where);
}

// ---------------------------------------------------------------- batches
static int bfail(cola_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  g_err = m;
  return code;
}

#define BCK(expr)                                                                               \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) return bfail(b, COLA_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Contexts one multi-simulation launch can serve: the same buffer layout and
// the same launch-time constants (time grids, cosmologies, models and step
// counts may differ: those are read through each simulation's header).
static bool same_shape(const cola_ctx* a, const cola_ctx* c) {
  return a->cfg.Np == c->cfg.Np && a->cfg.Nmesh == c->cfg.Nmesh && a->cfg.Lbox == c->cfg.Lbox &&
         a->cfg.nk_table == c->cfg.nk_table && a->cfg.seed_precision == c->cfg.seed_precision &&
         a->lpt_fast == c->lpt_fast && a->model.filter == c->model.filter;  // one smoothing window per launch
}

static cola_batch_plan normal_plan(const cola_batch* b, cola_batch_plan p) {
  const int n = (int)b->ctx.size();
  if (!b->uniform || p.group < 1) p.group = b->uniform ? n : 1;
  p.group = std::min(p.group, n);
  const int groups = (n + p.group - 1) / p.group;
  p.chains = std::max(1, std::min(p.chains < 1 ? 1 : p.chains, groups));
  p.grid_cap = std::max(0, p.grid_cap);
  p.deposit_box = std::max(0, std::min(p.deposit_box, 16384)) & ~3;
  p.gather_box = std::max(0, std::min(p.gather_box, 8192)) & ~3;
  return p;
}

static int chain_streams(cola_batch* b, int C) {
  while ((int)b->chain_st.size() < C) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    BCK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->chain_st.push_back(s);
    BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->join.push_back(ev);
  }
  return COLA_OK;
}

// Groups of a plan: consecutive runs of plan.group contexts.  Shift arrays
// (byte offsets of each member's allocation from its subset's first member)
// are gathered into `hsh`; the Multi pointers are fixed up once the device
// copy of hsh exists.
struct GroupPlan {
  Group g;
  size_t off[5];  // offsets into hsh of all, unscreened, fr_screened, dgp_screened, screened
};

static void plan_groups(const std::vector<cola_ctx*>& ctxs, int group, std::vector<GroupPlan>& out,
                        std::vector<int64_t>& hsh) {
  const int n = (int)ctxs.size();
  for (int j0 = 0; j0 < n; j0 += group) {
    const int j1 = std::min(n, j0 + group);
    GroupPlan gp;
    std::vector<cola_ctx*> lists[5];
    for (int i = j0; i < j1; ++i) {
      cola_ctx* c = ctxs[i];
      const bool scr = c->model.kind != COLA_LCDM && c->model.screening;
      lists[0].push_back(c);
      if (!scr) lists[1].push_back(c);
      else if (chameleon_kind(c->model.kind)) lists[2].push_back(c);
      else lists[3].push_back(c);
      if (scr) lists[4].push_back(c);
    }
    Group::Sub* subs[5] = {nullptr, &gp.g.unscreened, &gp.g.fr_screened, &gp.g.dgp_screened, &gp.g.screened};
    for (int q = 0; q < 5; ++q) {
      gp.off[q] = hsh.size();
      if (lists[q].empty()) continue;
      const char* base = static_cast<const char*>(lists[q][0]->allocs[0]);
      for (cola_ctx* c : lists[q]) hsh.push_back(static_cast<const char*>(c->allocs[0]) - base);
      Multi m;
      m.nb = (int)lists[q].size();
      if (q == 0) {
        gp.g.lead = lists[q][0];
        gp.g.all = m;
      } else {
        subs[q]->lead = lists[q][0];
        subs[q]->m = m;
      }
    }
    out.push_back(gp);
  }
}

// Captures one step of every context under plan p (the step index comes from
// each context's device header, so the graph serves every step).
static int batch_capture(cola_batch* b, int n, const cola_batch_plan& p, int kind, cola_batch::Graph* out) {
  std::vector<GroupPlan> groups;
  std::vector<int64_t> hsh;
  plan_groups(b->ctx, p.group, groups, hsh);
  CHECK_RC(chain_streams(b, p.chains));
  int64_t* dsh = nullptr;
  if (!hsh.empty()) {
    dsh = static_cast<int64_t*>(dev_alloc_on(b->ctx[0], hsh.size() * sizeof(int64_t), b->cap_st));
    if (!dsh) return bfail(b, COLA_ENOMEM, "batch capture: shift array allocation failed");
    out->shifts = dsh;
    BCK(cudaMemcpyAsync(dsh, hsh.data(), hsh.size() * sizeof(int64_t), cudaMemcpyHostToDevice, b->cap_st));
    BCK(cudaStreamSynchronize(b->cap_st));
  }
  for (GroupPlan& gp : groups) {
    Multi* ms[5] = {&gp.g.all, &gp.g.unscreened.m, &gp.g.fr_screened.m, &gp.g.dgp_screened.m,
                    &gp.g.screened.m};
    for (int q = 0; q < 5; ++q) ms[q]->shift = ms[q]->nb > 1 ? dsh + gp.off[q] : nullptr;
  }
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeRelaxed));
  int rc = COLA_OK;
  const int C = p.chains;
  cudaError_t e = cudaEventRecord(b->fork, b->cap_st);
  for (int c = 0; c < C && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(b->chain_st[c], b->fork, 0);
  set_grid_cap(p.grid_cap);
  set_particle_plan(p.deposit_box, p.gather_box);
  for (size_t j = 0; j < groups.size() && e == cudaSuccess && rc == COLA_OK; ++j) {
    cola_ctx* lead = groups[j].g.lead;
    cudaStream_t saved = lead->st;
    const bool prof = lead->prof;
    lead->st = b->chain_st[j % C];
    lead->prof = false;
    rc = enqueue_kind(groups[j].g, n, kind);
    lead->st = saved;
    lead->prof = prof;
    if (rc != COLA_OK) b->err = lead->err;
  }
  set_grid_cap(0);
  set_particle_plan(0, 0);
  for (int c = 0; c < C && e == cudaSuccess; ++c) {
    e = cudaEventRecord(b->join[c], b->chain_st[c]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_st, b->join[c], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->cap_st, &graph);
  if (rc != COLA_OK) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, rc, "batch capture: " + b->err);
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, COLA_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, COLA_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return COLA_OK;
}

static int batch_graph(cola_batch* b, const cola_batch_plan& p, cudaGraphExec_t* ex, int kind = BK_STEP) {
  const auto key = std::make_tuple(p.group, p.chains, p.grid_cap, p.deposit_box, p.gather_box, kind);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cola_batch::Graph g;
    int rc = batch_capture(b, b->step, p, kind, &g);
    if (rc != COLA_OK) {
      if (g.shifts) dev_free_on(b->ctx[0], g.shifts, b->cap_st);
      return rc;
    }
    it = b->graphs.emplace(key, g).first;
  }
  *ex = it->second.exec;
  return COLA_OK;
}

// Profiling: when the first context has stage timing enabled, the groups of
// the plan are launched directly (no graph) one after another on the batch's
// stream, so the first group's stage events cover its multi-simulation launches.
static int batch_eager(cola_batch* b, const cola_batch_plan& p, int n, int kind) {
  std::vector<GroupPlan> groups;
  std::vector<int64_t> hsh;
  plan_groups(b->ctx, p.group, groups, hsh);
  int64_t* dsh = nullptr;
  if (!hsh.empty()) {
    dsh = static_cast<int64_t*>(dev_alloc_on(b->ctx[0], hsh.size() * sizeof(int64_t), b->cap_st));
    if (!dsh) return bfail(b, COLA_ENOMEM, "batch step: shift array allocation failed");
    BCK(write_words(dsh, hsh.data(), (int64_t)hsh.size(), b->cap_st));
  }
  int rc = COLA_OK;
  for (GroupPlan& gp : groups) {
    Multi* ms[5] = {&gp.g.all, &gp.g.unscreened.m, &gp.g.fr_screened.m, &gp.g.dgp_screened.m,
                    &gp.g.screened.m};
    for (int q = 0; q < 5; ++q) ms[q]->shift = ms[q]->nb > 1 ? dsh + gp.off[q] : nullptr;
    cola_ctx* lead = gp.g.lead;
    cudaStream_t saved = lead->st;
    lead->st = b->cap_st;
    set_grid_cap(p.grid_cap);
    set_particle_plan(p.deposit_box, p.gather_box);
    rc = enqueue_kind(gp.g, n, kind);
    set_grid_cap(0);
    set_particle_plan(0, 0);
    lead->st = saved;
    if (rc != COLA_OK) {
      b->err = lead->err;
      break;
    }
  }
  dev_free_on(b->ctx[0], dsh, b->cap_st);
  return rc == COLA_OK ? COLA_OK : bfail(b, rc, "batch step: " + b->err);
}

// One launch sequence of `kind` (a whole step by default); every kind but the
// head of a fused run ends one step.
static int batch_launch(cola_batch* b, const cola_batch_plan& p, int kind = BK_STEP) {
  const int n = b->step;
  const bool eager = b->ctx[0]->prof;
  cudaGraphExec_t ex = nullptr;
  if (!eager) CHECK_RC(batch_graph(b, p, &ex, kind));
  // ordered after earlier work on the caller's stream, and before later work on it
  BCK(cudaEventRecord(b->ev_in, b->st));
  BCK(cudaStreamWaitEvent(b->cap_st, b->ev_in, 0));
  if (eager) CHECK_RC(batch_eager(b, p, n, kind));
  else BCK(cudaGraphLaunch(ex, b->cap_st));
  BCK(cudaEventRecord(b->ev_out, b->cap_st));
  BCK(cudaStreamWaitEvent(b->st, b->ev_out, 0));
  const int n1 = kind == BK_HEAD ? n : n + 1;
  b->step = n1;
  for (cola_ctx* ctx : b->ctx) {
    ctx->step = n1;
    ctx->hh.step = n1;
  }
  // later per-context calls on the contexts' own streams see the step
  for (cola_ctx* ctx : b->ctx)
    if (ctx->st != b->st) BCK(cudaStreamWaitEvent(ctx->st, b->ev_out, 0));
  return COLA_OK;
}

int cola_batch_create(cola_ctx* const* ctxs, int32_t n, const cola_batch_plan* plan, void* stream,
                      cola_batch** out) {
  if (!out) return fail(nullptr, COLA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1 || n > 65535) return fail(nullptr, COLA_EINVAL, "need 1 <= n <= 65535 contexts");
  for (int i = 0; i < n; ++i) {
    const cola_ctx* c = ctxs[i];
    if (!c) return fail(nullptr, COLA_EINVAL, "NULL context in batch");
    if (!c->ic_done) return fail(nullptr, COLA_ESTATE, "every context of a batch needs cola_ic");
    if (c->cfg.nsteps != ctxs[0]->cfg.nsteps || c->step != ctxs[0]->step)
      return fail(nullptr, COLA_EINVAL, "contexts of a batch need equal nsteps and steps done");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(nullptr, COLA_EINVAL, "a context appears twice in the batch");
  }
  cola_batch* b = new cola_batch();
  b->ctx.assign(ctxs, ctxs + n);
  b->st = static_cast<cudaStream_t>(stream);
  b->step = ctxs[0]->step;
  b->uniform = true;
  for (int i = 1; i < n; ++i) b->uniform = b->uniform && same_shape(ctxs[0], ctxs[i]);
  b->plan = normal_plan(b, plan ? *plan : cola_batch_plan{0, 1, 0, 0, 0});
  auto bail = [&](cudaError_t e) {
    g_err = std::string("cola_batch_create: ") + cudaGetErrorString(e);
    cola_batch_free(b);
    return COLA_ECUDA;
  };
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e);
  e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e);
  e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e);
  e = cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(e);
  // work already queued on the contexts' own streams precedes the first batch step
  for (cola_ctx* ctx : b->ctx) {
    if (ctx->st == b->st) continue;
    e = cudaEventRecord(b->fork, ctx->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->fork, 0);
    if (e != cudaSuccess) return bail(e);
  }
  *out = b;
  return COLA_OK;
}

int cola_batch_set_plan(cola_batch* b, const cola_batch_plan* plan) {
  if (!b || !plan) return fail(nullptr, COLA_EINVAL, "batch or plan is NULL");
  b->plan = normal_plan(b, *plan);
  return COLA_OK;
}

int cola_batch_get_plan(const cola_batch* b, cola_batch_plan* out) {
  if (!b || !out) return fail(nullptr, COLA_EINVAL, "batch or out is NULL");
  *out = b->plan;
  return COLA_OK;
}

int cola_batch_step(cola_batch* b, int32_t nsteps) {
  if (!b) return fail(nullptr, COLA_EINVAL, "batch is NULL");
  const int total = b->ctx[0]->cfg.nsteps;
  if (nsteps < 0) nsteps = total - b->step;
  if (b->step + nsteps > total) return bfail(b, COLA_EINVAL, "past the last step");
  for (cola_ctx* c : b->ctx) c->kslot = 0;  // single batch steps keep the kick fields in lr[3..5]
  // two or more steps with the direct particle kernels: the kick of each step but
  // the last and the drift + deposit of the next in one pass (enqueue_group_mid)
  bool fused = nsteps >= 2 && b->plan.deposit_box == 0 && b->plan.gather_box == 0;
  for (const cola_ctx* c : b->ctx) fused = fused && fused_steps_ok(c, nsteps);
  if (!fused) {
    for (int i = 0; i < nsteps; ++i) CHECK_RC(batch_launch(b, b->plan));
    return COLA_OK;
  }
  CHECK_RC(batch_launch(b, b->plan, BK_HEAD));
  int cur = 0;
  for (int i = 1; i < nsteps; ++i) {
    CHECK_RC(batch_launch(b, b->plan, cur ? BK_MID1 : BK_MID0));
    cur = 1 - cur;
  }
  CHECK_RC(batch_launch(b, b->plan, cur ? BK_TAIL1 : BK_TAIL0));
  for (cola_ctx* c : b->ctx) c->kslot = cur;  // the last step's kick fields
  return COLA_OK;
}

int cola_batch_autotune(cola_batch* b, int32_t max_steps, cola_batch_plan* best_out) {
  if (!b) return fail(nullptr, COLA_EINVAL, "batch is NULL");
  for (cola_ctx* c : b->ctx) c->kslot = 0;  // batch steps keep the kick fields in lr[3..5]
  const int n = (int)b->ctx.size();
  const int total = b->ctx[0]->cfg.nsteps;
  const int sms = 152;
  std::vector<cola_batch_plan> cand;
  if (b->uniform) {
    // one group over everything; halves and quarters on concurrent chains;
    // small groups on many chains with a capped grid (more on-chip reuse)
    cand = {{n, 1, 0, 0, 0}, {(n + 1) / 2, 2, 0, 0, 0}, {(n + 3) / 4, 4, 0, 0, 0}, {(n + 7) / 8, 4, 0, 0, 0},
            {std::max(1, n / 32), 8, sms, 0, 0}, {1, 32, sms, 0, 0}};
  } else {
    cand = {{1, 32, sms, 0, 0}, {1, 64, sms / 2, 0, 0}, {1, 16, 2 * sms, 0, 0}, {1, 128, sms / 4, 0, 0},
            {1, 8, 0, 0, 0}, {1, 32, 0, 0, 0}};
  }
  auto same = [](const cola_batch_plan& a, const cola_batch_plan& q) {
    return a.group == q.group && a.chains == q.chains && a.grid_cap == q.grid_cap &&
           a.deposit_box == q.deposit_box && a.gather_box == q.gather_box;
  };
  std::vector<cola_batch_plan> plans;
  for (const auto& c : cand) {
    const cola_batch_plan p = normal_plan(b, c);
    bool dup = false;
    for (const auto& q : plans) dup = dup || same(q, p);
    if (!dup) plans.push_back(p);
  }
  const int budget = std::min<int>(max_steps > 0 ? max_steps : total, total - b->step);
  double best = 1e300;
  cola_batch_plan bestp = b->plan;
  int used = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  int rc = COLA_OK;
  // one real step under plan p, timed on the caller's stream (capture outside the timing)
  auto time_plan = [&](const cola_batch_plan& p, float& ms) -> int {
    cudaGraphExec_t ex = nullptr;
    int r = batch_graph(b, p, &ex);
    if (r != COLA_OK) return r;
    cudaError_t e = cudaEventRecord(e0, b->st);
    if (e == cudaSuccess) {
      r = batch_launch(b, p);
      if (r != COLA_OK) return r;
      e = cudaEventRecord(e1, b->st);  // the caller's stream waits for the graph
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return bfail(b, COLA_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    ++used;
    return COLA_OK;
  };
  auto consider = [&](const cola_batch_plan& p) -> int {
    if (used >= budget) return COLA_OK;
    float ms = 0.f;
    CHECK_RC(time_plan(p, ms));
    if (ms < best) {
      best = ms;
      bestp = p;
    }
    return COLA_OK;
  };
  // 1. the launch grouping
  for (const auto& p : plans)
    if ((rc = consider(p)) != COLA_OK) break;
  // 2. the particle kernels with the best grouping: that plan is timed again
  //    first (later steps cost more once particles cluster), then deposit bins
  //    and gather boxes against it
  if (rc == COLA_OK && used + 1 < budget) {
    float ms = 0.f;
    rc = time_plan(bestp, ms);
    if (rc == COLA_OK) best = ms;
    for (int v : {4096, 16384})
      if (rc == COLA_OK) rc = consider(normal_plan(b, {bestp.group, bestp.chains, bestp.grid_cap, v, 0}));
    const int dep = bestp.deposit_box;
    for (int v : {4096, 8192})
      if (rc == COLA_OK) rc = consider(normal_plan(b, {bestp.group, bestp.chains, bestp.grid_cap, dep, v}));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != COLA_OK) return rc;
  b->plan = bestp;
  if (best_out) *best_out = bestp;
  return COLA_OK;
}

int cola_batch_pk(cola_batch* b, int32_t nbins, double* k, double* pk, int64_t* nmodes) {
  if (!b) return fail(nullptr, COLA_EINVAL, "batch is NULL");
  if (nbins < 1 || nbins > kMaxBins) return bfail(b, COLA_EINVAL, "nbins out of range 1..2000");
  const int n = (int)b->ctx.size();
  if (!b->uniform) {
    for (int i = 0; i < n; ++i) {
      cola_ctx* c = b->ctx[i];
      int rc = cola_pk(c, nbins, k ? k + (size_t)i * nbins : nullptr, pk ? pk + (size_t)i * nbins : nullptr,
                       nmodes ? nmodes + (size_t)i * nbins : nullptr);
      if (rc != COLA_OK) return bfail(b, rc, c->err);
    }
    return COLA_OK;
  }
  cola_ctx* lead = b->ctx[0];
  const int N = lead->Nm;
  const int64_t stride = 3 * (int64_t)kMaxBins;
  // [n][stride] accumulators, then the n shifts
  if (!b->pk_acc) {
    b->pk_acc = static_cast<double*>(dev_alloc_on(lead, ((size_t)n * stride + n) * sizeof(double), b->st));
    if (!b->pk_acc) return bfail(b, COLA_ENOMEM, "batch P(k): accumulator allocation failed");
  }
  std::vector<int64_t> hsh(n);
  const char* base = static_cast<const char*>(lead->allocs[0]);
  for (int i = 0; i < n; ++i) hsh[i] = static_cast<const char*>(b->ctx[i]->allocs[0]) - base;
  int64_t* dsh = n > 1 ? reinterpret_cast<int64_t*>(b->pk_acc + (size_t)n * stride) : nullptr;
  cudaStream_t st = b->st;
  if (dsh) BCK(cudaMemcpyAsync(dsh, hsh.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  Multi m;
  m.shift = dsh;
  m.nb = n;
  const PartParams pp = part_params(lead);
  const ForceParams fp = force_params(lead, lead->a[lead->step]);
  BCK(zero_f32(lead->rho, lead->M, st, m));
  BCK(part_deposit(pp, lead->s[0], lead->s[1], lead->s[2], lead->rho, lead->P, st, m));
  BCK(fft_xr2c(N, lead->rho, lead->Cw, fp.inv_rhobar, -1.f, lead->tw_nm, st, m));
  BCK(fft_col(N, lead->Cw, 1, false, lead->tw_nm, st, m));
  BCK(fft_col(N, lead->Cw, 2, false, lead->tw_nm, st, m));
  BCK(cudaMemset2DAsync(b->pk_acc, stride * sizeof(double), 0, 3 * nbins * sizeof(double), n, st));
  const double L = lead->L, N3 = (double)N * N * N;
  BCK(pk_bin(N, lead->Cw, nbins, b->pk_acc, L * L * L / (N3 * N3), st, m, stride));
  std::vector<double> h((size_t)n * 3 * nbins);
  BCK(cudaMemcpy2DAsync(h.data(), 3 * nbins * sizeof(double), b->pk_acc, stride * sizeof(double),
                        3 * nbins * sizeof(double), n, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  const double kf = 2.0 * kPi / L;
  for (int i = 0; i < n; ++i) {
    const double* r = h.data() + (size_t)i * 3 * nbins;
    for (int q = 0; q < nbins; ++q) {
      const double cnt = r[q];
      const size_t o = (size_t)i * nbins + q;
      if (k) k[o] = cnt > 0 ? r[2 * nbins + q] / cnt * kf : NAN;
      if (pk) pk[o] = cnt > 0 ? r[nbins + q] / cnt : NAN;
      if (nmodes) nmodes[o] = (int64_t)llround(cnt);
    }
  }
  return COLA_OK;
}

// Runs enqueue(group) on `stream` for every group of the n distinct contexts
// (one group per shape, in order of first appearance), ordered after the work
// already queued on each context's own stream and before the work queued on
// it later.  The shift arrays travel in launch parameters into a
// stream-ordered allocation.  Reports failures through g_err.
static int run_on_groups(cola_ctx* const* ctxs, int32_t n, void* stream, const char* who,
                         const std::function<int(const Group&)>& enqueue) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto ck = [who](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return COLA_OK;
    g_err = std::string(who) + ": " + what + ": " + cudaGetErrorString(e);
    return COLA_ECUDA;
  };
  for (int i = 0; i < n; ++i) {
    cola_ctx* c = ctxs[i];
    if (c->st == st) continue;
    if (!c->ev_order) CHECK_RC(ck(cudaEventCreateWithFlags(&c->ev_order, cudaEventDisableTiming), "event"));
    CHECK_RC(ck(cudaEventRecord(c->ev_order, c->st), "event record"));
    CHECK_RC(ck(cudaStreamWaitEvent(st, c->ev_order, 0), "stream wait"));
  }
  std::vector<std::vector<cola_ctx*>> buckets;
  for (int i = 0; i < n; ++i) {
    bool placed = false;
    for (auto& bk : buckets)
      if (same_shape(bk[0], ctxs[i])) {
        bk.push_back(ctxs[i]);
        placed = true;
        break;
      }
    if (!placed) buckets.push_back({ctxs[i]});
  }
  std::vector<GroupPlan> groups;
  std::vector<int64_t> hsh;
  for (const auto& bk : buckets) plan_groups(bk, (int)bk.size(), groups, hsh);
  int64_t* dsh = nullptr;
  if (!hsh.empty()) {
    dsh = static_cast<int64_t*>(dev_alloc_on(ctxs[0], hsh.size() * sizeof(int64_t), st));
    if (!dsh) {
      g_err = std::string(who) + ": shift buffer allocation failed";
      return COLA_ENOMEM;
    }
    int rc0 = ck(write_words(dsh, hsh.data(), (int64_t)hsh.size(), st), "shift upload");
    if (rc0 != COLA_OK) {
      dev_free_on(ctxs[0], dsh, st);
      return rc0;
    }
  }
  int rc = COLA_OK;
  for (GroupPlan& gp : groups) {
    Multi* ms[5] = {&gp.g.all, &gp.g.unscreened.m, &gp.g.fr_screened.m, &gp.g.dgp_screened.m,
                    &gp.g.screened.m};
    for (int q = 0; q < 5; ++q) ms[q]->shift = ms[q]->nb > 1 ? dsh + gp.off[q] : nullptr;
    cola_ctx* lead = gp.g.lead;
    cudaStream_t saved = lead->st;
    lead->st = st;
    rc = enqueue(gp.g);
    lead->st = saved;
    if (rc != COLA_OK) {
      g_err = std::string(who) + ": " + lead->err;
      break;
    }
  }
  dev_free_on(ctxs[0], dsh, st);
  if (rc != COLA_OK) return rc;
  for (int i = 0; i < n; ++i) {
    cola_ctx* c = ctxs[i];
    if (c->st == st) continue;
    CHECK_RC(ck(cudaEventRecord(c->ev_order, st), "event record"));
    CHECK_RC(ck(cudaStreamWaitEvent(c->st, c->ev_order, 0), "stream wait"));
  }
  return COLA_OK;
}

static int check_distinct(cola_ctx* const* ctxs, int32_t n) {
  if (!ctxs || n < 1 || n > 65535) return fail(nullptr, COLA_EINVAL, "need 1 <= n <= 65535 contexts");
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(nullptr, COLA_EINVAL, "NULL context");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(nullptr, COLA_EINVAL, "a context appears twice");
  }
  return COLA_OK;
}

int cola_step_many(cola_ctx* const* ctxs, int32_t n, void* stream) {
  CHECK_RC(check_distinct(ctxs, n));
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]->ic_done) return fail(nullptr, COLA_ESTATE, "cola_step_many before cola_ic");
    if (ctxs[i]->step >= ctxs[i]->cfg.nsteps) return fail(nullptr, COLA_EINVAL, "a context is past its last step");
  }
  CHECK_RC(run_on_groups(ctxs, n, stream, "cola_step_many",
                         [](const Group& g) { return enqueue_group_step(g, g.lead->step); }));
  for (int i = 0; i < n; ++i) {
    ctxs[i]->step += 1;
    ctxs[i]->hh.step = ctxs[i]->step;
    ctxs[i]->kslot = 0;
  }
  return COLA_OK;
}

int cola_ic_many(cola_ctx* const* ctxs, int32_t n, void* stream) {
  CHECK_RC(check_distinct(ctxs, n));
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]->model_set) return fail(nullptr, COLA_ESTATE, "cola_ic_many before cola_set_model");
    if (ctxs[i]->ic_done) return fail(nullptr, COLA_ESTATE, "cola_ic_many on a context that has its ICs");
  }
  // step 0 in every header, on each context's own stream (run_on_groups orders it before the ICs)
  for (int i = 0; i < n; ++i) {
    ctxs[i]->hh.step = 0;
    cudaError_t e = set_header(ctxs[i]->hdr, ctxs[i]->hh, ctxs[i]->st);
    if (e != cudaSuccess) return fail(nullptr, COLA_ECUDA, std::string("cola_ic_many: ") + cudaGetErrorString(e));
  }
  CHECK_RC(run_on_groups(ctxs, n, stream, "cola_ic_many", [](const Group& g) { return ic_group(g, false); }));
  for (int i = 0; i < n; ++i) {
    ctxs[i]->step = 0;
    ctxs[i]->ic_done = true;
  }
  return COLA_OK;
}

int32_t cola_batch_steps_done(const cola_batch* b) { return b ? b->step : -1; }

void cola_batch_free(cola_batch* b) {
  if (!b) return;
  if (b->cap_st) cudaStreamSynchronize(b->cap_st);
  cudaStreamSynchronize(b->st);
  for (auto& kv : b->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    dev_free_on(b->ctx[0], kv.second.shifts, b->cap_st);
  }
  dev_free_on(b->ctx[0], b->pk_acc, b->st);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (cudaStream_t s : b->chain_st) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  cudaGetLastError();
  delete b;
}

int cola_profile_enable(cola_ctx* ctx, int32_t on) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->stages.empty()) ctx->stages.resize(ST_COUNT);
  for (auto& stg : ctx->stages) {
    for (auto& pr : stg.pending) {
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
    stg = cola_ctx::Stage();
  }
  ctx->prof = on != 0;
  return COLA_OK;
}

int32_t cola_profile_nstages(void) { return ST_COUNT; }

const char* cola_profile_stage_name(int32_t i) {
  return (i >= 0 && i < ST_COUNT) ? kStageNames[i] : "";
}

int cola_profile_read(cola_ctx* ctx, double* ms, int64_t* launches, double* bytes_per_launch) {
  if (!ctx) return fail(nullptr, COLA_EINVAL, "ctx is NULL");
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->stages.empty()) ctx->stages.resize(ST_COUNT);
  for (int i = 0; i < ST_COUNT; ++i) {
    auto& stg = ctx->stages[i];
    for (auto& pr : stg.pending) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, pr.first, pr.second));
      stg.ms += t;
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
    stg.pending.clear();
    if (ms) ms[i] = stg.ms;
    if (launches) launches[i] = stg.launches;
    if (bytes_per_launch) bytes_per_launch[i] = stg.launches ? stg.bytes / (double)stg.launches : 0.0;
  }
  return COLA_OK;
}

int cola_host_growth(const cola_config* cfg, const cola_model* model, double* out,
                     double* k_nodes_out) {
  g_err.clear();
  int rc = validate_cfg(cfg, nullptr);
  if (rc) return rc;
  rc = validate_model(model, nullptr);
  if (rc) return rc;
  if (!out) return fail(nullptr, COLA_EINVAL, "out is NULL");
  Growth g;
  std::vector<double> k;
  rc = validate_model_range(*cfg, *model, nullptr);
  if (rc) return rc;
  growth_for(*cfg, hmodel(*model), g, &k, nullptr, nullptr);
  const int nk = cfg->nk_table;
  for (int n = 0; n <= cfg->nsteps; ++n) {
    const std::vector<double>* cols[6] = {&g.D1, &g.dD1, &g.ddD1, &g.D2, &g.dD2, &g.ddD2};
    for (int q = 0; q < 6; ++q)
      std::memcpy(out + ((size_t)n * 6 + q) * nk, cols[q]->data() + (size_t)n * nk, nk * sizeof(double));
  }
  if (k_nodes_out) std::memcpy(k_nodes_out, k.data(), nk * sizeof(double));
  return COLA_OK;
}

int64_t cola_device_bytes(const cola_config* cfg) {
  if (validate_cfg(cfg, nullptr) != COLA_OK) return -1;
  cola_ctx probe;
  Layout lay;
  context_layout(&probe, *cfg, lay);
  return (int64_t)lay.size;
}

int cola_host_timesteps(const cola_config* cfg, double* out) {
  g_err.clear();
  int rc = validate_cfg(cfg, nullptr);
  if (rc) return rc;
  if (!out) return fail(nullptr, COLA_EINVAL, "out is NULL");
  const std::vector<double> a = a_nodes(*cfg);
  for (int n = 0; n < cfg->nsteps; ++n) {
    const double a0 = a[n], a1 = a[n + 1], am = 0.5 * (a0 + a1);
    out[4 * n + 0] = a1;
    out[4 * n + 1] = hdtau(a0, am, cfg->Omega_m);
    out[4 * n + 2] = hdtau(a0, a1, cfg->Omega_m);
    out[4 * n + 3] = hdtau(am, a1, cfg->Omega_m);
  }
  return COLA_OK;
}

}  // extern "C"
