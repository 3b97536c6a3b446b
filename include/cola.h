/*
 * cola.h - C ABI of libcola: one COLA particle-mesh simulation with
 * scale-dependent growth and approximate screening on one GB300 (sm_103a).
 *
 * Method: Winther, Koyama, Manera, Wright & Zhao, "COLA with scale-dependent
 * growth: applications to screened modified gravity models" (arXiv:1703.00879).
 * Section references below are to that paper.
 *
 * Conventions shared by every entry point
 *   - Units: lengths Mpc/h, wavenumbers h/Mpc, time 1/H0 (H0 = 1); the time
 *     variable is tau with dtau = dt/a^2 (Sec. 1).  Velocities returned by
 *     cola_snapshot are peculiar velocities in km/s.
 *   - Particles: Np^3 unit-mass particles, particle p = (z*Np + y)*Np + x sits
 *     at the Lagrangian lattice point q = (x, y, z) * Lbox/Np.
 *   - Mesh arrays: Nmesh^3, indexed [z][y][x] with x fastest.  Half spectra:
 *     [kz][ky][kx], kx = 0..N/2 fastest (N/2+1 entries per row), complex
 *     numbers as interleaved float pairs.  Forward transforms are
 *     unnormalised (sum x e^{-ikx}).
 *   - Return value: COLA_OK (0) on success, a negative COLA_E* code on
 *     failure; no call aborts or prints.  The message of the last failure is
 *     returned by cola_last_error (a context-free failure, e.g. in cola_init
 *     before the context exists, is reported by cola_last_error(NULL)).
 *   - Memory: every device byte a context uses comes through the alloc/free
 *     callbacks given to cola_init (NULL callbacks: cudaMallocAsync /
 *     cudaFreeAsync on the stream).  The per-context buffers, including the
 *     context's copy of its twiddle, growth and per-step tables, are ONE
 *     allocation, released in cola_free.  Batches and multi-context calls
 *     allocate their small shift and P(k) arrays through the first context's
 *     callbacks.  The library itself never calls cudaMalloc or cudaFree; the
 *     host keeps computed growth tables in a bounded host cache and stages
 *     uploads through a pinned host ring per device, allocated at the first
 *     cola_init on that device,
 *     so creating, stepping and freeing contexts never synchronises the
 *     device.  Buffers passed in by the caller stay owned by the caller.
 *   - Allocator contract: alloc(bytes, stream, user) returns memory usable on
 *     `stream`, aligned to 256 bytes as cudaMalloc's is (cola_init releases a
 *     misaligned block and fails with COLA_EINVAL); free(ptr, stream, user)
 *     releases it in stream order (later work on `stream` may reuse it,
 *     earlier work still sees it), as PyTorch's caching allocator and
 *     cudaFreeAsync do.
 *   - Streams: all device work is enqueued on the stream given to cola_init
 *     (borrowed, never destroyed).  Calls that take or return HOST buffers
 *     wait on the host for that stream before returning (bounded by
 *     cola_set_wait_limit); calls with DEVICE buffers do not.
 *   - No CPU fallback: every step of the method runs in the library's CUDA
 *     kernels; without a usable GPU cola_init fails with COLA_ECUDA.
 */
#ifndef COLA_H
#define COLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  COLA_OK = 0,
  COLA_EINVAL = -1,   /* bad argument or unsupported size */
  COLA_ENOMEM = -2,   /* the allocator returned NULL */
  COLA_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
  COLA_ESTATE = -4,   /* calls made in the wrong order */
  COLA_ETIMEOUT = -5  /* a host wait for device work ran past the context's wait limit
                         (cola_set_wait_limit); the work stays queued */
};

/* Model kinds. */
enum { COLA_LCDM = 0, COLA_FOFR = 1, COLA_NDGP = 2, COLA_SYMM = 3, COLA_MB = 4 };

/* Where a caller-owned buffer lives. */
enum { COLA_HOST = 0, COLA_DEVICE = 1 };

/* Precision of the stored k-space LPT potentials (the seed fields). */
enum { COLA_SEED_FP32 = 0, COLA_SEED_BF16 = 1, COLA_SEED_FP16 = 2 };

typedef struct cola_ctx cola_ctx;

/* Device allocator: return `bytes` of device memory usable on `stream`, or NULL. */
typedef void* (*cola_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*cola_free_fn)(void* ptr, void* stream, void* user);

/* Run configuration.  Flat LCDM background (Omega_L = 1 - Omega_m, App. B);
 * Gaussian initial field with the Eisenstein-Hu no-wiggle spectrum
 * normalised to sigma8 at z = 0 and scaled to z_ini with the LCDM growth
 * factor; nsteps COLA steps uniform in a from z_ini to z_final. */
typedef struct {
  double Omega_m, Omega_b, h, n_s, sigma8;
  double Lbox;             /* box side [Mpc/h] */
  int32_t Np;              /* particles per side: power of two, 32..512 */
  int32_t Nmesh;           /* PM mesh cells per side: power of two, 32..1024 */
  double z_ini, z_final;
  int32_t nsteps;          /* >= 1 */
  uint64_t seed;           /* Philox-4x32-10 key of the white noise */
  int32_t seed_precision;  /* COLA_SEED_* */
  int32_t nk_table;        /* log-k nodes of the growth tables, >= 16 (1024 typical) */
} cola_config;

/* Gravity model (Sec. 5, Sec. 6, App. B). */
typedef struct {
  int32_t kind;            /* COLA_LCDM, COLA_FOFR (Hu-Sawicky n = 1), COLA_NDGP, COLA_SYMM, COLA_MB */
  double fR0;              /* |f_R0| (f(R) only, > 0) */
  double rcH0;             /* r_c H0 (nDGP only, > 0) */
  int32_t screening;       /* 1: approximate screening of the fifth force (Sec. 6) */
  int32_t filter;          /* smoothing window of the Vainshtein density (App. B), x = kR:
                              0 Gaussian exp(-x^2/2), 1 top-hat 3 (sin x - x cos x)/x^3,
                              2 sharp-k (1 for x <= 1, else 0; the cut decided in single
                              precision); any other value fails with COLA_EINVAL */
  double R_smooth;         /* smoothing radius [Mpc/h] (nDGP screening) */
  int32_t scale_dependent; /* 1: per-k growth D(k,a) (Sec. 4); 0: LCDM growth factors */
  /* Symmetron, the App. C {m(a), beta(a)} model with chameleon-type screening:
     beta(a) = beta_star sqrt(u), m^2(a) = (m_star H0)^2 u, u = 1 - (a_star / a)^3,
     both 0 for a <= a_star.  Fifth force C = 2 beta^2 with range 1/m;
     eps = min(1, Phi_crit / |Phi_N|) with Phi_crit = 3 Omega_m / (a_star^3 m_star^2),
     the App. C integral from a_star. */
  double beta_star;        /* coupling beta at late times, > 0 (symmetron only) */
  double m_star;           /* mass at late times over H0, > 0 (symmetron only); range 2997.92458 / m_star Mpc/h */
  double a_star;           /* symmetry-breaking scale factor in (0, 1] (symmetron only) */
  /* General {m(a), beta(a)} model (App. C), COLA_MB, with chameleon-type screening:
     beta(a) and m(a) / H0 at mb_n scale factors mb_a[0] < ... < mb_a[mb_n - 1],
     2 <= mb_n <= 4096, covering the run's [a_ini, a_final]; beta >= 0, m > 0.
     beta and m^2 are linear in a between nodes (dm^2/da the slope of the node
     interval).  mu = 1 + 2 beta^2 k^2 / (k^2 + a^2 m^2), C = 2 beta^2, range 1/m;
     Phi_crit(a) = mb_phicrit0 + 9 Omega_m / (2 beta(a)) int_{mb_a[0]}^a beta /
     (m^2 / H0^2 a'^4) da'.  The three arrays are caller-owned host memory, read
     during cola_set_model / cola_host_growth only; a violation fails with COLA_EINVAL. */
  const double* mb_a;
  const double* mb_beta;
  const double* mb_m;
  int32_t mb_n;
  double mb_phicrit0;      /* Phi_crit(mb_a[0]) >= 0 */
} cola_model;

/* Creates a context: validates the configuration, allocates every device
 * buffer of the run (particles, LPT grid, PM mesh) in one call of `alloc`,
 * and computes the background quantities.  `stream` is a cudaStream_t (NULL =
 * legacy default stream).  On success *out owns the context; on failure
 * *out is NULL and nothing is leaked.  Errors: COLA_EINVAL (sizes not powers of
 * two in 32..1024, nsteps < 1, nonsensical cosmology), COLA_ENOMEM, COLA_ECUDA. */
int cola_init(const cola_config* cfg, cola_alloc_fn alloc, cola_free_fn free_fn, void* user,
              void* stream, cola_ctx** out);

/* Sets the gravity model and solves, in double precision on the host, the
 * growth ODEs of Sec. 4.1 (D1'' = kappa mu(k,a) D1) and Eq. fofrapprox
 * (approximate second-order D2 with gamma_2(k, k/sqrt2, k/sqrt2, a)) on
 * nk_table log-spaced k nodes at every step boundary (once per distinct
 * configuration and model: the host keeps the result in a bounded cache), and
 * copies the float tables into the context's own allocation, asynchronously
 * on its stream.  Never synchronises the device.  Must precede cola_ic.  Errors: COLA_EINVAL (unknown kind,
 * non-positive fR0/rcH0/R_smooth where needed), COLA_ESTATE (after cola_ic). */
int cola_set_model(cola_ctx* ctx, const cola_model* model);

/* Scale-independent LPT fast path (on = 1; 0 restores the default).  When the
 * growth of the model does not depend on k (LCDM; nDGP; any model with
 * scale_dependent = 0) the LPT fields of every step are c1 Psi1 + c2 Psi2 of
 * the real-space 2LPT displacements Psi_i = grad phi_i (Sec. 4.1 with
 * D(k, a) = D(a)): Psi1 and Psi2 are transformed once, at cola_ic, and kept
 * per particle, and each step forms its drift and kick fields in the particle
 * kernels instead of running the six LPT inverse transforms.  The results
 * equal those of the default path up to FP32 rounding.  COLA_F_LPT_DISP /
 * COLA_F_LPT_ACC export the last step's fields formed the same way.  Must
 * follow cola_set_model and precede cola_ic.  Errors: COLA_EINVAL (the growth
 * depends on k), COLA_ESTATE (no model yet, or after cola_ic). */
int cola_set_lpt_fast(cola_ctx* ctx, int32_t on);

/* Initial conditions (Sec. 3, Sec. 4.1, App. A): Philox white noise on the Np^3
 * lattice, delta(k) with P_ini(k), phi1 = delta/k^2, phi2 from the 2LPT
 * source (Eq. lcdm2lpt); stores phi1(k), phi2(k) (the k-space seed fields),
 * places particles on the 2LPT trajectory at a_ini and evaluates the initial
 * force.  Errors: COLA_ESTATE (no model), COLA_ECUDA. */
int cola_ic(cola_ctx* ctx);

/* Same as cola_ic but with caller-provided potentials phi1(k), phi2(k):
 * Np*Np*(Np/2+1) complex values each (interleaved float pairs, unnormalised
 * forward-DFT convention, phi(k=0) ignored), on the host or the device. */
int cola_ic_from_potentials(cola_ctx* ctx, const float* phi1, const float* phi2, int32_t where);

/* Advances `nsteps` COLA steps (Sec. 2, App. A; -1 = to z_final): per step the
 * LPT reweight and inverse FFTs of the displacement and acceleration fields,
 * the drift with CIC deposit, the forward FFT, the screened Poisson solve,
 * the force inverse FFTs and the CIC gather with the kick.  Within one call of
 * two or more steps (FP32 fields, per-k LPT path) the kick of each step but
 * the last and the drift + deposit of the next run as one pass over the
 * particles, with the next step's LPT fields formed first; the state after the
 * call is that of the same number of single steps (up to the order of the
 * deposit's float additions).  Asynchronous on the stream.  Errors:
 * COLA_ESTATE (before cola_ic), COLA_EINVAL (past the last step), COLA_ECUDA. */
int cola_step(cola_ctx* ctx, int32_t nsteps);

/* Particle positions (wrapped into [0, Lbox), [Np^3][3] floats, Mpc/h) and
 * peculiar velocities ([Np^3][3] floats, km/s) at the current scale factor,
 * written to caller-owned buffers on the host or device; either pointer may
 * be NULL.  Host buffers wait for the stream (bounded by cola_set_wait_limit).
 * Page-locked host buffers that the device can address (cudaHostAlloc, or
 * registered and mapped) are written by the snapshot kernel directly, without
 * a device staging buffer or a copy; other host buffers are staged and copied.
 * If the wait gives up (COLA_ETIMEOUT) the device may still be writing the
 * buffers: keep them until the stream has drained. */
int cola_snapshot(cola_ctx* ctx, float* pos, float* vel, int32_t where);

/* Matter power spectrum of the current particles: CIC on the Nmesh mesh,
 * deconvolved by the CIC window, linear bins b = 0..nbins-1 covering
 * |k| in [(b+1/2) k_F, (b+3/2) k_F), k_F = 2 pi/Lbox, no shot-noise
 * subtraction.  Host arrays of nbins entries (k = mean |k| of the bin's modes,
 * pk in (Mpc/h)^3, nmodes = number of modes); any may be NULL.  Waits for the
 * stream (bounded by cola_set_wait_limit: on COLA_ETIMEOUT the outputs are not
 * written).  Errors: COLA_EINVAL, COLA_ESTATE (no ICs, or a cola_pk_async result
 * still pending), COLA_ECUDA, COLA_ETIMEOUT. */
int cola_pk(cola_ctx* ctx, int32_t nbins, double* k, double* pk, int64_t* nmodes);

/* Non-blocking P(k): cola_pk_async enqueues the same computation and a copy
 * of the bin sums into a pinned host buffer owned by the context, and returns
 * at once; cola_pk_ready returns 1 when that copy has landed (0 while pending);
 * cola_pk_result waits for it if needed (bounded by cola_set_wait_limit; on
 * COLA_ETIMEOUT the request stays pending and may be collected later) and fills
 * k, pk, nmodes like cola_pk.  One request per context may be pending.  Errors:
 * COLA_EINVAL, COLA_ESTATE (no ICs; a request already pending / none pending),
 * COLA_ECUDA, COLA_ETIMEOUT. */
int cola_pk_async(cola_ctx* ctx, int32_t nbins);
int cola_pk_ready(cola_ctx* ctx);
int cola_pk_result(cola_ctx* ctx, double* k, double* pk, int64_t* nmodes);

/* Moves the context to another stream: work already queued on the old stream
 * runs before anything later enqueued on the new one (an event wait, no host
 * synchronisation).  Errors: COLA_EINVAL, COLA_ECUDA. */
int cola_set_stream(cola_ctx* ctx, void* stream);

/* Failure detection: the number of non-finite values (NaN, +-Inf) in the particle
 * state (displacement, residual velocity and residual acceleration: 9 Np^3 floats),
 * counted on the device, in *nonfinite (0: the state is finite).  A run that went
 * unstable (too few steps for its model, a corrupted import) shows here before
 * its P(k) does.  Waits for the stream (bounded by cola_set_wait_limit).  The paper
 * has no counterpart.  Errors: COLA_EINVAL, COLA_ESTATE (no ICs yet, or a
 * cola_pk_async result pending), COLA_ECUDA (also, with *nonfinite set, when a
 * transform kernel on this device ever gave up on a tile load after its one-second
 * wait: every result since is invalid), COLA_ETIMEOUT. */
int cola_check_state(cola_ctx* ctx, int64_t* nonfinite);

/* Bounded host waits.  Every call that waits on the host for the context's
 * stream (host-buffer snapshots, exports and imports, cola_pk, cola_pk_result,
 * cola_wait) gives up after `seconds` with COLA_ETIMEOUT when seconds > 0
 * (0, the default: wait without limit).  The device work stays queued and
 * completes later; the context stays usable.  After a timed-out call with a
 * caller-owned HOST destination, that buffer is written when the queued copy
 * completes: keep it alive and call cola_wait (returns COLA_OK once the stream
 * has drained) before reading or releasing it.  The paper has no counterpart:
 * this serves callers with a latency budget, such as a request loop.  Errors:
 * COLA_EINVAL (negative or non-finite limit). */
int cola_set_wait_limit(cola_ctx* ctx, double seconds);
int cola_wait(cola_ctx* ctx);

/* Self-test of the one wait on the device.  The transform passes that stage their
 * tiles with TMA wait on an mbarrier for each tile's copies, for one second at
 * most; a CTA whose wait runs out is counted and stops, and cola_check_state
 * reports COLA_ECUDA.  This call runs that wait, with limit `seconds`
 * (0 < seconds <= 10), on a barrier phase that no copy completes, on the current
 * device's per-thread default stream, and waits for it: *timed_out = 1 when the
 * wait gave up (the expected result), 0 otherwise.  Nothing is allocated and no
 * context is needed.  Errors: COLA_EINVAL (limit out of range, NULL timed_out),
 * COLA_ECUDA. */
int cola_selftest_wait(double seconds, int* timed_out);

/* Current scale factor (NaN for a NULL context) and completed steps. */
double cola_scale_factor(const cola_ctx* ctx);
int32_t cola_steps_done(const cola_ctx* ctx);

/* Message of the last failure on ctx (or of the last context-free failure for
 * NULL); empty string if none.  Owned by the library. */
const char* cola_last_error(const cola_ctx* ctx);

/* Releases every device buffer of the context through the free callback and
 * destroys it.  Synchronises the stream first.  NULL is a no-op. */
void cola_free(cola_ctx* ctx);

/* ---------------------------------------------------------------------
 * State access (checkpoint/resume and per-stage inspection).
 * --------------------------------------------------------------------- */

/* Internal arrays that cola_export / cola_import copy.  Layouts:
 *   COLA_F_DISP, COLA_F_DV, COLA_F_ACC : [3][Np^3] floats (SoA x, y, z): the
 *       displacement s = x - q, the COLA residual velocity delta_v = dx/dtau
 *       - dPsi_LPT/dtau, and the last residual acceleration (force - A_LPT).
 *   COLA_F_RHO     : [Nmesh^3] floats, CIC mass per cell of the last deposit.
 *   COLA_F_DELTAK  : [Nmesh][Nmesh][Nmesh/2+1] complex, DFT of delta of the
 *                    last force evaluation (unnormalised).
 *   COLA_F_FORCE   : [3][Nmesh^3] floats, the last mesh force -grad Phi_tot.
 *   COLA_F_PHI1, COLA_F_PHI2 : [Np][Np][Np/2+1] complex, the seed potentials.
 *   COLA_F_LPT_DISP, COLA_F_LPT_ACC : [3][Np^3] floats, the last LPT
 *       displacement increment and LPT acceleration fields at the lattice. */
enum {
  COLA_F_DISP = 0, COLA_F_DV = 1, COLA_F_ACC = 2, COLA_F_RHO = 3, COLA_F_DELTAK = 4,
  COLA_F_FORCE = 5, COLA_F_PHI1 = 6, COLA_F_PHI2 = 7, COLA_F_LPT_DISP = 8, COLA_F_LPT_ACC = 9
};

/* Copies internal array `which` to a caller-owned buffer (host or device).
 * Errors: COLA_EINVAL (unknown array), COLA_ESTATE (array not computed yet). */
int cola_export(cola_ctx* ctx, int32_t which, void* dst, int32_t where);

/* Restores the particle state (COLA_F_DISP, COLA_F_DV, COLA_F_ACC from the
 * same step) and the step counter, e.g. from a checkpoint of an identical
 * run.  cola_ic must have run (the seed potentials are needed). */
int cola_import_state(cola_ctx* ctx, const float* disp, const float* dv, const float* acc,
                      int32_t steps_done, int32_t where);

/* ---------------------------------------------------------------------
 * Stage entry points (the same kernels as cola_step, on caller data).
 * --------------------------------------------------------------------- */

/* 3-D FFT on the context's Nmesh mesh.  dir = +1: real [N^3] -> half spectrum
 * [N][N][N/2+1] complex (unnormalised forward); dir = -1: half spectrum ->
 * real (unnormalised inverse; imaginary parts of the kx = 0 and kx = N/2
 * entries are ignored after the ky, kz transforms).  in/out on the host or
 * device (both on the same side). */
int cola_fft(cola_ctx* ctx, int32_t dir, const void* in, void* out, int32_t where);

/* CIC deposit of n positions ([n][3] floats, Mpc/h, any real values; wrapped
 * periodically) with unit mass onto the Nmesh mesh; writes [Nmesh^3] floats. */
int cola_cic_deposit(cola_ctx* ctx, const float* pos, int64_t n, float* rho, int32_t where);

/* Mesh force of App. B for the current model at scale factor a from a given
 * CIC density (mass per cell, [Nmesh^3] floats, mean Np^3/Nmesh^3): writes
 * [3][Nmesh^3] floats -grad Phi_tot. */
int cola_force_from_density(cola_ctx* ctx, const float* rho, double a, float* force,
                            int32_t where);

/* ---------------------------------------------------------------------
 * Batches: many simulations of one shape advanced together (ensembles).
 * --------------------------------------------------------------------- */
typedef struct cola_batch cola_batch;

/* How one batch step is launched.  The contexts, in batch order, are split
 * into groups of `group` consecutive contexts; every kernel of the step runs
 * ONCE per group over all of its contexts (a tile index that spans the
 * group's simulations; the model-dependent force stages run once per model
 * subset of the group).  Multi-simulation groups need contexts of one shape:
 * equal Np, Nmesh, Lbox, nk_table and seed_precision (seeds, models and
 * cosmologies may differ); otherwise groups have one context.  Groups are
 * spread round-robin over `chains` concurrent streams; `grid_cap` > 0 bounds
 * the persistent grid of every FFT pass so concurrent groups share the SMs.
 * deposit_box / gather_box choose the particle kernels of the step: 0 the
 * direct ones (CIC deposit by global atomics merged within each warp; gather
 * by direct loads of the mesh); > 0 the shared-memory box kernels, where each
 * CTA takes an 8 x 8 x 8 block of the Lagrangian lattice and bins its deposit
 * in, or stages its gather from, a box of at most that many mesh cells in
 * shared memory (deposit <= 16384, gather <= 8192; larger values are clamped,
 * values are rounded down to a multiple of 4; a block whose box does not fit
 * uses the direct path).  The results agree to float rounding either way. */
typedef struct {
  int32_t group;       /* contexts per group; <= 0: all (one shape) or 1 */
  int32_t chains;      /* concurrent streams, >= 1 */
  int32_t grid_cap;    /* CTAs per FFT pass, 0 = no cap */
  int32_t deposit_box; /* shared-memory deposit bins (cells), 0 = direct atomics */
  int32_t gather_box;  /* shared-memory gather box (cells), 0 = direct loads */
} cola_batch_plan;

/* Groups 1..65535 distinct contexts that completed cola_ic, have equal nsteps
 * and steps done, and live on the current device.  Each step of
 * cola_batch_step is ONE CUDA graph launch on `stream` that advances every
 * context by one step: the launch sequence of the plan (NULL: one group over
 * all contexts of one shape, else one context per group on one chain) is
 * captured once, instantiated and replayed for every step (the step index
 * and each simulation's per-step parameters are read on the device).
 * Contexts whose own stream differs from `stream` get ordered behind each
 * batch step.  The batch borrows the contexts (free the batch before them).
 * Errors: COLA_EINVAL, COLA_ESTATE, COLA_ECUDA (message via cola_last_error(NULL)). */
int cola_batch_create(cola_ctx* const* ctxs, int32_t n, const cola_batch_plan* plan, void* stream,
                      cola_batch** out);
int cola_batch_set_plan(cola_batch* b, const cola_batch_plan* plan);
int cola_batch_get_plan(const cola_batch* b, cola_batch_plan* out);
/* Advances every context by nsteps (-1: to the last step).  With two or more
 * steps, direct particle kernels (deposit_box = gather_box = 0) and every
 * context on the FP32 per-k LPT path, the step boundaries are fused as in
 * cola_step (the kick of each step but the last and the drift + deposit of
 * the next in one pass): nsteps + 1 graph launches, the same state as nsteps
 * single steps up to the order of the deposit's float additions.  When stage
 * timing is enabled on the first context (cola_profile_enable), the steps are
 * launched without a graph, group after group on one stream, so that the
 * first group's stage timings (covering all of its simulations) are recorded. */
int cola_batch_step(cola_batch* b, int32_t nsteps);
/* Autotuner: times up to max_steps real steps (they advance the batch), one
 * per candidate plan, and keeps the fastest for later steps; *best_out
 * receives it (may be NULL).  Candidates: first the launch grouping (one
 * group over everything; halves and quarters on concurrent chains; small
 * groups on many chains with a capped grid), then, with the best grouping,
 * the particle kernels (deposit bins of 4096 and 16384 cells against direct
 * atomics, gather boxes of 4096 and 8192 cells against direct loads). */
int cola_batch_autotune(cola_batch* b, int32_t max_steps, cola_batch_plan* best_out);
/* Matter power spectrum of every context (same estimator and bins as
 * cola_pk), computed by multi-simulation launches with one synchronisation:
 * k, pk, nmodes are host arrays [n][nbins] in batch order (each may be NULL). */
int cola_batch_pk(cola_batch* b, int32_t nbins, double* k, double* pk, int64_t* nmodes);
int32_t cola_batch_steps_done(const cola_batch* b);
void cola_batch_free(cola_batch* b);

/* Continuous batching: advances each of n distinct contexts (each after
 * cola_ic and before its last step) by ONE step, enqueued on `stream`.
 * Contexts of one shape (equal Np, Nmesh, Lbox, nk_table, seed_precision;
 * their models, seeds, step counts and progress may differ) share one
 * multi-simulation launch sequence.  No graph, no device allocation beyond
 * a stream-ordered shift array, no host synchronisation: a serving loop
 * calls it once per tick over whatever requests are in flight.  Work queued
 * on a context's own stream before the call runs before its step, work
 * queued after the call runs after it.  Errors: COLA_EINVAL (NULL, duplicate,
 * finished or too many contexts), COLA_ESTATE (no ICs), COLA_ECUDA;
 * message via cola_last_error(NULL). */
int cola_step_many(cola_ctx* const* ctxs, int32_t n, void* stream);

/* Initial conditions of n distinct contexts (each after cola_set_model and
 * before cola_ic) with multi-simulation launches on `stream`: what cola_ic
 * computes for each, from each context's own seed, spectrum and model,
 * contexts of one shape (as for cola_step_many) sharing every launch.  No
 * host synchronisation; ordering with the contexts' own streams as for
 * cola_step_many.  Errors: COLA_EINVAL, COLA_ESTATE (no model, or ICs already
 * done), COLA_ECUDA; message via cola_last_error(NULL). */
int cola_ic_many(cola_ctx* const* ctxs, int32_t n, void* stream);

/* ---------------------------------------------------------------------
 * Per-stage device timing: CUDA events recorded on the context's stream
 * around each launch group of cola_step (and of cola_ic's force evaluation).
 * --------------------------------------------------------------------- */

/* on = 1 clears the accumulators and starts recording; on = 0 stops. */
int cola_profile_enable(cola_ctx* ctx, int32_t on);

/* Number of stages and the name of stage i (static strings). */
int32_t cola_profile_nstages(void);
const char* cola_profile_stage_name(int32_t i);

/* Synchronises the stream and returns, per stage, the accumulated device
 * milliseconds, the number of kernel launches, and the mean algorithmic
 * bytes per launch: the stage's algorithmic bytes (each array the stage
 * needs read once and written once, whatever the number of kernels it takes;
 * CIC deposit counts the mesh read and written once) divided by its launches,
 * so launches x bytes_per_launch is the stage's algorithmic traffic.  Arrays
 * of cola_profile_nstages() entries; any may be NULL. */
int cola_profile_read(cola_ctx* ctx, double* ms, int64_t* launches, double* bytes_per_launch);

/* ---------------------------------------------------------------------
 * Allocation-free power spectrum.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a P(k) - cudaFree (and cudaMalloc when a pool grows) synchronises the whole
 * device and would stall the other streams of a latency-bound serving loop,
 * a process whose device memory is held by another allocator may get no
 * fresh memory, and a diagnostic inside a long run must not fail on an
 * allocation.
 *
 * It computes what cola_pk computes (CIC deposit, CIC-deconvolved |delta(k)|^2,
 * the same bins) for caller-given positions, using only a file-scope device
 * scratch array of fixed size that every GPU loading the library holds until
 * the process exits (about 18.6 MB: room for a COLA_PK_NOALLOC_MAX_NMESH^3
 * mesh, its half spectrum, twiddles and 2000 bins).
 *   pos    : DEVICE pointer, [n][3] floats, Mpc/h (wrapped periodically), n > 0
 *   nmesh  : power of two in 32..COLA_PK_NOALLOC_MAX_NMESH; larger meshes are
 *            rejected with COLA_EINVAL
 *   Lbox   : box side [Mpc/h];  nbins: 1..2000
 *   k, pk, nmodes : HOST arrays of nbins entries (any may be NULL), as cola_pk
 *   stream : cudaStream_t for the work.  The call copies its bin sums to the
 *            host and synchronises this stream before returning, so it must
 *            not be called while the stream is being captured into a graph.
 * No cudaMalloc, cudaFree or allocating library routine is called.  The
 * scratch is reserved when its module loads; with CUDA's lazy module loading
 * that would be the first use, so cola_init loads it, once per device, with
 * that device current (a failure there makes cola_init return COLA_ECUDA).
 * A caller that never creates a context reserves it with its first
 * cola_pk_noalloc call on the device, which may then fail with COLA_ECUDA if
 * the device is out of memory.  Every call asks for the scratch's device
 * address (cudaGetSymbolAddress) with the device current, so no cached
 * address outlives a device reset.  All calls on a device share the scratch
 * and it keeps the last call's contents (each call clears what must start at
 * zero), so calls whose device work could overlap race and must not be
 * issued.  Errors: COLA_EINVAL, COLA_ECUDA; message in cola_last_error(NULL).
 * --------------------------------------------------------------------- */
#define COLA_PK_NOALLOC_MAX_NMESH 128
int cola_pk_noalloc(const float* pos, int64_t n, int32_t nmesh, double Lbox, int32_t nbins,
                    double* k, double* pk, int64_t* nmodes, void* stream);

/* ---------------------------------------------------------------------
 * Host-only helpers (no GPU needed): the double-precision quantities the
 * library computes on the host and uploads.  Same validation as cola_init /
 * cola_set_model.
 * --------------------------------------------------------------------- */

/* Growth tables of Sec. 4.1 and Eq. fofrapprox at the nsteps+1 step boundaries
 * a_n = a_ini + n (a_final - a_ini)/nsteps, on the nk_table log-spaced nodes
 * k_j = k0 exp(j dlnk), k0 = pi/Lbox, k_last = 1.01 sqrt(3) pi Np/Lbox.
 * out: [nsteps+1][6][nk_table] doubles = D1, dD1/dtau, d2D1/dtau2, D2,
 * dD2/dtau, d2D2/dtau2 (D1 = 1, D2 = -3/7 at a_ini).  k_nodes (optional):
 * [nk_table] wavenumbers in h/Mpc. */
int cola_host_growth(const cola_config* cfg, const cola_model* model, double* out,
                     double* k_nodes);

/* Device bytes cola_init allocates for cfg: the one allocation holding every
 * buffer of a context, its own copy of the twiddle, growth and per-step tables
 * included (for admission control); -1 if cfg is invalid. */
int64_t cola_device_bytes(const cola_config* cfg);

/* Time integrals of the kick-drift-kick step (Sec. 2; dtau = dt/a^2):
 * out: [nsteps][4] doubles = a_{n+1}, Delta tau(a_n, a_{n+1/2}),
 * Delta tau(a_n, a_{n+1}), Delta tau(a_{n+1/2}, a_{n+1}), a_{n+1/2} = (a_n + a_{n+1})/2. */
int cola_host_timesteps(const cola_config* cfg, double* out);

#ifdef __cplusplus
}
#endif

#endif /* COLA_H */
