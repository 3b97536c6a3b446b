// Internal declarations shared by the host code and the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector_types.h>

#include <string>

namespace cola {

// Row pitch (in complex elements) of every half spectrum: N/2+1 rounded up to
// 16 so that column tiles of 2..16 elements never straddle a row.
__host__ __device__ constexpr int64_t half_pitch(int N) { return ((N / 2 + 1 + 15) / 16) * 16; }
inline int64_t half_elems(int N) { return (int64_t)N * N * half_pitch(N); }

// Half-spectrum layout.  The rows (z, y) of the planes z = 2j and 2j + 1 are
// interleaved in chunks of 8 complex values (64 bytes):
//   element (z, y, kx) at ((z >> 1) N + y) 2P + (kx >> 3) 16 + (z & 1) 8 + (kx & 7),
// P = half_pitch(N).  A pass along z then reads 128 contiguous bytes per pair of
// planes where the plain [z][y][kx] order gives 64-byte pieces one plane
// (N P 8 bytes) apart.  Rows are also numbered pair-major,
// q = ((z >> 1) N + y) 2 + (z & 1), so that TW consecutive rows q (TW even)
// fill a contiguous block of TW P elements.
__host__ __device__ inline int64_t hcol(int kx) { return (int64_t)(kx >> 3) * 16 + (kx & 7); }
__host__ __device__ inline int64_t hrow(int z, int y, int N, int64_t P) {
  return ((int64_t)(z >> 1) * N + y) * 2 * P + (z & 1) * 8;
}
__host__ __device__ inline int64_t hidx(int z, int y, int kx, int N, int64_t P) {
  return hrow(z, y, N, P) + hcol(kx);
}
// start of pair-major row q, and the index z N + y of the real-space row it belongs to
__host__ __device__ inline int64_t hrow_q(int64_t q, int64_t P) { return (q >> 1) * 2 * P + (q & 1) * 8; }
__host__ __device__ inline int64_t real_row_q(int64_t q, int N) {
  const int64_t pr = q >> 1;  // (z >> 1) N + y
  return ((pr / N) * 2 + (q & 1)) * N + pr % N;
}

struct SimHeader;

// Parameters of one force evaluation (App. B field equation).
struct ForceParams {
  float kf;          // 2 pi / L
  float kappa_norm;  // kappa(a) / N^3 (the inverse transforms are unnormalised)
  float C;           // fifth-force coupling C(a) (0 for LCDM)
  float a2m2;        // a^2 m^2(a)  [(h/Mpc)^2]
  float inv_rhobar;  // Nmesh^3 / Np^3
  float fr_thr;      // f(R), symmetron: Phi_crit(a) a^2 c^2, threshold on |Phi_N| in code units
  float dgp_coef;    // nDGP: 8 (r_c H0)^2 Omega_m / (9 beta^2)
  float R2half;      // nDGP: R_smooth^2 / 2
  float norm;        // 1 / N^3
  int model;         // screening family: 0 none (LCDM), 1 chameleon-type (f(R), symmetron), 2 Vainshtein (nDGP)
  int screened;      // 1: screened fifth force
  int filter;        // nDGP: smoothing window of the density, 0 Gaussian, 1 top-hat, 2 sharp-k
  // When hdr is set, kernels replace every value above by the simulation's
  // own: the current step's entry hdr->dfp[hdr->step], or hdr->fp_ini when ini
  // is set (hdr moved by the simulation's shift).
  const SimHeader* hdr;
  int ini;
};

// Eisenstein-Hu no-wiggle spectrum of the initial conditions.
struct EHDev {
  double theta2, s, alpha, Omh, h, ns, amp;  // amp: A (D(a_ini)/D(1))^2
  double N3_over_L3;
};

// Per-simulation device header: where its per-step parameters live and how many
// steps it has done.  Kernels that serve every step read their parameters
// through it, so one captured launch sequence serves every step.  The second
// group of fields parameterises the initial conditions, so that one launch
// sequence can set up many simulations.
struct SimHeader {
  const ForceParams* dfp;  // [nsteps]: force parameters at a_{n+1}
  const float* ddt;        // [nsteps][3]: half kick, drift, half kick time integrals
  const float4* tab;       // [nsteps+2][nk] LPT reweight table (row 0: a_ini, row n+1: step n,
                           // row nsteps+1: (1, 0, 0, 1), the Psi1 / Psi2 pass)
  const float4* vtab;      // [nsteps+2][nk] velocity table (last row unused)
  int step;                // steps done
  float seed_scale[2];     // dequantisation scales of the 16-bit seeds (written on the device)
  float seed_target;       // 16-bit seeds: the largest |component| maps to this
  unsigned long long seed; // white-noise seed
  EHDev eh;                // spectrum of the initial conditions
  ForceParams fp_ini;      // force parameters at a_ini
  // Reduced-precision LPT fields (16-bit per-step drift and kick fields, one
  // FP32 scale per field; written on the device only): lq_scale quantises the
  // next pass, lq_used dequantises the fields of the current step, lq_amax
  // collects the largest |value| a pass writes (delayed scaling).
  float lq_scale[6];
  float lq_used[6];
  float lq_amax[6];
  // per table row n: (max_k |c1|, max_k |e1|), the growth coefficient of Psi1 in
  // the drift and in the kick fields; their ratio between consecutive rows
  // predicts how the fields grow from one pass to the next
  const float2* lqg;
};

// One launch over several simulations of one shape.  Each simulation's
// buffers sit at the same offsets of its own allocation, so simulation b's
// pointers are simulation 0's moved by shift[b] bytes.  shift == nullptr: a
// single simulation.  Read-only tables equal in every simulation of a launch
// (twiddles) are read from the first simulation's copy, unmoved; per-simulation
// parameters are reached through the moved SimHeader.
struct Multi {
  const int64_t* shift = nullptr;
  int nb = 1;
};

template <class T>
__host__ __device__ __forceinline__ T* moved(T* p, int64_t by) {
  return p ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + by) : p;
}
__device__ __forceinline__ int64_t shift_of(const Multi& m, int b) { return m.shift ? m.shift[b] : 0; }


__device__ __forceinline__ void resolve(ForceParams& fp, int64_t by) {
  if (fp.hdr) {
    const SimHeader* h = moved(fp.hdr, by);
    fp = fp.ini ? h->fp_ini : h->dfp[h->step];
  }
}


// Parameters of the per-k LPT reweight (Sec. 4.1): table of float4 per log-k node.
struct LptParams {
  const SimHeader* hdr;  // table and seed scales of the simulation (moved per simulation)
  int vel;               // 0: hdr->tab, 1: hdr->vtab
  int row0;              // table row; plus hdr->step when add_step
  int add_step;
  const float4* row;     // resolved table row (set on the device when hdr is resolved)
  float scale[2];        // resolved seed scales
  float lnk0, inv_dlnk;
  int nk;
  float kf;           // 2 pi / L
  float norm;         // 1 / Np^3
  int seed_prec;      // 0 fp32, 1 bf16, 2 fp16
};

__device__ __forceinline__ void resolve(LptParams& lp, int64_t by) {
  if (lp.hdr) {
    const SimHeader* h = moved(lp.hdr, by);
    lp.row = (lp.vel ? h->vtab : h->tab) + (size_t)(lp.row0 + (lp.add_step ? h->step : 0)) * lp.nk;
    lp.scale[0] = h->seed_scale[0];
    lp.scale[1] = h->seed_scale[1];
    lp.hdr = nullptr;
  }
}

// Lattice/particle parameters.
struct PartParams {
  int Np, Nm, lgNp;
  float cellscale;  // Nm / L
  float L;
};

// ------------------------------------------------------------------ FFT passes
// All launchers return cudaGetLastError() of their launch.
cudaError_t fft_xr2c(int N, const float* in, float2* out, float scale, float offset,
                     const float2* tw, cudaStream_t s, Multi m = {});
cudaError_t fft_xc2r(int N, const float2* in, float* out, float kfs, const float2* tw,
                     cudaStream_t s, Multi m = {});
// up to six independent c2r row passes in one launch
cudaError_t fft_xc2r_multi(int N, int njobs, const float2* const* in, float* const* out,
                           const float* kfs, const float2* tw, cudaStream_t s, Multi m = {});
// N >= 256: c2r of the rows of a (x derivative i kfs kx on load) and of b into the
// (x, y) pairs of one interleaved real field xy (2 floats per cell, N^3 cells).
cudaError_t fft_xc2r_pair(int N, const float2* a, const float2* b, float* xy, float kfs, const float2* tw,
                          cudaStream_t s, Multi m = {});
// the same with 16-bit outputs (prec 1 bf16, 2 fp16): job j writes value / hdr->lq_scale[j]
// and adds its largest |value| into hdr->lq_amax[j] (hdr moved per simulation)
cudaError_t fft_xc2r_multi16(int N, int njobs, const float2* const* in, void* const* out,
                             const float* kfs, int prec, const SimHeader* hdr, const float2* tw,
                             cudaStream_t s, Multi m = {});
// axis 1 = y, 2 = z; in place
cudaError_t fft_col(int N, float2* data, int axis, bool inv, const float2* tw, cudaStream_t s,
                    Multi m = {});
// y inverse pass producing the plain transform (out_plain may alias in) and the
// transform of (i kfs f_y) times the input (out_deriv).
cudaError_t fft_yinv2(int N, const float2* in, float2* out_plain, float2* out_deriv, float kfs,
                      const float2* tw, cudaStream_t s, Multi m = {});
// Screening field: forward z of delta (after x, y) -> delta(k) stored in dk_out;
// Phi_N(k) (f(R)) or W(kR) delta(k) (nDGP) -> inverse z -> w_out.
cudaError_t mesh_z_screen_field(int N, const float2* in, float2* dk_out, float2* w_out,
                                const ForceParams& fp, const float2* tw, cudaStream_t s,
                                Multi m = {});
// S = delta eps: c2r of the screening field rows, eps, times delta from rho, r2c.
cudaError_t mesh_x_screen_source(int N, const float2* w_in, const float* rho, float2* s_out,
                                 const ForceParams& fp, const float2* tw, cudaStream_t s,
                                 Multi m = {});
// Forward z of the source (S or delta), Phi_tot(k) and -i kz Phi_tot, inverse z.
// dk (delta(k) after the forward z pass) is read when screened, may be null otherwise.
cudaError_t mesh_z_force(int N, const float2* in, const float2* dk, float2* phi_out,
                         float2* phiz_out, const ForceParams& fp, const float2* tw, cudaStream_t s,
                         Multi m = {});
// LPT: phi1, phi2 -> (c1 phi1 + c2 phi2), i kz (...), (e1 phi1 + e2 phi2), i kz (...),
// each inverse-transformed along z.  phi1/phi2 point to float2 (fp32) or
// 2 x 16-bit pairs (bf16/fp16) according to lp.seed_prec.
// zero_dst: optionally also zero zero_floats floats at zero_dst (each simulation's, moved by
// its shift) in the same launch, by bulk stores riding on the pass; *zeroed = whether it did
// (it does where the pass runs one CTA per SM, N >= 512 on 4-column tiles).
cudaError_t lpt_z(int N, const void* phi1, const void* phi2, float2* o0, float2* o1, float2* o2,
                  float2* o3, const LptParams& lp, const float2* tw, cudaStream_t s,
                  Multi m = {}, float* zero_dst = nullptr, int64_t zero_floats = 0,
                  bool* zeroed = nullptr);

// ------------------------------------------------------------------ particles
cudaError_t part_deposit(const PartParams& pp, const float* sx, const float* sy, const float* sz,
                         float* rho, int64_t P, cudaStream_t s, Multi m = {});
// Kick/drift time integrals: hdr->ddt[3 hdr->step + j] of the simulation when
// hdr is set (j = 0 first half kick, 1 drift, 2 second half kick), else the
// given values.
struct StepDt {
  const SimHeader* hdr;
  float dtk, dtd;
  // 0: the LPT field arguments of the drift / kick are FP32 arrays; 1 bf16, 2
  // fp16: 16-bit arrays dequantised with hdr->lq_used (fields 0..2 drift,
  // 3..5 kick; needs hdr)
  int lq = 0;
};
// Scale-independent LPT fields (the fast path for k-independent growth): the
// LPT fields of a step are c1 Psi1 + c2 Psi2 of the real-space fields
// Psi_i = grad phi_i kept per particle (Sec. 4.1 with D(k, a) = D(a)).  When
// `on`, a kernel reads the coefficients from row row0 (+ the simulation's step
// when add_step) of its growth table (tab, or vtab when vel) at k index 0:
// (c1, c2) = .xy for the drift, (e1, e2) = .zw for the kick, (dD1, dD2) = .xy
// of vtab for the snapshot velocity.  The kernel's own LPT field pointers then
// hold Psi1 and q2 holds Psi2; hdr and q2 move with each simulation's shift.
struct LptMix {
  const SimHeader* hdr;
  const float* q2[3];
  int on, vel, row0, add_step, nk;
};
// Growth-table coefficients of an LptMix for the simulation moved by `by`.
__device__ __forceinline__ float4 mix_coeffs(const LptMix& x, int64_t by) {
  const SimHeader* h = moved(x.hdr, by);
  const int row = x.row0 + (x.add_step ? h->step : 0);
  return (x.vel ? h->vtab : h->tab)[(size_t)row * x.nk];
}
cudaError_t part_drift_deposit(const PartParams& pp, float* sx, float* sy, float* sz, float* vx,
                               float* vy, float* vz, const float* ax, const float* ay,
                               const float* az, const float* dpx, const float* dpy,
                               const float* dpz, float* rho, StepDt dt, int64_t P,
                               cudaStream_t s, Multi m = {}, LptMix mix = {});
// The force mesh: F_x, F_y in F0, F1, or (pairs) the (F_x, F_y) pairs interleaved in F0
// (one float2 per cell; F1 unused); F_z in Fz.
cudaError_t part_gather_kick(const PartParams& pp, const float* sx, const float* sy,
                             const float* sz, float* vx, float* vy, float* vz, float* ax,
                             float* ay, float* az, const float* Ax, const float* Ay,
                             const float* Az, const float* F0, const float* F1, const float* Fz, bool pairs,
                             StepDt dt, int64_t P, cudaStream_t s, Multi m = {}, LptMix mix = {});
// End of step n (hdr->step = n) and start of step n + 1 in one pass: kick with A_n,
// closing half kick and drift of step n + 1 with its drift field dp, CIC deposit into rho
// (zeroed by the caller); acc is not written.  FP32 fields, lattice of Np^3 particles.
cudaError_t part_kick_drift_deposit(const PartParams& pp, float* sx, float* sy, float* sz, float* vx,
                                    float* vy, float* vz, const float* Ax, const float* Ay,
                                    const float* Az, const float* dpx, const float* dpy,
                                    const float* dpz, const float* F0, const float* F1, const float* Fz,
                                    bool pairs, float* rho, const SimHeader* hdr, int64_t P, cudaStream_t s,
                                    Multi m = {});
// The (x, y) pairs of fxy (n cells) into x[0..n) and y[0..n) (either may be null).
cudaError_t split_pairs(const float2* fxy, float* x, float* y, int64_t n, cudaStream_t s);
// Per simulation: lq_used = lq_scale (the scale the fields just written, table
// row step + 1, carry), lq_scale = lq_amax x (growth of the next row over this
// one, lqg) / target for the next pass (unchanged if nothing was written),
// lq_amax = 0.  target: the predicted largest value maps to it (fp16 2^10, a
// factor 64 below the format's largest finite value; bf16 1).
cudaError_t lq_update(SimHeader* hdr, int prec, int nsteps, cudaStream_t s, Multi m = {});
// Initial scales from six FP32 fields of P values (the LPT fields at a_ini, row
// 0): lq_scale = lq_used = max |field| x (growth of row 1 over row 0) / target,
// lq_amax = 0.
cudaError_t lq_init(SimHeader* hdr, const float* const* fields, int64_t P, int prec, cudaStream_t s,
                    Multi m = {});
// FP32 copy of the 16-bit field f (dequantised with lq_used[f]), one simulation.
cudaError_t lq_dequant(const void* src, float* dst, int64_t P, int prec, const SimHeader* hdr, int f,
                       cudaStream_t s);

// *out = the number of non-finite values among nf (<= 9) device arrays of n floats.
cudaError_t count_nonfinite(const float* const* f, int nf, int64_t n, unsigned long long* out, cudaStream_t s);
// *dst (host) = the number of transform CTAs on this device whose TMA tile-load
// wait ran out (one second) since the library was loaded; stream-ordered copy.
cudaError_t tile_load_failures(unsigned* dst, cudaStream_t s);
// N <= 128: the x (r2c, in scale + offset) and y forward transforms of a real N^3 field
// in one pass, one CTA per z-plane (out: interleaved half spectrum, z not transformed).
cudaError_t fft_plane_r2c(int N, const float* in, float2* out, float scale, float offset, const float2* tw,
                          cudaStream_t s, Multi m = {});
// N <= 128: the force's y and x inverse steps in one pass per z-plane: from Phi and
// -i kz Phi (z already inverse-transformed), fx = c2r(yinv(Phi)) with i kfs kx,
// fy = c2r(yinv(i kfs ky Phi)), fz = c2r(yinv(-i kz Phi)).
cudaError_t fft_plane_force(int N, const float2* phi, const float2* phiz, float* fx, float* fy, float* fz,
                            float kfs, const float2* tw, cudaStream_t s, Multi m = {});
// N <= 128: the six LPT field outputs of run_lpt in one pass per (z-plane, field) from
// lc[0..3] after the z inverse: out = {d_x lc0, d_y lc0, lc1, d_x lc2, d_y lc2, lc3}
// (d_x, d_y: i kfs kx, i kfs ky), real N^3 fields.  With zero_dst, the launch also clears
// zero_dst[0, zero_floats) of every simulation (*zeroed = true) when zero_floats is a
// multiple of 4 and zero_dst is 16-byte aligned.
cudaError_t fft_plane_lpt(int N, const float2* const* lc, float* const* out, float kfs, const float2* tw,
                          cudaStream_t s, Multi m = {}, float* zero_dst = nullptr, int64_t zero_floats = 0,
                          bool* zeroed = nullptr);
// N <= 128: the screening source in one pass per z-plane: from the screening field w
// (z already inverse-transformed), y and x inverse, S = delta eps(w) with delta from
// rho, x (r2c) and y forward into s_out (z not transformed).
cudaError_t fft_plane_screen(int N, const float2* w_in, const float* rho, float2* s_out, const ForceParams& fp,
                             const float2* tw, cudaStream_t s, Multi m = {});
// Runs the transform kernels' bounded mbarrier wait on a phase that never completes
// (limit `seconds`, 0 < seconds <= 10, on the per-thread default stream; waits for it); *timed_out = 1 when it gave up.
cudaError_t wait_probe(double seconds, int* timed_out);

// hdr->step += 1 (end of a step)
cudaError_t step_advance(SimHeader* hdr, cudaStream_t s, Multi m = {});
// hdr = v (one simulation), except the seed scales, which keep their device values
cudaError_t set_header(SimHeader* hdr, const SimHeader& v, cudaStream_t s);
// dst[0..n) = src[0..n) (host values) by kernels whose launch parameters carry
// the values: stream-ordered, without a host synchronisation
cudaError_t write_words(int64_t* dst, const int64_t* src, int64_t n, cudaStream_t s);
// n floats at p set to zero in every simulation
cudaError_t zero_f32(float* p, int64_t n, cudaStream_t s, Multi m = {});
cudaError_t part_snapshot(const PartParams& pp, const float* sx, const float* sy, const float* sz,
                          const float* vx, const float* vy, const float* vz, const float* lx,
                          const float* ly, const float* lz, float vscale, float* pos, float* vel,
                          int64_t P, cudaStream_t s, LptMix mix = {});
// out_d = c1 Psi1_d + c2 Psi2_d (acc = 0) or e1 Psi1_d + e2 Psi2_d (acc = 1) for
// one simulation, coefficients as LptMix (psi1: the Psi1 fields)
cudaError_t lpt_mix(int64_t P, const float* const* psi1, const LptMix& mix, int acc, float* const* out,
                    cudaStream_t s);
cudaError_t pos_deposit(int Nm, float cellscale, const float* pos, int64_t n, float* rho,
                        cudaStream_t s);
// acc_stride > 0: simulation b accumulates into acc + b acc_stride (acc not
// moved); 0: into acc moved by its shift.
cudaError_t pk_bin(int N, const float2* dk, int nbins, double* acc, double norm,
                   cudaStream_t s, Multi m = {}, int64_t acc_stride = 0);

// ------------------------------------------------------------------ initial conditions
// The initial-condition launchers run over m's simulations; where a value
// differs between simulations (seed, spectrum, seed scales) it is read from
// each simulation's header when hdr is given.
cudaError_t ic_noise(int N, uint64_t seed, float* out, cudaStream_t s, Multi m = {},
                     const SimHeader* hdr = nullptr);
// delta(k) = G(k) sqrt(P(k) N^3/L^3); phi1 = delta/k^2 (k = 0 -> 0), in place on c.
// work: device scratch of 3 (N/2)^2 + 1 doubles per simulation (the factor per |n|^2).
cudaError_t ic_phi1(int N, float2* c, float kf, const EHDev& eh, double* work, cudaStream_t s,
                    Multi m = {}, const SimHeader* hdr = nullptr);
// out = -k_i k_j / N^3 * phi1 with the Nyquist rule for i != j.
cudaError_t ic_hessian(int N, const float2* phi1, float2* out, int i, int j, float kf,
                       cudaStream_t s, Multi m = {});
cudaError_t ic_source(int64_t n, const float* hxx, const float* hyy, const float* hzz,
                      const float* hxy, const float* hxz, const float* hyz, float* src,
                      cudaStream_t s, Multi m = {});
// phi2 = -src(k)/k^2 in place.
cudaError_t ic_phi2(int N, float2* c, float kf, cudaStream_t s, Multi m = {});
cudaError_t ic_particles(int64_t P, const float* px, const float* py, const float* pz, float* sx,
                         float* sy, float* sz, float* vx, float* vy, float* vz,
                         cudaStream_t s, Multi m = {}, LptMix mix = {});
// pack a dense [N][N][N/2+1] half spectrum into / out of the padded layout
cudaError_t half_pack(int N, const float2* dense, float2* padded, cudaStream_t s);
cudaError_t half_unpack(int N, const float2* padded, float2* dense, cudaStream_t s);
// reduced-precision seeds: the largest |component| of field f (into absmax),
// then hdr->seed_scale[f] = absmax / hdr->seed_target (1 if absmax = 0), then
// the 16-bit copy of the field divided by that scale
cudaError_t seed_absmax(int N, const float2* src, float* out_absmax, cudaStream_t s, Multi m = {});
cudaError_t seed_scale_set(SimHeader* hdr, const float* absmax, int f, cudaStream_t s, Multi m = {});
cudaError_t seed_quantise(int N, const float2* src, void* dst, int prec, const SimHeader* hdr, int f,
                          cudaStream_t s, Multi m = {});

// Caps the persistent grid of the FFT-pass kernels launched by the calling
// thread (0 = no cap: resident CTAs x SMs).
void set_grid_cap(int max_ctas);
// Particle kernels the calling thread's step launches use: deposit_box /
// gather_box > 0 selects the shared-memory box kernels with that many cells
// (rounded down to a multiple of 4; at most 16384 / 8192), 0 the direct ones.
void set_particle_plan(int deposit_box, int gather_box);

// Loads the allocation-free P(k) scratch on the current device (once per
// device; later calls return at once).  COLA_OK or COLA_ECUDA.
int pk_noalloc_reserve();

// Sets the message cola_last_error(NULL) returns (calling thread).
void set_context_free_error(const std::string& msg);

}  // namespace cola
