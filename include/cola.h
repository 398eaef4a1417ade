/*
 * cola.h — C ABI of the GB300 (sm_103a) COLA particle-mesh library.
 *
 * The method is COLA (COmoving Lagrangian Acceleration) as used by Koda et al. 2015,
 * "Fast and accurate mock catalogue generation for low-mass galaxies" (arXiv:1507.05329):
 * particles move relative to their 2LPT trajectories (§2.1), the residual is integrated with the
 * kick and drift of §2.2 eqs. (cola-kick) and (cola-drift) on the time grid a_i = i/n_step
 * (eq. drift-a), and the force is a particle-mesh (PM) force on a uniform mesh (§2.3).
 *
 * Conventions used by every call
 *   - Units: H0 = 1; lengths in PM mesh cells (L/N); time variable a; canonical velocity
 *     v = a^2 dx/dt (§2.2, eq. motion).
 *   - Particles: n = np^3, particle id = (ix*np + iy)*np + iz on the Lagrangian lattice q.
 *     Every particle array is structure-of-arrays float32 [3][n] (x block, then y, then z),
 *     a DEVICE pointer owned by the caller, 16-byte aligned.
 *       s    : total displacement x - q (mesh cells);
 *       v    : residual canonical velocity v_res = v - a^2 dx_2LPT/dt (§2.1);
 *       psi1 : first-order 2LPT displacement Psi1 (mesh cells);
 *       psi2 : second-order 2LPT displacement Psi2 (mesh cells), x_2LPT = q + D1 Psi1 + D2 Psi2.
 *   - Mesh arrays are [N][N][N] C order (z fastest).  Half spectra are [N][N][N/2+1] complex
 *     (interleaved float re, im), the k_z >= 0 half as in §3.3.
 *   - Calls are asynchronous on the context's CUDA stream unless stated; the caller must keep
 *     buffers alive until the stream has finished with them.
 *   - Errors: every int-returning call returns a cola_status.  Argument errors are found on the
 *     host before anything is launched.  Device-side conditions (fixed-point overflow,
 *     non-finite particle state) set a sticky flag that cola_sync() reports.
 *   - One context per device and stream; a context is not thread safe.  Besides the contexts the
 *     library keeps only process-wide records of which kernels already had their shared-memory
 *     limit raised on which device, and the static scratch array of the allocation-free entry
 *     point (cola_power_spectrum_noalloc, at the end of this header).
 */
#ifndef COLA_H
#define COLA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    COLA_OK = 0,
    COLA_ERR_INVALID = 1,     /* bad argument or size (reported on the host, nothing launched) */
    COLA_ERR_OOM = 2,         /* device allocation failed */
    COLA_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    COLA_ERR_OVERFLOW = 4,    /* a fixed-point mesh cell overflowed (more than 2^22 particles) */
    COLA_ERR_NONFINITE = 5,   /* a particle position or velocity became NaN or infinite */
    COLA_ERR_INTERNAL = 6     /* a bounded device loop hit its limit (never expected; result invalid) */
} cola_status;

/* Parameters of one realisation (§1 cosmology, §2.2 time stepping, §2.3 box and mesh).
 * Flat LCDM with Omega_Lambda = 1 - omega_m; linear P(k) = A k^n_s T_BBKS(k)^2 normalised to
 * sigma8 at a = 1.  Requirements (checked by cola_create): np >= 2 and nmesh >= 4 even, both with
 * no prime factor above 5, nmesh <= 4096, np <= 2048, (nmesh * 2^20) % np == 0, nstep >= 1. */
typedef struct {
    double omega_m;       /* matter density today */
    double h;             /* H0 / (100 km/s/Mpc), enters only Gamma = omega_m h of BBKS */
    double n_s;           /* spectral index */
    double sigma8;        /* rms of the linear density in 8 Mpc/h spheres at a = 1 */
    double box;           /* box side L in Mpc/h */
    int np;               /* particles per side */
    int nmesh;            /* PM mesh cells per side */
    int nstep;            /* n_step of eq. (drift-a); a_i = i / nstep */
    double nlpt;          /* n_LPT of eqs. (ansatz-drift), (ansatz-kick); the paper uses -2.5 */
    int ic_mode;          /* 0: eq. (initial_time), v_res = 0 at a_{1/2};
                             1: Appendix A eq. (initial_time_original), v_res = 0 at a_1 */
    int drift_ansatz;     /* 0: eq. (ansatz-drift); 1: v_res constant during a drift (§2.1) */
    unsigned long long seed;  /* seed of the white noise drawn when a call gets white_noise == NULL */
} cola_params;

typedef struct cola_ctx cola_ctx;

/* Create a context on the current CUDA device for the given stream (cudaStream_t, NULL =
 * legacy default stream).  Validates the parameters, computes every FP64 time coefficient on
 * the host and allocates the device meshes (about 20 N^3 bytes plus the P(k) and FFT tables).
 * The context owns those allocations.  Returns COLA_ERR_INVALID or COLA_ERR_OOM on failure and
 * leaves *out NULL. */
int cola_create(const cola_params* params, void* stream, cola_ctx** out);

/* Free a context and its device memory (synchronises its stream first).  NULL is a no-op. */
void cola_destroy(cola_ctx* ctx);

/* Wait for the context's stream, then report and clear the sticky device error flag. */
int cola_sync(cola_ctx* ctx);

/* Human-readable text of a cola_status (static storage). */
const char* cola_strerror(int status);

/* FP64 scalars of COLA step i (1 <= i <= nstep), host only, no context needed.
 * out[0..11] = a_i, a_lo, a_hi, force_scale = (3/2) Om / a_i, c1, c2 (2LPT acceleration
 * coefficients, F_2LPT = c1 Psi1 + c2 Psi2), kick factor of eq. (cola-kick) from a_lo to a_hi,
 * drift factor of eq. (cola-drift) from a_i to a_{i+1}, dD1, dD2 (growth increments over the
 * drift), D1(a_i), D2(a_i).  The last step has drift = dD1 = dD2 = 0.  i = 0 returns the
 * initial-condition scalars: out[0] = a_1, out[10] = D1(a_1), out[11] = D2(a_1), and out[8],
 * out[9] = a^2 dD1/dt, a^2 dD2/dt at a = 1 (the 2LPT velocity factors of the final output).
 * Returns COLA_ERR_INVALID for a bad index or nout < 12. */
int cola_step_scalars(const cola_params* params, int i, double* out, int nout);

/* Linear matter power spectrum at a = 1 of the parameters' cosmology (§1 cosmology; P(k) = A k^n_s
 * T_BBKS(k)^2 with Gamma = omega_m h, A from sigma8), host only, no context needed.  k: nk
 * wavenumbers >= 0 in h/Mpc; power (may be NULL) receives P(k) in (Mpc/h)^3, transfer (may be
 * NULL) T_BBKS(k).  The white-noise amplitudes of cola_ic_2lpt are sqrt(P(k)/V_cell) of these values.
 * Returns COLA_ERR_INVALID for invalid parameters or a negative or non-finite k. */
int cola_linear_power(const cola_params* params, const double* k, int nk, double* power, double* transfer);

/* Seeded white noise (§2.3: the initial conditions are Gaussian random modes drawn from a seed; the
 * paper does not name its generator).  One unit Gaussian per lattice site, from the counter-based
 * generator Philox-4x32-10 (Salmon, Moraes, Dror & Shaw 2011) and the Box-Muller transform: site i
 * (particle id) takes counter j = i/4 = (j mod 2^32, j div 2^32, 0, 0) under key (seed mod 2^32,
 * seed div 2^32); output words (x0, x1) give sites 4j, 4j+1 and (x2, x3) sites 4j+2, 4j+3 as
 * (r cos 2 pi u2, r sin 2 pi u2), r = sqrt(-2 ln u1), u1 = ((a >> 8) + 1) 2^-24, u2 = (b >> 8) 2^-24,
 * evaluated in FP32.  The field is a pure function of (seed, i).
 * cola_white_noise writes params->seed's field to out (device float32 [np^3]) on `stream`
 * (cudaStream_t); only np and seed are used (params must still be valid).
 * cola_philox_words writes the raw words of counters first .. first+count-1 under `seed` to out
 * (device uint32 [count][4]).  Both are asynchronous; COLA_ERR_INVALID for bad arguments. */
int cola_white_noise(const cola_params* params, float* out, void* stream);
int cola_philox_words(unsigned long long seed, long long first, long long count, unsigned* out, void* stream);

/* S0 — 2LPT initial conditions (§2.1 growing mode; §2.3 2LPTic-style Gaussian modes).
 * white_noise: device float32 [n], unit Gaussian, one value per lattice site (input), or NULL to
 * draw the field of params.seed (cola_white_noise) inside the call.
 * Writes psi1, psi2, s = D1(a_1) Psi1 + D2(a_1) Psi2 and v = 0 (eq. initial_time). */
int cola_ic_2lpt(cola_ctx* ctx, const float* white_noise, float* s, float* v,
                 float* psi1, float* psi2);

/* S1 alone — CIC deposit of the particles at displacement s into rho (device uint64 [N^3]),
 * which is overwritten.  Fixed point: mesh coordinate G = (q*R + rint(s*2^20)) mod N*2^20,
 * R = (N/np)*2^20; cell G>>20; 14-bit weights; every particle adds exactly 2^42 (§2.3, §3.3
 * CIC; the fixed-point form is this library's, deterministic and exact). */
int cola_deposit(cola_ctx* ctx, const float* s, unsigned long long* rho);

/* S1+S2 — deposit, then the forward 3D FFT of the density contrast
 * delta = rho N^3 / (n 2^42) - 1.  delta_k: device float32 [N][N][N/2+1][2] (unnormalised DFT,
 * X(k) = sum_x delta(x) exp(-i k.x)). */
int cola_density_spectrum(cola_ctx* ctx, const float* s, float* delta_k);

/* S2 and S3 on a given fixed-point density mesh, in place of the deposit (for checks of the FFT and
 * Poisson passes on a known density, e.g. a sum of plane waves, at any mesh size).  rho: device
 * uint64 [N][N][N], read only, interpreted as the deposit's output (delta = rho N^3 / (n 2^42) - 1,
 * n = np^3; no total-mass check).  The passes are the context's schedule, as in cola_pm_force.
 * cola_density_spectrum_of_mesh writes the forward spectrum as cola_density_spectrum does.
 * cola_pm_force_of_mesh writes F_j at the m mesh cells cells[i] = (ix N + iy) N + iz (device int64
 * [m], each in [0, N^3)) to force (device float32 [3][m]), a as in cola_pm_force. */
int cola_density_spectrum_of_mesh(cola_ctx* ctx, const unsigned long long* rho, float* delta_k);
int cola_pm_force_of_mesh(cola_ctx* ctx, const unsigned long long* rho, double a, const long long* cells, long long m,
                          float* force);

/* S1-S3 (+ interpolation) — PM force at the particles (§2.2 Poisson equation and eq. motion):
 * F = -grad phi with nabla^2 phi = (3/2) Om a^-1 delta, Green function -1/k^2, 4-point
 * central-difference gradient kernel, CIC interpolation with the deposit's weights.
 * force: device float32 [3][n] in mesh cells per unit time squared. */
int cola_pm_force(cola_ctx* ctx, const float* s, double a, float* force);

/* S1-S5 — COLA step i (1 <= i <= nstep): force at a_i, kick v_res from a_{i-1/2} to a_{i+1/2}
 * (eq. cola-kick, F_res = F - F_2LPT), drift s from a_i to a_{i+1} (eq. cola-drift) adding the
 * 2LPT growth increments.  The last step kicks to a_nstep and does not drift.  In place on s, v. */
int cola_step(cola_ctx* ctx, int i, float* s, float* v, const float* psi1, const float* psi2);

/* A whole realisation: cola_ic_2lpt (white_noise NULL: the field of params.seed), then steps
 * 1..nstep, then (if pk != NULL) the power spectrum of the final positions into pk (device double
 * [3][nbins]). */
int cola_run(cola_ctx* ctx, const float* white_noise, float* s, float* v, float* psi1,
             float* psi2, double* pk, int nbins);

/* The number of kernels one cola_run call with these arguments launches (written to *kernels): the
 * call is captured into a CUDA graph on a private stream, its kernel nodes are counted and the
 * graph is destroyed unexecuted, so no buffer is touched.  Memset and copy nodes are not kernels.
 * Call it after one plain cola_run with the same nbins (the capture cannot upload new P(k) bin
 * edges or set first-use kernel attributes).  Profiling counters are left as they were.
 * COLA_ERR_INVALID for a NULL kernels or an nbins different from the last P(k) call's. */
int cola_run_kernel_count(cola_ctx* ctx, const float* white_noise, float* s, float* v, float* psi1,
                          float* psi2, double* pk, int nbins, long long* kernels);

/* S6 — matter power spectrum of the particles at displacement s (§3.3): CIC deposit, FFT, the
 * modes {kz>0} U {kz=0,ky>0} U {kz=0,ky=0,kx>0}, nbins log-spaced bins between 2 pi/L and
 * pi N/L decided on the integer |m|^2, P = V |delta_k|^2 / N^6 averaged per bin.
 * pk: device double [3][nbins] = mean |k| (h/Mpc), P (Mpc/h)^3, mode count.  1 <= nbins <= 128.
 * The reduction order is fixed, so the result is bit-reproducible.  A call with a different nbins
 * than the previous one synchronises the stream once to upload the new bin edges. */
int cola_power_spectrum(cola_ctx* ctx, const float* s, double* pk, int nbins);

/* ---- Execution schedule and autotuner (not part of the method: choices among kernels that
 * compute the same result; every schedule gives a bit-identical density mesh and the same forces
 * to FP32 rounding order) ---------------------------------------------------------------------
 * Bits of a schedule:
 *   COLA_SCHED_BINNED_DEPOSIT : particles binned into mesh tiles each step, tile-wise deposit in
 *                               shared memory (else one global 64-bit atomic per CIC corner).
 *                               Available when the tile geometry fits (cola_create decides).
 *   COLA_SCHED_TILE_GATHER    : tile-wise gather from shared memory (requires the binned deposit
 *                               and tiles of at least 4 cells along z).
 *   COLA_SCHED_PIPELINED_FFT  : persistent cp.async-pipelined strided FFT passes (else one CTA per
 *                               tile of pencils).
 *   COLA_SCHED_PIPE_EPT8      : the pipelined passes give each thread 8 complex values per stage
 *                               instead of 16 (twice the threads on the same tile); requires
 *                               COLA_SCHED_PIPELINED_FFT.
 *   COLA_SCHED_PIPELINED_GATHER: the tile gather runs on persistent CTAs that copy the next tile's
 *                               forces while interpolating the current one (requires
 *                               COLA_SCHED_TILE_GATHER).
 *   COLA_SCHED_GREEN_EPT8     : the fused x + Green + inverse-x pass gives each thread 8 complex values
 *                               per stage instead of 16 (narrower tiles, fewer registers per thread).
 *   COLA_SCHED_C2R_EPT8       : the same for the contiguous-axis C2R passes of the three forces.
 *   COLA_SCHED_ROWS_PIPE      : the C2R passes run on persistent CTAs that copy the next tile's rows
 *                               (cp.async) while transforming the current one.
 *   bits COLA_SCHED_BUDGET_SHIFT..+1 : shared-memory budget per CTA of the pipelined passes,
 *                               0: 160 KB, 1: 96 KB, 2: 64 KB (sets their tile width); must be 0
 *                               without COLA_SCHED_PIPELINED_FFT.
 *   COLA_SCHED_R2C_EPT8       : 8 complex values per thread per stage in the contiguous-axis R2C
 *                               pass of the density.
 *   COLA_SCHED_WIDE_TILES     : tiles of 8 pencils (one CTA of up to 768 threads per SM) in the
 *                               16-element Green pass and the one-CTA-per-tile strided passes where
 *                               the default tile is narrower (meshes of 769 to 1536 cells), so that
 *                               every row segment moved is 64 bytes; on by default.
 *   COLA_SCHED_PIPE_INPLACE   : the pipelined passes keep two tile buffers (staging and one work buffer
 *                               that the middle stages overwrite) in up to 210 KB, which holds tiles of
 *                               8 pencils of 1536; requires COLA_SCHED_PIPELINED_FFT, budget bits 0 and
 *                               no COLA_SCHED_PIPE_EPT8.
 * cola_create picks a schedule from the sizes (in-place pipelined passes for meshes of 769 to 1536
 * cells, the binned deposit and tile gather where the tiles are dense enough); cola_get_schedule reads
 * it and cola_set_schedule replaces it (COLA_ERR_INVALID for an unavailable or malformed schedule).
 * cola_autotune times `reps` PM force evaluations (deposit, FFTs, Poisson + gradient, gather) at
 * displacements s (device float32 [3][np^3]; an evolved state is representative, a lattice is not)
 * in a coordinate search from the current schedule: the deposit/gather choice, then the strided
 * passes (pipelining, elements per thread, budget or in-place tiles), then the Green pass, then the tile width, then
 * the C2R passes (elements per thread, pipelining), then the R2C pass, each
 * with the others fixed.  It keeps the fastest, writes it to *best (may be NULL), and writes the
 * schedules it timed and their milliseconds per evaluation, in timing order, to
 * scheds[0..max_candidates) and ms[0..max_candidates) (either may be NULL).  Returns the number of
 * schedules timed, or minus a cola_status.  It synchronises the stream and allocates a temporary
 * force array: call it outside graph capture. */
#define COLA_SCHED_BINNED_DEPOSIT 1
#define COLA_SCHED_TILE_GATHER 2
#define COLA_SCHED_PIPELINED_FFT 4
#define COLA_SCHED_PIPE_EPT8 8
#define COLA_SCHED_PIPELINED_GATHER 16
#define COLA_SCHED_GREEN_EPT8 32
#define COLA_SCHED_C2R_EPT8 64
#define COLA_SCHED_ROWS_PIPE 128
#define COLA_SCHED_BUDGET_SHIFT 8
#define COLA_SCHED_R2C_EPT8 1024
#define COLA_SCHED_WIDE_TILES 2048
#define COLA_SCHED_PIPE_INPLACE 4096
int cola_get_schedule(cola_ctx* ctx, int* schedule);
int cola_set_schedule(cola_ctx* ctx, int schedule);
int cola_autotune(cola_ctx* ctx, const float* s, int reps, int* best, int* scheds, double* ms, int max_candidates);

/* ---- Reverse mode (not in the paper: the transpose of its forward model) ------------------
 * The forward being differentiated is cola_run's: 2LPT (§2.1, §2.3), then n_step COLA steps
 * (§2.2, eqs. cola-kick / cola-drift) with the PM force of §2.2/§2.3.  The adjoint treats the CIC
 * weights as the continuous piecewise-linear functions of position that the 14-bit fixed-point
 * weights approximate (their exact derivative is zero almost everywhere); the derivative of a
 * weight is +-1 times the other two axes' weights, taken in the cell the forward's fixed-point
 * coordinate selects.  Linear k-space maps are transposed as y -> irfft(conj(M) rfft(y)), valid for
 * the Hermitian multipliers used here.  Float atomics sum the adjoint deposit, so adjoints agree
 * with the exact transpose to FP32 rounding but are not bit-reproducible. */

/* cola_run without P(k), storing the positions at which each step evaluates its force.
 *   ckpt : device float32 [nstep][3][np^3], 16-byte aligned (12 nstep np^3 bytes, caller-owned);
 *          ckpt[i-1] receives s at a_i before step i.
 * Other arguments and results as cola_run.  Asynchronous on the context's stream. */
int cola_run_checkpointed(cola_ctx* ctx, const float* white_noise, float* s, float* v, float* psi1, float* psi2,
                          float* ckpt);

/* Vector-Jacobian product of cola_run_checkpointed with respect to the white noise.
 *   white_noise : the same device float32 [np^3] input as the forward (the 2LPT Hessians are
 *                 recomputed from it), or NULL if the forward drew the field of params.seed.
 *   ckpt        : the forward's checkpoints; the PM force of each step is recomputed from them.
 *   lam_s       : cotangent of the final s, device float32 [3][np^3] (required).
 *   lam_v, lam_psi1, lam_psi2 : cotangents of the final v_res, Psi1 and Psi2 (device float32
 *                 [3][np^3]); NULL means zero.
 *   lam_wn      : out, dL/d(white noise), device float32 [np^3].
 * Inputs are not modified.  The first call allocates the adjoint work space (60 np^3 bytes plus
 * three complex meshes, 24 nmesh^2 (nmesh/2+1) bytes); it lives until cola_destroy.  The 2LPT part
 * reuses the context's mesh arena, so the context's meshes are undefined afterwards.
 * All pointers 16-byte aligned; COLA_ERR_INVALID for a NULL or misaligned required pointer. */
int cola_adjoint(cola_ctx* ctx, const float* white_noise, const float* ckpt, const float* lam_s, const float* lam_v,
                 const float* lam_psi1, const float* lam_psi2, float* lam_wn);

/* Density contrast of the particles on an ngrid^3 CIC grid covering the box (the differentiable
 * loss's field): grid coordinate y = (q + s) ngrid / nmesh with continuous CIC weights rounded to
 * multiples of 2^-32 and summed exactly in 64-bit integers (bit-reproducible),
 * delta = ngrid^3 rho / np^3 - 1.
 *   s     : device float32 [3][np^3] displacements (mesh cells).
 *   delta : out, device float32 [ngrid][ngrid][ngrid] (row-major, z fastest).
 * 1 <= ngrid <= nmesh.  Uses the context's density mesh as scratch. */
int cola_grid_density(cola_ctx* ctx, const float* s, int ngrid, float* delta);

/* Transpose of cola_grid_density at s: lam_s = d(sum_g lam_delta_g delta_g)/ds, with the
 * continuous-weight derivative (one-sided at cell faces).  lam_s is overwritten. */
int cola_grid_density_adjoint(cola_ctx* ctx, const float* s, int ngrid, const float* lam_delta, float* lam_s);

/* ---- Batched realisations in one CUDA graph (the paper's many mock catalogues, §3) ----------
 * A batch owns one context per realisation and `nstreams` non-blocking lanes.  Realisations are
 * assigned to lanes longest-first (cost ~ particles + mesh cells x log N) and run back to back on
 * their lane; lanes run concurrently.  cola_batch_run enqueues cola_run (2LPT + n_step PM steps +
 * P(k) in nbins bins) of every realisation, forked from and joined back into `stream`:
 *   use_graph = 0 : plain launches;
 *   use_graph = 1 : the first call runs once eagerly (warm-up, then synchronises), captures the
 *                   whole launch sequence into a CUDA graph and launches it; later calls only
 *                   launch the graph (one host call for all realisations).
 * io[i] holds realisation i's device buffers (as for cola_run: white noise [np^3] or NULL for the
 * field of params[i].seed, s, v, psi1, psi2 [3][np^3] float32, pk double [3][nbins]); all 16-byte
 * aligned, caller-owned, fixed for the
 * batch's lifetime (the graph records the pointers).  params[i] is realisation i's parameters
 * (sizes may differ).  Contexts hold their own meshes: the batch needs the sum of the members'
 * context memory.  All calls are asynchronous on `stream` except create, sync and tune.
 * cola_batch_sync waits for `stream` and returns the first member's error flag (as cola_sync).
 * cola_batch_tune runs cola_autotune once per distinct (np, nmesh) on that member's current s
 * (run the batch first, so positions are evolved), gives the winner to every member of that
 * shape and drops the captured graph (the next graph run captures again).
 * cola_batch_info reports member i's lane and schedule and the captured graph's node count
 * (0 before capture); any output pointer may be NULL. */
typedef struct cola_batch cola_batch;
typedef struct {
  const float* white_noise;
  float* s;
  float* v;
  float* psi1;
  float* psi2;
  double* pk;
} cola_batch_io;
int cola_batch_create(const cola_params* params, const cola_batch_io* io, int count, int nbins, int nstreams,
                      void* stream, cola_batch** out);
int cola_batch_run(cola_batch* batch, int use_graph);
int cola_batch_sync(cola_batch* batch);
int cola_batch_tune(cola_batch* batch, int reps);
int cola_batch_info(cola_batch* batch, int i, int* lane, int* schedule, size_t* graph_nodes);
void cola_batch_destroy(cola_batch* batch);

/* P(k) as cola_power_spectrum, with options:
 *   COLA_PK_CIC_CORRECT : correct each mode for the CIC smoothing and aliasing and subtract shot
 *                         noise (the paper corrects with Jing 2005, §3.3; this is that correction for
 *                         a locally flat spectrum): P = P_raw / C2(k) - V/n with
 *                         C2 = prod_i (1 - (2/3) sin^2(pi m_i / N)), the CIC window squared summed
 *                         over all aliases.  P can then be negative where the signal is below shot noise.
 * Other flag bits give COLA_ERR_INVALID. */
#define COLA_PK_CIC_CORRECT 1
int cola_power_spectrum_ex(cola_ctx* ctx, const float* s, double* pk, int nbins, int flags);

/* Snapshot between two force times (§2.2: the kick/drift equations interpolate the particles to
 * output redshifts between steps).  Input: the state right after cola_step(i): s (at a_{i+1}, or at
 * a_{n_step} = 1 after the last step), v = v_res at a_{i+1/2}, psi1, psi2.  Output at
 * a_i <= a_snap <= a_{i+1} (a_snap = 1 after the last step):
 *   s_out = s_i + drift(a_i -> a_snap) v_res + (D1(a_snap) - D1(a_i)) Psi1 + (D2(a_snap) - D2(a_i)) Psi2,
 *   v_out = v_res + a^2 dD1/dt Psi1 + a^2 dD2/dt Psi2 at a_snap (canonical velocity; may be NULL),
 * the drift integral of eq. (cola-drift) with the step's a_{i+1/2} and ansatz, evaluated up to
 * a_snap; the residual velocity between kicks is v_res(a_{i+1/2}).  COLA_ERR_INVALID if a_snap is
 * outside the step's interval.  s_out must not alias s. */
int cola_snapshot(cola_ctx* ctx, int i, double a_snap, const float* s, const float* v, const float* psi1,
                  const float* psi2, float* s_out, float* v_out);

/* cola_run that also writes snapshots at nsnap increasing scale factors a_snap[k] in [a_1, 1]
 * (the paper writes its density fields at z = 0.73, 0.6, 0.44 and 0):
 *   s_snap : device float32 [nsnap][3][np^3] (required), v_snap : same shape or NULL,
 *   pk_snap: device double [nsnap][3][nbins] or NULL, computed with cola_power_spectrum_ex(pk_flags).
 * s, v, psi1, psi2 end at a = 1 as after cola_run. */
int cola_run_snapshots(cola_ctx* ctx, const float* white_noise, float* s, float* v, float* psi1, float* psi2,
                       const double* a_snap, int nsnap, float* s_snap, float* v_snap, double* pk_snap, int nbins,
                       int pk_flags);

/* Friends-of-friends haloes (§2.3, run on the fly by the paper; §3.2: linking length b = 0.2 times
 * the mean particle separation, 0.37 for 2LPT).  Links are decided exactly on the deposit's
 * fixed-point coordinates G (20 fractional bits per mesh cell): friends when the periodic
 * minimum-image distance satisfies d^2 <= l^2 in integers, l = rint(b (nmesh/np) 2^20).  Groups are
 * the connected components (friends of friends), labelled by their smallest particle id, so the
 * output is unique and bit-reproducible.
 *   s          : device float32 [3][np^3] displacements (mesh cells).
 *   b          : linking length in mean particle separations, 0 < b, l <= 2^30.
 *   n_min      : smallest halo (>= 1).
 *   label, size: out, device int32 [np^3]: group label and member count of each particle.
 *   halo_label, halo_size : out, device int32 [capacity] or NULL; halo_pos : out, device double
 *                [3][capacity] or NULL, the periodic centre of mass in mesh cells in [0, nmesh)
 *                (G_root + exact integer sum of minimum-image offsets / size, in FP64).  Haloes
 *                (groups of >= n_min members) are listed in increasing label order; only the first
 *                `capacity` are written.
 *   nhalo      : out, device int32: the number of haloes (may exceed capacity).
 * Work space (about 52 B per particle plus the search cells) is allocated on first use and kept
 * until cola_destroy; requires np^3 < 2^31.  Asynchronous on the context's stream. */
int cola_fof(cola_ctx* ctx, const float* s, double b, int n_min, int* label, int* size, int* halo_label,
             int* halo_size, double* halo_pos, int capacity, int* nhalo);

/* Stage timing and launch counting (not part of the method: measurement support).
 * Stages: 0 deposit, 1 forward z (R2C), 2 forward y, 3 x + Green + gradient + inverse x,
 * 4 inverse y, 5 inverse z (C2R), 6 gather + kick + drift (or force gather), 7 x passes outside
 * the fused stage 3 (P(k), density spectrum, 2LPT), 8 2LPT element-wise kernels, 9 P(k) binning,
 * 10 mesh clearing (memset, direct deposit only), 11 spatial binning of the particles (count, scan,
 * scatter), 12 reverse-mode and loss-grid kernels (adjoint element-wise maps, adjoint scatter and
 * gather, loss-grid deposit), 13 friends-of-friends, 14 the 2LPT lattice transforms (forward and
 * adjoint).  Stages 1, 2, 4, 5 and 7 also count the adjoint's mesh transforms.
 * cola_profile_enable(ctx, 1) resets the totals and brackets every later launch with CUDA events
 * on the context's stream; 0 stops timing (launches are always counted).  cola_profile_read
 * synchronises the stream and writes per-stage total milliseconds and launch counts for the first
 * nstages stages (either pointer may be NULL).  Returns the number of stages (15), or minus a
 * cola_status on failure. */
#define COLA_NUM_STAGES 15
int cola_profile_enable(cola_ctx* ctx, int on);
int cola_profile_read(cola_ctx* ctx, double* ms, long long* launches, int nstages);

/* Allocation-free power spectrum (this entry point has no counterpart in the paper).
 *
 * For callers that cannot allocate device memory: code that runs inside a CUDA-graph capture and
 * must replay without a memory pool, plug-ins whose host framework owns the whole device heap,
 * and real-time loops that forbid allocator calls (cudaMalloc also synchronises the device).
 * It computes what cola_power_spectrum computes, without a context and without any allocation:
 * its scratch (density mesh, spectrum, partial sums, twiddles, bin edges) is one static device
 * array of COLA_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until exit.
 *   params : only np, nmesh and box are used; nmesh <= COLA_NOALLOC_MAX_MESH, np <= COLA_NOALLOC_MAX_NP
 *            (fewer than 2^22 particles: the fixed-point mesh cannot overflow), same size rules as
 *            cola_create.  Larger sizes return COLA_ERR_INVALID before anything is launched.
 *   s      : device float32 [3][np^3] displacements (mesh cells), 16-byte aligned.
 *   pk     : device double [3][nbins], as for cola_power_spectrum; 1 <= nbins <= 128.
 *   stream : cudaStream_t to enqueue on (NULL = legacy default stream).
 * Asynchronous: results are ready when the stream reaches them.  The call runs on the current
 * device, whose copy of the array it uses: s, pk and the stream must belong to that device.  The
 * first call on each device resolves the array's device address (cudaGetSymbolAddress), and each
 * kernel's first launch on a device raises its shared-memory limit (host-side attribute calls, no
 * allocation); make that first call before any stream capture.  Every call shares the array:
 * calls that overlap on the GPU (other streams or threads) race and give wrong results. */
#define COLA_NOALLOC_MAX_MESH 64
#define COLA_NOALLOC_MAX_NP 128
#define COLA_NOALLOC_SCRATCH_BYTES 3670016
int cola_power_spectrum_noalloc(const cola_params* params, const float* s, double* pk, int nbins,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* COLA_H */
