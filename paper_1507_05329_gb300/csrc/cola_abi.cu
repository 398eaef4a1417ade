// C ABI of the COLA particle-mesh library (declared in include/cola.h).
//
// One realisation per context.  The context owns the PM meshes and tables; the caller owns every
// particle array.  Each call enqueues kernels on the context's stream:
//   S0 cola_ic_2lpt ........ white noise -> delta_L -> Psi1, Psi2 (§2.1, §2.3)
//   S1 deposit ............. CIC, 64-bit fixed point (§2.3, §3.3)
//   S2 forward FFT ......... z (R2C, fused fixed-point -> delta), y
//   S3 Poisson + gradient .. x forward fused with -1/k^2, the 4-point gradient and inverse x (F_x;
//                            F_y and F_z from one shared transform);
//                            then inverse y and C2R z for each component (§2.2 Poisson equation)
//   S4+S5 gather/kick/drift  CIC interpolation + eqs. (cola-kick), (cola-drift) (§2.1, §2.2)
//   S6 power spectrum ...... §3.3
#include "cola_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

using namespace cola;

namespace {

#define COLA_TRY(expr)              \
  do {                              \
    const int _st = (expr);         \
    if (_st != COLA_OK) return _st; \
  } while (0)

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return COLA_OK;
  std::fprintf(stderr, "cola: %s: %s\n", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? COLA_ERR_OOM : COLA_ERR_CUDA;
}

bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

int validate(const cola_params* p) {
  if (!p) return COLA_ERR_INVALID;
  if (p->np < 2 || p->np > 2048 || p->np % 2 || !smooth235(p->np)) return COLA_ERR_INVALID;
  if (p->nmesh < 4 || p->nmesh > 4096 || p->nmesh % 2 || !smooth235(p->nmesh)) return COLA_ERR_INVALID;
  if ((((long long)p->nmesh) << 20) % p->np) return COLA_ERR_INVALID;
  if (p->nstep < 1 || p->nstep > 10000) return COLA_ERR_INVALID;
  if (!(p->omega_m > 0.0 && p->omega_m <= 1.0) || !(p->box > 0.0) || !(p->h > 0.0) || !(p->sigma8 >= 0.0))
    return COLA_ERR_INVALID;
  if (!(p->nlpt != 0.0) || !std::isfinite(p->nlpt) || !std::isfinite(p->n_s)) return COLA_ERR_INVALID;
  if (p->ic_mode < 0 || p->ic_mode > 1 || p->drift_ansatz < 0 || p->drift_ansatz > 1) return COLA_ERR_INVALID;
  return COLA_OK;
}

Grid3 make_grid(int n) {
  Grid3 g;
  g.n = n;
  g.nc = n / 2 + 1;
  g.pc = (g.nc + 1) & ~1;   // even: complex rows start on 16-byte boundaries
  return g;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int kPkBlocks = 1216;   // 8 CTAs of 256 threads per SM: enough loads in flight
constexpr int kPkMaxBins = 128;

// Integer |m|^2 lower edges of nbins log bins between |m| = 1 and |m| = N/2.
void bin_edges(int nmesh, int nbins, long long* e) {
  const double half = nmesh / 2.0;
  for (int b = 0; b <= nbins; ++b) {
    const double e2 = std::pow(half, 2.0 * b / nbins);
    e[b] = (long long)std::ceil(e2 - 1e-9);
  }
}

enum Stage {
  kStDeposit = 0, kStFwdZ = 1, kStFwdY = 2, kStGreenX = 3, kStInvY = 4, kStInvZ = 5, kStGather = 6,
  kStFwdX = 7, kStIc = 8, kStPk = 9, kStClear = 10, kStBin = 11, kStAdjoint = 12, kStFof = 13, kStIcFft = 14
};

// While the 2LPT lattice (N_p^3) transforms run, the FFT passes count as their own stage, so that
// the PM-step stages hold mesh-size launches only.
struct LatticeScope {
  cola_ctx* c;
  explicit LatticeScope(cola_ctx* ctx) : c(ctx) { c->lattice_fft = true; }
  ~LatticeScope() { c->lattice_fft = false; }
};

cudaEvent_t take_event(cola_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Counts the launch of one stage and, while profiling, brackets it with events on the stream.
template <class F>
int staged(cola_ctx* c, int stage, F&& launch) {
  if (c->lattice_fft && (stage == kStFwdZ || stage == kStFwdY || stage == kStFwdX || stage == kStInvY ||
                         stage == kStInvZ))
    stage = kStIcFft;
  c->stage_launches[stage] += 1;
  if (!c->prof) return launch();
  cola_ctx::Mark m{stage, take_event(c), take_event(c)};
  cudaEventRecord(m.a, c->stream);
  const int st = launch();
  cudaEventRecord(m.b, c->stream);
  c->marks.push_back(m);
  return st;
}

#define STAGED(stage, expr) staged(c, (stage), [&]() { return (expr); })

int check_ptr(const void* p) { return (p && ((uintptr_t)p % 16 == 0)) ? COLA_OK : COLA_ERR_INVALID; }

// S1 + S2 (z, y): deposit and the first two forward passes into cbuf[2].
// S1 into rho: tile-wise (binning, then one plain store per cell) or direct atomics.
int deposit_mesh(cola_ctx* c, const float* s, unsigned long long* rho) {
  if (c->binned) {
    COLA_TRY(STAGED(kStBin, launch_binning(c->pg, c->bg, s, c->bb, c->stream)));
    return STAGED(kStDeposit, launch_deposit_tiles(c->pg, c->bg, s, c->bb, rho, c->stream));
  }
  const size_t n3 = (size_t)c->mesh.n * c->mesh.n * c->mesh.n;
  COLA_TRY(STAGED(kStClear, cuda_status(cudaMemsetAsync(rho, 0, n3 * sizeof(unsigned long long), c->stream), "memset")));
  return STAGED(kStDeposit, launch_deposit(c->pg, s, rho, c->flags, c->stream));
}

// S4 (+S5): gather at the particles deposited by the last deposit_mesh call on the same s.
int gather(cola_ctx* c, const float* s_in, float* force, float* s, float* v, const float* psi1, const float* psi2,
           const KickDrift* kd) {
  const float* f[3] = {reinterpret_cast<float*>(c->cbuf[0]), reinterpret_cast<float*>(c->cbuf[1]),
                       reinterpret_cast<float*>(c->cbuf[2])};
  if (c->binned && c->tile_gather)
    return STAGED(kStGather, launch_gather_tiles(c->pg, c->bg, c->bb, f, 2LL * c->mesh.pc, s_in, force, s, v, psi1,
                                                 psi2, kd, c->flags, c->stream, c->gather_pipe));
  return STAGED(kStGather, launch_gather(c->pg, f, 2LL * c->mesh.pc, s_in, force, s, v, psi1, psi2, kd, c->flags,
                                         c->stream));
}

// S2 (z, y) of a fixed-point mesh into cbuf[2]; with check_mass, the exact total-mass (overflow)
// check of the deposit rides along the z pass.
int forward_yz(cola_ctx* c, const unsigned long long* rho, bool check_mass) {
  const Grid3& g = c->mesh;
  const size_t n3 = (size_t)g.n * g.n * g.n;
  const float scale = (float)((double)n3 / ((double)c->pg.npart * 4398046511104.0));   // N^3 / (n 2^42)
  COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(c->mplan, g, kSrcFixedPoint, rho, g.n, scale, c->cbuf[2], c->stream,
                                           check_mass ? c->mass_acc : nullptr)));
  if (check_mass) COLA_TRY(launch_mass_check(c->pg, nullptr, false, c->mass_acc, c->flags, c->stream));
  COLA_TRY(STAGED(kStFwdY, launch_pencils(c->mplan, g, 1, -1, c->cbuf[2], c->stream)));
  return COLA_OK;
}

int deposit_and_forward_yz(cola_ctx* c, const float* s) {
  if (c->binned) {
    // the tile deposit writes the density contrast itself (half the bytes of the fixed-point mesh, and
    // the z pass reads float rows); its exact 128-bit mass total feeds the overflow check
    const Grid3& g = c->mesh;
    const size_t n3 = (size_t)g.n * g.n * g.n;
    const float scale = (float)((double)n3 / ((double)c->pg.npart * 4398046511104.0));   // N^3 / (n 2^42)
    float* delta = reinterpret_cast<float*>(c->rho);
    COLA_TRY(STAGED(kStBin, launch_binning(c->pg, c->bg, s, c->bb, c->stream)));
    COLA_TRY(STAGED(kStDeposit, launch_deposit_tiles(c->pg, c->bg, s, c->bb, nullptr, c->stream, delta, scale,
                                                     c->tile_mass)));
    COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(c->mplan, g, kSrcFloat, delta, g.n, 1.0f, c->cbuf[2], c->stream)));
    COLA_TRY(launch_mass_reduce(c->tile_mass, c->bg.tiles, c->mass_acc, c->stream));
    COLA_TRY(launch_mass_check(c->pg, nullptr, false, c->mass_acc, c->flags, c->stream));
    return STAGED(kStFwdY, launch_pencils(c->mplan, g, 1, -1, c->cbuf[2], c->stream));
  }
  COLA_TRY(deposit_mesh(c, s, c->rho));
  return forward_yz(c, c->rho, true);
}

// S3 after forward_yz: the three force components as real fields in cbuf[0..2] (rows of 2 pc floats).
// With save_spectrum the fast Green kernels also leave the density's forward spectrum in the
// (already consumed) fixed-point mesh buffer and c->spec_saved says so.
int green_and_inverse(cola_ctx* c, double force_scale, bool save_spectrum = false) {
  const Grid3& g = c->mesh;
  float2* const outs[3] = {c->cbuf[0], c->cbuf[1], c->cbuf[2]};
  bool saved = false;
  COLA_TRY(STAGED(kStGreenX, launch_green_x(c->mplan, g, c->cbuf[2], outs, c->dtab, (float)force_scale, c->stream,
                                            save_spectrum ? reinterpret_cast<float2*>(c->rho) : nullptr, &saved)));
  c->spec_saved = saved;
  for (int j = 0; j < 3; ++j) {
    COLA_TRY(STAGED(kStInvY, launch_pencils(c->mplan, g, 1, +1, c->cbuf[j], c->stream)));
    COLA_TRY(STAGED(kStInvZ, launch_c2r_rows(c->mplan, g, c->cbuf[j], c->stream)));
  }
  return COLA_OK;
}

// S1-S3: the three force components as real fields in cbuf[0..2] (rows of 2 pc floats).
int force_mesh(cola_ctx* c, const float* s, double force_scale, bool save_spectrum = false) {
  COLA_TRY(deposit_and_forward_yz(c, s));
  return green_and_inverse(c, force_scale, save_spectrum);
}

int inverse3d(cola_ctx* c, const Grid3& g, const FftPlan& p, float2* b) {
  COLA_TRY(STAGED(kStFwdX, launch_pencils(p, g, 0, +1, b, c->stream)));
  COLA_TRY(STAGED(kStInvY, launch_pencils(p, g, 1, +1, b, c->stream)));
  return STAGED(kStInvZ, launch_c2r_rows(p, g, b, c->stream));
}

// A 2LPT field: inverse3d of mul times the lattice spectrum src, into dst, and, with particles, into
// that particle array (dense, times scale).  Where the plan allows, the multiply rides in the first
// inverse pass and the last pass writes the particle layout itself; else separate kernels do.
int inverse3d_mul(cola_ctx* c, const Grid3& g, const FftPlan& p, const float2* src, const IcMul& mul, float2* dst,
                  float scale = 1.0f, float* particles = nullptr) {
  if (pencils_x_mul_ok(p, g)) {
    COLA_TRY(STAGED(kStFwdX, launch_pencils_x_mul(p, g, src, mul, dst, c->stream)));
  } else {
    COLA_TRY(STAGED(kStIc, launch_ic_multiply(g, src, dst, (IcField)mul.kind, mul.ci, mul.cj, mul.scale, c->stream)));
    COLA_TRY(STAGED(kStFwdX, launch_pencils(p, g, 0, +1, dst, c->stream)));
  }
  COLA_TRY(STAGED(kStInvY, launch_pencils(p, g, 1, +1, dst, c->stream)));
  if (!particles) return STAGED(kStInvZ, launch_c2r_rows(p, g, dst, c->stream));
  if (c2r_rows_dense_ok(p, g)) return STAGED(kStInvZ, launch_c2r_rows_dense(p, g, dst, scale, particles, c->stream));
  COLA_TRY(STAGED(kStInvZ, launch_c2r_rows(p, g, dst, c->stream)));
  return STAGED(kStIc, launch_ic_to_particles(g, dst, scale, particles, c->stream));
}

int forward3d_yx(cola_ctx* c, const Grid3& g, const FftPlan& p, float2* b) {
  COLA_TRY(STAGED(kStFwdY, launch_pencils(p, g, 1, -1, b, c->stream)));
  return STAGED(kStFwdX, launch_pencils(p, g, 0, -1, b, c->stream));
}

// W(k) = R2C of the lattice white noise into B0: the caller's field wn, or (wn == NULL) the field
// of params.seed drawn into B0's real rows first (the R2C then runs in place).
int noise_spectrum(cola_ctx* c, const float* wn, float2* b0) {
  const Grid3& g = c->lat;
  if (wn) return STAGED(kStFwdZ, launch_r2c_rows(c->lplan, g, kSrcFloat, wn, g.n, 1.0f, b0, c->stream));
  float* rows = reinterpret_cast<float*>(b0);
  COLA_TRY(STAGED(kStIc, launch_white_noise(c->p.seed, c->p.np, 2LL * g.pc, rows, c->stream)));
  return STAGED(kStFwdZ, launch_r2c_rows(c->lplan, g, kSrcFloat, rows, 2LL * g.pc, 1.0f, b0, c->stream));
}

}  // namespace

extern "C" const char* cola_strerror(int status) {
  switch (status) {
    case COLA_OK: return "ok";
    case COLA_ERR_INVALID: return "invalid argument or size";
    case COLA_ERR_OOM: return "device allocation failed";
    case COLA_ERR_CUDA: return "CUDA runtime error";
    case COLA_ERR_OVERFLOW: return "fixed-point density overflow";
    case COLA_ERR_NONFINITE: return "non-finite particle position or velocity";
    case COLA_ERR_INTERNAL: return "internal iteration limit reached";
    default: return "unknown status";
  }
}

extern "C" int cola_step_scalars(const cola_params* params, int i, double* out, int nout) {
  if (validate(params) != COLA_OK || !out || nout < 12 || i < 0 || i > params->nstep) return COLA_ERR_INVALID;
  const Cosmo cosmo(params->omega_m, params->h, params->n_s, params->sigma8);
  for (int k = 0; k < 12; ++k) out[k] = 0.0;
  if (i == 0) {
    const double a1 = 1.0 / params->nstep;
    out[0] = a1;
    out[8] = cosmo.d1_da(1.0) * hubble(1.0, params->omega_m);
    out[9] = cosmo.d2_da(1.0) * hubble(1.0, params->omega_m);
    out[10] = cosmo.d1(a1);
    out[11] = cosmo.d2(a1);
    return COLA_OK;
  }
  const StepScalars s = step_scalars(*params, cosmo, i);
  const double v[12] = {s.a, s.a_lo, s.a_hi, s.force_scale, s.c1, s.c2, s.kick, s.drift, s.dd1, s.dd2, s.d1, s.d2};
  for (int k = 0; k < 12; ++k) out[k] = v[k];
  return COLA_OK;
}

extern "C" int cola_linear_power(const cola_params* params, const double* k, int nk, double* power,
                                 double* transfer) {
  if (validate(params) != COLA_OK || nk < 0 || (nk > 0 && !k)) return COLA_ERR_INVALID;
  const Cosmo cosmo(params->omega_m, params->h, params->n_s, params->sigma8);
  for (int i = 0; i < nk; ++i) {
    if (!(k[i] >= 0.0) || !std::isfinite(k[i])) return COLA_ERR_INVALID;
    if (power) power[i] = cosmo.power(k[i]);
    if (transfer) transfer[i] = cosmo.transfer(k[i]);
  }
  return COLA_OK;
}

extern "C" int cola_white_noise(const cola_params* params, float* out, void* stream) {
  if (validate(params) != COLA_OK) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(out));
  return launch_white_noise(params->seed, params->np, params->np, out, static_cast<cudaStream_t>(stream));
}

extern "C" int cola_philox_words(unsigned long long seed, long long first, long long count, unsigned* out,
                                 void* stream) {
  if (first < 0 || count < 0 || (count > 0 && check_ptr(out) != COLA_OK)) return COLA_ERR_INVALID;
  if (count == 0) return COLA_OK;
  return launch_philox_words(seed, first, count, out, static_cast<cudaStream_t>(stream));
}

extern "C" void cola_destroy(cola_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  if (c->edges_host) cudaFreeHost(c->edges_host);
  fft_plan_free(&c->mplan);
  fft_plan_free(&c->lplan);
  void* bufs[] = {c->arena,    c->dtab,     c->amp_m2,  c->edges, c->pk_partials, c->pk_geom,
                  c->flags,    c->mass_acc, c->bin_mem, c->adj_mem,     c->fof_mem,  c->fof_sums};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete c;
}

extern "C" int cola_create(const cola_params* params, void* stream, cola_ctx** out) {
  if (!out) return COLA_ERR_INVALID;
  *out = nullptr;
  COLA_TRY(validate(params));
  cola_ctx* c = new (std::nothrow) cola_ctx;
  if (!c) return COLA_ERR_OOM;
  c->p = *params;
  c->stream = static_cast<cudaStream_t>(stream);
  c->mesh = make_grid(params->nmesh);
  c->lat = make_grid(params->np);
  c->pg.np = params->np;
  c->pg.n = params->nmesh;
  c->pg.r_fixed = (((long long)params->nmesh) << 20) / params->np;
  c->pg.npart = (long long)params->np * params->np * params->np;
  auto fail = [&](int st) {
    cola_destroy(c);
    return st;
  };
  int st = fft_plan_init(&c->mplan, params->nmesh);
  if (st == COLA_OK) st = fft_plan_init(&c->lplan, params->np);
  if (st != COLA_OK) return fail(st);

  // host FP64 tables
  const Cosmo cosmo(params->omega_m, params->h, params->n_s, params->sigma8);
  c->steps.resize(params->nstep + 1);
  for (int i = 1; i <= params->nstep; ++i) c->steps[i] = step_scalars(*params, cosmo, i);
  {
    const double a1 = 1.0 / params->nstep;
    c->steps[0] = StepScalars{};
    c->steps[0].a = a1;
    c->steps[0].d1 = cosmo.d1(a1);
    c->steps[0].d2 = cosmo.d2(a1);
    c->vel_f1 = cosmo.d1_da(1.0) * hubble(1.0, params->omega_m);
    c->vel_f2 = cosmo.d2_da(1.0) * hubble(1.0, params->omega_m);
  }

  // device memory: meshes and the IC work space share one arena
  const size_t cbytes = align256(c->mesh.complex_elems() * sizeof(float2));
  const size_t nm3 = (size_t)params->nmesh * params->nmesh * params->nmesh;
  const size_t mesh_bytes = align256(nm3 * sizeof(unsigned long long)) + 3 * cbytes;
  const size_t lbytes = align256(c->lat.complex_elems() * sizeof(float2));
  const size_t ic_bytes = 8 * lbytes;
  c->arena_bytes = mesh_bytes > ic_bytes ? mesh_bytes : ic_bytes;
  if ((st = cuda_status(cudaMalloc(&c->arena, c->arena_bytes), "cudaMalloc arena")) != COLA_OK) return fail(st);
  char* base = static_cast<char*>(c->arena);
  c->rho = reinterpret_cast<unsigned long long*>(base);
  for (int j = 0; j < 3; ++j)
    c->cbuf[j] = reinterpret_cast<float2*>(base + align256(nm3 * sizeof(unsigned long long)) + j * cbytes);

  // gradient kernel per storage index: D(m) = (8 sin k - sin 2k)/6, k = 2 pi m / N, 0 at Nyquist
  {
    const int n = params->nmesh;
    std::vector<float> d(n);
    for (int j = 0; j < n; ++j) {
      const int m = j < n / 2 ? j : j - n;
      const double k = 2.0 * M_PI * m / n;
      d[j] = (2 * j == n) ? 0.0f : (float)((8.0 * std::sin(k) - std::sin(2.0 * k)) / 6.0);
    }
    if ((st = cuda_status(cudaMalloc(&c->dtab, n * sizeof(float)), "cudaMalloc dtab")) != COLA_OK) return fail(st);
    cudaMemcpy(c->dtab, d.data(), n * sizeof(float), cudaMemcpyHostToDevice);
  }
  // sqrt(P(k) / V_cell) / np^3 per integer |m|^2 of the lattice, k = 2 pi |m| / L
  {
    const int npd = params->np;
    const long long m2max = 3LL * (npd / 2) * (npd / 2);
    std::vector<float> amp(m2max + 1);
    const double vcell = std::pow(params->box / npd, 3);
    const double n3 = (double)npd * npd * npd;
    amp[0] = 0.0f;
    for (long long m2 = 1; m2 <= m2max; ++m2) {
      const double k = 2.0 * M_PI * std::sqrt((double)m2) / params->box;
      amp[m2] = (float)(std::sqrt(cosmo.power(k) / vcell) / n3);
    }
    if ((st = cuda_status(cudaMalloc(&c->amp_m2, amp.size() * sizeof(float)), "cudaMalloc amp")) != COLA_OK)
      return fail(st);
    cudaMemcpy(c->amp_m2, amp.data(), amp.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  c->pk_blocks = kPkBlocks;
  if ((st = cuda_status(cudaMalloc(&c->edges, (kPkMaxBins + 1) * sizeof(long long)), "cudaMalloc")) != COLA_OK ||
      (st = cuda_status(cudaMalloc(&c->pk_partials, (size_t)kPkBlocks * 2 * kPkMaxBins * sizeof(double)),
                        "cudaMalloc")) != COLA_OK ||
      (st = cuda_status(cudaMalloc(&c->pk_geom, 2 * kPkMaxBins * sizeof(double)), "cudaMalloc")) != COLA_OK ||
      (st = cuda_status(cudaMalloc(&c->flags, sizeof(int)), "cudaMalloc")) != COLA_OK ||
      (st = cuda_status(cudaMalloc(&c->mass_acc, 2 * kMassSlots * sizeof(unsigned long long)), "cudaMalloc")) != COLA_OK)
    return fail(st);
  cudaMemset(c->flags, 0, sizeof(int));
  cudaMemset(c->mass_acc, 0, 2 * kMassSlots * sizeof(unsigned long long));
  // tile binning buffers: 6 per-tile arrays, n primary entries and up to 7n spill entries
  if (bin_geometry(params->nmesh, params->np, &c->bg)) {
    const size_t tiles = (size_t)c->bg.tiles + 1;
    const size_t nseg = (tiles + 4095) / 4096 + 1;
    const size_t bytes = 6 * align256(tiles * sizeof(unsigned)) + align256((size_t)c->pg.npart * 4) +
                         align256((size_t)c->pg.npart * 28) + align256(2 * nseg * sizeof(unsigned)) +
                         align256(tiles * 2 * sizeof(unsigned long long)) + align256((size_t)c->pg.npart * 8);
    if ((st = cuda_status(cudaMalloc(&c->bin_mem, bytes), "cudaMalloc bins")) != COLA_OK) return fail(st);
    char* q = static_cast<char*>(c->bin_mem);
    unsigned** arr[6] = {&c->bb.cnt_p, &c->bb.cnt_s, &c->bb.off_p, &c->bb.off_s, &c->bb.cur_p, &c->bb.cur_s};
    for (int i = 0; i < 6; ++i) {
      *arr[i] = reinterpret_cast<unsigned*>(q);
      q += align256(tiles * sizeof(unsigned));
    }
    c->bb.ent_p = reinterpret_cast<unsigned*>(q);
    q += align256((size_t)c->pg.npart * 4);
    c->bb.ent_s = reinterpret_cast<unsigned*>(q);
    q += align256((size_t)c->pg.npart * 28);
    c->bb.seg = reinterpret_cast<unsigned*>(q);
    q += align256(2 * nseg * sizeof(unsigned));
    c->tile_mass = reinterpret_cast<unsigned long long*>(q);
    q += align256(tiles * 2 * sizeof(unsigned long long));
    c->bb.rec = reinterpret_cast<unsigned long long*>(q);
    c->binned = true;
    c->tile_gather = tile_gather_pays(c->bg, c->pg.npart);
  }
  // meshes (and 2LPT lattices) of 769 to 1536 cells: the in-place pipelined strided passes hold
  // tiles of 8 pencils (64-byte row segments) where the three-buffer ones hold 4 (at 1536: 185.6
  // against 203.2 ms per PM force evaluation on 1024^3 particles)
  auto inplace_pays = [](int n) { return n > 768 && n * 8 <= 12288; };
  c->mplan.pipe_inplace = inplace_pays(params->nmesh);
  c->lplan.pipe_inplace = inplace_pays(params->np);
  if ((st = cuda_status(cudaMallocHost(&c->edges_host, (kPkMaxBins + 1) * sizeof(long long)), "cudaMallocHost")) !=
      COLA_OK)
    return fail(st);
  bin_edges(params->nmesh, 64, c->edges_host);
  c->edges_nbins = 64;
  cudaMemcpy(c->edges, c->edges_host, 65 * sizeof(long long), cudaMemcpyHostToDevice);
  if ((st = cuda_status(cudaDeviceSynchronize(), "create")) != COLA_OK) return fail(st);
  *out = c;
  return COLA_OK;
}

extern "C" int cola_sync(cola_ctx* c) {
  if (!c) return COLA_ERR_INVALID;
  COLA_TRY(cuda_status(cudaStreamSynchronize(c->stream), "stream sync"));
  int flags = 0;
  COLA_TRY(cuda_status(cudaMemcpy(&flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost), "flags"));
  if (flags) cudaMemset(c->flags, 0, sizeof(int));
  if (flags & 1) return COLA_ERR_OVERFLOW;
  if (flags & 2) return COLA_ERR_NONFINITE;
  if (flags & 4) return COLA_ERR_INTERNAL;
  return COLA_OK;
}

extern "C" int cola_ic_2lpt(cola_ctx* c, const float* wn, float* s, float* v, float* psi1, float* psi2) {
  if (!c) return COLA_ERR_INVALID;
  if (wn) COLA_TRY(check_ptr(wn));
  for (const void* p : {(const void*)s, (const void*)v, (const void*)psi1, (const void*)psi2})
    COLA_TRY(check_ptr(p));
  const LatticeScope scope(c);
  const Grid3& g = c->lat;
  const FftPlan& P = c->lplan;
  const size_t lbytes = align256(g.complex_elems() * sizeof(float2));
  float2* B[8];
  for (int i = 0; i < 8; ++i) B[i] = reinterpret_cast<float2*>(static_cast<char*>(c->arena) + i * lbytes);
  const long long n = c->pg.npart;
  const float r = (float)c->p.nmesh / (float)c->p.np;   // lattice spacings -> mesh cells
  // white noise -> W(k) -> delta_L(k) / np^3
  COLA_TRY(noise_spectrum(c, wn, B[0]));
  COLA_TRY(forward3d_yx(c, g, P, B[0]));
  COLA_TRY(STAGED(kStIc, launch_ic_amplitude(g, B[0], c->amp_m2, c->stream)));
  // Psi1 = i k delta_L / k^2
  for (int j = 0; j < 3; ++j) {
    COLA_TRY(inverse3d_mul(c, g, P, B[0], IcMul{kIcPsi1, j, 0, 1.0f}, B[7], r, psi1 + j * n));
  }
  // phi1_ij = k_i k_j delta_L / k^2 in real space, then the second-order source
  const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int h = 0; h < 6; ++h) {
    COLA_TRY(inverse3d_mul(c, g, P, B[0], IcMul{kIcHess, pairs[h][0], pairs[h][1], 1.0f}, B[1 + h]));
  }
  float2* const hs[6] = {B[1], B[2], B[3], B[4], B[5], B[6]};
  COLA_TRY(STAGED(kStIc, launch_ic_source(g, hs, B[7], c->stream)));
  COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(P, g, kSrcFloat, B[7], 2LL * g.pc, 1.0f, B[7], c->stream)));
  COLA_TRY(forward3d_yx(c, g, P, B[7]));
  // Psi2 = -i k S(k) / k^2
  const float inv_n3 = (float)(1.0 / ((double)g.n * g.n * g.n));
  for (int j = 0; j < 3; ++j) {
    COLA_TRY(inverse3d_mul(c, g, P, B[7], IcMul{kIcPsi2, j, 0, inv_n3}, B[1], r, psi2 + j * n));
  }
  const StepScalars& s0 = c->steps[0];
  return STAGED(kStIc, launch_ic_positions(n, psi1, psi2, (float)s0.d1, (float)s0.d2, s, v, c->stream));
}

extern "C" int cola_deposit(cola_ctx* c, const float* s, unsigned long long* rho) {
  if (!c) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(s));
  COLA_TRY(check_ptr(rho));
  const size_t n3 = (size_t)c->mesh.n * c->mesh.n * c->mesh.n;
  (void)n3;
  COLA_TRY(deposit_mesh(c, s, rho));
  return launch_mass_check(c->pg, rho, true, c->mass_acc, c->flags, c->stream);
}

extern "C" int cola_density_spectrum(cola_ctx* c, const float* s, float* delta_k) {
  if (!c) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(s));
  COLA_TRY(check_ptr(delta_k));
  COLA_TRY(deposit_and_forward_yz(c, s));
  COLA_TRY(STAGED(kStFwdX, launch_pencils(c->mplan, c->mesh, 0, -1, c->cbuf[2], c->stream)));
  return launch_dense_spectrum(c->mesh, c->cbuf[2], delta_k, c->stream);
}

extern "C" int cola_density_spectrum_of_mesh(cola_ctx* c, const unsigned long long* rho, float* delta_k) {
  if (!c) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(rho));
  COLA_TRY(check_ptr(delta_k));
  COLA_TRY(forward_yz(c, rho, false));
  COLA_TRY(STAGED(kStFwdX, launch_pencils(c->mplan, c->mesh, 0, -1, c->cbuf[2], c->stream)));
  return launch_dense_spectrum(c->mesh, c->cbuf[2], delta_k, c->stream);
}

extern "C" int cola_pm_force_of_mesh(cola_ctx* c, const unsigned long long* rho, double a, const long long* cells,
                                     long long m, float* force) {
  if (!c || !(a > 0.0) || m < 0) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(rho));
  if (m > 0) {
    COLA_TRY(check_ptr(cells));
    COLA_TRY(check_ptr(force));
  }
  COLA_TRY(forward_yz(c, rho, false));
  COLA_TRY(green_and_inverse(c, 1.5 * c->p.omega_m / a));
  const float* f[3] = {reinterpret_cast<float*>(c->cbuf[0]), reinterpret_cast<float*>(c->cbuf[1]),
                       reinterpret_cast<float*>(c->cbuf[2])};
  return launch_sample_mesh(c->mesh, f, cells, m, force, c->stream);
}

extern "C" int cola_pm_force(cola_ctx* c, const float* s, double a, float* force) {
  if (!c || !(a > 0.0)) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(s));
  COLA_TRY(check_ptr(force));
  COLA_TRY(force_mesh(c, s, 1.5 * c->p.omega_m / a));
  return gather(c, s, force, nullptr, nullptr, nullptr, nullptr, nullptr);
}

namespace {
// COLA step i; save_spectrum keeps the density spectrum of s (see green_and_inverse).
int step_impl(cola_ctx* c, int i, float* s, float* v, const float* psi1, const float* psi2, bool save_spectrum) {
  if (!c || i < 1 || i > c->p.nstep) return COLA_ERR_INVALID;
  for (const void* p : {(const void*)s, (const void*)v, (const void*)psi1, (const void*)psi2})
    COLA_TRY(check_ptr(p));
  const StepScalars& ss = c->steps[i];
  COLA_TRY(force_mesh(c, s, ss.force_scale, save_spectrum));
  const KickDrift kd{(float)ss.kick, (float)ss.drift, (float)ss.dd1, (float)ss.dd2, (float)ss.c1, (float)ss.c2};
  return gather(c, nullptr, nullptr, s, v, psi1, psi2, &kd);
}

// S6 binning of a forward density spectrum dk (complex N x N x pc) into pk.
int pk_from_spectrum(cola_ctx* c, const float2* dk, double* pk, int nbins, int flags) {
  if (nbins != c->edges_nbins) {
    // the pinned host copy may still feed an earlier upload: wait for it before rewriting it
    COLA_TRY(cuda_status(cudaStreamSynchronize(c->stream), "pk edges"));
    bin_edges(c->mesh.n, nbins, c->edges_host);
    COLA_TRY(cuda_status(cudaMemcpyAsync(c->edges, c->edges_host, (nbins + 1) * sizeof(long long),
                                         cudaMemcpyHostToDevice, c->stream), "edges"));
    c->edges_nbins = nbins;
  }
  const double nn = c->mesh.n;
  const double vol = std::pow(c->p.box, 3);
  const double pscale = vol / (nn * nn * nn * nn * nn * nn);
  const double kfund = 2.0 * M_PI / c->p.box;
  const int corr = (flags & COLA_PK_CIC_CORRECT) ? 1 : 0;
  if (c->pk_geom_nbins != nbins) {   // once per bin count: mode counts and mean |k| of the bins
    COLA_TRY(STAGED(kStPk, launch_pk_geometry(c->mesh, c->edges, nbins, c->pk_partials, c->pk_blocks, c->pk_geom,
                                              c->stream)));
    c->pk_geom_nbins = nbins;
  }
  COLA_TRY(STAGED(kStPk, launch_pk_bins(c->mesh, dk, c->edges, nbins, corr, c->pk_partials, c->pk_blocks,
                                        c->stream)));
  return STAGED(kStPk, launch_pk_finish(c->pk_partials, c->pk_blocks, nbins, c->pk_geom, kfund, pscale,
                                        corr ? vol / (double)c->pg.npart : 0.0, pk, c->stream));
}
}  // namespace

extern "C" int cola_step(cola_ctx* c, int i, float* s, float* v, const float* psi1, const float* psi2) {
  return step_impl(c, i, s, v, psi1, psi2, false);
}

extern "C" int cola_power_spectrum_ex(cola_ctx* c, const float* s, double* pk, int nbins, int flags) {
  if (!c || nbins < 1 || nbins > kPkMaxBins || (flags & ~COLA_PK_CIC_CORRECT)) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(s));
  COLA_TRY(check_ptr(pk));
  COLA_TRY(deposit_and_forward_yz(c, s));
  COLA_TRY(STAGED(kStFwdX, launch_pencils(c->mplan, c->mesh, 0, -1, c->cbuf[2], c->stream)));
  return pk_from_spectrum(c, c->cbuf[2], pk, nbins, flags);
}

extern "C" int cola_power_spectrum(cola_ctx* c, const float* s, double* pk, int nbins) {
  return cola_power_spectrum_ex(c, s, pk, nbins, 0);
}

extern "C" int cola_snapshot(cola_ctx* c, int i, double a_snap, const float* s, const float* v, const float* psi1,
                             const float* psi2, float* s_out, float* v_out) {
  if (!c || i < 1 || i > c->p.nstep) return COLA_ERR_INVALID;
  for (const void* p : {(const void*)s, (const void*)v, (const void*)psi1, (const void*)psi2, (const void*)s_out})
    COLA_TRY(check_ptr(p));
  if (v_out) COLA_TRY(check_ptr(v_out));
  const StepScalars& ss = c->steps[i];
  const bool last = i == c->p.nstep;
  const double a_next = last ? ss.a : (double)(i + 1) / c->p.nstep;
  if (!(a_snap >= ss.a - 1e-12 && a_snap <= a_next + 1e-12)) return COLA_ERR_INVALID;
  const Cosmo cosmo(c->p.omega_m, c->p.h, c->p.n_s, c->p.sigma8);
  // the state holds s at a_next and v_res at a_{i+1/2}: step back from a_next to a_snap
  double alpha = 0.0, b1 = 0.0, b2 = 0.0;
  if (!last) {
    alpha = -cosmo.drift(a_snap, a_next, ss.a_hi, c->p.nlpt, c->p.drift_ansatz);
    b1 = cosmo.d1(a_snap) - cosmo.d1(a_next);
    b2 = cosmo.d2(a_snap) - cosmo.d2(a_next);
  }
  const double f = a_snap * a_snap * a_snap * hubble(a_snap, c->p.omega_m);   // a^2 d/dt = a^3 H d/da
  const double g1 = f * cosmo.d1_da(a_snap), g2 = f * cosmo.d2_da(a_snap);
  return STAGED(kStIc, launch_snapshot(c->pg.npart, s, v, psi1, psi2, (float)alpha, (float)b1, (float)b2, (float)g1,
                                       (float)g2, s_out, v_out, c->stream));
}

extern "C" int cola_run(cola_ctx* c, const float* wn, float* s, float* v, float* psi1, float* psi2, double* pk,
                        int nbins) {
  if (!c) return COLA_ERR_INVALID;
  if (pk && (nbins < 1 || nbins > kPkMaxBins || check_ptr(pk) != COLA_OK)) return COLA_ERR_INVALID;
  COLA_TRY(cola_ic_2lpt(c, wn, s, v, psi1, psi2));
  for (int i = 1; i < c->p.nstep; ++i) COLA_TRY(step_impl(c, i, s, v, psi1, psi2, false));
  // the last step kicks to a = 1 without drifting, so the positions it deposits are the final ones:
  // its density spectrum, kept by the Green pass, gives P(k) without a second deposit and FFT
  COLA_TRY(step_impl(c, c->p.nstep, s, v, psi1, psi2, pk != nullptr));
  if (pk) {
    if (c->spec_saved) COLA_TRY(pk_from_spectrum(c, reinterpret_cast<const float2*>(c->rho), pk, nbins, 0));
    else COLA_TRY(cola_power_spectrum(c, s, pk, nbins));
  }
  return COLA_OK;
}

extern "C" int cola_run_kernel_count(cola_ctx* c, const float* wn, float* s, float* v, float* psi1, float* psi2,
                                     double* pk, int nbins, long long* kernels) {
  if (!c || !kernels || (pk && nbins != c->edges_nbins)) return COLA_ERR_INVALID;
  *kernels = 0;
  cudaStream_t cap = nullptr;
  COLA_TRY(cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stream"));
  const cudaStream_t saved = c->stream;
  const bool prof = c->prof;
  long long launches[COLA_NUM_STAGES];
  std::copy(c->stage_launches, c->stage_launches + COLA_NUM_STAGES, launches);
  c->stream = cap;
  c->prof = false;   // no timing events inside the capture
  int st = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed), "begin capture");
  if (st == COLA_OK) {
    const int run_st = cola_run(c, wn, s, v, psi1, psi2, pk, nbins);
    cudaGraph_t g = nullptr;
    const int end_st = cuda_status(cudaStreamEndCapture(cap, &g), "end capture");
    st = run_st != COLA_OK ? run_st : end_st;
    size_t nn = 0;
    if (st == COLA_OK) st = cuda_status(cudaGraphGetNodes(g, nullptr, &nn), "graph nodes");
    if (st == COLA_OK && nn) {
      std::vector<cudaGraphNode_t> nodes(nn);
      st = cuda_status(cudaGraphGetNodes(g, nodes.data(), &nn), "graph nodes");
      for (size_t i = 0; st == COLA_OK && i < nn; ++i) {
        cudaGraphNodeType ty;
        st = cuda_status(cudaGraphNodeGetType(nodes[i], &ty), "node type");
        if (st == COLA_OK && ty == cudaGraphNodeTypeKernel) ++*kernels;
      }
    }
    if (g) cudaGraphDestroy(g);
  }
  c->stream = saved;
  c->prof = prof;
  std::copy(launches, launches + COLA_NUM_STAGES, c->stage_launches);
  cudaStreamDestroy(cap);
  return st;
}

extern "C" int cola_run_snapshots(cola_ctx* c, const float* wn, float* s, float* v, float* psi1, float* psi2,
                                  const double* a_snap, int nsnap, float* s_snap, float* v_snap, double* pk_snap,
                                  int nbins, int pk_flags) {
  if (!c || nsnap < 1 || !a_snap || !s_snap) return COLA_ERR_INVALID;
  const double a1 = 1.0 / c->p.nstep;
  for (int k = 0; k < nsnap; ++k)
    if (!(a_snap[k] >= a1 && a_snap[k] <= 1.0 + 1e-12) || (k > 0 && !(a_snap[k] > a_snap[k - 1])))
      return COLA_ERR_INVALID;
  const size_t pbytes = (size_t)3 * c->pg.npart * sizeof(float);
  COLA_TRY(cola_ic_2lpt(c, wn, s, v, psi1, psi2));
  int k = 0;
  for (int i = 1; i <= c->p.nstep; ++i) {
    COLA_TRY(cola_step(c, i, s, v, psi1, psi2));
    const double a_next = i == c->p.nstep ? 1.0 : (double)(i + 1) / c->p.nstep;
    for (; k < nsnap && a_snap[k] <= a_next + 1e-12; ++k) {
      float* so = reinterpret_cast<float*>(reinterpret_cast<char*>(s_snap) + k * pbytes);
      float* vo = v_snap ? reinterpret_cast<float*>(reinterpret_cast<char*>(v_snap) + k * pbytes) : nullptr;
      COLA_TRY(cola_snapshot(c, i, a_snap[k], s, v, psi1, psi2, so, vo));
      if (pk_snap) COLA_TRY(cola_power_spectrum_ex(c, so, pk_snap + (size_t)k * 3 * nbins, nbins, pk_flags));
    }
  }
  return COLA_OK;
}

// ---- execution schedule and autotuner ---------------------------------------------------------
namespace {
constexpr int kPipeBudgetsKb[3] = {160, 96, 64};

int schedule_of(const cola_ctx* c) {
  int k = 0;
  while (k < 2 && kPipeBudgetsKb[k] != c->mplan.pipe_kb) ++k;
  return (c->binned ? COLA_SCHED_BINNED_DEPOSIT : 0) | (c->tile_gather ? COLA_SCHED_TILE_GATHER : 0) |
         (c->mplan.pipe ? COLA_SCHED_PIPELINED_FFT : 0) | (c->mplan.pipe_ept == 8 ? COLA_SCHED_PIPE_EPT8 : 0) |
         (c->gather_pipe ? COLA_SCHED_PIPELINED_GATHER : 0) | (c->mplan.green_ept == 8 ? COLA_SCHED_GREEN_EPT8 : 0) |
         (c->mplan.row_ept == 8 ? COLA_SCHED_C2R_EPT8 : 0) | (c->mplan.row_pipe ? COLA_SCHED_ROWS_PIPE : 0) |
         (k << COLA_SCHED_BUDGET_SHIFT) | (c->mplan.r2c_ept == 8 ? COLA_SCHED_R2C_EPT8 : 0) |
         (c->mplan.wide ? COLA_SCHED_WIDE_TILES : 0) | (c->mplan.pipe_inplace ? COLA_SCHED_PIPE_INPLACE : 0);
}

bool schedule_valid(const cola_ctx* c, int sc) {
  if (sc & ~(COLA_SCHED_BINNED_DEPOSIT | COLA_SCHED_TILE_GATHER | COLA_SCHED_PIPELINED_FFT | COLA_SCHED_PIPE_EPT8 |
             COLA_SCHED_PIPELINED_GATHER | COLA_SCHED_GREEN_EPT8 | COLA_SCHED_C2R_EPT8 | COLA_SCHED_ROWS_PIPE |
             (3 << COLA_SCHED_BUDGET_SHIFT) | COLA_SCHED_R2C_EPT8 | COLA_SCHED_WIDE_TILES | COLA_SCHED_PIPE_INPLACE))
    return false;
  if ((sc & COLA_SCHED_PIPELINED_GATHER) && !(sc & COLA_SCHED_TILE_GATHER)) return false;
  if ((sc & COLA_SCHED_PIPE_EPT8) && !(sc & COLA_SCHED_PIPELINED_FFT)) return false;   // unused knob
  if ((sc & COLA_SCHED_BINNED_DEPOSIT) && !c->bin_mem) return false;
  if ((sc & COLA_SCHED_TILE_GATHER) && !(sc & COLA_SCHED_BINNED_DEPOSIT)) return false;
  if ((sc & COLA_SCHED_TILE_GATHER) && c->bg.lz < 2) return false;   // 16-byte staging copies along z
  if (((sc >> COLA_SCHED_BUDGET_SHIFT) & 3) > 2) return false;
  if (!(sc & COLA_SCHED_PIPELINED_FFT) && ((sc >> COLA_SCHED_BUDGET_SHIFT) & 3)) return false;   // unused knob
  if ((sc & COLA_SCHED_PIPE_INPLACE) && (!(sc & COLA_SCHED_PIPELINED_FFT) || (sc & COLA_SCHED_PIPE_EPT8) ||
                                          ((sc >> COLA_SCHED_BUDGET_SHIFT) & 3)))
    return false;   // its own budget, 16 elements per thread
  return true;
}

void apply_schedule(cola_ctx* c, int sc) {
  c->binned = (sc & COLA_SCHED_BINNED_DEPOSIT) != 0;
  c->tile_gather = (sc & COLA_SCHED_TILE_GATHER) != 0;
  c->mplan.pipe = (sc & COLA_SCHED_PIPELINED_FFT) != 0;
  c->mplan.pipe_kb = kPipeBudgetsKb[(sc >> COLA_SCHED_BUDGET_SHIFT) & 3];
  c->mplan.pipe_ept = (sc & COLA_SCHED_PIPE_EPT8) ? 8 : 16;
  c->gather_pipe = (sc & COLA_SCHED_PIPELINED_GATHER) != 0;
  c->mplan.green_ept = (sc & COLA_SCHED_GREEN_EPT8) ? 8 : 16;
  c->mplan.row_ept = (sc & COLA_SCHED_C2R_EPT8) ? 8 : 16;
  c->mplan.r2c_ept = (sc & COLA_SCHED_R2C_EPT8) ? 8 : 16;
  c->mplan.wide = (sc & COLA_SCHED_WIDE_TILES) != 0;
  c->mplan.pipe_inplace = (sc & COLA_SCHED_PIPE_INPLACE) != 0;
  c->mplan.row_pipe = (sc & COLA_SCHED_ROWS_PIPE) != 0;
}
}  // namespace

extern "C" int cola_get_schedule(cola_ctx* c, int* schedule) {
  if (!c || !schedule) return COLA_ERR_INVALID;
  *schedule = schedule_of(c);
  return COLA_OK;
}

extern "C" int cola_set_schedule(cola_ctx* c, int schedule) {
  if (!c || !schedule_valid(c, schedule)) return COLA_ERR_INVALID;
  apply_schedule(c, schedule);
  return COLA_OK;
}

extern "C" int cola_autotune(cola_ctx* c, const float* s, int reps, int* best, int* scheds, double* ms,
                             int max_candidates) {
  if (!c || reps < 1 || max_candidates < 0) return -COLA_ERR_INVALID;
  if (check_ptr(s) != COLA_OK) return -COLA_ERR_INVALID;
  const int keep = schedule_of(c);
  float* force = nullptr;
  if (cuda_status(cudaMalloc(&force, (size_t)3 * c->pg.npart * sizeof(float)), "cudaMalloc tune") != COLA_OK)
    return -COLA_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool prof = c->prof;
  c->prof = false;
  const double fs = 1.5 * c->p.omega_m;   // force at a = 1
  int st = COLA_OK;
  std::vector<std::pair<int, float>> timed;   // schedule, ms per force evaluation
  auto time_of = [&](int sc) -> float {
    for (const auto& t : timed)
      if (t.first == sc) return t.second;
    apply_schedule(c, sc);
    st = force_mesh(c, s, fs);   // warm-up (lazy kernel attributes, caches)
    if (st == COLA_OK) st = gather(c, s, force, nullptr, nullptr, nullptr, nullptr, nullptr);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && st == COLA_OK; ++r) {
      st = force_mesh(c, s, fs);
      if (st == COLA_OK) st = gather(c, s, force, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    cudaEventRecord(e1, c->stream);
    if (st == COLA_OK) st = cuda_status(cudaEventSynchronize(e1), "tune");
    float t = 0.0f;
    if (st == COLA_OK) cudaEventElapsedTime(&t, e0, e1);
    t /= reps;
    timed.push_back({sc, t});
    return t;
  };
  // coordinate search from the current schedule: one group of knobs at a time, the others fixed
  const int kB1 = 1 << COLA_SCHED_BUDGET_SHIFT, kB2 = 2 << COLA_SCHED_BUDGET_SHIFT;
  const int P = COLA_SCHED_PIPELINED_FFT, E = COLA_SCHED_PIPE_EPT8, I = COLA_SCHED_PIPE_INPLACE;
  const std::vector<std::pair<int, std::vector<int>>> groups = {
      {COLA_SCHED_BINNED_DEPOSIT | COLA_SCHED_TILE_GATHER | COLA_SCHED_PIPELINED_GATHER,
       {0, COLA_SCHED_BINNED_DEPOSIT, COLA_SCHED_BINNED_DEPOSIT | COLA_SCHED_TILE_GATHER,
        COLA_SCHED_BINNED_DEPOSIT | COLA_SCHED_TILE_GATHER | COLA_SCHED_PIPELINED_GATHER}},
      {P | E | I | (3 << COLA_SCHED_BUDGET_SHIFT), {0, P, P | E, P | kB1, P | kB1 | E, P | kB2, P | kB2 | E, P | I}},
      {COLA_SCHED_GREEN_EPT8, {0, COLA_SCHED_GREEN_EPT8}},
      {COLA_SCHED_WIDE_TILES, {0, COLA_SCHED_WIDE_TILES}},
      {COLA_SCHED_C2R_EPT8 | COLA_SCHED_ROWS_PIPE,
       {0, COLA_SCHED_C2R_EPT8, COLA_SCHED_ROWS_PIPE, COLA_SCHED_C2R_EPT8 | COLA_SCHED_ROWS_PIPE}},
      {COLA_SCHED_R2C_EPT8, {0, COLA_SCHED_R2C_EPT8}}};
  int cur = keep;
  for (const auto& g : groups) {
    int arg = -1;
    float tbest = 0.0f;
    for (int opt : g.second) {
      const int sc = (cur & ~g.first) | opt;
      if (!schedule_valid(c, sc)) continue;
      const float t = time_of(sc);
      if (st != COLA_OK) break;
      if (arg < 0 || t < tbest) {
        arg = sc;
        tbest = t;
      }
    }
    if (st != COLA_OK) break;
    if (arg >= 0) cur = arg;
  }
  c->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(force);
  if (st != COLA_OK) {
    apply_schedule(c, keep);
    return -st;
  }
  apply_schedule(c, cur);
  if (best) *best = cur;
  for (size_t i = 0; i < timed.size() && (int)i < max_candidates; ++i) {
    if (scheds) scheds[i] = timed[i].first;
    if (ms) ms[i] = timed[i].second;
  }
  return (int)timed.size();
}

// ---- friends-of-friends ------------------------------------------------------------------------
namespace {

int fof_workspace(cola_ctx* c, const FofGeom& f, int capacity) {
  const long long n = c->pg.npart;
  if (!c->fof_mem || c->fof_ncells < f.ncells) {
    if (c->fof_mem) {
      COLA_TRY(cuda_status(cudaStreamSynchronize(c->stream), "fof realloc"));
      cudaFree(c->fof_mem);
      c->fof_mem = nullptr;
    }
    const long long nseg = ((n > f.ncells ? n : f.ncells) + 4095) / 4096 + 1;
    const size_t b8 = align256((size_t)n * 8), b4 = align256((size_t)(n + 1) * 4);
    const size_t bc = align256((size_t)(f.ncells + 1) * 4);
    const size_t bytes = 3 * b8 + 7 * b4 + 3 * bc + align256((size_t)nseg * 4);
    void* mem = nullptr;
    COLA_TRY(cuda_status(cudaMalloc(&mem, bytes), "cudaMalloc fof"));
    c->fof_mem = mem;
    c->fof_ncells = f.ncells;
    char* q = static_cast<char*>(mem);
    for (int a = 0; a < 3; ++a, q += b8) c->fb.g[a] = reinterpret_cast<long long*>(q);
    int** ints[3] = {&c->fb.key, &c->fb.sorted, &c->fb.parent};
    for (int i = 0; i < 3; ++i, q += b4) *ints[i] = reinterpret_cast<int*>(q);
    unsigned** uns[4] = {&c->fb.cnt, &c->fb.flag, &c->fb.hoff, &c->fb.hcur};
    for (int i = 0; i < 4; ++i, q += b4) *uns[i] = reinterpret_cast<unsigned*>(q);
    unsigned** cells[3] = {&c->fb.counts, &c->fb.off, &c->fb.cur};
    for (int i = 0; i < 3; ++i, q += bc) *cells[i] = reinterpret_cast<unsigned*>(q);
    c->fb.seg = reinterpret_cast<unsigned*>(q);
  }
  if (capacity > c->fof_sums_cap) {
    if (c->fof_sums) {
      COLA_TRY(cuda_status(cudaStreamSynchronize(c->stream), "fof realloc"));
      cudaFree(c->fof_sums);
      c->fof_sums = nullptr;
      c->fof_sums_cap = 0;
    }
    void* mem = nullptr;
    COLA_TRY(cuda_status(cudaMalloc(&mem, (size_t)3 * capacity * sizeof(unsigned long long)), "cudaMalloc fof"));
    c->fof_sums = mem;
    c->fof_sums_cap = capacity;
  }
  c->fb.sums = static_cast<unsigned long long*>(c->fof_sums);
  return COLA_OK;
}

}  // namespace

extern "C" int cola_fof(cola_ctx* c, const float* s, double b, int n_min, int* label, int* size, int* halo_label,
                        int* halo_size, double* halo_pos, int capacity, int* nhalo) {
  if (!c || !(b > 0.0) || n_min < 1 || capacity < 0 || c->pg.npart > 0x7fffffffLL) return COLA_ERR_INVALID;
  for (const void* p : {(const void*)s, (const void*)label, (const void*)size, (const void*)nhalo})
    COLA_TRY(check_ptr(p));
  for (const void* p : {(const void*)halo_label, (const void*)halo_size, (const void*)halo_pos})
    if (p) COLA_TRY(check_ptr(p));
  FofGeom f;
  if (!fof_geometry(c->p.nmesh, c->p.np, b, &f)) return COLA_ERR_INVALID;
  COLA_TRY(fof_workspace(c, f, capacity));
  return STAGED(kStFof, launch_fof(c->pg, f, s, c->fb, n_min, label, size, halo_label, halo_size, halo_pos, capacity,
                                   nhalo, c->flags, c->stream));
}

// ---- reverse mode ---------------------------------------------------------------------------
namespace {

// Adjoint work space: lam_s, lam_v, lam_Psi1, lam_Psi2, lam_F ([3][n] each) and three mesh spectra.
int adjoint_workspace(cola_ctx* c) {
  if (c->adj_mem) return COLA_OK;
  const size_t pbytes = align256((size_t)3 * c->pg.npart * sizeof(float));
  const size_t cbytes = align256(c->mesh.complex_elems() * sizeof(float2));
  void* mem = nullptr;
  COLA_TRY(cuda_status(cudaMalloc(&mem, 5 * pbytes + 3 * cbytes), "cudaMalloc adjoint"));
  c->adj_mem = mem;
  char* q = static_cast<char*>(mem);
  for (int i = 0; i < 5; ++i) c->lam[i] = reinterpret_cast<float*>(q + i * pbytes);
  for (int j = 0; j < 3; ++j) c->adj_mesh[j] = reinterpret_cast<float2*>(q + 5 * pbytes + j * cbytes);
  return COLA_OK;
}

int copy_or_zero(cola_ctx* c, float* dst, const float* src, size_t bytes) {
  if (src) return cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy");
  return cuda_status(cudaMemsetAsync(dst, 0, bytes, c->stream), "memset");
}

// Reverse pass of PM step i at checkpoint s_i: lam_s += d(lam_F . F(s_i))/ds_i.
int pm_force_adjoint(cola_ctx* c, const float* s_i, double force_scale) {
  const Grid3& g = c->mesh;
  COLA_TRY(force_mesh(c, s_i, force_scale));   // F on the mesh, cbuf[0..2]
  COLA_TRY(STAGED(kStClear, cuda_status(cudaMemsetAsync(c->adj_mesh[0], 0,
                                                        3 * align256(g.complex_elems() * sizeof(float2)), c->stream),
                                        "memset")));
  float* const m[3] = {reinterpret_cast<float*>(c->adj_mesh[0]), reinterpret_cast<float*>(c->adj_mesh[1]),
                       reinterpret_cast<float*>(c->adj_mesh[2])};
  COLA_TRY(STAGED(kStAdjoint, launch_adj_deposit(c->pg, s_i, c->lam[4], m, 2LL * g.pc, c->stream)));
  for (int j = 0; j < 3; ++j) {
    COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(c->mplan, g, kSrcFloat, c->adj_mesh[j], 2LL * g.pc, 1.0f, c->adj_mesh[j],
                                             c->stream)));
    COLA_TRY(forward3d_yx(c, g, c->mplan, c->adj_mesh[j]));
  }
  const double kf = 2.0 * M_PI / g.n;
  const double n3 = (double)g.n * g.n * g.n;
  COLA_TRY(STAGED(kStAdjoint, launch_adj_combine(g, c->adj_mesh, c->dtab, (float)(force_scale / (kf * kf * n3)),
                                                 c->adj_mesh[0], c->stream)));
  COLA_TRY(inverse3d(c, g, c->mplan, c->adj_mesh[0]));
  const float* f[3] = {reinterpret_cast<float*>(c->cbuf[0]), reinterpret_cast<float*>(c->cbuf[1]),
                       reinterpret_cast<float*>(c->cbuf[2])};
  return STAGED(kStAdjoint, launch_adj_gather(c->pg, s_i, c->lam[4], f, m[0], 2LL * g.pc,
                                              (float)(n3 / (double)c->pg.npart), c->lam[0], c->stream));
}

// Transpose of the 2LPT maps white noise -> (Psi1, Psi2) at lam_Psi1 = lam[2], lam_Psi2 = lam[3].
int lpt_adjoint(cola_ctx* c, const float* wn, float* lam_wn) {
  const LatticeScope scope(c);
  const Grid3& g = c->lat;
  const FftPlan& P = c->lplan;
  const size_t lbytes = align256(g.complex_elems() * sizeof(float2));
  float2* B[8];
  for (int i = 0; i < 8; ++i) B[i] = reinterpret_cast<float2*>(static_cast<char*>(c->arena) + i * lbytes);
  const long long n = c->pg.npart;
  const float r = (float)c->p.nmesh / (float)c->p.np;
  const float inv_n3 = (float)(1.0 / ((double)g.n * g.n * g.n));
  // delta_L(k) / np^3 as in the forward
  COLA_TRY(noise_spectrum(c, wn, B[0]));
  COLA_TRY(forward3d_yx(c, g, P, B[0]));
  COLA_TRY(STAGED(kStIc, launch_ic_amplitude(g, B[0], c->amp_m2, c->stream)));
  // lam_S = sum_j (transpose of Psi2_j = -i kodd_j / k^2 S) lam_Psi2_j
  for (int j = 0; j < 3; ++j) {
    COLA_TRY(STAGED(kStAdjoint, launch_particles_to_field(g, c->lam[3] + j * n, r, B[1], c->stream)));
    COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(P, g, kSrcFloat, B[1], 2LL * g.pc, 1.0f, B[1], c->stream)));
    COLA_TRY(forward3d_yx(c, g, P, B[1]));
    COLA_TRY(STAGED(kStIc, launch_ic_multiply(g, B[1], B[7], kIcPsi1, j, 0, inv_n3, c->stream, j > 0)));
  }
  COLA_TRY(inverse3d(c, g, P, B[7]));
  // the six Hessians, then lam_h = lam_S dS/dh in place
  const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int h = 0; h < 6; ++h) {
    COLA_TRY(STAGED(kStIc, launch_ic_multiply(g, B[0], B[1 + h], kIcHess, pairs[h][0], pairs[h][1], 1.0f, c->stream)));
    COLA_TRY(inverse3d(c, g, P, B[1 + h]));
  }
  float2* const hs[6] = {B[1], B[2], B[3], B[4], B[5], B[6]};
  COLA_TRY(STAGED(kStAdjoint, launch_ic_source_adjoint(g, B[7], hs, c->stream)));
  // acc(k) = sum_h H_h F(lam_h) + sum_j (i kodd_j / k^2)^* r F(lam_Psi1_j); lam_w = inverse(amp acc)
  for (int h = 0; h < 6; ++h) {
    COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(P, g, kSrcFloat, B[1 + h], 2LL * g.pc, 1.0f, B[1 + h], c->stream)));
    COLA_TRY(forward3d_yx(c, g, P, B[1 + h]));
    COLA_TRY(STAGED(kStIc, launch_ic_multiply(g, B[1 + h], B[0], kIcHess, pairs[h][0], pairs[h][1], 1.0f, c->stream,
                                              h > 0)));
  }
  for (int j = 0; j < 3; ++j) {
    COLA_TRY(STAGED(kStAdjoint, launch_particles_to_field(g, c->lam[2] + j * n, r, B[7], c->stream)));
    COLA_TRY(STAGED(kStFwdZ, launch_r2c_rows(P, g, kSrcFloat, B[7], 2LL * g.pc, 1.0f, B[7], c->stream)));
    COLA_TRY(forward3d_yx(c, g, P, B[7]));
    COLA_TRY(STAGED(kStIc, launch_ic_multiply(g, B[7], B[0], kIcPsi2, j, 0, 1.0f, c->stream, true)));
  }
  COLA_TRY(STAGED(kStIc, launch_ic_amplitude(g, B[0], c->amp_m2, c->stream)));
  COLA_TRY(inverse3d(c, g, P, B[0]));
  return STAGED(kStIc, launch_ic_to_particles(g, B[0], 1.0f, lam_wn, c->stream));
}

}  // namespace

extern "C" int cola_run_checkpointed(cola_ctx* c, const float* wn, float* s, float* v, float* psi1, float* psi2,
                                     float* ckpt) {
  if (!c) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(ckpt));
  const size_t pbytes = (size_t)3 * c->pg.npart * sizeof(float);
  COLA_TRY(cola_ic_2lpt(c, wn, s, v, psi1, psi2));
  for (int i = 1; i <= c->p.nstep; ++i) {
    COLA_TRY(cuda_status(cudaMemcpyAsync(reinterpret_cast<char*>(ckpt) + (i - 1) * pbytes, s, pbytes,
                                         cudaMemcpyDeviceToDevice, c->stream), "checkpoint"));
    COLA_TRY(cola_step(c, i, s, v, psi1, psi2));
  }
  return COLA_OK;
}

extern "C" int cola_adjoint(cola_ctx* c, const float* wn, const float* ckpt, const float* lam_s, const float* lam_v,
                            const float* lam_psi1, const float* lam_psi2, float* lam_wn) {
  if (!c) return COLA_ERR_INVALID;
  if (wn) COLA_TRY(check_ptr(wn));
  for (const void* p : {(const void*)ckpt, (const void*)lam_s, (const void*)lam_wn})
    COLA_TRY(check_ptr(p));
  for (const void* p : {(const void*)lam_v, (const void*)lam_psi1, (const void*)lam_psi2})
    if (p) COLA_TRY(check_ptr(p));
  COLA_TRY(adjoint_workspace(c));
  const long long n = c->pg.npart;
  const size_t pbytes = (size_t)3 * n * sizeof(float);
  COLA_TRY(copy_or_zero(c, c->lam[0], lam_s, pbytes));
  COLA_TRY(copy_or_zero(c, c->lam[1], lam_v, pbytes));
  COLA_TRY(copy_or_zero(c, c->lam[2], lam_psi1, pbytes));
  COLA_TRY(copy_or_zero(c, c->lam[3], lam_psi2, pbytes));
  for (int i = c->p.nstep; i >= 1; --i) {
    const StepScalars& ss = c->steps[i];
    COLA_TRY(STAGED(kStAdjoint, launch_adj_step(3 * n, c->lam[0], c->lam[1], c->lam[2], c->lam[3], c->lam[4], ss,
                                                c->stream)));
    const float* s_i = reinterpret_cast<const float*>(reinterpret_cast<const char*>(ckpt) + (i - 1) * pbytes);
    COLA_TRY(pm_force_adjoint(c, s_i, ss.force_scale));
  }
  const StepScalars& s0 = c->steps[0];
  COLA_TRY(STAGED(kStAdjoint, launch_adj_ic(3 * n, c->lam[0], c->lam[2], c->lam[3], (float)s0.d1, (float)s0.d2,
                                            c->stream)));
  return lpt_adjoint(c, wn, lam_wn);
}

extern "C" int cola_grid_density(cola_ctx* c, const float* s, int ngrid, float* delta) {
  if (!c || ngrid < 1 || ngrid > c->mesh.n) return COLA_ERR_INVALID;
  COLA_TRY(check_ptr(s));
  COLA_TRY(check_ptr(delta));
  return STAGED(kStAdjoint, launch_grid_density(c->pg, s, ngrid, c->rho, delta, c->stream));
}

extern "C" int cola_grid_density_adjoint(cola_ctx* c, const float* s, int ngrid, const float* lam_delta,
                                         float* lam_s) {
  if (!c || ngrid < 1 || ngrid > c->mesh.n) return COLA_ERR_INVALID;
  for (const void* p : {(const void*)s, (const void*)lam_delta, (const void*)lam_s}) COLA_TRY(check_ptr(p));
  return STAGED(kStAdjoint, launch_grid_density_adjoint(c->pg, s, ngrid, lam_delta, lam_s, c->stream));
}

extern "C" int cola_profile_enable(cola_ctx* c, int on) {
  if (!c) return COLA_ERR_INVALID;
  if (on) {
    COLA_TRY(cuda_status(cudaStreamSynchronize(c->stream), "profile sync"));
    for (auto& m : c->marks) {
      c->event_pool.push_back(m.a);
      c->event_pool.push_back(m.b);
    }
    c->marks.clear();
    for (int i = 0; i < COLA_NUM_STAGES; ++i) {
      c->stage_ms[i] = 0.0;
      c->stage_launches[i] = 0;
    }
  }
  c->prof = on != 0;
  return COLA_OK;
}

extern "C" int cola_profile_read(cola_ctx* c, double* ms, long long* launches, int nstages) {
  if (!c || nstages < 0) return -COLA_ERR_INVALID;
  if (cuda_status(cudaStreamSynchronize(c->stream), "profile read") != COLA_OK) return -COLA_ERR_CUDA;
  for (auto& m : c->marks) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, m.a, m.b);
    c->stage_ms[m.stage] += t;
    c->event_pool.push_back(m.a);
    c->event_pool.push_back(m.b);
  }
  c->marks.clear();
  for (int i = 0; i < nstages && i < COLA_NUM_STAGES; ++i) {
    if (ms) ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->stage_launches[i];
  }
  return COLA_NUM_STAGES;
}
