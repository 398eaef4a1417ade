// Internal declarations shared by the library's translation units (host-visible only).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "../../include/cola.h"

namespace cola {

double hubble(double a, double om);

// FP64 background cosmology and linear power (host only).
struct Cosmo {
  double om, h, ns, sigma8;
  double i1 = 0.0;   // growth integral at a = 1
  double amp = 0.0;  // P(k) amplitude A from sigma8
  Cosmo(double om, double h, double ns, double sigma8);
  double transfer(double k) const;
  double power(double k) const;
  double omega_a(double a) const;
  double d1(double a) const;
  double d1_da(double a) const;
  double d2(double a) const;
  double d2_da(double a) const;
  double drift(double a0, double a1, double ahalf, double nlpt, int ansatz) const;
  double kick(double alo, double ahi, double ai, double nlpt) const;
};

struct StepScalars {
  double a, a_lo, a_hi, force_scale, c1, c2, kick, drift, dd1, dd2, d1, d2;
};

StepScalars step_scalars(const cola_params& p, const Cosmo& c, int i);

// ---------------------------------------------------------------------------------------------
// FFT plan: one transform length, its radix stages and the twiddle table exp(-2 pi i t / n).
// ---------------------------------------------------------------------------------------------
constexpr int kMaxStages = 12;

struct FftDev {
  int n;
  int nstages;
  int radix[kMaxStages];
  const float2* tw;   // device table, n entries
};

struct FftPlan {
  FftDev dev{};
  float2* tw = nullptr;   // owned device memory
  // padded shared-tile row steps of each stage along n/R and along ns (0: padding not affine),
  // computed once by fft_plan_init for the fast-path kernels
  int nbp[kMaxStages] = {};
  int nsp[kMaxStages] = {};
  int w_pencil = 8;       // pencils per CTA in the strided passes
  int w_rows = 4;         // row pairs per CTA in the contiguous (R2C / C2R) passes
  int ept = 16;           // complex elements per thread
  // schedule (chosen by cola_set_schedule / cola_autotune): persistent pipelined strided passes
  // on/off, and their shared-memory budget per CTA (sets the tile width)
  bool pipe = true;
  int pipe_kb = 160;
  int pipe_ept = 16;      // complex elements per thread of the pipelined passes (16 or 8)
  int green_ept = 16;     // complex elements per thread of the Green pass (16 or 8)
  int row_ept = 16;       // complex elements per thread of the C2R row passes (16 or 8)
  int r2c_ept = 16;       // complex elements per thread of the R2C row pass (16 or 8)
  bool row_pipe = false;  // persistent C2R passes with a staging buffer for the next tile
  bool wide = true;       // tiles of 8 pencils in the one-CTA-per-tile strided and Green passes
  bool pipe_inplace = false;  // pipelined passes: one work buffer overwritten in place, 210 KB budget
};

// Factor n into radices {16, 8, 5, 4, 3, 2}; returns false if n has another prime factor.
bool fft_factor(int n, std::vector<int>* radices);
int fft_plan_init(FftPlan* plan, int n);   // allocates the twiddle table; returns cola_status
void fft_plan_steps(FftPlan* plan);        // fills nbp / nsp from dev.n and dev.radix (host only)
void fft_plan_free(FftPlan* plan);
void fft_set_smem_limits();                // raise the dynamic shared-memory limit of the FFT kernels

// True the first time it is called for `key` on the current device (thread safe).  Kernel attributes
// (the dynamic shared-memory limit) are per device, so every setter is keyed by (device, kernel).
bool first_use_on_device(const void* key);

// Geometry of a 3D field of side n in the in-place real-to-complex layout:
// complex rows of pc = (n/2+1 rounded up to even) entries, real rows of 2*pc floats.
struct Grid3 {
  int n;
  int nc;            // n/2 + 1 valid complex entries per row
  int pc;            // padded complex row length
  size_t rows() const { return (size_t)n * n; }
  size_t complex_elems() const { return rows() * pc; }
};

// Sources of the contiguous-axis forward transform.
enum RowSource { kSrcFixedPoint = 0, kSrcFloat = 1 };

// Launchers (fft.cu).  All take the stream explicitly.
// Forward R2C along z of n^2 rows; src is uint64 (scaled: value*scale - 1) or float rows with
// the given row stride (floats or uint64 elements).  dst: complex grid rows of stride pc.
int launch_r2c_rows(const FftPlan& p, const Grid3& g, RowSource kind, const void* src,
                    long long src_row_stride, float scale, float2* dst, cudaStream_t st,
                    unsigned long long* mass_acc = nullptr);
// Inverse C2R along z, in place on a complex grid (real rows of stride 2*pc floats).
int launch_c2r_rows(const FftPlan& p, const Grid3& g, float2* data, cudaStream_t st);
// The C2R rows of data (not modified) written to out as dense rows of n floats times scale, where the
// plan has a specialised kernel for it (c2r_rows_dense_ok); the same floats as launch_c2r_rows then
// launch_ic_to_particles.
bool c2r_rows_dense_ok(const FftPlan& p, const Grid3& g);
// The inverse x pass of mul times the lattice spectrum src into dst (src unchanged) where the plan has
// a specialised in-place pipelined kernel for it (pencils_x_mul_ok); the same floats as
// launch_ic_multiply followed by launch_pencils(axis 0, +1).
struct IcMul;
bool pencils_x_mul_ok(const FftPlan& p, const Grid3& g);
int launch_pencils_x_mul(const FftPlan& p, const Grid3& g, const float2* src, const IcMul& mul, float2* dst,
                         cudaStream_t st);
int launch_c2r_rows_dense(const FftPlan& p, const Grid3& g, const float2* data, float scale, float* out,
                          cudaStream_t st);
// C2C along y (axis 1) or x (axis 0) of the complex grid; dir = -1 forward, +1 inverse.
int launch_pencils(const FftPlan& p, const Grid3& g, int axis, int dir, float2* data,
                   cudaStream_t st);
// Forward x transform, then for each j in {x, y, z}: out_j = i D(k_j) scale delta(k)/k^2
// (k in rad/cell, D the 4-point gradient kernel), then the inverse x transform of out_j.
// out[2] may alias in.  With spec_out (a complex grid that aliases none of the others) the fast
// kernels also write the forward spectrum delta(k) there and set *spec_saved.
int launch_green_x(const FftPlan& p, const Grid3& g, const float2* in, float2* const out[3],
                   const float* dtab, float scale, cudaStream_t st, float2* spec_out = nullptr,
                   bool* spec_saved = nullptr);

// Launchers (particles.cu).
struct ParticleGeom {
  int np;             // particles per side
  int n;              // mesh cells per side
  long long r_fixed;  // (n/np) * 2^20
  long long npart;    // np^3
};

int launch_deposit(const ParticleGeom& pg, const float* s, unsigned long long* rho, int* flags,
                   cudaStream_t st);
// Sets flags bit 0 if the 128-bit total in acc (accumulated by the fixed-point R2C pass, or by
// summing rho here when sum_mesh) differs from n 2^42, i.e. if some cell wrapped; resets acc.
int launch_mass_check(const ParticleGeom& pg, const unsigned long long* rho, bool sum_mesh, unsigned long long* acc,
                      int* flags, cudaStream_t st);
// Adds the 128-bit sum of m (lo, hi) pairs to the accumulator acc (kMassSlots pairs).
int launch_mass_reduce(const unsigned long long* pairs, long long m, unsigned long long* acc, cudaStream_t st);

// Fixed-point particle coordinates shared by the deposit, the gathers, the adjoint and FoF: a
// particle at lattice index q (per axis) and displacement s (mesh cells) sits at
// G = (q R + rint(s 2^20)) mod N 2^20, R = (N/np) 2^20; its cell is G >> 20 and its 14-bit CIC
// weight fraction (G >> 6) & (2^14 - 1).  Every kernel must take the same integers, which makes the
// deposit bit-exact and the interpolation use the deposit's own weights.
constexpr int kFracBits = 20;
constexpr long long kFracOne = 1LL << kFracBits;
constexpr int kWeightOne = 1 << 14;

#ifdef __CUDACC__
// G of one axis.  A NaN or huge s wraps into [0, modulus) (the final % catches what one
// conditional add cannot), so no kernel can index outside the mesh.
__device__ __forceinline__ long long fixed_coord(int q, float s, long long r_fixed, long long modulus) {
  long long g = (long long)q * r_fixed + __float2ll_rn(s * (float)kFracOne);
  if (g < 0) g += modulus;
  else if (g >= modulus) g -= modulus;
  if ((unsigned long long)g >= (unsigned long long)modulus) {
    g %= modulus;
    if (g < 0) g += modulus;
  }
  return g;
}

// The same G with 32-bit integer arithmetic where that is exact, else fixed_coord.  |s| < lim cells
// with lim = min(N, 2047 - N) keeps q R + rint(s 2^20) inside (-N 2^20, 2047 2^20) (no int32
// overflow) and one conditional add or subtract from [0, N 2^20); s 2^20 is exact in FP32 (a power of
// two scaling) and fits an int32, so its round-to-nearest-even is the one fixed_coord takes.  NaN and
// infinite s fail the test and take fixed_coord: the result is bit-identical for every input.
struct FixedGeo {
  long long r_fixed, modulus;
  float lim;   // 0 when N >= 1024 + 1023 (no 32-bit fast path)
};
__host__ __device__ __forceinline__ FixedGeo fixed_geo(int nmesh, long long r_fixed) {
  const int room = 2047 - nmesh;
  const int lim = room < nmesh ? room : nmesh;
  return FixedGeo{r_fixed, (long long)nmesh << kFracBits, lim > 0 ? (float)lim : 0.0f};
}
// Cell G >> 20 and 14-bit weight fraction (G >> 6) & (2^14 - 1) of one axis.  F32 (meshes below
// 2048 cells, where every G fits an int) takes the 32-bit path when |s| < lim.
template <bool F32>
__device__ __forceinline__ void cell_frac(int q, float s, const FixedGeo& f, int* cell, int* frac) {
  if (F32) {
    int g;
    if (fabsf(s) < f.lim) {
      const int m = (int)f.modulus;
      g = q * (int)f.r_fixed + __float2int_rn(s * (float)kFracOne);
      if (g < 0) g += m;
      else if (g >= m) g -= m;
    } else {
      g = (int)fixed_coord(q, s, f.r_fixed, f.modulus);
    }
    *cell = g >> kFracBits;
    *frac = (g >> (kFracBits - 14)) & (kWeightOne - 1);
  } else {
    const long long g = fixed_coord(q, s, f.r_fixed, f.modulus);
    *cell = (int)(g >> kFracBits);
    *frac = (int)((g >> (kFracBits - 14)) & (kWeightOne - 1));
  }
}
#endif

#ifdef __CUDACC__
// Density contrast of one fixed-point mesh cell, delta = rho scale - 1 (scale = N^3 / (n 2^42)), the
// same float in every kernel that forms it (the tile deposit, the R2C passes, the generic FFT): rho
// is converted as hi 2^32 + lo with two exact-range 32-bit conversions and one fused multiply-add
// (FP32 units only; a 64-bit integer conversion runs on GB300's few FP64 units), then one more FMA.
__device__ __forceinline__ float fixed_to_delta(unsigned long long v, float scale) {
  const float f = __fmaf_rn(__uint2float_rn((unsigned)(v >> 32)), 4294967296.0f, __uint2float_rn((unsigned)v));
  return __fmaf_rn(f, scale, -1.0f);
}

// The 128-bit mass accumulator is kMassSlots (lo, hi) pairs, one chosen per CTA, so that the atomics of
// many CTAs do not all land on one address; launch_mass_check sums the slots.
constexpr int kMassSlots = 128;
__device__ __forceinline__ unsigned long long* mass_slot(unsigned long long* acc) {
  return acc + 2 * (blockIdx.x & (kMassSlots - 1));
}

// Adds a thread's 128-bit partial (lo, hi) to the accumulator pair acc[0..1] (exact, any order).
// Called by every thread of full warps.
__device__ __forceinline__ void mass_accumulate(unsigned long long lo, unsigned long long hi, unsigned long long* acc) {
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, off);
    const unsigned long long ohi = __shfl_down_sync(0xffffffffu, hi, off);
    lo += olo;
    hi += ohi + (lo < olo);
  }
  if ((threadIdx.x & 31) == 0 && (lo | hi)) {
    const unsigned long long old = atomicAdd(acc, lo);
    atomicAdd(acc + 1, hi + (old + lo < old));
  }
}
#endif
struct KickDrift {
  float kick, drift, dd1, dd2, c1, c2;
};
// Interpolates the three real force fields (rows of stride rs floats) at the particles; with
// kd == nullptr writes the force to out[3][n], else applies the COLA kick and drift in place.
int launch_gather(const ParticleGeom& pg, const float* const f[3], long long rs, const float* s_in,
                  float* force_out, float* s, float* v, const float* psi1, const float* psi2,
                  const KickDrift* kd, int* flags, cudaStream_t st);

// Spatial binning by tiles of T x T mesh columns (binning.cu).
struct BinGeom {
  int lt;      // log2 T (tile side across z)
  int lz;      // log2 TZ (tile length along z)
  int nt;      // tiles per axis across z (N / T)
  int nz;      // tiles along z (N / TZ)
  int tiles;   // nt^2 nz
};
struct BinBuffers {
  unsigned *cnt_p = nullptr, *cnt_s = nullptr;   // counts per tile (primary, spill)
  unsigned *off_p = nullptr, *off_s = nullptr;   // offsets, tiles + 1
  unsigned *cur_p = nullptr, *cur_s = nullptr;   // scatter cursors
  unsigned *ent_p = nullptr, *ent_s = nullptr;   // packed lattice coordinates (n primary, up to 7n spill)
  unsigned* seg = nullptr;                        // scan segment sums (2 lists)
  unsigned long long* rec = nullptr;              // [n] rank in the primary tile << 32 | flags << 26 | tile
};
bool bin_geometry(int nmesh, int np, BinGeom* b);
size_t bin_smem_bytes(const BinGeom& b, int nmesh);
bool tile_gather_pays(const BinGeom& b, long long npart);   // else gather in lattice order
int launch_binning(const ParticleGeom& pg, const BinGeom& b, const float* s, BinBuffers& bb, cudaStream_t st);
// delta_out == nullptr: writes the fixed-point mesh rho.  Else writes the density contrast
// fixed_to_delta(rho, scale) as dense float rows to delta_out (rho is not written) and each tile's
// exact 128-bit total to tile_mass[2 tile .. 2 tile + 1] (for launch_mass_reduce).
int launch_deposit_tiles(const ParticleGeom& pg, const BinGeom& b, const float* s, const BinBuffers& bb,
                         unsigned long long* rho, cudaStream_t st, float* delta_out = nullptr, float scale = 0.0f,
                         unsigned long long* tile_mass = nullptr);
int launch_gather_tiles(const ParticleGeom& pg, const BinGeom& b, const BinBuffers& bb, const float* const f[3],
                        long long rs, const float* s_in, float* force_out, float* s, float* v, const float* psi1,
                        const float* psi2, const KickDrift* kd, int* flags, cudaStream_t st,
                        bool pipelined = false);

// 2LPT helpers on the lattice grid (side np).
enum IcField { kIcPsi1 = 0, kIcHess = 1, kIcPsi2 = 2 };
// One 2LPT spectral multiply: field kind, components ci, cj and a scale (see ic_multiply_mode).
struct IcMul {
  int kind, ci, cj;
  float scale;
};
#ifdef __CUDACC__
__device__ __forceinline__ int signed_mode(int i, int n) { return i < n / 2 ? i : i - n; }
// The 2LPT multiplier of mode m (integer wave numbers, m[2] >= 0) applied to z: Psi1_j = i k_j / k^2,
// Psi2_j = -i k_j / k^2 (times scale), Hessian_ij = k_i k_j / k^2; the Nyquist plane of an odd
// derivative is zeroed and k = 0 gives 0.  One definition for the multiply kernel and the inverse
// pass that fuses it, so both compute the same floats.
__device__ __forceinline__ float2 ic_multiply_mode(float2 z, const int (&m)[3], int n, const IcMul& mp) {
  const float kf = 6.283185307179586f / n;
  const float m2 = (float)m[0] * m[0] + (float)m[1] * m[1] + (float)m[2] * m[2];
  float2 out = make_float2(0.f, 0.f);
  if (m2 > 0.f) {
    const float inv_k2 = 1.0f / (m2 * kf * kf);
    const int nyq = n / 2;
    const float koi = (m[mp.ci] == nyq || m[mp.ci] == -nyq) ? 0.f : m[mp.ci] * kf;
    if (mp.kind == kIcPsi1) {
      const float c = koi * inv_k2 * mp.scale;   // i c z
      out = make_float2(-c * z.y, c * z.x);
    } else if (mp.kind == kIcPsi2) {
      const float c = -koi * inv_k2 * mp.scale;
      out = make_float2(-c * z.y, c * z.x);
    } else {
      float kk;
      if (mp.ci == mp.cj) kk = (m[mp.ci] * kf) * (m[mp.ci] * kf);
      else {
        const float koj = (m[mp.cj] == nyq || m[mp.cj] == -nyq) ? 0.f : m[mp.cj] * kf;
        kk = koi * koj;
      }
      const float c = kk * inv_k2 * mp.scale;
      out = make_float2(c * z.x, c * z.y);
    }
  }
  return out;
}
#endif
int launch_ic_amplitude(const Grid3& g, float2* wk, const float* amp_m2, cudaStream_t st);
int launch_ic_multiply(const Grid3& g, const float2* src, float2* dst, IcField kind, int i, int j,
                       float scale, cudaStream_t st, bool accumulate = false);
int launch_ic_source(const Grid3& g, float2* const h[6], float2* dst, cudaStream_t st);
int launch_ic_to_particles(const Grid3& g, const float2* field, float scale, float* dst,
                           cudaStream_t st);
int launch_ic_positions(long long npart, const float* psi1, const float* psi2, float d1, float d2,
                        float* s, float* v, cudaStream_t st);

// Seeded white noise (rng.cu): Philox-4x32-10 keyed by the seed, Box-Muller, one Gaussian per lattice
// site written to out[row * row_stride + iz]; and the raw words of counters first .. first+count-1.
int launch_white_noise(unsigned long long seed, int np, long long row_stride, float* out, cudaStream_t st);
int launch_philox_words(unsigned long long seed, long long first, long long count, unsigned* out, cudaStream_t st);

// Adjoint (adjoint.cu).
int launch_adj_step(long long n3, const float* lam_s, float* lam_v, float* lam_p1, float* lam_p2, float* lam_f,
                    const StepScalars& sc, cudaStream_t st);
int launch_adj_deposit(const ParticleGeom& pg, const float* s, const float* lam_f, float* const m[3], long long rs,
                       cudaStream_t st);
int launch_adj_combine(const Grid3& g, float2* const l[3], const float* dtab, float g_scale, float2* out,
                       cudaStream_t st);
int launch_adj_gather(const ParticleGeom& pg, const float* s, const float* lam_f, const float* const f[3],
                      const float* lam_delta, long long rs, float norm, float* lam_s, cudaStream_t st);
int launch_adj_ic(long long n3, const float* lam_s, float* lam_p1, float* lam_p2, float d1, float d2, cudaStream_t st);
int launch_particles_to_field(const Grid3& g, const float* src, float scale, float2* dst, cudaStream_t st);
int launch_ic_source_adjoint(const Grid3& g, const float2* lam_src, float2* const h[6], cudaStream_t st);
int launch_grid_density(const ParticleGeom& pg, const float* s, int ngrid, unsigned long long* scratch, float* delta,
                        cudaStream_t st);
int launch_grid_density_adjoint(const ParticleGeom& pg, const float* s, int ngrid, const float* lam_delta,
                                float* lam_s, cudaStream_t st);

// Snapshot between force times: s_out = s + alpha v + b1 psi1 + b2 psi2; v_out = v + g1 psi1 + g2 psi2
// (v_out may be null).
int launch_snapshot(long long npart, const float* s, const float* v, const float* psi1, const float* psi2, float alpha,
                    float b1, float b2, float g1, float g2, float* s_out, float* v_out, cudaStream_t st);

// Friends-of-friends (fof.cu): geometry of the cell search and work buffers.
struct FofGeom {
  long long modulus = 0;   // N 2^20
  long long ell = 0;       // linking length in fixed-point units
  long long ncells = 0;    // ncs^3
  int ncs = 0;             // cells per axis, side >= ell
};
struct FofBuffers {
  long long* g[3] = {nullptr, nullptr, nullptr};   // fixed-point coordinates [n] per axis
  int* key = nullptr;                              // cell of each particle
  int* sorted = nullptr;                           // particle ids sorted by cell
  int* parent = nullptr;                           // union-find forest
  unsigned* cnt = nullptr;                         // members per root
  unsigned* flag = nullptr;                        // 1 for roots of haloes
  unsigned* hoff = nullptr;                        // [n + 1] halo index of each root
  unsigned* hcur = nullptr;
  unsigned* counts = nullptr;                      // [ncells] particles per cell
  unsigned* off = nullptr;                         // [ncells + 1]
  unsigned* cur = nullptr;
  unsigned* seg = nullptr;                         // scan segment sums
  unsigned long long* sums = nullptr;              // [3][capacity] offset sums of the haloes
};
bool fof_geometry(int nmesh, int np, double b, FofGeom* f);
int launch_fof(const ParticleGeom& pg, const FofGeom& f, const float* s, const FofBuffers& fb, int n_min, int* label,
               int* size, int* halo_label, int* halo_size, double* halo_pos, int capacity, int* nhalo, int* flags,
               cudaStream_t st);
// Exclusive scan of m counts into off[0..m] and a copy cur[0..m) (binning.cu); seg holds
// ceil(m / 4096) partial sums.
int launch_excl_scan(const unsigned* cnt, int m, unsigned* seg, unsigned* off, unsigned* cur, cudaStream_t st);

// Power spectrum binning of a forward spectrum (side n).  launch_pk_geometry writes the bins' sum of
// |m| and mode count (they depend only on n and the edges) to geom[2][nbins]; launch_pk_bins sums the
// modes' power (over C2 when cic_correct) into partials[nblocks][nbins]; launch_pk_finish combines
// them into pk[3][nbins] (mean |k| = kfund mean |m|, P = pscale mean power - shot, counts).
// partials holds 2 nblocks nbins doubles (the geometry pass uses both halves).
int launch_pk_geometry(const Grid3& g, const long long* edges, int nbins, double* partials, int nblocks,
                       double* geom, cudaStream_t st);
int launch_pk_bins(const Grid3& g, const float2* dk, const long long* edges, int nbins, int cic_correct,
                   double* partials, int nblocks, cudaStream_t st);
int launch_pk_finish(const double* partials, int nblocks, int nbins, const double* geom, double kfund, double pscale,
                     double shot, double* pk, cudaStream_t st);
int launch_dense_spectrum(const Grid3& g, const float2* src, float* dst, cudaStream_t st);
// out[3][m] = the three real force fields f (rows of 2 pc floats) at mesh cells (ix N + iy) N + iz.
int launch_sample_mesh(const Grid3& g, const float* const f[3], const long long* cells, long long m, float* out,
                       cudaStream_t st);

}  // namespace cola

// The context (cola_abi.cu).
struct cola_ctx {
  cola_params p;
  cudaStream_t stream = nullptr;
  cola::Grid3 mesh{}, lat{};
  cola::FftPlan mplan, lplan;
  cola::ParticleGeom pg{};
  std::vector<cola::StepScalars> steps;   // index 1..nstep; [0] holds initial-condition scalars
  double vel_f1 = 0.0, vel_f2 = 0.0;      // a^2 dD/dt at a = 1
  // device memory
  void* arena = nullptr;                  // meshes (and the IC work space, aliased)
  size_t arena_bytes = 0;
  unsigned long long* rho = nullptr;      // [N^3]
  float2* cbuf[3] = {nullptr, nullptr, nullptr};   // complex N x N x pc each
  float* dtab = nullptr;                  // gradient kernel per storage index, N entries
  float* amp_m2 = nullptr;                // sqrt(P(k)/V_cell) per integer m^2 of the lattice
  long long* edges = nullptr;             // P(k) bin edges in m^2 (device), up to 129
  long long* edges_host = nullptr;        // pinned host copy of the current edges
  int edges_nbins = 0;
  double* pk_partials = nullptr;
  int pk_blocks = 0;
  double* pk_geom = nullptr;              // [2][nbins]: sum of |m| and mode count per bin
  int pk_geom_nbins = 0;                  // bins the geometry was computed for (0: none yet)
  bool spec_saved = false;                // the last force evaluation left delta(k) in the rho buffer
  int* flags = nullptr;                   // sticky device error flags
  unsigned long long* mass_acc = nullptr; // 128-bit total of the fixed-point mesh (overflow check)
  unsigned long long* tile_mass = nullptr;  // [tiles][2] 128-bit totals of the tile deposit
  bool binned = false;                    // tile-wise deposit (else direct atomics)
  bool tile_gather = false;               // tile-wise gather from shared memory (else lattice order)
  bool gather_pipe = false;               // ... by persistent CTAs that stage the next tile meanwhile
  cola::BinGeom bg{};
  cola::BinBuffers bb;
  void* bin_mem = nullptr;
  // measurement support
  bool prof = false;
  bool lattice_fft = false;   // the 2LPT lattice transforms are running (their own stage)
  double stage_ms[COLA_NUM_STAGES] = {};
  long long stage_launches[COLA_NUM_STAGES] = {};
  struct Mark { int stage; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  // adjoint work space (allocated by the first cola_adjoint call)
  void* adj_mem = nullptr;
  float* lam[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // lam_s, lam_v, lam_psi1, lam_psi2, lam_F
  float2* adj_mesh[3] = {nullptr, nullptr, nullptr};
  // friends-of-friends work space (allocated by cola_fof, grown when a call needs more)
  void* fof_mem = nullptr;
  long long fof_ncells = 0;                // cell capacity of fof_mem
  void* fof_sums = nullptr;
  int fof_sums_cap = 0;
  cola::FofBuffers fb;
};
