// Particle-side kernels of the COLA step (sm_103a): CIC deposit, CIC gather fused with the COLA
// kick and drift, the 2LPT initial-condition helpers, and the power-spectrum binning.
//
//   deposit ............ §2.3 PM mesh, §3.3 CIC; deterministic 64-bit fixed point (exact sums)
//   gather/kick/drift .. §2.1 residual force F_res = F - F_2LPT; §2.2 eqs. (cola-kick), (cola-drift)
//   2LPT ............... §2.1 growing mode x = q + D1 Psi1 + D2 Psi2; §2.3 2LPTic-style fields
//   P(k) ............... §3.3 half-space modes and bin averages
#include "cola_internal.h"

#include <cstdio>

namespace cola {
namespace {


int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "cola: launch of %s failed: %s\n", what, cudaGetErrorString(e));
    return COLA_ERR_CUDA;
  }
  return COLA_OK;
}

unsigned grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  const long long cap = 152LL * 16 * 4;   // enough resident CTAs; kernels grid-stride beyond it
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

// Particles are processed by lattice rows: blockIdx.x (grid-stride) indexes the row (qx, qy) and
// the threads walk qz, so the lattice index needs one division per row and none per particle.
constexpr int kRowThreads = 256;

__global__ void __launch_bounds__(kRowThreads) k_deposit(ParticleGeom pg, const float* __restrict__ s,
                                                        unsigned long long* rho) {
  const long long n = pg.npart;
  const long long modulus = (long long)pg.n << kFracBits;
  const int nm = pg.n, np = pg.np;
  const long long nrows = (long long)np * np;
  for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int qx = (int)(row / np), qy = (int)(row - (long long)qx * np);
    for (int qz = threadIdx.x; qz < np; qz += blockDim.x) {
      const long long id = row * np + qz;
      const int q[3] = {qx, qy, qz};
      int c[3];
      unsigned long long w1[3], w0[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long g = fixed_coord(q[a], __ldg(s + a * n + id), pg.r_fixed, modulus);
        c[a] = (int)(g >> kFracBits);
        w1[a] = (unsigned long long)((g >> (kFracBits - 14)) & (kWeightOne - 1));
        w0[a] = kWeightOne - w1[a];
      }
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int ix = (c[0] + dx) == nm ? 0 : c[0] + dx;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int iy = (c[1] + dy) == nm ? 0 : c[1] + dy;
          const unsigned long long wxy = (dx ? w1[0] : w0[0]) * (dy ? w1[1] : w0[1]);
          unsigned long long* rrow = rho + ((long long)ix * nm + iy) * nm;
#pragma unroll
          for (int dz = 0; dz < 2; ++dz) {
            const int iz = (c[2] + dz) == nm ? 0 : c[2] + dz;
            const unsigned long long w = wxy * (dz ? w1[2] : w0[2]);
            if (w) atomicAdd(rrow + iz, w);   // result unused: compiles to a reduction (no return trip)
          }
        }
      }
    }
  }
}

// CIC gather of the three force fields, optionally fused with the COLA kick and drift.
template <bool KICK>
__global__ void __launch_bounds__(kRowThreads) k_gather(ParticleGeom pg, const float* __restrict__ f0,
                                                       const float* __restrict__ f1, const float* __restrict__ f2,
                                                       long long rs, const float* __restrict__ s_in,
                                                       float* __restrict__ force_out, float* s, float* v,
                                                       const float* __restrict__ psi1,
                                                       const float* __restrict__ psi2, KickDrift kd, int* flags) {
  const long long n = pg.npart;
  const long long modulus = (long long)pg.n << kFracBits;
  const int nm = pg.n, np = pg.np;
  const long long nrows = (long long)np * np;
  const float inv_one = 1.0f / kWeightOne;
  bool bad = false;
  for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int qx = (int)(row / np), qy = (int)(row - (long long)qx * np);
#pragma unroll 2
    for (int qz = threadIdx.x; qz < np; qz += blockDim.x) {
      const long long id = row * np + qz;
      const int q[3] = {qx, qy, qz};
      const float* sp = KICK ? s : s_in;
      float sv[3];
      int c[3];
      float w1[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sv[a] = sp[a * n + id];
        const long long g = fixed_coord(q[a], sv[a], pg.r_fixed, modulus);
        c[a] = (int)(g >> kFracBits);
        w1[a] = (float)((int)(g >> (kFracBits - 14)) & (kWeightOne - 1)) * inv_one;
      }
      float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int ix = (c[0] + dx) == nm ? 0 : c[0] + dx;
        const float wx = dx ? w1[0] : 1.0f - w1[0];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int iy = (c[1] + dy) == nm ? 0 : c[1] + dy;
          const float wxy = wx * (dy ? w1[1] : 1.0f - w1[1]);
          const long long rbase = ((long long)ix * nm + iy) * rs;
          const int iz0 = c[2], iz1 = (c[2] + 1) == nm ? 0 : c[2] + 1;
          const float wz1 = w1[2], wz0 = 1.0f - w1[2];
          fx += wxy * (wz0 * __ldg(f0 + rbase + iz0) + wz1 * __ldg(f0 + rbase + iz1));
          fy += wxy * (wz0 * __ldg(f1 + rbase + iz0) + wz1 * __ldg(f1 + rbase + iz1));
          fz += wxy * (wz0 * __ldg(f2 + rbase + iz0) + wz1 * __ldg(f2 + rbase + iz1));
        }
      }
      if (!KICK) {
        force_out[id] = fx;
        force_out[n + id] = fy;
        force_out[2 * n + id] = fz;
      } else {
        const float fp[3] = {fx, fy, fz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float p1 = __ldg(psi1 + a * n + id), p2 = __ldg(psi2 + a * n + id);
          const float fres = fp[a] - (kd.c1 * p1 + kd.c2 * p2);
          const float vn = v[a * n + id] + kd.kick * fres;
          const float sn = sv[a] + kd.drift * vn + kd.dd1 * p1 + kd.dd2 * p2;
          v[a * n + id] = vn;
          s[a * n + id] = sn;
          bad |= !isfinite(vn) || !isfinite(sn);
        }
      }
    }
  }
  if (KICK && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 2);
}

// Exact overflow check of a fixed-point mesh: the 128-bit sum of the (possibly wrapped) cells
// equals n 2^42 exactly unless some cell wrapped past 2^64 (each wrap removes 2^64).
__global__ void k_mass_check(const unsigned long long* __restrict__ acc, unsigned long long expect_lo,
                             unsigned long long expect_hi, unsigned long long* acc_reset, int* flags) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long lo = 0ULL, hi = 0ULL;
    for (int k = 0; k < kMassSlots; ++k) {
      const unsigned long long l = acc[2 * k];
      lo += l;
      hi += acc[2 * k + 1] + (lo < l);
    }
    if (lo != expect_lo || hi != expect_hi) atomicOr(flags, 1);
    for (int k = 0; k < 2 * kMassSlots; ++k) acc_reset[k] = 0ULL;
  }
}

__global__ void k_mesh_sum(const unsigned long long* __restrict__ rho, long long cells, unsigned long long* acc) {
  unsigned long long lo = 0, hi = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long v = rho[i];
    lo += v;
    hi += (lo < v);
  }
  mass_accumulate(lo, hi, mass_slot(acc));
}

// ---- 2LPT helpers on the lattice grid (side n = np, half spectrum rows of pc) --------------

__global__ void k_ic_amplitude(int n, int pc, int nc, float2* wk, const float* __restrict__ amp_m2) {
  const long long total = (long long)n * n * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(t % nc);
    const long long row = t / nc;
    const int my = signed_mode((int)(row % n), n), mx = signed_mode((int)(row / n), n);
    const long long m2 = (long long)mx * mx + (long long)my * my + (long long)kz * kz;
    float2 z = wk[row * pc + kz];
    const float a = amp_m2[m2];
    wk[row * pc + kz] = make_float2(z.x * a, z.y * a);
  }
}

// dst(k) = M(k) src(k): Psi1 component i: i kodd_i / k^2; Hessian (i, j): k_i k_j / k^2 (diagonal
// uses the full k_i, off-diagonal the Nyquist-zeroed kodd); Psi2 component i: -i kodd_i / k^2.
// k in radians per lattice spacing, times 'scale'.
__global__ void k_ic_multiply(int n, int pc, int nc, const float2* __restrict__ src, float2* dst, IcMul mp,
                              int accumulate) {
  const long long total = (long long)n * n * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(t % nc);
    const long long row = t / nc;
    const int m[3] = {signed_mode((int)(row / n), n), signed_mode((int)(row % n), n), kz};
    float2 out = ic_multiply_mode(src[row * pc + kz], m, n, mp);
    if (accumulate) {
      const float2 o = dst[row * pc + kz];
      out = make_float2(out.x + o.x, out.y + o.y);
    }
    dst[row * pc + kz] = out;
  }
}

// S = h00 h11 + h00 h22 + h11 h22 - h01^2 - h02^2 - h12^2 on real rows of stride 2 pc.
__global__ void k_ic_source(int n, int pc, const float* __restrict__ h0, const float* __restrict__ h1,
                            const float* __restrict__ h2, const float* __restrict__ h3,
                            const float* __restrict__ h4, const float* __restrict__ h5, float* dst) {
  const long long total = (long long)n * n * n;
  const long long rs = 2LL * pc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = (t / n) * rs + (t % n);
    const float a = h0[i], b = h1[i], c = h2[i], d = h3[i], e = h4[i], f = h5[i];
    dst[i] = a * b + a * c + b * c - d * d - e * e - f * f;
  }
}

__global__ void k_ic_to_particles(int n, int pc, const float* __restrict__ field, float scale, float* dst) {
  const long long total = (long long)n * n * n;
  const long long rs = 2LL * pc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = field[(t / n) * rs + (t % n)] * scale;
}

__global__ void k_ic_positions(long long n3, const float* __restrict__ psi1, const float* __restrict__ psi2,
                               float d1, float d2, float* s, float* v) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    s[t] = d1 * psi1[t] + d2 * psi2[t];
    v[t] = 0.0f;
  }
}

// s_out = s + alpha v + b1 psi1 + b2 psi2;  v_out = v + g1 psi1 + g2 psi2   (all [3][n])
__global__ void k_snapshot(long long n3, const float* __restrict__ s, const float* __restrict__ v,
                           const float* __restrict__ psi1, const float* __restrict__ psi2, float alpha, float b1,
                           float b2, float g1, float g2, float* s_out, float* v_out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const float p1 = psi1[t], p2 = psi2[t], vv = v[t];
    s_out[t] = s[t] + alpha * vv + b1 * p1 + b2 * p2;
    if (v_out) v_out[t] = vv + g1 * p1 + g2 * p2;
  }
}

// ---- power spectrum ------------------------------------------------------------------------
constexpr int kPkThreads = 256;
constexpr int kPkWarps = kPkThreads / 32;
constexpr int kMaxBins = 128;

// Each warp walks whole k_z rows; along a row |m|^2 grows with k_z, so equal bins are contiguous
// runs of lanes.  A segmented scan in a fixed shuffle order sums each run, whose last lane adds it
// to the warp's own histogram; warps and blocks are then summed in index order, so the reduction
// order is fixed and the result is bit-reproducible.
//
// The work is split in two.  The bins' geometry (mode count and sum of |m|, exact integers and
// FP64 square roots) depends only on the mesh and the bin edges: k_pk_geometry computes it once per
// context and bin count.  The per-call pass k_pk_power only sums |delta_k|^2 (over C2 with
// cic_correct): FP32 within a warp's run of at most 32 modes, FP64 from the run on.  GB300 has few
// FP64 units, so the per-mode FP64 square root and FP64 shuffles of a single pass made it
// FP64-bound (73 ms at 1536^3 against ~2 ms for its 14.5 GB of reads).
// cic_correct: per mode |delta_k|^2 / C2(m), C2 = prod_i (1 - (2/3) sin^2(pi m_i / n)) the CIC
// window squared summed over its aliases (Jing 2005 for a locally flat spectrum); the shot noise
// V / particles is subtracted from the bin mean.

// bin of |m|^2 = m2 among edges[0..nbins] (edges[b] <= m2 < edges[b+1]), -1 outside
__device__ __forceinline__ int pk_bin_of(long long m2, const long long* edges, int nbins) {
  if (m2 < edges[0] || m2 >= edges[nbins]) return -1;
  int lo = 0, hi = nbins;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (m2 >= edges[mid]) lo = mid; else hi = mid;
  }
  return lo;
}

// the half space of §3.3: {kz > 0} U {kz = 0, ky > 0} U {kz = ky = 0, kx > 0}
__device__ __forceinline__ bool pk_half(int mx, int my, int kz) { return kz > 0 || my > 0 || (my == 0 && mx > 0); }

__global__ void __launch_bounds__(kPkThreads) k_pk_geometry(int n, int nc, const long long* __restrict__ edges_g,
                                                            int nbins, double* partials) {
  __shared__ long long edges[kMaxBins + 1];
  __shared__ double hk[kPkWarps][kMaxBins];
  __shared__ long long hc[kPkWarps][kMaxBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i <= nbins; i += blockDim.x) edges[i] = edges_g[i];
  for (int i = threadIdx.x; i < kPkWarps * kMaxBins; i += blockDim.x) {
    (&hk[0][0])[i] = 0.0;
    (&hc[0][0])[i] = 0;
  }
  __syncthreads();
  const long long nrows = (long long)n * n;
  for (long long row = (long long)blockIdx.x * kPkWarps + warp; row < nrows;
       row += (long long)gridDim.x * kPkWarps) {
    const int mx = signed_mode((int)(row / n), n), my = signed_mode((int)(row % n), n);
    for (int kz0 = 0; kz0 < nc; kz0 += 32) {
      const int kz = kz0 + lane;
      int bin = -1;
      double kk = 0.0;
      if (kz < nc && pk_half(mx, my, kz)) {
        const long long m2 = (long long)mx * mx + (long long)my * my + (long long)kz * kz;
        bin = pk_bin_of(m2, edges, nbins);
        if (bin >= 0) kk = sqrt((double)m2);
      }
      long long c = bin >= 0 ? 1 : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int ob = __shfl_up_sync(0xffffffffu, bin, d);
        const double ok = __shfl_up_sync(0xffffffffu, kk, d);
        const long long oc = __shfl_up_sync(0xffffffffu, c, d);
        if (lane >= d && ob == bin) {
          kk += ok;
          c += oc;
        }
      }
      const int nb_next = __shfl_down_sync(0xffffffffu, bin, 1);
      if (bin >= 0 && (lane == 31 || nb_next != bin)) {
        hk[warp][bin] += kk;
        hc[warp][bin] += c;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    double sk = 0.0;
    long long sc = 0;
    for (int w = 0; w < kPkWarps; ++w) {
      sk += hk[w][b];
      sc += hc[w][b];
    }
    double* out = partials + (size_t)blockIdx.x * 2 * nbins;
    out[b] = sk;
    out[nbins + b] = (double)sc;
  }
}

// geom[0..nbins) = sum of |m| per bin, geom[nbins..2 nbins) = mode count (exact in FP64)
__global__ void k_pk_geometry_finish(const double* __restrict__ partials, int nblocks, int nbins, double* geom) {
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    double sk = 0.0, sc = 0.0;
    for (int i = 0; i < nblocks; ++i) {
      sk += partials[(size_t)i * 2 * nbins + b];
      sc += partials[(size_t)i * 2 * nbins + nbins + b];
    }
    geom[b] = sk;
    geom[nbins + b] = sc;
  }
}

constexpr int kPkUnroll = 4;   // k_z chunks of 32 whose loads a lane issues before scanning them

__global__ void __launch_bounds__(kPkThreads) k_pk_power(int n, int pc, int nc, const float2* __restrict__ dk,
                                                         const long long* __restrict__ edges_g, int nbins,
                                                         int cic_correct, double* partials) {
  __shared__ long long edges[kMaxBins + 1];
  __shared__ double hp[kPkWarps][kMaxBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i <= nbins; i += blockDim.x) edges[i] = edges_g[i];
  for (int i = threadIdx.x; i < kPkWarps * kMaxBins; i += blockDim.x) (&hp[0][0])[i] = 0.0;
  __syncthreads();
  const long long nrows = (long long)n * n;
  const float inv_n = 1.0f / (float)n;
  for (long long row = (long long)blockIdx.x * kPkWarps + warp; row < nrows;
       row += (long long)gridDim.x * kPkWarps) {
    const int mx = signed_mode((int)(row / n), n), my = signed_mode((int)(row % n), n);
    const long long mxy = (long long)mx * mx + (long long)my * my;
    float cxy = 1.0f;
    if (cic_correct) {
      const float sx = sinpif((float)mx * inv_n), sy = sinpif((float)my * inv_n);
      cxy = (1.0f - (2.0f / 3.0f) * sx * sx) * (1.0f - (2.0f / 3.0f) * sy * sy);
    }
    const float2* rowp = dk + row * pc;
    int bin = -2;   // the lane's current bin along the row (-2: not searched yet)
    for (int kz0 = 0; kz0 < nc; kz0 += 32 * kPkUnroll) {
      // the chunk's loads first (streaming: the spectrum is read once), then one scan per 32 modes
      float2 z[kPkUnroll];
#pragma unroll
      for (int u = 0; u < kPkUnroll; ++u) {
        const int kz = kz0 + 32 * u + lane;
        z[u] = kz < nc ? __ldcs(rowp + kz) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kPkUnroll; ++u) {
        const int kz = kz0 + 32 * u + lane;
        int b = -1;
        float p = 0.0f;
        if (kz < nc && pk_half(mx, my, kz)) {
          const long long m2 = mxy + (long long)kz * kz;
          // |m|^2 grows along the row: advance the previous bin instead of searching again
          if (bin < 0 || m2 < edges[bin]) bin = pk_bin_of(m2, edges, nbins);
          else
            while (bin >= 0 && m2 >= edges[bin + 1]) bin = bin + 1 < nbins ? bin + 1 : -1;
          b = bin;
          if (b >= 0) {
            p = z[u].x * z[u].x + z[u].y * z[u].y;
            if (cic_correct) {
              const float sz = sinpif((float)kz * inv_n);
              p = p / (cxy * (1.0f - (2.0f / 3.0f) * sz * sz));
            }
          }
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int ob = __shfl_up_sync(0xffffffffu, b, d);
          const float op = __shfl_up_sync(0xffffffffu, p, d);
          if (lane >= d && ob == b) p += op;
        }
        const int nb_next = __shfl_down_sync(0xffffffffu, b, 1);
        if (b >= 0 && (lane == 31 || nb_next != b)) hp[warp][b] += (double)p;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    double sp = 0.0;
    for (int w = 0; w < kPkWarps; ++w) sp += hp[w][b];
    partials[(size_t)blockIdx.x * nbins + b] = sp;
  }
}

// pk[0..nbins) = mean |k| (h/Mpc), pk[nbins..) = P = pscale * mean power - shot, pk[2 nbins..) = modes
__global__ void k_pk_finish(const double* __restrict__ partials, int nblocks, int nbins,
                            const double* __restrict__ geom, double kfund, double pscale, double shot, double* pk) {
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    double sp = 0.0;
    for (int i = 0; i < nblocks; ++i) sp += partials[(size_t)i * nbins + b];
    const double sk = geom[b], sc = geom[nbins + b];
    pk[b] = sc > 0 ? sk / sc * kfund : 0.0;
    pk[nbins + b] = sc > 0 ? pscale * sp / sc - shot : 0.0;
    pk[2 * nbins + b] = sc;
  }
}

// out[j m + i] = F_j at mesh cell cells[i] = (ix N + iy) N + iz of the real fields (rows of rs floats)
__global__ void k_sample_mesh(int n, long long rs, const float* __restrict__ f0, const float* __restrict__ f1,
                              const float* __restrict__ f2, const long long* __restrict__ cells, long long m,
                              float* __restrict__ out) {
  const long long n3 = (long long)n * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
    long long c = cells[t];
    c = c < 0 ? 0 : (c >= n3 ? n3 - 1 : c);   // the host validates the cells; never read outside
    const long long row = c / n, z = c - row * n;
    const long long o = row * rs + z;
    out[t] = f0[o];
    out[m + t] = f1[o];
    out[2 * m + t] = f2[o];
  }
}

__global__ void k_dense_spectrum(int n, int pc, int nc, const float2* __restrict__ src, float2* dst) {
  const long long total = (long long)n * n * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = src[(t / nc) * pc + (t % nc)];
}

}  // namespace

unsigned rows_grid(const ParticleGeom& pg) {
  const long long rows = (long long)pg.np * pg.np;
  const long long cap = 152LL * 64;
  return (unsigned)(rows < cap ? rows : cap);
}

int launch_deposit(const ParticleGeom& pg, const float* s, unsigned long long* rho, int* flags, cudaStream_t st) {
  (void)flags;
  const int th = pg.np < kRowThreads ? ((pg.np + 31) / 32) * 32 : kRowThreads;
  k_deposit<<<rows_grid(pg), th, 0, st>>>(pg, s, rho);
  return check_launch("deposit");
}

// 128-bit sum of m (lo, hi) pairs into the accumulator slots
__global__ void k_mass_reduce(const unsigned long long* __restrict__ pairs, long long m, unsigned long long* acc) {
  unsigned long long lo = 0, hi = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long l = pairs[2 * i];
    lo += l;
    hi += pairs[2 * i + 1] + (lo < l);
  }
  mass_accumulate(lo, hi, mass_slot(acc));
}

int launch_mass_reduce(const unsigned long long* pairs, long long m, unsigned long long* acc, cudaStream_t st) {
  k_mass_reduce<<<grid_for(m, 256), 256, 0, st>>>(pairs, m, acc);
  return check_launch("mass_reduce");
}

int launch_mass_check(const ParticleGeom& pg, const unsigned long long* rho, bool sum_mesh, unsigned long long* acc,
                      int* flags, cudaStream_t st) {
  if (sum_mesh) {
    const long long cells = (long long)pg.n * pg.n * pg.n;
    k_mesh_sum<<<grid_for(cells, 256), 256, 0, st>>>(rho, cells, acc);
    const int e = check_launch("mesh_sum");
    if (e != COLA_OK) return e;
  }
  // expected total: n 2^42 as a 128-bit number
  const unsigned long long n = (unsigned long long)pg.npart;
  const unsigned long long lo = n << 42, hi = n >> 22;
  k_mass_check<<<1, 32, 0, st>>>(acc, lo, hi, acc, flags);
  return check_launch("mass_check");
}

int launch_gather(const ParticleGeom& pg, const float* const f[3], long long rs, const float* s_in,
                  float* force_out, float* s, float* v, const float* psi1, const float* psi2,
                  const KickDrift* kd, int* flags, cudaStream_t st) {
  const unsigned g = rows_grid(pg);
  const int th = pg.np < kRowThreads ? ((pg.np + 31) / 32) * 32 : kRowThreads;
  if (kd)
    k_gather<true><<<g, th, 0, st>>>(pg, f[0], f[1], f[2], rs, nullptr, nullptr, s, v, psi1, psi2, *kd, flags);
  else
    k_gather<false><<<g, th, 0, st>>>(pg, f[0], f[1], f[2], rs, s_in, force_out, nullptr, nullptr, nullptr,
                                      nullptr, KickDrift{}, flags);
  return check_launch("gather");
}

int launch_ic_amplitude(const Grid3& g, float2* wk, const float* amp_m2, cudaStream_t st) {
  k_ic_amplitude<<<grid_for((long long)g.rows() * g.nc, 256), 256, 0, st>>>(g.n, g.pc, g.nc, wk, amp_m2);
  return check_launch("ic_amplitude");
}

int launch_ic_multiply(const Grid3& g, const float2* src, float2* dst, IcField kind, int i, int j, float scale,
                       cudaStream_t st, bool accumulate) {
  k_ic_multiply<<<grid_for((long long)g.rows() * g.nc, 256), 256, 0, st>>>(g.n, g.pc, g.nc, src, dst,
                                                                           IcMul{(int)kind, i, j, scale},
                                                                           accumulate ? 1 : 0);
  return check_launch("ic_multiply");
}

int launch_ic_source(const Grid3& g, float2* const h[6], float2* dst, cudaStream_t st) {
  auto f = [](float2* p) { return reinterpret_cast<const float*>(p); };
  k_ic_source<<<grid_for((long long)g.rows() * g.n, 256), 256, 0, st>>>(
      g.n, g.pc, f(h[0]), f(h[1]), f(h[2]), f(h[3]), f(h[4]), f(h[5]), reinterpret_cast<float*>(dst));
  return check_launch("ic_source");
}

int launch_ic_to_particles(const Grid3& g, const float2* field, float scale, float* dst, cudaStream_t st) {
  k_ic_to_particles<<<grid_for((long long)g.rows() * g.n, 256), 256, 0, st>>>(
      g.n, g.pc, reinterpret_cast<const float*>(field), scale, dst);
  return check_launch("ic_to_particles");
}

int launch_ic_positions(long long npart, const float* psi1, const float* psi2, float d1, float d2, float* s,
                        float* v, cudaStream_t st) {
  k_ic_positions<<<grid_for(3 * npart, 256), 256, 0, st>>>(3 * npart, psi1, psi2, d1, d2, s, v);
  return check_launch("ic_positions");
}

int launch_snapshot(long long npart, const float* s, const float* v, const float* psi1, const float* psi2, float alpha,
                    float b1, float b2, float g1, float g2, float* s_out, float* v_out, cudaStream_t st) {
  k_snapshot<<<grid_for(3 * npart, 256), 256, 0, st>>>(3 * npart, s, v, psi1, psi2, alpha, b1, b2, g1, g2, s_out,
                                                       v_out);
  return check_launch("snapshot");
}

int launch_pk_geometry(const Grid3& g, const long long* edges, int nbins, double* partials, int nblocks,
                       double* geom, cudaStream_t st) {
  k_pk_geometry<<<nblocks, kPkThreads, 0, st>>>(g.n, g.nc, edges, nbins, partials);
  k_pk_geometry_finish<<<1, 128, 0, st>>>(partials, nblocks, nbins, geom);
  return check_launch("pk_geometry");
}

int launch_pk_bins(const Grid3& g, const float2* dk, const long long* edges, int nbins, int cic_correct,
                   double* partials, int nblocks, cudaStream_t st) {
  k_pk_power<<<nblocks, kPkThreads, 0, st>>>(g.n, g.pc, g.nc, dk, edges, nbins, cic_correct, partials);
  return check_launch("pk_bins");
}

int launch_pk_finish(const double* partials, int nblocks, int nbins, const double* geom, double kfund, double pscale,
                     double shot, double* pk, cudaStream_t st) {
  k_pk_finish<<<1, 128, 0, st>>>(partials, nblocks, nbins, geom, kfund, pscale, shot, pk);
  return check_launch("pk_finish");
}

int launch_sample_mesh(const Grid3& g, const float* const f[3], const long long* cells, long long m, float* out,
                       cudaStream_t st) {
  if (m <= 0) return COLA_OK;
  k_sample_mesh<<<grid_for(m, 256), 256, 0, st>>>(g.n, 2LL * g.pc, f[0], f[1], f[2], cells, m, out);
  return check_launch("sample_mesh");
}

int launch_dense_spectrum(const Grid3& g, const float2* src, float* dst, cudaStream_t st) {
  k_dense_spectrum<<<grid_for((long long)g.rows() * g.nc, 256), 256, 0, st>>>(g.n, g.pc, g.nc, src,
                                                                              reinterpret_cast<float2*>(dst));
  return check_launch("dense_spectrum");
}

}  // namespace cola
