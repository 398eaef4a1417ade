// Hand-written adjoint (reverse mode) of the COLA run, and the CIC density of the differentiable
// loss.  The paper has no adjoint; this is the transpose of the forward of §2.1/§2.2 (kick, drift,
// PM force) and of the 2LPT maps (§2.1), for the continuous-CIC model: the fixed-point deposit is
// piecewise constant in position, so the adjoint uses the derivative of the continuous CIC weights
// (+-1 times the other axes' weights, one-sided at cell faces, cell chosen by the forward's
// fixed-point coordinate).  Reverse pass per step i (checkpointed positions s_i):
//   lam_v += drift lam_s;  lam_Psi += dD lam_s                 (transpose of the drift)
//   lam_F = kick lam_v;    lam_Psi -= c lam_F                  (transpose of the kick)
//   recompute F(s_i) on the mesh; deposit lam_F on three meshes; lam_delta = sum_j conj(i D_j g) lam_F_j
//   lam_s += sum_c grad W(x - c) [lam_F . F_c + (N^3/n) lam_delta_c]
// Float atomics sum the deposits, so the adjoint is accurate to FP32 rounding but not
// bit-reproducible from run to run.
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
  const long long cap = 152LL * 16 * 4;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ void lattice_of(long long id, int np, int* q) {
  const long long np2 = (long long)np * np;
  q[0] = (int)(id / np2);
  const long long rem = id - (long long)q[0] * np2;
  q[1] = (int)(rem / np);
  q[2] = (int)(rem - (long long)q[1] * np);
}

// cell and weight of cell c+1 per axis, from the forward's fixed-point coordinate
__device__ __forceinline__ void cic_cell(const ParticleGeom& pg, long long id, const float* s, long long n, int* c,
                                         float* w1) {
  int q[3];
  lattice_of(id, pg.np, q);
  const long long modulus = (long long)pg.n << kFracBits;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long g = fixed_coord(q[a], s[a * n + id], pg.r_fixed, modulus);
    c[a] = (int)(g >> kFracBits);
    w1[a] = (float)((int)(g >> (kFracBits - 14)) & (kWeightOne - 1)) * (1.0f / kWeightOne);
  }
}

// lam_v += drift lam_s; lam_p1 += dd1 lam_s; lam_p2 += dd2 lam_s; lam_f = kick lam_v;
// lam_p1 -= c1 lam_f; lam_p2 -= c2 lam_f   (all [3][n])
__global__ void k_adj_step(long long n3, const float* __restrict__ lam_s, float* lam_v, float* lam_p1, float* lam_p2,
                           float* lam_f, float drift, float dd1, float dd2, float kick, float c1, float c2) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3; t += (long long)gridDim.x * blockDim.x) {
    const float ls = lam_s[t];
    const float lv = lam_v[t] + drift * ls;
    const float lf = kick * lv;
    lam_v[t] = lv;
    lam_f[t] = lf;
    lam_p1[t] += dd1 * ls - c1 * lf;
    lam_p2[t] += dd2 * ls - c2 * lf;
  }
}

// deposit the three components of lam_f with CIC weights onto three real meshes (rows of rs)
__global__ void k_adj_deposit(ParticleGeom pg, const float* __restrict__ s, const float* __restrict__ lam_f, float* m0,
                              float* m1, float* m2, long long rs) {
  const long long n = pg.npart;
  const int nm = pg.n;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    int c[3];
    float w1[3];
    cic_cell(pg, id, s, n, c, w1);
    const float l0 = lam_f[id], l1 = lam_f[n + id], l2 = lam_f[2 * n + id];
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int ix = (c[0] + dx) == nm ? 0 : c[0] + dx;
      const float wx = dx ? w1[0] : 1.0f - w1[0];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int iy = (c[1] + dy) == nm ? 0 : c[1] + dy;
        const float wxy = wx * (dy ? w1[1] : 1.0f - w1[1]);
        const long long row = ((long long)ix * nm + iy) * rs;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int iz = (c[2] + dz) == nm ? 0 : c[2] + dz;
          const float w = wxy * (dz ? w1[2] : 1.0f - w1[2]);
          atomicAdd(m0 + row + iz, w * l0);
          atomicAdd(m1 + row + iz, w * l1);
          atomicAdd(m2 + row + iz, w * l2);
        }
      }
    }
  }
}

// out(k) = sum_j conj(i D(m_j) g) L_j(k) = -i g sum_j D(m_j) L_j(k), g = g_scale / |m|^2; out may be L_0
__global__ void k_adj_combine(int n, int pc, int nc, const float2* l0, const float2* l1, const float2* l2,
                              const float* __restrict__ dtab, float g_scale, float2* out) {
  const long long total = (long long)n * n * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(t % nc);
    const long long row = t / nc;
    const int ix = (int)(row / n), iy = (int)(row % n);
    const int mx = ix < n / 2 ? ix : ix - n, my = iy < n / 2 ? iy : iy - n;
    const int m2 = mx * mx + my * my + kz * kz;
    const long long e = row * pc + kz;
    const float g = m2 > 0 ? g_scale / (float)m2 : 0.0f;
    const float2 a = l0[e], b = l1[e], cc = l2[e];
    const float dx = dtab[ix], dy = dtab[iy], dz = dtab[kz];
    const float re = dx * a.x + dy * b.x + dz * cc.x, im = dx * a.y + dy * b.y + dz * cc.y;
    out[e] = make_float2(g * im, -g * re);   // -i g (re + i im)
  }
}

// lam_s += sum_c grad W(x - c) [lam_f . F_c + norm lam_delta_c]
__global__ void k_adj_gather(ParticleGeom pg, const float* __restrict__ s, const float* __restrict__ lam_f,
                             const float* __restrict__ f0, const float* __restrict__ f1, const float* __restrict__ f2,
                             const float* __restrict__ ld, long long rs, float norm, float* lam_s) {
  const long long n = pg.npart;
  const int nm = pg.n;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    int c[3];
    float w1[3];
    cic_cell(pg, id, s, n, c, w1);
    const float l0 = lam_f[id], l1 = lam_f[n + id], l2 = lam_f[2 * n + id];
    float gxs = 0.f, gys = 0.f, gzs = 0.f;
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int ix = (c[0] + dx) == nm ? 0 : c[0] + dx;
      const float wx = dx ? w1[0] : 1.0f - w1[0], gx = dx ? 1.0f : -1.0f;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int iy = (c[1] + dy) == nm ? 0 : c[1] + dy;
        const float wy = dy ? w1[1] : 1.0f - w1[1], gy = dy ? 1.0f : -1.0f;
        const long long row = ((long long)ix * nm + iy) * rs;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int iz = (c[2] + dz) == nm ? 0 : c[2] + dz;
          const float wz = dz ? w1[2] : 1.0f - w1[2], gz = dz ? 1.0f : -1.0f;
          const long long e = row + iz;
          const float v = l0 * __ldg(f0 + e) + l1 * __ldg(f1 + e) + l2 * __ldg(f2 + e) + norm * __ldg(ld + e);
          gxs += gx * wy * wz * v;
          gys += wx * gy * wz * v;
          gzs += wx * wy * gz * v;
        }
      }
    }
    lam_s[id] += gxs;
    lam_s[n + id] += gys;
    lam_s[2 * n + id] += gzs;
  }
}

// lam_p1 += d1 lam_s; lam_p2 += d2 lam_s   (initial condition s_1 = D1 Psi1 + D2 Psi2)
__global__ void k_adj_ic(long long n3, const float* __restrict__ lam_s, float* lam_p1, float* lam_p2, float d1, float d2) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3; t += (long long)gridDim.x * blockDim.x) {
    lam_p1[t] += d1 * lam_s[t];
    lam_p2[t] += d2 * lam_s[t];
  }
}

// particle array [n] -> real lattice field (rows of 2 pc floats), times scale
__global__ void k_particles_to_field(int n, int pc, const float* __restrict__ src, float scale, float* dst) {
  const long long total = (long long)n * n * n;
  const long long rs = 2LL * pc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    dst[(t / n) * rs + (t % n)] = src[t] * scale;
}

// Transpose of the second-order source S = h00 h11 + h00 h22 + h11 h22 - h01^2 - h02^2 - h12^2
// (§2.1): the six Hessian fields h (rows of 2 pc floats) are replaced in place by lam_S dS/dh.
__global__ void k_ic_source_adjoint(int n, int pc, const float* __restrict__ lam_src, float* h0, float* h1, float* h2,
                                    float* h3, float* h4, float* h5) {
  const long long total = (long long)n * n * n;
  const long long rs = 2LL * pc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long i = (t / n) * rs + (t % n);
    const float l = lam_src[i];
    const float a = h0[i], b = h1[i], c = h2[i], d = h3[i], e = h4[i], f = h5[i];
    h0[i] = l * (b + c);
    h1[i] = l * (a + c);
    h2[i] = l * (a + b);
    h3[i] = -2.0f * l * d;
    h4[i] = -2.0f * l * e;
    h5[i] = -2.0f * l * f;
  }
}

// ---- CIC density contrast of the loss grid (continuous weights) and its adjoint ---------------
// grid coordinate y = (q N/np + s) ngrid / N, wrapped into [0, ngrid)
__device__ __forceinline__ void grid_cell(const ParticleGeom& pg, long long id, const float* s, long long n, int ng,
                                          double ratio, int* c, float* t) {
  int q[3];
  lattice_of(id, pg.np, q);
  const double r = (double)pg.n / pg.np;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double y = ((double)q[a] * r + (double)s[a * n + id]) * ratio;
    y -= floor(y / ng) * ng;
    double fy = floor(y);
    double tt = y - fy;
    int ci = (fy >= 0.0 && fy < (double)ng) ? (int)fy : 0;   // y == ng after rounding, or not finite
    if (!(fy >= 0.0 && fy < (double)ng)) tt = 0.0;
    c[a] = ci;
    t[a] = (float)tt;
  }
}

// Continuous CIC weights rounded to multiples of 2^-32 and summed with 64-bit integer atomics:
// the sum is exact and independent of the order, so the loss grid is bit-reproducible.
__global__ void k_grid_deposit(ParticleGeom pg, const float* __restrict__ s, int ng, double ratio,
                               unsigned long long* rho) {
  const long long n = pg.npart;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    int c[3];
    float t[3];
    grid_cell(pg, id, s, n, ng, ratio, c, t);
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int ix = (c[0] + dx) == ng ? 0 : c[0] + dx;
      const float wx = dx ? t[0] : 1.0f - t[0];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int iy = (c[1] + dy) == ng ? 0 : c[1] + dy;
        const float wxy = wx * (dy ? t[1] : 1.0f - t[1]);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int iz = (c[2] + dz) == ng ? 0 : c[2] + dz;
          const float w = wxy * (dz ? t[2] : 1.0f - t[2]);
          const unsigned long long q = (unsigned long long)__double2ll_rn((double)w * 4294967296.0);
          if (q) atomicAdd(rho + ((long long)ix * ng + iy) * ng + iz, q);
        }
      }
    }
  }
}

// delta = rho scale - 1, scale = ng^3 / (n 2^32), in FP64
__global__ void k_grid_finish(long long cells, const unsigned long long* __restrict__ rho, double scale,
                              float* delta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells; i += (long long)gridDim.x * blockDim.x)
    delta[i] = (float)((double)rho[i] * scale - 1.0);
}

__global__ void k_grid_adjoint(ParticleGeom pg, const float* __restrict__ s, int ng, double ratio,
                               const float* __restrict__ lam_delta, float gscale, float* lam_s) {
  const long long n = pg.npart;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    int c[3];
    float t[3];
    grid_cell(pg, id, s, n, ng, ratio, c, t);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int ix = (c[0] + dx) == ng ? 0 : c[0] + dx;
      const float wx = dx ? t[0] : 1.0f - t[0], gx = dx ? 1.0f : -1.0f;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int iy = (c[1] + dy) == ng ? 0 : c[1] + dy;
        const float wy = dy ? t[1] : 1.0f - t[1], gy = dy ? 1.0f : -1.0f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int iz = (c[2] + dz) == ng ? 0 : c[2] + dz;
          const float wz = dz ? t[2] : 1.0f - t[2], gz = dz ? 1.0f : -1.0f;
          const float v = __ldg(lam_delta + ((long long)ix * ng + iy) * ng + iz);
          g0 += gx * wy * wz * v;
          g1 += wx * gy * wz * v;
          g2 += wx * wy * gz * v;
        }
      }
    }
    lam_s[id] = g0 * gscale;
    lam_s[n + id] = g1 * gscale;
    lam_s[2 * n + id] = g2 * gscale;
  }
}

}  // namespace

int launch_adj_step(long long n3, const float* lam_s, float* lam_v, float* lam_p1, float* lam_p2, float* lam_f,
                    const StepScalars& sc, cudaStream_t st) {
  k_adj_step<<<grid_for(n3, 256), 256, 0, st>>>(n3, lam_s, lam_v, lam_p1, lam_p2, lam_f, (float)sc.drift,
                                                (float)sc.dd1, (float)sc.dd2, (float)sc.kick, (float)sc.c1,
                                                (float)sc.c2);
  return check_launch("adj_step");
}

int launch_adj_deposit(const ParticleGeom& pg, const float* s, const float* lam_f, float* const m[3], long long rs,
                       cudaStream_t st) {
  k_adj_deposit<<<grid_for(pg.npart, 256), 256, 0, st>>>(pg, s, lam_f, m[0], m[1], m[2], rs);
  return check_launch("adj_deposit");
}

int launch_adj_combine(const Grid3& g, float2* const l[3], const float* dtab, float g_scale, float2* out,
                       cudaStream_t st) {
  k_adj_combine<<<grid_for((long long)g.rows() * g.nc, 256), 256, 0, st>>>(g.n, g.pc, g.nc, l[0], l[1], l[2], dtab,
                                                                           g_scale, out);
  return check_launch("adj_combine");
}

int launch_adj_gather(const ParticleGeom& pg, const float* s, const float* lam_f, const float* const f[3],
                      const float* lam_delta, long long rs, float norm, float* lam_s, cudaStream_t st) {
  k_adj_gather<<<grid_for(pg.npart, 256), 256, 0, st>>>(pg, s, lam_f, f[0], f[1], f[2], lam_delta, rs, norm, lam_s);
  return check_launch("adj_gather");
}

int launch_adj_ic(long long n3, const float* lam_s, float* lam_p1, float* lam_p2, float d1, float d2, cudaStream_t st) {
  k_adj_ic<<<grid_for(n3, 256), 256, 0, st>>>(n3, lam_s, lam_p1, lam_p2, d1, d2);
  return check_launch("adj_ic");
}

int launch_particles_to_field(const Grid3& g, const float* src, float scale, float2* dst, cudaStream_t st) {
  k_particles_to_field<<<grid_for((long long)g.rows() * g.n, 256), 256, 0, st>>>(g.n, g.pc, src, scale,
                                                                                  reinterpret_cast<float*>(dst));
  return check_launch("particles_to_field");
}

int launch_grid_density(const ParticleGeom& pg, const float* s, int ngrid, unsigned long long* scratch, float* delta,
                        cudaStream_t st) {
  const long long cells = (long long)ngrid * ngrid * ngrid;
  if (cudaMemsetAsync(scratch, 0, cells * sizeof(unsigned long long), st) != cudaSuccess) return COLA_ERR_CUDA;
  const double ratio = (double)ngrid / pg.n;
  k_grid_deposit<<<grid_for(pg.npart, 256), 256, 0, st>>>(pg, s, ngrid, ratio, scratch);
  k_grid_finish<<<grid_for(cells, 256), 256, 0, st>>>(cells, scratch, (double)cells / ((double)pg.npart * 4294967296.0),
                                                      delta);
  return check_launch("grid_density");
}

int launch_ic_source_adjoint(const Grid3& g, const float2* lam_src, float2* const h[6], cudaStream_t st) {
  float* f[6];
  for (int i = 0; i < 6; ++i) f[i] = reinterpret_cast<float*>(h[i]);
  k_ic_source_adjoint<<<grid_for((long long)g.rows() * g.n, 256), 256, 0, st>>>(
      g.n, g.pc, reinterpret_cast<const float*>(lam_src), f[0], f[1], f[2], f[3], f[4], f[5]);
  return check_launch("ic_source_adjoint");
}

int launch_grid_density_adjoint(const ParticleGeom& pg, const float* s, int ngrid, const float* lam_delta,
                                float* lam_s, cudaStream_t st) {
  const double ratio = (double)ngrid / pg.n;
  const double cells = (double)ngrid * ngrid * ngrid;
  k_grid_adjoint<<<grid_for(pg.npart, 256), 256, 0, st>>>(pg, s, ngrid, ratio, lam_delta,
                                                          (float)(cells / (double)pg.npart * ratio), lam_s);
  return check_launch("grid_density_adjoint");
}

}  // namespace cola
