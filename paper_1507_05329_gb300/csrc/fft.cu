// Hand-written mixed-radix 3D FFT passes for the PM force (sm_103a).
//
// The paper's PM force spends 66% of its time in FFTW (§2.3, Table 1).  Here each 1D pass of the
// 3D transform is one kernel that reads a tile of W pencils from HBM once, transforms it in shared
// memory with Stockham autosort stages of radix 16/8/5/4/3/2, and writes it once:
//   * contiguous axis (z): pairs of real rows packed as one complex row (R2C / C2R);
//   * strided axes (y, x): W adjacent complex columns per tile, so each row segment is a
//     contiguous W*8-byte run;
//   * the last forward pass (x) is fused with the Poisson Green function, the 4-point gradient
//     kernel and the three inverse x transforms of the force components (§2.2 Poisson equation).
// Shared-memory layout of a tile: element (j, w) at ((j + j/16) * W + w); the skew of one W-row
// every 16 rows keeps the stride-R writes of the first Stockham stages off a single bank group.
#include "cola_internal.h"

#include <cmath>
#include <cstdio>

namespace cola {
namespace {

constexpr int kEpt = 16;   // complex elements per thread (register staging of a stage)
constexpr int kMaxThreads = 384;   // largest tile (6144 elements) / kEpt

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i (forward, DIR < 0) or +i (inverse, DIR > 0)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
template <int DIR>
__device__ __forceinline__ float2 rot(float2 a, float c, float s) {   // a * (c + i*DIR*s)
  return DIR < 0 ? make_float2(a.x * c + a.y * s, a.y * c - a.x * s)
                 : make_float2(a.x * c - a.y * s, a.y * c + a.x * s);
}

// ---- small DFTs in registers, natural order in and out; sign of the exponent = DIR ----------
template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 t = v[0];
    v[0] = t + v[1];
    v[1] = t - v[1];
  }
};

template <int DIR> struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3];
    const float2 t3 = mul_i<DIR>(v[1] - v[3]);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  }
};

template <int DIR> struct Dft<8, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    const float c = 0.70710678118654752f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, DIR>::run(e);
    Dft<4, DIR>::run(o);
    o[1] = rot<DIR>(o[1], c, c);
    o[2] = mul_i<DIR>(o[2]);
    o[3] = rot<DIR>(o[3], -c, c);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = e[k] + o[k];
      v[k + 4] = e[k] - o[k];
    }
  }
};

template <int DIR> struct Dft<16, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    // w16^k = cos(pi k / 8) + i DIR sin(pi k / 8), k = 0..7
    const float cs[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                         0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f};
    const float sn[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                         1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
    float2 e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    Dft<8, DIR>::run(e);
    Dft<8, DIR>::run(o);
#pragma unroll
    for (int k = 1; k < 8; ++k) o[k] = rot<DIR>(o[k], cs[k], sn[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = e[k] + o[k];
      v[k + 8] = e[k] - o[k];
    }
  }
};

template <int DIR> struct Dft<3, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    const float h = 0.86602540378443865f;   // sqrt(3)/2
    const float2 s = v[1] + v[2], d = v[1] - v[2];
    const float2 m = v[0] - 0.5f * s;
    const float2 t = h * mul_i<DIR>(d);
    v[0] = v[0] + s;
    v[1] = m + t;
    v[2] = m - t;
  }
};

template <int DIR> struct Dft<5, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;
    const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;
    const float2 a1 = v[1] + v[4], b1 = v[1] - v[4], a2 = v[2] + v[3], b2 = v[2] - v[3];
    const float2 m1 = v[0] + c1 * a1 + c2 * a2;
    const float2 m2 = v[0] + c2 * a1 + c1 * a2;
    const float2 t1 = mul_i<DIR>(s1 * b1 + s2 * b2);
    const float2 t2 = mul_i<DIR>(s2 * b1 - s1 * b2);
    v[0] = v[0] + a1 + a2;
    v[1] = m1 + t1;
    v[4] = m1 - t1;
    v[2] = m2 + t2;
    v[3] = m2 - t2;
  }
};

__device__ __forceinline__ int saddr(int j, int w, int lw) { return ((j + (j >> 4)) << lw) + w; }

// One Stockham stage on W pencils of length n (Govindaraju et al. 2008 formulation): butterfly b
// reads x[b + r n/R], twiddles by w_n^(r k n/(Ns R)) with k = b mod Ns, and writes
// y[(b - k) R + k + r Ns].  Ping-pong between two shared buffers, one barrier per stage.
template <int R, int DIR>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ x, float2* __restrict__ y, int n, int lw,
                                          int ns, const float2* __restrict__ tw, int tid, int nthreads) {
  const int nb = n / R;
  const int total = nb << lw;
  const int tstride = n / (ns * R);
  const int wmask = (1 << lw) - 1;
  for (int idx = tid; idx < total; idx += nthreads) {
    const int w = idx & wmask, b = idx >> lw;
    const int k = b % ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[saddr(b + r * nb, w, lw)];
    if (ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 t = __ldg(&tw[r * k * tstride]);
        if (DIR > 0) t.y = -t.y;
        v[r] = cmul(v[r], t);
      }
    }
    Dft<R, DIR>::run(v);
    const int base = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[saddr(base + r * ns, w, lw)] = v[r];
  }
  __syncthreads();
}

// All stages of the plan; the data starts in buffer a and the returned pointer holds the result.
template <int DIR>
__device__ float2* fft_smem(float2* a, float2* b, const FftDev& p, int lw, int tid, int nthreads) {
  int ns = 1;
  for (int st = 0; st < p.nstages; ++st) {
    const int r = p.radix[st];
    switch (r) {
      case 16: fft_stage<16, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
      case 8: fft_stage<8, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
      case 5: fft_stage<5, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
      case 4: fft_stage<4, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
      case 3: fft_stage<3, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
      default: fft_stage<2, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
    }
    float2* t = a;
    a = b;
    b = t;
    ns *= r;
  }
  return a;
}

__device__ __forceinline__ int tile_elems(int n, int lw) { return (n + n / 16 + 1) << lw; }

// ---- contiguous axis: pairs of real rows as one complex row ----------------------------------
template <int SRC>
__global__ void __launch_bounds__(kMaxThreads, 2) k_r2c_rows(FftDev p, int lw, const void* __restrict__ src, long long src_rs, float scale,
                           float2* __restrict__ dst, int pc, long long nrows, unsigned long long* mass_acc) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, wmask = (1 << lw) - 1;
  const long long row0 = (long long)blockIdx.x << (lw + 1);
  unsigned long long mlo = 0, mhi = 0;
  for (int idx = tid; idx < (n << lw); idx += nt) {
    const int w = idx & wmask, j = idx >> lw;
    const long long ra = row0 + 2 * w;
    float a = 0.0f, b = 0.0f;
    if (SRC == kSrcFixedPoint) {
      const unsigned long long* s = static_cast<const unsigned long long*>(src);
      if (ra < nrows) {
        const unsigned long long va = s[ra * src_rs + j];
        a = __ull2float_rn(va) * scale - 1.0f;
        mlo += va;
        mhi += (mlo < va);
      }
      if (ra + 1 < nrows) {
        const unsigned long long vb = s[(ra + 1) * src_rs + j];
        b = __ull2float_rn(vb) * scale - 1.0f;
        mlo += vb;
        mhi += (mlo < vb);
      }
    } else {
      const float* s = static_cast<const float*>(src);
      if (ra < nrows) a = s[ra * src_rs + j] * scale;
      if (ra + 1 < nrows) b = s[(ra + 1) * src_rs + j] * scale;
    }
    sm[saddr(j, w, lw)] = make_float2(a, b);
  }
  if (SRC == kSrcFixedPoint && mass_acc) mass_accumulate(mlo, mhi, mass_acc);
  __syncthreads();
  const float2* res = fft_smem<-1>(sm, sm + tile_elems(n, lw), p, lw, tid, nt);
  const int nh = n / 2;
  for (int idx = tid; idx < ((nh + 1) << lw); idx += nt) {
    const int w = idx & wmask, k = idx >> lw;
    const long long ra = row0 + 2 * w;
    const float2 zk = res[saddr(k, w, lw)];
    const float2 zn = res[saddr(k == 0 ? 0 : n - k, w, lw)];
    // A = (Z_k + conj Z_{n-k}) / 2,  B = (Z_k - conj Z_{n-k}) / 2i
    const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
    const float2 B = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    if (ra < nrows) dst[ra * pc + k] = A;
    if (ra + 1 < nrows) dst[(ra + 1) * pc + k] = B;
  }
}

__global__ void __launch_bounds__(kMaxThreads, 2) k_c2r_rows(FftDev p, int lw, float2* data, int pc, long long nrows) {
  extern __shared__ float2 sm[];
  const int n = p.n, nh = n / 2, tid = threadIdx.x, nt = blockDim.x, wmask = (1 << lw) - 1;
  const long long row0 = (long long)blockIdx.x << (lw + 1);
  for (int idx = tid; idx < (n << lw); idx += nt) {
    const int w = idx & wmask, k = idx >> lw;
    const long long ra = row0 + 2 * w;
    const int kk = k <= nh ? k : n - k;
    float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
    if (ra < nrows) A = data[ra * pc + kk];
    if (ra + 1 < nrows) B = data[(ra + 1) * pc + kk];
    if (kk == 0 || kk == nh) { A.y = 0.f; B.y = 0.f; }   // self-conjugate bins are real
    float2 c;
    if (k <= nh) c = make_float2(A.x - B.y, A.y + B.x);   // A + iB
    else c = make_float2(A.x + B.y, B.x - A.y);           // conj(A) + i conj(B)
    sm[saddr(k, w, lw)] = c;
  }
  __syncthreads();
  const float2* res = fft_smem<+1>(sm, sm + tile_elems(n, lw), p, lw, tid, nt);
  float* out = reinterpret_cast<float*>(data);
  const long long rs = 2LL * pc;
  for (int idx = tid; idx < (n << lw); idx += nt) {
    const int w = idx & wmask, j = idx >> lw;
    const long long ra = row0 + 2 * w;
    const float2 c = res[saddr(j, w, lw)];
    if (ra < nrows) out[ra * rs + j] = c.x;
    if (ra + 1 < nrows) out[(ra + 1) * rs + j] = c.y;
  }
}

// ---- strided axes: W adjacent columns, transform along j ----------------------------------
template <int DIR>
__global__ void __launch_bounds__(kMaxThreads, 2) k_pencils(FftDev p, int lw, float2* data, long long jstride, long long ostride, int nc) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, wmask = (1 << lw) - 1;
  const int col0 = blockIdx.x << lw;
  float2* base = data + (long long)blockIdx.y * ostride + col0;
  for (int idx = tid; idx < (n << lw); idx += nt) {
    const int w = idx & wmask, j = idx >> lw;
    sm[saddr(j, w, lw)] = (col0 + w < nc) ? base[j * jstride + w] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res = fft_smem<DIR>(sm, sm + tile_elems(n, lw), p, lw, tid, nt);
  for (int idx = tid; idx < (n << lw); idx += nt) {
    const int w = idx & wmask, j = idx >> lw;
    if (col0 + w < nc) base[j * jstride + w] = res[saddr(j, w, lw)];
  }
}

// ---- x pass fused with the Green function and gradient kernel ------------------------------
// Tile: W adjacent k_z columns of the plane y = blockIdx.y, transformed along x.  After the
// forward x transform the tile holds delta(k) for known (m_x, m_y, m_z); each component
//   F_j(k) = i D(m_j) g_scale delta(k) / |m|^2,   D(m) = (8 sin k - sin 2k)/6, k = 2 pi m / n
// (g_scale = force_scale / (kf^2 n^3), kf = 2 pi / n, the 1/n^3 normalising the inverse 3D
// transform) is inverse-transformed along x and stored.  out2 may alias in.
__global__ void __launch_bounds__(kMaxThreads, 1) k_green_x(FftDev p, int lw, const float2* in, float2* out0, float2* out1, float2* out2,
                          int pc, int nc, const float* __restrict__ dtab, float g_scale) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, wmask = (1 << lw) - 1;
  const int col0 = blockIdx.x << lw;
  const int y = blockIdx.y;
  const long long jstride = (long long)n * pc;
  const long long boff = (long long)y * pc + col0;
  const int total = n << lw;
  for (int idx = tid; idx < total; idx += nt) {
    const int w = idx & wmask, j = idx >> lw;
    sm[saddr(j, w, lw)] = (col0 + w < nc) ? in[boff + j * jstride + w] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* const buf0 = sm;
  float2* const buf1 = sm + tile_elems(n, lw);
  const float2* spec = fft_smem<-1>(buf0, buf1, p, lw, tid, nt);
  const int my = y < n / 2 ? y : y - n;
  float2 gd[kEpt];
#pragma unroll
  for (int e = 0; e < kEpt; ++e) {
    const int idx = tid + e * nt;
    gd[e] = make_float2(0.f, 0.f);
    if (idx < total) {
      const int w = idx & wmask, j = idx >> lw;
      const int mx = j < n / 2 ? j : j - n;
      const int mz = col0 + w;
      const int m2 = mx * mx + my * my + mz * mz;
      const float g = m2 > 0 ? g_scale / (float)m2 : 0.0f;
      gd[e] = g * spec[saddr(j, w, lw)];
    }
  }
  __syncthreads();
  const float dy = dtab[y];
#pragma unroll 1
  for (int comp = 0; comp < 3; ++comp) {
#pragma unroll
    for (int e = 0; e < kEpt; ++e) {
      const int idx = tid + e * nt;
      if (idx < total) {
        const int w = idx & wmask, j = idx >> lw;
        const int mz = col0 + w;
        const float d = comp == 0 ? dtab[j] : (comp == 1 ? dy : (mz < nc ? dtab[mz] : 0.0f));
        buf0[saddr(j, w, lw)] = make_float2(-d * gd[e].y, d * gd[e].x);   // i D g delta
      }
    }
    __syncthreads();
    const float2* res = fft_smem<+1>(buf0, buf1, p, lw, tid, nt);
    float2* o = comp == 0 ? out0 : (comp == 1 ? out1 : out2);
    for (int idx = tid; idx < total; idx += nt) {
      const int w = idx & wmask, j = idx >> lw;
      if (col0 + w < nc) o[boff + j * jstride + w] = res[saddr(j, w, lw)];
    }
    __syncthreads();
  }
}

// =============================================================================================
// Fast path: plans whose every stage has ns = (product of earlier radices) a power of two, i.e.
// n = 2^a * (1, 3 or 5) with the odd factor as the last stage.  No runtime division; the first
// stage loads from global memory into registers and the last stage stores from registers.
// Inverse transforms run the transposed stages in reverse order with conjugate twiddles
// (F is symmetric, so conj(F) = conj(S_0^T) ... conj(S_{m-1}^T)); the first of them reads exactly
// the elements the forward's last butterfly produced, which keeps the Green multiply in registers.
// =============================================================================================
struct FastPlan {
  int n, nst;
  int radix[kMaxStages];
  int lns[kMaxStages];    // log2 of ns at each stage
  int tstr[kMaxStages];   // twiddle stride n / (ns R)
  const float2* tw;
};

template <int DIR>
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int t) {
  float2 v = __ldg(&tw[t]);
  if (DIR > 0) v.y = -v.y;
  return v;
}

// forward (decimation in time) stage s
template <int R, int DIR, class Src, class Dst>
__device__ __forceinline__ void fwd_stage(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                          int nthreads) {
  constexpr int kB = (kEpt + R - 1) / R;
  const int nb = p.n / R, total = nb << lw, lns = p.lns[s], tstr = p.tstr[s];
  const int wm = (1 << lw) - 1, km = (1 << lns) - 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nthreads;
    if (idx < total) {
      const int w = idx & wm, b = idx >> lw, k = b & km;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src(b + r * nb, w);
      if (lns) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twid<DIR>(p.tw, r * k * tstr));
      }
      Dft<R, DIR>::run(v);
      const int base = (((b >> lns) * R) << lns) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst(base + (r << lns), w, v[r]);
    }
  }
}

// transposed stage s (used in reverse order for the inverse transform)
template <int R, int DIR, class Src, class Dst>
__device__ __forceinline__ void tr_stage(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                         int nthreads) {
  constexpr int kB = (kEpt + R - 1) / R;
  const int nb = p.n / R, total = nb << lw, lns = p.lns[s], tstr = p.tstr[s];
  const int wm = (1 << lw) - 1, km = (1 << lns) - 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nthreads;
    if (idx < total) {
      const int w = idx & wm, b = idx >> lw, k = b & km;
      const int base = (((b >> lns) * R) << lns) + k;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src(base + (r << lns), w);
      Dft<R, DIR>::run(v);
      if (lns) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twid<DIR>(p.tw, r * k * tstr));
      }
#pragma unroll
      for (int r = 0; r < R; ++r) dst(b + r * nb, w, v[r]);
    }
  }
}

template <bool TR, int DIR, class Src, class Dst>
__device__ __forceinline__ void any_stage(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                          int nt) {
  switch (p.radix[s]) {
    case 16: TR ? tr_stage<16, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<16, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 8: TR ? tr_stage<8, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<8, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 5: TR ? tr_stage<5, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<5, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 4: TR ? tr_stage<4, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<4, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 3: TR ? tr_stage<3, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<3, DIR>(p, s, lw, src, dst, tid, nt); break;
    default: TR ? tr_stage<2, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<2, DIR>(p, s, lw, src, dst, tid, nt); break;
  }
}

struct SmemR {
  const float2* s;
  int lw;
  __device__ __forceinline__ float2 operator()(int j, int w) const { return s[saddr(j, w, lw)]; }
};
struct SmemW {
  float2* s;
  int lw;
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const { s[saddr(j, w, lw)] = v; }
};

// Forward transform of a tile: stage 0 reads gsrc, the last stage writes gdst, shared memory
// (buffers a, b) in between.  Ends with a barrier only when the caller asks (sync_end).
template <int DIR, class GSrc, class GDst>
__device__ __forceinline__ void fwd_tile(const FastPlan& p, int lw, float2* a, float2* b, const GSrc& gsrc,
                                         const GDst& gdst, int tid, int nt) {
  const int m = p.nst;
  if (m == 1) {
    any_stage<false, DIR>(p, 0, lw, gsrc, gdst, tid, nt);
    return;
  }
  any_stage<false, DIR>(p, 0, lw, gsrc, SmemW{a, lw}, tid, nt);
  __syncthreads();
  for (int s = 1; s < m - 1; ++s) {
    any_stage<false, DIR>(p, s, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  any_stage<false, DIR>(p, m - 1, lw, SmemR{a, lw}, gdst, tid, nt);
}

// Inverse transform of a tile by the transposed stages m-1 .. 0.
template <int DIR, class GSrc, class GDst>
__device__ __forceinline__ void inv_tile(const FastPlan& p, int lw, float2* a, float2* b, const GSrc& gsrc,
                                         const GDst& gdst, int tid, int nt) {
  const int m = p.nst;
  if (m == 1) {
    any_stage<true, DIR>(p, 0, lw, gsrc, gdst, tid, nt);
    return;
  }
  any_stage<true, DIR>(p, m - 1, lw, gsrc, SmemW{a, lw}, tid, nt);
  __syncthreads();
  for (int s = m - 2; s > 0; --s) {
    any_stage<true, DIR>(p, s, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  any_stage<true, DIR>(p, 0, lw, SmemR{a, lw}, gdst, tid, nt);
}

// ---- global-memory views ---------------------------------------------------------------------
struct PencilG {   // W adjacent columns of a strided pencil, masked beyond nc
  float2* base;
  long long jstride;
  int cols_left;   // nc - col0
  __device__ __forceinline__ float2 operator()(int j, int w) const {
    return w < cols_left ? base[j * jstride + w] : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const {
    if (w < cols_left) base[j * jstride + w] = v;
  }
};

template <int SRC>
struct RowPairSrc {   // complex (row 2w, row 2w+1) at column j of real rows
  const void* src;
  long long rs, row0, nrows;
  float scale;
  mutable unsigned long long mlo = 0, mhi = 0;   // 128-bit sum of the fixed-point values read
  __device__ __forceinline__ float2 operator()(int j, int w) const {
    const long long ra = row0 + 2 * w;
    float a = 0.f, b = 0.f;
    if (SRC == kSrcFixedPoint) {
      const unsigned long long* s = static_cast<const unsigned long long*>(src);
      if (ra < nrows) {
        const unsigned long long va = s[ra * rs + j];
        a = __ull2float_rn(va) * scale - 1.0f;
        mlo += va;
        mhi += (mlo < va);
      }
      if (ra + 1 < nrows) {
        const unsigned long long vb = s[(ra + 1) * rs + j];
        b = __ull2float_rn(vb) * scale - 1.0f;
        mlo += vb;
        mhi += (mlo < vb);
      }
    } else {
      const float* s = static_cast<const float*>(src);
      if (ra < nrows) a = s[ra * rs + j] * scale;
      if (ra + 1 < nrows) b = s[(ra + 1) * rs + j] * scale;
    }
    return make_float2(a, b);
  }
};

struct HalfPairSrc {   // C[k] = A[k] + i B[k] of two Hermitian half rows (C2R input)
  const float2* data;
  int pc, n;
  long long row0, nrows;
  __device__ __forceinline__ float2 operator()(int k, int w) const {
    const long long ra = row0 + 2 * w;
    const int nh = n / 2;
    const int kk = k <= nh ? k : n - k;
    float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
    if (ra < nrows) A = data[ra * pc + kk];
    if (ra + 1 < nrows) B = data[(ra + 1) * pc + kk];
    if (kk == 0 || kk == nh) {
      A.y = 0.f;
      B.y = 0.f;
    }
    return k <= nh ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
  }
};

struct RealPairDst {   // (re, im) -> real rows (2w, 2w+1)
  float* out;
  long long rs, row0, nrows;
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const {
    const long long ra = row0 + 2 * w;
    if (ra < nrows) out[ra * rs + j] = v.x;
    if (ra + 1 < nrows) out[(ra + 1) * rs + j] = v.y;
  }
};

__device__ __forceinline__ int fast_tile_elems(int n, int lw) { return (n + n / 16 + 1) << lw; }

template <int SRC>
__global__ void __launch_bounds__(kMaxThreads, 2) k_r2c_fast(FastPlan p, int lw, const void* __restrict__ src,
                                                              long long src_rs, float scale, float2* __restrict__ dst,
                                                              int pc, long long nrows, unsigned long long* mass_acc) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, wmask = (1 << lw) - 1;
  const long long row0 = (long long)blockIdx.x << (lw + 1);
  float2* a = sm;
  float2* b = sm + fast_tile_elems(n, lw);
  RowPairSrc<SRC> g{src, src_rs, row0, nrows, scale};
  // the untangle needs Z[k] and Z[n-k] together: every stage, the last included, ends in shared memory
  float2* cur = a;
  float2* nxt = b;
  any_stage<false, -1>(p, 0, lw, g, SmemW{cur, lw}, tid, nt);
  if (SRC == kSrcFixedPoint && mass_acc) mass_accumulate(g.mlo, g.mhi, mass_acc);
  for (int s = 1; s < p.nst; ++s) {
    __syncthreads();
    any_stage<false, -1>(p, s, lw, SmemR{cur, lw}, SmemW{nxt, lw}, tid, nt);
    float2* t = cur;
    cur = nxt;
    nxt = t;
  }
  const float2* res = cur;
  __syncthreads();
  const int nh = n / 2;
  for (int idx = tid; idx < ((nh + 1) << lw); idx += nt) {
    const int w = idx & wmask, k = idx >> lw;
    const long long ra = row0 + 2 * w;
    const float2 zk = res[saddr(k, w, lw)];
    const float2 zn = res[saddr(k == 0 ? 0 : n - k, w, lw)];
    const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
    const float2 B = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    if (ra < nrows) dst[ra * pc + k] = A;
    if (ra + 1 < nrows) dst[(ra + 1) * pc + k] = B;
  }
}

__global__ void __launch_bounds__(kMaxThreads, 2) k_c2r_fast(FastPlan p, int lw, float2* data, int pc, long long nrows) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x;
  const long long row0 = (long long)blockIdx.x << (lw + 1);
  const HalfPairSrc g{data, pc, n, row0, nrows};
  // all reads of this CTA's rows happen in the first stage; the output overwrites the same rows
  const RealPairDst d{reinterpret_cast<float*>(data), 2LL * pc, row0, nrows};
  if (p.nst == 1) {
    // single stage reads and writes the same rows: stage through shared memory
    any_stage<true, +1>(p, 0, lw, g, SmemW{sm, lw}, tid, nt);
    __syncthreads();
    for (int idx = tid; idx < (n << lw); idx += nt) d(idx >> lw, idx & ((1 << lw) - 1), sm[saddr(idx >> lw, idx & ((1 << lw) - 1), lw)]);
    return;
  }
  inv_tile<+1>(p, lw, sm, sm + fast_tile_elems(n, lw), g, d, tid, nt);
}

template <int DIR>
__global__ void __launch_bounds__(kMaxThreads, 2) k_pencils_fast(FastPlan p, int lw, float2* data, long long jstride,
                                                                  long long ostride, int nc) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x;
  const int col0 = blockIdx.x << lw;
  const PencilG g{data + (long long)blockIdx.y * ostride + col0, jstride, nc - col0};
  if (p.nst == 1) {
    // the same tile is read and written: stage through shared memory
    if (DIR < 0) any_stage<false, DIR>(p, 0, lw, g, SmemW{sm, lw}, tid, nt);
    else any_stage<true, DIR>(p, 0, lw, g, SmemW{sm, lw}, tid, nt);
    __syncthreads();
    for (int idx = tid; idx < (n << lw); idx += nt) g(idx >> lw, idx & ((1 << lw) - 1), sm[saddr(idx >> lw, idx & ((1 << lw) - 1), lw)]);
    return;
  }
  if (DIR < 0) fwd_tile<DIR>(p, lw, sm, sm + fast_tile_elems(n, lw), g, g, tid, nt);
  else inv_tile<DIR>(p, lw, sm, sm + fast_tile_elems(n, lw), g, g, tid, nt);
}

// x pass fused with Green function and gradient kernel, spectrum kept in registers between the
// forward transform's last stage and the inverse transforms' first (transposed) stage.
template <int RL>
__device__ __forceinline__ void green_body(const FastPlan& p, int lw, const float2* in, float2* out0, float2* out1,
                                           float2* out2, int pc, int nc, const float* __restrict__ dtab,
                                           float g_scale) {
  extern __shared__ float2 sm[];
  constexpr int kB = (kEpt + RL - 1) / RL;
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, m = p.nst;
  const int col0 = blockIdx.x << lw, y = blockIdx.y;
  const long long jstride = (long long)n * pc;
  const long long boff = (long long)y * pc + col0;
  float2* a = sm;
  float2* b = sm + fast_tile_elems(n, lw);
  const PencilG gin{const_cast<float2*>(in) + boff, jstride, nc - col0};
  const int nb = n / RL, total = nb << lw, wm = (1 << lw) - 1;
  const int ls = p.lns[m - 1], tstr = p.tstr[m - 1];
  float2 spec[kB][RL];
  // forward stages 0 .. m-2 (shared memory), last stage into registers
  const float2* last_in = nullptr;
  if (m > 1) {
    any_stage<false, -1>(p, 0, lw, gin, SmemW{a, lw}, tid, nt);
    __syncthreads();
    for (int s = 1; s < m - 1; ++s) {
      any_stage<false, -1>(p, s, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
      __syncthreads();
      float2* t = a;
      a = b;
      b = t;
    }
    last_in = a;
  }
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nt;
    if (idx < total) {
      const int w = idx & wm, bb = idx >> lw;   // last stage: bb < ns, k = bb
#pragma unroll
      for (int r = 0; r < RL; ++r) spec[i][r] = m > 1 ? last_in[saddr(bb + r * nb, w, lw)] : gin(bb + r * nb, w);
      if (ls) {
#pragma unroll
        for (int r = 1; r < RL; ++r) spec[i][r] = cmul(spec[i][r], twid<-1>(p.tw, r * bb * tstr));
      }
      Dft<RL, -1>::run(spec[i]);
      // element j = bb + r*ns_last: multiply by g_scale / |m|^2 (the common factor of F_j)
      const int my = y < n / 2 ? y : y - n, mz = col0 + w;
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int j = bb + (r << ls);
        const int mx = j < n / 2 ? j : j - n;
        const int m2 = mx * mx + my * my + mz * mz;
        spec[i][r] = (m2 > 0 ? g_scale / (float)m2 : 0.0f) * spec[i][r];
      }
    }
  }
  __syncthreads();   // the forward's shared buffers are free from here on
  const float dy = dtab[y];
  a = sm;
  b = sm + fast_tile_elems(n, lw);
#pragma unroll 1
  for (int comp = 0; comp < 3; ++comp) {
    float2* o = comp == 0 ? out0 : (comp == 1 ? out1 : out2);
    const PencilG gout{o + boff, jstride, nc - col0};
    float2* cur = a;
    float2* nxt = b;
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const int idx = tid + i * nt;
      if (idx < total) {
        const int w = idx & wm, bb = idx >> lw;
        const int mz = col0 + w;
        float2 v[RL];
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int j = bb + (r << ls);
          const float d = comp == 0 ? dtab[j] : (comp == 1 ? dy : (mz < nc ? dtab[mz] : 0.0f));
          v[r] = make_float2(-d * spec[i][r].y, d * spec[i][r].x);   // i D g delta
        }
        // transposed last stage (first of the inverse): inputs are exactly v
        Dft<RL, +1>::run(v);
        if (ls) {
#pragma unroll
          for (int r = 1; r < RL; ++r) v[r] = cmul(v[r], twid<+1>(p.tw, r * bb * tstr));
        }
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          if (m > 1) cur[saddr(bb + r * nb, w, lw)] = v[r];
          else gout(bb + r * nb, w, v[r]);
        }
      }
    }
    if (m > 1) {
      __syncthreads();
      for (int s = m - 2; s > 0; --s) {
        any_stage<true, +1>(p, s, lw, SmemR{cur, lw}, SmemW{nxt, lw}, tid, nt);
        __syncthreads();
        float2* t = cur;
        cur = nxt;
        nxt = t;
      }
      any_stage<true, +1>(p, 0, lw, SmemR{cur, lw}, gout, tid, nt);
      __syncthreads();   // before the next component reuses the buffers
    }
  }
}

__global__ void __launch_bounds__(kMaxThreads, 1) k_green_fast(FastPlan p, int lw, const float2* in, float2* out0,
                                                               float2* out1, float2* out2, int pc, int nc,
                                                               const float* __restrict__ dtab, float g_scale) {
  switch (p.radix[p.nst - 1]) {
    case 16: green_body<16>(p, lw, in, out0, out1, out2, pc, nc, dtab, g_scale); break;
    case 8: green_body<8>(p, lw, in, out0, out1, out2, pc, nc, dtab, g_scale); break;
    case 5: green_body<5>(p, lw, in, out0, out1, out2, pc, nc, dtab, g_scale); break;
    case 4: green_body<4>(p, lw, in, out0, out1, out2, pc, nc, dtab, g_scale); break;
    case 3: green_body<3>(p, lw, in, out0, out1, out2, pc, nc, dtab, g_scale); break;
    default: green_body<2>(p, lw, in, out0, out1, out2, pc, nc, dtab, g_scale); break;
  }
}

struct TileShape {
  int lw;
  int threads;
  size_t smem;
};

constexpr int kTileElems = 6144;    // complex elements per tile (two buffers: about 100 KB of shared memory)

TileShape tile_shape(int n, int wmax) {
  int lw = 0;
  while ((2 << lw) <= wmax && n * (2 << lw) <= kTileElems) ++lw;
  TileShape t;
  t.lw = lw;
  int th = ((n << lw) + kEpt - 1) / kEpt;
  th = ((th + 31) / 32) * 32;
  t.threads = th < 32 ? 32 : th;
  t.smem = 2 * (size_t)(n + n / 16 + 1) * (1u << lw) * sizeof(float2);
  return t;
}

// Fast path eligibility: every stage's ns is a power of two.
bool fast_plan(const FftPlan& pl, FastPlan* fp) {
  const FftDev& d = pl.dev;
  int ns = 1;
  fp->n = d.n;
  fp->nst = d.nstages;
  fp->tw = d.tw;
  for (int s = 0; s < d.nstages; ++s) {
    if (ns & (ns - 1)) return false;
    int l = 0;
    while ((1 << l) < ns) ++l;
    fp->radix[s] = d.radix[s];
    fp->lns[s] = l;
    fp->tstr[s] = d.n / (ns * d.radix[s]);
    ns *= d.radix[s];
  }
  for (int s = d.nstages; s < kMaxStages; ++s) fp->radix[s] = 1, fp->lns[s] = 0, fp->tstr[s] = 0;
  return true;
}

TileShape fast_shape(int n, int wmax, int nbuf) {
  TileShape t = tile_shape(n, wmax);
  t.smem = (size_t)nbuf * (size_t)(n + n / 16 + 1) * (1u << t.lw) * sizeof(float2);
  return t;
}

int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "cola: launch of %s failed: %s\n", what, cudaGetErrorString(e));
    return COLA_ERR_CUDA;
  }
  return COLA_OK;
}

int largest_pow2_le(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

}  // namespace

bool fft_factor(int n, std::vector<int>* radices) {
  radices->clear();
  if (n < 2) return false;
  int m = n, p2 = 0;
  while (m % 2 == 0) { m /= 2; ++p2; }
  int n5 = 0, n3 = 0;
  while (m % 5 == 0) { m /= 5; ++n5; }
  while (m % 3 == 0) { m /= 3; ++n3; }
  if (m != 1) return false;
  // powers of two: the fewest stages of radix <= 16, as even as possible
  if (p2 > 0) {
    const int nst = (p2 + 3) / 4;
    int left = p2;
    for (int s = 0; s < nst; ++s) {
      const int e = (left + (nst - s) - 1) / (nst - s);
      radices->push_back(1 << e);
      left -= e;
    }
  }
  for (int i = 0; i < n5; ++i) radices->push_back(5);
  for (int i = 0; i < n3; ++i) radices->push_back(3);
  return (int)radices->size() <= kMaxStages;
}

int fft_plan_init(FftPlan* plan, int n) {
  std::vector<int> rad;
  if (!fft_factor(n, &rad)) return COLA_ERR_INVALID;
  plan->dev.n = n;
  plan->dev.nstages = (int)rad.size();
  for (int i = 0; i < kMaxStages; ++i) plan->dev.radix[i] = i < (int)rad.size() ? rad[i] : 1;
  std::vector<float2> h(n);
  for (int t = 0; t < n; ++t) {
    const double ang = -2.0 * M_PI * (double)t / (double)n;
    h[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  if (cudaMalloc(&plan->tw, n * sizeof(float2)) != cudaSuccess) return COLA_ERR_OOM;
  if (cudaMemcpy(plan->tw, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
    return COLA_ERR_CUDA;
  plan->dev.tw = plan->tw;
  static bool attrs_set = false;
  if (!attrs_set) {
    const int mx = 227 * 1024;
    cudaFuncSetAttribute(k_r2c_rows<kSrcFixedPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_r2c_rows<kSrcFloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_c2r_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_pencils<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_pencils<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_green_x, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_r2c_fast<kSrcFixedPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_r2c_fast<kSrcFloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_c2r_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_pencils_fast<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_pencils_fast<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_green_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attrs_set = true;
  }
  return COLA_OK;
}

void fft_set_smem_limits() {
  const int mx = 227 * 1024;
  cudaFuncSetAttribute(k_r2c_rows<kSrcFixedPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_r2c_rows<kSrcFloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_c2r_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pencils<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pencils<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_green_x, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_r2c_fast<kSrcFixedPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_r2c_fast<kSrcFloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_c2r_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pencils_fast<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pencils_fast<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_green_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

void fft_plan_free(FftPlan* plan) {
  if (plan->tw) cudaFree(plan->tw);
  plan->tw = nullptr;
}

int launch_r2c_rows(const FftPlan& p, const Grid3& g, RowSource kind, const void* src,
                    long long src_row_stride, float scale, float2* dst, cudaStream_t st,
                    unsigned long long* mass_acc) {
  const long long nrows = (long long)g.rows();
  FastPlan fp;
  if (fast_plan(p, &fp)) {
    const TileShape t = fast_shape(g.n, 1 << 20, fp.nst >= 2 ? 2 : 1);
    const long long blocks = (nrows + (2LL << t.lw) - 1) / (2LL << t.lw);
    if (kind == kSrcFixedPoint)
      k_r2c_fast<kSrcFixedPoint><<<(unsigned)blocks, t.threads, t.smem, st>>>(fp, t.lw, src, src_row_stride, scale,
                                                                              dst, g.pc, nrows, mass_acc);
    else
      k_r2c_fast<kSrcFloat><<<(unsigned)blocks, t.threads, t.smem, st>>>(fp, t.lw, src, src_row_stride, scale, dst,
                                                                         g.pc, nrows, nullptr);
    return check_launch("r2c_fast");
  }
  const TileShape t = tile_shape(g.n, 1 << 20);
  const long long blocks = (nrows + (2LL << t.lw) - 1) / (2LL << t.lw);
  if (kind == kSrcFixedPoint)
    k_r2c_rows<kSrcFixedPoint><<<(unsigned)blocks, t.threads, t.smem, st>>>(p.dev, t.lw, src, src_row_stride,
                                                                            scale, dst, g.pc, nrows, mass_acc);
  else
    k_r2c_rows<kSrcFloat><<<(unsigned)blocks, t.threads, t.smem, st>>>(p.dev, t.lw, src, src_row_stride, scale,
                                                                       dst, g.pc, nrows, nullptr);
  return check_launch("r2c_rows");
}

int launch_c2r_rows(const FftPlan& p, const Grid3& g, float2* data, cudaStream_t st) {
  const long long nrows = (long long)g.rows();
  FastPlan fp;
  if (fast_plan(p, &fp)) {
    const TileShape t = fast_shape(g.n, 1 << 20, fp.nst >= 3 ? 2 : 1);
    const long long blocks = (nrows + (2LL << t.lw) - 1) / (2LL << t.lw);
    k_c2r_fast<<<(unsigned)blocks, t.threads, t.smem, st>>>(fp, t.lw, data, g.pc, nrows);
    return check_launch("c2r_fast");
  }
  const TileShape t = tile_shape(g.n, 1 << 20);
  const long long blocks = (nrows + (2LL << t.lw) - 1) / (2LL << t.lw);
  k_c2r_rows<<<(unsigned)blocks, t.threads, t.smem, st>>>(p.dev, t.lw, data, g.pc, nrows);
  return check_launch("c2r_rows");
}

int launch_pencils(const FftPlan& p, const Grid3& g, int axis, int dir, float2* data, cudaStream_t st) {
  const long long plane = (long long)g.n * g.pc;
  const long long jstride = axis == 1 ? g.pc : plane;
  const long long ostride = axis == 1 ? plane : g.pc;
  FastPlan fp;
  if (fast_plan(p, &fp)) {
    const TileShape t = fast_shape(g.n, largest_pow2_le(g.nc), fp.nst >= 3 ? 2 : 1);
    dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
    if (dir < 0) k_pencils_fast<-1><<<grid, t.threads, t.smem, st>>>(fp, t.lw, data, jstride, ostride, g.nc);
    else k_pencils_fast<+1><<<grid, t.threads, t.smem, st>>>(fp, t.lw, data, jstride, ostride, g.nc);
    return check_launch("pencils_fast");
  }
  const TileShape t = tile_shape(g.n, largest_pow2_le(g.nc));
  dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
  if (dir < 0)
    k_pencils<-1><<<grid, t.threads, t.smem, st>>>(p.dev, t.lw, data, jstride, ostride, g.nc);
  else
    k_pencils<+1><<<grid, t.threads, t.smem, st>>>(p.dev, t.lw, data, jstride, ostride, g.nc);
  return check_launch("pencils");
}

int launch_green_x(const FftPlan& p, const Grid3& g, const float2* in, float2* const out[3],
                   const float* dtab, float scale, cudaStream_t st) {
  const double kf = 2.0 * M_PI / g.n;
  const double n3 = (double)g.n * g.n * g.n;
  const float g_scale = (float)((double)scale / (kf * kf * n3));
  FastPlan fp;
  if (fast_plan(p, &fp)) {
    const TileShape t = fast_shape(g.n, largest_pow2_le(g.nc), fp.nst >= 3 ? 2 : 1);
    dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
    k_green_fast<<<grid, t.threads, t.smem, st>>>(fp, t.lw, in, out[0], out[1], out[2], g.pc, g.nc, dtab, g_scale);
    return check_launch("green_fast");
  }
  const TileShape t = tile_shape(g.n, largest_pow2_le(g.nc));
  dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
  k_green_x<<<grid, t.threads, t.smem, st>>>(p.dev, t.lw, in, out[0], out[1], out[2], g.pc, g.nc, dtab, g_scale);
  return check_launch("green_x");
}

}  // namespace cola
