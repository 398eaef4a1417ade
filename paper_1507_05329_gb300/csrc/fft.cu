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
                           float2* __restrict__ dst, int pc, long long nrows) {
  extern __shared__ float2 sm[];
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, wmask = (1 << lw) - 1;
  const long long row0 = (long long)blockIdx.x << (lw + 1);
  for (int idx = tid; idx < (n << lw); idx += nt) {
    const int w = idx & wmask, j = idx >> lw;
    const long long ra = row0 + 2 * w;
    float a = 0.0f, b = 0.0f;
    if (SRC == kSrcFixedPoint) {
      const unsigned long long* s = static_cast<const unsigned long long*>(src);
      if (ra < nrows) a = __ull2float_rn(s[ra * src_rs + j]) * scale - 1.0f;
      if (ra + 1 < nrows) b = __ull2float_rn(s[(ra + 1) * src_rs + j]) * scale - 1.0f;
    } else {
      const float* s = static_cast<const float*>(src);
      if (ra < nrows) a = s[ra * src_rs + j] * scale;
      if (ra + 1 < nrows) b = s[(ra + 1) * src_rs + j] * scale;
    }
    sm[saddr(j, w, lw)] = make_float2(a, b);
  }
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
}

void fft_plan_free(FftPlan* plan) {
  if (plan->tw) cudaFree(plan->tw);
  plan->tw = nullptr;
}

int launch_r2c_rows(const FftPlan& p, const Grid3& g, RowSource kind, const void* src,
                    long long src_row_stride, float scale, float2* dst, cudaStream_t st) {
  const long long nrows = (long long)g.rows();
  const TileShape t = tile_shape(g.n, 1 << 20);
  const long long blocks = (nrows + (2LL << t.lw) - 1) / (2LL << t.lw);
  if (kind == kSrcFixedPoint)
    k_r2c_rows<kSrcFixedPoint><<<(unsigned)blocks, t.threads, t.smem, st>>>(p.dev, t.lw, src, src_row_stride,
                                                                            scale, dst, g.pc, nrows);
  else
    k_r2c_rows<kSrcFloat><<<(unsigned)blocks, t.threads, t.smem, st>>>(p.dev, t.lw, src, src_row_stride, scale,
                                                                       dst, g.pc, nrows);
  return check_launch("r2c_rows");
}

int launch_c2r_rows(const FftPlan& p, const Grid3& g, float2* data, cudaStream_t st) {
  const long long nrows = (long long)g.rows();
  const TileShape t = tile_shape(g.n, 1 << 20);
  const long long blocks = (nrows + (2LL << t.lw) - 1) / (2LL << t.lw);
  k_c2r_rows<<<(unsigned)blocks, t.threads, t.smem, st>>>(p.dev, t.lw, data, g.pc, nrows);
  return check_launch("c2r_rows");
}

int launch_pencils(const FftPlan& p, const Grid3& g, int axis, int dir, float2* data, cudaStream_t st) {
  const TileShape t = tile_shape(g.n, largest_pow2_le(g.nc));
  const long long plane = (long long)g.n * g.pc;
  const long long jstride = axis == 1 ? g.pc : plane;
  const long long ostride = axis == 1 ? plane : g.pc;
  dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
  if (dir < 0)
    k_pencils<-1><<<grid, t.threads, t.smem, st>>>(p.dev, t.lw, data, jstride, ostride, g.nc);
  else
    k_pencils<+1><<<grid, t.threads, t.smem, st>>>(p.dev, t.lw, data, jstride, ostride, g.nc);
  return check_launch("pencils");
}

int launch_green_x(const FftPlan& p, const Grid3& g, const float2* in, float2* const out[3],
                   const float* dtab, float scale, cudaStream_t st) {
  const TileShape t = tile_shape(g.n, largest_pow2_le(g.nc));
  dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
  const double kf = 2.0 * M_PI / g.n;
  const double n3 = (double)g.n * g.n * g.n;
  const float g_scale = (float)((double)scale / (kf * kf * n3));
  k_green_x<<<grid, t.threads, t.smem, st>>>(p.dev, t.lw, in, out[0], out[1], out[2], g.pc, g.nc, dtab, g_scale);
  return check_launch("green_x");
}

}  // namespace cola
