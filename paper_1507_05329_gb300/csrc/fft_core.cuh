// Device building blocks of the hand-written mixed-radix 3D FFT passes (sm_103a), shared by the
// FFT translation units.  Hand-written mixed-radix 3D FFT passes for the PM force:
//
// The paper's PM force spends 66% of its time in FFTW (§2.3, Table 1).  Here each 1D pass of the
// 3D transform is one kernel that reads a tile of W pencils from HBM once, transforms it in shared
// memory with Stockham autosort stages of radix 16/8/5/4/3/2, and writes it once:
//   * contiguous axis (z): pairs of real rows packed as one complex row (R2C / C2R);
//   * strided axes (y, x): W adjacent complex columns per tile, so each row segment is a
//     contiguous W*8-byte run;
//   * the last forward pass (x) is fused with the Poisson Green function, the 4-point gradient
//     kernel and the inverse x transforms of the force components (§2.2 Poisson equation): F_x
//     has its own, F_y and F_z share one (their gradient factors are constant along x).
// Shared-memory layout of a tile: element (j, w) at ((j + j/16) * W + w); the skew of one W-row
// every 16 rows keeps the stride-R writes of the first Stockham stages off a single bank group.
#pragma once
#include "cola_internal.h"

#include <cmath>
#include <cstdio>
#include <mutex>
#include <unordered_set>

namespace cola {
namespace fftk {

constexpr int kEpt = 16;   // complex elements per thread (register staging of a stage)
constexpr int kMaxThreads = 384;   // largest tile (6144 elements) / kEpt
constexpr int kWideThreads = 768;  // wide tiles: 8 pencils of up to 1536 elements / kEpt

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

// 6 = 2 x 3: radix 2 first, a_j = x_j + x_{j+3} and b_j = (x_j - x_{j+3}) w6^j, then a 3-point DFT of
// each; the even outputs come from a, the odd from b.
template <int DIR> struct Dft<6, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    const float h = 0.86602540378443865f;   // sqrt(3)/2
    float2 a[3] = {v[0] + v[3], v[1] + v[4], v[2] + v[5]};
    float2 b[3] = {v[0] - v[3], v[1] - v[4], v[2] - v[5]};
    b[1] = cmul(b[1], make_float2(0.5f, DIR * h));
    b[2] = cmul(b[2], make_float2(-0.5f, DIR * h));
    Dft<3, DIR>::run(a);
    Dft<3, DIR>::run(b);
    v[0] = a[0];
    v[1] = b[0];
    v[2] = a[1];
    v[3] = b[1];
    v[4] = a[2];
    v[5] = b[2];
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
      case 6: fft_stage<6, DIR>(a, b, p.n, lw, ns, p.tw, tid, nthreads); break;
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
  // Padded row steps of a shared tile (saddr) along the stage's two strides, 0 where the padding
  // is not affine along them: rows j0 + r n/R sit at saddr(j0) + r nbp W, rows j0 + r ns at
  // saddr(j0) + r nsp W (checked exhaustively on the host when the plan is made).
  int nbp[kMaxStages];
  int nsp[kMaxStages];
  const float2* tw;
};

// The three-stage plans that have kernels specialised for them: 1 = 16 x 8 x 8 (1024 points),
// 2 = 16 x 16 x 5 (1280), 3 = 16 x 16 x 6 (1536); 0 for any other plan.
inline int plan3_id(const FastPlan& fp) {
  if (fp.nst != 3 || fp.radix[0] != 16) return 0;
  if (fp.radix[1] == 8 && fp.radix[2] == 8) return 1;
  if (fp.radix[1] == 16 && fp.radix[2] == 5) return 2;
  if (fp.radix[1] == 16 && fp.radix[2] == 6) return 3;
  return 0;
}

template <int DIR>
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int t) {
  float2 v = __ldg(&tw[t]);
  if (DIR > 0) v.y = -v.y;
  return v;
}

// Twiddle multiplies of butterfly k of stage s, v[r] *= w^(r k tstr_s) (conjugated for DIR > 0),
// r = 1..R-1.  TWF: all R-1 twiddles are loaded before the first multiply (fewer registers held
// across the loads in the strided y passes); else each load feeds its multiply.  Same products.
template <int R, int DIR, bool TWF>
__device__ __forceinline__ void apply_twiddles(const FastPlan& p, int s, int k, float2 (&v)[R]) {
  const int tstr = p.tstr[s];
  if constexpr (TWF) {
    float2 t[R];
#pragma unroll
    for (int r = 1; r < R; ++r) t[r] = twid<DIR>(p.tw, r * k * tstr);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], t[r]);
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twid<DIR>(p.tw, r * k * tstr));
  }
}
template <int R, int DIR, bool TWF>
__device__ __forceinline__ void apply_twiddles2(const FastPlan& p, int s, int k, float2 (&va)[R], float2 (&vb)[R]) {
  const int tstr = p.tstr[s];
  if constexpr (TWF) {
    float2 t[R];
#pragma unroll
    for (int r = 1; r < R; ++r) t[r] = twid<DIR>(p.tw, r * k * tstr);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      va[r] = cmul(va[r], t[r]);
      vb[r] = cmul(vb[r], t[r]);
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const float2 t = twid<DIR>(p.tw, r * k * tstr);
      va[r] = cmul(va[r], t);
      vb[r] = cmul(vb[r], t);
    }
  }
}

struct SmemR {
  const float2* s;
  int lw;
  __device__ __forceinline__ float2 operator()(int j, int w) const { return s[saddr(j, w, lw)]; }
  __device__ __forceinline__ float4 ld2(int j, int w) const {
    return *reinterpret_cast<const float4*>(s + saddr(j, w, lw));
  }
};
struct SmemW {
  float2* s;
  int lw;
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const { s[saddr(j, w, lw)] = v; }
  __device__ __forceinline__ void st2(int j, int w, float4 v) const {
    *reinterpret_cast<float4*>(s + saddr(j, w, lw)) = v;
  }
};
template <class T>
struct SmemAcc {
  static constexpr bool value = false;
};
template <>
struct SmemAcc<SmemR> {
  static constexpr bool value = true;
};
template <>
struct SmemAcc<SmemW> {
  static constexpr bool value = true;
};

// Rows j0 + r d (r < R) of column w.  In a shared tile whose padding is affine along d (padded
// step dp > 0) the addresses are one pointer plus multiples of a fixed step; elsewhere each row
// goes through the accessor.
template <int R, class Src>
__device__ __forceinline__ void load_rows(const Src& src, int j0, int d, int dp, int lw, int w, float2 (&v)[R]) {
  if constexpr (SmemAcc<Src>::value) {
    if (dp) {
      const float2* q = src.s + saddr(j0, w, lw);
      const int st = dp << lw;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = q[r * st];
      return;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = src(j0 + r * d, w);
}
template <int R, class Dst>
__device__ __forceinline__ void store_rows(const Dst& dst, int j0, int d, int dp, int lw, int w, const float2 (&v)[R]) {
  if constexpr (SmemAcc<Dst>::value) {
    if (dp) {
      float2* q = dst.s + saddr(j0, w, lw);
      const int st = dp << lw;
#pragma unroll
      for (int r = 0; r < R; ++r) q[r * st] = v[r];
      return;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) dst(j0 + r * d, w, v[r]);
}

// Pencil pairs: with two or more pencils per tile a thread takes the same butterfly of two
// adjacent pencils, so the twiddles and index arithmetic are shared and every shared/global
// access moves 16 bytes.
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// Column pairs (w, w + 1) of rows j0 + r d, as load_rows and store_rows (w even: 16-byte accesses).
template <int R, class Src>
__device__ __forceinline__ void load_rows2(const Src& src, int j0, int d, int dp, int lw, int w, float2 (&va)[R],
                                           float2 (&vb)[R]) {
  if constexpr (SmemAcc<Src>::value) {
    if (dp) {
      const float2* q = src.s + saddr(j0, w, lw);
      const int st = dp << lw;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float4 t = *reinterpret_cast<const float4*>(q + r * st);
        va[r] = make_float2(t.x, t.y);
        vb[r] = make_float2(t.z, t.w);
      }
      return;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float4 t = src.ld2(j0 + r * d, w);
    va[r] = make_float2(t.x, t.y);
    vb[r] = make_float2(t.z, t.w);
  }
}
template <int R, class Dst>
__device__ __forceinline__ void store_rows2(const Dst& dst, int j0, int d, int dp, int lw, int w, const float2 (&va)[R],
                                            const float2 (&vb)[R]) {
  if constexpr (SmemAcc<Dst>::value) {
    if (dp) {
      float2* q = dst.s + saddr(j0, w, lw);
      const int st = dp << lw;
#pragma unroll
      for (int r = 0; r < R; ++r) *reinterpret_cast<float4*>(q + r * st) = pack2(va[r], vb[r]);
      return;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) dst.st2(j0 + r * d, w, pack2(va[r], vb[r]));
}

template <int R, int DIR, class Src, class Dst, int EPT, bool TWF = false>
__device__ __forceinline__ void fwd_stage_pairs(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst,
                                                int tid, int nthreads) {
  constexpr int kB = (EPT + 2 * R - 1) / (2 * R);
  const int nb = p.n / R, lwp = lw - 1, total = nb << lwp, lns = p.lns[s];
  const int wm = (1 << lwp) - 1, km = (1 << lns) - 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nthreads;
    if (idx < total) {
      const int w = (idx & wm) << 1, b = idx >> lwp, k = b & km;
      float2 va[R], vb[R];
      load_rows2<R>(src, b, nb, p.nbp[s], lw, w, va, vb);
      if (lns) apply_twiddles2<R, DIR, TWF>(p, s, k, va, vb);
      Dft<R, DIR>::run(va);
      Dft<R, DIR>::run(vb);
      const int base = (((b >> lns) * R) << lns) + k;
      store_rows2<R>(dst, base, 1 << lns, p.nsp[s], lw, w, va, vb);
    }
  }
}

template <int R, int DIR, class Src, class Dst, int EPT, bool TWF = false>
__device__ __forceinline__ void tr_stage_pairs(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst,
                                               int tid, int nthreads) {
  constexpr int kB = (EPT + 2 * R - 1) / (2 * R);
  const int nb = p.n / R, lwp = lw - 1, total = nb << lwp, lns = p.lns[s];
  const int wm = (1 << lwp) - 1, km = (1 << lns) - 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nthreads;
    if (idx < total) {
      const int w = (idx & wm) << 1, b = idx >> lwp, k = b & km;
      const int base = (((b >> lns) * R) << lns) + k;
      float2 va[R], vb[R];
      load_rows2<R>(src, base, 1 << lns, p.nsp[s], lw, w, va, vb);
      Dft<R, DIR>::run(va);
      Dft<R, DIR>::run(vb);
      if (lns) apply_twiddles2<R, DIR, TWF>(p, s, k, va, vb);
      store_rows2<R>(dst, b, nb, p.nbp[s], lw, w, va, vb);
    }
  }
}

// forward (decimation in time) stage s
template <int R, int DIR, class Src, class Dst, int EPT = kEpt, bool TWF = false>
__device__ __forceinline__ void fwd_stage(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                          int nthreads) {
  if (R <= 8 && lw >= 1 && 2 * R <= EPT) {   // pairs of columns: 2R elements per butterfly task
    fwd_stage_pairs<R, DIR, Src, Dst, EPT, TWF>(p, s, lw, src, dst, tid, nthreads);
    return;
  }
  constexpr int kB = (EPT + R - 1) / R;
  const int nb = p.n / R, total = nb << lw, lns = p.lns[s];
  const int wm = (1 << lw) - 1, km = (1 << lns) - 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nthreads;
    if (idx < total) {
      const int w = idx & wm, b = idx >> lw, k = b & km;
      float2 v[R];
      load_rows<R>(src, b, nb, p.nbp[s], lw, w, v);
      if (lns) apply_twiddles<R, DIR, TWF>(p, s, k, v);
      Dft<R, DIR>::run(v);
      const int base = (((b >> lns) * R) << lns) + k;
      store_rows<R>(dst, base, 1 << lns, p.nsp[s], lw, w, v);
    }
  }
}

// transposed stage s (used in reverse order for the inverse transform)
template <int R, int DIR, class Src, class Dst, int EPT = kEpt, bool TWF = false>
__device__ __forceinline__ void tr_stage(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                         int nthreads) {
  if (R <= 8 && lw >= 1 && 2 * R <= EPT) {   // pairs of columns: 2R elements per butterfly task
    tr_stage_pairs<R, DIR, Src, Dst, EPT, TWF>(p, s, lw, src, dst, tid, nthreads);
    return;
  }
  constexpr int kB = (EPT + R - 1) / R;
  const int nb = p.n / R, total = nb << lw, lns = p.lns[s];
  const int wm = (1 << lw) - 1, km = (1 << lns) - 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nthreads;
    if (idx < total) {
      const int w = idx & wm, b = idx >> lw, k = b & km;
      const int base = (((b >> lns) * R) << lns) + k;
      float2 v[R];
      load_rows<R>(src, base, 1 << lns, p.nsp[s], lw, w, v);
      Dft<R, DIR>::run(v);
      if (lns) apply_twiddles<R, DIR, TWF>(p, s, k, v);
      store_rows<R>(dst, b, nb, p.nbp[s], lw, w, v);
    }
  }
}

// MAXR: the largest radix the kernel is compiled for (8 or 16); radix-16 code is left out of the
// kernels of plans that do not use it, which keeps their register count down.
template <bool TR, int DIR, int MAXR, class Src, class Dst>
__device__ __forceinline__ void any_stage(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                          int nt) {
  switch (p.radix[s]) {
    case 16:
      if constexpr (MAXR >= 16) {
        TR ? tr_stage<16, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<16, DIR>(p, s, lw, src, dst, tid, nt);
      }
      break;
    case 8: TR ? tr_stage<8, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<8, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 6: TR ? tr_stage<6, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<6, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 5: TR ? tr_stage<5, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<5, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 4: TR ? tr_stage<4, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<4, DIR>(p, s, lw, src, dst, tid, nt); break;
    case 3: TR ? tr_stage<3, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<3, DIR>(p, s, lw, src, dst, tid, nt); break;
    default: TR ? tr_stage<2, DIR>(p, s, lw, src, dst, tid, nt) : fwd_stage<2, DIR>(p, s, lw, src, dst, tid, nt); break;
  }
}

template <bool TR, int DIR, int MAXR, int EPT, class Src, class Dst>
__device__ __forceinline__ void any_stage_e(const FastPlan& p, int s, int lw, const Src& src, const Dst& dst, int tid,
                                            int nt) {
  switch (p.radix[s]) {
    case 16:
      if constexpr (MAXR >= 16) {
        TR ? tr_stage<16, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt)
           : fwd_stage<16, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt);
      }
      break;
    case 8: TR ? tr_stage<8, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt) : fwd_stage<8, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt); break;
    case 6: TR ? tr_stage<6, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt) : fwd_stage<6, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt); break;
    case 5: TR ? tr_stage<5, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt) : fwd_stage<5, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt); break;
    case 4: TR ? tr_stage<4, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt) : fwd_stage<4, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt); break;
    case 3: TR ? tr_stage<3, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt) : fwd_stage<3, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt); break;
    default: TR ? tr_stage<2, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt) : fwd_stage<2, DIR, Src, Dst, EPT>(p, s, lw, src, dst, tid, nt); break;
  }
}


// A stage that overwrites its input buffer: each thread reads the rows of all its butterflies into
// registers, the block synchronises, and the results go back to the same buffer (one work buffer
// instead of two, one barrier more).  Only middle stages, whose radix is a power of two in a fast
// plan, so a thread's EPT = 16 values fill one register array whatever the radix; the barrier sits
// outside the radix switch.  The caller synchronises before the next stage reads.
template <int R, bool TR, int EPT>
__device__ __forceinline__ void inplace_read(const FastPlan& p, int s, int lw, const float2* buf, int tid, int nt,
                                             float2 (&v)[EPT]) {
  constexpr int kB = EPT / R;
  const int nb = p.n / R, total = nb << lw, lns = p.lns[s];
  const int wm = (1 << lw) - 1, km = (1 << lns) - 1;
  const SmemR src{buf, lw};
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nt;
    if (idx < total) {
      const int w = idx & wm, b = idx >> lw, k = b & km;
      float2 t[R];
      if (TR) load_rows<R>(src, (((b >> lns) * R) << lns) + k, 1 << lns, p.nsp[s], lw, w, t);
      else load_rows<R>(src, b, nb, p.nbp[s], lw, w, t);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i * R + r] = t[r];
    }
  }
}

template <int R, int DIR, bool TR, int EPT>
__device__ __forceinline__ void inplace_write(const FastPlan& p, int s, int lw, float2* buf, int tid, int nt,
                                              const float2 (&v)[EPT]) {
  constexpr int kB = EPT / R;
  const int nb = p.n / R, total = nb << lw, lns = p.lns[s];
  const int wm = (1 << lw) - 1, km = (1 << lns) - 1;
  const SmemW dst{buf, lw};
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nt;
    if (idx < total) {
      const int w = idx & wm, b = idx >> lw, k = b & km;
      float2 t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = v[i * R + r];
      if (!TR && lns) apply_twiddles<R, DIR, true>(p, s, k, t);
      Dft<R, DIR>::run(t);
      if (TR && lns) apply_twiddles<R, DIR, true>(p, s, k, t);
      if (TR) store_rows<R>(dst, b, nb, p.nbp[s], lw, w, t);
      else store_rows<R>(dst, (((b >> lns) * R) << lns) + k, 1 << lns, p.nsp[s], lw, w, t);
    }
  }
}

template <bool TR, int DIR, int MAXR, int EPT>
__device__ __forceinline__ void inplace_stage(const FastPlan& p, int s, int lw, float2* buf, int tid, int nt) {
  static_assert(EPT == 16, "in-place stages hold 16 values per thread");
  float2 v[EPT];
  const int R = p.radix[s];
  if (MAXR >= 16 && R == 16) inplace_read<(MAXR >= 16 ? 16 : 8), TR, EPT>(p, s, lw, buf, tid, nt, v);
  else if (R == 8) inplace_read<8, TR, EPT>(p, s, lw, buf, tid, nt, v);
  else if (R == 4) inplace_read<4, TR, EPT>(p, s, lw, buf, tid, nt, v);
  else inplace_read<2, TR, EPT>(p, s, lw, buf, tid, nt, v);
  __syncthreads();
  if (MAXR >= 16 && R == 16) inplace_write<(MAXR >= 16 ? 16 : 8), DIR, TR, EPT>(p, s, lw, buf, tid, nt, v);
  else if (R == 8) inplace_write<8, DIR, TR, EPT>(p, s, lw, buf, tid, nt, v);
  else if (R == 4) inplace_write<4, DIR, TR, EPT>(p, s, lw, buf, tid, nt, v);
  else inplace_write<2, DIR, TR, EPT>(p, s, lw, buf, tid, nt, v);
}


// Forward transform of a tile: stage 0 reads gsrc, the last stage writes gdst, shared memory
// (buffers a, b) in between.  Ends with a barrier only when the caller asks (sync_end).
template <int DIR, int MAXR, class GSrc, class GDst, int EPT = kEpt>
__device__ __forceinline__ void fwd_tile(const FastPlan& p, int lw, float2* a, float2* b, const GSrc& gsrc,
                                         const GDst& gdst, int tid, int nt) {
  const int m = p.nst;
  if (m == 1) {
    any_stage_e<false, DIR, MAXR, EPT>(p, 0, lw, gsrc, gdst, tid, nt);
    return;
  }
  any_stage_e<false, DIR, MAXR, EPT>(p, 0, lw, gsrc, SmemW{a, lw}, tid, nt);
  __syncthreads();
  for (int s = 1; s < m - 1; ++s) {
    any_stage_e<false, DIR, MAXR, EPT>(p, s, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  any_stage_e<false, DIR, MAXR, EPT>(p, m - 1, lw, SmemR{a, lw}, gdst, tid, nt);
}

// Inverse transform of a tile by the transposed stages m-1 .. 0.  R0, R1, R2 > 0: the plan has exactly
// three stages of those radices (compile-time stage code, the same butterflies in the same order).
template <int DIR, int MAXR, class GSrc, class GDst, int EPT = kEpt, int R0 = 0, int R1 = 0, int R2 = 0>
__device__ __forceinline__ void inv_tile(const FastPlan& p, int lw, float2* a, float2* b, const GSrc& gsrc,
                                         const GDst& gdst, int tid, int nt) {
  if constexpr (R0 > 0) {
    tr_stage<R2, DIR, GSrc, SmemW, EPT>(p, 2, lw, gsrc, SmemW{a, lw}, tid, nt);
    __syncthreads();
    tr_stage<R1, DIR, SmemR, SmemW, EPT>(p, 1, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
    __syncthreads();
    tr_stage<R0, DIR, SmemR, GDst, EPT>(p, 0, lw, SmemR{b, lw}, gdst, tid, nt);
    return;
  }
  const int m = p.nst;
  if (m == 1) {
    any_stage_e<true, DIR, MAXR, EPT>(p, 0, lw, gsrc, gdst, tid, nt);
    return;
  }
  any_stage_e<true, DIR, MAXR, EPT>(p, m - 1, lw, gsrc, SmemW{a, lw}, tid, nt);
  __syncthreads();
  for (int s = m - 2; s > 0; --s) {
    any_stage_e<true, DIR, MAXR, EPT>(p, s, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  any_stage_e<true, DIR, MAXR, EPT>(p, 0, lw, SmemR{a, lw}, gdst, tid, nt);
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
  __device__ __forceinline__ float4 ld2(int j, int w) const {
    if (w + 1 < cols_left) return *reinterpret_cast<const float4*>(base + j * jstride + w);
    return pack2((*this)(j, w), (*this)(j, w + 1));
  }
  __device__ __forceinline__ void st2(int j, int w, float4 v) const {
    if (w + 1 < cols_left) *reinterpret_cast<float4*>(base + j * jstride + w) = v;
    else if (w < cols_left) base[j * jstride + w] = make_float2(v.x, v.y);
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
        a = fixed_to_delta(va, scale);
        mlo += va;
        mhi += (mlo < va);
      }
      if (ra + 1 < nrows) {
        const unsigned long long vb = s[(ra + 1) * rs + j];
        b = fixed_to_delta(vb, scale);
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
  __device__ __forceinline__ float4 ld2(int j, int w) const { return pack2((*this)(j, w), (*this)(j, w + 1)); }
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
  __device__ __forceinline__ float4 ld2(int k, int w) const { return pack2((*this)(k, w), (*this)(k, w + 1)); }
};

struct RealPairDst {   // (re, im) -> real rows (2w, 2w+1)
  float* out;
  long long rs, row0, nrows;
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const {
    const long long ra = row0 + 2 * w;
    if (ra < nrows) out[ra * rs + j] = v.x;
    if (ra + 1 < nrows) out[(ra + 1) * rs + j] = v.y;
  }
  __device__ __forceinline__ void st2(int j, int w, float4 v) const {
    (*this)(j, w, make_float2(v.x, v.y));
    (*this)(j, w + 1, make_float2(v.z, v.w));
  }
};

struct DenseScaledDst {   // (re, im) -> scale x (re, im) in dense rows (2w, 2w+1) of n floats
  float* out;
  long long n, row0, nrows;
  float scale;
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const {
    const long long ra = row0 + 2 * w;
    if (ra < nrows) out[ra * n + j] = v.x * scale;
    if (ra + 1 < nrows) out[(ra + 1) * n + j] = v.y * scale;
  }
  __device__ __forceinline__ void st2(int j, int w, float4 v) const {
    (*this)(j, w, make_float2(v.x, v.y));
    (*this)(j, w + 1, make_float2(v.z, v.w));
  }
};

__device__ __forceinline__ int fast_tile_elems(int n, int lw) { return (n + n / 16 + 1) << lw; }

// Writes i dy v to base1 and i dz[w] v to base2 (W adjacent columns of two strided pencils).
struct PencilG2 {
  float2* base1;
  float2* base2;
  long long jstride;
  int cols_left;   // nc - col0
  float dy;
  const float* dz;   // gradient kernel at the tile's columns
  __device__ __forceinline__ void operator()(int j, int w, float2 v) const {
    if (w < cols_left) {
      const float d = dz[w];
      base1[j * jstride + w] = make_float2(-dy * v.y, dy * v.x);
      base2[j * jstride + w] = make_float2(-d * v.y, d * v.x);
    }
  }
  __device__ __forceinline__ void st2(int j, int w, float4 v) const {
    if (w + 1 < cols_left) {
      const float d0 = dz[w], d1 = dz[w + 1];
      *reinterpret_cast<float4*>(base1 + j * jstride + w) = make_float4(-dy * v.y, dy * v.x, -dy * v.w, dy * v.z);
      *reinterpret_cast<float4*>(base2 + j * jstride + w) = make_float4(-d0 * v.y, d0 * v.x, -d1 * v.w, d1 * v.z);
    } else {
      (*this)(j, w, make_float2(v.x, v.y));
    }
  }
};

// Inverse x transform of the register-resident spectrum (times i D_x(k_x) when GRADX) into gout:
// the transposed last stage straight from registers, then the remaining stages in shared memory.
// R0, R1 > 0: the plan has exactly three stages of radices R0, R1, RL (compile-time stage code).
template <int RL, int MAXR, int EPT, bool GRADX, class GDst, int R0 = 0, int R1 = 0>
__device__ __forceinline__ void green_inverse(const FastPlan& p, int lw, const float2 (&spec)[(EPT + RL - 1) / RL][RL],
                                              const float* __restrict__ dtab, const GDst& gout, float2* a, float2* b) {
  constexpr int kB = (EPT + RL - 1) / RL;
  const int n = p.n, tid = threadIdx.x, nt = blockDim.x, m = p.nst;
  const int nb = n / RL, total = nb << lw, wm = (1 << lw) - 1;
  const int ls = p.lns[m - 1], tstr = p.tstr[m - 1];
  float2* cur = a;
  float2* nxt = b;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    const int idx = tid + i * nt;
    if (idx < total) {
      const int w = idx & wm, bb = idx >> lw;
      float2 v[RL];
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        if (GRADX) {
          const float d = dtab[bb + (r << ls)];
          v[r] = make_float2(-d * spec[i][r].y, d * spec[i][r].x);   // i D g delta
        } else {
          v[r] = spec[i][r];
        }
      }
      // transposed last stage (first of the inverse): inputs are exactly v
      Dft<RL, +1>::run(v);
      if (ls) {
#pragma unroll
        for (int r = 1; r < RL; ++r) v[r] = cmul(v[r], twid<+1>(p.tw, r * bb * tstr));
      }
      if (m > 1) store_rows<RL>(SmemW{cur, lw}, bb, nb, p.nbp[m - 1], lw, w, v);
      else store_rows<RL>(gout, bb, nb, 0, lw, w, v);
    }
  }
  if constexpr (R0 > 0) {
    // the middle stage in place in cur (its values read into registers, then written back): the other
    // buffer stays free for the parked spectrum
    __syncthreads();
    {
      float2 w16[EPT];
      inplace_read<R1, true, EPT>(p, 1, lw, cur, tid, nt, w16);
      __syncthreads();
      inplace_write<R1, +1, true, EPT>(p, 1, lw, cur, tid, nt, w16);
    }
    __syncthreads();
    tr_stage<R0, +1, SmemR, GDst, EPT>(p, 0, lw, SmemR{cur, lw}, gout, tid, nt);
    __syncthreads();   // before the next inverse reuses the buffer
  } else if (m > 1) {
    __syncthreads();
    for (int s = m - 2; s > 0; --s) {
      any_stage_e<true, +1, MAXR, EPT>(p, s, lw, SmemR{cur, lw}, SmemW{nxt, lw}, tid, nt);
      __syncthreads();
      float2* t = cur;
      cur = nxt;
      nxt = t;
    }
    any_stage_e<true, +1, MAXR, EPT>(p, 0, lw, SmemR{cur, lw}, gout, tid, nt);
    __syncthreads();   // before the next inverse reuses the buffers
  }
}

// x pass fused with Green function and gradient kernel, spectrum kept in registers between the
// forward transform's last stage and the inverse transforms' first (transposed) stage.  EPT:
// complex elements per thread per stage (16, or 8: twice the threads, half the registers held).
// R0, R1 > 0: the plan has exactly three stages of radices R0, R1, RL (compile-time stage code, the
// same butterflies in the same order: bit-identical results).
template <int RL, int MAXR, int EPT, int R0 = 0, int R1 = 0>
__device__ __forceinline__ void green_body(const FastPlan& p, int lw, const float2* in, float2* out0, float2* out1,
                                           float2* out2, int pc, int nc, const float* __restrict__ dtab,
                                           float g_scale, float2* spec_out) {
  extern __shared__ float2 sm[];
  constexpr int kB = (EPT + RL - 1) / RL;
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
  if constexpr (R0 > 0) {
    fwd_stage<R0, -1, PencilG, SmemW, EPT>(p, 0, lw, gin, SmemW{a, lw}, tid, nt);
    __syncthreads();
    fwd_stage<R1, -1, SmemR, SmemW, EPT>(p, 1, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
    __syncthreads();
    last_in = b;
  } else if (m > 1) {
    any_stage_e<false, -1, MAXR, EPT>(p, 0, lw, gin, SmemW{a, lw}, tid, nt);
    __syncthreads();
    for (int s = 1; s < m - 1; ++s) {
      any_stage_e<false, -1, MAXR, EPT>(p, s, lw, SmemR{a, lw}, SmemW{b, lw}, tid, nt);
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
      if (m > 1) load_rows<RL>(SmemR{last_in, lw}, bb, nb, p.nbp[m - 1], lw, w, spec[i]);
      else load_rows<RL>(gin, bb, nb, 0, lw, w, spec[i]);
      if (ls) {
#pragma unroll
        for (int r = 1; r < RL; ++r) spec[i][r] = cmul(spec[i][r], twid<-1>(p.tw, r * bb * tstr));
      }
      Dft<RL, -1>::run(spec[i]);
      if (spec_out && w < nc - col0) {   // the forward spectrum itself, for a P(k) of the same density
#pragma unroll
        for (int r = 0; r < RL; ++r) spec_out[(long long)(bb + (r << ls)) * jstride + boff + w] = spec[i][r];
      }
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
  // D_y(k_y) and D_z(k_z) are constant along an x pencil, so F_y and F_z are i D_y H and i D_z H of
  // one inverse H = IFFT_x(g delta): two inverse transforms instead of three
  if constexpr (R0 > 0) {
    // three-stage plans: the spectrum is parked in the second buffer (element (r, idx) at r total + idx)
    // while the first inverse runs in place in the first, so it is not held in registers across it
    float2* park = sm + fast_tile_elems(n, lw);
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const int idx = tid + i * nt;
      if (idx < total) {
#pragma unroll
        for (int r = 0; r < RL; ++r) park[r * total + idx] = spec[i][r];
      }
    }
    green_inverse<RL, MAXR, EPT, true, PencilG, R0, R1>(p, lw, spec, dtab, PencilG{out0 + boff, jstride, nc - col0}, sm,
                                                        nullptr);
    float2 spec2[kB][RL];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const int idx = tid + i * nt;
      if (idx < total) {
#pragma unroll
        for (int r = 0; r < RL; ++r) spec2[i][r] = park[r * total + idx];
      }
    }
    green_inverse<RL, MAXR, EPT, false, PencilG2, R0, R1>(
        p, lw, spec2, dtab, PencilG2{out1 + boff, out2 + boff, jstride, nc - col0, dtab[y], dtab + col0}, sm, nullptr);
  } else {
    green_inverse<RL, MAXR, EPT, true, PencilG, R0, R1>(p, lw, spec, dtab, PencilG{out0 + boff, jstride, nc - col0},
                                                        sm, sm + fast_tile_elems(n, lw));
    green_inverse<RL, MAXR, EPT, false, PencilG2, R0, R1>(
        p, lw, spec, dtab, PencilG2{out1 + boff, out2 + boff, jstride, nc - col0, dtab[y], dtab + col0}, sm,
        sm + fast_tile_elems(n, lw));
  }
}

// =============================================================================================
// Persistent, software-pipelined strided passes.  Each CTA walks tiles t = blockIdx.x + i gridDim.x.
// The tile's W columns are fetched with cp.async (16-byte chunks, zero fill beyond nc) into a
// staging buffer S; after stage 0 has consumed S the copy of the next tile is issued, so the HBM
// reads of tile i+1 overlap the shared-memory stages and the global stores of tile i.
// =============================================================================================
constexpr int kPipeEpt = 16;             // complex elements per thread per stage (default; 8 also built)
constexpr int kPipeThreads = 768;

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issue the copy of tile (chunk, outer) into S: n rows of W complex, as W/2 16-byte pieces per row.
__device__ __forceinline__ void fetch_tile(float2* S, const float2* data, long long jstride, long long ostride, int nc,
                                           int n, int lw, int chunk, int outer, int tid, int nt) {
  const int W = 1 << lw, col0 = chunk << lw;
  const float2* base = data + (long long)outer * ostride + col0;
  const int pieces = n * (W >> 1);
  for (int q = tid; q < pieces; q += nt) {
    const int j = q / (W >> 1), w = (q - j * (W >> 1)) * 2;
    const int valid = nc - col0 - w;   // complex values available from this column on
    const int bytes = valid >= 2 ? 16 : (valid == 1 ? 8 : 0);
    cp_async16(S + saddr(j, w, lw), bytes ? (const void*)(base + j * jstride + w) : (const void*)base, bytes);
  }
  cp_async_commit();
}


// Issue the copy of `rows` consecutive complex half rows (row0 ..) of stride pc into S, row-major
// with stride pc, as 16-byte pieces (pc is even); rows past nrows are zero-filled.
__device__ __forceinline__ void fetch_rows(float2* S, const float2* data, int pc, long long row0, long long nrows,
                                           int rows, int tid, int nt) {
  const int per = pc >> 1;
  for (int q = tid; q < rows * per; q += nt) {
    const int r = q / per, c = (q - r * per) * 2;
    const bool ok = row0 + r < nrows;
    cp_async16(S + (long long)r * pc + c, ok ? (const void*)(data + (row0 + r) * pc + c) : (const void*)data,
               ok ? 16 : 0);
  }
  cp_async_commit();
}

// C[k] = A[k] + i B[k] of two Hermitian half rows, read from the staged copy (HalfPairSrc's
// expansion; staged rows past nrows are zero).
struct HalfPairS {
  const float2* s;
  int pc, n;
  __device__ __forceinline__ float2 operator()(int k, int w) const {
    const int nh = n / 2, kk = k <= nh ? k : n - k;
    float2 A = s[(2 * w) * pc + kk], B = s[(2 * w + 1) * pc + kk];
    if (kk == 0 || kk == nh) {
      A.y = 0.f;
      B.y = 0.f;
    }
    return k <= nh ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
  }
  __device__ __forceinline__ float4 ld2(int k, int w) const { return pack2((*this)(k, w), (*this)(k, w + 1)); }
};

// Raises a kernel's dynamic shared-memory limit the first time it is launched on the current
// device (host side; the attribute is per device).
template <class K>
inline void ensure_smem(K kernel) {
  if (first_use_on_device(reinterpret_cast<const void*>(kernel)))
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace fftk

// Launchers of the kernels compiled in the separate FFT translation units.
template <int MAXR, int EPT>
void fast_r2c_launch(const fftk::FastPlan& fp, int lw, unsigned blocks, int threads, size_t smem, int kind,
                     const void* src, long long rs, float scale, float2* dst, int pc, long long nrows,
                     unsigned long long* acc, cudaStream_t st);
template <int MAXR, int EPT>
void fast_c2r_launch(const fftk::FastPlan& fp, int lw, unsigned blocks, int threads, size_t smem, float2* data, int pc,
                     long long nrows, cudaStream_t st);
template <int MAXR>
void fast_pencils_launch(const fftk::FastPlan& fp, int lw, dim3 grid, int threads, size_t smem, int dir, float2* data,
                         long long jstride, long long ostride, int nc, cudaStream_t st);
template <int MAXR, int EPT>
void fast_green_launch(const fftk::FastPlan& fp, int lw, dim3 grid, int threads, size_t smem, const float2* in,
                       float2* const out[3], int pc, int nc, const float* dtab, float g_scale, float2* spec_out,
                       cudaStream_t st);
template <int MAXR>
void c2r_pipe_launch(const fftk::FastPlan& fp, int lw, int ctas, int threads, size_t smem, int ept, float2* data, int pc,
                     long long nrows, long long ntiles, cudaStream_t st);
// The R2C rows of a plan with specialised kernels (plan3_id) by its kernel (as
// fast_r2c_launch<16, EPT>); false (nothing launched) for any other plan.
template <int EPT>
bool plan3_r2c_launch(const fftk::FastPlan& fp, int lw, unsigned blocks, int threads, size_t smem, int kind,
                      const void* src, long long rs, float scale, float2* dst, int pc, long long nrows,
                      unsigned long long* acc, cudaStream_t st);
// The C2R rows of a plan with specialised kernels (plan3_id) by its kernel (EPT elements per
// thread, as fast_c2r_launch<16, EPT>); false (nothing launched) for any other plan.
// out != nullptr: the real rows go to out as dense rows of n floats times scale (the particle
// arrays' layout) and data is only read.
template <int EPT>
bool plan3_c2r_launch(const fftk::FastPlan& fp, int lw, unsigned blocks, int threads, size_t smem, float2* data, int pc,
                      long long nrows, cudaStream_t st, float* out = nullptr, float scale = 1.0f);
// The fused Green pass of a plan with specialised kernels (plan3_id) on tiles of 8 pencils (16 elements
// per thread) by its kernel; false (nothing launched) otherwise.
bool plan3_green_launch(const fftk::FastPlan& fp, int lw, dim3 grid, int threads, size_t smem, const float2* in,
                        float2* const out[3], int pc, int nc, const float* dtab, float g_scale, float2* spec_out,
                        cudaStream_t st);
// The in-place pipelined pass of a plan with specialised kernels (plan3_id) on tiles of 8 pencils (lw 3,
// 16 elements per thread) by its kernel; false (nothing launched) for any other plan or shape.
// mul (inverse passes only): the tile is read from src and multiplied by the 2LPT factor *mul of its
// mode before the transform, which is written to data.
bool plan3_pencils_launch(const fftk::FastPlan& fp, int lw, int ctas, int threads, size_t smem, int dir, float2* data,
                          long long jstride, long long ostride, int nc, int nchunks, int ntiles, cudaStream_t st,
                          const float2* src = nullptr, const IcMul* mul = nullptr);
template <int MAXR>
void pipe_pencils_launch(const fftk::FastPlan& fp, int lw, int ctas, int threads, size_t smem, int dir, int ept,
                         bool inplace, float2* data, long long jstride, long long ostride, int nc, int nchunks,
                         int ntiles, cudaStream_t st);
void generic_r2c_launch(const FftDev& d, int lw, unsigned blocks, int threads, size_t smem, int kind, const void* src,
                        long long rs, float scale, float2* dst, int pc, long long nrows, unsigned long long* acc,
                        cudaStream_t st);
void generic_c2r_launch(const FftDev& d, int lw, unsigned blocks, int threads, size_t smem, float2* data, int pc,
                        long long nrows, cudaStream_t st);
void generic_pencils_launch(const FftDev& d, int lw, dim3 grid, int threads, size_t smem, int dir, float2* data,
                            long long jstride, long long ostride, int nc, cudaStream_t st);
void generic_green_launch(const FftDev& d, int lw, dim3 grid, int threads, size_t smem, const float2* in,
                          float2* const out[3], int pc, int nc, const float* dtab, float g_scale, cudaStream_t st);
void generic_set_smem_limits();

}  // namespace cola
