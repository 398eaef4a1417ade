// Generic FFT kernels: any 2/3/5-smooth length (runtime radix plans, register-staged Stockham
// stages).  Used for lengths whose plans the fast kernels do not cover.
#include "fft_core.cuh"

namespace cola {
using namespace fftk;
namespace {
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
        a = fixed_to_delta(va, scale);
        mlo += va;
        mhi += (mlo < va);
      }
      if (ra + 1 < nrows) {
        const unsigned long long vb = s[(ra + 1) * src_rs + j];
        b = fixed_to_delta(vb, scale);
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
  if (SRC == kSrcFixedPoint && mass_acc) mass_accumulate(mlo, mhi, mass_slot(mass_acc));
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

}  // namespace

void generic_set_smem_limits() {
  const int mx = 227 * 1024;
  cudaFuncSetAttribute(k_r2c_rows<kSrcFixedPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_r2c_rows<kSrcFloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_c2r_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pencils<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pencils<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_green_x, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

void generic_r2c_launch(const FftDev& d, int lw, unsigned blocks, int threads, size_t smem, int kind, const void* src,
                        long long rs, float scale, float2* dst, int pc, long long nrows, unsigned long long* acc,
                        cudaStream_t st) {
  if (kind == kSrcFixedPoint)
    k_r2c_rows<kSrcFixedPoint><<<blocks, threads, smem, st>>>(d, lw, src, rs, scale, dst, pc, nrows, acc);
  else
    k_r2c_rows<kSrcFloat><<<blocks, threads, smem, st>>>(d, lw, src, rs, scale, dst, pc, nrows, nullptr);
}

void generic_c2r_launch(const FftDev& d, int lw, unsigned blocks, int threads, size_t smem, float2* data, int pc,
                        long long nrows, cudaStream_t st) {
  k_c2r_rows<<<blocks, threads, smem, st>>>(d, lw, data, pc, nrows);
}

void generic_pencils_launch(const FftDev& d, int lw, dim3 grid, int threads, size_t smem, int dir, float2* data,
                            long long jstride, long long ostride, int nc, cudaStream_t st) {
  if (dir < 0) k_pencils<-1><<<grid, threads, smem, st>>>(d, lw, data, jstride, ostride, nc);
  else k_pencils<+1><<<grid, threads, smem, st>>>(d, lw, data, jstride, ostride, nc);
}

void generic_green_launch(const FftDev& d, int lw, dim3 grid, int threads, size_t smem, const float2* in,
                          float2* const out[3], int pc, int nc, const float* dtab, float g_scale, cudaStream_t st) {
  k_green_x<<<grid, threads, smem, st>>>(d, lw, in, out[0], out[1], out[2], pc, nc, dtab, g_scale);
}

}  // namespace cola
