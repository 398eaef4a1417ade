// Seeded Gaussian white noise of the initial conditions (§2.3: Gaussian random modes from a seed).
//
// The paper does not name its generator; this library draws the real-space white noise of the
// N_p^3 Lagrangian lattice from the counter-based generator Philox-4x32-10 (Salmon, Moraes, Dror &
// Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3"), written here from that description:
//   round:  (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
//           M0 = 0xD2511F53, M1 = 0xCD9E8D57; ten rounds, the key advancing by the Weyl constants
//           (0x9E3779B9, 0xBB67AE85) between rounds.
// Site i (particle id) takes counter j = i / 4 = (j lo, j hi, 0, 0) under key (seed lo, seed hi);
// words (x0, x1) serve sites 4j, 4j+1 and (x2, x3) sites 4j+2, 4j+3 through Box-Muller:
// u1 = ((a >> 8) + 1) 2^-24 in (0, 1], u2 = (b >> 8) 2^-24, r = sqrt(-2 ln u1), the pair
// (r cos 2 pi u2, r sin 2 pi u2).  No state: every site is a pure function of (seed, i), so any
// launch shape gives the same field.
#include "cola_internal.h"

#include <cstdio>

namespace cola {
namespace {

struct Words4 {
  unsigned x[4];
};

__device__ __forceinline__ Words4 philox4x32_10(unsigned c0, unsigned c1, unsigned c2, unsigned c3, unsigned k0,
                                                unsigned k1) {
  constexpr unsigned kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u, kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kW0;
      k1 += kW1;
    }
    const unsigned hi0 = __umulhi(kM0, c0), lo0 = kM0 * c0;
    const unsigned hi1 = __umulhi(kM1, c2), lo1 = kM1 * c2;
    const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Words4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ void box_muller(unsigned a, unsigned b, float* z0, float* z1) {
  const float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;   // exact: 24-bit integers
  const float u2 = (float)(b >> 8) * 0x1p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  *z0 = r * cs;
  *z1 = r * sn;
}

// out: real rows of the lattice (site i = row * np + iz at row * rs + iz)
__global__ void k_white_noise(unsigned k0, unsigned k1, long long n, int np, long long rs, float* __restrict__ out) {
  const long long m = (n + 3) >> 2;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
    const Words4 w = philox4x32_10((unsigned)j, (unsigned)(j >> 32), 0u, 0u, k0, k1);
    float z[4];
    box_muller(w.x[0], w.x[1], &z[0], &z[1]);
    box_muller(w.x[2], w.x[3], &z[2], &z[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long i = 4 * j + q;
      if (i < n) {
        const long long row = i / np;
        out[row * rs + (i - row * np)] = z[q];
      }
    }
  }
}

__global__ void k_philox_words(unsigned k0, unsigned k1, long long first, long long count, unsigned* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    const long long j = first + t;
    const Words4 w = philox4x32_10((unsigned)j, (unsigned)(j >> 32), 0u, 0u, k0, k1);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[4 * t + q] = w.x[q];
  }
}

unsigned grid_of(long long work) {
  const long long b = (work + 255) / 256;
  return (unsigned)(b < 152LL * 32 ? (b > 0 ? b : 1) : 152LL * 32);
}

}  // namespace

int launch_white_noise(unsigned long long seed, int np, long long row_stride, float* out, cudaStream_t st) {
  const long long n = (long long)np * np * np;
  k_white_noise<<<grid_of((n + 3) / 4), 256, 0, st>>>((unsigned)seed, (unsigned)(seed >> 32), n, np, row_stride, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "cola: launch of white_noise failed: %s\n", cudaGetErrorString(e));
    return COLA_ERR_CUDA;
  }
  return COLA_OK;
}

int launch_philox_words(unsigned long long seed, long long first, long long count, unsigned* out, cudaStream_t st) {
  k_philox_words<<<grid_of(count), 256, 0, st>>>((unsigned)seed, (unsigned)(seed >> 32), first, count, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "cola: launch of philox_words failed: %s\n", cudaGetErrorString(e));
    return COLA_ERR_CUDA;
  }
  return COLA_OK;
}

}  // namespace cola
