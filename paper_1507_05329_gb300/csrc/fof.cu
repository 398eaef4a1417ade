// Friends-of-friends halo finding (§2.3: run on the fly, 19% of the paper's time; §3.2: linking
// length 0.2 times the mean particle separation) on the fixed-point coordinates of the deposit.
//
// Two particles are friends when their periodic distance is at most l; groups are the connected
// components.  Distances are exact integers: G = (q R + rint(s 2^20)) mod N 2^20 per axis,
// l = rint(b (N/N_p) 2^20), and the test d^2 <= l^2 runs in 64-bit integers, so no rounding
// decides a link and the result is bit-identical to any exact implementation.
//   1. G per particle and a cell of side >= l (ncs cells per axis, ncs^3 <= 2^27), counting sort
//      of the particle ids by cell;
//   2. every particle scans the 27 (fewer if ncs < 3) neighbouring cells for friends j > i and
//      joins the two trees (lock-free union-find: a root is hooked, by CAS, to the smaller root);
//   3. full path compression: label = root = smallest id of the group (canonical);
//   4. group sizes by atomics; groups of >= n_min members compacted in increasing label order by
//      a scan; centre of mass from exact 64-bit sums of minimum-image offsets to the root.
#include "cola_internal.h"

#include <cstdio>

namespace cola {
namespace {

constexpr int kFlagIterations = 4;   // union-find did not converge (never expected; reported)

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

// minimum image of a difference in (-modulus, modulus)
__device__ __forceinline__ long long wrap(long long d, long long modulus) {
  const long long h = modulus / 2;
  if (d > h) d -= modulus;
  else if (d < -h) d += modulus;
  return d;
}

// root of x; path splitting (each visited node is pointed at its grandparent).  Parents never
// exceed their children, so the walk ends within n hops.
__device__ __forceinline__ int find_root(int* parent, int x) {
  volatile int* p = parent;
  int cur = x, nxt = p[cur];
  while (nxt != cur) {
    const int nn = p[nxt];
    if (nn != nxt) p[cur] = nn;
    cur = nxt;
    nxt = nn;
  }
  return cur;
}

__device__ __forceinline__ void unite(int* parent, int a, int b, int* flags) {
  for (int it = 0; it < (1 << 22); ++it) {
    a = find_root(parent, a);
    b = find_root(parent, b);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + a, a, b) == a) return;   // hook the larger root under the smaller
  }
  atomicOr(flags, kFlagIterations);
}

__global__ void k_fof_prepare(ParticleGeom pg, const float* __restrict__ s, long long modulus, int ncs,
                              long long* g0, long long* g1, long long* g2, int* key, unsigned* counts,
                              int* parent) {
  const long long n = pg.npart;
  const long long np2 = (long long)pg.np * pg.np;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int qx = (int)(id / np2);
    const long long rem = id - (long long)qx * np2;
    const int qy = (int)(rem / pg.np), qz = (int)(rem - (long long)qy * pg.np);
    const long long a = fixed_coord(qx, s[id], pg.r_fixed, modulus);
    const long long b = fixed_coord(qy, s[n + id], pg.r_fixed, modulus);
    const long long c = fixed_coord(qz, s[2 * n + id], pg.r_fixed, modulus);
    g0[id] = a;
    g1[id] = b;
    g2[id] = c;
    const int cx = (int)(a * ncs / modulus), cy = (int)(b * ncs / modulus), cz = (int)(c * ncs / modulus);
    const int k = (cx * ncs + cy) * ncs + cz;
    key[id] = k;
    atomicAdd(counts + k, 1u);
    parent[id] = (int)id;
  }
}

__global__ void k_fof_scatter(long long n, const int* __restrict__ key, unsigned* cur, int* sorted) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x)
    sorted[atomicAdd(cur + key[id], 1u)] = (int)id;
}

__global__ void k_fof_link(long long n, const long long* __restrict__ g0, const long long* __restrict__ g1,
                           const long long* __restrict__ g2, const int* __restrict__ key,
                           const unsigned* __restrict__ off, const int* __restrict__ sorted, int ncs,
                           long long modulus, long long ell, int* parent, int* flags) {
  const long long ell2 = ell * ell;
  const int lo = ncs >= 3 ? -1 : 0, hi = ncs >= 2 ? 1 : 0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int k = key[id];
    const int cz = k % ncs, cy = (k / ncs) % ncs, cx = k / (ncs * ncs);
    const long long a = g0[id], b = g1[id], c = g2[id];
    for (int dx = lo; dx <= hi; ++dx) {
      const int x = (cx + dx + ncs) % ncs;
      for (int dy = lo; dy <= hi; ++dy) {
        const int y = (cy + dy + ncs) % ncs;
        for (int dz = lo; dz <= hi; ++dz) {
          const int cell = (x * ncs + y) * ncs + (cz + dz + ncs) % ncs;
          const unsigned e = off[cell + 1];
          for (unsigned t = off[cell]; t < e; ++t) {
            const int j = sorted[t];
            if (j <= id) continue;
            const long long d0 = wrap(g0[j] - a, modulus);
            if (d0 > ell || d0 < -ell) continue;
            const long long d1 = wrap(g1[j] - b, modulus);
            if (d1 > ell || d1 < -ell) continue;
            const long long d2 = wrap(g2[j] - c, modulus);
            if (d2 > ell || d2 < -ell) continue;
            if (d0 * d0 + d1 * d1 + d2 * d2 <= ell2) unite(parent, (int)id, j, flags);
          }
        }
      }
    }
  }
}

// label (a separate array: path splitting keeps rewriting parent while roots are written out)
__global__ void k_fof_label(long long n, int* parent, int* label, unsigned* cnt) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int r = find_root(parent, (int)id);
    label[id] = r;
    atomicAdd(cnt + r, 1u);
  }
}

__global__ void k_fof_size(long long n, const int* __restrict__ label, const unsigned* __restrict__ cnt, int n_min,
                           int* size, unsigned* halo_flag) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int r = label[id];
    const unsigned c = cnt[r];
    size[id] = (int)c;
    halo_flag[id] = (r == id && c >= (unsigned)n_min) ? 1u : 0u;
  }
}

__global__ void k_fof_halo_sums(long long n, const int* __restrict__ label, const unsigned* __restrict__ cnt, int n_min,
                                const unsigned* __restrict__ hoff, const long long* __restrict__ g0,
                                const long long* __restrict__ g1, const long long* __restrict__ g2,
                                long long modulus, int capacity, unsigned long long* sums) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int r = label[id];
    if (cnt[r] < (unsigned)n_min) continue;
    const unsigned h = hoff[r];
    if (h >= (unsigned)capacity) continue;
    atomicAdd(sums + h, (unsigned long long)wrap(g0[id] - g0[r], modulus));
    atomicAdd(sums + capacity + h, (unsigned long long)wrap(g1[id] - g1[r], modulus));
    atomicAdd(sums + 2LL * capacity + h, (unsigned long long)wrap(g2[id] - g2[r], modulus));
  }
}

__global__ void k_fof_halo_finish(long long n, const unsigned* __restrict__ halo_flag, const unsigned* __restrict__ cnt,
                                  const unsigned* __restrict__ hoff, const long long* __restrict__ g0,
                                  const long long* __restrict__ g1, const long long* __restrict__ g2,
                                  long long modulus, int capacity, const unsigned long long* __restrict__ sums,
                                  int* halo_label, int* halo_size, double* halo_pos, int* nhalo) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    if (id == 0) *nhalo = (int)hoff[n];
    if (!halo_flag[id]) continue;
    const unsigned h = hoff[id];
    if (h >= (unsigned)capacity) continue;
    const unsigned c = cnt[id];
    if (halo_label) halo_label[h] = (int)id;
    if (halo_size) halo_size[h] = (int)c;
    if (halo_pos) {
      const long long g[3] = {g0[id], g1[id], g2[id]};
      const double mod = (double)modulus;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double com = (double)g[a] + (double)(long long)sums[a * (long long)capacity + h] / (double)c;
        double m = fmod(com, mod);
        if (m < 0.0) m += mod;
        halo_pos[a * (long long)capacity + h] = m / (double)(1LL << kFracBits);
      }
    }
  }
}

}  // namespace

bool fof_geometry(int nmesh, int np, double b, FofGeom* f) {
  const long long modulus = (long long)nmesh << kFracBits;
  const double ell = rint(b * ((double)nmesh / np) * (double)(1LL << kFracBits));
  if (!(ell >= 1.0) || ell > (double)(1LL << 30)) return false;   // d^2 sums stay below 2^62
  f->modulus = modulus;
  f->ell = (long long)ell;
  long long ncs = modulus / f->ell;                                 // cells of side >= l
  if (ncs > 512) ncs = 512;
  if (ncs < 1) ncs = 1;
  f->ncs = (int)ncs;
  f->ncells = (long long)ncs * ncs * ncs;
  return true;
}

int launch_fof(const ParticleGeom& pg, const FofGeom& f, const float* s, const FofBuffers& fb, int n_min, int* label,
               int* size, int* halo_label, int* halo_size, double* halo_pos, int capacity, int* nhalo, int* flags,
               cudaStream_t st) {
  const long long n = pg.npart;
  int e;
  if (cudaMemsetAsync(fb.counts, 0, f.ncells * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(fb.cnt, 0, n * sizeof(unsigned), st) != cudaSuccess)
    return COLA_ERR_CUDA;
  const unsigned gp = grid_for(n, 256);
  k_fof_prepare<<<gp, 256, 0, st>>>(pg, s, f.modulus, f.ncs, fb.g[0], fb.g[1], fb.g[2], fb.key, fb.counts,
                                    fb.parent);
  if ((e = check_launch("fof_prepare")) != COLA_OK) return e;
  if ((e = launch_excl_scan(fb.counts, (int)f.ncells, fb.seg, fb.off, fb.cur, st)) != COLA_OK) return e;
  k_fof_scatter<<<gp, 256, 0, st>>>(n, fb.key, fb.cur, fb.sorted);
  k_fof_link<<<gp, 256, 0, st>>>(n, fb.g[0], fb.g[1], fb.g[2], fb.key, fb.off, fb.sorted, f.ncs, f.modulus, f.ell,
                                 fb.parent, flags);
  k_fof_label<<<gp, 256, 0, st>>>(n, fb.parent, label, fb.cnt);
  k_fof_size<<<gp, 256, 0, st>>>(n, label, fb.cnt, n_min, size, fb.flag);
  if ((e = check_launch("fof_link")) != COLA_OK) return e;
  if ((e = launch_excl_scan(fb.flag, (int)n, fb.seg, fb.hoff, fb.hcur, st)) != COLA_OK) return e;
  const int cap = capacity > 0 ? capacity : 0;
  if (cap > 0 && halo_pos) {
    if (cudaMemsetAsync(fb.sums, 0, 3ULL * cap * sizeof(unsigned long long), st) != cudaSuccess) return COLA_ERR_CUDA;
    k_fof_halo_sums<<<gp, 256, 0, st>>>(n, label, fb.cnt, n_min, fb.hoff, fb.g[0], fb.g[1], fb.g[2], f.modulus, cap,
                                        fb.sums);
  }
  k_fof_halo_finish<<<gp, 256, 0, st>>>(n, fb.flag, fb.cnt, fb.hoff, fb.g[0], fb.g[1], fb.g[2], f.modulus, cap, fb.sums,
                                        halo_label, halo_size, cap > 0 ? halo_pos : nullptr, nhalo);
  return check_launch("fof_halos");
}

}  // namespace cola
