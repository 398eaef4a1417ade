// Spatial binning of particles by mesh column tiles, and the tile-wise CIC deposit and gather.
//
// The particle arrays stay in Lagrangian order (particle id = lattice index).  At late times the
// particles of one lattice plane are spread over tens of mesh planes (§2.3 mesh; displacements of
// ~8 cells rms at a = 1 for the 0.78 Mpc/h cells of the 1536^3 mesh), so visiting them in lattice
// order touches far more mesh than the L2 holds.  Each step therefore
//   1. counts particles per tile of T x T x TZ mesh cells (T = 8 across, TZ = 32 along z) from the
//      fixed-point base cell (the same integer cell as the deposit), with warp-aggregated atomics;
//   2. scans the counts into offsets;
//   3. scatters packed lattice coordinates into their tile's list.  A particle whose base cell
//      lies on an upper face of its tile also goes, as a "spill" entry, to the neighbouring tiles
//      its cloud reaches (at most seven);
//   4. deposits tile by tile: one CTA sums the 8 fixed-point weights of its primary and spill
//      particles that fall inside the tile in shared memory (64-bit integers, exact) and writes
//      the whole tile once with plain stores: no clearing pass and no global atomics on the mesh;
//   5. gathers the force and applies the kick and drift tile by tile (primary entries only): the
//      CTA first copies the tile's force values with a one-cell halo ((T+1)^2 (TZ+1) x 3 floats,
//      32 KB) into shared memory with coalesced loads, then interpolates from shared memory.  The
//      tile index runs fastest along z, so neighbouring tiles (which share halos) run together.
// The order of particles inside a tile's list depends on atomic timing, but neither result does:
// integer sums are order independent and every particle's gather is computed on its own.
#include "cola_internal.h"

#include <cstdio>
#include <type_traits>

namespace cola {
namespace {

constexpr int kThreads = 256;
// Deposit accumulator columns of TZ + 1 cells: without the pad every column of a tile started on the
// same shared-memory bank, and a warp's lanes from two columns with equal z conflicted (24.4 against
// 26.7 ms at 1024^3/1536^3).
constexpr int kDepositPad = 1;
#ifndef COLA_DEPOSIT_MIN_BLOCKS
#define COLA_DEPOSIT_MIN_BLOCKS 8   // resident deposit CTAs per SM the register budget is sized for
#endif

int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "cola: launch of %s failed: %s\n", what, cudaGetErrorString(e));
    return COLA_ERR_CUDA;
  }
  return COLA_OK;
}

// Bin entries hold the lattice coordinates packed as qx << 20 | qy << 10 | qz (np <= 1024).
__device__ __forceinline__ unsigned pack_q(int qx, int qy, int qz) {
  return ((unsigned)qx << 20) | ((unsigned)qy << 10) | (unsigned)qz;
}
__device__ __forceinline__ void unpack_q(unsigned e, int np, int* q, long long* id) {
  q[0] = (int)(e >> 20);
  q[1] = (int)((e >> 10) & 1023u);
  q[2] = (int)(e & 1023u);
  *id = ((long long)q[0] * np + q[1]) * np + q[2];
}

constexpr int kGatherEnt = 1024;   // entries staged in shared memory per tile (4 KB)

// Exact 64-bit shared-memory add from two native 32-bit atomics (low word with carry out).
__device__ __forceinline__ void smem_add64(unsigned long long* p, unsigned long long w) {
  unsigned* h = reinterpret_cast<unsigned*>(p);
  const unsigned lo = (unsigned)w, hi = (unsigned)(w >> 32);
  const unsigned old = atomicAdd(h, lo);
  const unsigned carry = (old + lo) < old ? 1u : 0u;
  if (hi + carry) atomicAdd(h + 1, hi + carry);
}

// warp-aggregated increment of counter[key] for the lanes whose key >= 0; returns the lane's slot
// (old value + rank among equal keys) when want_slot.
__device__ __forceinline__ unsigned agg_inc(unsigned* counter, int key, bool want_slot) {
  const unsigned active = __activemask();
  const unsigned grp = __match_any_sync(active, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  unsigned base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(counter + key, (unsigned)__popc(grp));
  if (!want_slot) return 0;
  base = __shfl_sync(grp, base, leader);
  return base + __popc(grp & ((1u << lane) - 1u));
}

// Bin keys of one particle: primary tile and up to seven spill tiles (-1 = none).  Tile index
// (bx * nt + by) * nz + bz runs fastest along z.
// LT, LZ: compile-time log2 of the tile sides (the common 8 x 8 x 32 tiles), or 0 to read them from b.
template <int LT, int LZ>
__device__ __forceinline__ void tile_keys(const BinGeom& b, int cx, int cy, int cz, int* k) {
  const int lt = LT ? LT : b.lt, lz = LZ ? LZ : b.lz;
  const int bx = cx >> lt, by = cy >> lt, bz = cz >> lz;
  const int m = (1 << lt) - 1, mz = (1 << lz) - 1;
  // with a single tile along an axis the cloud wraps inside the tile itself: no spill there
  const bool sx = b.nt > 1 && (cx & m) == m, sy = b.nt > 1 && (cy & m) == m, sz = b.nz > 1 && (cz & mz) == mz;
  const int bxs[2] = {bx, bx + 1 == b.nt ? 0 : bx + 1};
  const int bys[2] = {by, by + 1 == b.nt ? 0 : by + 1};
  const int bzs[2] = {bz, bz + 1 == b.nz ? 0 : bz + 1};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c >> 2, dy = (c >> 1) & 1, dz = c & 1;
    const bool ok = (!dx || sx) && (!dy || sy) && (!dz || sz);
    k[c] = ok ? (bxs[dx] * b.nt + bys[dy]) * b.nz + bzs[dz] : -1;
  }
}

// Spill keys of a particle from its primary tile key and its three upper-face flags (the keys
// tile_keys gives, without the particle's position).
__device__ __forceinline__ void keys_from_record(const BinGeom& b, unsigned key, unsigned flags, int* k) {
  const int bz = (int)(key % (unsigned)b.nz), bxy = (int)(key / (unsigned)b.nz);
  const int bx = bxy / b.nt, by = bxy - bx * b.nt;
  const bool sx = flags & 1u, sy = flags & 2u, sz = flags & 4u;
  const int bxs[2] = {bx, bx + 1 == b.nt ? 0 : bx + 1};
  const int bys[2] = {by, by + 1 == b.nt ? 0 : by + 1};
  const int bzs[2] = {bz, bz + 1 == b.nz ? 0 : bz + 1};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c >> 2, dy = (c >> 1) & 1, dz = c & 1;
    const bool ok = (!dx || sx) && (!dy || sy) && (!dz || sz);
    k[c] = ok ? (bxs[dx] * b.nt + bys[dy]) * b.nz + bzs[dz] : -1;
  }
}

// Count pass: per-tile primary and spill counts; every particle's rank within its primary tile (the
// aggregated atomic's return) is recorded with its tile key and upper-face flags, so that the scatter
// pass needs neither the positions nor atomics for the primary entries.
//   rec[id] = rank << 32 | flags << 26 | key   (key < 2^26 tiles, flags: x, y, z upper face)
template <int LT, int LZ, bool F32>
__global__ void __launch_bounds__(kThreads) k_bin_count(ParticleGeom pg, BinGeom b, FixedGeo fg,
                                                        const float* __restrict__ s, unsigned* cnt_p, unsigned* cnt_s,
                                                        unsigned long long* __restrict__ rec) {
  const long long n = pg.npart;
  const int np = pg.np;
  const long long nrows = (long long)np * np;
  const int lt = LT ? LT : b.lt, lz = LZ ? LZ : b.lz;
  const int m = (1 << lt) - 1, mz = (1 << lz) - 1;
  // the block walks (row, chunk) pairs; the positions of the next pair are loaded before this
  // pair's atomics, so the two latencies overlap
  const int nch = (np + (int)blockDim.x - 1) / (int)blockDim.x;
  long long row = blockIdx.x;
  int ch = 0;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f;
  auto load = [&](long long r, int c, float& a0, float& a1, float& a2) {
    const int qz = c * (int)blockDim.x + (int)threadIdx.x;
    if (qz < np) {
      const long long id = r * np + qz;
      a0 = __ldg(s + id);
      a1 = __ldg(s + n + id);
      a2 = __ldg(s + 2 * n + id);
    }
  };
  if (row < nrows) load(row, 0, p0, p1, p2);
  while (row < nrows) {
    long long nrow = row;
    int nchk = ch + 1;
    if (nchk == nch) {
      nchk = 0;
      nrow += gridDim.x;
    }
    float n0 = 0.f, n1 = 0.f, n2 = 0.f;
    if (nrow < nrows) load(nrow, nchk, n0, n1, n2);
    const int qx = (int)(row / np), qy = (int)(row - (long long)qx * np);
    // whole warps walk the row together so that the warp-aggregated atomics see full warps
    const int qz = ch * (int)blockDim.x + (int)threadIdx.x;
    const bool live = qz < np;
    int k[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    unsigned flags = 0;
    if (live) {
      int cx, cy, cz, f;
      cell_frac<F32>(qx, p0, fg, &cx, &f);
      cell_frac<F32>(qy, p1, fg, &cy, &f);
      cell_frac<F32>(qz, p2, fg, &cz, &f);
      tile_keys<LT, LZ>(b, cx, cy, cz, k);
      flags = (b.nt > 1 && (cx & m) == m ? 1u : 0u) | (b.nt > 1 && (cy & m) == m ? 2u : 0u) |
              (b.nz > 1 && (cz & mz) == mz ? 4u : 0u);
    }
    if (__any_sync(__activemask(), live)) {
      // primary keys are shared by runs of lanes: one aggregated atomic per run
      const unsigned rank = agg_inc(cnt_p, k[0], true);
      if (live) rec[row * np + qz] = ((unsigned long long)rank << 32) | ((unsigned long long)flags << 26) | (unsigned)k[0];
    }
    // spill keys are sparse: one atomic per entry (its result unused)
#pragma unroll
    for (int e = 1; e < 8; ++e)
      if (k[e] >= 0) atomicAdd(cnt_s + k[e], 1u);
    row = nrow;
    ch = nchk;
    p0 = n0;
    p1 = n1;
    p2 = n2;
  }
}

// Scatter pass from the records: primary entries straight to offset + rank, spill entries through
// the spill cursors.
__global__ void __launch_bounds__(kThreads) k_bin_scatter(ParticleGeom pg, BinGeom b,
                                                          const unsigned long long* __restrict__ rec,
                                                          const unsigned* __restrict__ off_p, unsigned* cur_s,
                                                          unsigned* ent_p, unsigned* ent_s) {
  const int np = pg.np;
  const long long nrows = (long long)np * np;
  constexpr int U = 2;   // records in flight per thread: their loads, then their offset lookups
  for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int qx = (int)(row / np), qy = (int)(row - (long long)qx * np);
    for (int q0 = threadIdx.x; q0 < np; q0 += U * blockDim.x) {
      unsigned long long r[U];
      unsigned base[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int qz = q0 + u * (int)blockDim.x;
        r[u] = qz < np ? __ldcs(rec + row * np + qz) : 0ULL;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int qz = q0 + u * (int)blockDim.x;
        base[u] = qz < np ? __ldg(off_p + ((unsigned)r[u] & ((1u << 26) - 1u))) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int qz = q0 + u * (int)blockDim.x;
        if (qz >= np) continue;
        const unsigned key = (unsigned)r[u] & ((1u << 26) - 1u), flags = ((unsigned)r[u] >> 26) & 7u;
        const unsigned packed = pack_q(qx, qy, qz);
        ent_p[base[u] + (unsigned)(r[u] >> 32)] = packed;
        if (flags) {
          int k[8];
          keys_from_record(b, key, flags, k);
#pragma unroll
          for (int e = 1; e < 8; ++e)
            if (k[e] >= 0) ent_s[atomicAdd(cur_s + k[e], 1u)] = packed;
        }
      }
    }
  }
}

// Exclusive scan of the two per-tile count arrays into offsets (length m+1) and scatter cursors,
// in three coalesced phases: per-segment sums, a scan of the segment sums, per-segment scans.
constexpr int kScanThreads = 512;
constexpr int kScanSeg = kScanThreads * 8;   // counts per segment

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* total) {
  __shared__ unsigned wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned w = lane < kScanThreads / 32 ? wsum[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += o;
    }
    if (lane < kScanThreads / 32) wsum[lane] = w;
  }
  __syncthreads();
  const unsigned before = warp ? wsum[warp - 1] : 0;
  *total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return before + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const unsigned* __restrict__ cnt_p,
                                                           const unsigned* __restrict__ cnt_s, int m,
                                                           unsigned* seg_sums) {
  const int list = blockIdx.y;
  const unsigned* cnt = list ? cnt_s : cnt_p;
  const int base = blockIdx.x * kScanSeg;
  unsigned v = 0;
  for (int i = threadIdx.x; i < kScanSeg; i += kScanThreads)
    if (base + i < m) v += cnt[base + i];
  unsigned tot;
  block_excl_scan(v, &tot);
  if (threadIdx.x == 0) seg_sums[list * gridDim.x + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_segs(unsigned* seg_sums, int nseg) {
  const int list = blockIdx.x;
  unsigned* ss = seg_sums + list * nseg;
  unsigned carry = 0;
  for (int b = 0; b < nseg; b += kScanThreads) {
    const unsigned v = b + (int)threadIdx.x < nseg ? ss[b + threadIdx.x] : 0;
    unsigned tot;
    const unsigned ex = block_excl_scan(v, &tot);
    if (b + (int)threadIdx.x < nseg) ss[b + threadIdx.x] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const unsigned* __restrict__ cnt_p,
                                                            const unsigned* __restrict__ cnt_s, int m,
                                                            const unsigned* __restrict__ seg_sums, unsigned* off_p,
                                                            unsigned* off_s, unsigned* cur_p, unsigned* cur_s) {
  const int list = blockIdx.y;
  const unsigned* cnt = list ? cnt_s : cnt_p;
  unsigned* off = list ? off_s : off_p;
  unsigned* cur = list ? cur_s : cur_p;
  const int base = blockIdx.x * kScanSeg;
  // each thread scans 8 consecutive counts; the thread totals are scanned across the block
  unsigned c[8], v = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = base + threadIdx.x * 8 + k;
    c[k] = i < m ? cnt[i] : 0;
    v += c[k];
  }
  unsigned tot;
  unsigned run = seg_sums[list * gridDim.x + blockIdx.x] + block_excl_scan(v, &tot);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = base + threadIdx.x * 8 + k;
    if (i < m) {
      off[i] = run;
      cur[i] = run;
    }
    run += c[k];
    if (i == m - 1) off[m] = run;
  }
}

// Tile-wise deposit: shared accumulator [T][T][TZ] of 64-bit fixed-point sums.  The tile's primary
// and spill entries form one index range, so a CTA's threads run out of work together.
template <int LT, int LZ, bool F32>
__global__ void __launch_bounds__(kThreads, COLA_DEPOSIT_MIN_BLOCKS) k_deposit_tiles(ParticleGeom pg, BinGeom b, FixedGeo fg,
                                                           const float* __restrict__ s,
                                                           const unsigned* __restrict__ off_p,
                                                           const unsigned* __restrict__ ent_p,
                                                           const unsigned* __restrict__ off_s,
                                                           const unsigned* __restrict__ ent_s,
                                                           unsigned long long* rho, float* delta_out, float scale,
                                                           unsigned long long* tile_mass) {
  extern __shared__ unsigned long long acc[];
  const int lt = LT ? LT : b.lt, lz = LZ ? LZ : b.lz;
  const int nm = pg.n, T = 1 << lt, TZ = 1 << lz;
  const int tile = blockIdx.x;
  const int bz = tile % b.nz, bxy = tile / b.nz;
  const int bx = bxy / b.nt, by = bxy - bx * b.nt;
  const int x0 = bx << lt, y0 = by << lt, z0 = bz << lz;
  const int cells = (T * T) << lz;
  const int cs = TZ + kDepositPad;   // accumulator column stride (padding spreads columns over banks)
  for (int i = threadIdx.x; i < T * T * cs; i += blockDim.x) acc[i] = 0ULL;
  __syncthreads();
  const long long n = pg.npart;
  const unsigned p0 = off_p[tile], np_t = off_p[tile + 1] - p0;
  const unsigned s0 = off_s[tile], total = np_t + (off_s[tile + 1] - s0);
  for (unsigned k = threadIdx.x; k < total; k += blockDim.x) {
    int q[3];
    long long id;
    unpack_q(k < np_t ? ent_p[p0 + k] : ent_s[s0 + (k - np_t)], pg.np, q, &id);
    int c[3];
    unsigned w1[3], w0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int f;
      cell_frac<F32>(q[a], __ldg(s + a * n + id), fg, &c[a], &f);
      w1[a] = (unsigned)f;
      w0[a] = kWeightOne - w1[a];
    }
    int lz2[2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
      int iz = c[2] + dz;
      if (iz == nm) iz = 0;
      lz2[dz] = iz - z0;
    }
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      int ix = c[0] + dx;
      if (ix == nm) ix = 0;
      const int lx = ix - x0;
      if (lx < 0 || lx >= T) continue;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        int iy = c[1] + dy;
        if (iy == nm) iy = 0;
        const int ly = iy - y0;
        if (ly < 0 || ly >= T) continue;
        const unsigned wxy = (dx ? w1[0] : w0[0]) * (dy ? w1[1] : w0[1]);   // <= 2^28
        unsigned long long* col = acc + (lx * T + ly) * cs;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const unsigned long long w = (unsigned long long)wxy * (dz ? w1[2] : w0[2]);   // <= 2^42
          if (w && lz2[dz] >= 0 && lz2[dz] < TZ) smem_add64(col + lz2[dz], w);
        }
      }
    }
  }
  __syncthreads();
  // the tile owns its cells: plain, coalesced stores of T*T column segments of TZ cells
  if (!delta_out) {
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int col = i >> lz, z = i & (TZ - 1);
      const int lx = col >> lt, ly = col & (T - 1);
      rho[((long long)(x0 + lx) * nm + (y0 + ly)) * nm + z0 + z] = acc[col * cs + z];
    }
    return;
  }
  // the density contrast instead of the fixed-point values, and the exact 128-bit total for the
  // overflow check (every thread of the CTA's full warps reaches the warp reduction)
  unsigned long long lo = 0ULL, hi = 0ULL;
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    const int col = i >> lz, z = i & (TZ - 1);
    const int lx = col >> lt, ly = col & (T - 1);
    const unsigned long long v = acc[col * cs + z];
    lo += v;
    hi += (lo < v);
    delta_out[((long long)(x0 + lx) * nm + (y0 + ly)) * nm + z0 + z] = fixed_to_delta(v, scale);
  }
  // the CTA's total (warp shuffles, then the warps' partials in shared memory) and one slot update
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, off);
    const unsigned long long ohi = __shfl_down_sync(0xffffffffu, hi, off);
    lo += olo;
    hi += ohi + (lo < olo);
  }
  __shared__ unsigned long long wpart[2 * (kThreads / 32)];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    wpart[2 * warp] = lo;
    wpart[2 * warp + 1] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tlo = 0ULL, thi = 0ULL;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tlo += wpart[2 * w];
      thi += wpart[2 * w + 1] + (tlo < wpart[2 * w]);
    }
    tile_mass[2 * blockIdx.x] = tlo;   // one pair per tile, no atomics; launch_mass_reduce sums them
    tile_mass[2 * blockIdx.x + 1] = thi;
  }
}

// Tile-wise gather (+ kick and drift) over the primary entries of each tile, from a shared copy
// of the tile's force values with a one-cell halo on the upper side of every axis.
// Shared copy: 3 components x (T+1)^2 rows of hz = TZ + 1 floats, rows padded to hp (16 B).
struct GatherTile {
  int x0, y0, z0;
};

// floats of one tile's staged forces: 3 components x (T+1)^2 rows of hp
__host__ __device__ __forceinline__ int gather_floats(const BinGeom& b) {
  const int hx = (1 << b.lt) + 1, hp = ((1 << b.lz) + 1 + 3) & ~3;
  return 3 * hx * hx * hp;
}
template <int LT, int LZ>
__device__ __forceinline__ int gather_floats_t(const BinGeom& b) {
  const int hx = (1 << (LT ? LT : b.lt)) + 1, hp = ((1 << (LZ ? LZ : b.lz)) + 1 + 3) & ~3;
  return 3 * hx * hx * hp;
}

__device__ __forceinline__ GatherTile gather_tile_origin(const BinGeom& b, int tile) {
  const int bz = tile % b.nz, bxy = tile / b.nz;
  const int bx = bxy / b.nt, by = bxy - bx * b.nt;
  return GatherTile{bx << b.lt, by << b.lt, bz << b.lz};
}

// Issue (and commit as one group) the asynchronous copies of a tile's forces into fsm: TZ/4
// chunks of 16 bytes per row (rows start 16-byte aligned: z0 is a multiple of TZ and real rows
// hold 2 pc floats, pc even) plus the 4-byte periodic halo cell.
template <int LT, int LZ>
__device__ __forceinline__ void gather_stage(float* fsm, const BinGeom& b, int nm, const GatherTile& t,
                                             const float* __restrict__ f0, const float* __restrict__ f1,
                                             const float* __restrict__ f2, long long rs) {
  const int hx = (1 << (LT ? LT : b.lt)) + 1, zl = 1 << (LZ ? LZ : b.lz), hp = (zl + 1 + 3) & ~3;
  const int rows = 3 * hx * hx, chunks = (zl >> 2) + 1;
  for (int op = threadIdx.x; op < rows * chunks; op += blockDim.x) {
    const int r = op / chunks, ch = op - r * chunks;
    const int comp = r / (hx * hx), col = r - comp * hx * hx;
    const int lx = col / hx, ly = col - lx * hx;
    int gx = t.x0 + lx, gy = t.y0 + ly;
    if (gx >= nm) gx -= nm;
    if (gy >= nm) gy -= nm;
    const float* f = comp == 0 ? f0 : (comp == 1 ? f1 : f2);
    const float* row = f + ((long long)gx * nm + gy) * rs;
    float* dst = fsm + r * hp;
    if (ch < (zl >> 2)) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + 4 * ch);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(row + t.z0 + 4 * ch) : "memory");
    } else {
      const int gzz = t.z0 + zl == nm ? 0 : t.z0 + zl;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + zl);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(row + gzz) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

constexpr int kBulkWaitLimit = 1 << 22;   // polls of a staging barrier before the CTA gives up

// Stage a tile's forces as gather_stage does, by bulk copies: one cp.async.bulk of TZ cells per force
// row (3 (T+1)^2 rows, a row per thread), all completing on the mbarrier at bar_sa, plus each row's
// periodic halo cell by a 4-byte cp.async (committed as one group).  Rows start 16-byte aligned (z0 a
// multiple of TZ >= 4, rows of 2 pc floats with pc even) and TZ cells are a multiple of 16 bytes.
// Called by every thread of the block; contains a barrier.
template <int LT, int LZ>
__device__ __forceinline__ void gather_stage_bulk(float* fsm, unsigned bar_sa, const BinGeom& b, int nm,
                                                  const GatherTile& t, const float* __restrict__ f0,
                                                  const float* __restrict__ f1, const float* __restrict__ f2,
                                                  long long rs) {
  const int hx = (1 << (LT ? LT : b.lt)) + 1, zl = 1 << (LZ ? LZ : b.lz), hp = (zl + 1 + 3) & ~3;
  const int rows = 3 * hx * hx;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_sa) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar_sa),
                 "r"(rows * zl * 4)
                 : "memory");
  }
  __syncthreads();   // the barrier expects every row's bytes before any copy is issued
  const int gzz = t.z0 + zl == nm ? 0 : t.z0 + zl;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const int comp = r / (hx * hx), col = r - comp * hx * hx;
    const int lx = col / hx, ly = col - lx * hx;
    int gx = t.x0 + lx, gy = t.y0 + ly;
    if (gx >= nm) gx -= nm;
    if (gy >= nm) gy -= nm;
    const float* f = comp == 0 ? f0 : (comp == 1 ? f1 : f2);
    const float* row = f + ((long long)gx * nm + gy) * rs;
    const unsigned sa = (unsigned)__cvta_generic_to_shared(fsm + r * hp);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(sa),
                 "l"(row + t.z0), "r"(zl * 4), "r"(bar_sa)
                 : "memory");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa + 4u * zl), "l"(row + gzz) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Bounded wait for phase `parity` of the mbarrier at bar_sa; false if the limit was reached.
__device__ __forceinline__ bool bulk_wait(unsigned bar_sa, unsigned parity) {
  for (int it = 0; it < kBulkWaitLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar_sa), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Interpolate the staged forces at the tile's particles e0..e1 (and kick and drift).  Returns
// whether a non-finite state was written.
template <bool KICK, int LT, int LZ, bool F32>
__device__ __forceinline__ bool gather_particles(const float* fsm, const ParticleGeom& pg, const BinGeom& b,
                                                 const FixedGeo& fg, const GatherTile& t, unsigned e0, unsigned e1,
                                                 const unsigned* __restrict__ ent_p, const unsigned* ent_s,
                                                 unsigned ne, const float* __restrict__ s_in,
                                                 float* __restrict__ force_out, float* s, float* v,
                                                 const float* __restrict__ psi1, const float* __restrict__ psi2,
                                                 const KickDrift& kd) {
  const int hx = (1 << (LT ? LT : b.lt)) + 1, hp = ((1 << (LZ ? LZ : b.lz)) + 1 + 3) & ~3;
  const long long n = pg.npart;
  const float inv_one = 1.0f / kWeightOne;
  bool bad = false;
  const float* sp = KICK ? s : s_in;
  // rolling prefetch: the next particle's entry and position are loaded while this one is
  // interpolated
  int qn[3] = {0, 0, 0};
  long long idn = 0;
  float sn[3] = {0.f, 0.f, 0.f};
  auto fetch = [&](unsigned e) {
    unpack_q(e - e0 < ne ? ent_s[e - e0] : ent_p[e], pg.np, qn, &idn);
#pragma unroll
    for (int a = 0; a < 3; ++a) sn[a] = sp[a * n + idn];
  };
  if (e0 + threadIdx.x < e1) fetch(e0 + threadIdx.x);
  for (unsigned e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int q[3] = {qn[0], qn[1], qn[2]};
    const long long id = idn;
    float sv[3] = {sn[0], sn[1], sn[2]};
    float pv1[3], pv2[3], vv[3];
    if (KICK) {
      // issue every particle load up front: their latency overlaps the interpolation below
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pv1[a] = __ldg(psi1 + a * n + id);
        pv2[a] = __ldg(psi2 + a * n + id);
        vv[a] = v[a * n + id];
      }
    }
    if (e + blockDim.x < e1) fetch(e + blockDim.x);
    int c[3];
    float w1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int f;
      cell_frac<F32>(q[a], sv[a], fg, &c[a], &f);
      w1[a] = (float)f * inv_one;
    }
    const int lx = c[0] - t.x0, ly = c[1] - t.y0, lz = c[2] - t.z0;   // base cell inside the tile
    float fr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const float wx = dx ? w1[0] : 1.0f - w1[0];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float wxy = wx * (dy ? w1[1] : 1.0f - w1[1]);
        const int o = ((lx + dx) * hx + (ly + dy)) * hp + lz;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          const float* p = fsm + comp * (hx * hx * hp) + o;
          fr[comp] += wxy * ((1.0f - w1[2]) * p[0] + w1[2] * p[1]);
        }
      }
    }
    if (!KICK) {
      force_out[id] = fr[0];
      force_out[n + id] = fr[1];
      force_out[2 * n + id] = fr[2];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float p1 = pv1[a], p2 = pv2[a];
        const float fres = fr[a] - (kd.c1 * p1 + kd.c2 * p2);
        const float vn = vv[a] + kd.kick * fres;
        const float sn = sv[a] + kd.drift * vn + kd.dd1 * p1 + kd.dd2 * p2;
        v[a * n + id] = vn;
        s[a * n + id] = sn;
        bad |= !isfinite(vn) || !isfinite(sn);
      }
    }
  }
  return bad;
}

// One CTA per tile.
template <bool KICK, int LT, int LZ, bool F32>
__global__ void __launch_bounds__(kThreads) k_gather_tiles(ParticleGeom pg, BinGeom b, FixedGeo fg,
                                                          const unsigned* __restrict__ off_p,
                                                          const unsigned* __restrict__ ent_p,
                                                          const float* __restrict__ f0, const float* __restrict__ f1,
                                                          const float* __restrict__ f2, long long rs,
                                                          const float* __restrict__ s_in, float* __restrict__ force_out,
                                                          float* s, float* v, const float* __restrict__ psi1,
                                                          const float* __restrict__ psi2, KickDrift kd, int* flags) {
  extern __shared__ __align__(16) float fsm[];
  const int tile = blockIdx.x;
  const unsigned e0 = off_p[tile], e1 = off_p[tile + 1];
  if (e0 == e1) return;                          // empty (uniform across the block)
  const GatherTile t = gather_tile_origin(b, tile);
  // the tile's first kGatherEnt entries travel with the forces: one dependent global load fewer
  unsigned* ent_s = reinterpret_cast<unsigned*>(fsm + gather_floats_t<LT, LZ>(b));
  const unsigned ne = e1 - e0 < (unsigned)kGatherEnt ? e1 - e0 : (unsigned)kGatherEnt;
  for (unsigned i = threadIdx.x; i < ne; i += blockDim.x) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(ent_s + i);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(ent_p + e0 + i) : "memory");
  }
  // the forces by bulk copies on an mbarrier placed after the staged entries (8-byte aligned)
  const unsigned bar_sa = (unsigned)__cvta_generic_to_shared(ent_s + kGatherEnt);
  gather_stage_bulk<LT, LZ>(fsm, bar_sa, b, pg.n, t, f0, f1, f2, rs);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  const bool ok = bulk_wait(bar_sa, 0);
  if (__syncthreads_or(!ok)) {
    // the staging never completed (not expected): report, give the copies one more bounded wait, stop
    if (threadIdx.x == 0) atomicOr(flags, 4);
    bulk_wait(bar_sa, 0);
    return;
  }
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(bar_sa) : "memory");
  const bool bad = gather_particles<KICK, LT, LZ, F32>(fsm, pg, b, fg, t, e0, e1, ent_p, ent_s, ne, s_in, force_out,
                                                       s, v, psi1, psi2, kd);
  if (KICK && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 2);
}

// Persistent variant: each CTA walks tiles t = blockIdx.x + i gridDim.x with two staging buffers;
// the next non-empty tile's forces are copied (cp.async) while the current tile's particles run.
template <bool KICK, int LT, int LZ, bool F32>
__global__ void __launch_bounds__(kThreads) k_gather_tiles_pipe(ParticleGeom pg, BinGeom b, FixedGeo fg,
                                                               const unsigned* __restrict__ off_p,
                                                               const unsigned* __restrict__ ent_p,
                                                               const float* __restrict__ f0,
                                                               const float* __restrict__ f1,
                                                               const float* __restrict__ f2, long long rs,
                                                               const float* __restrict__ s_in,
                                                               float* __restrict__ force_out, float* s, float* v,
                                                               const float* __restrict__ psi1,
                                                               const float* __restrict__ psi2, KickDrift kd,
                                                               int* flags) {
  extern __shared__ __align__(16) float fsm[];
  const int hx = (1 << b.lt) + 1, hp = ((1 << b.lz) + 1 + 3) & ~3;
  float* bcur = fsm;
  float* bnext = fsm + 3 * hx * hx * hp;
  const int ntiles = b.tiles;
  // first non-empty tile of this CTA
  auto next_tile = [&](int t) {
    while (t < ntiles && off_p[t] == off_p[t + 1]) t += gridDim.x;
    return t;
  };
  int t = next_tile(blockIdx.x);
  if (t >= ntiles) return;
  gather_stage<LT, LZ>(bcur, b, pg.n, gather_tile_origin(b, t), f0, f1, f2, rs);
  bool bad = false;
  while (t < ntiles) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();   // tile t staged; every thread is done with the other buffer
    const int tn = next_tile(t + gridDim.x);
    if (tn < ntiles) gather_stage<LT, LZ>(bnext, b, pg.n, gather_tile_origin(b, tn), f0, f1, f2, rs);
    bad |= gather_particles<KICK, LT, LZ, F32>(bcur, pg, b, fg, gather_tile_origin(b, t), off_p[t], off_p[t + 1], ent_p,
                                               nullptr, 0u,
                                  s_in, force_out, s, v, psi1, psi2, kd);
    float* tmp = bcur;
    bcur = bnext;
    bnext = tmp;
    t = tn;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (KICK && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 2);
}

}  // namespace

bool bin_geometry(int nmesh, int np, BinGeom* b) {
  if (np > 1024) return false;                       // packed 10-bit lattice coordinates
  int lt = 3;                                        // T = 8 cells across, or the largest power of
  while (lt > 0 && nmesh % (1 << lt)) --lt;          // two dividing N
  int lz = 5;                                        // TZ = 32 cells along z, likewise
  while (lz > 0 && nmesh % (1 << lz)) --lz;
  if (lz == 0 || lt == 0) return false;
  b->lt = lt;
  b->lz = lz;
  b->nt = nmesh >> lt;
  b->nz = nmesh >> lz;
  const long long tiles = (long long)b->nt * b->nt * b->nz;
  if (tiles > (1LL << 26)) return false;
  b->tiles = (int)tiles;
  return true;
}

size_t bin_smem_bytes(const BinGeom& b, int nmesh) {
  (void)nmesh;
  return (size_t)(1 << b.lt) * (1 << b.lt) * ((1 << b.lz) + kDepositPad) * sizeof(unsigned long long);
}

// z-tiles per gather CTA
int gather_group(const BinGeom& b) {
  (void)b;
  return 1;
}

size_t gather_smem_bytes(const BinGeom& b) {
  const size_t hx = (1 << b.lt) + 1, hz = ((size_t)gather_group(b) << b.lz) + 1;
  const size_t hp = (hz + 3) & ~(size_t)3;
  return 3 * hx * hx * hp * sizeof(float);
}

bool tile_gather_pays(const BinGeom& b, long long npart) {
  // staging a tile's forces costs about as much as gathering a few hundred particles directly;
  // the 16-byte copies also need rows of at least 4 cells along z
  const long long groups = (long long)b.tiles / gather_group(b);
  return b.lz >= 2 && npart >= 384LL * groups;
}

int launch_excl_scan(const unsigned* cnt, int m, unsigned* seg, unsigned* off, unsigned* cur, cudaStream_t st) {
  const int nseg = (m + kScanSeg - 1) / kScanSeg;
  k_scan_sums<<<dim3(nseg, 1), kScanThreads, 0, st>>>(cnt, cnt, m, seg);
  k_scan_segs<<<1, kScanThreads, 0, st>>>(seg, nseg);
  k_scan_apply<<<dim3(nseg, 1), kScanThreads, 0, st>>>(cnt, cnt, m, seg, off, off, cur, cur);
  return check_launch("excl_scan");
}

namespace {
template <int V>
using IntC = std::integral_constant<int, V>;

// Calls go(LT, LZ, F32) with the compile-time instance that matches the geometry: the common
// 8 x 8 x 32 tiles or run-time tile sides, and the 32-bit fixed-point path below 2048 cells.
template <class Go>
void with_instance(const BinGeom& b, int nmesh, Go&& go) {
  const bool common = b.lt == 3 && b.lz == 5;
  const bool f32 = nmesh < 2048;
  if (common && f32) go(IntC<3>{}, IntC<5>{}, std::true_type{});
  else if (common) go(IntC<3>{}, IntC<5>{}, std::false_type{});
  else if (f32) go(IntC<0>{}, IntC<0>{}, std::true_type{});
  else go(IntC<0>{}, IntC<0>{}, std::false_type{});
}

template <class K>
void smem_limit(K kernel, int bytes) {
  if (first_use_on_device(reinterpret_cast<const void*>(kernel)))
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
}  // namespace

int launch_binning(const ParticleGeom& pg, const BinGeom& b, const float* s, BinBuffers& bb, cudaStream_t st) {
  const long long rows = (long long)pg.np * pg.np;
  const unsigned grid = (unsigned)(rows < 152LL * 64 ? rows : 152LL * 64);
  const int th = pg.np < kThreads ? ((pg.np + 31) / 32) * 32 : kThreads;
  const FixedGeo fg = fixed_geo(pg.n, pg.r_fixed);
  if (cudaMemsetAsync(bb.cnt_p, 0, (size_t)b.tiles * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(bb.cnt_s, 0, (size_t)b.tiles * sizeof(unsigned), st) != cudaSuccess)
    return COLA_ERR_CUDA;
  with_instance(b, pg.n, [&](auto lt, auto lz, auto f32) {
    k_bin_count<decltype(lt)::value, decltype(lz)::value, decltype(f32)::value>
        <<<grid, th, 0, st>>>(pg, b, fg, s, bb.cnt_p, bb.cnt_s, bb.rec);
  });
  int e = check_launch("bin_count");
  if (e != COLA_OK) return e;
  const int nseg = (b.tiles + kScanSeg - 1) / kScanSeg;
  k_scan_sums<<<dim3(nseg, 2), kScanThreads, 0, st>>>(bb.cnt_p, bb.cnt_s, b.tiles, bb.seg);
  k_scan_segs<<<2, kScanThreads, 0, st>>>(bb.seg, nseg);
  k_scan_apply<<<dim3(nseg, 2), kScanThreads, 0, st>>>(bb.cnt_p, bb.cnt_s, b.tiles, bb.seg, bb.off_p, bb.off_s,
                                                       bb.cur_p, bb.cur_s);
  if ((e = check_launch("bin_scan")) != COLA_OK) return e;
  k_bin_scatter<<<grid, th, 0, st>>>(pg, b, bb.rec, bb.off_p, bb.cur_s, bb.ent_p, bb.ent_s);
  return check_launch("bin_scatter");
}

int launch_deposit_tiles(const ParticleGeom& pg, const BinGeom& b, const float* s, const BinBuffers& bb,
                         unsigned long long* rho, cudaStream_t st, float* delta_out, float scale,
                         unsigned long long* tile_mass) {
  if (delta_out && !tile_mass) return COLA_ERR_INVALID;
  const FixedGeo fg = fixed_geo(pg.n, pg.r_fixed);
  with_instance(b, pg.n, [&](auto lt, auto lz, auto f32) {
    auto k = k_deposit_tiles<decltype(lt)::value, decltype(lz)::value, decltype(f32)::value>;
    smem_limit(k, 64 * 1024);
    k<<<b.tiles, kThreads, bin_smem_bytes(b, pg.n), st>>>(pg, b, fg, s, bb.off_p, bb.ent_p, bb.off_s, bb.ent_s, rho,
                                                          delta_out, scale, tile_mass);
  });
  return check_launch("deposit_tiles");
}

int launch_gather_tiles(const ParticleGeom& pg, const BinGeom& b, const BinBuffers& bb, const float* const f[3],
                        long long rs, const float* s_in, float* force_out, float* s, float* v, const float* psi1,
                        const float* psi2, const KickDrift* kd, int* flags, cudaStream_t st, bool pipelined) {
  const size_t sm = gather_smem_bytes(b);
  const size_t sm_ent = (size_t)gather_floats(b) * sizeof(float) + kGatherEnt * sizeof(unsigned) + 16;   // + mbarrier
  const KickDrift k = kd ? *kd : KickDrift{};
  const FixedGeo fg = fixed_geo(pg.n, pg.r_fixed);
  if (pipelined) {
    // two staging buffers per CTA: as many CTAs per SM as the shared memory holds (at most 4)
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = (int)((227 * 1024) / (2 * sm + 1024));
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
    const int ctas = b.tiles < sms * per_sm ? b.tiles : sms * per_sm;
    with_instance(b, pg.n, [&](auto lt, auto lz, auto f32) {
      constexpr int LT = decltype(lt)::value, LZ = decltype(lz)::value;
      constexpr bool F32 = decltype(f32)::value;
      if (kd) {
        auto kern = k_gather_tiles_pipe<true, LT, LZ, F32>;
        smem_limit(kern, 128 * 1024);
        kern<<<ctas, kThreads, 2 * sm, st>>>(pg, b, fg, bb.off_p, bb.ent_p, f[0], f[1], f[2], rs, nullptr, nullptr, s,
                                             v, psi1, psi2, k, flags);
      } else {
        auto kern = k_gather_tiles_pipe<false, LT, LZ, F32>;
        smem_limit(kern, 128 * 1024);
        kern<<<ctas, kThreads, 2 * sm, st>>>(pg, b, fg, bb.off_p, bb.ent_p, f[0], f[1], f[2], rs, s_in, force_out,
                                             nullptr, nullptr, nullptr, nullptr, k, flags);
      }
    });
    return check_launch("gather_tiles_pipe");
  }
  with_instance(b, pg.n, [&](auto lt, auto lz, auto f32) {
    constexpr int LT = decltype(lt)::value, LZ = decltype(lz)::value;
    constexpr bool F32 = decltype(f32)::value;
    if (kd) {
      auto kern = k_gather_tiles<true, LT, LZ, F32>;
      smem_limit(kern, 64 * 1024);
      kern<<<b.tiles, kThreads, sm_ent, st>>>(pg, b, fg, bb.off_p, bb.ent_p, f[0], f[1], f[2], rs, nullptr, nullptr, s,
                                              v, psi1, psi2, k, flags);
    } else {
      auto kern = k_gather_tiles<false, LT, LZ, F32>;
      smem_limit(kern, 64 * 1024);
      kern<<<b.tiles, kThreads, sm_ent, st>>>(pg, b, fg, bb.off_p, bb.ent_p, f[0], f[1], f[2], rs, s_in, force_out,
                                              nullptr, nullptr, nullptr, nullptr, k, flags);
    }
  });
  return check_launch("gather_tiles");
}

}  // namespace cola
