// Allocation-free power spectrum for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA-graph capture that must
// stay replayable without a memory pool, plug-ins of host frameworks that own the whole device
// heap, or real-time loops that forbid allocator calls and their implicit synchronisation.  For
// them cola_power_spectrum_noalloc measures P(k) of a small realisation without a context: every
// scratch buffer it needs (the fixed-point density mesh, the half spectrum, the per-block partial
// sums, the bins' geometry, the FFT twiddles and the bin edges) lives in one file-scope device array of fixed size.
//
// That array costs COLA_NOALLOC_SCRATCH_BYTES (about 3.4 MB) on every GPU that loads the library,
// for as long as the process lives.  All calls share it and it keeps the last call's contents:
// the density mesh is cleared by every call, everything else is fully rewritten, and calls that
// overlap on the GPU (other streams, other host threads) race on it.
#include "cola_internal.h"

#include <cmath>
#include <cstdio>
#include <mutex>

namespace cola {
namespace {

constexpr int kMaxMesh = COLA_NOALLOC_MAX_MESH;
constexpr int kMaxBins = 128;
constexpr int kBlocks = 64;   // P(k) partial-sum blocks

constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kRhoBytes = round256((size_t)kMaxMesh * kMaxMesh * kMaxMesh * sizeof(unsigned long long));
constexpr size_t kSpecBytes = round256((size_t)kMaxMesh * kMaxMesh * (kMaxMesh / 2 + 2) * sizeof(float2));
constexpr size_t kPartBytes = round256((size_t)kBlocks * 2 * kMaxBins * sizeof(double));
constexpr size_t kEdgeBytes = round256((kMaxBins + 1) * sizeof(long long));
constexpr size_t kTwBytes = round256(kMaxMesh * sizeof(float2));
constexpr size_t kGeomBytes = round256(2 * kMaxBins * sizeof(double));
constexpr size_t kFlagBytes = 256;
constexpr size_t kOffSpec = kRhoBytes;
constexpr size_t kOffPart = kOffSpec + kSpecBytes;
constexpr size_t kOffEdge = kOffPart + kPartBytes;
constexpr size_t kOffTw = kOffEdge + kEdgeBytes;
constexpr size_t kOffGeom = kOffTw + kTwBytes;
constexpr size_t kOffFlag = kOffGeom + kGeomBytes;
constexpr size_t kTotal = kOffFlag + kFlagBytes;
static_assert(kTotal <= COLA_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the documented size");

__device__ __align__(256) unsigned char g_scratch[COLA_NOALLOC_SCRATCH_BYTES];

struct EdgeTable {
  long long e[kMaxBins + 1];
};

// Per-call tables: twiddles exp(-2 pi i t / n) (FP64 sincospi rounded to float) and bin edges.
__global__ void k_static_tables(int n, float2* tw, EdgeTable edges, int nedges, long long* edges_out) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
  }
  for (int b = threadIdx.x; b < nedges; b += blockDim.x) edges_out[b] = edges.e[b];
}

// Host-side stand-in of g_scratch is not a device address: resolve it once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_base[kMaxDevices] = {};

int scratch_base(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return COLA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_base[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) {
      std::fprintf(stderr, "cola: cudaGetSymbolAddress(scratch) failed: %s\n", cudaGetErrorString(e));
      return COLA_ERR_CUDA;
    }
    g_base[dev] = static_cast<unsigned char*>(ptr);
    fft_set_smem_limits();
  }
  *out = g_base[dev];
  return COLA_OK;
}

bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" int cola_power_spectrum_noalloc(const cola_params* p, const float* s, double* pk, int nbins,
                                           void* stream) {
  if (!p || !s || !pk || ((uintptr_t)s % 16) || ((uintptr_t)pk % 16)) return COLA_ERR_INVALID;
  if (p->nmesh < 4 || p->nmesh > kMaxMesh || p->nmesh % 2 || !smooth235(p->nmesh)) return COLA_ERR_INVALID;
  if (p->np < 2 || p->np > COLA_NOALLOC_MAX_NP || p->np % 2 || !smooth235(p->np)) return COLA_ERR_INVALID;
  if ((((long long)p->nmesh) << 20) % p->np) return COLA_ERR_INVALID;
  if (nbins < 1 || nbins > kMaxBins || !(p->box > 0.0)) return COLA_ERR_INVALID;
  unsigned char* base = nullptr;
  const int st0 = scratch_base(&base);
  if (st0 != COLA_OK) return st0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = p->nmesh;

  FftPlan plan;
  std::vector<int> rad;
  if (!fft_factor(n, &rad)) return COLA_ERR_INVALID;
  plan.dev.n = n;
  plan.dev.nstages = (int)rad.size();
  for (int i = 0; i < kMaxStages; ++i) plan.dev.radix[i] = i < (int)rad.size() ? rad[i] : 1;
  plan.dev.tw = reinterpret_cast<const float2*>(base + kOffTw);
  fft_plan_steps(&plan);

  Grid3 g;
  g.n = n;
  g.nc = n / 2 + 1;
  g.pc = (g.nc + 1) & ~1;
  ParticleGeom pg;
  pg.np = p->np;
  pg.n = n;
  pg.r_fixed = (((long long)n) << 20) / p->np;
  pg.npart = (long long)p->np * p->np * p->np;

  EdgeTable edges;
  const double half = n / 2.0;
  for (int b = 0; b <= nbins; ++b) edges.e[b] = (long long)std::ceil(std::pow(half, 2.0 * b / nbins) - 1e-9);

  auto* rho = reinterpret_cast<unsigned long long*>(base);
  auto* spec = reinterpret_cast<float2*>(base + kOffSpec);
  auto* part = reinterpret_cast<double*>(base + kOffPart);
  auto* edg = reinterpret_cast<long long*>(base + kOffEdge);
  auto* tw = reinterpret_cast<float2*>(base + kOffTw);
  auto* flags = reinterpret_cast<int*>(base + kOffFlag);
  auto* geom = reinterpret_cast<double*>(base + kOffGeom);

  const size_t n3 = (size_t)n * n * n;
  if (cudaMemsetAsync(rho, 0, n3 * sizeof(unsigned long long), st) != cudaSuccess) return COLA_ERR_CUDA;
  k_static_tables<<<1, 128, 0, st>>>(n, tw, edges, nbins + 1, edg);
  if (cudaGetLastError() != cudaSuccess) return COLA_ERR_CUDA;
  int r = launch_deposit(pg, s, rho, flags, st);
  const float scale = (float)((double)n3 / ((double)pg.npart * 4398046511104.0));
  if (r == COLA_OK) r = launch_r2c_rows(plan, g, kSrcFixedPoint, rho, n, scale, spec, st);
  if (r == COLA_OK) r = launch_pencils(plan, g, 1, -1, spec, st);
  if (r == COLA_OK) r = launch_pencils(plan, g, 0, -1, spec, st);
  const double pscale = std::pow(p->box, 3) / std::pow((double)n, 6);
  if (r == COLA_OK) r = launch_pk_geometry(g, edg, nbins, part, kBlocks, geom, st);
  if (r == COLA_OK) r = launch_pk_bins(g, spec, edg, nbins, 0, part, kBlocks, st);
  if (r == COLA_OK) r = launch_pk_finish(part, kBlocks, nbins, geom, 2.0 * M_PI / p->box, pscale, 0.0, pk, st);
  return r;
}
