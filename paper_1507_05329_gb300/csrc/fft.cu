// Host side of the FFT passes: plans (factorisation, twiddle tables), tile shapes and the choice
// among the pipelined, fast and generic kernels of each pass.
#include "fft_core.cuh"

#include <mutex>
#include <set>
#include <utility>

namespace cola {
using namespace fftk;
namespace {

struct TileShape {
  int lw;
  int threads;
  size_t smem;
};

constexpr int kTileElems = 6144;    // complex elements per tile (two buffers: about 100 KB of shared memory)
constexpr int kWideElems = 12288;   // wide tiles: 8 pencils of up to 1536 (two buffers: about 200 KB)

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


int largest_pow2_le(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

// Persistent pipelined strided passes: three tile buffers (staging, ping, pong) per CTA, or two
// (staging and one work buffer that the middle stages overwrite) in a budget of kInplaceKb.
struct PipeShape {
  int lw, threads, nchunks, ntiles, ctas;
  size_t smem;
};

constexpr int kInplaceKb = 210;   // two tiles of 8 pencils of 1536

PipeShape pipe_shape(const Grid3& g, int budget_kb, int ept, bool inplace) {
  PipeShape ps;
  const size_t nbuf = inplace ? 2 : 3;
  if (inplace) budget_kb = kInplaceKb;
  int lw = 1;   // W >= 2: 16-byte copies
  while ((2 << lw) <= largest_pow2_le(g.nc) &&
         nbuf * (g.n + g.n / 16 + 1) * (2 << lw) * 8 <= (size_t)budget_kb * 1024 &&
         ((long long)g.n * (2 << lw) + ept - 1) / ept <= kPipeThreads)
    ++lw;
  ps.lw = lw;
  ps.smem = nbuf * (g.n + g.n / 16 + 1) * (1 << lw) * sizeof(float2);
  int th = ((g.n << lw) + ept - 1) / ept;
  th = ((th + 31) / 32) * 32;
  ps.threads = th < 64 ? 64 : (th > kPipeThreads ? kPipeThreads : th);
  ps.nchunks = (g.nc + (1 << lw) - 1) >> lw;
  ps.ntiles = ps.nchunks * g.n;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = ps.smem <= 72 * 1024 ? 3 : (ps.smem <= 110 * 1024 ? 2 : 1);
  if (per_sm * ps.threads > 2048) per_sm = 2048 / ps.threads > 0 ? 2048 / ps.threads : 1;
  ps.ctas = ps.ntiles < sms * per_sm ? ps.ntiles : sms * per_sm;
  return ps;
}

// The pipelined kernels need at least two columns per tile and a whole tile per thread set.
bool pipe_ok(const FftPlan& p, const Grid3& g) {
  if (!p.pipe || g.nc < 2) return false;
  const PipeShape ps = pipe_shape(g, p.pipe_kb, p.pipe_ept, p.pipe_inplace);
  return (long long)ps.threads * p.pipe_ept >= (long long)(g.n << ps.lw) && ps.smem <= kInplaceKb * 1024;
}

int max_radix(const FastPlan& fp) {
  int m = 2;
  for (int s = 0; s < fp.nst; ++s) m = fp.radix[s] > m ? fp.radix[s] : m;
  return m;
}

// Row index of a shared tile with one padding row per 16 (the device's saddr without the column).
int padded_row(int j) { return j + (j >> 4); }

// Padded step along stride d for the butterflies of a radix-R stage whose first rows are `starts`:
// the step that every row j0 + r d (r < R) of every butterfly lands on, or 0 when the padding is not
// affine along d.  Checked row by row, so a plan never takes the fixed-step addressing unless it
// gives exactly the rows saddr gives.
int affine_step(const std::vector<int>& starts, int d, int R) {
  const int step = padded_row(starts[0] + d) - padded_row(starts[0]);
  for (int j0 : starts)
    for (int r = 0; r < R; ++r)
      if (padded_row(j0 + r * d) != padded_row(j0) + r * step) return 0;
  return step;
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
    const int R = d.radix[s];
    fp->radix[s] = R;
    fp->lns[s] = l;
    fp->tstr[s] = d.n / (ns * R);
    fp->nbp[s] = pl.nbp[s];
    fp->nsp[s] = pl.nsp[s];
    ns *= R;
  }
  for (int s = d.nstages; s < kMaxStages; ++s)
    fp->radix[s] = 1, fp->lns[s] = 0, fp->tstr[s] = 0, fp->nbp[s] = 0, fp->nsp[s] = 0;
  return true;
}

TileShape fast_shape(int n, int wmax, int nbuf) {
  TileShape t = tile_shape(n, wmax);
  t.smem = (size_t)nbuf * (size_t)(n + n / 16 + 1) * (1u << t.lw) * sizeof(float2);
  return t;
}

// Tiles of 8 pencils for the strided passes whose default tile is narrower (n > 768): every row
// segment a tile reads and writes is then 64 bytes (two DRAM sectors) instead of 32, at one CTA of
// up to kWideThreads threads per SM.  Measured at n = 1536: the Green pass 41.0 -> 30.8 ms.
TileShape wide_shape(const FftPlan& p, const Grid3& g, const TileShape& t, int nbuf) {
  if (!p.wide || t.lw >= 3 || g.n * 8 > kWideElems || g.nc < 8) return t;
  TileShape w;
  w.lw = 3;
  const int th = ((g.n << 3) + kEpt - 1) / kEpt;
  w.threads = ((th + 31) / 32) * 32;
  w.smem = (size_t)nbuf * (size_t)(g.n + g.n / 16 + 1) * 8 * sizeof(float2);
  return w;
}

int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "cola: launch of %s failed: %s\n", what, cudaGetErrorString(e));
    return COLA_ERR_CUDA;
  }
  return COLA_OK;
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
  // one factor 3 and no 5: when the powers of two would need one stage more for their last factor
  // 2 (p2 = 1 mod 4, e.g. 1536 = 8 8 8 3), that 2 joins the 3 in a last radix-6 stage (16 16 6)
  const bool radix6 = n3 == 1 && n5 == 0 && p2 % 4 == 1;
  if (radix6) {
    --p2;
    n3 = 0;
  }
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
  if (radix6) radices->push_back(6);
  return (int)radices->size() <= kMaxStages;
}

// Affine row steps of the stages with a power-of-two ns (the fast-path stages): butterfly b < n/R
// touches rows b + r n/R and ((b >> l) R << l) + (b mod ns) + r ns, ns = 2^l.
void fft_plan_steps(FftPlan* plan) {
  const int n = plan->dev.n, m = plan->dev.nstages;
  for (int s = 0; s < kMaxStages; ++s) plan->nbp[s] = plan->nsp[s] = 0;
  for (int s = 0, ns = 1; s < m && !(ns & (ns - 1)); ns *= plan->dev.radix[s], ++s) {
    int l = 0;
    while ((1 << l) < ns) ++l;
    const int R = plan->dev.radix[s], nb = n / R;
    std::vector<int> by_nb(nb), by_ns(nb);
    for (int b = 0; b < nb; ++b) {
      by_nb[b] = b;
      by_ns[b] = (((b >> l) * R) << l) + (b & (ns - 1));
    }
    plan->nbp[s] = affine_step(by_nb, nb, R);
    plan->nsp[s] = affine_step(by_ns, ns, R);
  }
}

int fft_plan_init(FftPlan* plan, int n) {
  std::vector<int> rad;
  if (!fft_factor(n, &rad)) return COLA_ERR_INVALID;
  plan->dev.n = n;
  plan->dev.nstages = (int)rad.size();
  for (int i = 0; i < kMaxStages; ++i) plan->dev.radix[i] = i < (int)rad.size() ? rad[i] : 1;
  fft_plan_steps(plan);
  std::vector<float2> h(n);
  for (int t = 0; t < n; ++t) {
    const double ang = -2.0 * M_PI * (double)t / (double)n;
    h[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  if (cudaMalloc(&plan->tw, n * sizeof(float2)) != cudaSuccess) return COLA_ERR_OOM;
  if (cudaMemcpy(plan->tw, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
    return COLA_ERR_CUDA;
  plan->dev.tw = plan->tw;
  if (first_use_on_device(reinterpret_cast<const void*>(&generic_set_smem_limits))) generic_set_smem_limits();
  return COLA_OK;
}

bool first_use_on_device(const void* key) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  std::lock_guard<std::mutex> lock(mu);
  return done.insert({dev, key}).second;
}

void fft_set_smem_limits() { generic_set_smem_limits(); }

void fft_plan_free(FftPlan* plan) {
  if (plan->tw) cudaFree(plan->tw);
  plan->tw = nullptr;
}

// Row tiles with 8 elements per thread hold at most kTileElems / 2 elements (384 threads).
TileShape row_shape(int ept, const Grid3& g, int nbuf) {
  if (ept == 8 && g.n <= kTileElems / 2) {
    TileShape t = fast_shape(g.n, largest_pow2_le(kTileElems / 2 / g.n), nbuf);
    const int th = ((g.n << t.lw) + 7) / 8;
    t.threads = ((th + 31) / 32) * 32;
    return t;
  }
  return fast_shape(g.n, 1 << 20, nbuf);
}

int launch_r2c_rows(const FftPlan& p, const Grid3& g, RowSource kind, const void* src,
                    long long src_row_stride, float scale, float2* dst, cudaStream_t st,
                    unsigned long long* mass_acc) {
  const long long nrows = (long long)g.rows();
  FastPlan fp;
  if (fast_plan(p, &fp)) {
    const TileShape t = row_shape(p.r2c_ept, g, fp.nst >= 2 ? 2 : 1);
    const bool e8 = p.r2c_ept == 8 && g.n <= kTileElems / 2;
    const unsigned blocks = (unsigned)((nrows + (2LL << t.lw) - 1) / (2LL << t.lw));
    unsigned long long* acc = kind == kSrcFixedPoint ? mass_acc : nullptr;
    if (max_radix(fp) > 8) {
      if (e8 ? plan3_r2c_launch<8>(fp, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc,
                                   nrows, acc, st)
             : plan3_r2c_launch<16>(fp, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc,
                                    nrows, acc, st))
        return check_launch("r2c_plan3");
      if (e8) fast_r2c_launch<16, 8>(fp, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc, nrows, acc, st);
      else fast_r2c_launch<16, 16>(fp, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc, nrows, acc, st);
    } else {
      if (e8) fast_r2c_launch<8, 8>(fp, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc, nrows, acc, st);
      else fast_r2c_launch<8, 16>(fp, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc, nrows, acc, st);
    }
    return check_launch("r2c_fast");
  }
  const TileShape t = tile_shape(g.n, 1 << 20);
  const unsigned blocks = (unsigned)((nrows + (2LL << t.lw) - 1) / (2LL << t.lw));
  generic_r2c_launch(p.dev, t.lw, blocks, t.threads, t.smem, kind, src, src_row_stride, scale, dst, g.pc, nrows,
                     kind == kSrcFixedPoint ? mass_acc : nullptr, st);
  return check_launch("r2c_rows");
}

int launch_c2r_rows(const FftPlan& p, const Grid3& g, float2* data, cudaStream_t st) {
  const long long nrows = (long long)g.rows();
  FastPlan fp;
  if (p.row_pipe && fast_plan(p, &fp)) {
    // persistent CTAs: the widest tile (2W rows) with the staging copy and the stage buffers in
    // 110 KB and at most kPipeThreads threads
    const int ept = p.row_ept, nbuf = fp.nst >= 3 ? 2 : 1;
    auto smem_of = [&](int lw) {
      return ((size_t)(2 << lw) * g.pc + (size_t)nbuf * (g.n + g.n / 16 + 1) * (1u << lw)) * sizeof(float2);
    };
    auto threads_of = [&](int lw) { return (((g.n << lw) + ept - 1) / ept + 31) / 32 * 32; };
    int lw = 0;
    while ((2LL << (lw + 1)) <= nrows && smem_of(lw + 1) <= 110 * 1024 && threads_of(lw + 1) <= kPipeThreads) ++lw;
    const int th = threads_of(lw) < 64 ? 64 : threads_of(lw);
    if (th <= kPipeThreads && (long long)th * ept >= (long long)(g.n << lw)) {
      const size_t smem = smem_of(lw);
      const long long ntiles = (nrows + (2LL << lw) - 1) / (2LL << lw);
      int dev = 0, sms = 152;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      int per_sm = (int)((227 * 1024) / (smem + 1024));
      if (per_sm * th > 2048) per_sm = 2048 / th;
      if (per_sm > 3) per_sm = 3;
      if (per_sm < 1) per_sm = 1;
      const int ctas = (int)(ntiles < (long long)sms * per_sm ? ntiles : (long long)sms * per_sm);
      if (max_radix(fp) > 8) c2r_pipe_launch<16>(fp, lw, ctas, th, smem, ept, data, g.pc, nrows, ntiles, st);
      else c2r_pipe_launch<8>(fp, lw, ctas, th, smem, ept, data, g.pc, nrows, ntiles, st);
      return check_launch("c2r_pipe");
    }
  }
  if (fast_plan(p, &fp)) {
    const TileShape t = row_shape(p.row_ept, g, fp.nst >= 3 ? 2 : 1);
    const bool e8 = p.row_ept == 8 && g.n <= kTileElems / 2;
    const unsigned blocks = (unsigned)((nrows + (2LL << t.lw) - 1) / (2LL << t.lw));
    if (max_radix(fp) > 8) {
      if (e8 ? plan3_c2r_launch<8>(fp, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st)
             : plan3_c2r_launch<16>(fp, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st))
        return check_launch("c2r_plan3");
      if (e8) fast_c2r_launch<16, 8>(fp, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st);
      else fast_c2r_launch<16, 16>(fp, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st);
    } else {
      if (e8) fast_c2r_launch<8, 8>(fp, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st);
      else fast_c2r_launch<8, 16>(fp, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st);
    }
    return check_launch("c2r_fast");
  }
  const TileShape t = tile_shape(g.n, 1 << 20);
  const unsigned blocks = (unsigned)((nrows + (2LL << t.lw) - 1) / (2LL << t.lw));
  generic_c2r_launch(p.dev, t.lw, blocks, t.threads, t.smem, data, g.pc, nrows, st);
  return check_launch("c2r_rows");
}

bool pencils_x_mul_ok(const FftPlan& p, const Grid3& g) {
  FastPlan fp;
  if (!(fast_plan(p, &fp) && pipe_ok(p, g) && p.pipe_inplace && p.pipe_ept == 16 && plan3_id(fp) != 0)) return false;
  const PipeShape ps = pipe_shape(g, p.pipe_kb, p.pipe_ept, p.pipe_inplace);
  return ps.lw == 3 && ps.threads * 16 == (g.n << ps.lw);
}

int launch_pencils_x_mul(const FftPlan& p, const Grid3& g, const float2* src, const IcMul& mul, float2* dst,
                         cudaStream_t st) {
  FastPlan fp;
  if (!pencils_x_mul_ok(p, g) || !fast_plan(p, &fp)) return COLA_ERR_INVALID;
  const PipeShape ps = pipe_shape(g, p.pipe_kb, p.pipe_ept, p.pipe_inplace);
  const long long plane = (long long)g.n * g.pc;
  if (!plan3_pencils_launch(fp, ps.lw, ps.ctas, ps.threads, ps.smem, +1, dst, plane, g.pc, g.nc, ps.nchunks, ps.ntiles,
                            st, src, &mul))
    return COLA_ERR_INVALID;
  return check_launch("pencils_x_mul");
}

bool c2r_rows_dense_ok(const FftPlan& p, const Grid3& g) {
  FastPlan fp;
  return !p.row_pipe && fast_plan(p, &fp) && plan3_id(fp) != 0 && g.nc >= 2;
}

int launch_c2r_rows_dense(const FftPlan& p, const Grid3& g, const float2* data, float scale, float* out,
                          cudaStream_t st) {
  FastPlan fp;
  if (!c2r_rows_dense_ok(p, g) || !fast_plan(p, &fp)) return COLA_ERR_INVALID;
  const long long nrows = (long long)g.rows();
  const TileShape t = row_shape(p.row_ept, g, 2);
  const bool e8 = p.row_ept == 8 && g.n <= kTileElems / 2;
  const unsigned blocks = (unsigned)((nrows + (2LL << t.lw) - 1) / (2LL << t.lw));
  float2* d = const_cast<float2*>(data);   // only read when out is given
  const bool ok = e8 ? plan3_c2r_launch<8>(fp, t.lw, blocks, t.threads, t.smem, d, g.pc, nrows, st, out, scale)
                     : plan3_c2r_launch<16>(fp, t.lw, blocks, t.threads, t.smem, d, g.pc, nrows, st, out, scale);
  return ok ? check_launch("c2r_dense") : COLA_ERR_INVALID;
}

int launch_pencils(const FftPlan& p, const Grid3& g, int axis, int dir, float2* data, cudaStream_t st) {
  const long long plane = (long long)g.n * g.pc;
  const long long jstride = axis == 1 ? g.pc : plane;
  const long long ostride = axis == 1 ? plane : g.pc;
  FastPlan fp;
  if (fast_plan(p, &fp) && pipe_ok(p, g)) {
    const PipeShape ps = pipe_shape(g, p.pipe_kb, p.pipe_ept, p.pipe_inplace);
    if (p.pipe_inplace && p.pipe_ept == 16 &&
        plan3_pencils_launch(fp, ps.lw, ps.ctas, ps.threads, ps.smem, dir, data, jstride, ostride, g.nc, ps.nchunks,
                             ps.ntiles, st))
      return check_launch("pencils_plan3");
    if (max_radix(fp) > 8)
      pipe_pencils_launch<16>(fp, ps.lw, ps.ctas, ps.threads, ps.smem, dir, p.pipe_ept, p.pipe_inplace, data, jstride,
                              ostride, g.nc, ps.nchunks, ps.ntiles, st);
    else
      pipe_pencils_launch<8>(fp, ps.lw, ps.ctas, ps.threads, ps.smem, dir, p.pipe_ept, p.pipe_inplace, data, jstride,
                             ostride, g.nc, ps.nchunks, ps.ntiles, st);
    return check_launch("pencils_pipe");
  }
  if (fast_plan(p, &fp)) {
    const int nbuf = fp.nst >= 3 ? 2 : 1;
    const TileShape t = wide_shape(p, g, fast_shape(g.n, largest_pow2_le(g.nc), nbuf), nbuf);
    dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
    if (max_radix(fp) > 8)
      fast_pencils_launch<16>(fp, t.lw, grid, t.threads, t.smem, dir, data, jstride, ostride, g.nc, st);
    else
      fast_pencils_launch<8>(fp, t.lw, grid, t.threads, t.smem, dir, data, jstride, ostride, g.nc, st);
    return check_launch("pencils_fast");
  }
  const TileShape t = tile_shape(g.n, largest_pow2_le(g.nc));
  dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
  generic_pencils_launch(p.dev, t.lw, grid, t.threads, t.smem, dir, data, jstride, ostride, g.nc, st);
  return check_launch("pencils");
}

int launch_green_x(const FftPlan& p, const Grid3& g, const float2* in, float2* const out[3],
                   const float* dtab, float scale, cudaStream_t st, float2* spec_out, bool* spec_saved) {
  if (spec_saved) *spec_saved = false;
  const double kf = 2.0 * M_PI / g.n;
  const double n3 = (double)g.n * g.n * g.n;
  const float g_scale = (float)((double)scale / (kf * kf * n3));
  FastPlan fp;
  if (fast_plan(p, &fp)) {
    if (p.green_ept == 8 && g.n <= kTileElems / 2) {
      // half the elements per thread: tiles of at most 3072 elements keep 384 threads
      const TileShape t = fast_shape(g.n, largest_pow2_le(g.nc) < kTileElems / 2 / g.n ?
                                          largest_pow2_le(g.nc) : largest_pow2_le(kTileElems / 2 / g.n),
                                     fp.nst >= 3 ? 2 : 1);
      int th = ((g.n << t.lw) + 7) / 8;
      th = ((th + 31) / 32) * 32;
      dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
      if (max_radix(fp) > 8)
        fast_green_launch<16, 8>(fp, t.lw, grid, th, t.smem, in, out, g.pc, g.nc, dtab, g_scale, spec_out, st);
      else
        fast_green_launch<8, 8>(fp, t.lw, grid, th, t.smem, in, out, g.pc, g.nc, dtab, g_scale, spec_out, st);
      if (spec_saved) *spec_saved = spec_out != nullptr;
      return check_launch("green_fast8");
    }
    const int nbuf = fp.nst >= 3 ? 2 : 1;
    const TileShape t = wide_shape(p, g, fast_shape(g.n, largest_pow2_le(g.nc), nbuf), nbuf);
    dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
    if (plan3_green_launch(fp, t.lw, grid, t.threads, t.smem, in, out, g.pc, g.nc, dtab, g_scale, spec_out, st)) {
      if (spec_saved) *spec_saved = spec_out != nullptr;
      return check_launch("green_plan3");
    }
    if (max_radix(fp) > 8)
      fast_green_launch<16, 16>(fp, t.lw, grid, t.threads, t.smem, in, out, g.pc, g.nc, dtab, g_scale, spec_out, st);
    else
      fast_green_launch<8, 16>(fp, t.lw, grid, t.threads, t.smem, in, out, g.pc, g.nc, dtab, g_scale, spec_out, st);
    if (spec_saved) *spec_saved = spec_out != nullptr;
    return check_launch("green_fast");
  }
  const TileShape t = tile_shape(g.n, largest_pow2_le(g.nc));
  dim3 grid((g.nc + (1 << t.lw) - 1) >> t.lw, g.n);
  generic_green_launch(p.dev, t.lw, grid, t.threads, t.smem, in, out, g.pc, g.nc, dtab, g_scale, st);
  return check_launch("green_x");
}

}  // namespace cola
