// Host side of the SegSALSA-STR library: planning, workspace, iteration loop, C ABI.
//
// One iteration of SALSA (eqs. 12-14) is, in launch order,
//   [k > 0]  row FFT forward (gathers rhs^k from the sweep's tile partials) -> column solve
//            -> row FFT inverse: z^{k+1} = (3 I + J^T J)^{-1} G^T (u^k + d^k)       (eq. 12)
//   sweep:   u^{k+1}, d^{k+1} and the tile partials of rhs^{k+1}                  (eqs. 13-14)
// For k = 0 the z-update is the identity (u^0 = G z^0, d^0 = 0), so it is skipped.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/segsalsa_str.h"
#include "aux.cuh"
#include "fft.cuh"
#include "zfused.cuh"
#include "launch.h"
#include "mlr.cuh"
#include "adjoint.cuh"
#include "wide.cuh"

namespace sgs {

enum Kind { KIND_SWEEP = 0, KIND_ROWF = 1, KIND_COL = 2, KIND_ROWI = 3, KIND_DIAG = 4, KIND_OTHER = 5,
            KIND_MLR = 6, KIND_ADJ = 7, KIND_ZF = 8 };
constexpr int NKIND = 9;
constexpr int MAXCOV = 2;           // tile covers per row / column in the partial gather
constexpr int TRACE_CAP = 128;      // device trace records before a flush to the host
// Images from this many pixels up run the pipelined row passes unless the tiling says otherwise.
constexpr long long ROWPIPE_DEFAULT_PIXELS = 1LL << 62;

static thread_local std::string g_last_error;

static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct SolverBase {
  virtual ~SolverBase() {}
  std::string err;
  virtual int set_probs(const void* p, int layout, int on_device) = 0;
  virtual int solve(int iters, double* trace, int every, int* nrec) = 0;
  virtual int get_labels(int32_t* lab, int on_device) = 0;
  virtual int get_z(void* z, int layout, int on_device) = 0;
  virtual int get_iteration(int* k) const = 0;
  virtual int get_state(void* z, void* d1, void* d2, void* d3, void* d4, void* rhs, int dev) = 0;
  virtual int set_state(const void* z, const void* d1, const void* d2, const void* d3,
                        const void* d4, const void* rhs, int k, int dev) = 0;
  virtual int linear_solve(const void* rhs, void* z, int dev) = 0;
  virtual int set_spectra(const void* x, const void* w, const float* bias, int d, int dev) = 0;
  virtual int get_probs(void* p, int layout, int dev) = 0;
  virtual int set_profiling(int on) = 0;
  virtual int kernel_stats(int64_t* launches, double* ms) = 0;
  virtual int reset_stats() = 0;
  virtual int traffic(double* sweep, double* iter) const = 0;
  virtual segsalsa_str_tiling tiling() const = 0;
  // batch support: every call below enqueues on the given stream and never synchronizes
  virtual bool ready() const = 0;                      // set_probs has been called
  virtual bool graphable() const = 0;                  // next iteration is a plain one (k >= 1)
  virtual int enqueue_iterations(int len, cudaStream_t s) = 0;  // launches only; state unchanged
  virtual void advance(int len) = 0;                   // account for `len` enqueued iterations
  virtual int enqueue_eager_iteration(cudaStream_t s) = 0;       // one iteration, state advanced
  virtual int enqueue_read_err(int* host, cudaStream_t s) = 0;   // copy the device error flag
  virtual int clear_err(cudaStream_t s) = 0;
  virtual void invalidate() = 0;                       // forget p and the iterates
  virtual int set_g4(int mode) = 0;
  virtual int set_wait_budget(long long cycles, int probe) = 0;
  virtual int set_log_probs(const void* logp, int layout, int dev) = 0;
  virtual int set_lambda(double lam) = 0;
  virtual int set_weights(const double* w) = 0;
  virtual int backward(int iters, const void* zbar, int layout, void* glogp, double* glam,
                       double* gom, int every, int dev) = 0;
  virtual int generation() const = 0;                  // changes when launches change
  int fail(int code, const std::string& m) { err = m; return code; }
};

// Validation of the parameters shared by create and workspace_bytes.
static int check_params(const segsalsa_str_params* pr, std::string& msg) {
  if (!pr) { msg = "params is NULL"; return SEGSALSA_ERR_ARG; }
  if (pr->M < 0 || pr->M > 5) { msg = "M must be in [0, 5]"; return SEGSALSA_ERR_ARG; }
  if (pr->K < 2 || pr->K > 32) { msg = "K must be in [2, 32]"; return SEGSALSA_ERR_ARG; }
  const int minsz = 2 * pr->M + 2;
  if (pr->H < minsz || pr->W < minsz) { msg = "H and W must be >= 2M+2"; return SEGSALSA_ERR_ARG; }
  if ((long long)pr->H * pr->W > (1LL << 30)) { msg = "image too large"; return SEGSALSA_ERR_ARG; }
  if (pr->H > 65535 || pr->W > 65535) { msg = "H and W must be <= 65535"; return SEGSALSA_ERR_ARG; }
  if (!(pr->lambda >= 0.0) || !std::isfinite(pr->lambda)) { msg = "lambda must be finite and >= 0"; return SEGSALSA_ERR_ARG; }
  if (!(pr->mu > 0.0) || !std::isfinite(pr->mu)) { msg = "mu must be finite and > 0"; return SEGSALSA_ERR_ARG; }
  if (pr->schatten_p != 1 && pr->schatten_p != 2 && pr->schatten_p != SEGSALSA_SCHATTEN_INF) {
    msg = "schatten_p must be 1, 2 or SEGSALSA_SCHATTEN_INF"; return SEGSALSA_ERR_ARG;
  }
  if (pr->precision != SEGSALSA_FP32 && pr->precision != SEGSALSA_FP64) {
    msg = "precision must be SEGSALSA_FP32 or SEGSALSA_FP64"; return SEGSALSA_ERR_ARG;
  }
  const int L = (2 * pr->M + 1) * (2 * pr->M + 1);
  if (pr->weights) {
    for (int j = 0; j < L; ++j)
      if (!std::isfinite(pr->weights[j])) { msg = "weights must be finite"; return SEGSALSA_ERR_ARG; }
  } else if (!(pr->sigma > 0.0) || !std::isfinite(pr->sigma)) {
    msg = "sigma must be finite and > 0 when weights is NULL"; return SEGSALSA_ERR_ARG;
  }
  return SEGSALSA_OK;
}

// Shift weights: given, or omega_j = sqrt(normalised Gaussian) (the weighted shifts of Sec. 3).
static std::vector<double> make_weights(const segsalsa_str_params* pr) {
  const int M = pr->M, P = 2 * M + 1;
  std::vector<double> w(P * P);
  if (pr->weights) {
    for (int j = 0; j < P * P; ++j) w[j] = pr->weights[j];
    return w;
  }
  double s = 0.0;
  for (int dy = -M; dy <= M; ++dy)
    for (int dx = -M; dx <= M; ++dx) {
      const double g = std::exp(-(double)(dy * dy + dx * dx) / (2.0 * pr->sigma * pr->sigma));
      w[(dy + M) * P + dx + M] = g;
      s += g;
    }
  for (auto& v : w) v = std::sqrt(v / s);
  return w;
}

// Everything decided from the parameters before memory exists.
struct Plan {
  int H, W, K, M, L, n, G, NC;
  int ntx, nty, THmax, EHmax, EWmax, ntiles;
  size_t sweep_smem, sweep_smem_diag;
  int Wh, Mf, blue, QB, nqblk;
  RowLaunch row;
  // pipelined row passes (persistent CTAs): on/off, vertical-cover stage slots, shared memory
  // of the forward (enough for the partial and the dense source) and inverse kernels, grids
  int rp, rp_nslot;
  size_t rp_smem_f, rp_smem_i;
  int rp_grid_f, rp_grid_i;
  // power-of-two rows: compile-time Stockham kernels with the first stage fused into the load
  int p2, QBi;             // QBi: class pairs per CTA of the inverse power-of-two pass
  size_t p2_smem, p2_smem_i;
  int CB, NSEG, SL, col_threads, ncolblk;
  int row_threads, col_rows;   // target threads of a row-pass CTA; rows per column segment
  size_t col_smem;
  // z-update fused over a cluster (0: three passes), its class-pair groups, threads, memory
  int zf_cs, zf_qg, zf_rmax, zf_groups, zf_threads;
  size_t zf_smem;
  // z-update as one launch of persistent CTAs taking the units of the three passes in order
  // (ordered tickets; the one-unit row form only)
  int zs, zs_threads, zs_grid;
  size_t zs_smem;
  int nproj_blk, nprior_blk;
  // wide patches (M >= 3): two-launch sweep (gram + transpose tiles) writing a dense rhs
  int wide, wntx1, wntiles1, wnblk2;
  std::vector<int> covY, covX;  // [H][MAXCOV], [W][MAXCOV]
};

static bool build_cover(int N, int ntile, int lo, int hi, std::vector<int>& cov) {
  cov.assign((size_t)N * MAXCOV, -1);
  std::vector<int> cnt(N, 0);
  for (int t = 0; t < ntile; ++t) {
    const int a = (int)(((long long)t * N) / ntile), b = (int)(((long long)(t + 1) * N) / ntile);
    const int ext = (b - a) + lo + hi;
    for (int e = 0; e < ext; ++e) {
      const int x = wrap_idx(a - lo + e, N);
      if (cnt[x] >= MAXCOV) return false;
      cov[(size_t)x * MAXCOV + cnt[x]++] = (t << 16) | e;
    }
  }
  return true;
}

// Tiling fields accepted by the *_tiled calls (0 = default).
static int check_tiling(const segsalsa_str_tiling* t, std::string& msg) {
  if (!t) return SEGSALSA_OK;
  if (t->tile_rows && (t->tile_rows < 4 || t->tile_rows > 32)) { msg = "tile_rows must be 0 or 4..32"; return SEGSALSA_ERR_ARG; }
  if (t->row_pairs < 0 || t->row_pairs > 64) { msg = "row_pairs must be 0..64"; return SEGSALSA_ERR_ARG; }
  if (t->col_block < 0 || t->col_block > 8) { msg = "col_block must be 0..8"; return SEGSALSA_ERR_ARG; }
  if (t->row_threads && (t->row_threads < 64 || t->row_threads > 1024)) { msg = "row_threads must be 0 or 64..1024"; return SEGSALSA_ERR_ARG; }
  if (t->col_rows && (t->col_rows < 2 || t->col_rows > 4096)) { msg = "col_rows must be 0 or 2..4096"; return SEGSALSA_ERR_ARG; }
  if (t->zfuse && t->zfuse != 1 && t->zfuse != 2 && t->zfuse != 3 && t->zfuse != 4 && t->zfuse != 8 &&
      t->zfuse != 16) {
    msg = "zfuse must be 0, 1, 2, 3, 4, 8 or 16"; return SEGSALSA_ERR_ARG;
  }
  if (t->row_pipe < 0 || t->row_pipe > 3) { msg = "row_pipe must be 0, 1, 2 or 3"; return SEGSALSA_ERR_ARG; }
  return SEGSALSA_OK;
}

static int floor_pow2(int v) {
  int r = 1;
  while (2 * r <= v) r *= 2;
  return r;
}

template <typename T>
static int make_plan(const segsalsa_str_params* pr, Plan& pl, std::string& msg,
                     const segsalsa_str_tiling* tl = nullptr) {
  if (int rc = check_tiling(tl, msg)) return rc;
  pl.H = pr->H; pl.W = pr->W; pl.K = pr->K; pl.M = pr->M;
  pl.L = (2 * pl.M + 1) * (2 * pl.M + 1);
  pl.n = pl.H * pl.W;
  const int K = pl.K, M = pl.M, H = pl.H, W = pl.W;
  pl.G = K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  // columns per tile: 256/G, fewer when a CTA's shared memory (two row stages, the z tile and
  // the accumulators) would not fit
  const int cand[] = {16, 12, 8, 6, 4};
  for (pl.NC = 256 / pl.G; pl.NC > 1; --pl.NC) {
    const size_t s = sweep_smem_bytes<T>(pl.NC, 16 + 2 * M + 1, pl.NC + 2 * M + 1, pl.G, pl.L, K, true);
    if (s <= 220 * 1024) break;
  }
  pl.ntx = (W + pl.NC - 1) / pl.NC;
  // tile height: the largest of {16, 12, 8, 6, 4} that still gives two CTAs per SM (152 SMs);
  // with more than one tile row every tile must be at least 2M+1 rows high
  pl.THmax = 0;
  int fallback = 0;
  for (int th : cand) {
    const int nty = (H + th - 1) / th;
    if (nty > 1 && H / nty < 2 * M + 1) continue;
    fallback = th;
    if ((long long)nty * pl.ntx >= 304) { pl.THmax = th; break; }
  }
  if (!pl.THmax) pl.THmax = fallback ? fallback : H;
  if (tl && tl->tile_rows) {
    // requested height, raised until every tile of a multi-row tiling has >= 2M+1 rows
    int th = tl->tile_rows;
    while (th < H && (H + th - 1) / th > 1 && H / ((H + th - 1) / th) < 2 * M + 1) ++th;
    pl.THmax = std::min(th, H);
  }
  pl.nty = (H + pl.THmax - 1) / pl.THmax;
  pl.EHmax = pl.THmax + 2 * M + 1;
  pl.EWmax = pl.NC + 2 * M + 1;
  pl.sweep_smem = sweep_smem_bytes<T>(pl.NC, pl.EHmax, pl.EWmax, pl.G, pl.L, K, false);
  pl.sweep_smem_diag = sweep_smem_bytes<T>(pl.NC, pl.EHmax, pl.EWmax, pl.G, pl.L, K, true);
  pl.wide = M >= 3;
  pl.wntx1 = (W + 256 / pl.G - 1) / (256 / pl.G);
  pl.wntiles1 = pl.wntx1 * ((H + WG_TH - 1) / WG_TH);
  // transpose: the gram tiles again (one row of 256 / G targets), at most 8 blocks per SM
  pl.wnblk2 = std::max(1, std::min(152 * 8, pl.wntiles1));
  if (pl.wide) {
    if (wide_gram_smem<T>(M, pl.G) > 227 * 1024) {
      msg = "wide-patch tiles do not fit in shared memory"; return SEGSALSA_ERR_ARG;
    }
  } else if (pl.sweep_smem_diag > 227 * 1024) {
    msg = "tile does not fit in shared memory"; return SEGSALSA_ERR_ARG;
  }
  pl.ntiles = pl.ntx * pl.nty;
  if ((long long)pl.ntiles * pl.EHmax * pl.EWmax * K >= (1LL << 31)) { msg = "image too large for 32-bit partial offsets"; return SEGSALSA_ERR_ARG; }
  if (M >= 3) {
    // the wide-patch sweep writes a dense rhs: no tile partials to gather (trivial covers)
    pl.covY.assign((size_t)H * MAXCOV, -1);
    pl.covX.assign((size_t)W * MAXCOV, -1);
    for (int y = 0; y < H; ++y) pl.covY[(size_t)y * MAXCOV] = 0;
    for (int x = 0; x < W; ++x) pl.covX[(size_t)x * MAXCOV] = 0;
  } else if (!build_cover(H, pl.nty, M, M + 1, pl.covY) || !build_cover(W, pl.ntx, M, M + 1, pl.covX)) {
    msg = "image too small for the tiling"; return SEGSALSA_ERR_ARG;
  }
  // row FFT
  pl.Wh = W / 2 + 1;
  {
    FftPlan<T> fp{};
    if (!make_fft_plan<T>(W, fp)) { msg = "no FFT plan for this row length"; return SEGSALSA_ERR_ARG; }
    pl.Mf = fp.Mf;
    pl.blue = fp.blue;
  }
  if (pl.Mf > 8192) { msg = "row length too large for the shared-memory FFT"; return SEGSALSA_ERR_ARG; }
  const int Q = (K + 1) / 2;
  // small images (latency bound): fewer class pairs per CTA until the grid has two CTAs per SM
  // (145 x 145, K = 16: two pairs per CTA, 33.4 us per iteration of one solve against 35.0 us
  // with four pairs, one CTA per SM; a target of eight per SM, one pair per CTA, measured 12 %
  // slower with earlier kernels); larger ones: as many as fit (contiguous 64-byte pixel reads,
  // fewer CTAs)
  const bool small_image = (long long)H * W < 65536;
  pl.QB = row_pairs_per_cta(pl.Mf, Q, small_image ? H : (1 << 30));
  if (tl && tl->row_pairs) {
    const int qmax = row_pairs_per_cta(pl.Mf, Q, 1 << 30, 8192 * 4 / (int)sizeof(T), false);  // the most a CTA takes
    pl.QB = std::min(floor_pow2(tl->row_pairs), qmax);
  }
  pl.nqblk = (Q + pl.QB - 1) / pl.QB;
  // row CTAs: 256 threads below a megapixel (several CTAs per SM hide the per-stage barrier
  // latency), 1024 above (long rows, more work per CTA)
  const bool large_image = (long long)H * W >= (1LL << 20);
  pl.row_threads = large_image ? 1024 : 256;
  if (tl && tl->row_threads) pl.row_threads = floor_pow2(tl->row_threads);
  pl.row = row_launch_config<T>(W, pl.Mf, pl.blue, pl.QB, pl.row_threads);
  if (pl.row.smem > 227 * 1024) { msg = "row too long for the shared-memory FFT"; return SEGSALSA_ERR_ARG; }
  // pipelined row passes: on request (row_pipe = 2) or by default (row_pipe = 0) for images
  // of ROWPIPE_DEFAULT_PIXELS and more; the stage takes both vertical covers of a row at once
  // while two CTAs still share an SM
  {
    const int req = tl ? tl->row_pipe : 0;
    // by default for rows of 2048 and more (measured faster there; shorter power-of-two rows
    // run the one-unit kernels with more pairs per CTA at least as fast)
    pl.p2 = (((req == 0 && W >= 2048) || req == 3) && p2_ok<T>(W, pl.blue, pl.QB, K)) ? 1 : 0;
    // pair count of the power-of-two kernels, unless the tiling fixes it: the largest of 4, 2, 1
    // whose CTA (W / 8 x pairs threads, two transform buffers) fits (2048-point rows, K = 16:
    // four pairs, forward 294 -> 256 us and inverse 216 -> 206 us at 2048 x 2048)
    if (pl.p2 && !(tl && tl->row_pairs)) {
      for (int qb : {4, 2, 1}) {
        if (!p2_ok<T>(W, pl.blue, qb, K) || W / 8 * qb > 1024 ||
            p2_smem_bytes<T>(W, qb) > 227 * 1024 || qb > Q)
          continue;
        pl.QB = qb;
        break;
      }
      pl.nqblk = (Q + pl.QB - 1) / pl.QB;
      pl.row = row_launch_config<T>(W, pl.Mf, pl.blue, pl.QB, pl.row_threads);
    }
    pl.QBi = pl.QB;
    pl.p2_smem = p2_smem_bytes<T>(W, pl.QB);
    pl.p2_smem_i = p2_smem_bytes<T>(W, pl.QBi);
    if (std::max(pl.p2_smem, pl.p2_smem_i) > 227 * 1024) pl.p2 = 0;
    pl.rp = (req == 2 || (req == 0 && !pl.p2 && (long long)H * W >= ROWPIPE_DEFAULT_PIXELS)) ? 1 : 0;
    const size_t two = rowpipe_smem_bytes<T>(true, W, pl.Mf, pl.Wh, pl.QB, pl.ntx, pl.EWmax, 2, false);
    pl.rp_nslot = two <= 112 * 1024 ? 2 : 1;
    pl.rp_smem_f = std::max(
        rowpipe_smem_bytes<T>(true, W, pl.Mf, pl.Wh, pl.QB, pl.ntx, pl.EWmax, pl.rp_nslot, false),
        rowpipe_smem_bytes<T>(true, W, pl.Mf, pl.Wh, pl.QB, pl.ntx, pl.EWmax, 1, true));
    pl.rp_smem_i = rowpipe_smem_bytes<T>(false, W, pl.Mf, pl.Wh, pl.QB, pl.ntx, pl.EWmax, 1, false);
    if (std::max(pl.rp_smem_f, pl.rp_smem_i) > 227 * 1024) pl.rp = 0;
    pl.rp_grid_f = pl.rp_grid_i = 0;  // set at create (occupancy of the device)
  }
  // column solve: column blocks of CB complex values, all H rows in shared memory (<= 64 KiB
  // so that several CTAs share an SM), NSEG segments per column
  pl.CB = sizeof(T) == 4 ? 8 : 4;
  while ((size_t)H * pl.CB * sizeof(cplx<T>) > 64 * 1024 && pl.CB > 1) pl.CB /= 2;
  if ((size_t)H * pl.CB * sizeof(cplx<T>) > 200 * 1024) { msg = "image too tall for the column solve"; return SEGSALSA_ERR_ARG; }
  // small images: thinner column blocks until the grid has one CTA per SM
  while (small_image && pl.CB > 1 && (long long)pl.Wh * K / pl.CB < 152) pl.CB /= 2;
  if (tl && tl->col_block) {
    pl.CB = floor_pow2(tl->col_block);
    while ((size_t)H * pl.CB * sizeof(cplx<T>) > 200 * 1024 && pl.CB > 1) pl.CB /= 2;
  }
  pl.col_smem = (size_t)H * pl.CB * sizeof(cplx<T>);
  const int nseq = 2 * pl.CB;
  // segment length: 8 rows below a megapixel (short serial chains), 32 rows above (the two
  // warm-up recursions per segment then cost less than the segment itself)
  pl.col_rows = large_image ? 32 : 8;
  if (tl && tl->col_rows) pl.col_rows = tl->col_rows;
  pl.NSEG = std::max(1, std::min(H / pl.col_rows, 1024 / nseq));
  col_segments(H, pl.NSEG, nseq, (int)sizeof(T), pl.SL, pl.NSEG);
  pl.col_threads = (nseq * pl.NSEG + 31) / 32 * 32;
  // the one-launch z-update runs the column units on its CTAs of at most ZSEQ_MAX_THREADS:
  // longer segments where the column pass would need more (a three-launch handle given the
  // reported col_rows plans the same segments)
  if (tl && tl->zfuse == 3 && !pl.p2 && !pl.rp) {
    while (pl.col_threads > ZSEQ_MAX_THREADS && pl.col_rows < H) {
      ++pl.col_rows;
      pl.NSEG = std::max(1, std::min(H / pl.col_rows, 1024 / nseq));
      col_segments(H, pl.NSEG, nseq, (int)sizeof(T), pl.SL, pl.NSEG);
      pl.col_threads = (nseq * pl.NSEG + 31) / 32 * 32;
    }
  }
  pl.ncolblk = (pl.Wh * K + pl.CB - 1) / pl.CB;
  // z-update in one launch, on request only (measured slower than the three passes at every
  // shape tried): clusters of CS CTAs (one band of rows each) per class pair, when a band's
  // transforms and half spectra fit in shared memory (the handle falls back to three passes
  // if the device cannot hold the cluster).
  pl.zf_cs = pl.zf_qg = pl.zf_rmax = pl.zf_groups = pl.zf_threads = 0;
  pl.zf_smem = 0;
  {
    const int req = tl ? tl->zfuse : 0;
    std::vector<int> cands;
    if (req > 1 && req != 3) cands = {req};
    const bool direct = !pl.blue && largest_prime_factor(pl.Mf) > 7;
    for (int cs : cands) {
      const int rmax = (H + cs - 1) / cs;
      if (H < 2 * cs || (long long)pl.Mf * rmax > 65536) continue;
      const size_t sm = zf_smem_bytes<T>(W, pl.Mf, pl.blue, pl.Wh, rmax, 1, 1);
      if (sm > 160 * 1024) continue;
      const int elems = pl.Mf * rmax;
      const int t = ((direct ? elems / 2 : elems / 8) + 31) / 32 * 32;
      pl.zf_cs = cs;
      pl.zf_qg = 1;
      pl.zf_rmax = rmax;
      pl.zf_groups = Q;
      pl.zf_threads = std::max(128, std::min(512, t));
      pl.zf_smem = sm;
      break;
    }
  }
  // the three passes in one launch of persistent CTAs (one-unit row form only; grid set at
  // create from the device's occupancy)
  pl.zs = pl.zs_threads = pl.zs_grid = 0;
  pl.zs_smem = 0;
  {
    const int req = tl ? tl->zfuse : 0;
    if (req == 3 && !pl.p2 && !pl.rp && !pl.zf_cs && pl.col_threads <= ZSEQ_MAX_THREADS) {
      pl.zs = 1;
      pl.zs_threads = std::min(ZSEQ_MAX_THREADS, (std::max(pl.row.threads, pl.col_threads) + 31) / 32 * 32);
      pl.zs_smem = std::max(pl.row.smem, pl.col_smem);
      if (pl.zs_smem > 227 * 1024) pl.zs = 0;
    }
  }
  // diagnostics
  // one pixel per thread (projection) and tiles of PRIOR_TH x PRIOR_TW pixels (prior): one
  // round per block up to eight blocks per SM, grid-stride rounds beyond (small images need
  // every SM: four rounds per block left 20 blocks for 145 x 145, 27 instead of 15 us)
  const int cap = 152 * 8;
  pl.nproj_blk = std::max(1, std::min(cap, (pl.n + AUX_THREADS - 1) / AUX_THREADS));
  {
    const int pt = ((H + PRIOR_TH - 1) / PRIOR_TH) * ((W + PRIOR_TW - 1) / PRIOR_TW);
    pl.nprior_blk = std::max(1, std::min(cap, pt));
  }
  return SEGSALSA_OK;
}

// Carves the workspace (dry run: only sizes).
struct Carver {
  char* base;
  size_t off = 0;
  template <class U> U* take(size_t count) {
    off = align_up(off, 256);
    U* p = base ? reinterpret_cast<U*>(base + off) : nullptr;
    off += count * sizeof(U);
    return p;
  }
};

template <typename T>
struct Buffers {
  T *p, *z, *dloc, *d2, *P, *P2, *zp, *tmp, *rhsd;
  T* dcmp;  // compact local duals [n][K + 2] (d3, c1, c4) of the affine fused sweep
  T* wbuf;  // wide patches: scratch [n][L][K][2] (the old d2 of a traced sweep; checkpoint read-out)
  T* coef;  // wide patches: [n][4] the 2 x 2 prox matrix A of the last sweep (d2 = V (A - I))
  cplx<T>* S;
  int32_t* lab;
  double *dsq, *dproj, *dprior, *dtrace;
  int* flag;
  int* err;  // set by kernels whose bounded waits gave up
  unsigned int* zctr;  // [4] work-ticket counters of the one-launch z-update (0 between launches)
  T* omega;
  int *covY, *covX, *offX;
  T *beta, *gain, *wfac;
  int* nwarm;
  cplx<T>*tw, *chirp, *bhat;
};

template <typename T>
static size_t carve(const Plan& pl, char* base, Buffers<T>& b) {
  Carver c{base};
  const size_t nK = (size_t)pl.n * pl.K;
  // p, dloc and d2 are read by 16-byte-rounded bulk copies: 64 bytes of slack after each
  b.p = c.take<T>(nK + 64 / sizeof(T));
  b.z = c.take<T>(nK);
  b.dloc = c.take<T>(3 * nK + 64 / sizeof(T));
  b.dcmp = c.take<T>((size_t)pl.n * (pl.K + 2) + 64 / sizeof(T));
  b.d2 = c.take<T>(2 * (size_t)pl.L * nK + 64 / sizeof(T));
  const size_t tslot = (size_t)pl.ntiles * pl.EHmax * pl.EWmax * pl.K;
  b.P = c.take<T>(tslot);
  b.P2 = c.take<T>(tslot);
  b.zp = c.take<T>(nK);
  b.tmp = c.take<T>(nK);
  b.rhsd = c.take<T>(nK);
  b.S = c.take<cplx<T>>((size_t)pl.H * pl.Wh * pl.K);
  b.wbuf = pl.wide ? c.take<T>(2 * (size_t)pl.L * nK) : nullptr;
  b.coef = pl.wide ? c.take<T>(4 * (size_t)pl.n) : nullptr;
  b.lab = c.take<int32_t>(pl.n);
  b.dsq = c.take<double>(std::max(pl.ntiles, pl.wntiles1));
  b.dproj = c.take<double>(4 * (size_t)pl.nproj_blk);
  b.dprior = c.take<double>(pl.nprior_blk);
  b.dtrace = c.take<double>(6 * (size_t)TRACE_CAP);
  b.flag = c.take<int>(1);
  b.err = c.take<int>(1);
  b.zctr = c.take<unsigned int>(4);
  b.omega = c.take<T>(pl.L);
  b.covY = c.take<int>((size_t)pl.H * MAXCOV);
  b.covX = c.take<int>((size_t)pl.W * MAXCOV);
  b.offX = c.take<int>((size_t)pl.W * MAXCOV);
  b.beta = c.take<T>(pl.Wh);
  b.gain = c.take<T>(pl.Wh);
  b.wfac = c.take<T>(pl.Wh);
  b.nwarm = c.take<int>(pl.Wh);
  b.tw = c.take<cplx<T>>(pl.Mf);
  b.chirp = c.take<cplx<T>>(pl.W);
  b.bhat = c.take<cplx<T>>(pl.Mf);
  return align_up(c.off, 256);
}

#define SGS_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(SEGSALSA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <typename T>
class Solver : public SolverBase {
 public:
  Plan pl;
  Buffers<T> b{};
  std::vector<double> omega;
  double lambda = 0, mu = 1, c_omega = 0;
  int sp = 1;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  void* ws = nullptr;
  bool own_ws = false;
  int iter = 0;
  bool have_probs = false;
  bool rhs_dense = false;  // next z-update reads b.rhsd instead of the partials
  // the local duals are held in compact form (b.dcmp, written by the affine fused sweep)
  // rather than in full form (b.dloc: set_probs, set_state, the simplex and wide sweeps)
  bool dl_cmp = false;

  // The form of the local duals the handle's sweeps keep from iteration to iteration (graphs
  // are captured in it): compact for the affine fused sweep, full otherwise.
  bool dl_steady() const { return pl.wide || (g4 == SEGSALSA_G4_SIMPLEX ? !dl_cmp : dl_cmp); }
  int64_t nlaunch[NKIND] = {0};
  double ms[NKIND] = {0};
  bool profiling = false;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> evs;
  std::vector<cudaEvent_t> evpool;
  // CUDA graphs of iteration chunks: key (length, traced) -> executable graph and the launch
  // counts per kind it contains
  struct Chunk {
    cudaGraphExec_t exec = nullptr;
    int64_t launches[NKIND] = {0};
  };
  std::map<std::pair<int, int>, Chunk> chunks;
  double* trace_host = nullptr;  // pinned staging for trace records
  void* mlr_buf = nullptr;       // device staging of host spectra / weights / biases
  size_t mlr_cap = 0;
  int trace_host_cap = 0;
  bool use_graphs = true;
  int g4 = SEGSALSA_G4_AFFINE;   // MPO of g4: affine set (eq. 10) or probability simplex
  int gen = 0;
  long long wait_budget = WAIT_BUDGET_CYCLES;  // bounded device-side waits (clock cycles)
  int wait_probe = 0;            // 1: the next bulk-copy waits cannot complete (wait test)

  ~Solver() override {
    if (st) cudaStreamSynchronize(st);
    for (auto& kv : chunks)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (trace_host) cudaFreeHost(trace_host);
    if (mlr_buf) cudaFree(mlr_buf);
    for (auto& e : evs) { cudaEventDestroy(std::get<1>(e)); cudaEventDestroy(std::get<2>(e)); }
    for (auto e : evpool) cudaEventDestroy(e);
    if (own_ws && ws) cudaFree(ws);
    if (own_stream && st) cudaStreamDestroy(st);
  }

  int init(const segsalsa_str_params* pr, void* workspace, size_t wsbytes,
           const segsalsa_str_tiling* tl = nullptr) {
    std::string msg;
    int rc = make_plan<T>(pr, pl, msg, tl);
    if (rc) return fail(rc, msg);
    omega = make_weights(pr);
    lambda = pr->lambda;
    mu = pr->mu;
    sp = pr->schatten_p == SEGSALSA_SCHATTEN_INF ? 0 : pr->schatten_p;
    c_omega = 0.0;
    for (double w : omega) c_omega += w * w;
    const size_t need = carve<T>(pl, nullptr, b);
    if (workspace) {
      if (wsbytes < need) return fail(SEGSALSA_ERR_OOM, "workspace too small");
      if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(SEGSALSA_ERR_ARG, "workspace must be 256-byte aligned");
      ws = workspace;
    } else {
      cudaError_t e = cudaMalloc(&ws, need);
      if (e != cudaSuccess) { ws = nullptr; return fail(SEGSALSA_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
      own_ws = true;
    }
    carve<T>(pl, reinterpret_cast<char*>(ws), b);
    if (pr->stream) st = reinterpret_cast<cudaStream_t>(pr->stream);
    else { SGS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own_stream = true; }
    if (pl.wide) SGS_CUDA(prepare_wide<T>(pl.M, pl.G));
    else if (pl.K == pl.G && pl.NC == 256 / pl.G) SGS_CUDA(prepare_sweep_keq<T>(pl.M, pl.G, pl.sweep_smem, pl.sweep_smem_diag));
    else SGS_CUDA(prepare_sweep<T>(pl.M, pl.G, pl.sweep_smem, pl.sweep_smem_diag));
    SGS_CUDA(prepare_fft<T>(pl.row, pl.col_smem));
    if (pl.zf_cs && zfused_max_clusters<T>(pl.zf_cs, pl.zf_threads, pl.zf_smem) < 1) pl.zf_cs = 0;
    if (pl.zs) {
      int dev = 0, nsm = 0, nb = 0;
      SGS_CUDA(cudaGetDevice(&dev));
      SGS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      ZseqArgs<T> none{};
      SGS_CUDA(launch_zseq<T>(none, 0, pl.zs_threads, pl.zs_smem, st, &nb));
      const long long most = std::max<long long>(std::max<long long>((long long)pl.nqblk * pl.H, pl.ncolblk), 1);
      pl.zs_grid = (int)std::min<long long>(most, (long long)nb * nsm);
      if (nb < 1) pl.zs = 0;
    }
    {
      // the prior's blocks walk the tiles: one wave of them, so that no SM runs a second
      // round of blocks after the others are done (never more than the planned partials)
      int dev = 0, nsm = 0, nb = 0;
      SGS_CUDA(cudaGetDevice(&dev));
      SGS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      SGS_CUDA(prior_blocks_per_sm<T>(pl.M, pl.G, &nb));
      if (nb >= 1) pl.nprior_blk = std::max(1, std::min(pl.nprior_blk, nb * nsm));
    }
    if (pl.rp) {
      // one wave of persistent CTAs; three launches of the one-unit kernels if none fits
      int dev = 0, nsm = 0, nbf = 0, nbi = 0;
      SGS_CUDA(cudaGetDevice(&dev));
      SGS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      SGS_CUDA(row_pipe_blocks_per_sm<T>(true, pl.rp_smem_f, &nbf));
      SGS_CUDA(row_pipe_blocks_per_sm<T>(false, pl.rp_smem_i, &nbi));
      const long long units = (long long)pl.nqblk * pl.H;
      pl.rp_grid_f = (int)std::min<long long>(units, (long long)nbf * nsm);
      pl.rp_grid_i = (int)std::min<long long>(units, (long long)nbi * nsm);
      if (nbf < 1 || nbi < 1) pl.rp = 0;
    }
    return upload_tables();
  }

  int upload_tables() {
    const int H = pl.H, W = pl.W, Wh = pl.Wh, Mf = pl.Mf;
    std::vector<T> om(pl.L);
    for (int j = 0; j < pl.L; ++j) om[j] = (T)omega[j];
    SGS_CUDA(cudaMemcpyAsync(b.omega, om.data(), sizeof(T) * pl.L, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemsetAsync(b.err, 0, sizeof(int), st));
    SGS_CUDA(cudaMemsetAsync(b.zctr, 0, 4 * sizeof(unsigned int), st));
    SGS_CUDA(cudaMemcpyAsync(b.covY, pl.covY.data(), sizeof(int) * pl.covY.size(), cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemcpyAsync(b.covX, pl.covX.data(), sizeof(int) * pl.covX.size(), cudaMemcpyHostToDevice, st));
    {
      std::vector<int> off(pl.covX.size());
      for (size_t i = 0; i < off.size(); ++i) {
        const int cx = pl.covX[i];
        off[i] = cx < 0 ? -1 : ((cx >> 16) * pl.EHmax * pl.EWmax + (cx & 0xffff)) * pl.K;
      }
      SGS_CUDA(cudaMemcpyAsync(b.offX, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, st));
      SGS_CUDA(cudaStreamSynchronize(st));  // `off` leaves scope
    }
    // column solve coefficients, per kx: (a + 2c) - c (S + S^-1) = (c/beta)(1 - beta S)(1 - beta/S)
    std::vector<T> beta(Wh), gain(Wh), wfac(Wh);
    std::vector<int> nwarm(Wh);
    const double tol = sizeof(T) == 4 ? 1e-9 : 1e-18;
    const double c = c_omega;
    for (int kx = 0; kx < Wh; ++kx) {
      const double s = std::sin(M_PI * kx / W);
      const double alpha = 3.0 + c * (4.0 * s * s + 2.0);
      if (c > 0.0) {
        const double t = alpha / c;
        const double bt = 2.0 / (t + std::sqrt(t * t - 4.0));
        const double gn = 2.0 / (alpha + std::sqrt(alpha * alpha - 4.0 * c * c));
        int nw = (int)std::ceil(std::log(tol * (1.0 - bt)) / std::log(bt));
        double wf = 1.0;
        if (nw >= H || nw < 0) { nw = H; wf = 1.0 / (1.0 - std::pow(bt, H)); }
        beta[kx] = (T)bt; gain[kx] = (T)gn; wfac[kx] = (T)wf; nwarm[kx] = nw;
      } else {
        beta[kx] = 0; gain[kx] = (T)(1.0 / alpha); wfac[kx] = 1; nwarm[kx] = 0;
      }
    }
    SGS_CUDA(cudaMemcpyAsync(b.beta, beta.data(), sizeof(T) * Wh, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemcpyAsync(b.gain, gain.data(), sizeof(T) * Wh, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemcpyAsync(b.wfac, wfac.data(), sizeof(T) * Wh, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemcpyAsync(b.nwarm, nwarm.data(), sizeof(int) * Wh, cudaMemcpyHostToDevice, st));
    // FFT tables (FP64 on the host)
    std::vector<cplx<T>> tw(Mf), chirp(W), bhat(Mf);
    for (int m = 0; m < Mf; ++m) {
      const double ang = -2.0 * M_PI * (double)m / Mf;
      tw[m] = mkc<T>((T)std::cos(ang), (T)std::sin(ang));
    }
    if (pl.blue) {
      std::vector<std::complex<double>> ch(W), bb(Mf, 0.0), twd(Mf);
      for (int m = 0; m < W; ++m) {
        const long long q = ((long long)m * m) % (2LL * W);
        const double ang = M_PI * (double)q / W;
        ch[m] = std::complex<double>(std::cos(ang), std::sin(ang));
        chirp[m] = mkc<T>((T)ch[m].real(), (T)ch[m].imag());
      }
      for (int m = 0; m < W; ++m) bb[m] = ch[m];
      for (int m = 1; m < W; ++m) bb[Mf - m] = ch[m];
      for (int m = 0; m < Mf; ++m) {
        const double ang = -2.0 * M_PI * (double)m / Mf;
        twd[m] = std::complex<double>(std::cos(ang), std::sin(ang));
      }
      for (int k = 0; k < Mf; ++k) {
        std::complex<double> acc = 0.0;
        for (int m = 0; m < Mf; ++m) acc += bb[m] * twd[((long long)k * m) % Mf];
        acc /= (double)Mf;
        bhat[k] = mkc<T>((T)acc.real(), (T)acc.imag());
      }
    } else {
      for (int m = 0; m < W; ++m) chirp[m] = mkc<T>(T(1), T(0));
      for (int m = 0; m < Mf; ++m) bhat[m] = mkc<T>(T(1), T(0));
    }
    SGS_CUDA(cudaMemcpyAsync(b.tw, tw.data(), sizeof(cplx<T>) * Mf, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemcpyAsync(b.chirp, chirp.data(), sizeof(cplx<T>) * W, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaMemcpyAsync(b.bhat, bhat.data(), sizeof(cplx<T>) * Mf, cudaMemcpyHostToDevice, st));
    SGS_CUDA(cudaStreamSynchronize(st));
    return SEGSALSA_OK;
  }

  // ---------------------------------------------------------------- launch bookkeeping
  cudaEvent_t get_event() {
    if (!evpool.empty()) { cudaEvent_t e = evpool.back(); evpool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  template <class F> cudaError_t launch(int kind, F&& f) {
    nlaunch[kind]++;
    if (!profiling) return f();
    cudaEvent_t a = get_event(), c = get_event();
    cudaEventRecord(a, st);
    cudaError_t e = f();
    cudaEventRecord(c, st);
    evs.emplace_back(kind, a, c);
    return e;
  }
#define SGS_LAUNCH(kind, expr) SGS_CUDA(launch(kind, [&]() -> cudaError_t { expr; return cudaGetLastError(); }))

  FftPlan<T> fft_plan() const {
    FftPlan<T> f{};
    make_fft_plan<T>(pl.W, f);
    f.tw = b.tw; f.chirp = b.chirp; f.bhat = b.bhat;
    return f;
  }
  RowArgs<T> row_args(const T* src, T* zout) const {
    RowArgs<T> a{};
    a.H = pl.H; a.W = pl.W; a.K = pl.K; a.Wh = pl.Wh; a.QB = pl.QB; a.smem_tables = pl.row.tables;
    a.lgB = 0;
    while ((1 << a.lgB) < pl.QB) ++a.lgB;
    a.mgB = div_magic(pl.QB);
    a.pl = fft_plan();
    a.src = src; a.P = b.P; a.ntx = pl.ntx; a.EHmax = pl.EHmax; a.EWmax = pl.EWmax;
    a.covY = b.covY; a.covX = b.covX; a.offX = b.offX; a.S = b.S; a.z = zout;
    a.nq = pl.nqblk; a.units = pl.nqblk * pl.H; a.nslot = pl.rp_nslot;
    return a;
  }

  // Bring the full form up to date (d1 = c1 p, d4 = c4 1) and make it the one in use.
  int dl_to_full() {
    if (!dl_cmp) return SEGSALSA_OK;
    const size_t nK = (size_t)pl.n * pl.K;
    const int blocks = (int)std::min<size_t>((nK + AUX_THREADS - 1) / AUX_THREADS, 152 * 8);
    SGS_LAUNCH(KIND_OTHER, (k_dl_expand<T><<<blocks, AUX_THREADS, 0, st>>>(b.dcmp, b.p, b.dloc, pl.n, pl.K)));
    dl_cmp = false;
    return SEGSALSA_OK;
  }

  // z = (3 I + J^T J)^{-1} rhs; rhs dense (src) or the sweep's rhs (src == nullptr: the tile
  // partials, or the dense rhs of the wide-patch sweep)
  int z_update(const T* src, T* zout) {
    if (!src && pl.wide) src = b.rhsd;
    const RowArgs<T> ra = row_args(src, zout);
    if (pl.zf_cs) {
      ZfArgs<T> za{};
      za.r = ra;
      za.r.smem_tables = 1;
      za.beta = b.beta; za.gain = b.gain; za.wfac = b.wfac; za.nwarm = b.nwarm;
      za.CS = pl.zf_cs; za.QG = pl.zf_qg; za.RMAX = pl.zf_rmax;
      za.mgB = div_magic(pl.zf_rmax * pl.zf_qg);
      SGS_CUDA(launch(KIND_ZF, [&]() { return launch_zfused<T>(za, pl.zf_groups, pl.zf_threads, pl.zf_smem, st); }));
      return SEGSALSA_OK;
    }
    ColArgs<T> ca{};
    ca.H = pl.H; ca.C = pl.Wh * pl.K; ca.K = pl.K; ca.CB = pl.CB; ca.NSEG = pl.NSEG; ca.SL = pl.SL;
    ca.beta = b.beta; ca.gain = b.gain; ca.wfac = b.wfac; ca.nwarm = b.nwarm; ca.S = b.S;
    if (pl.zs) {
      ZseqArgs<T> za{};
      za.f = ra; za.i = ra; za.c = ca;
      za.nqf = za.nqi = pl.nqblk;
      za.nf = za.ni = pl.nqblk * pl.H;
      za.nc = pl.ncolblk;
      za.ctr = b.zctr; za.err = b.err;
      za.budget = wait_budget;
      za.probe = wait_probe ? 1 : 0;
      SGS_CUDA(launch(KIND_ZF, [&]() { return launch_zseq<T>(za, pl.zs_grid, pl.zs_threads, pl.zs_smem, st); }));
      return SEGSALSA_OK;
    }
    const dim3 rg(pl.nqblk, pl.H);
    // the power-of-two kernels move a class block of a pixel as one vector: a caller's dense
    // rhs or z must be aligned to it
    const uintptr_t va = (uintptr_t)std::min<size_t>(16, 2 * pl.QB * sizeof(T)) - 1;
    const bool p2 = pl.p2 && ((reinterpret_cast<uintptr_t>(src) & va) == 0) &&
                    ((reinterpret_cast<uintptr_t>(zout) & va) == 0);
    if (p2)
      SGS_CUDA(launch(KIND_ROWF, [&]() { return launch_row_p2<T>(true, ra, rg, pl.p2_smem, st); }));
    else if (pl.rp)
      SGS_CUDA(launch(KIND_ROWF, [&]() { return launch_row_pipe<T>(true, ra, pl.rp_grid_f, pl.rp_smem_f, st); }));
    else
      SGS_CUDA(launch(KIND_ROWF, [&]() { return launch_row<T>(true, ra, rg, pl.row, st); }));
    SGS_CUDA(launch(KIND_COL, [&]() { return launch_col<T>(ca, pl.ncolblk, pl.col_threads, pl.col_smem, st); }));
    if (p2) {
      RowArgs<T> ri = ra;
      ri.QB = pl.QBi;
      ri.lgB = 0;
      while ((1 << ri.lgB) < pl.QBi) ++ri.lgB;
      ri.mgB = div_magic(pl.QBi);
      const dim3 rgi((pl.K / 2 + pl.QBi - 1) / pl.QBi, pl.H);
      SGS_CUDA(launch(KIND_ROWI, [&]() { return launch_row_p2<T>(false, ri, rgi, pl.p2_smem_i, st); }));
    }
    else if (pl.rp)
      SGS_CUDA(launch(KIND_ROWI, [&]() { return launch_row_pipe<T>(false, ra, pl.rp_grid_i, pl.rp_smem_i, st); }));
    else
      SGS_CUDA(launch(KIND_ROWI, [&]() { return launch_row<T>(false, ra, rg, pl.row, st); }));
    return SEGSALSA_OK;
  }

  int sweep(bool diag) {
    int rc;
    if (pl.wide) {
      if ((rc = dl_to_full())) return rc;     // the wide kernels keep the full form
      WideArgs<T> w{};
      w.H = pl.H; w.W = pl.W; w.K = pl.K; w.M = pl.M; w.L = pl.L;
      w.z = b.z; w.p = b.p; w.dloc = b.dloc; w.V = b.d2; w.coef = b.coef; w.scratch = b.wbuf;
      w.rhs = b.rhsd;
      w.gtd = b.P2; w.diag_sq = b.dsq; w.omega = b.omega;
      w.tau = (T)(lambda / mu); w.mu = (T)mu; w.invK = (T)(1.0 / pl.K); w.sp = sp;
      w.ntx1 = pl.wntx1; w.ntiles1 = pl.wntiles1; w.nblk2 = pl.wnblk2;
      // three kernels per sweep (gram, shifted sums, differences); counted as sweep launches
      nlaunch[KIND_SWEEP] += 2;
      SGS_CUDA(launch(KIND_SWEEP, [&]() {
        return launch_wide<T>(w, pl.G, diag, g4 == SEGSALSA_G4_SIMPLEX, st);
      }));
      return SEGSALSA_OK;
    }
    const bool simplex = g4 == SEGSALSA_G4_SIMPLEX;
    // the simplex sweep reads and writes the full form of the local duals; the affine sweep
    // reads either form and writes the compact one
    if (simplex && (rc = dl_to_full())) return rc;
    SweepArgs<T> a{};
    a.H = pl.H; a.W = pl.W; a.K = pl.K; a.NC = pl.NC; a.ntx = pl.ntx; a.nty = pl.nty;
    a.EHmax = pl.EHmax; a.EWmax = pl.EWmax;
    a.z = b.z; a.p = b.p; a.dloc = b.dloc; a.d2 = b.d2; a.P = b.P; a.P2 = b.P2;
    a.dcmp = b.dcmp;
    a.cin = (!simplex && dl_cmp) ? 1 : 0;
    a.diag_sq = b.dsq; a.omega = b.omega;
    a.tau = (T)(lambda / mu); a.mu = (T)mu; a.invK = (T)(1.0 / pl.K); a.sp = sp;
    a.err = b.err;
    a.budget = wait_budget;
    a.probe = wait_probe ? 16u : 0u;
    const size_t smem = diag ? pl.sweep_smem_diag : pl.sweep_smem;
    SGS_CUDA(launch(KIND_SWEEP, [&]() {
      if (simplex) return launch_sweep_simplex<T>(a, pl.M, pl.G, diag, pl.ntiles, smem, st);
      return pl.K == pl.G && pl.NC == 256 / pl.G ? launch_sweep_keq<T>(a, pl.M, pl.G, diag, pl.ntiles, smem, st)
                          : launch_sweep<T>(a, pl.M, pl.G, diag, pl.ntiles, smem, st);
    }));
    if (!simplex) dl_cmp = true;
    return SEGSALSA_OK;
  }

  int diagnostics(int k, int rec) {
    const int n = pl.n, K = pl.K;
    SGS_CUDA(launch(KIND_DIAG, [&]() { return launch_project_g<T>(pl.G, pl.nproj_blk, st, b.z, b.p, b.zp, n, K, (const T*)b.P2, pl.wide ? (const T*)b.P2 : nullptr, (const int*)b.covY, (const int*)b.offX, pl.W, pl.ntx, pl.EHmax, pl.EWmax, b.dproj); }));
    SGS_CUDA(launch(KIND_DIAG, [&]() { return launch_prior<T>(pl.M, pl.G, pl.nprior_blk, st, b.zp, b.omega, pl.H, pl.W, K, sp, b.dprior); }));
    SGS_CUDA(launch(KIND_DIAG, [&]() { return launch_pdl(k_finalize_trace, dim3(1), dim3(FT_THREADS), 0, st, (const double*)b.dsq, pl.wide ? pl.wntiles1 : pl.ntiles, (const double*)b.dproj, pl.nproj_blk, (const double*)b.dprior, pl.nprior_blk, (double)k, mu, lambda, b.dtrace + 6 * rec); }));
    return SEGSALSA_OK;
  }

  // ---------------------------------------------------------------------- API methods
  int copy_in(T* dst, const void* src, size_t count, int dev) {
    SGS_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return SEGSALSA_OK;
  }
  int copy_out(void* dst, const T* src, size_t count, int dev) {
    SGS_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return SEGSALSA_OK;
  }
  int grid1(size_t count) const { return (int)((count + AUX_THREADS - 1) / AUX_THREADS); }

  int set_probs(const void* p, int layout, int dev) override {
    if (!p) return fail(SEGSALSA_ERR_ARG, "p is NULL");
    if (layout != SEGSALSA_LAYOUT_KHW && layout != SEGSALSA_LAYOUT_HWK) return fail(SEGSALSA_ERR_ARG, "bad layout");
    const int n = pl.n, K = pl.K;
    const size_t nK = (size_t)n * K;
    int rc;
    if (layout == SEGSALSA_LAYOUT_HWK) {
      if ((rc = copy_in(b.tmp, p, nK, dev))) return rc;
    } else {
      if ((rc = copy_in(b.zp, p, nK, dev))) return rc;
      SGS_LAUNCH(KIND_OTHER, (k_khw_to_hwk<T><<<grid1(nK), AUX_THREADS, 0, st>>>(b.zp, b.tmp, n, K)));
    }
    return commit_probs();
  }

  // Validate the probabilities staged in b.tmp (pixel-major) and start a new solve from them.
  int commit_probs() {
    const int n = pl.n, K = pl.K;
    const size_t nK = (size_t)n * K;
    SGS_CUDA(cudaMemsetAsync(b.flag, 0, sizeof(int), st));
    SGS_LAUNCH(KIND_OTHER, (k_check_probs<T><<<grid1(n), AUX_THREADS, 0, st>>>(b.tmp, n, K, b.flag)));
    int flag = 0;
    SGS_CUDA(cudaMemcpyAsync(&flag, b.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGS_CUDA(cudaStreamSynchronize(st));
    if (flag & 1) return fail(SEGSALSA_ERR_ARG, "p has non-finite entries");
    if (flag & 2) return fail(SEGSALSA_ERR_ARG, "p has negative entries");
    if (flag & 4) return fail(SEGSALSA_ERR_ARG, "p has a pixel without a positive entry");
    SGS_CUDA(cudaMemcpyAsync(b.p, b.tmp, sizeof(T) * nK, cudaMemcpyDeviceToDevice, st));
    SGS_LAUNCH(KIND_OTHER, (k_init_z<T><<<grid1(n), AUX_THREADS, 0, st>>>(b.p, b.z, n, K)));
    SGS_CUDA(cudaMemsetAsync(b.dloc, 0, sizeof(T) * 3 * nK, st));
    dl_cmp = false;
    SGS_CUDA(cudaMemsetAsync(b.d2, 0, sizeof(T) * 2 * pl.L * nK, st));
    if (pl.wide) SGS_CUDA(cudaMemsetAsync(b.coef, 0, sizeof(T) * 4 * (size_t)n, st));  // V = 0: d2 = 0
    SGS_CUDA(cudaStreamSynchronize(st));
    iter = 0;
    rhs_dense = false;
    have_probs = true;
    return SEGSALSA_OK;
  }

  int set_spectra(const void* x, const void* w, const float* bias, int d, int dev) override {
    if (!x || !w) return fail(SEGSALSA_ERR_ARG, "x and w are required");
    if (d < 1 || d > MLR_MAXD) return fail(SEGSALSA_ERR_ARG, "d must be in [1, 256]");
    const size_t n = (size_t)pl.n, K = (size_t)pl.K;
    const size_t xb = n * d * 2, wb = K * d * 2, bb = K * sizeof(float);
    const uint16_t* xd = static_cast<const uint16_t*>(x);
    const uint16_t* wd = static_cast<const uint16_t*>(w);
    const float* bd = bias;
    // the kernel bulk-copies x and w from 16-byte aligned addresses: the weights always go
    // through the handle's staging buffer, x when it is host data or not so aligned
    const bool stage_x = !dev || (reinterpret_cast<uintptr_t>(x) & 15) != 0;
    const size_t need = align_up(xb, 256) + align_up(wb, 256) + bb;
    if (need > mlr_cap) {
      if (mlr_buf) cudaFree(mlr_buf);
      mlr_buf = nullptr;
      mlr_cap = 0;
      cudaError_t e = cudaMalloc(&mlr_buf, need);
      if (e != cudaSuccess) { mlr_buf = nullptr; return fail(SEGSALSA_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
      mlr_cap = need;
    }
    char* base = static_cast<char*>(mlr_buf);
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (stage_x) {
      SGS_CUDA(cudaMemcpyAsync(base, x, xb, kind, st));
      xd = reinterpret_cast<const uint16_t*>(base);
    }
    SGS_CUDA(cudaMemcpyAsync(base + align_up(xb, 256), w, wb, kind, st));
    wd = reinterpret_cast<const uint16_t*>(base + align_up(xb, 256));
    if (bias && !dev) {
      float* bdev = reinterpret_cast<float*>(base + align_up(xb, 256) + align_up(wb, 256));
      SGS_CUDA(cudaMemcpyAsync(bdev, bias, bb, kind, st));
      bd = bdev;
    }
    MlrArgs a{};
    a.x = xd; a.w = wd; a.bias = bd; a.p = b.tmp; a.err = b.err;
    a.n = pl.n; a.d = d; a.dpad = (d + 15) / 16 * 16; a.K = pl.K; a.npad = pl.K <= 16 ? 16 : 32;
    a.budget = wait_budget;
    a.probe = wait_probe ? 16u : 0u;
    SGS_CUDA(launch(KIND_MLR, [&]() { return launch_mlr<T>(a, st); }));
    int errflag = 0;
    SGS_CUDA(cudaMemcpyAsync(&errflag, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGS_CUDA(cudaStreamSynchronize(st));
    if (errflag) {
      cudaMemsetAsync(b.err, 0, sizeof(int), st);
      return fail(SEGSALSA_ERR_TIMEOUT, "the tensor-core wait gave up (bounded wait exceeded)");
    }
    return commit_probs();
  }

  int get_probs(void* p, int layout, int dev) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "no state: call set_probs first");
    if (!p) return fail(SEGSALSA_ERR_ARG, "p is NULL");
    if (layout != SEGSALSA_LAYOUT_KHW && layout != SEGSALSA_LAYOUT_HWK) return fail(SEGSALSA_ERR_ARG, "bad layout");
    const size_t nK = (size_t)pl.n * pl.K;
    int rc;
    if (layout == SEGSALSA_LAYOUT_HWK) {
      if ((rc = copy_out(p, b.p, nK, dev))) return rc;
    } else {
      SGS_LAUNCH(KIND_OTHER, (k_hwk_to_khw<T><<<grid1(nK), AUX_THREADS, 0, st>>>(b.p, b.tmp, pl.n, pl.K)));
      if ((rc = copy_out(p, b.tmp, nK, dev))) return rc;
    }
    SGS_CUDA(cudaStreamSynchronize(st));
    return SEGSALSA_OK;
  }

  // One iteration launched eagerly: z-update (skipped at k = 0), sweep, and when traced the
  // diagnostics writing trace slot `rec`.
  int iteration(bool traced, int rec) {
    int rc;
    if (iter > 0) {
      if ((rc = z_update(rhs_dense ? b.rhsd : nullptr, b.z))) return rc;
      rhs_dense = false;
    }
    if ((rc = sweep(traced))) return rc;
    if (traced && (rc = diagnostics(iter + 1, rec))) return rc;
    ++iter;
    return SEGSALSA_OK;
  }

  // Executable graph of `len` iterations (k >= 1), the last one traced into slot 0 if `traced`.
  int get_chunk(int len, bool traced, Chunk*& out) {
    auto key = std::make_pair(len, traced ? 1 : 0);
    auto it = chunks.find(key);
    if (it != chunks.end()) { out = &it->second; return SEGSALSA_OK; }
    Chunk c;
    int64_t before[NKIND];
    for (int i = 0; i < NKIND; ++i) before[i] = nlaunch[i];
    const int saved_iter = iter;
    SGS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = SEGSALSA_OK;
    for (int i = 0; i < len && !rc; ++i) {
      const bool tr = traced && i == len - 1;
      if ((rc = z_update(nullptr, b.z))) break;
      if ((rc = sweep(tr))) break;
      if (tr) rc = diagnostics(0, 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    iter = saved_iter;
    for (int i = 0; i < NKIND; ++i) {
      c.launches[i] = nlaunch[i] - before[i];
      nlaunch[i] = before[i];
    }
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(SEGSALSA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SEGSALSA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    out = &chunks.emplace(key, c).first->second;
    return SEGSALSA_OK;
  }

  int ensure_trace_host(int n) {
    if (n <= trace_host_cap) return SEGSALSA_OK;
    if (trace_host) cudaFreeHost(trace_host);
    trace_host = nullptr;
    trace_host_cap = 0;
    SGS_CUDA(cudaMallocHost(&trace_host, sizeof(double) * 6 * (size_t)n));
    trace_host_cap = n;
    return SEGSALSA_OK;
  }

  int solve(int iters, double* trace, int every, int* nrec) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "solve before set_probs");
    if (iters < 0) return fail(SEGSALSA_ERR_ARG, "iters must be >= 0");
    if (trace && every < 1) return fail(SEGSALSA_ERR_ARG, "trace_every must be >= 1");
    int rc;
    const int maxrec = trace ? iters / every + 2 : 0;
    if (trace && (rc = ensure_trace_host(maxrec))) return rc;
    int written = 0;
    std::vector<int> rec_k;
    rec_k.reserve(maxrec);
    const int untraced_chunk = 16;
    int it = 0;
    while (it < iters) {
      const int left = iters - it;
      // a whole traced period (or an untraced block) that ends before or at the last iteration
      // (graphs are captured with the local duals in their steady form: after set_probs,
      // set_state or a switch of g4 the first iteration runs eagerly)
      const bool can_graph = use_graphs && !profiling && iter >= 1 && !rhs_dense && dl_steady();
      int len = 0;
      if (can_graph) {
        if (trace) {
          if (iter % every == 0 && every <= left && every > 1) len = every;
        } else if (left >= untraced_chunk) {
          len = untraced_chunk;
        }
      }
      if (len > 0) {
        Chunk* c = nullptr;
        if ((rc = get_chunk(len, trace != nullptr, c))) return rc;
        SGS_CUDA(cudaGraphLaunch(c->exec, st));
        for (int i = 0; i < NKIND; ++i) nlaunch[i] += c->launches[i];
        iter += len;
        it += len;
        if (trace) {
          SGS_CUDA(cudaMemcpyAsync(trace_host + 6 * (size_t)written, b.dtrace, sizeof(double) * 6,
                                   cudaMemcpyDeviceToHost, st));
          rec_k.push_back(iter);
          ++written;
        }
        continue;
      }
      const bool tr = trace && (((iter + 1) % every) == 0 || it == iters - 1);
      if ((rc = iteration(tr, 0))) return rc;
      ++it;
      if (tr) {
        SGS_CUDA(cudaMemcpyAsync(trace_host + 6 * (size_t)written, b.dtrace, sizeof(double) * 6,
                                 cudaMemcpyDeviceToHost, st));
        rec_k.push_back(iter);
        ++written;
      }
    }
    int errflag = 0;
    SGS_CUDA(cudaMemcpyAsync(&errflag, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGS_CUDA(cudaStreamSynchronize(st));
    if (errflag) {
      cudaMemsetAsync(b.err, 0, sizeof(int), st);
      cudaMemsetAsync(b.zctr, 0, 4 * sizeof(unsigned int), st);
      return fail(SEGSALSA_ERR_TIMEOUT, "a device-side wait gave up (bounded wait exceeded)");
    }
    if (trace) {
      for (int r = 0; r < written; ++r) {
        for (int j = 0; j < 6; ++j) trace[6 * r + j] = trace_host[6 * r + j];
        trace[6 * r] = (double)rec_k[r];
      }
    }
    if (nrec) *nrec = written;
    if (trace)
      for (int i = 0; i < 6 * written; ++i)
        if (!std::isfinite(trace[i])) return fail(SEGSALSA_ERR_NUMERIC, "non-finite value in the iterates");
    return SEGSALSA_OK;
  }

  int get_labels(int32_t* lab, int dev) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "no state: call set_probs first");
    if (!lab) return fail(SEGSALSA_ERR_ARG, "labels is NULL");
    SGS_LAUNCH(KIND_OTHER, (k_labels<T><<<grid1(pl.n), AUX_THREADS, 0, st>>>(b.z, pl.n, pl.K, b.lab)));
    SGS_CUDA(cudaMemcpyAsync(lab, b.lab, sizeof(int32_t) * pl.n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    SGS_CUDA(cudaStreamSynchronize(st));
    return SEGSALSA_OK;
  }

  int get_z(void* z, int layout, int dev) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "no state: call set_probs first");
    if (!z) return fail(SEGSALSA_ERR_ARG, "z is NULL");
    if (layout != SEGSALSA_LAYOUT_KHW && layout != SEGSALSA_LAYOUT_HWK) return fail(SEGSALSA_ERR_ARG, "bad layout");
    const size_t nK = (size_t)pl.n * pl.K;
    int rc;
    if (layout == SEGSALSA_LAYOUT_HWK) {
      if ((rc = copy_out(z, b.z, nK, dev))) return rc;
    } else {
      SGS_LAUNCH(KIND_OTHER, (k_hwk_to_khw<T><<<grid1(nK), AUX_THREADS, 0, st>>>(b.z, b.tmp, pl.n, pl.K)));
      if ((rc = copy_out(z, b.tmp, nK, dev))) return rc;
    }
    SGS_CUDA(cudaStreamSynchronize(st));
    return SEGSALSA_OK;
  }

  int get_iteration(int* k) const override {
    if (!k) return SEGSALSA_ERR_ARG;
    *k = iter;
    return SEGSALSA_OK;
  }

  int get_state(void* z, void* d1, void* d2, void* d3, void* d4, void* rhs, int dev) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "no state: call set_probs first");
    const size_t nK = (size_t)pl.n * pl.K;
    int rc;
    if ((d1 || d3 || d4) && (rc = dl_to_full())) return rc;   // d1, d3, d4 from the full form
    if (z && (rc = copy_out(z, b.z, nK, dev))) return rc;
    if (d2 && pl.wide) {
      // the wide sweep stores d2 as (V, A): d2 = V (A - I)
      T* dst = dev ? reinterpret_cast<T*>(d2) : b.wbuf;
      SGS_CUDA(launch_wide_dual<T>(b.d2, b.coef, dst, pl.n, pl.L * pl.K, st));
      if (!dev && (rc = copy_out(d2, b.wbuf, 2 * pl.L * nK, 0))) return rc;
    } else if (d2 && (rc = copy_out(d2, b.d2, 2 * pl.L * nK, dev))) {
      return rc;
    }
    void* dl[3] = {d1, d3, d4};
    for (int j = 0; j < 3; ++j) {
      if (!dl[j]) continue;
      // dloc is [n][3][K]: gather plane j
      SGS_CUDA(cudaMemcpy2DAsync(b.tmp, sizeof(T) * pl.K, b.dloc + (size_t)j * pl.K, sizeof(T) * 3 * pl.K,
                                 sizeof(T) * pl.K, pl.n, cudaMemcpyDeviceToDevice, st));
      if ((rc = copy_out(dl[j], b.tmp, nK, dev))) return rc;
      SGS_CUDA(cudaStreamSynchronize(st));
    }
    if (rhs) {
      if (rhs_dense || pl.wide) {
        if ((rc = copy_out(rhs, b.rhsd, nK, dev))) return rc;
      } else {
        const RowArgs<T> ra = row_args(nullptr, b.tmp);
        SGS_LAUNCH(KIND_OTHER, (k_gather_dense<T><<<grid1(nK), AUX_THREADS, 0, st>>>(ra)));
        if ((rc = copy_out(rhs, b.tmp, nK, dev))) return rc;
      }
    }
    SGS_CUDA(cudaStreamSynchronize(st));
    return SEGSALSA_OK;
  }

  int set_state(const void* z, const void* d1, const void* d2, const void* d3, const void* d4,
                const void* rhs, int k, int dev) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "set_probs must come first (p is kept)");
    if (!z || !d1 || !d2 || !d3 || !d4) return fail(SEGSALSA_ERR_ARG, "z, d1..d4 are required");
    if (k < 0) return fail(SEGSALSA_ERR_ARG, "k must be >= 0");
    if (k > 0 && !rhs) return fail(SEGSALSA_ERR_ARG, "rhs is required when k > 0");
    const size_t nK = (size_t)pl.n * pl.K;
    int rc;
    if ((rc = copy_in(b.z, z, nK, dev))) return rc;
    if ((rc = copy_in(b.d2, d2, 2 * pl.L * nK, dev))) return rc;
    dl_cmp = false;                 // d1, d3, d4 arrive in full form
    if (pl.wide) SGS_CUDA(launch_wide_coef_identity<T>(b.coef, pl.n, st));  // V = d2, A = 2I
    const void* dl[3] = {d1, d3, d4};
    for (int j = 0; j < 3; ++j) {
      if ((rc = copy_in(b.tmp, dl[j], nK, dev))) return rc;
      SGS_CUDA(cudaMemcpy2DAsync(b.dloc + (size_t)j * pl.K, sizeof(T) * 3 * pl.K, b.tmp, sizeof(T) * pl.K,
                                 sizeof(T) * pl.K, pl.n, cudaMemcpyDeviceToDevice, st));
    }
    if (k > 0) {
      if ((rc = copy_in(b.rhsd, rhs, nK, dev))) return rc;
      rhs_dense = true;
    } else {
      rhs_dense = false;
    }
    SGS_CUDA(cudaStreamSynchronize(st));
    iter = k;
    return SEGSALSA_OK;
  }

  int linear_solve(const void* rhs, void* z, int dev) override {
    if (!rhs || !z) return fail(SEGSALSA_ERR_ARG, "rhs and z are required");
    const size_t nK = (size_t)pl.n * pl.K;
    int rc;
    const T* src = reinterpret_cast<const T*>(rhs);
    if (!dev) {
      if ((rc = copy_in(b.tmp, rhs, nK, 0))) return rc;
      src = b.tmp;
    }
    T* out = dev ? reinterpret_cast<T*>(z) : b.zp;
    if ((rc = z_update(src, out))) return rc;
    if (!dev && (rc = copy_out(z, b.zp, nK, 0))) return rc;
    if (pl.zs) {  // the one-launch form waits between its passes (bounded)
      int errflag = 0;
      SGS_CUDA(cudaMemcpyAsync(&errflag, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
      SGS_CUDA(cudaStreamSynchronize(st));
      if (errflag) {
        cudaMemsetAsync(b.err, 0, sizeof(int), st);
        cudaMemsetAsync(b.zctr, 0, 4 * sizeof(unsigned int), st);
        return fail(SEGSALSA_ERR_TIMEOUT, "a device-side wait gave up (bounded wait exceeded)");
      }
    }
    SGS_CUDA(cudaStreamSynchronize(st));
    return SEGSALSA_OK;
  }

  int set_profiling(int on) override {
    profiling = on != 0;
    return SEGSALSA_OK;
  }
  int kernel_stats(int64_t* launches, double* msout) override {
    if (!launches) return fail(SEGSALSA_ERR_ARG, "launches is NULL");
    SGS_CUDA(cudaStreamSynchronize(st));
    for (auto& e : evs) {
      float t = 0.f;
      SGS_CUDA(cudaEventElapsedTime(&t, std::get<1>(e), std::get<2>(e)));
      ms[std::get<0>(e)] += t;
      evpool.push_back(std::get<1>(e));
      evpool.push_back(std::get<2>(e));
    }
    evs.clear();
    for (int i = 0; i < NKIND; ++i) {
      launches[i] = nlaunch[i];
      if (msout) msout[i] = ms[i];
    }
    return SEGSALSA_OK;
  }
  int reset_stats() override {
    int64_t tmpl[NKIND];
    int rc = kernel_stats(tmpl, nullptr);
    if (rc) return rc;
    for (int i = 0; i < NKIND; ++i) { nlaunch[i] = 0; ms[i] = 0; }
    return SEGSALSA_OK;
  }
  segsalsa_str_tiling tiling() const override {
    segsalsa_str_tiling t;
    t.tile_rows = pl.THmax; t.row_pairs = pl.QB; t.col_block = pl.CB;
    t.row_threads = pl.row_threads; t.col_rows = pl.col_rows;
    t.zfuse = pl.zs ? 3 : pl.zf_cs ? pl.zf_cs : 1;
    t.row_pipe = pl.p2 ? 3 : pl.rp ? 2 : 1;
    return t;
  }

  // ------------------------------------------------------------------ batch support
  bool ready() const override { return have_probs; }
  bool graphable() const override { return have_probs && iter >= 1 && !rhs_dense && dl_steady(); }
  int enqueue_iterations(int len, cudaStream_t s) override {
    cudaStream_t keep = st;
    const bool keep_prof = profiling;
    int64_t before[NKIND];
    for (int i = 0; i < NKIND; ++i) before[i] = nlaunch[i];
    st = s;
    profiling = false;
    int rc = SEGSALSA_OK;
    for (int i = 0; i < len && !rc; ++i) {
      rc = z_update(nullptr, b.z);
      if (!rc) rc = sweep(false);
    }
    st = keep;
    profiling = keep_prof;
    for (int i = 0; i < NKIND; ++i) nlaunch[i] = before[i];
    return rc;
  }
  void advance(int len) override {
    iter += len;
    if (pl.zs || pl.zf_cs) {
      nlaunch[KIND_ZF] += len;
    } else {
      nlaunch[KIND_ROWF] += len; nlaunch[KIND_COL] += len; nlaunch[KIND_ROWI] += len;
    }
    nlaunch[KIND_SWEEP] += pl.wide ? 3 * len : len;
  }
  int enqueue_eager_iteration(cudaStream_t s) override {
    cudaStream_t keep = st;
    const bool keep_prof = profiling;
    st = s;
    profiling = false;
    const int rc = iteration(false, 0);
    st = keep;
    profiling = keep_prof;
    return rc;
  }
  int enqueue_read_err(int* host, cudaStream_t s) override {
    SGS_CUDA(cudaMemcpyAsync(host, b.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    return SEGSALSA_OK;
  }
  int clear_err(cudaStream_t s) override {
    SGS_CUDA(cudaMemsetAsync(b.err, 0, sizeof(int), s));
    SGS_CUDA(cudaMemsetAsync(b.zctr, 0, 4 * sizeof(unsigned int), s));
    return SEGSALSA_OK;
  }
  void invalidate() override { have_probs = false; iter = 0; rhs_dense = false; }
  int generation() const override { return gen; }
  int set_wait_budget(long long cycles, int probe) override {
    if (cycles < 1) return fail(SEGSALSA_ERR_ARG, "the wait budget must be at least one cycle");
    if (probe != 0 && probe != 1) return fail(SEGSALSA_ERR_ARG, "probe must be 0 or 1");
    SGS_CUDA(cudaStreamSynchronize(st));
    drop_chunks();                 // the graphs hold the old kernel arguments
    wait_budget = cycles;
    wait_probe = probe;
    return SEGSALSA_OK;
  }

  int set_g4(int mode) override {
    if (mode != SEGSALSA_G4_AFFINE && mode != SEGSALSA_G4_SIMPLEX) return fail(SEGSALSA_ERR_ARG, "bad g4 mode");
    if (mode == g4) return SEGSALSA_OK;
    if (mode == SEGSALSA_G4_SIMPLEX && !pl.wide)  // the wide kernels are prepared at create
      SGS_CUDA(prepare_sweep_simplex<T>(pl.M, pl.G, pl.sweep_smem, pl.sweep_smem_diag));
    SGS_CUDA(cudaStreamSynchronize(st));
    for (auto& kv : chunks)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    chunks.clear();
    g4 = mode;
    ++gen;
    return SEGSALSA_OK;
  }

  void drop_chunks() {
    for (auto& kv : chunks)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    chunks.clear();
    ++gen;
  }

  int set_log_probs(const void* logp, int layout, int dev) override {
    if (!logp) return fail(SEGSALSA_ERR_ARG, "log p is NULL");
    if (layout != SEGSALSA_LAYOUT_KHW && layout != SEGSALSA_LAYOUT_HWK) return fail(SEGSALSA_ERR_ARG, "bad layout");
    const size_t nK = (size_t)pl.n * pl.K;
    int rc;
    T* src = b.zp;
    if (layout == SEGSALSA_LAYOUT_HWK) {
      if ((rc = copy_in(b.zp, logp, nK, dev))) return rc;
    } else {
      if ((rc = copy_in(b.tmp, logp, nK, dev))) return rc;
      SGS_LAUNCH(KIND_OTHER, (k_khw_to_hwk<T><<<grid1(nK), AUX_THREADS, 0, st>>>(b.tmp, b.zp, pl.n, pl.K)));
    }
    const AdjShape sh{pl.H, pl.W, pl.K, pl.n};
    SGS_LAUNCH(KIND_OTHER, launch_exp_logp<T>(sh, pl.G, src, b.tmp, st));
    return commit_probs();
  }

  int set_lambda(double lam) override {
    if (!(lam >= 0.0) || !std::isfinite(lam)) return fail(SEGSALSA_ERR_ARG, "lambda must be finite and >= 0");
    SGS_CUDA(cudaStreamSynchronize(st));
    lambda = lam;
    drop_chunks();
    return SEGSALSA_OK;
  }

  int set_weights(const double* w) override {
    if (!w) return fail(SEGSALSA_ERR_ARG, "weights is NULL");
    for (int j = 0; j < pl.L; ++j)
      if (!std::isfinite(w[j])) return fail(SEGSALSA_ERR_ARG, "weights must be finite");
    SGS_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < pl.L; ++j) omega[j] = w[j];
    c_omega = 0.0;
    for (double v : omega) c_omega += v * v;
    drop_chunks();
    return upload_tables();
  }

  // Reverse pass of `iters` iterations from the current p (see adjoint.cuh for the algebra).
  int backward(int iters, const void* zbar, int layout, void* glogp, double* glam, double* gom,
               int every, int dev) override {
    if (!have_probs) return fail(SEGSALSA_ERR_STATE, "backward before set_probs");
    if (iters < 1) return fail(SEGSALSA_ERR_ARG, "iters must be >= 1");
    if (every < 1) return fail(SEGSALSA_ERR_ARG, "checkpoint_every must be >= 1");
    if (!zbar || !glogp) return fail(SEGSALSA_ERR_ARG, "zbar and grad_logp are required");
    if (layout != SEGSALSA_LAYOUT_KHW && layout != SEGSALSA_LAYOUT_HWK) return fail(SEGSALSA_ERR_ARG, "bad layout");
    if (pl.wide) return fail(SEGSALSA_ERR_ARG, "the reverse pass covers patches up to 5 x 5 (M <= 2)");
    const int K = pl.K, L = pl.L, n = pl.n;
    const size_t nK = (size_t)n * K, nloc = 3 * nK, n2 = 2 * (size_t)L * nK;
    const size_t tslot = (size_t)pl.ntiles * pl.EHmax * pl.EWmax * K;
    const size_t st_elems = nK + nloc + n2 + tslot;          // z, d1/d3/d4, d2, rhs partials
    const int nseg = (iters + every - 1) / every;
    const int blocks = (n + ADJ_THREADS / pl.G - 1) / (ADJ_THREADS / pl.G);
    const size_t npart = (size_t)blocks * (L + 2);
    // device memory of the pass (released at the end)
    Carver cv{nullptr};
    auto plan = [&](Carver& c, T*& ck, T*& fin, T*& zs, T*& dls, T*& d2s, T*& vbl, T*& vb2,
                    T*& zb, T*& bb, T*& glp, double*& part, double*& acc) {
      ck = c.take<T>((size_t)nseg * st_elems);
      fin = c.take<T>(st_elems);
      zs = c.take<T>((size_t)(every + 2) * nK);
      dls = c.take<T>((size_t)(every + 1) * nloc);
      d2s = c.take<T>((size_t)(every + 1) * n2);
      vbl = c.take<T>(2 * nloc);   // vbar local blocks, two buffers
      vb2 = c.take<T>(2 * n2);     // vbar d2 blocks, two buffers (pairs stay 2 T aligned)
      zb = c.take<T>(nK);
      bb = c.take<T>(nK);
      glp = c.take<T>(nK);
      part = c.take<double>(npart);
      acc = c.take<double>(L + 2);
    };
    T *ck, *fin, *zs, *dls, *d2s, *vbl, *vb2, *zb, *bb, *glp;
    double *part, *acc;
    plan(cv, ck, fin, zs, dls, d2s, vbl, vb2, zb, bb, glp, part, acc);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, cv.off);
    if (e != cudaSuccess) return fail(SEGSALSA_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    struct Free { void* m; ~Free() { cudaFree(m); } } guard{mem};
    Carver cm{static_cast<char*>(mem)};
    plan(cm, ck, fin, zs, dls, d2s, vbl, vb2, zb, bb, glp, part, acc);
    auto save = [&](T* dst) -> cudaError_t {
      cudaError_t r;
      if (dl_to_full()) return cudaErrorUnknown;   // checkpoints hold the full form
      if ((r = cudaMemcpyAsync(dst, b.z, sizeof(T) * nK, cudaMemcpyDeviceToDevice, st))) return r;
      if ((r = cudaMemcpyAsync(dst + nK, b.dloc, sizeof(T) * nloc, cudaMemcpyDeviceToDevice, st))) return r;
      if ((r = cudaMemcpyAsync(dst + nK + nloc, b.d2, sizeof(T) * n2, cudaMemcpyDeviceToDevice, st))) return r;
      return cudaMemcpyAsync(dst + nK + nloc + n2, b.P, sizeof(T) * tslot, cudaMemcpyDeviceToDevice, st);
    };
    auto load = [&](const T* src) -> cudaError_t {
      cudaError_t r;
      if ((r = cudaMemcpyAsync(b.z, src, sizeof(T) * nK, cudaMemcpyDeviceToDevice, st))) return r;
      if ((r = cudaMemcpyAsync(b.dloc, src + nK, sizeof(T) * nloc, cudaMemcpyDeviceToDevice, st))) return r;
      dl_cmp = false;
      if ((r = cudaMemcpyAsync(b.d2, src + nK + nloc, sizeof(T) * n2, cudaMemcpyDeviceToDevice, st))) return r;
      return cudaMemcpyAsync(b.P, src + nK + nloc + n2, sizeof(T) * tslot, cudaMemcpyDeviceToDevice, st);
    };
    int rc;
    // forward from z^0 = p / 1^T p, d^0 = 0, with a checkpoint every `every` iterations
    SGS_LAUNCH(KIND_OTHER, (k_init_z<T><<<grid1(n), AUX_THREADS, 0, st>>>(b.p, b.z, n, K)));
    SGS_CUDA(cudaMemsetAsync(b.dloc, 0, sizeof(T) * nloc, st));
    dl_cmp = false;
    SGS_CUDA(cudaMemsetAsync(b.d2, 0, sizeof(T) * n2, st));
    iter = 0;
    rhs_dense = false;
    for (int k = 0; k < iters; k += every) {
      SGS_CUDA(save(ck + (size_t)(k / every) * st_elems));
      if ((rc = solve(std::min(every, iters - k), nullptr, 0, nullptr))) return rc;
    }
    SGS_CUDA(save(fin));
    // seed: zbar^T, pixel-major
    if (layout == SEGSALSA_LAYOUT_HWK) {
      if ((rc = copy_in(zb, zbar, nK, dev))) return rc;
    } else {
      if ((rc = copy_in(b.tmp, zbar, nK, dev))) return rc;
      SGS_LAUNCH(KIND_OTHER, (k_khw_to_hwk<T><<<grid1(nK), AUX_THREADS, 0, st>>>(b.tmp, zb, n, K)));
    }
    SGS_CUDA(cudaMemsetAsync(glp, 0, sizeof(T) * nK, st));
    SGS_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (L + 2), st));
    const AdjShape sh{pl.H, pl.W, K, n};
    bool first = true;
    int cur = 0;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int k0 = seg * every;
      const int k1 = std::min(k0 + every, iters - 1);
      if (k1 < k0 + 1) continue;                              // no unit in this segment
      // recompute z^k, d^k (k0 <= k <= k1) and z^{k1+1} from the checkpoint
      SGS_CUDA(load(ck + (size_t)seg * st_elems));
      iter = k0;
      rhs_dense = false;
      for (int k = k0; k <= k1; ++k) {
        const int i = k - k0;
        SGS_CUDA(cudaMemcpyAsync(zs + (size_t)i * nK, b.z, sizeof(T) * nK, cudaMemcpyDeviceToDevice, st));
        if ((rc = dl_to_full())) return rc;           // the reverse units read the full form
        SGS_CUDA(cudaMemcpyAsync(dls + (size_t)i * nloc, b.dloc, sizeof(T) * nloc, cudaMemcpyDeviceToDevice, st));
        SGS_CUDA(cudaMemcpyAsync(d2s + (size_t)i * n2, b.d2, sizeof(T) * n2, cudaMemcpyDeviceToDevice, st));
        if (k < k1) {
          if ((rc = iteration(false, 0))) return rc;
        } else {
          if ((rc = z_update(nullptr, b.z))) return rc;         // z^{k1+1} (k1 >= 1)
          SGS_CUDA(cudaMemcpyAsync(zs + (size_t)(i + 1) * nK, b.z, sizeof(T) * nK, cudaMemcpyDeviceToDevice, st));
        }
      }
      // reverse units k1 .. k0+1
      for (int k = k1; k >= k0 + 1; --k) {
        const int i = k - k0;
        if ((rc = z_update(zb, bb))) return rc;                 // bbar = A^{-1} zbar^{k+1}
        AdjArgs<T> a{};
        a.s = sh;
        a.zk = zs + (size_t)i * nK;
        a.zk1 = zs + (size_t)(i + 1) * nK;
        a.p = b.p;
        a.dloc = dls + (size_t)(i - 1) * nloc;
        a.d2 = d2s + (size_t)(i - 1) * n2;
        a.bbar = bb;
        a.vn_loc = first ? nullptr : vbl + (size_t)(cur ^ 1) * nloc;
        a.vn_2 = first ? nullptr : vb2 + (size_t)(cur ^ 1) * n2;
        a.v_loc = vbl + (size_t)cur * nloc;
        a.v_2 = vb2 + (size_t)cur * n2;
        // the (h, v) pairs of the d2 layouts move as single 2 T accesses
        const uintptr_t pairs = reinterpret_cast<uintptr_t>(a.d2) | reinterpret_cast<uintptr_t>(a.v_2) |
                                reinterpret_cast<uintptr_t>(a.vn_2);
        if (pairs & (2 * sizeof(T) - 1)) return fail(SEGSALSA_ERR_CUDA, "reverse pass: unaligned d2 buffers");
        a.glogp = glp;
        a.part = part;
        a.omega = b.omega;
        a.tau = (T)(lambda / mu);
        a.mu = (T)mu;
        a.invK = (T)(1.0 / K);
        a.sp = sp;
        a.simplex = g4 == SEGSALSA_G4_SIMPLEX ? 1 : 0;
        SGS_LAUNCH(KIND_ADJ, launch_adj_vjp<T>(a, pl.M, pl.G, blocks, st));
        // the unit's block partials into the running FP64 sums; units run in the order
        // k = iters - 1 .. 1 whatever the checkpoint interval, so the sums are too
        SGS_LAUNCH(KIND_ADJ, launch_adj_sum(part, blocks, L + 2, acc, st));
        SGS_LAUNCH(KIND_ADJ, launch_adj_gt<T>(sh, pl.M, a.v_loc, a.v_2, b.omega, zb, st));
        first = false;
        cur ^= 1;
      }
    }
    // z^1 = z^0 = p / 1^T p: the rest of zbar flows into log p
    SGS_LAUNCH(KIND_ADJ, launch_adj_init<T>(sh, pl.G, b.p, zb, glp, st));
    if (layout == SEGSALSA_LAYOUT_HWK) {
      if ((rc = copy_out(glogp, glp, nK, dev))) return rc;
    } else {
      SGS_LAUNCH(KIND_OTHER, (k_hwk_to_khw<T><<<grid1(nK), AUX_THREADS, 0, st>>>(glp, b.tmp, n, K)));
      if ((rc = copy_out(glogp, b.tmp, nK, dev))) return rc;
    }
    // the handle ends where the forward pass ended: iteration `iters`
    SGS_CUDA(load(fin));
    iter = iters;
    rhs_dense = false;
    std::vector<double> sums(L + 2);   // tau, omega_0..omega_{L-1}, S
    SGS_CUDA(cudaMemcpyAsync(sums.data(), acc, sizeof(double) * (L + 2), cudaMemcpyDeviceToHost, st));
    SGS_CUDA(cudaStreamSynchronize(st));
    if (glam) *glam = sums[0] / mu;
    if (gom)
      for (int j = 0; j < L; ++j) gom[j] = sums[1 + j] - 2.0 * omega[j] * sums[L + 1];
    return SEGSALSA_OK;
  }

  int traffic(double* sw, double* it) const override {
    const double unit = (double)sizeof(T) * pl.n * pl.K;
    // per pixel and class: d2 read and written (4L values), z, p, rhs (3), d3 read and written
    // (2), and d1, d4 either per class (4 more: the simplex and wide sweeps) or as the two
    // per-pixel scalars of the compact form, read and written (4 per pixel: the affine sweep)
    const bool compact = !pl.wide && g4 != SEGSALSA_G4_SIMPLEX;
    const double s = compact ? unit * (4.0 * pl.L + 5.0) + 4.0 * sizeof(T) * pl.n
                             : unit * (4.0 * pl.L + 9.0);
    if (sw) *sw = s;
    if (it) *it = s + 2.0 * unit;
    return SEGSALSA_OK;
  }
};

static int create_any(const segsalsa_str_params* pr, void* ws, size_t wsb,
                      std::unique_ptr<SolverBase>& out, std::string& msg,
                      const segsalsa_str_tiling* tl = nullptr) {
  int rc = check_params(pr, msg);
  if (rc) return rc;
  if ((rc = check_tiling(tl, msg))) return rc;
  if (pr->precision == SEGSALSA_FP32) {
    auto s = std::make_unique<Solver<float>>();
    rc = s->init(pr, ws, wsb, tl);
    if (rc) { msg = s->err; return rc; }
    out = std::move(s);
  } else {
    auto s = std::make_unique<Solver<double>>();
    rc = s->init(pr, ws, wsb, tl);
    if (rc) { msg = s->err; return rc; }
    out = std::move(s);
  }
  return SEGSALSA_OK;
}

}  // namespace sgs

struct segsalsa_str {
  std::unique_ptr<sgs::SolverBase> impl;
};

// ------------------------------------------------------------------------------ batches
//
// A batch keeps one solver per image and a few "lanes" (streams). Images are assigned to lanes
// by longest-processing-time-first on a per-iteration cost (bytes moved plus a fixed launch
// term), so that the lanes carry about the same work. A chunk of `len` iterations of the whole
// batch is captured once into a CUDA graph: the master stream forks to every lane, each lane
// runs its images one after the other (all `len` iterations of an image in a row, so that a
// small image's working set stays in L2), and the lanes join back. The chains of different
// lanes run concurrently; replaying the graph costs one launch per chunk.
namespace sgs {

struct TuneKey {
  int precision, M, K, size_class;
  bool operator<(const TuneKey& o) const {
    return std::tie(precision, M, K, size_class) < std::tie(o.precision, o.M, o.K, o.size_class);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, segsalsa_str_tiling> g_tune_cache;
static thread_local std::string g_batch_error;

static int size_class_of(int H, int W) {
  const long long n = (long long)H * W;
  int l = 0;
  while ((2LL << l) <= n) ++l;  // l = floor(log2 n)
  return l / 2;
}
static TuneKey tune_key(const segsalsa_str_params& p) {
  return TuneKey{p.precision, p.M, p.K, size_class_of(p.H, p.W)};
}
static bool same_tiling(const segsalsa_str_tiling& a, const segsalsa_str_tiling& b) {
  return a.tile_rows == b.tile_rows && a.row_pairs == b.row_pairs && a.col_block == b.col_block &&
         a.row_threads == b.row_threads && a.col_rows == b.col_rows && a.zfuse == b.zfuse &&
         a.row_pipe == b.row_pipe;
}

constexpr int BATCH_CHUNK = 64;         // iterations per captured graph
constexpr int BATCH_DEFAULT_LANES = 16;

}  // namespace sgs

struct segsalsa_str_batch {
  std::string err;
  int n = 0;
  std::vector<segsalsa_str_params> params;
  std::vector<std::vector<double>> weights;  // the callers' weights, copied
  std::vector<std::unique_ptr<segsalsa_str>> img;
  std::vector<segsalsa_str_tiling> req;      // requested tiling of each image (0 = default)
  cudaStream_t ms = nullptr;
  bool own_ms = false;
  int nlanes = 0;
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  std::vector<std::vector<int>> lane_img;
  std::map<int, cudaGraphExec_t> graphs;     // by chunk length
  std::vector<int> graph_gen;                // image generations the graphs were captured at
  int* err_host = nullptr;                   // pinned, one flag per image

  int fail(int code, const std::string& m) { err = m; return code; }
#define SGB_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(SEGSALSA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

  ~segsalsa_str_batch() {
    if (ms) cudaStreamSynchronize(ms);
    drop_graphs();
    img.clear();
    for (auto e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (auto s : lanes) cudaStreamDestroy(s);
    if (err_host) cudaFreeHost(err_host);
    if (own_ms && ms) cudaStreamDestroy(ms);
  }

  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }

  // per-iteration cost used to balance the lanes: algorithmic bytes plus ~8 MB for the four
  // launches' fixed latency
  double cost(int i) const {
    const auto& p = params[i];
    const int L = (2 * p.M + 1) * (2 * p.M + 1);
    const double es = p.precision == SEGSALSA_FP32 ? 4.0 : 8.0;
    return es * (4.0 * L + 11.0) * (double)p.H * p.W * p.K + 8.0e6;
  }

  int make_image(int i, const segsalsa_str_tiling* t, std::unique_ptr<sgs::SolverBase>& out) {
    std::string msg;
    segsalsa_str_params pr = params[i];
    pr.weights = weights[i].empty() ? nullptr : weights[i].data();
    pr.stream = nullptr;
    const int rc = sgs::create_any(&pr, nullptr, 0, out, msg, t);
    if (rc) return fail(rc, "image " + std::to_string(i) + ": " + msg);
    return SEGSALSA_OK;
  }

  int init(int count, const segsalsa_str_params* pr, const segsalsa_str_tiling* tl, void* stream) {
    n = count;
    params.assign(pr, pr + n);
    weights.resize(n);
    req.resize(n);
    for (int i = 0; i < n; ++i) {
      std::string msg;
      if (int rc = sgs::check_params(&pr[i], msg)) return fail(rc, "image " + std::to_string(i) + ": " + msg);
      if (pr[i].stream) return fail(SEGSALSA_ERR_ARG, "image " + std::to_string(i) + ": params.stream must be NULL in a batch");
      if (tl)
        if (int rc = sgs::check_tiling(&tl[i], msg)) return fail(rc, "image " + std::to_string(i) + ": " + msg);
      const int L = (2 * pr[i].M + 1) * (2 * pr[i].M + 1);
      if (pr[i].weights) weights[i].assign(pr[i].weights, pr[i].weights + L);
      params[i].weights = nullptr;
      if (tl) {
        req[i] = tl[i];
      } else {
        std::lock_guard<std::mutex> g(sgs::g_tune_mu);
        auto it = sgs::g_tune_cache.find(sgs::tune_key(pr[i]));
        req[i] = it != sgs::g_tune_cache.end() ? it->second : segsalsa_str_tiling{0, 0, 0, 0, 0};
      }
    }
    for (int i = 0; i < n; ++i) {
      std::unique_ptr<sgs::SolverBase> s;
      if (int rc = make_image(i, &req[i], s)) return rc;
      img.emplace_back(new segsalsa_str);
      img.back()->impl = std::move(s);
    }
    if (stream) ms = reinterpret_cast<cudaStream_t>(stream);
    else { SGB_CUDA(cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking)); own_ms = true; }
    SGB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    SGB_CUDA(cudaMallocHost(&err_host, sizeof(int) * n));
    return set_lanes(std::min(n, sgs::BATCH_DEFAULT_LANES));
  }

  // Longest-processing-time-first assignment of the images to `want` lanes.
  int set_lanes(int want) {
    if (want < 1) return fail(SEGSALSA_ERR_ARG, "lanes must be >= 1");
    want = std::min(want, n);
    while ((int)lanes.size() < want) {
      cudaStream_t s;
      SGB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      lanes.push_back(s);
      cudaEvent_t e;
      SGB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      join.push_back(e);
    }
    nlanes = want;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    lane_img.assign(nlanes, {});
    std::vector<double> load(nlanes, 0.0);
    for (int i : order) {
      const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lane_img[j].push_back(i);
      load[j] += cost(i);
    }
    drop_graphs();
    return SEGSALSA_OK;
  }

  // Fork from the master stream to the lanes, run `body(lane, stream)`, join back.
  template <class F> int on_lanes(F&& body) {
    SGB_CUDA(cudaEventRecord(fork, ms));
    int rc = SEGSALSA_OK;
    for (int j = 0; j < nlanes; ++j) {
      SGB_CUDA(cudaStreamWaitEvent(lanes[j], fork, 0));
      if (!rc) rc = body(j, lanes[j]);
      SGB_CUDA(cudaEventRecord(join[j], lanes[j]));
      SGB_CUDA(cudaStreamWaitEvent(ms, join[j], 0));
    }
    return rc;
  }

  int image_fail(int i) {
    return fail(SEGSALSA_ERR_CUDA, "image " + std::to_string(i) + ": " + img[i]->impl->err);
  }

  int get_graph(int len, cudaGraphExec_t& out) {
    bool stale = (int)graph_gen.size() != n;
    for (int i = 0; i < n && !stale; ++i) stale = graph_gen[i] != img[i]->impl->generation();
    if (stale) {
      drop_graphs();
      graph_gen.resize(n);
      for (int i = 0; i < n; ++i) graph_gen[i] = img[i]->impl->generation();
    }
    auto it = graphs.find(len);
    if (it != graphs.end()) { out = it->second; return SEGSALSA_OK; }
    SGB_CUDA(cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal));
    int bad = -1;
    const int rc = on_lanes([&](int j, cudaStream_t s) {
      for (int i : lane_img[j])
        if (img[i]->impl->enqueue_iterations(len, s)) { bad = i; return SEGSALSA_ERR_CUDA; }
      return SEGSALSA_OK;
    });
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ms, &g);
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (bad >= 0) return image_fail(bad);
      if (rc) return rc;
      return fail(SEGSALSA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return fail(SEGSALSA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    graphs[len] = ex;
    out = ex;
    return SEGSALSA_OK;
  }

  int check_errs() {
    for (int i = 0; i < n; ++i)
      if (img[i]->impl->enqueue_read_err(err_host + i, ms)) return image_fail(i);
    SGB_CUDA(cudaStreamSynchronize(ms));
    int rc = SEGSALSA_OK;
    for (int i = 0; i < n; ++i)
      if (err_host[i]) {
        img[i]->impl->clear_err(ms);
        if (!rc) rc = fail(SEGSALSA_ERR_TIMEOUT, "image " + std::to_string(i) + ": a device-side wait gave up (bounded wait exceeded)");
      }
    cudaStreamSynchronize(ms);
    return rc;
  }

  // Enqueue `iters` iterations of every image on the master stream (no synchronization).
  int enqueue_solve(int iters) {
    if (iters <= 0) return SEGSALSA_OK;
    int left = iters;
    bool eager = false;
    for (int i = 0; i < n; ++i) eager = eager || !img[i]->impl->graphable();
    if (eager) {
      // one eager iteration of every image: afterwards all of them are at a plain iteration
      int bad = -1;
      const int rc = on_lanes([&](int j, cudaStream_t s) {
        for (int i : lane_img[j])
          if (img[i]->impl->enqueue_eager_iteration(s)) { bad = i; return SEGSALSA_ERR_CUDA; }
        return SEGSALSA_OK;
      });
      if (bad >= 0) return image_fail(bad);
      if (rc) return rc;
      --left;
    }
    while (left > 0) {
      const int len = std::min(left, sgs::BATCH_CHUNK);
      cudaGraphExec_t g;
      if (int rc = get_graph(len, g)) return rc;
      SGB_CUDA(cudaGraphLaunch(g, ms));
      for (int i = 0; i < n; ++i) img[i]->impl->advance(len);
      left -= len;
    }
    return SEGSALSA_OK;
  }

  int solve(int iters) {
    if (iters < 0) return fail(SEGSALSA_ERR_ARG, "iters must be >= 0");
    for (int i = 0; i < n; ++i)
      if (!img[i]->impl->ready()) return fail(SEGSALSA_ERR_STATE, "image " + std::to_string(i) + ": set_probs first");
    if (int rc = enqueue_solve(iters)) return rc;
    return check_errs();
  }

  // ------------------------------------------------------------------------ autotuner
  // Deterministic strictly positive probabilities for the timing runs (the cost of an
  // iteration does not depend on the values).
  int synthetic_probs(int i) {
    const auto& p = params[i];
    const size_t nK = (size_t)p.H * p.W * p.K;
    uint32_t x = 2463534242u + 977u * (uint32_t)i;
    auto next = [&]() { x ^= x << 13; x ^= x >> 17; x ^= x << 5; return 0.05 + (x >> 8) * (1.0 / 16777216.0); };
    int rc;
    if (p.precision == SEGSALSA_FP32) {
      std::vector<float> v(nK);
      for (auto& e : v) e = (float)next();
      rc = img[i]->impl->set_probs(v.data(), SEGSALSA_LAYOUT_HWK, 0);
    } else {
      std::vector<double> v(nK);
      for (auto& e : v) e = next();
      rc = img[i]->impl->set_probs(v.data(), SEGSALSA_LAYOUT_HWK, 0);
    }
    if (rc) return fail(rc, "image " + std::to_string(i) + ": " + img[i]->impl->err);
    return SEGSALSA_OK;
  }

  int rebuild(int i, const segsalsa_str_tiling& t) {
    std::unique_ptr<sgs::SolverBase> s;
    if (int rc = make_image(i, &t, s)) return rc;
    SGB_CUDA(cudaStreamSynchronize(ms));
    img[i]->impl = std::move(s);
    req[i] = t;
    drop_graphs();
    return synthetic_probs(i);
  }

  // Device time of `trial` batch iterations (best of two graph replays after a warm one).
  int time_batch(int trial, double& ms_out) {
    if (int rc = enqueue_solve(1)) return rc;  // brings every image to a plain iteration
    cudaGraphExec_t g;
    if (int rc = get_graph(trial, g)) return rc;
    cudaEvent_t a, c;
    SGB_CUDA(cudaEventCreate(&a));
    SGB_CUDA(cudaEventCreate(&c));
    double best = 1e300;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
      e = cudaEventRecord(a, ms);
      if (e == cudaSuccess) e = cudaGraphLaunch(g, ms);
      if (e == cudaSuccess) e = cudaEventRecord(c, ms);
      if (e == cudaSuccess) e = cudaEventSynchronize(c);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, c);
      if (e == cudaSuccess && r > 0) best = std::min(best, (double)t);
      for (int i = 0; i < n; ++i) img[i]->impl->advance(trial);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(c);
    if (e != cudaSuccess) return fail(SEGSALSA_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    if (int rc = check_errs()) return rc;
    ms_out = best;
    return SEGSALSA_OK;
  }

  int autotune(int trial, segsalsa_str_tiling* chosen) {
    if (trial < 1) return fail(SEGSALSA_ERR_ARG, "trial_iters must be >= 1");
    for (int i = 0; i < n; ++i)
      if (int rc = synthetic_probs(i)) return rc;
    double best;
    if (int rc = time_batch(trial, best)) return rc;
    // lanes first
    {
      std::set<int> cand = {4, 8, 16, 32, n};
      int keep = nlanes;
      for (int L : cand) {
        if (L > n || L == nlanes || L < 1) continue;
        const int prev = nlanes;
        if (int rc = set_lanes(L)) return rc;
        double t;
        if (int rc = time_batch(trial, t)) return rc;
        if (t < best * 0.98) { best = t; keep = L; }
        else if (int rc = set_lanes(prev)) return rc;
      }
      if (nlanes != keep)
        if (int rc = set_lanes(keep)) return rc;
    }
    // then the tiling of each class, largest total work first
    std::map<sgs::TuneKey, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) groups[sgs::tune_key(params[i])].push_back(i);
    std::vector<std::pair<double, sgs::TuneKey>> order;
    for (auto& kv : groups) {
      double w = 0;
      for (int i : kv.second) w += cost(i);
      order.push_back({-w, kv.first});
    }
    std::sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    const int cand_rows[] = {4, 6, 8, 12, 16, 24, 32};
    const int cand_pairs[] = {1, 2, 4, 8, 16};
    const int cand_cols[] = {1, 2, 4, 8};
    const int cand_rthr[] = {128, 256, 512, 1024};
    const int cand_seg[] = {8, 16, 32};
    const int cand_pipe[] = {1, 2, 3};
    for (auto& o : order) {
      const std::vector<int>& mem = groups[o.second];
      segsalsa_str_tiling cur = req[mem[0]];
      // resolved tilings already timed for this class
      std::set<std::vector<int>> seen;
      auto resolved = [&](const segsalsa_str_tiling& t, std::vector<int>& key) {
        key.clear();
        for (int i : mem) {
          segsalsa_str_params pr = params[i];
          pr.weights = weights[i].empty() ? nullptr : weights[i].data();
          sgs::Plan pl;
          std::string msg;
          const int rc = pr.precision == SEGSALSA_FP32 ? sgs::make_plan<float>(&pr, pl, msg, &t)
                                                       : sgs::make_plan<double>(&pr, pl, msg, &t);
          if (rc) return false;
          key.push_back(pl.THmax); key.push_back(pl.QB); key.push_back(pl.CB);
          key.push_back(pl.row.threads); key.push_back(pl.NSEG); key.push_back(pl.zf_cs);
          key.push_back(pl.rp);
          key.push_back(pl.p2);
        }
        return true;
      };
      std::vector<int> key;
      if (resolved(cur, key)) seen.insert(key);
      for (int f = 0; f < 6; ++f) {
        const int* cvs[6] = {cand_rows, cand_pairs, cand_cols, cand_rthr, cand_seg, cand_pipe};
        const int ncs[6] = {7, 5, 4, 4, 3, 3};
        const int* cv = cvs[f];
        const int nc = ncs[f];
        segsalsa_str_tiling keep = cur;
        for (int c = 0; c < nc; ++c) {
          segsalsa_str_tiling t = cur;
          int* fld[6] = {&t.tile_rows, &t.row_pairs, &t.col_block, &t.row_threads, &t.col_rows,
                         &t.row_pipe};
          *fld[f] = cv[c];
          if (!resolved(t, key) || seen.count(key)) continue;
          seen.insert(key);
          bool ok = true;
          for (int i : mem) {
            const int rc = rebuild(i, t);
            if (rc == SEGSALSA_ERR_ARG) { ok = false; break; }
            if (rc) return rc;
          }
          double tm = 1e300;
          if (ok)
            if (int rc = time_batch(trial, tm)) return rc;
          if (ok && tm < best * 0.98) { best = tm; keep = t; }
        }
        cur = keep;
        for (int i : mem)
          if (!sgs::same_tiling(req[i], cur))
            if (int rc = rebuild(i, cur)) return rc;
      }
      std::lock_guard<std::mutex> g(sgs::g_tune_mu);
      sgs::g_tune_cache[o.second] = cur;
    }
    for (int i = 0; i < n; ++i) {
      img[i]->impl->invalidate();
      if (chosen) chosen[i] = img[i]->impl->tiling();
    }
    drop_graphs();
    SGB_CUDA(cudaStreamSynchronize(ms));
    return SEGSALSA_OK;
  }
#undef SGB_CUDA
};

extern "C" {

int segsalsa_str_workspace_bytes_tiled(const segsalsa_str_params* pr, const segsalsa_str_tiling* tl,
                                       size_t* bytes) {
  std::string msg;
  int rc = sgs::check_params(pr, msg);
  if (!rc && !bytes) { rc = SEGSALSA_ERR_ARG; msg = "bytes is NULL"; }
  if (!rc) {
    sgs::Plan pl;
    if (pr->precision == SEGSALSA_FP32) {
      rc = sgs::make_plan<float>(pr, pl, msg, tl);
      sgs::Buffers<float> b{};
      if (!rc) *bytes = sgs::carve<float>(pl, nullptr, b);
    } else {
      rc = sgs::make_plan<double>(pr, pl, msg, tl);
      sgs::Buffers<double> b{};
      if (!rc) *bytes = sgs::carve<double>(pl, nullptr, b);
    }
  }
  if (rc) sgs::g_last_error = msg;
  return rc;
}

int segsalsa_str_workspace_bytes(const segsalsa_str_params* pr, size_t* bytes) {
  return segsalsa_str_workspace_bytes_tiled(pr, nullptr, bytes);
}

int segsalsa_str_create_tiled(const segsalsa_str_params* pr, const segsalsa_str_tiling* tl, void* ws,
                              size_t wsb, segsalsa_str_t** out) {
  if (!out) { sgs::g_last_error = "out is NULL"; return SEGSALSA_ERR_ARG; }
  *out = nullptr;
  std::unique_ptr<sgs::SolverBase> impl;
  std::string msg;
  int rc = sgs::create_any(pr, ws, wsb, impl, msg, tl);
  if (rc) { sgs::g_last_error = msg; return rc; }
  auto* h = new segsalsa_str;
  h->impl = std::move(impl);
  *out = h;
  return SEGSALSA_OK;
}

int segsalsa_str_create(const segsalsa_str_params* pr, void* ws, size_t wsb, segsalsa_str_t** out) {
  return segsalsa_str_create_tiled(pr, nullptr, ws, wsb, out);
}

int segsalsa_str_get_tiling(const segsalsa_str_t* h, segsalsa_str_tiling* t) {
  if (!h || !t) return SEGSALSA_ERR_ARG;
  *t = h->impl->tiling();
  return SEGSALSA_OK;
}

#define SGS_H(h) if (!(h)) return SEGSALSA_ERR_ARG

int segsalsa_str_set_probs(segsalsa_str_t* h, const void* p, int32_t layout, int32_t dev) {
  SGS_H(h); return h->impl->set_probs(p, layout, dev);
}
int segsalsa_str_solve(segsalsa_str_t* h, int32_t iters, double* trace, int32_t every, int32_t* nrec) {
  SGS_H(h); return h->impl->solve(iters, trace, every, nrec);
}
int segsalsa_str_solve_until(segsalsa_str_t* h, int32_t max_iters, double tol_primal,
                             double tol_dual, int32_t check_every, int32_t* iters_done,
                             double* last_record) {
  SGS_H(h);
  sgs::SolverBase& s = *h->impl;
  if (max_iters < 0) return s.fail(SEGSALSA_ERR_ARG, "max_iters must be >= 0");
  if (check_every < 1) return s.fail(SEGSALSA_ERR_ARG, "check_every must be >= 1");
  if (!(tol_primal >= 0.0) || !(tol_dual >= 0.0) || !std::isfinite(tol_primal) ||
      !std::isfinite(tol_dual))
    return s.fail(SEGSALSA_ERR_ARG, "tolerances must be finite and >= 0");
  int done = 0;
  double rec[12] = {0};
  double last[6] = {0};
  bool have = false;
  while (done < max_iters) {
    const int len = std::min(check_every, max_iters - done);
    int n = 0;
    const int rc = s.solve(len, rec, len, &n);
    if (rc) return rc;
    done += len;
    if (n > 0) {
      for (int j = 0; j < 6; ++j) last[j] = rec[6 * (n - 1) + j];
      have = true;
      if (last[1] <= tol_primal && last[2] <= tol_dual) break;
    }
  }
  if (iters_done) *iters_done = done;
  if (last_record)
    for (int j = 0; j < 6; ++j) last_record[j] = have ? last[j] : std::nan("");
  return SEGSALSA_OK;
}
int segsalsa_str_get_labels(segsalsa_str_t* h, int32_t* lab, int32_t dev) {
  SGS_H(h); return h->impl->get_labels(lab, dev);
}
int segsalsa_str_get_z(segsalsa_str_t* h, void* z, int32_t layout, int32_t dev) {
  SGS_H(h); return h->impl->get_z(z, layout, dev);
}
int segsalsa_str_get_iteration(const segsalsa_str_t* h, int32_t* k) {
  SGS_H(h); return h->impl->get_iteration(k);
}
int segsalsa_str_get_state(segsalsa_str_t* h, void* z, void* d1, void* d2, void* d3, void* d4,
                           void* rhs, int32_t dev) {
  SGS_H(h); return h->impl->get_state(z, d1, d2, d3, d4, rhs, dev);
}
int segsalsa_str_set_state(segsalsa_str_t* h, const void* z, const void* d1, const void* d2,
                           const void* d3, const void* d4, const void* rhs, int32_t k, int32_t dev) {
  SGS_H(h); return h->impl->set_state(z, d1, d2, d3, d4, rhs, k, dev);
}
int segsalsa_str_linear_solve(segsalsa_str_t* h, const void* rhs, void* z, int32_t dev) {
  SGS_H(h); return h->impl->linear_solve(rhs, z, dev);
}
int segsalsa_str_set_spectra(segsalsa_str_t* h, const void* x, const void* w, const float* bias,
                             int32_t d, int32_t dev) {
  SGS_H(h); return h->impl->set_spectra(x, w, bias, d, dev);
}
int segsalsa_str_get_probs(segsalsa_str_t* h, void* p, int32_t layout, int32_t dev) {
  SGS_H(h); return h->impl->get_probs(p, layout, dev);
}
int segsalsa_str_set_wait_budget(segsalsa_str_t* h, int64_t cycles, int32_t probe) {
  SGS_H(h); return h->impl->set_wait_budget((long long)cycles, probe);
}
int segsalsa_str_set_g4(segsalsa_str_t* h, int32_t mode) {
  SGS_H(h); return h->impl->set_g4(mode);
}
int segsalsa_str_set_log_probs(segsalsa_str_t* h, const void* logp, int32_t layout, int32_t dev) {
  SGS_H(h); return h->impl->set_log_probs(logp, layout, dev);
}
int segsalsa_str_set_lambda(segsalsa_str_t* h, double lambda) {
  SGS_H(h); return h->impl->set_lambda(lambda);
}
int segsalsa_str_set_weights(segsalsa_str_t* h, const double* weights) {
  SGS_H(h); return h->impl->set_weights(weights);
}
int segsalsa_str_backward(segsalsa_str_t* h, int32_t iters, const void* zbar, int32_t layout,
                          void* grad_logp, double* grad_lambda, double* grad_weights,
                          int32_t checkpoint_every, int32_t dev) {
  SGS_H(h);
  return h->impl->backward(iters, zbar, layout, grad_logp, grad_lambda, grad_weights,
                           checkpoint_every, dev);
}
int segsalsa_str_set_profiling(segsalsa_str_t* h, int32_t on) {
  SGS_H(h); return h->impl->set_profiling(on);
}
int segsalsa_str_kernel_stats(segsalsa_str_t* h, int64_t* launches, double* ms) {
  SGS_H(h); return h->impl->kernel_stats(launches, ms);
}
int segsalsa_str_reset_stats(segsalsa_str_t* h) {
  SGS_H(h); return h->impl->reset_stats();
}
int segsalsa_str_traffic_model(const segsalsa_str_t* h, double* sw, double* it) {
  SGS_H(h); return h->impl->traffic(sw, it);
}
void segsalsa_str_destroy(segsalsa_str_t* h) { delete h; }

int segsalsa_str_batch_create(int32_t n, const segsalsa_str_params* params,
                              const segsalsa_str_tiling* tiling, void* stream,
                              segsalsa_str_batch_t** out) {
  if (!out) { sgs::g_batch_error = "out is NULL"; return SEGSALSA_ERR_ARG; }
  *out = nullptr;
  if (n < 1 || !params) { sgs::g_batch_error = "n_images must be >= 1 and params non-NULL"; return SEGSALSA_ERR_ARG; }
  auto b = std::make_unique<segsalsa_str_batch>();
  const int rc = b->init(n, params, tiling, stream);
  if (rc) { sgs::g_batch_error = b->err; return rc; }
  *out = b.release();
  return SEGSALSA_OK;
}
int segsalsa_str_batch_image(segsalsa_str_batch_t* b, int32_t i, segsalsa_str_t** h) {
  if (!b) return SEGSALSA_ERR_ARG;
  if (!h || i < 0 || i >= b->n) return b->fail(SEGSALSA_ERR_ARG, "image index out of range or h NULL");
  *h = b->img[i].get();
  return SEGSALSA_OK;
}
int segsalsa_str_batch_solve(segsalsa_str_batch_t* b, int32_t iters) {
  if (!b) return SEGSALSA_ERR_ARG;
  return b->solve(iters);
}
int segsalsa_str_batch_autotune(segsalsa_str_batch_t* b, int32_t trial_iters, segsalsa_str_tiling* chosen) {
  if (!b) return SEGSALSA_ERR_ARG;
  return b->autotune(trial_iters, chosen);
}
int segsalsa_str_batch_set_lanes(segsalsa_str_batch_t* b, int32_t lanes) {
  if (!b) return SEGSALSA_ERR_ARG;
  return b->set_lanes(lanes);
}
int segsalsa_str_batch_get_lanes(const segsalsa_str_batch_t* b, int32_t* lanes) {
  if (!b || !lanes) return SEGSALSA_ERR_ARG;
  *lanes = b->nlanes;
  return SEGSALSA_OK;
}
void segsalsa_str_batch_destroy(segsalsa_str_batch_t* b) { delete b; }
const char* segsalsa_str_batch_last_error(const segsalsa_str_batch_t* b) {
  if (!b) return sgs::g_batch_error.c_str();
  return b->err.c_str();
}
const char* segsalsa_str_last_error(const segsalsa_str_t* h) {
  if (!h) return sgs::g_last_error.c_str();
  return h->impl->err.c_str();
}

}  // extern "C"
