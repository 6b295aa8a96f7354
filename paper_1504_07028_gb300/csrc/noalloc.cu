// Allocation-free z-update: segsalsa_str_linear_solve_static.
//
// Who needs this: code that runs where device allocation is not allowed or not possible --
// inside a region that must not call cudaMalloc (it synchronises the device and can fail
// under a fixed memory budget), under an external allocator that owns all device memory, or
// from a plug-in that has no handle and cannot keep one. Such callers pass their own rhs and
// z buffers; the scratch this operation needs (the row spectrum and the transform tables)
// lives in one file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
//
// The kernels are the library's own row-DFT and column-solve passes; only the memory they
// work in differs. Host code never dereferences g_static_scratch: the array's name on the
// host is a stand-in, not a device address, so its device address is looked up with
// cudaGetSymbolAddress on every call (with the caller's device current; the lookup allocates
// nothing). The transform tables kept in the array are rebuilt whenever the geometry, the
// device address or the CUDA context changes (a device reset reloads the module with the
// array zeroed).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/segsalsa_str.h"
#include "fft.cuh"

namespace sgs {
namespace {

constexpr size_t kSpecMaxComplex = size_t(2) << 20;                 // 2 Mi complex = 16 MiB
constexpr size_t kSpecBytes = kSpecMaxComplex * sizeof(float2);
constexpr size_t kTableBytes = size_t(512) << 10;                   // 512 KiB of tables
constexpr int kMaxDev = kMaxDevices;

static __device__ __align__(256) unsigned char g_static_scratch[kSpecBytes + kTableBytes];

struct DevCache {
  unsigned char* base = nullptr;  // device address of g_static_scratch on this device
  unsigned long long ctx = 0;     // context the tables were built in
  int H = -1, W = -1;             // geometry whose tables are in the array
  double c = -1.0;
};
static DevCache g_cache[kMaxDev];
static std::mutex g_cache_mu;     // host-side bookkeeping only; GPU-side overlap still races

// Table region layout (offsets in bytes from the table base, 256-aligned pieces).
struct TableLayout {
  size_t tw, chirp, bhat, beta, gain, wfac, nwarm, twd, end;
};
__host__ __device__ inline size_t al256(size_t v) { return (v + 255) / 256 * 256; }
__host__ __device__ inline TableLayout table_layout(int W, int Mf, int Wh) {
  TableLayout t{};
  size_t o = 0;
  t.tw = o;    o = al256(o + sizeof(float2) * Mf);
  t.chirp = o; o = al256(o + sizeof(float2) * W);
  t.bhat = o;  o = al256(o + sizeof(float2) * Mf);
  t.beta = o;  o = al256(o + sizeof(float) * Wh);
  t.gain = o;  o = al256(o + sizeof(float) * Wh);
  t.wfac = o;  o = al256(o + sizeof(float) * Wh);
  t.nwarm = o; o = al256(o + sizeof(int) * Wh);
  t.twd = o;   o = al256(o + sizeof(double2) * Mf);
  t.end = o;
  return t;
}

// Twiddles (FP64 and FP32), chirp and column coefficients, one thread per index.
__global__ void k_static_tables(unsigned char* tb, int H, int W, int Mf, int Wh, int blue,
                                double c) {
  const TableLayout L = table_layout(W, Mf, Wh);
  float2* tw = reinterpret_cast<float2*>(tb + L.tw);
  double2* twd = reinterpret_cast<double2*>(tb + L.twd);
  float2* chirp = reinterpret_cast<float2*>(tb + L.chirp);
  float* beta = reinterpret_cast<float*>(tb + L.beta);
  float* gain = reinterpret_cast<float*>(tb + L.gain);
  float* wfac = reinterpret_cast<float*>(tb + L.wfac);
  int* nwarm = reinterpret_cast<int*>(tb + L.nwarm);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Mf) {
    double s, co;
    sincospi(-2.0 * (double)i / Mf, &s, &co);
    twd[i] = make_double2(co, s);
    tw[i] = make_float2((float)co, (float)s);
  }
  if (i < W) {
    double s = 0.0, co = 1.0;
    if (blue) sincospi((double)(((long long)i * i) % (2LL * W)) / W, &s, &co);
    chirp[i] = make_float2((float)co, (float)s);
  }
  if (i < Wh) {
    const double sn = sinpi((double)i / W);
    const double alpha = 3.0 + c * (4.0 * sn * sn + 2.0);
    if (c > 0.0) {
      const double t = alpha / c;
      const double bt = 2.0 / (t + sqrt(t * t - 4.0));
      int nw = (int)ceil(log(1e-9 * (1.0 - bt)) / log(bt));
      double wf = 1.0;
      if (nw >= H || nw < 0) { nw = H; wf = 1.0 / (1.0 - pow(bt, (double)H)); }
      beta[i] = (float)bt;
      gain[i] = (float)(2.0 / (alpha + sqrt(alpha * alpha - 4.0 * c * c)));
      wfac[i] = (float)wf;
      nwarm[i] = nw;
    } else {
      beta[i] = 0.f; gain[i] = (float)(1.0 / alpha); wfac[i] = 1.f; nwarm[i] = 0;
    }
  }
}

// Bluestein filter spectrum bhat = DFT(b) / Mf in FP64 (needs the FP64 twiddles).
__global__ void k_static_bhat(unsigned char* tb, int W, int Mf, int Wh, int blue) {
  const TableLayout L = table_layout(W, Mf, Wh);
  const double2* twd = reinterpret_cast<const double2*>(tb + L.twd);
  float2* bhat = reinterpret_cast<float2*>(tb + L.bhat);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Mf) return;
  if (!blue) { bhat[k] = make_float2(1.f, 0.f); return; }
  double ar = 0.0, ai = 0.0;
  for (int m = 0; m < Mf; ++m) {
    int src = -1;  // b[m] = chirp[m] (m < W), b[Mf - m] = chirp[m] (1 <= m < W)
    if (m < W) src = m;
    else if (Mf - m < W) src = Mf - m;
    if (src < 0) continue;
    double s, co;
    sincospi((double)(((long long)src * src) % (2LL * W)) / W, &s, &co);
    const double2 w = twd[(int)(((long long)k * m) % Mf)];
    ar += co * w.x - s * w.y;
    ai += co * w.y + s * w.x;
  }
  bhat[k] = make_float2((float)(ar / Mf), (float)(ai / Mf));
}

}  // namespace
}  // namespace sgs

extern "C" int segsalsa_str_linear_solve_static(const float* rhs, float* z, int32_t H, int32_t W,
                                                int32_t K, double c_omega, void* stream) {
  using namespace sgs;
  if (!rhs || !z || H < 2 || W < 2 || K < 1 || K > 32 || !(c_omega >= 0.0) ||
      !std::isfinite(c_omega))
    return SEGSALSA_ERR_ARG;
  if (W > 8192) return SEGSALSA_ERR_OOM;
  const int Wh = W / 2 + 1;
  FftPlan<float> pl{};
  if (!make_fft_plan<float>(W, pl) || pl.Mf > 8192) return SEGSALSA_ERR_OOM;
  const int Mf = pl.Mf, blue = pl.blue;
  if ((size_t)H * Wh * K > kSpecMaxComplex) return SEGSALSA_ERR_OOM;
  if (table_layout(W, Mf, Wh).end > kTableBytes) return SEGSALSA_ERR_OOM;
  const int CB = 8;
  const size_t col_smem = (size_t)H * CB * sizeof(float2);
  if (col_smem > 200 * 1024) return SEGSALSA_ERR_OOM;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return SEGSALSA_ERR_CUDA;
  // the device address of the array in the current context (this also creates the context
  // on first use), then the context's identity
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_static_scratch) != cudaSuccess || !sym) return SEGSALSA_ERR_CUDA;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lk(g_cache_mu);
  DevCache& dc = g_cache[dev];
  if (dc.base != sym || dc.ctx != ctx || ctx == 0) {
    dc.base = reinterpret_cast<unsigned char*>(sym);
    dc.ctx = ctx;
    dc.H = dc.W = -1;  // tables unknown: rebuild
  }
  unsigned char* spec = dc.base;
  unsigned char* tb = dc.base + kSpecBytes;
  const TableLayout TL = table_layout(W, Mf, Wh);
  bool rebuilt = false;
  if (dc.H != H || dc.W != W || dc.c != c_omega) {
    const int n = (Mf > W ? Mf : W);
    k_static_tables<<<(n + 255) / 256, 256, 0, st>>>(tb, H, W, Mf, Wh, blue, c_omega);
    k_static_bhat<<<(Mf + 127) / 128, 128, 0, st>>>(tb, W, Mf, Wh, blue);
    if (cudaGetLastError() != cudaSuccess) return SEGSALSA_ERR_CUDA;
    dc.H = H; dc.W = W; dc.c = c_omega;
    rebuilt = true;
  }

  pl.tw = reinterpret_cast<const float2*>(tb + TL.tw);
  pl.chirp = reinterpret_cast<const float2*>(tb + TL.chirp);
  pl.bhat = reinterpret_cast<const float2*>(tb + TL.bhat);

  const int Q = (K + 1) / 2;
  const int QB = row_pairs_per_cta(Mf, Q);
  const int nq = (Q + QB - 1) / QB;
  const RowLaunch rl = row_launch_config<float>(W, Mf, blue, QB);
  if (rl.smem > 227 * 1024) return SEGSALSA_ERR_OOM;

  RowArgs<float> ra{};
  ra.H = H; ra.W = W; ra.K = K; ra.Wh = Wh; ra.QB = QB; ra.smem_tables = rl.tables; ra.pl = pl;
  ra.lgB = 0;
  while ((1 << ra.lgB) < QB) ++ra.lgB;
  ra.mgB = div_magic(QB);
  ra.src = rhs; ra.S = reinterpret_cast<cplx<float>*>(spec); ra.z = z;
  ColArgs<float> ca{};
  ca.H = H; ca.C = Wh * K; ca.K = K; ca.CB = CB;
  ca.NSEG = H / 24 < 1 ? 1 : (H / 24 > 1024 / (2 * CB) ? 1024 / (2 * CB) : H / 24);
  col_segments(H, ca.NSEG, 2 * CB, (int)sizeof(float), ca.SL, ca.NSEG);
  ca.beta = reinterpret_cast<const float*>(tb + TL.beta);
  ca.gain = reinterpret_cast<const float*>(tb + TL.gain);
  ca.wfac = reinterpret_cast<const float*>(tb + TL.wfac);
  ca.nwarm = reinterpret_cast<const int*>(tb + TL.nwarm);
  ca.S = ra.S;
  const int col_threads = (2 * CB * ca.NSEG + 31) / 32 * 32;
  const int ncolblk = (Wh * K + CB - 1) / CB;

  const dim3 rg(nq, H);
  // the forward row pass copies the tables before its programmatic-dependency wait, so right
  // after a rebuild it must be an ordinary launch (it then starts once k_static_bhat is done)
  if (launch_row<float>(true, ra, rg, rl, st, !rebuilt) != cudaSuccess ||
      launch_col<float>(ca, ncolblk, col_threads, col_smem, st) != cudaSuccess ||
      launch_row<float>(false, ra, rg, rl, st) != cudaSuccess)
    return SEGSALSA_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? SEGSALSA_OK : SEGSALSA_ERR_CUDA;
}
