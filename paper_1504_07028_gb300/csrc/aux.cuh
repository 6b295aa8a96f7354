// Auxiliary kernels of SegSALSA-STR: input checks, z^0, layout changes, label readout and the
// traced diagnostics (primal / dual residual, objective (7) at the simplex projection).
#pragma once

#include "common.cuh"
#include "sweep.cuh"

namespace sgs {

constexpr int AUX_THREADS = 256;

// Input check of p (eq. 7 needs p_i^T z_i > 0 on the feasible set): bit 0 non-finite,
// bit 1 negative entry, bit 2 a pixel without a positive entry. p is pixel-major.
template <typename T>
__global__ void k_check_probs(const T* p, int n, int K, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  bool pos = false;
  for (int k = 0; k < K; ++k) {
    const T v = p[(size_t)i * K + k];
    if (!isfinite(v)) f |= 1;
    else if (v < T(0)) f |= 2;
    else if (v > T(0)) pos = true;
  }
  if (!pos) f |= 4;
  if (f) atomicOr(flags, f);
}

// z^0 = p_i / 1^T p_i (pixel-major).
template <typename T>
__global__ void k_init_z(const T* p, T* z, int n, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = T(0);
  for (int k = 0; k < K; ++k) s += p[(size_t)i * K + k];
  const T inv = T(1) / s;
  for (int k = 0; k < K; ++k) z[(size_t)i * K + k] = p[(size_t)i * K + k] * inv;
}

// (K, n) <-> (n, K)
template <typename T>
__global__ void k_khw_to_hwk(const T* src, T* dst, int n, int K) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n * K) return;
  const size_t pix = i / K, k = i % K;
  dst[i] = src[k * n + pix];
}
template <typename T>
__global__ void k_hwk_to_khw(const T* src, T* dst, int n, int K) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n * K) return;
  const size_t k = i / n, pix = i % n;
  dst[i] = src[pix * K + k];
}

// argmax_k z_k, ties to the lowest k.
template <typename T>
__global__ void k_labels(const T* z, int n, int K, int32_t* lab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T* zi = z + (size_t)i * K;
  T best = zi[0];
  int arg = 0;
  for (int k = 1; k < K; ++k) {
    const T v = zi[k];
    if (v > best) { best = v; arg = k; }
  }
  lab[i] = arg;
}

// Euclidean projection of every pixel vector onto the probability simplex (Michelot's
// active-set iteration: theta = (sum of the active entries - 1) / |active|, drop entries
// <= theta, repeat; exact after at most K rounds), plus per-block partials of
// min z, max |1^T z - 1| and sum_i -ln(p_i^T proj(z_i)).
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS) k_project(const T* z, const T* p, T* zp, int n,
                                                        int K, double* part /*[blocks][3]*/) {
  __shared__ double red32[32];
  T vmin = T(1e30), vdev = T(0), vdata = T(0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T* zi = z + (size_t)i * K;
    T v[32];
    unsigned act = 0;
    T s = T(0);
    for (int k = 0; k < K; ++k) {
      v[k] = zi[k];
      s += v[k];
      vmin = fmin(vmin, v[k]);
      act |= 1u << k;
    }
    vdev = fmax(vdev, fabs(s - T(1)));
    T theta = T(0);
    for (int round = 0; round <= K; ++round) {
      T sa = T(0);
      int na = 0;
      for (int k = 0; k < K; ++k)
        if (act >> k & 1u) { sa += v[k]; ++na; }
      theta = (sa - T(1)) / T(na);
      unsigned nact = act;
      for (int k = 0; k < K; ++k)
        if ((act >> k & 1u) && v[k] <= theta) nact &= ~(1u << k);
      if (nact == act || nact == 0) break;
      act = nact;
    }
    T pz = T(0);
    for (int k = 0; k < K; ++k) {
      const T q = fmax(v[k] - theta, T(0));
      zp[(size_t)i * K + k] = q;
      pz += p[(size_t)i * K + k] * q;
    }
    vdata -= log(pz);
  }
  const double a = block_min_d((double)vmin, red32);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 0] = a;
  const double b = block_max_d((double)vdev, red32);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 1] = b;
  const double c = block_sum_d((double)vdata, red32);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 2] = c;
}

// sum_i ||[J zp]_i||_{S_p} per block (zp pixel-major), via the 2x2 Gram matrix of eq. (5).
// Per-pixel arithmetic in T, block sums in double; grid-stride over pixels.
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS) k_prior(const T* zp, const T* omega, int H, int W,
                                                      int K, int M, int sp, double* part) {
  __shared__ double red32[32];
  T val = T(0);
  const int P = 2 * M + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H * W; i += gridDim.x * blockDim.x) {
    const int y = i / W, x = i % W;
    T a = T(0), b = T(0), c = T(0);
    for (int dy = -M; dy <= M; ++dy)
      for (int dx = -M; dx <= M; ++dx) {
        const T w = omega[(dy + M) * P + (dx + M)];
        const int y0 = wrap_idx(y + dy, H), x0 = wrap_idx(x + dx, W);
        const int y1 = wrap_idx(y0 + 1, H), x1 = wrap_idx(x0 + 1, W);
        const T* z00 = zp + ((size_t)y0 * W + x0) * K;
        const T* z01 = zp + ((size_t)y0 * W + x1) * K;
        const T* z10 = zp + ((size_t)y1 * W + x0) * K;
        for (int k = 0; k < K; ++k) {
          const T h = w * (z01[k] - z00[k]);
          const T v = w * (z10[k] - z00[k]);
          a += h * h;
          b += h * v;
          c += v * v;
        }
      }
    const T hd = T(0.5) * (a - c);
    const T r = sqrt(hd * hd + b * b);
    const T s1 = sqrt(fmax(T(0.5) * (a + c) + r, T(0)));
    const T s2 = sqrt(fmax(T(0.5) * (a + c) - r, T(0)));
    val += (sp == 1) ? s1 + s2 : (sp == 2) ? sqrt(fmax(a + c, T(0))) : s1;
  }
  const double t = block_sum_d((double)val, red32);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Sum of squares of G^T d, gathered from the tile partials P2 like the row pass does.
template <typename T>
__global__ void __launch_bounds__(AUX_THREADS) k_gather_sq(const T* P2, const int* covY,
                                                          const int* covX, int H, int W, int K,
                                                          int ntx, int EHmax, int EWmax,
                                                          double* part) {
  __shared__ double red32[32];
  T val = T(0);
  const size_t tot = (size_t)H * W * K;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % K);
    const size_t pix = i / K;
    const int y = (int)(pix / W), x = (int)(pix % W);
    T v = T(0);
    for (int iy = 0; iy < 2; ++iy) {
      const int cy = covY[2 * y + iy];
      if (cy < 0) continue;
      for (int ix = 0; ix < 2; ++ix) {
        const int cx = covX[2 * x + ix];
        if (cx < 0) continue;
        const size_t t = (size_t)(cy >> 16) * ntx + (cx >> 16);
        v += P2[((t * EHmax + (cy & 0xffff)) * EWmax + (cx & 0xffff)) * K + k];
      }
    }
    val += v * v;
  }
  const double t = block_sum_d((double)val, red32);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// One trace record (k, primal, dual, objective, min z, max |1^T z - 1|), reducing the block
// partials in a fixed order.
__global__ void k_finalize_trace(const double* sq, int nsq, const double* gsq, int ngsq,
                                 const double* proj, int nproj, const double* prior, int nprior,
                                 double k, double mu, double lambda, double* rec) {
  __shared__ double red32[32];
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0, mn = 1e300, mx = 0.0;
  for (int i = threadIdx.x; i < nsq; i += blockDim.x) a += sq[i];
  for (int i = threadIdx.x; i < ngsq; i += blockDim.x) b += gsq[i];
  for (int i = threadIdx.x; i < nproj; i += blockDim.x) {
    mn = fmin(mn, proj[3 * i]);
    mx = fmax(mx, proj[3 * i + 1]);
    c += proj[3 * i + 2];
  }
  for (int i = threadIdx.x; i < nprior; i += blockDim.x) d += prior[i];
  a = block_sum_d(a, red32);
  if (threadIdx.x == 0) rec[1] = sqrt(a);
  b = block_sum_d(b, red32);
  if (threadIdx.x == 0) rec[2] = mu * sqrt(b);
  c = block_sum_d(c, red32);
  d = block_sum_d(d, red32);
  if (threadIdx.x == 0) rec[3] = c + lambda * d;
  mn = block_min_d(mn, red32);
  if (threadIdx.x == 0) rec[4] = mn;
  mx = block_max_d(mx, red32);
  if (threadIdx.x == 0) { rec[5] = mx; rec[0] = k; }
}

}  // namespace sgs
