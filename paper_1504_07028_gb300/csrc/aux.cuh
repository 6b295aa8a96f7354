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
// <= theta, repeat; exact after at most K rounds), plus per-block partials of min z,
// max |1^T z - 1|, sum_i -ln(p_i^T proj(z_i)) and ||G^T d||^2 (G^T d gathered from the tile
// partials P2 in the row pass's order: covY vertical covers per row, offX per-column tile
// offsets). G lanes per pixel, class k on lane k.
template <typename T, int G>
__global__ void __launch_bounds__(AUX_THREADS) k_project(const T* z, const T* p, T* zp, int n,
                                                        int K, const T* P2, const int* covY,
                                                        const int* offX, int W, int ntx,
                                                        int EHmax, int EWmax,
                                                        double* part /*[blocks][4]*/) {
  __shared__ double red32[32];
  constexpr int PPB = AUX_THREADS / G;
  const int g = threadIdx.x % G;
  T vmin = T(1e30), vdev = T(0), vdata = T(0), vgsq = T(0);
  pdl_wait();
  for (int i0 = blockIdx.x * PPB; i0 < n; i0 += gridDim.x * PPB) {
    const int i = i0 + threadIdx.x / G;
    const bool ok = i < n && g < K;
    const T v = ok ? z[(size_t)i * K + g] : T(0);
    const T pk = ok ? p[(size_t)i * K + g] : T(0);
    bool act = ok;
    const T s = group_sum<G>(v);
    T theta = T(0);
    for (int round = 0; round <= K; ++round) {
      const T sa = group_sum<G>(act ? v : T(0));
      const T na = group_sum<G>(act ? T(1) : T(0));
      theta = (sa - T(1)) / fmax(na, T(1));
      const bool nact = act && v > theta;
      const bool changed = act && !nact;
      act = nact;
      if (!__any_sync(0xffffffffu, changed)) break;  // warp-uniform exit (groups share shuffles)
    }
    const T q = ok ? fmax(v - theta, T(0)) : T(0);
    if (ok) zp[(size_t)i * K + g] = q;
    const T pz = group_sum<G>(pk * q);
    if (ok) {
      vmin = fmin(vmin, v);
      const int y = i / W, x = i - y * W;
      const int c0 = covY[2 * y], c1 = covY[2 * y + 1];
      const int rb0 = c0 < 0 ? -1 : (((c0 >> 16) * ntx * EHmax) + (c0 & 0xffff)) * EWmax * K;
      const int rb1 = c1 < 0 ? -1 : (((c1 >> 16) * ntx * EHmax) + (c1 & 0xffff)) * EWmax * K;
      const int o0 = offX[2 * x], o1 = offX[2 * x + 1];
      T gd = T(0);
      if (rb0 >= 0) {
        if (o0 >= 0) gd += P2[rb0 + o0 + g];
        if (o1 >= 0) gd += P2[rb0 + o1 + g];
      }
      if (rb1 >= 0) {
        if (o0 >= 0) gd += P2[rb1 + o0 + g];
        if (o1 >= 0) gd += P2[rb1 + o1 + g];
      }
      vgsq += gd * gd;
    }
    if (i < n && g == 0) {
      vdev = fmax(vdev, fabs(s - T(1)));
      vdata -= log(pz);
    }
  }
  const double a = block_min_w<T>(vmin, red32);
  if (threadIdx.x == 0) part[4 * blockIdx.x + 0] = a;
  const double b = block_max_w<T>(vdev, red32);
  if (threadIdx.x == 0) part[4 * blockIdx.x + 1] = b;
  const double c = block_sum_w<T>(vdata, red32);
  if (threadIdx.x == 0) part[4 * blockIdx.x + 2] = c;
  const double d = block_sum_w<T>(vgsq, red32);
  if (threadIdx.x == 0) part[4 * blockIdx.x + 3] = d;
}

// sum_i ||[J zp]_i||_{S_p} per block (zp pixel-major), via the 2x2 Gram matrix of eq. (5):
// G lanes per pixel (class k on lane k) accumulate their 2L Jacobian entries, a G-lane sum
// gives the Gram matrix. Block sums in double.
template <typename T, int M, int G>
__global__ void __launch_bounds__(AUX_THREADS) k_prior(const T* zp, const T* omega, int H, int W,
                                                      int K, int sp, double* part) {
  __shared__ double red32[32];
  constexpr int PPB = AUX_THREADS / G;
  constexpr int P = 2 * M + 1;
  const int g = threadIdx.x % G;
  const int n = H * W;
  T val = T(0);
  pdl_wait();
  for (int i0 = blockIdx.x * PPB; i0 < n; i0 += gridDim.x * PPB) {
    const int i = i0 + threadIdx.x / G;
    const bool ok = i < n && g < K;
    const int y = ok ? i / W : 0, x = ok ? i % W : 0;
    T zv[P + 1][P + 1];
    int xs[P + 1];
#pragma unroll
    for (int dx = 0; dx <= P; ++dx) {
      int xx = x - M + dx;
      xx += (xx < 0) ? W : 0;
      xx -= (xx >= W) ? W : 0;
      xs[dx] = xx;
    }
#pragma unroll
    for (int dy = 0; dy <= P; ++dy) {
      int yy = y - M + dy;
      yy += (yy < 0) ? H : 0;
      yy -= (yy >= H) ? H : 0;
      const size_t row = (size_t)yy * W;
#pragma unroll
      for (int dx = 0; dx <= P; ++dx)
        zv[dy][dx] = (ok && !(dy == P && dx == P)) ? zp[(row + xs[dx]) * K + g] : T(0);
    }
    T a = T(0), b = T(0), c = T(0);
#pragma unroll
    for (int dy = 0; dy < P; ++dy)
#pragma unroll
      for (int dx = 0; dx < P; ++dx) {
        const T w = omega[dy * P + dx];
        const T h = w * (zv[dy][dx + 1] - zv[dy][dx]);
        const T v = w * (zv[dy + 1][dx] - zv[dy][dx]);
        a += h * h;
        b += h * v;
        c += v * v;
      }
    a = group_sum<G>(a);
    b = group_sum<G>(b);
    c = group_sum<G>(c);
    if (i < n && g == 0) {
      const T hd = T(0.5) * (a - c);
      const T r = sqrt(hd * hd + b * b);
      const T s1 = sqrt(fmax(T(0.5) * (a + c) + r, T(0)));
      const T s2 = sqrt(fmax(T(0.5) * (a + c) - r, T(0)));
      val += (sp == 1) ? s1 + s2 : (sp == 2) ? sqrt(fmax(a + c, T(0))) : s1;
    }
  }
  const double t = block_sum_w<T>(val, red32);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <typename T, int G>
inline void launch_project(int blocks, cudaStream_t st, const T* z, const T* p, T* zp, int n,
                           int K, const T* P2, const int* covY, const int* offX, int W, int ntx,
                           int EHmax, int EWmax, double* part) {
  launch_pdl(k_project<T, G>, dim3(blocks), dim3(AUX_THREADS), 0, st, z, p, zp, n, K, P2, covY,
             offX, W, ntx, EHmax, EWmax, part);
}
template <typename T>
inline cudaError_t launch_project_g(int G, int blocks, cudaStream_t st, const T* z, const T* p,
                                    T* zp, int n, int K, const T* P2, const int* covY,
                                    const int* offX, int W, int ntx, int EHmax, int EWmax,
                                    double* part) {
  switch (G) {
    case 4: launch_project<T, 4>(blocks, st, z, p, zp, n, K, P2, covY, offX, W, ntx, EHmax, EWmax, part); break;
    case 8: launch_project<T, 8>(blocks, st, z, p, zp, n, K, P2, covY, offX, W, ntx, EHmax, EWmax, part); break;
    case 16: launch_project<T, 16>(blocks, st, z, p, zp, n, K, P2, covY, offX, W, ntx, EHmax, EWmax, part); break;
    default: launch_project<T, 32>(blocks, st, z, p, zp, n, K, P2, covY, offX, W, ntx, EHmax, EWmax, part); break;
  }
  return cudaGetLastError();
}
template <typename T, int M>
inline void launch_prior_m(int G, int blocks, cudaStream_t st, const T* zp, const T* om, int H,
                           int W, int K, int sp, double* part) {
  switch (G) {
    case 4: launch_pdl(k_prior<T, M, 4>, dim3(blocks), dim3(AUX_THREADS), 0, st, zp, om, H, W, K, sp, part); break;
    case 8: launch_pdl(k_prior<T, M, 8>, dim3(blocks), dim3(AUX_THREADS), 0, st, zp, om, H, W, K, sp, part); break;
    case 16: launch_pdl(k_prior<T, M, 16>, dim3(blocks), dim3(AUX_THREADS), 0, st, zp, om, H, W, K, sp, part); break;
    default: launch_pdl(k_prior<T, M, 32>, dim3(blocks), dim3(AUX_THREADS), 0, st, zp, om, H, W, K, sp, part); break;
  }
}
template <typename T>
inline cudaError_t launch_prior(int M, int G, int blocks, cudaStream_t st, const T* zp,
                                const T* om, int H, int W, int K, int sp, double* part) {
  switch (M) {
    case 0: launch_prior_m<T, 0>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    case 1: launch_prior_m<T, 1>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    default: launch_prior_m<T, 2>(G, blocks, st, zp, om, H, W, K, sp, part); break;
  }
  return cudaGetLastError();
}

// One trace record (k, primal, dual, objective, min z, max |1^T z - 1|), reducing the block
// partials in a fixed order. One warp: each lane sums a strided subset in FP64 (four independent
// chains), then shuffles; no block barriers (the partials number a few hundred to a few
// thousand, and FP64 is a narrow pipe on this part).
__global__ void __launch_bounds__(32) k_finalize_trace(
    const double* sq, int nsq, const double* proj, int nproj, const double* prior, int nprior,
    double k, double mu, double lambda, double* rec) {
  const int l = threadIdx.x;
  auto sum = [&](const double* v, int n, int stride, int off) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = l; i0 < n; i0 += 4 * 32) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + 32 * u;
        if (i < n) acc[u] += v[stride * i + off];
      }
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
  };
  pdl_wait();
  double a = sum(sq, nsq, 1, 0);
  double b = sum(proj, nproj, 4, 3);
  double c = sum(proj, nproj, 4, 2);
  double d = sum(prior, nprior, 1, 0);
  double mn = 1e300, mx = 0.0;
  for (int i = l; i < nproj; i += 32) {
    mn = fmin(mn, proj[4 * i]);
    mx = fmax(mx, proj[4 * i + 1]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (l == 0) {
    rec[0] = k;
    rec[1] = sqrt(a);
    rec[2] = mu * sqrt(b);
    rec[3] = c + lambda * d;
    rec[4] = mn;
    rec[5] = mx;
  }
}

}  // namespace sgs
