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

// The full form of the local duals ([n][3][K]: d1, d3, d4) from the compact form the affine
// sweep writes ([n][K + 2]: d3, c1, c4; d1 = c1 p, d4 = c4 1), with the sweep's own product
// for d1, so that either form gives the next sweep the same values.
template <typename T>
__global__ void k_dl_expand(const T* __restrict__ dc, const T* __restrict__ p, T* __restrict__ dl,
                            int n, int K) {
  const size_t tot = (size_t)n * K;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / K;
    const int k = (int)(i - pix * K);
    const T* c = dc + pix * (K + 2);
    T* o = dl + pix * 3 * K + k;
    o[0] = c[K] * p[i];
    o[K] = c[k];
    o[2 * K] = c[K + 1];
  }
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

// v mod n for v >= -n: one conditional correction in the common case, a division only when v
// is two periods or more past the end (halo entries of a partial tile on a narrow image).
__device__ __forceinline__ int wrap_near(int v, int n) {
  if (v < 0) v += n;
  if (v >= n) {
    v -= n;
    if (v >= n) v %= n;
  }
  return v;
}

// G consecutive values of a pixel's classes (K valid, the rest zero): 16-byte loads when the
// row of K values is 16-byte aligned and a whole number of vectors, scalar loads otherwise.
template <typename T, int G>
__device__ __forceinline__ void load_classes(const T* __restrict__ src, int K, T (&v)[G]) {
  constexpr int VE = 16 / sizeof(T);
  if (K % VE == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
    for (int k0 = 0; k0 < G; k0 += VE) {
      if (k0 < K) {
        if constexpr (sizeof(T) == 4) {
          const float4 w = __ldg(reinterpret_cast<const float4*>(src + k0));
          v[k0] = w.x; v[k0 + 1] = w.y; v[k0 + 2] = w.z; v[k0 + 3] = w.w;
        } else {
          const double2 w = __ldg(reinterpret_cast<const double2*>(src + k0));
          v[k0] = w.x; v[k0 + 1] = w.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e) v[k0 + e] = T(0);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < G; ++k) v[k] = k < K ? __ldg(src + k) : T(0);
  }
}

// The 16 / sizeof(T) classes k0, k0 + 1, ... of a pixel's row of K values (zero past K): one
// 16-byte load when they are whole and aligned, scalar loads otherwise.
template <typename T>
__device__ __forceinline__ void load_chunk(const T* __restrict__ row, int k0, int K,
                                           T (&c)[16 / sizeof(T)]) {
  constexpr int VE = 16 / sizeof(T);
  const T* src = row + k0;
  if (k0 + VE <= K && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    if constexpr (sizeof(T) == 4) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(src));
      c[0] = w.x; c[1] = w.y; c[2] = w.z; c[3] = w.w;
    } else {
      const double2 w = __ldg(reinterpret_cast<const double2*>(src));
      c[0] = w.x; c[1] = w.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < VE; ++e) c[e] = k0 + e < K ? __ldg(src + e) : T(0);
  }
}

// Euclidean projection of every pixel vector onto the probability simplex (Michelot's
// active-set iteration: theta = (sum of the active entries - 1) / |active|, drop entries
// <= theta, repeat; exact after at most K rounds), plus per-block partials of min z,
// max |1^T z - 1|, sum_i -ln(p_i^T proj(z_i)) and ||G^T d||^2 (G^T d gathered from the tile
// partials P2 in the row pass's order: covY vertical covers per row, offX per-column tile
// offsets; or read from the dense gtd [n][K] when it is given). One pixel per thread, its G
// class values in registers (classes >= K are zero), the active set as a bit mask.
template <typename T, int G>
__global__ void __launch_bounds__(AUX_THREADS) k_project(const T* z, const T* p, T* zp, int n,
                                                        int K, const T* P2, const T* gtd,
                                                        const int* covY,
                                                        const int* offX, int W, int ntx,
                                                        int EHmax, int EWmax,
                                                        double* part /*[blocks][4]*/) {
  __shared__ double red32[32];
  T vmin = T(1e30), vdev = T(0), vdata = T(0), vgsq = T(0);
  const uint32_t all = K >= 32 ? 0xffffffffu : ((1u << K) - 1u);
  pdl_wait();
  constexpr int VE = 16 / sizeof(T);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T v[G], pk[G];
    load_classes<T, G>(z + (size_t)i * K, K, v);
    load_classes<T, G>(p + (size_t)i * K, K, pk);
    // ||G^T d||^2 first: its loads do not depend on the projection, so they are in flight
    // together with those of z and p
    if (gtd) {
#pragma unroll
      for (int k0 = 0; k0 < G; k0 += VE) {
        if (k0 >= K) break;
        T gd[VE];
        load_chunk<T>(gtd + (size_t)i * K, k0, K, gd);
#pragma unroll
        for (int e = 0; e < VE; ++e) vgsq += gd[e] * gd[e];
      }
    } else {
      // G^T d at pixel i: the (at most 2 x 2) covering partials, in the row pass's order
      const int y = i / W, x = i - y * W;
      const int c0 = covY[2 * y], c1 = covY[2 * y + 1];
      const int rb0 = (((c0 >> 16) * ntx * EHmax) + (c0 & 0xffff)) * EWmax * K;
      const int rb1 = c1 < 0 ? -1 : (((c1 >> 16) * ntx * EHmax) + (c1 & 0xffff)) * EWmax * K;
      const int o0 = offX[2 * x], o1 = offX[2 * x + 1];
#pragma unroll
      for (int k0 = 0; k0 < G; k0 += VE) {
        if (k0 >= K) break;
        T g00[VE], g01[VE], g10[VE], g11[VE];
        load_chunk<T>(P2 + rb0 + o0, k0, K, g00);
        if (o1 >= 0) load_chunk<T>(P2 + rb0 + o1, k0, K, g01);
        if (rb1 >= 0) load_chunk<T>(P2 + rb1 + o0, k0, K, g10);
        if (rb1 >= 0 && o1 >= 0) load_chunk<T>(P2 + rb1 + o1, k0, K, g11);
#pragma unroll
        for (int e = 0; e < VE; ++e) {
          T gd = g00[e];
          if (o1 >= 0) gd += g01[e];
          if (rb1 >= 0) gd += g10[e];
          if (rb1 >= 0 && o1 >= 0) gd += g11[e];
          vgsq += gd * gd;
        }
      }
    }
    T s = T(0), mn = v[0];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      s += v[k];
      if (k < K) mn = fmin(mn, v[k]);
    }
    uint32_t act = all;
    T theta = T(0);
    for (int round = 0; round <= K; ++round) {
      T sa = T(0), na = T(0);
#pragma unroll
      for (int k = 0; k < G; ++k)
        if ((act >> k) & 1u) { sa += v[k]; na += T(1); }
      theta = (sa - T(1)) / fmax(na, T(1));
      uint32_t nact = 0;
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (((act >> k) & 1u) && v[k] > theta) nact |= 1u << k;
      if (nact == act) break;
      act = nact;
    }
    T pz = T(0), q[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      q[k] = fmax(v[k] - theta, T(0));
      if (k < K) pz += pk[k] * q[k];
    }
    // the projection out in 16-byte vectors where the pixel's row allows it
    T* zo = zp + (size_t)i * K;
    if (K % VE == 0 && (reinterpret_cast<uintptr_t>(zo) & 15) == 0) {
#pragma unroll
      for (int k0 = 0; k0 < G; k0 += VE) {
        if (k0 >= K) break;
        if constexpr (sizeof(T) == 4)
          *reinterpret_cast<float4*>(zo + k0) = make_float4(q[k0], q[k0 + 1], q[k0 + 2], q[k0 + 3]);
        else
          *reinterpret_cast<double2*>(zo + k0) = make_double2(q[k0], q[k0 + 1]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (k < K) zo[k] = q[k];
    }
    vmin = fmin(vmin, mn);
    vdev = fmax(vdev, fabs(s - T(1)));
    vdata -= log(pz);
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

// sum_i ||[J zp]_i||_{S_p} per block (zp pixel-major). The Gram matrix of pixel i's patch
// Jacobian (eq. 5) is sum_j omega_j^2 T(i + s_j), where T(m) = sum_k (grad z_k)(grad z_k)^T
// at pixel m (forward differences): the structure tensor of Sec. 3. A block takes tiles of
// PRIOR_TH x PRIOR_TW pixels: it first forms the three entries of T on the tile and its
// M-pixel halo in shared memory (one pixel per thread, classes in registers), then every
// pixel sums the L weighted taps and takes the norm from the two eigenvalues.
constexpr int PRIOR_TH = 8, PRIOR_TW = 32;  // PRIOR_TH * PRIOR_TW == AUX_THREADS
template <typename T, int M, int G>
__global__ void __launch_bounds__(AUX_THREADS) k_prior(const T* zp, const T* omega, int H, int W,
                                                      int K, int sp, double* part) {
  constexpr int P = 2 * M + 1;
  constexpr int RH = PRIOR_TH + 2 * M, RW = PRIOR_TW + 2 * M;
  // Where it fits, the tile's projected z (the tile, its halo and one more row and column for
  // the forward differences) is first copied into shared memory, each pixel read once from
  // global memory instead of three times; pixels padded by one 16-byte chunk so that
  // consecutive pixels' chunks fall on different banks. Same differences, same sums.
  constexpr int VE = 16 / sizeof(T);
  constexpr int ZH = RH + 1, ZW = RW + 1, PS = G + VE;
  constexpr bool ZTILE = (size_t)ZH * ZW * PS * sizeof(T) <= 32 * 1024;
  __shared__ double red32[32];
  __shared__ T sA[RH * RW], sB[RH * RW], sC[RH * RW];
  __shared__ T w2[P * P];
  __shared__ __align__(16) T sZ[ZTILE ? ZH * ZW * PS : VE];
  for (int j = threadIdx.x; j < P * P; j += blockDim.x) w2[j] = omega[j] * omega[j];
  const int ntx = (W + PRIOR_TW - 1) / PRIOR_TW;
  const int ntiles = ((H + PRIOR_TH - 1) / PRIOR_TH) * ntx;
  T val = T(0);
  pdl_wait();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int y0 = (tile / ntx) * PRIOR_TH, x0 = (tile % ntx) * PRIOR_TW;
    __syncthreads();  // the previous tile's reads of sA/sB/sC (and sZ) are done, w2 written
    if constexpr (ZTILE) {
      constexpr int NCH = G / VE;
      for (int i = threadIdx.x; i < ZH * ZW * NCH; i += blockDim.x) {
        const int pix = i / NCH, ch = i - pix * NCH;
        const int ry = pix / ZW, rx = pix - ry * ZW;
        const int y = wrap_near(y0 - M + ry, H), x = wrap_near(x0 - M + rx, W);
        T cz[VE];
        if (ch * VE < K) {
          load_chunk<T>(zp + ((size_t)y * W + x) * K, ch * VE, K, cz);
        } else {
#pragma unroll
          for (int e = 0; e < VE; ++e) cz[e] = T(0);
        }
        T* dz = sZ + pix * PS + ch * VE;
        if constexpr (sizeof(T) == 4)
          *reinterpret_cast<float4*>(dz) = make_float4(cz[0], cz[1], cz[2], cz[3]);
        else
          *reinterpret_cast<double2*>(dz) = make_double2(cz[0], cz[1]);
      }
      __syncthreads();
      for (int r = threadIdx.x; r < RH * RW; r += blockDim.x) {
        const int ry = r / RW, rx = r - ry * RW;
        const T* zc = sZ + (ry * ZW + rx) * PS;   // pixel (ry, rx); + PS: (ry, rx + 1)
        const T* zv = zc + ZW * PS;               // (ry + 1, rx)
        T a = T(0), b = T(0), c = T(0);
#pragma unroll
        for (int k0 = 0; k0 < G; k0 += VE) {
          if (k0 >= K) break;
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            const T h = zc[PS + k0 + e] - zc[k0 + e], v = zv[k0 + e] - zc[k0 + e];
            a += h * h;
            b += h * v;
            c += v * v;
          }
        }
        sA[r] = a;
        sB[r] = b;
        sC[r] = c;
      }
    } else {
      for (int r = threadIdx.x; r < RH * RW; r += blockDim.x) {
        const int ry = r / RW, rx = r - ry * RW;
        const int y = wrap_near(y0 - M + ry, H), x = wrap_near(x0 - M + rx, W);  // M < H, W
        const int xh = x + 1 == W ? 0 : x + 1, yv = y + 1 == H ? 0 : y + 1;
        const T* rc = zp + ((size_t)y * W + x) * K;
        const T* rh = zp + ((size_t)y * W + xh) * K;
        const T* rv = zp + ((size_t)yv * W + x) * K;
        T a = T(0), b = T(0), c = T(0);
#pragma unroll
        for (int k0 = 0; k0 < G; k0 += VE) {
          if (k0 >= K) break;
          T zc[VE], zh[VE], zv[VE];
          load_chunk<T>(rc, k0, K, zc);
          load_chunk<T>(rh, k0, K, zh);
          load_chunk<T>(rv, k0, K, zv);
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            const T h = zh[e] - zc[e], v = zv[e] - zc[e];
            a += h * h;
            b += h * v;
            c += v * v;
          }
        }
        sA[r] = a;
        sB[r] = b;
        sC[r] = c;
      }
    }
    __syncthreads();
    const int ty = threadIdx.x / PRIOR_TW, tx = threadIdx.x - ty * PRIOR_TW;
    if (y0 + ty < H && x0 + tx < W) {
      T a = T(0), b = T(0), c = T(0);
#pragma unroll
      for (int dy = 0; dy < P; ++dy)
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
          const T w = w2[dy * P + dx];
          const int r = (ty + dy) * RW + tx + dx;
          a += w * sA[r];
          b += w * sB[r];
          c += w * sC[r];
        }
      const T hd = T(0.5) * (a - c);
      const T rr = sqrt(hd * hd + b * b);
      const T s1 = sqrt(fmax(T(0.5) * (a + c) + rr, T(0)));
      const T s2 = sqrt(fmax(T(0.5) * (a + c) - rr, T(0)));
      val += (sp == 1) ? s1 + s2 : (sp == 2) ? sqrt(fmax(a + c, T(0))) : s1;
    }
  }
  const double t = block_sum_w<T>(val, red32);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <typename T, int G>
inline void launch_project(int blocks, cudaStream_t st, const T* z, const T* p, T* zp, int n,
                           int K, const T* P2, const T* gtd, const int* covY, const int* offX,
                           int W, int ntx, int EHmax, int EWmax, double* part) {
  launch_pdl(k_project<T, G>, dim3(blocks), dim3(AUX_THREADS), 0, st, z, p, zp, n, K, P2, gtd,
             covY, offX, W, ntx, EHmax, EWmax, part);
}
template <typename T>
inline cudaError_t launch_project_g(int G, int blocks, cudaStream_t st, const T* z, const T* p,
                                    T* zp, int n, int K, const T* P2, const T* gtd,
                                    const int* covY, const int* offX, int W, int ntx, int EHmax,
                                    int EWmax, double* part) {
  switch (G) {
    case 4: launch_project<T, 4>(blocks, st, z, p, zp, n, K, P2, gtd, covY, offX, W, ntx, EHmax, EWmax, part); break;
    case 8: launch_project<T, 8>(blocks, st, z, p, zp, n, K, P2, gtd, covY, offX, W, ntx, EHmax, EWmax, part); break;
    case 16: launch_project<T, 16>(blocks, st, z, p, zp, n, K, P2, gtd, covY, offX, W, ntx, EHmax, EWmax, part); break;
    default: launch_project<T, 32>(blocks, st, z, p, zp, n, K, P2, gtd, covY, offX, W, ntx, EHmax, EWmax, part); break;
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
template <typename T, int M>
inline cudaError_t prior_blocks_per_sm_m(int G, int* nb) {
  switch (G) {
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_prior<T, M, 4>, AUX_THREADS, 0);
    case 8: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_prior<T, M, 8>, AUX_THREADS, 0);
    case 16: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_prior<T, M, 16>, AUX_THREADS, 0);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_prior<T, M, 32>, AUX_THREADS, 0);
  }
}
// Resident blocks per SM of the prior kernel (its tile loop is sized to one wave of them).
template <typename T>
inline cudaError_t prior_blocks_per_sm(int M, int G, int* nb) {
  switch (M) {
    case 0: return prior_blocks_per_sm_m<T, 0>(G, nb);
    case 1: return prior_blocks_per_sm_m<T, 1>(G, nb);
    case 2: return prior_blocks_per_sm_m<T, 2>(G, nb);
    case 3: return prior_blocks_per_sm_m<T, 3>(G, nb);
    case 4: return prior_blocks_per_sm_m<T, 4>(G, nb);
    default: return prior_blocks_per_sm_m<T, 5>(G, nb);
  }
}
template <typename T>
inline cudaError_t launch_prior(int M, int G, int blocks, cudaStream_t st, const T* zp,
                                const T* om, int H, int W, int K, int sp, double* part) {
  switch (M) {
    case 0: launch_prior_m<T, 0>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    case 1: launch_prior_m<T, 1>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    case 2: launch_prior_m<T, 2>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    case 3: launch_prior_m<T, 3>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    case 4: launch_prior_m<T, 4>(G, blocks, st, zp, om, H, W, K, sp, part); break;
    default: launch_prior_m<T, 5>(G, blocks, st, zp, om, H, W, K, sp, part); break;
  }
  return cudaGetLastError();
}

// One trace record (k, primal, dual, objective, min z, max |1^T z - 1|), reducing the block
// partials in a fixed order: FT_THREADS threads each sum a strided subset in FP64 (four
// independent chains, so that loads are in flight together: one warp took 79 us for the 16384
// tile partials of a 2048 x 2048 image, bound by load latency), then a fixed shuffle tree per
// warp and the warp results in warp order.
constexpr int FT_THREADS = 1024;

__global__ void __launch_bounds__(FT_THREADS) k_finalize_trace(
    const double* sq, int nsq, const double* proj, int nproj, const double* prior, int nprior,
    double k, double mu, double lambda, double* rec) {
  __shared__ double red[6][FT_THREADS / 32];
  const int t = threadIdx.x, l = t & 31, w = t >> 5;
  auto sum = [&](const double* v, int n, int stride, int off) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = t; i0 < n; i0 += 4 * FT_THREADS) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + FT_THREADS * u;
        if (i < n) acc[u] += v[stride * i + off];
      }
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
  };
  pdl_wait();
  double v[6];
  v[0] = sum(sq, nsq, 1, 0);
  v[1] = sum(proj, nproj, 4, 3);
  v[2] = sum(proj, nproj, 4, 2);
  v[3] = sum(prior, nprior, 1, 0);
  v[4] = 1e300;
  v[5] = 0.0;
  for (int i = t; i < nproj; i += FT_THREADS) {
    v[4] = fmin(v[4], proj[4 * i]);
    v[5] = fmax(v[5], proj[4 * i + 1]);
  }
  auto tree = [&](double (&x)[6]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
      x[4] = fmin(x[4], __shfl_xor_sync(0xffffffffu, x[4], o));
      x[5] = fmax(x[5], __shfl_xor_sync(0xffffffffu, x[5], o));
    }
  };
  tree(v);
  if (l == 0)
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q][w] = v[q];
  __syncthreads();
  if (w == 0) {
    double x[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) x[q] = red[q][l];
    tree(x);
    if (l == 0) {
      rec[0] = k;
      rec[1] = sqrt(x[0]);
      rec[2] = mu * sqrt(x[1]);
      rec[3] = x[2] + lambda * x[3];
      rec[4] = x[4];
      rec[5] = x[5];
    }
  }
}

}  // namespace sgs
