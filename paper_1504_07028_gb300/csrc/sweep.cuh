// Fused SALSA sweep (u-update (13) + d-update (14) + right-hand side of the next z-update (12))
// for SegSALSA-STR, one launch per iteration.
//
// Per pixel i (Sec. 4):
//   v1 = z - d1,  v2 = J z - d2,  v3 = z - d3,  v4 = z - d4              (G z^{k+1} - d^k)
//   u1 = prox of -ln(p^T .)/mu at v1 (positive root of s^2 - (p^T v1) s - |p|^2/mu = 0)
//   u2 = Schatten-p prox of (lambda/mu)||.||_{S_p} at the (L K) x 2 matrix v2  (Sec. 3-4)
//   u3 = max(v3, 0);   u4 = v4 - (1^T v4 - 1)/K                          (MPOs of g3, g4)
//   d_j <- u_j - v_j  (= d_j - (G z - u_j), eq. 14)
//   rhs = (u1 + d1) + J^T (u2 + d2) + (u3 + d3) + (u4 + d4)              (G^T (u + d), eq. 12)
//
// Work mapping. A CTA owns a tile of pixels (balanced tiling of the image) and 256 threads:
// NC = 256/G columns x G lanes. The G lanes of a column hold the classes of one pixel (class
// k = lane), so the 2x2 Gram matrix [Jz]_i^T [Jz]_i of eq. (5) is a G-lane shuffle sum and
// each lane keeps its 2L Jacobian entries in registers. Each column walks down the tile rows.
// The Jacobian stencil reads z from a shared-memory copy of the tile plus its halo
// ([-M, M+1] around every pixel). J^T w is a scatter: pixel i sends +/- omega_j w to the
// (2M+2)^2 neighbours i + s_j (+ e_h / e_v). Each thread keeps those sums for the rows it can
// still touch in a (2M+2)x(2M+2) register window and flushes the finished top row into a
// shared accumulator over the tile plus halo (shared atomics, 2M+2 per pixel and class).
// The accumulator tile, halo included, is written to a partials buffer P; the row-FFT pass
// adds the overlapping tiles when it reads rhs (no global atomics, deterministic).
#pragma once

#include "common.cuh"

namespace sgs {

template <typename T>
struct SweepArgs {
  int H, W, K;
  int ntx, nty;          // tile grid
  int EHmax, EWmax;      // extents of the P tile slots (tile + halo), in pixels
  const T* z;            // [n][K]
  const T* p;            // [n][K]
  T* dloc;               // [n][3][K]  (d1, d3, d4)
  T* d2;                 // [n][L][K][2]
  T* P;                  // [tiles][EHmax][EWmax][K]  partial sums of G^T(u + d)
  T* P2;                 // DIAG: partial sums of G^T d (dual residual)
  double* diag_sq;       // DIAG: per tile sum of squared dual changes (primal residual)
  const T* omega;        // [L] shift weights
  T tau;                 // lambda / mu
  T mu;
  T invK;
  int sp;                // 1, 2, 0 = infinity
};

// Coefficients of u2 = V A for the prox of tau*||.||_{S_p} at V (R x 2) with Gram
// [[a, b], [b, c]] = V^T V. With V = U diag(s) W^T and shrunk values t, u2 = V W diag(g) W^T,
// g_i = t_i / s_i. Writing W diag(g) W^T = gbar I + kap [[hd, b], [b, -hd]], hd = (a - c)/2,
// kap = (g1 - g2) / (l1 - l2), the case formulas below have no cancellation at s1 = s2.
template <typename T>
__device__ __forceinline__ void schatten_coeffs(T a, T b, T c, T tau, int sp, T& A11, T& A12,
                                                T& A22) {
  const T tr = a + c;
  T gbar = T(0), kap = T(0);
  const T hd = T(0.5) * (a - c);
  if (sp == 2) {
    const T nf = sqrt(tr);
    gbar = (nf > tau) ? T(1) - tau / nf : T(0);
  } else if (tr > T(0)) {
    const T r = sqrt(hd * hd + b * b);             // (l1 - l2) / 2
    const T l1 = T(0.5) * tr + r;
    const T l2 = fmax(T(0.5) * tr - r, T(0));
    const T s1 = sqrt(l1), s2 = sqrt(l2);
    if (sp == 1) {
      if (s1 > tau) {
        if (s2 > tau) {
          const T q = s1 * s2;
          gbar = T(1) - tau * (s1 + s2) / (T(2) * q);
          kap = tau / (q * (s1 + s2));
        } else {
          const T g1 = T(1) - tau / s1;
          gbar = T(0.5) * g1;
          kap = (r > T(0)) ? g1 / (T(2) * r) : T(0);
        }
      }
    } else {  // p = infinity: t = s - proj_{tau B1}(s)
      if (s1 + s2 > tau) {
        if (s1 - s2 >= tau) {
          const T g1 = T(1) - tau / s1;  // g2 = 1
          gbar = T(0.5) * (g1 + T(1));
          kap = (r > T(0)) ? (g1 - T(1)) / (T(2) * r) : T(0);
        } else {
          const T t = T(0.5) * (s1 + s2 - tau);  // both shrink to t; here s2 > 0
          const T q = s1 * s2;
          gbar = t * (s1 + s2) / (T(2) * q);
          kap = -t / (q * (s1 + s2));
        }
      }
    }
  } else if (!(tau > T(0))) {
    gbar = T(1);
  }
  A11 = gbar + kap * hd;
  A22 = gbar - kap * hd;
  A12 = kap * b;
}

template <typename T> struct Vec2Of;
template <> struct Vec2Of<float> { using type = float2; };
template <> struct Vec2Of<double> { using type = double2; };

template <typename T, int M, int G, bool DIAG>
__global__ void __launch_bounds__(256, 2) k_sweep(const SweepArgs<T> a) {
  constexpr int L = (2 * M + 1) * (2 * M + 1);
  constexpr int NC = 256 / G;
  constexpr int E = 2 * M + 2;
  using V2 = typename Vec2Of<T>::type;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = a.EHmax * a.EWmax * G;
  T* zs = reinterpret_cast<T*>(smem_raw);
  T* acc = zs + slot;
  T* acc2 = acc + slot;                 // only used when DIAG
  T* om = acc + (DIAG ? 2 : 1) * slot;  // [L]
  __shared__ double red32[32];

  const int tile = blockIdx.x;
  const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
  const int y0 = (int)(((long long)ty * a.H) / a.nty);
  const int y1 = (int)(((long long)(ty + 1) * a.H) / a.nty);
  const int x0 = (int)(((long long)tx * a.W) / a.ntx);
  const int x1 = (int)(((long long)(tx + 1) * a.W) / a.ntx);
  const int TH = y1 - y0, TW = x1 - x0;
  const int EH = TH + 2 * M + 1, EW = TW + 2 * M + 1;
  const int K = a.K;

  for (int j = threadIdx.x; j < L; j += blockDim.x) om[j] = a.omega[j];
  for (int idx = threadIdx.x; idx < slot; idx += blockDim.x) {
    const int g = idx % G;
    const int e = idx / G;
    const int ex = e % a.EWmax, ey = e / a.EWmax;
    T v = T(0);
    if (g < K && ex < EW && ey < EH) {
      const int y = wrap_idx(y0 - M + ey, a.H), x = wrap_idx(x0 - M + ex, a.W);
      v = a.z[((size_t)y * a.W + x) * K + g];
    }
    zs[idx] = v;
    acc[idx] = T(0);
    if constexpr (DIAG) acc2[idx] = T(0);
  }
  __syncthreads();

  const int g = threadIdx.x % G, c = threadIdx.x / G;
  const bool colok = c < TW;
  const bool kok = colok && g < K;
  const int x = x0 + (colok ? c : 0);
  const int EWs = a.EWmax;

  T accW[E][E];
  constexpr int E2 = DIAG ? E : 1;
  T accW2[E2][E2];
#pragma unroll
  for (int r = 0; r < E; ++r)
#pragma unroll
    for (int s = 0; s < E; ++s) accW[r][s] = T(0);
#pragma unroll
  for (int r = 0; r < E2; ++r)
#pragma unroll
    for (int s = 0; s < E2; ++s) accW2[r][s] = T(0);
  T sq = T(0);
  const T tau = a.tau, mu = a.mu;

  for (int r = 0; r < TH; ++r) {
    const size_t pix = (size_t)(y0 + r) * a.W + x;
    // ---- loads: duals and p of this pixel / class
    V2 dv[L];
    const V2* d2p = reinterpret_cast<const V2*>(a.d2) + (pix * L) * K + g;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      if (kok) dv[j] = d2p[(size_t)j * K];
      else { dv[j].x = T(0); dv[j].y = T(0); }
    }
    T pk = T(0), d1 = T(0), d3 = T(0), d4 = T(0);
    if (kok) {
      pk = a.p[pix * K + g];
      const T* dl = a.dloc + pix * 3 * K + g;
      d1 = dl[0];
      d3 = dl[K];
      d4 = dl[2 * K];
    }
    // ---- v2 = J z - d2 (eq. 4), from the shared tile
    const T* zc = zs + ((r + M) * EWs + (c + M)) * G + g;
    T vh[L], vv[L];
#pragma unroll
    for (int dy = -M; dy <= M; ++dy)
#pragma unroll
      for (int dx = -M; dx <= M; ++dx) {
        const int j = (dy + M) * (2 * M + 1) + (dx + M);
        const T z00 = zc[(dy * EWs + dx) * G];
        const T z01 = zc[(dy * EWs + dx + 1) * G];
        const T z10 = zc[((dy + 1) * EWs + dx) * G];
        const T w = om[j];
        vh[j] = w * (z01 - z00) - dv[j].x;
        vv[j] = w * (z10 - z00) - dv[j].y;
      }
    // ---- Gram matrix (eq. 5) over the (j, k) rows of this pixel
    T ga = T(0), gb = T(0), gc = T(0);
#pragma unroll
    for (int j = 0; j < L; ++j) {
      ga += vh[j] * vh[j];
      gb += vh[j] * vv[j];
      gc += vv[j] * vv[j];
    }
    ga = group_sum<G>(ga);
    gb = group_sum<G>(gb);
    gc = group_sum<G>(gc);
    T A11, A12, A22;
    schatten_coeffs<T>(ga, gb, gc, tau, a.sp, A11, A12, A22);
    // ---- u2, d2 update, w = u2 + d2 and its J^T scatter into the window
    V2* d2w = reinterpret_cast<V2*>(a.d2) + (pix * L) * K + g;
#pragma unroll
    for (int dy = -M; dy <= M; ++dy)
#pragma unroll
      for (int dx = -M; dx <= M; ++dx) {
        const int j = (dy + M) * (2 * M + 1) + (dx + M);
        const T uh = vh[j] * A11 + vv[j] * A12;
        const T uv = vh[j] * A12 + vv[j] * A22;
        const T nh = uh - vh[j], nv = uv - vv[j];
        if constexpr (DIAG) {
          const T eh = nh - dv[j].x, ev = nv - dv[j].y;
          if (kok) sq += eh * eh + ev * ev;
        }
        if (kok) {
          V2 o; o.x = nh; o.y = nv;
          d2w[(size_t)j * K] = o;
        }
        const T w = om[j];
        const T wh = w * (uh + nh), wv = w * (uv + nv);
        accW[dy + M][dx + M + 1] += wh;
        accW[dy + M][dx + M] -= wh + wv;
        accW[dy + M + 1][dx + M] += wv;
        if constexpr (DIAG) {
          const T qh = w * nh, qv = w * nv;
          accW2[dy + M][dx + M + 1] += qh;
          accW2[dy + M][dx + M] -= qh + qv;
          accW2[dy + M + 1][dx + M] += qv;
        }
      }
    // ---- pixel-local MPOs of g1, g3, g4 and their duals
    const T z0 = zc[0];
    const T v1 = z0 - d1, v3 = z0 - d3, v4 = z0 - d4;
    const T pv = group_sum<G>(pk * v1);
    const T pp = group_sum<G>(pk * pk);
    const T s4 = group_sum<G>(kok ? v4 : T(0));
    const T q = T(4) * pp / mu;
    const T disc = sqrt(pv * pv + q);
    const T sroot = (pv >= T(0)) ? T(0.5) * (pv + disc) : (T(0.5) * q) / (disc - pv);
    const T u1 = v1 + pk / (mu * sroot);
    const T u3 = fmax(v3, T(0));
    const T u4 = v4 - (s4 - T(1)) * a.invK;
    const T n1 = u1 - v1, n3 = u3 - v3, n4 = u4 - v4;
    if (kok) {
      T* dl = a.dloc + pix * 3 * K + g;
      dl[0] = n1;
      dl[K] = n3;
      dl[2 * K] = n4;
      accW[M][M] += (u1 + n1) + (u3 + n3) + (u4 + n4);
      if constexpr (DIAG) {
        accW2[M][M] += n1 + n3 + n4;
        sq += (n1 - d1) * (n1 - d1) + (n3 - d3) * (n3 - d3) + (n4 - d4) * (n4 - d4);
      }
    }
    // ---- flush the finished top window row (tile row r + 0 - M + M = r in tile+halo rows)
    if (colok) {
      T* ar = acc + (r * EWs + c) * G + g;
#pragma unroll
      for (int s = 0; s < E; ++s) atomicAdd(ar + s * G, accW[0][s]);
      if constexpr (DIAG) {
        T* ar2 = acc2 + (r * EWs + c) * G + g;
#pragma unroll
        for (int s = 0; s < E; ++s) atomicAdd(ar2 + s * G, accW2[0][s]);
      }
    }
#pragma unroll
    for (int rr = 0; rr < E - 1; ++rr)
#pragma unroll
      for (int s = 0; s < E; ++s) accW[rr][s] = accW[rr + 1][s];
#pragma unroll
    for (int s = 0; s < E; ++s) accW[E - 1][s] = T(0);
    if constexpr (DIAG) {
#pragma unroll
      for (int rr = 0; rr < E - 1; ++rr)
#pragma unroll
        for (int s = 0; s < E; ++s) accW2[rr][s] = accW2[rr + 1][s];
#pragma unroll
      for (int s = 0; s < E; ++s) accW2[E - 1][s] = T(0);
    }
  }
  // remaining window rows: tile+halo rows TH .. TH + 2M
  if (colok) {
#pragma unroll
    for (int rr = 0; rr < E - 1; ++rr) {
      T* ar = acc + ((TH + rr) * EWs + c) * G + g;
#pragma unroll
      for (int s = 0; s < E; ++s) atomicAdd(ar + s * G, accW[rr][s]);
      if constexpr (DIAG) {
        T* ar2 = acc2 + ((TH + rr) * EWs + c) * G + g;
#pragma unroll
        for (int s = 0; s < E; ++s) atomicAdd(ar2 + s * G, accW2[rr][s]);
      }
    }
  }
  __syncthreads();
  // ---- write the tile (with halo) partial sums
  {
    T* Pt = a.P + (size_t)tile * a.EHmax * a.EWmax * K;
    T* Pt2 = DIAG ? a.P2 + (size_t)tile * a.EHmax * a.EWmax * K : nullptr;
    const int tot = EH * EW * K;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int k = idx % K;
      const int e = idx / K;
      const int ex = e % EW, ey = e / EW;
      const int so = (ey * EWs + ex);
      Pt[(size_t)so * K + k] = acc[so * G + k];
      if constexpr (DIAG) Pt2[(size_t)so * K + k] = acc2[so * G + k];
    }
  }
  if constexpr (DIAG) {
    const double t = block_sum_d((double)sq, red32);
    if (threadIdx.x == 0) a.diag_sq[tile] = t;
  }
}

template <typename T, int M, int G, bool DIAG>
inline cudaError_t launch_sweep_inst(const SweepArgs<T>& a, int tiles, size_t smem,
                                     cudaStream_t st) {
  auto kern = k_sweep<T, M, G, DIAG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<tiles, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int M, bool DIAG>
inline cudaError_t launch_sweep_g(const SweepArgs<T>& a, int G, int tiles, size_t smem,
                                  cudaStream_t st) {
  switch (G) {
    case 4: return launch_sweep_inst<T, M, 4, DIAG>(a, tiles, smem, st);
    case 8: return launch_sweep_inst<T, M, 8, DIAG>(a, tiles, smem, st);
    case 16: return launch_sweep_inst<T, M, 16, DIAG>(a, tiles, smem, st);
    case 32: return launch_sweep_inst<T, M, 32, DIAG>(a, tiles, smem, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool DIAG>
inline cudaError_t launch_sweep_md(const SweepArgs<T>& a, int M, int G, int tiles, size_t smem,
                                   cudaStream_t st) {
  switch (M) {
    case 0: return launch_sweep_g<T, 0, DIAG>(a, G, tiles, smem, st);
    case 1: return launch_sweep_g<T, 1, DIAG>(a, G, tiles, smem, st);
    case 2: return launch_sweep_g<T, 2, DIAG>(a, G, tiles, smem, st);
  }
  return cudaErrorInvalidValue;
}

// Shared memory of one sweep CTA in bytes.
template <typename T>
inline size_t sweep_smem_bytes(int EHmax, int EWmax, int G, int L, bool diag) {
  return sizeof(T) * ((size_t)(diag ? 3 : 2) * EHmax * EWmax * G + (size_t)L);
}

}  // namespace sgs
