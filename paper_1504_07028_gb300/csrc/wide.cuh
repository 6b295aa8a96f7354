// SALSA sweep (eqs. 12-14) for wide patches, (2M+1) x (2M+1) with M = 3, 4, 5 (the 7x7 to 11x11
// patches of Sec. 5's patch-size study). The fused sweep keeps a pixel's 2L Jacobian entries
// per class and its J^T scatter window in registers, which does not fit for L up to 121; here
// the same update is split into two launches that never hold more than one shift per thread:
//
//   k_wide_gram (one pixel per G lanes, class k on lane k, tiles of WG_TH rows):
//     pass 1 over the shifts: v2 = J z - d2, the Gram matrix [[a, b], [b, c]] = V^T V of
//     eq. (5) by a G-lane sum, and the Schatten-p prox coefficients u2 = V [[A11, A12],
//     [A12, A22]] (the closed form the fused sweep uses); pass 2 over the shifts: u2, the dual
//     update d2 <- u2 - v2 (in place: each entry is read and written by one thread) and
//     w = u2 + d2, stored for the transpose; then the pixel-local MPOs of g1, g3, g4 with their
//     duals and their part (u1 + d1) + (u3 + d3) + (u4 + d4) of the rhs.
//
//   k_wide_jt (one target pixel per G lanes): every target pixel m adds, shift by shift,
//       omega_j [w_h(m - s_j - e_h) - w_h(m - s_j) - w_v(m - s_j) + w_v(m - s_j - e_v)]
//     (J^T of eq. 12 as a gather, in a fixed order: deterministic); the w of neighbouring
//     targets overlap, so the repeated reads are served by L1. The result rhs = local part +
//     J^T w is dense; the z-update reads it directly.
//
// Traced variants also accumulate ||d^{k+1} - d^k||^2 per tile and write G^T d^{k+1}
// densely (dual residual).
#pragma once

#include "common.cuh"
#include "sweep.cuh"

namespace sgs {

constexpr int WG_TH = 1;   // rows of a gram tile (its columns: 256 / G)

template <typename T>
struct WideArgs {
  int H, W, K, M, L;
  const T* z;        // [n][K]
  const T* p;        // [n][K]
  T* dloc;           // [n][3][K]  (d1, d3, d4)
  T* d2;             // [n][L][K][2]
  T* wbuf;           // [n][L][K][2]: omega_j (u2 + d2) of the last sweep
  T* rhs;            // [n][K] dense rhs (local part from the gram kernel, completed by k_wide_jt)
  T* gtd;            // DIAG: [n][K] dense G^T d^{k+1}
  double* diag_sq;   // DIAG: per-tile sums of squared dual changes
  const T* omega;    // [L]
  T tau, mu, invK;
  int sp;
  int ntx1, ntiles1; // gram tiles: columns of tiles, count
  int nblk2;         // blocks of the transpose (grid-stride over pixels)
};

template <typename T>
__host__ __device__ inline size_t wide_gram_smem(int M, int G) {
  const int NC = 256 / G;
  return sizeof(T) * (size_t)(WG_TH + 2 * M + 1) * (NC + 2 * M + 1) * G;
}

template <typename T, int G, bool DIAG, bool SIMP>
__global__ void __launch_bounds__(256) k_wide_gram(const WideArgs<T> a) {
  constexpr int NC = 256 / G;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* zs = reinterpret_cast<T*>(smem_raw);
  __shared__ double red32[32];
  const int M = a.M, K = a.K, L = a.L;
  const int P = 2 * M + 1;
  const int EW = NC + 2 * M + 1, EH = WG_TH + 2 * M + 1;
  const int tile = blockIdx.x;
  const int y0 = (tile / a.ntx1) * WG_TH, x0 = (tile % a.ntx1) * NC;
  const int g = threadIdx.x % G, c = threadIdx.x / G;
  pdl_wait();
  // z tile with its halo (rows y0 - M .. y0 + WG_TH + M, periodic), classes on G lanes
  for (int idx = threadIdx.x; idx < EH * EW * G; idx += blockDim.x) {
    const int gg = idx % G, e = idx / G;
    const int ey = e / EW, ex = e - ey * EW;
    const bool v = gg < K;
    const int y = wrap_idx(y0 - M + ey, a.H), x = wrap_idx(x0 - M + ex, a.W);
    cp_async_zfill<sizeof(T)>(zs + idx, v ? a.z + ((size_t)y * a.W + x) * K + gg : a.z, v);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  const T tau = a.tau, mu = a.mu;
  T sq = T(0);
  const int x = x0 + c;
  const bool colok = x < a.W;
  const bool kok = colok && g < K;
  for (int r = 0; r < WG_TH; ++r) {
    const int y = y0 + r;
    if (y >= a.H) break;                                     // uniform over the block
    const size_t pix = (size_t)y * a.W + (colok ? x : 0);
    const T* zc = zs + ((r + M) * EW + (c + M)) * G + g;     // z at this pixel, class g
    using V2 = typename Vec2Of<T>::type;
    V2* d2p = reinterpret_cast<V2*>(a.d2) + pix * L * K + g;   // shift j at + j K
    V2* wp = reinterpret_cast<V2*>(a.wbuf) + pix * L * K + g;
    // pass 1: Gram matrix over the (j, k) rows of the pixel
    T ga = T(0), gb = T(0), gc = T(0);
    if (kok) {
#pragma unroll 8
      for (int j = 0; j < L; ++j) {
        const int jy = j / P;
        const T* zq = zc + ((jy - M) * EW + (j - jy * P - M)) * G;
        const T w = a.omega[j];
        const V2 dd = d2p[(size_t)j * K];
        const T vh = w * (zq[G] - zq[0]) - dd.x;
        const T vv = w * (zq[EW * G] - zq[0]) - dd.y;
        ga += vh * vh;
        gb += vh * vv;
        gc += vv * vv;
      }
    }
    ga = group_sum<G>(ga);
    gb = group_sum<G>(gb);
    gc = group_sum<G>(gc);
    T A11, A12, A22;
    schatten_coeffs<T>(ga, gb, gc, tau, a.sp, A11, A12, A22);
    // pass 2: u2 = V A, d2 <- u2 - v2, w = omega_j (u2 + d2)
    if (kok) {
#pragma unroll 8
      for (int j = 0; j < L; ++j) {
        const int jy = j / P;
        const T* zq = zc + ((jy - M) * EW + (j - jy * P - M)) * G;
        const T w = a.omega[j];
        const V2 od = d2p[(size_t)j * K];
        const T vh = w * (zq[G] - zq[0]) - od.x;
        const T vv = w * (zq[EW * G] - zq[0]) - od.y;
        const T uh = vh * A11 + vv * A12;
        const T uv = vh * A12 + vv * A22;
        V2 nd, wd;
        nd.x = uh - vh; nd.y = uv - vv;
        wd.x = w * (uh + nd.x); wd.y = w * (uv + nd.y);
        d2p[(size_t)j * K] = nd;
        wp[(size_t)j * K] = wd;
        if constexpr (DIAG)
          sq += (nd.x - od.x) * (nd.x - od.x) + (nd.y - od.y) * (nd.y - od.y);
      }
    }
    // pixel-local MPOs of g1, g3, g4 and their duals (as the fused sweep)
    T pk = T(0), d1 = T(0), d3 = T(0), d4 = T(0);
    if (kok) {
      pk = a.p[pix * K + g];
      const T* dl = a.dloc + pix * 3 * K + g;
      d1 = dl[0]; d3 = dl[K]; d4 = dl[2 * K];
    }
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
    T u4;
    if constexpr (!SIMP) {
      u4 = v4 - (s4 - T(1)) * a.invK;
    } else {
      (void)s4;
      bool act = kok;
      T theta = T(0);
      for (int pass = 0; pass < 32; ++pass) {
        const T cnt = group_sum<G>(act ? T(1) : T(0));
        const T sum = group_sum<G>(act ? v4 : T(0));
        theta = (cnt > T(0)) ? (sum - T(1)) / cnt : T(0);
        const bool nact = act && (v4 > theta);
        const bool changed = nact != act;
        act = nact;
        if (!__any_sync(0xffffffffu, changed)) break;
      }
      u4 = kok ? fmax(v4 - theta, T(0)) : T(0);
    }
    const T n1 = u1 - v1, n3 = u3 - v3, n4 = u4 - v4;
    if (kok) {
      T* dl = a.dloc + pix * 3 * K + g;
      dl[0] = n1; dl[K] = n3; dl[2 * K] = n4;
      a.rhs[pix * K + g] = (u1 + n1) + (u3 + n3) + (u4 + n4);
      if constexpr (DIAG) {
        a.gtd[pix * K + g] = n1 + n3 + n4;
        sq += (n1 - d1) * (n1 - d1) + (n3 - d3) * (n3 - d3) + (n4 - d4) * (n4 - d4);
      }
    }
  }
  pdl_trigger();
  if constexpr (DIAG) {
    const double t = block_sum_w<T>(sq, red32);
    if (threadIdx.x == 0) a.diag_sq[tile] = t;
  }
}

template <typename T, int G, bool DIAG>
__global__ void __launch_bounds__(256) k_wide_jt(const WideArgs<T> a) {
  using V2 = typename Vec2Of<T>::type;
  constexpr int PPB = 256 / G;
  const int K = a.K, M = a.M, P = 2 * M + 1, L = a.L;
  const int g = threadIdx.x % G;
  const V2* wv2 = reinterpret_cast<const V2*>(a.wbuf);
  const V2* dv2 = reinterpret_cast<const V2*>(a.d2);
  const int n = a.H * a.W;
  pdl_wait();  // w, d2 and the local rhs come from k_wide_gram
  for (int m0 = blockIdx.x * PPB; m0 < n; m0 += gridDim.x * PPB) {
    const int m = m0 + threadIdx.x / G;
    if (m >= n || g >= K) continue;   // no block-wide operations below
    const int my = m / a.W, mx = m - my * a.W;
    T acc = T(0), accd = T(0);
#pragma unroll 4
    for (int j = 0; j < L; ++j) {
      const int jy = j / P;
      const int dy = jy - M, dx = j - jy * P - M;
      // i0 = m - s_j, ih = i0 - e_h, iv = i0 - e_v (periodic; |s_j| <= M < H, W)
      int y0 = my - dy, x0 = mx - dx;
      y0 += (y0 < 0) ? a.H : 0;
      y0 -= (y0 >= a.H) ? a.H : 0;
      x0 += (x0 < 0) ? a.W : 0;
      x0 -= (x0 >= a.W) ? a.W : 0;
      const int xh = x0 == 0 ? a.W - 1 : x0 - 1, yv = y0 == 0 ? a.H - 1 : y0 - 1;
      const size_t o0 = (((size_t)y0 * a.W + x0) * L + j) * K + g;
      const size_t oh = (((size_t)y0 * a.W + xh) * L + j) * K + g;
      const size_t ov = (((size_t)yv * a.W + x0) * L + j) * K + g;
      const V2 w0 = wv2[o0];
      const T wh = a.wbuf[2 * oh], wv = a.wbuf[2 * ov + 1];
      acc += wh - w0.x - w0.y + wv;
      if constexpr (DIAG) {
        const T om = a.omega[j];
        const V2 d0 = dv2[o0];
        const T dh = a.d2[2 * oh], dv = a.d2[2 * ov + 1];
        accd += om * dh - om * d0.x - om * d0.y + om * dv;
      }
    }
    const size_t o = (size_t)m * K + g;
    a.rhs[o] += acc;
    if constexpr (DIAG) a.gtd[o] += accd;
  }
  pdl_trigger();
}

// Launch both kernels of one wide-patch sweep (defined in wide.cu for float and double).
template <typename T>
cudaError_t launch_wide(const WideArgs<T>& a, int G, bool diag, bool simplex, cudaStream_t st);
template <typename T>
cudaError_t prepare_wide(int M, int G);

}  // namespace sgs
