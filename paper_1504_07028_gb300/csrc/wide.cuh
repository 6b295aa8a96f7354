// SALSA sweep (eqs. 12-14) for wide patches, (2M+1) x (2M+1) with M = 3, 4, 5 (the 7x7 to 11x11
// patches of Sec. 5's patch-size study). The fused sweep keeps a pixel's 2L Jacobian entries
// per class and its J^T scatter window in registers, which does not fit for L up to 121; here
// the same update is split into two launches that never hold more than one shift per thread.
//
// Stored form of the prior's dual. The MPO of g2 maps the pixel's block v (2L rows of K) to
// u = v A with the symmetric 2 x 2 matrix A of the Schatten-p closed form, and the dual becomes
// d2' = u - v = v (A - I). The wide sweep therefore stores V = v (the last prox argument, in the
// d2 buffer, [n][L][K][2]) and A per pixel ([n][4]: A11, A12, A22, unused) instead of d2 itself:
// d2 = V (A - I) entry by entry. (A = 2I stores d2 = V; V = 0 stores d2 = 0 for any A.)
//
//   k_wide_gram (one pixel per G lanes, class k on lane k, tiles of WG_TH rows): one pass over
//     the shifts reads V and the pixel's A, forms the dual d2 = V (A - I) and the new argument
//     v = omega_j grad z(m + s_j) - d2 (eq. 13's J z - d2), stores v over V in place (each entry
//     is read and written by one thread) and sums the Gram matrix [[a, b], [b, c]] = v^T v of
//     eq. (5) by a G-lane sum; then the new A, and the pixel-local MPOs of g1, g3, g4 with their
//     duals and their part (u1 + d1) + (u3 + d3) + (u4 + d4) of the rhs.
//
//   J^T of eq. 12 on w = omega_j (u + d2') = omega_j (v A + (v A - v)), recomputed from the
//   stored v and A: (J^T w)(m) = sum_j [w_h(m - s_j - e_h) - w_h(m - s_j)
//   + w_v(m - s_j - e_v) - w_v(m - s_j)] = S_h(m - e_h) - S_h(m) + S_v(m - e_v) - S_v(m) with
//   S(p) = sum_j w(p - s_j, j), the backward differences of one shifted sum per component:
//
//   k_wide_jt (one pixel per G lanes, over the gram tiles): S_h, S_v of every pixel, one v load
//     and the A of the source (from a shared-memory window of the tile's sources) per shift, in
//     a fixed order (deterministic); nothing but S is written, so the overlapping reads of v
//     by neighbouring pixels do not race.
//   k_wide_diff (one pixel and class per thread): rhs += S_h(m - e_h) - S_h(m) + S_v(m - e_v)
//     - S_v(m). The result rhs = local part + J^T w is dense; the z-update reads it directly.
//
// Traced variants also accumulate ||d^{k+1} - d^k||^2 per tile (the gram kernel keeps the old
// dual in a scratch buffer for a second pass) and write G^T d^{k+1} densely (dual residual).
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
  T* V;              // [n][L][K][2]: the prior's last prox argument v (d2 = V (A - I))
  T* coef;           // [n][4]: A11, A12, A22 of that prox
  T* scratch;        // [n][L][K][2]: DIAG, the old dual d2 of the traced sweep (gram kernel);
                     // then S = (S_h, S_v) [n][K][2] and, DIAG, the same sums of omega_j d2'
                     // (transpose)
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
  const int NC = 256 / G, L = (2 * M + 1) * (2 * M + 1);
  // the z tile with its halo, then per shift its z-tile offset and omega_j
  return sizeof(T) * (size_t)(WG_TH + 2 * M + 1) * (NC + 2 * M + 1) * G +
         (size_t)L * (sizeof(int) + sizeof(T));
}

// A of pixel `pix` (two 2-vectors: (A11, A12), (A22, unused)).
template <typename T>
__device__ __forceinline__ void load_coef(const T* coef, size_t pix, T& a11, T& a12, T& a22) {
  using V2 = typename Vec2Of<T>::type;
  const V2* c = reinterpret_cast<const V2*>(coef) + 2 * pix;
  const V2 c0 = c[0], c1 = c[1];
  a11 = c0.x; a12 = c0.y; a22 = c1.x;
}

// The two components of u = v A in one fixed evaluation order (explicit fma), so that every
// kernel that forms u or the dual u - v from the stored (V, A) gets the same bits.
template <typename T>
__device__ __forceinline__ T prox_h(T vx, T vy, T a11, T a12) { return fma(vy, a12, vx * a11); }
template <typename T>
__device__ __forceinline__ T prox_v(T vx, T vy, T a12, T a22) { return fma(vy, a22, vx * a12); }

template <typename T, int G, bool DIAG, bool SIMP>
__global__ void __launch_bounds__(256) k_wide_gram(const WideArgs<T> a) {
  constexpr int NC = 256 / G;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* zs = reinterpret_cast<T*>(smem_raw);
  __shared__ double red32[32];
  const int M = a.M, K = a.K, L = a.L;
  const int P = 2 * M + 1;
  const int EW = NC + 2 * M + 1, EH = WG_TH + 2 * M + 1;
  T* om = zs + (size_t)EH * EW * G;                   // [L] omega_j
  int* zoff = reinterpret_cast<int*>(om + L);         // [L] z-tile offset of shift j
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    const int jy = j / P;
    zoff[j] = ((jy - M) * EW + (j - jy * P - M)) * G;
    om[j] = a.omega[j];
  }
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
    V2* vp = reinterpret_cast<V2*>(a.V) + pix * L * K + g;   // shift j at + j K
    V2* ep = reinterpret_cast<V2*>(a.scratch) + pix * L * K + g;
    T o11 = T(0), o12 = T(0), o22 = T(0);
    if (colok) load_coef(a.coef, pix, o11, o12, o22);
    // the dual of the last sweep, the new argument v (stored over V) and the Gram matrix
    T ga = T(0), gb = T(0), gc = T(0);
    if (kok) {
      constexpr int UB = 8;   // shifts whose V loads are issued together
      for (int j0 = 0; j0 < L; j0 += UB) {
        V2 vb[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u)
          if (j0 + u < L) vb[u] = vp[(size_t)(j0 + u) * K];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = j0 + u;
        if (j >= L) break;
        const T* zq = zc + zoff[j];
        const T w = om[j];
        const V2 vo = vb[u];
        V2 dd;
        dd.x = prox_h(vo.x, vo.y, o11, o12) - vo.x;
        dd.y = prox_v(vo.x, vo.y, o12, o22) - vo.y;
        V2 v;
        v.x = w * (zq[G] - zq[0]) - dd.x;
        v.y = w * (zq[EW * G] - zq[0]) - dd.y;
        vp[(size_t)j * K] = v;
        if constexpr (DIAG) ep[(size_t)j * K] = dd;
        ga += v.x * v.x;
        gb += v.x * v.y;
        gc += v.y * v.y;
      }
      }
    }
    ga = group_sum<G>(ga);
    gb = group_sum<G>(gb);
    gc = group_sum<G>(gc);
    T A11, A12, A22;
    schatten_coeffs<T>(ga, gb, gc, tau, a.sp, A11, A12, A22);
    if (colok && g == 0) {
      using V2c = typename Vec2Of<T>::type;
      V2c* cp = reinterpret_cast<V2c*>(a.coef) + 2 * pix;
      V2c c0, c1;
      c0.x = A11; c0.y = A12; c1.x = A22; c1.y = T(0);
      cp[0] = c0;
      cp[1] = c1;
    }
    if constexpr (DIAG) {
      // ||d2' - d2||^2 with d2' = v (A - I): v and the old dual read back (this thread's writes)
      if (kok) {
        for (int j = 0; j < L; ++j) {
          const V2 v = vp[(size_t)j * K], od = ep[(size_t)j * K];
          const T nx = prox_h(v.x, v.y, A11, A12) - v.x;
          const T ny = prox_v(v.x, v.y, A12, A22) - v.y;
          sq += (nx - od.x) * (nx - od.x) + (ny - od.y) * (ny - od.y);
        }
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

// Shared memory of k_wide_jt: the A of a tile's source window ((2M + 2) rows x (NC + 2M + 1)
// columns, four values each), then per shift its V offset for interior targets (8 bytes),
// omega_j, (dy, dx) and its window entry (4-byte values last: L is odd).
template <typename T>
__host__ __device__ inline size_t wide_jt_smem(int M, int G) {
  const int NC = 256 / G, L = (2 * M + 1) * (2 * M + 1);
  const size_t win = (size_t)(2 * M + 2) * (NC + 2 * M + 1) * 4 * sizeof(T);
  return win + (size_t)L * (sizeof(long long) + 3 * sizeof(int) + sizeof(T));
}

// The four stored values of one window entry (A11, A12, A22, unused) in one shared load.
template <typename T> struct Coef4;
template <> struct Coef4<float> {
  float a11, a12, a22, pad;
  __device__ static Coef4 at(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
  }
};
template <> struct Coef4<double> {
  double a11, a12, a22, pad;
  __device__ static Coef4 at(const double* p) {
    const double2 v = reinterpret_cast<const double2*>(p)[0], w = reinterpret_cast<const double2*>(p)[1];
    return {v.x, v.y, w.x, w.y};
  }
};

template <typename T, int G, bool DIAG>
__global__ void __launch_bounds__(256) k_wide_jt(const WideArgs<T> a) {
  using V2 = typename Vec2Of<T>::type;
  constexpr int NC = 256 / G;
  constexpr int UJ = 8;   // shifts whose v loads are issued together
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int K = a.K, M = a.M, P = 2 * M + 1, L = a.L;
  const int EWc = NC + 2 * M + 1, EHc = 2 * M + 2;
  T* cw = reinterpret_cast<T*>(smem_raw);                                   // [EHc][EWc][4]
  long long* offv = reinterpret_cast<long long*>(cw + (size_t)EHc * EWc * 4);  // [L]
  T* om = reinterpret_cast<T*>(offv + L);                                     // [L]
  int* dyx = reinterpret_cast<int*>(om + L);                                  // [L][2]
  int* woff = dyx + 2 * L;                                                    // [L]
  const int g = threadIdx.x % G, c = threadIdx.x / G;
  const V2* vv2 = reinterpret_cast<const V2*>(a.V);
  V2* S = reinterpret_cast<V2*>(a.scratch);                                   // [n][K]
  const size_t nK = (size_t)a.H * a.W * K;
  const long long LK = (long long)L * K;
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    const int jy = j / P, dy = jy - M, dx = j - jy * P - M;
    dyx[2 * j] = dy;
    dyx[2 * j + 1] = dx;
    offv[j] = (-(long long)dy * a.W - dx) * LK + (long long)j * K;   // V2 units, m - s_j
    woff[j] = 4 * ((M + 1 - dy) * EWc + (M + 1 - dx));   // window entry of m - s_j (column 0)
    om[j] = a.omega[j];
  }
  pdl_wait();  // v, A and the local rhs come from k_wide_gram
  for (int tile = blockIdx.x; tile < a.ntiles1; tile += gridDim.x) {
    const int y = tile / a.ntx1, x0 = (tile % a.ntx1) * NC;
    __syncthreads();  // the previous tile's window is no longer read
    // A of the sources m - s_j of the tile's pixels (periodic)
    for (int idx = threadIdx.x; idx < EHc * EWc; idx += blockDim.x) {
      const int ry = idx / EWc, rx = idx - ry * EWc;
      const int py = wrap_idx(y - M - 1 + ry, a.H), px = wrap_idx(x0 - M - 1 + rx, a.W);
      T a11, a12, a22;
      load_coef(a.coef, (size_t)py * a.W + px, a11, a12, a22);
      cw[4 * idx] = a11;
      cw[4 * idx + 1] = a12;
      cw[4 * idx + 2] = a22;
    }
    __syncthreads();
    const int x = x0 + c;
    if (x >= a.W || g >= K) continue;   // no block-wide operation before the next tile's
    const long long m = (long long)y * a.W + x;
    const bool inner = y >= M && y <= a.H - 1 - M && x >= M && x <= a.W - 1 - M;
    T sh = T(0), sv = T(0), dh = T(0), dv = T(0);
    for (int j0 = 0; j0 < L; j0 += UJ) {
      V2 v0[UJ];
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int j = j0 + u;
        if (j >= L) break;
        long long o0;
        if (inner) {
          o0 = m * LK + offv[j] + g;
        } else {
          int ys = y - dyx[2 * j], xs = x - dyx[2 * j + 1];   // m - s_j, periodic
          ys += (ys < 0) ? a.H : 0;
          ys -= (ys >= a.H) ? a.H : 0;
          xs += (xs < 0) ? a.W : 0;
          xs -= (xs >= a.W) ? a.W : 0;
          o0 = (((long long)ys * a.W + xs) * L + j) * K + g;
        }
        v0[u] = vv2[o0];
      }
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int j = j0 + u;
        if (j >= L) break;
        const Coef4<T> c0 = Coef4<T>::at(cw + woff[j] + 4 * c);
        const T ux = prox_h(v0[u].x, v0[u].y, c0.a11, c0.a12);
        const T uy = prox_v(v0[u].x, v0[u].y, c0.a12, c0.a22);
        const T nx = ux - v0[u].x, ny = uy - v0[u].y;
        const T o = om[j];
        sh += o * (ux + nx);
        sv += o * (uy + ny);
        if constexpr (DIAG) {
          dh += o * nx;
          dv += o * ny;
        }
      }
    }
    const size_t oo = (size_t)m * K + g;
    V2 r;
    r.x = sh; r.y = sv;
    S[oo] = r;
    if constexpr (DIAG) {
      r.x = dh; r.y = dv;
      S[nK + oo] = r;
    }
  }
  pdl_trigger();
}

// rhs(m) += S_h(m - e_h) - S_h(m) + S_v(m - e_v) - S_v(m) (and the same for G^T d2' into gtd).
template <typename T, bool DIAG>
__global__ void __launch_bounds__(256) k_wide_diff(const WideArgs<T> a) {
  using V2 = typename Vec2Of<T>::type;
  const V2* S = reinterpret_cast<const V2*>(a.scratch);
  const int K = a.K;
  const size_t nK = (size_t)a.H * a.W * K;
  pdl_wait();  // S comes from k_wide_jt
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nK;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t pix = i / K;
    const int k = (int)(i - pix * K);
    const int y = (int)(pix / a.W), x = (int)(pix - (size_t)y * a.W);
    const size_t ih = ((size_t)y * a.W + (x == 0 ? a.W - 1 : x - 1)) * K + k;
    const size_t iv = ((size_t)(y == 0 ? a.H - 1 : y - 1) * a.W + x) * K + k;
    const V2 s0 = S[i], shv = S[ih], svv = S[iv];
    a.rhs[i] += (shv.x - s0.x) + (svv.y - s0.y);
    if constexpr (DIAG) {
      const V2 d0 = S[nK + i], dhv = S[nK + ih], dvv = S[nK + iv];
      a.gtd[i] += (dhv.x - d0.x) + (dvv.y - d0.y);
    }
  }
  pdl_trigger();
}

// d2 = V (A - I) written out densely ([n][L][K][2]; checkpoint read-out).
template <typename T>
__global__ void k_wide_dual(const T* __restrict__ V, const T* __restrict__ coef, T* __restrict__ d2,
                            int n, int LK) {
  const size_t tot = (size_t)n * LK;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    T a11, a12, a22;
    load_coef(coef, i / LK, a11, a12, a22);
    const T vx = V[2 * i], vy = V[2 * i + 1];
    d2[2 * i] = prox_h(vx, vy, a11, a12) - vx;
    d2[2 * i + 1] = prox_v(vx, vy, a12, a22) - vy;
  }
}

// A = 2 I for every pixel, so that V holds d2 itself (checkpoint load).
template <typename T>
__global__ void k_wide_coef_identity(T* coef, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    coef[4 * (size_t)i] = T(2);
    coef[4 * (size_t)i + 1] = T(0);
    coef[4 * (size_t)i + 2] = T(2);
    coef[4 * (size_t)i + 3] = T(0);
  }
}

// Launch both kernels of one wide-patch sweep (defined in wide.cu for float and double).
template <typename T>
cudaError_t launch_wide(const WideArgs<T>& a, int G, bool diag, bool simplex, cudaStream_t st);
template <typename T>
cudaError_t prepare_wide(int M, int G);
// Dense d2 from the stored form (V, A), and the stored form of a given d2 (A = 2I).
template <typename T>
cudaError_t launch_wide_dual(const T* V, const T* coef, T* d2, int n, int LK, cudaStream_t st);
template <typename T>
cudaError_t launch_wide_coef_identity(T* coef, int n, cudaStream_t st);

}  // namespace sgs
