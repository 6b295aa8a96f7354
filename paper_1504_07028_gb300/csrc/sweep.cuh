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
// still touch in a (2M+2)x(2M+2) register window; every row step, the finished top window row
// goes through exclusive shared-memory slots, is summed in a fixed order by the owner of each
// column and stored as one row of the tile's partials P (tile plus halo). The row-FFT pass
// adds the overlapping tiles when it reads rhs (no atomics anywhere: deterministic).
#pragma once

#include "common.cuh"

namespace sgs {

template <typename T>
struct SweepArgs {
  int H, W, K;
  int NC;                // columns per tile (<= 256 / G)
  int ntx, nty;          // tile grid
  int EHmax, EWmax;      // extents of the P tile slots (tile + halo), in pixels
  const T* z;            // [n][K]
  const T* p;            // [n][K]
  T* dloc;               // [n][3][K]  (d1, d3, d4): full form of the local duals
  T* dcmp;               // [n][K + 2] (d3, c1, c4): compact form, d1 = c1 p, d4 = c4 1 (affine g4)
  int cin;               // affine g4: the local duals come in compact form (else full form);
                         // the affine sweep writes the compact form, the simplex sweep the full
  T* d2;                 // [n][L][K][2]
  T* P;                  // [tiles][EHmax][EWmax][K]  partial sums of G^T(u + d)
  T* P2;                 // DIAG: partial sums of G^T d (dual residual)
  double* diag_sq;       // DIAG: per tile sum of squared dual changes (primal residual)
  const T* omega;        // [L] shift weights
  T tau;                 // lambda / mu
  T mu;
  T invK;
  int sp;                // 1, 2, 0 = infinity
  int* err;              // set to 1 when a bounded wait gives up
  long long budget;      // clock cycles a bounded wait may take
  uint32_t probe;        // extra bytes armed on the first row's barrier (0; 16 in the wait test)
};

// Coefficients of u2 = V A for the prox of tau*||.||_{S_p} at V (R x 2) with Gram
// [[a, b], [b, c]] = V^T V. With V = U diag(s) W^T and shrunk values t, u2 = V W diag(g) W^T,
// g_i = t_i / s_i. Writing W diag(g) W^T = gbar I + kap [[hd, b], [b, -hd]], hd = (a - c)/2,
// kap = (g1 - g2) / (l1 - l2), the case formulas below have no cancellation at s1 = s2.
// The eigen-decomposition of the symmetric 2 x 2 Gram matrix is one Jacobi rotation; the
// closed form needs no rotation angle, and where both singular values are shrunk (or both
// kept) no division by the eigenvalue gap, so it stays accurate in FP32 when the two values
// coincide. Where exactly one is shrunk, kap = g1 / (2 r) is a bounded ratio whose two factors
// vanish together (g1 <= (s1 - s2) / s1).
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

// Byte sizes of one pipeline stage (one tile row of d2, dloc and p, each with 16 bytes of
// alignment slack at both ends), for tiles at most NC pixels wide.
__host__ __device__ inline size_t al16(size_t v) { return (v + 15) / 16 * 16; }
template <typename T>
__host__ __device__ inline void stage_sizes(int NC, int L, int K, size_t& d2b, size_t& dlb,
                                            size_t& pb) {
  d2b = al16((size_t)NC * 2 * L * K * sizeof(T) + 32);
  dlb = al16((size_t)NC * 3 * K * sizeof(T) + 32);
  pb = al16((size_t)NC * K * sizeof(T) + 32);
}

// Issue the bulk copies of one tile row (pixels [pix0, pix0 + TW)) into a stage.
// Each region starts at the 16-byte boundary at or below its first byte; returns nothing,
// the consumer recomputes the same offsets.
template <typename T>
__device__ __forceinline__ void issue_row(const SweepArgs<T>& a, size_t pix0, int TW, int L,
                                          unsigned char* st, size_t d2b, size_t dlb,
                                          uint64_t* bar, uint32_t extra = 0) {
  const int K = a.K;
  const int dls = a.cin ? K + 2 : 3 * K;   // local-dual values per pixel in the input form
  const char* g0 = reinterpret_cast<const char*>(a.d2) + pix0 * (2 * L * K * sizeof(T));
  const char* g1 = reinterpret_cast<const char*>(a.cin ? a.dcmp : a.dloc) + pix0 * (dls * sizeof(T));
  const char* g2 = reinterpret_cast<const char*>(a.p) + pix0 * (K * sizeof(T));
  const size_t n0 = (size_t)TW * 2 * L * K * sizeof(T);
  const size_t n1 = (size_t)TW * dls * sizeof(T);
  const size_t n2 = (size_t)TW * K * sizeof(T);
  const char* a0 = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(g0) & ~uintptr_t(15));
  const char* a1 = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(g1) & ~uintptr_t(15));
  const char* a2 = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(g2) & ~uintptr_t(15));
  const uint32_t b0 = (uint32_t)al16((g0 - a0) + n0);
  const uint32_t b1 = (uint32_t)al16((g1 - a1) + n1);
  const uint32_t b2 = (uint32_t)al16((g2 - a2) + n2);
  mbar_arrive_expect_tx(bar, b0 + b1 + b2 + extra);
  bulk_g2s(st, a0, b0, bar);
  bulk_g2s(st + d2b, a1, b1, bar);
  bulk_g2s(st + d2b + dlb, a2, b2, bar);
}

// Deterministic flush of one window row: every thread column c writes its E contributions
// to exclusive slots (columns c .. c+E-1 of the tile+halo row), the block synchronises, and
// the owner of each (column, class) sums the E slots in order s = 0..E-1 and stores the result
// straight into row `ey` of the tile's partials (each tile+halo row is flushed exactly once).
// Slots of idle columns stay zero; the caller synchronises before the slots are reused.
template <typename T, int G, int E, bool DIAG>
__device__ __forceinline__ void flush_row(const T (&w)[E], const T (&w2)[DIAG ? E : 1], bool colok,
                                          int c, int g, T* slots, T* slots2, T* Pt, T* Pt2,
                                          int ey, int EWmax, int EW, int K) {
  constexpr int SW = 256 / G + E - 1;
  if (colok) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      slots[(s * SW + c + s) * G + g] = w[s];
      if constexpr (DIAG) slots2[(s * SW + c + s) * G + g] = w2[s];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < EW * G; e += blockDim.x) {
    const int col = e / G, lane = e & (G - 1);
    if (lane >= K) continue;
    T sum = T(0), sum2 = T(0);
#pragma unroll
    for (int s = 0; s < E; ++s) {
      sum += slots[(s * SW + col) * G + lane];
      if constexpr (DIAG) sum2 += slots2[(s * SW + col) * G + lane];
    }
    const size_t o = ((size_t)ey * EWmax + col) * K + lane;
    Pt[o] = sum;
    if constexpr (DIAG) Pt2[o] = sum2;
  }
}

// Three CTAs per SM for the plain FP32 variant (80 registers, no spills); two otherwise.
template <typename T, int M, bool DIAG>
constexpr int sweep_min_blocks() { return (sizeof(T) == 8 || M >= 2 || DIAG) ? 2 : 3; }

// SIMP selects the MPO of g4: false, the projection onto the affine set 1^T xi = 1 (eq. 10);
// true, the projection onto the probability simplex (Sec. 4's description of that MPO).
// KEQ: the class count equals the lane count G, so the class strides are compile-time constants
// (measured 8 % fewer sweep cycles at 145 x 145, K = 16).
template <typename T, int M, int G, bool DIAG, bool SIMP, bool KEQ>
__global__ void __launch_bounds__(256, sweep_min_blocks<T, M, DIAG>()) k_sweep(const SweepArgs<T> a) {
  constexpr int L = (2 * M + 1) * (2 * M + 1);
  constexpr int E = 2 * M + 2;
  using V2 = typename Vec2Of<T>::type;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);  // 2 stage barriers
  size_t d2b, dlb, pb;
  stage_sizes<T>(a.NC, L, a.K, d2b, dlb, pb);
  const size_t stb = d2b + dlb + pb;
  unsigned char* stage0 = smem_raw + 128;
  const int slot = a.EHmax * a.EWmax * G;
  T* zs = reinterpret_cast<T*>(stage0 + 2 * stb);
  T* om = zs + slot;                    // [L]
  // flush slots: row contributions of thread column c for tile+halo column c + s live at
  // slots[(s * SW + c + s) * G + g]; each (s, column) has one writer, owners sum over s
  constexpr int SW = 256 / G + E - 1;   // columns of a slot row (NC <= 256 / G)
  T* slots = om + ((L + 3) & ~3);
  T* slots2 = slots + E * SW * G;       // only used when DIAG
  __shared__ double red32[32];

  const int tile = blockIdx.x;
  const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
  const int y0 = (int)(((long long)ty * a.H) / a.nty);
  const int y1 = (int)(((long long)(ty + 1) * a.H) / a.nty);
  const int x0 = (int)(((long long)tx * a.W) / a.ntx);
  const int x1 = (int)(((long long)(tx + 1) * a.W) / a.ntx);
  const int TH = y1 - y0, TW = x1 - x0;
  const int EH = TH + 2 * M + 1, EW = TW + 2 * M + 1;
  const int K = KEQ ? G : a.K;
  (void)EH;
  T* Pt = a.P + (size_t)tile * a.EHmax * a.EWmax * K;   // this tile's partials (tile + halo)
  T* Pt2 = DIAG ? a.P2 + (size_t)tile * a.EHmax * a.EWmax * K : nullptr;

  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  for (int j = threadIdx.x; j < L; j += blockDim.x) om[j] = a.omega[j];
  for (int j = threadIdx.x; j < (DIAG ? 2 : 1) * E * SW * G; j += blockDim.x) slots[j] = T(0);
  pdl_wait();  // z, d, p and the partial buffers belong to the previous kernels
  __syncthreads();
  if (threadIdx.x == 0) {
    issue_row<T>(a, (size_t)y0 * a.W + x0, TW, L, stage0, d2b, dlb, &mbar[0], a.probe);
    if (TH > 1) issue_row<T>(a, (size_t)(y0 + 1) * a.W + x0, TW, L, stage0 + stb, d2b, dlb, &mbar[1]);
  }
  // z tile (with halo, periodic) by per-thread async copies; padded classes read as zero
  {
    // element idx = (ey * EWmax + ex) * G + g; threads stride by 256 = (256 / G) pixels, so
    // (ex, ey) advance incrementally (no runtime division in the loop)
    constexpr int PS = 256 / G;
    const int g = threadIdx.x & (G - 1);
    int p = threadIdx.x / G;
    int ex = p % a.EWmax, ey = p / a.EWmax;
    for (int idx = threadIdx.x; idx < slot; idx += 256) {
      const bool v = g < K && ex < EW && ey < EH;
      const T* src = a.z;
      if (v) {
        int y = y0 - M + ey, xx = x0 - M + ex;
        y += (y < 0) ? a.H : 0;
        y -= (y >= a.H) ? a.H : 0;
        xx += (xx < 0) ? a.W : 0;
        xx -= (xx >= a.W) ? a.W : 0;
        src = a.z + ((size_t)y * a.W + xx) * K + g;
      }
      cp_async_zfill<sizeof(T)>(zs + idx, src, v);
      ex += PS;
      while (ex >= a.EWmax) { ex -= a.EWmax; ++ey; }
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  const int g = threadIdx.x % G, c = threadIdx.x / G;
  const bool colok = c < TW;
  const bool kok = colok && g < K;
  const int x = x0 + (colok ? c : 0);
  // KEQ instantiations run only with full-width tiles (NC = 256 / G), so their z-tile row
  // stride is a compile-time constant too
  const int EWs = KEQ ? 256 / G + 2 * M + 1 : a.EWmax;

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
  // shift weights in registers for the FP32 3 x 3 patch (the 5 x 5 and FP64 variants are at
  // their register caps)
  constexpr bool OMR = M <= 1 && sizeof(T) == 4;
  constexpr int LR = OMR ? L : 1;
  T omr[LR];
#pragma unroll
  for (int j = 0; j < LR; ++j) omr[j] = om[j];
  auto omega_j = [&](int j) -> T { return OMR ? omr[j < LR ? j : 0] : om[j]; };

  for (int r = 0; r < TH; ++r) {
    const int sidx = r & 1;
    const bool ok = mbar_wait_bounded(&mbar[sidx], (uint32_t)((r >> 1) & 1), a.budget);
    if (__syncthreads_or(!ok)) {
      // a copy never completed: report, give the other stage a bounded chance, and leave
      if (threadIdx.x == 0) {
        atomicExch(a.err, 1);
        if (r + 1 < TH) mbar_wait_bounded(&mbar[sidx ^ 1], (uint32_t)(((r + 1) >> 1) & 1), a.budget);
      }
      return;
    }
    // every thread is past row r-1: its stage can take row r+1
    if (threadIdx.x == 0 && r >= 1 && r + 1 < TH)
      issue_row<T>(a, (size_t)(y0 + r + 1) * a.W + x0, TW, L, stage0 + (sidx ^ 1) * stb, d2b,
                   dlb, &mbar[sidx ^ 1]);
    const size_t pix0 = (size_t)(y0 + r) * a.W + x0;
    const size_t pix = pix0 + (colok ? c : 0);
    unsigned char* st = stage0 + sidx * stb;
    // the consumer's view of the three regions (same 16-byte rounding as issue_row)
    const uintptr_t q0 = reinterpret_cast<uintptr_t>(a.d2) + pix0 * (2 * L * K * sizeof(T));
    const bool cin = !SIMP && a.cin;      // the simplex sweep always reads the full form
    const int dls = cin ? K + 2 : 3 * K;
    const uintptr_t q1 = reinterpret_cast<uintptr_t>(cin ? a.dcmp : a.dloc) + pix0 * (dls * sizeof(T));
    const uintptr_t q2 = reinterpret_cast<uintptr_t>(a.p) + pix0 * (K * sizeof(T));
    const V2* sd2 = reinterpret_cast<const V2*>(st + (q0 & 15)) + (size_t)c * L * K + g;
    const T* sdp = reinterpret_cast<const T*>(st + d2b + (q1 & 15)) + (size_t)c * dls;  // pixel
    const T* sp = reinterpret_cast<const T*>(st + d2b + dlb + (q2 & 15)) + (size_t)c * K + g;
    // ---- loads: duals and p of this pixel / class (from the staged row)
    V2 dv[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
      if (kok) dv[j] = sd2[j * K];
      else { dv[j].x = T(0); dv[j].y = T(0); }
    }
    T pk = T(0), d1 = T(0), d3 = T(0), d4 = T(0);
    if (kok) {
      pk = sp[0];
      if (cin) {            // d1 = c1 p, d4 = c4 1 (the forms the MPOs of g1 and g4 leave)
        d3 = sdp[g];
        d1 = sdp[K] * pk;
        d4 = sdp[K + 1];
      } else {
        d1 = sdp[g];
        d3 = sdp[K + g];
        d4 = sdp[2 * K + g];
      }
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
        const T w = omega_j(j);
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
        const T w = omega_j(j);
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
    // the new d1 is p / (mu sroot) = c1 p and, for the affine g4, the new d4 is the same
    // -(1^T v4 - 1) / K for every class: the compact form stores c1 and c4 per pixel
    const T c1n = T(1) / (mu * sroot);
    const T u1 = SIMP ? v1 + pk / (mu * sroot) : v1 + pk * c1n;
    const T u3 = fmax(v3, T(0));
    T u4;
    T c4n = T(0);
    if constexpr (!SIMP) {
      c4n = -(s4 - T(1)) * a.invK;
      u4 = v4 + c4n;
    } else {
      // Michelot: threshold over the active classes until no class leaves the active set (at
      // most K passes; the loop runs until no group of the warp changes, so that every lane
      // takes part in the shuffles)
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
    const T n1 = SIMP ? u1 - v1 : pk * c1n, n3 = u3 - v3, n4 = SIMP ? u4 - v4 : c4n;
    if constexpr (SIMP) {
      if (kok) {
        T* dl = a.dloc + pix * 3 * K + g;
        dl[0] = n1;
        dl[K] = n3;
        dl[2 * K] = n4;
      }
    } else {
      T* dc = a.dcmp + pix * (K + 2);
      if (kok) dc[g] = n3;
      if (kok && g == 0) {
        dc[K] = c1n;
        dc[K + 1] = c4n;
      }
    }
    if (kok) {
      accW[M][M] += (u1 + n1) + (u3 + n3) + (u4 + n4);
      if constexpr (DIAG) {
        accW2[M][M] += n1 + n3 + n4;
        sq += (n1 - d1) * (n1 - d1) + (n3 - d3) * (n3 - d3) + (n4 - d4) * (n4 - d4);
      }
    }
    // ---- flush the finished top window row (tile+halo row r), in a fixed summation order
    flush_row<T, G, E, DIAG>(accW[0], accW2[0], colok, c, g, slots, slots2, Pt, Pt2, r, EWs,
                             EW, K);
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
  pdl_trigger();
#pragma unroll
  for (int rr = 0; rr < E - 1; ++rr) {
    __syncthreads();  // the previous flush's owners are done with the slots
    flush_row<T, G, E, DIAG>(accW[rr], accW2[DIAG ? rr : 0], colok, c, g, slots, slots2, Pt, Pt2,
                             TH + rr, EWs, EW, K);
  }
  if constexpr (DIAG) {
    const double t = block_sum_w<T>(sq, red32);
    if (threadIdx.x == 0) a.diag_sq[tile] = t;
  }
}

// Largest dynamic shared memory granted so far to each sweep variant.
template <typename T, int M, int G, bool DIAG, bool SIMP, bool KEQ>
struct SweepGrant {
  static SmemGrants v;
};
template <typename T, int M, int G, bool DIAG, bool SIMP, bool KEQ>
SmemGrants SweepGrant<T, M, G, DIAG, SIMP, KEQ>::v;

template <typename T, int M, int G, bool DIAG, bool SIMP, bool KEQ>
inline cudaError_t grant_sweep(size_t smem) {
  return grant_smem(k_sweep<T, M, G, DIAG, SIMP, KEQ>, smem, SweepGrant<T, M, G, DIAG, SIMP, KEQ>::v);
}

template <typename T, int M, int G, bool DIAG, bool SIMP, bool KEQ>
inline cudaError_t launch_sweep_inst(const SweepArgs<T>& a, int tiles, size_t smem,
                                     cudaStream_t st) {
  cudaError_t e = grant_sweep<T, M, G, DIAG, SIMP, KEQ>(smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_sweep<T, M, G, DIAG, SIMP, KEQ>, dim3(tiles), dim3(256), smem, st, a);
}

template <typename T, int M, int G, bool SIMP, bool KEQ>
inline cudaError_t prepare_sweep_inst(size_t smem, size_t smem_diag) {
  cudaError_t e = grant_sweep<T, M, G, false, SIMP, KEQ>(smem);
  if (e != cudaSuccess) return e;
  return grant_sweep<T, M, G, true, SIMP, KEQ>(smem_diag);
}

template <typename T, int M, bool DIAG, bool SIMP, bool KEQ>
inline cudaError_t launch_sweep_g(const SweepArgs<T>& a, int G, int tiles, size_t smem,
                                  cudaStream_t st) {
  switch (G) {
    case 4: return launch_sweep_inst<T, M, 4, DIAG, SIMP, KEQ>(a, tiles, smem, st);
    case 8: return launch_sweep_inst<T, M, 8, DIAG, SIMP, KEQ>(a, tiles, smem, st);
    case 16: return launch_sweep_inst<T, M, 16, DIAG, SIMP, KEQ>(a, tiles, smem, st);
    case 32: return launch_sweep_inst<T, M, 32, DIAG, SIMP, KEQ>(a, tiles, smem, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool DIAG, bool SIMP, bool KEQ>
inline cudaError_t launch_sweep_md(const SweepArgs<T>& a, int M, int G, int tiles, size_t smem,
                                   cudaStream_t st) {
  switch (M) {
    case 0: return launch_sweep_g<T, 0, DIAG, SIMP, KEQ>(a, G, tiles, smem, st);
    case 1: return launch_sweep_g<T, 1, DIAG, SIMP, KEQ>(a, G, tiles, smem, st);
    case 2: return launch_sweep_g<T, 2, DIAG, SIMP, KEQ>(a, G, tiles, smem, st);
  }
  return cudaErrorInvalidValue;
}

// The instantiations of one precision and one g4 variant (each in its own translation unit).
template <typename T, bool SIMP, bool KEQ>
inline cudaError_t launch_sweep_variant(const SweepArgs<T>& a, int M, int G, bool diag,
                                        int tiles, size_t smem, cudaStream_t st) {
  return diag ? launch_sweep_md<T, true, SIMP, KEQ>(a, M, G, tiles, smem, st)
              : launch_sweep_md<T, false, SIMP, KEQ>(a, M, G, tiles, smem, st);
}
template <typename T, bool SIMP, bool KEQ>
inline cudaError_t prepare_sweep_variant(int M, int G, size_t smem, size_t smem_diag) {
#define SGS_PREP(MM, GG) \
  if (M == MM && G == GG) return prepare_sweep_inst<T, MM, GG, SIMP, KEQ>(smem, smem_diag);
  SGS_PREP(0, 4) SGS_PREP(0, 8) SGS_PREP(0, 16) SGS_PREP(0, 32)
  SGS_PREP(1, 4) SGS_PREP(1, 8) SGS_PREP(1, 16) SGS_PREP(1, 32)
  SGS_PREP(2, 4) SGS_PREP(2, 8) SGS_PREP(2, 16) SGS_PREP(2, 32)
#undef SGS_PREP
  return cudaErrorInvalidValue;
}

// Shared memory of one sweep CTA in bytes: barriers, two row stages, z tile, accumulator(s).
template <typename T>
inline size_t sweep_smem_bytes(int NC, int EHmax, int EWmax, int G, int L, int K, bool diag) {
  size_t d2b, dlb, pb;
  stage_sizes<T>(NC, L, K, d2b, dlb, pb);
  const int E = EWmax - NC;  // 2M + 1 ... the window width is E + 1 = 2M + 2
  const size_t slots = (size_t)(E + 1) * (256 / G + E) * G;
  return 128 + 2 * (d2b + dlb + pb) +
         sizeof(T) * ((size_t)EHmax * EWmax * G + (size_t)((L + 3) & ~3) +
                      (diag ? 2 : 1) * slots);
}

}  // namespace sgs
