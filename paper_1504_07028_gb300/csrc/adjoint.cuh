// Reverse pass of the unrolled SALSA iteration (12)-(14): the differentiable solver.
//
// The forward step k maps (w^k, d^k) to (w^{k+1}, d^{k+1}) with w = u + d:
//     z^{k+1} = A^{-1} G^T w^k,  A = G^T G = 3 I + J^T J            (eq. 12)
//     v = G z^{k+1} - d^k,  u^{k+1} = MPOs of g1..g4 at v            (eq. 13)
//     d^{k+1} = u^{k+1} - v,  w^{k+1} = 2 u^{k+1} - v                (eq. 14)
// and the output is z^T. Its adjoint runs backwards one unit per step: given zbar^{k+1},
//     bbar = A^{-1} zbar^{k+1}                       (A is symmetric: the z-update itself)
//     wbar^k = G bbar,  dbar^k = -vbar^{k+1}
//     ubar = 2 wbar^k + dbar^k,  vbar^k = -wbar^k - dbar^k + (dMPO/dv)^T ubar
//     zbar^k = G^T vbar^k
// with the parameter gradients collected on the way: log p through the MPO of g1 (and through
// z^0 = p / 1^T p at the end), lambda through the Schatten prox (tau = lambda / mu), and the
// shift weights omega through J in v = J z - d2, in b = G^T w and in A.
//
// k_adj_vjp does everything of one unit that is local to a pixel (the stencils J z^k and
// J bbar are read from the neighbours in global memory), k_adj_gt applies G^T, and the
// z-update kernels apply A^{-1}. The Schatten prox derivative is taken by forward-mode dual
// numbers through the same closed form the sweep evaluates (schatten_coeffs): the Jacobian of
// (A11, A12, A22) with respect to (a, b, c, tau) comes out of one evaluation.
#pragma once

#include "sweep.cuh"

namespace sgs {

// Value and four tangents (d/da, d/db, d/dc, d/dtau). Kept in a namespace of its own: its
// sqrt / fmax are found by argument-dependent lookup and hide nothing for plain numbers.
namespace dual {
template <typename T>
struct Dual4 {
  T v;
  T d[4];
  __device__ Dual4() : v(T(0)) { d[0] = d[1] = d[2] = d[3] = T(0); }
  __device__ Dual4(double x) : v(T(x)) { d[0] = d[1] = d[2] = d[3] = T(0); }
};
template <typename T> __device__ __forceinline__ Dual4<T> operator+(Dual4<T> x, Dual4<T> y) {
  Dual4<T> r; r.v = x.v + y.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = x.d[i] + y.d[i];
  return r;
}
template <typename T> __device__ __forceinline__ Dual4<T> operator-(Dual4<T> x, Dual4<T> y) {
  Dual4<T> r; r.v = x.v - y.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = x.d[i] - y.d[i];
  return r;
}
template <typename T> __device__ __forceinline__ Dual4<T> operator-(Dual4<T> x) {
  Dual4<T> r; r.v = -x.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = -x.d[i];
  return r;
}
template <typename T> __device__ __forceinline__ Dual4<T> operator*(Dual4<T> x, Dual4<T> y) {
  Dual4<T> r; r.v = x.v * y.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = x.d[i] * y.v + x.v * y.d[i];
  return r;
}
template <typename T> __device__ __forceinline__ Dual4<T> operator/(Dual4<T> x, Dual4<T> y) {
  Dual4<T> r; r.v = x.v / y.v;
  const T iy = T(1) / y.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = (x.d[i] - r.v * y.d[i]) * iy;
  return r;
}
template <typename T> __device__ __forceinline__ bool operator>(Dual4<T> x, Dual4<T> y) { return x.v > y.v; }
template <typename T> __device__ __forceinline__ bool operator>=(Dual4<T> x, Dual4<T> y) { return x.v >= y.v; }
template <typename T> __device__ __forceinline__ Dual4<T> sqrt(Dual4<T> x) {
  Dual4<T> r; r.v = ::sqrt(x.v);
  const T h = r.v > T(0) ? T(0.5) / r.v : T(0);   // a clamped zero carries no tangent
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = x.d[i] * h;
  return r;
}
template <typename T> __device__ __forceinline__ Dual4<T> fmax(Dual4<T> x, Dual4<T> y) {
  return x.v >= y.v ? x : y;
}
}  // namespace dual
using dual::Dual4;

struct AdjShape {
  int H, W, K, n;
};

// Inputs and outputs of one reverse unit (pixel-major layouts of the forward state).
template <typename T>
struct AdjArgs {
  AdjShape s;
  const T* zk;        // z^k            [n][K]
  const T* zk1;       // z^{k+1}        [n][K]
  const T* p;         // [n][K]
  const T* dloc;      // d^{k-1}: d1, d3, d4  [n][3][K]
  const T* d2;        // d^{k-1}: d2     [n][L][K][2]
  const T* bbar;      // A^{-1} zbar^{k+1}  [n][K]
  const T* vn_loc;    // vbar^{k+1} local blocks [n][3][K], or nullptr (zero)
  const T* vn_2;      // vbar^{k+1} d2 block [n][L][K][2], or nullptr
  T* v_loc;           // out: vbar^k [n][3][K]
  T* v_2;             // out: vbar^k [n][L][K][2]
  T* glogp;           // accumulated d/dlog p [n][K]
  double* part;       // block partials [NP][blocks]: tau, omega_0..omega_{L-1}, S (= <D bbar, D z^{k+1}>)
  const T* omega;
  T tau, mu, invK;
  int sp;
  int simplex;        // g4 on the probability simplex (else on the affine set 1^T xi = 1)
};

constexpr int ADJ_THREADS = 256;

// The (h, v) pair of one class in the [..][K][2] layouts, moved as one 8- or 16-byte access.
template <typename T> struct Pair2;
template <> struct Pair2<float> { using t = float2; };
template <> struct Pair2<double> { using t = double2; };
template <typename T>
__device__ __forceinline__ typename Pair2<T>::t ld_pair(const T* q) {
  return __ldg(reinterpret_cast<const typename Pair2<T>::t*>(q));
}
template <typename T>
__device__ __forceinline__ void st_pair(T* q, T h, T v) {
  typename Pair2<T>::t o;
  o.x = h;
  o.y = v;
  *reinterpret_cast<typename Pair2<T>::t*>(q) = o;
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <typename T, int M, int G>
__global__ void __launch_bounds__(ADJ_THREADS, 2) k_adj_vjp(const AdjArgs<T> a) {
  constexpr int L = (2 * M + 1) * (2 * M + 1);
  constexpr int E = 2 * M + 2;
  constexpr int NP = L + 2;
  constexpr int NWARP = ADJ_THREADS / 32;
  __shared__ double red[NWARP][NP];
  const int H = a.s.H, W = a.s.W, K = a.s.K;
  const int g = threadIdx.x & (G - 1);
  const int pix = blockIdx.x * (ADJ_THREADS / G) + threadIdx.x / G;
  const bool pok = pix < a.s.n;
  const bool kok = pok && g < K;
  const int y = pok ? pix / W : 0, x = pok ? pix - y * W : 0;
  // stencil windows of z^k and bbar over rows y-M .. y+M+1, columns x-M .. x+M+1
  T zw[E][E], bw[E][E];
#pragma unroll
  for (int r = 0; r < E; ++r)
#pragma unroll
    for (int c = 0; c < E; ++c) {
      const size_t q = ((size_t)wrapi(y - M + r, H) * W + wrapi(x - M + c, W)) * K + g;
      zw[r][c] = kok ? a.zk[q] : T(0);
      bw[r][c] = kok ? a.bbar[q] : T(0);
    }
  const size_t e = (size_t)pix * K + g;
  const T pk = kok ? a.p[e] : T(0);
  const size_t el = (size_t)pix * 3 * K + g;
  const T d1 = kok ? a.dloc[el] : T(0), d3 = kok ? a.dloc[el + K] : T(0),
          d4 = kok ? a.dloc[el + 2 * K] : T(0);
  const T zc = zw[M][M], bc = bw[M][M];
  // ---- forward MPOs at v = G z^k - d^{k-1}
  const T v1 = zc - d1, v3 = zc - d3, v4 = zc - d4;
  T vh[L], vv[L];
  const size_t e2 = (size_t)pix * L * K * 2 + 2 * g;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int dy = j / (2 * M + 1), dx = j % (2 * M + 1);
    const T w = a.omega[j];
    T dh = T(0), dv = T(0);
    if (kok) {
      const auto q = ld_pair(a.d2 + e2 + (size_t)j * K * 2);
      dh = q.x;
      dv = q.y;
    }
    vh[j] = w * (zw[dy][dx + 1] - zw[dy][dx]) - dh;
    vv[j] = w * (zw[dy + 1][dx] - zw[dy][dx]) - dv;
  }
  const T pv = group_sum<G>(pk * v1), pp = group_sum<G>(pk * pk);
  const T qq = T(4) * pp / a.mu;
  const T disc = sqrt(pv * pv + qq);
  const T t = (pv >= T(0)) ? T(0.5) * (pv + disc) : (T(0.5) * qq) / (disc - pv);
  T ga = T(0), gb = T(0), gc = T(0);
#pragma unroll
  for (int j = 0; j < L; ++j) { ga += vh[j] * vh[j]; gb += vh[j] * vv[j]; gc += vv[j] * vv[j]; }
  ga = group_sum<G>(ga); gb = group_sum<G>(gb); gc = group_sum<G>(gc);
  Dual4<T> Da(0.0), Db(0.0), Dc(0.0), Dt(0.0);
  Da.v = ga; Da.d[0] = T(1);
  Db.v = gb; Db.d[1] = T(1);
  Dc.v = gc; Dc.d[2] = T(1);
  Dt.v = a.tau; Dt.d[3] = T(1);
  Dual4<T> A11, A12, A22;
  schatten_coeffs<Dual4<T>>(Da, Db, Dc, Dt, a.sp, A11, A12, A22);
  const T s4 = group_sum<G>(kok ? v4 : T(0));
  // ---- adjoints of the outputs: wbar^k = G bbar, dbar^k = -vbar^{k+1}
  const T nd1 = a.vn_loc && kok ? a.vn_loc[el] : T(0);
  const T nd3 = a.vn_loc && kok ? a.vn_loc[el + K] : T(0);
  const T nd4 = a.vn_loc && kok ? a.vn_loc[el + 2 * K] : T(0);
  // block 1 (data term): ubar1 = 2 bbar - vbar1^{k+1}
  const T ub1 = T(2) * bc - nd1;
  const T su = group_sum<G>(kok ? ub1 * pk : T(0));
  const T vb1 = -bc + nd1 + (ub1 - su * pk / (a.mu * t * disc));
  if (kok) {
    const T dtdp = (a.mu * v1 * t + T(2) * pk) / (a.mu * disc);
    const T pbar = ub1 / (a.mu * t) - su / (a.mu * t * t) * dtdp;
    a.glogp[e] += pk * pbar;
  }
  // block 3 (positive orthant) and block 4 (affine set, or the probability simplex)
  const T ub3 = T(2) * bc - nd3;
  const T vb3 = -bc + nd3 + ((v3 > T(0)) ? ub3 : T(0));
  const T ub4 = T(2) * bc - nd4;
  T vb4;
  if (!a.simplex) {
    const T sub4 = group_sum<G>(kok ? ub4 : T(0));
    vb4 = -bc + nd4 + (ub4 - sub4 * a.invK);
  } else {
    // the projection max(v4 - theta, 0) moves the active classes S = {v4 > theta} by a
    // common shift: its Jacobian is I - 1 1^T / |S| on S and 0 elsewhere. The active set by
    // the sweep's fixed-point search (Michelot), in the same arithmetic.
    bool act = kok;
    for (int pass = 0; pass < 32; ++pass) {
      const T cnt = group_sum<G>(act ? T(1) : T(0));
      const T sum = group_sum<G>(act ? v4 : T(0));
      const T theta = (cnt > T(0)) ? (sum - T(1)) / cnt : T(0);
      const bool nact = act && (v4 > theta);
      const bool changed = nact != act;
      act = nact;
      if (!__any_sync(0xffffffffu, changed)) break;
    }
    const T cnt = group_sum<G>(act ? T(1) : T(0));
    const T sub4 = group_sum<G>(act ? ub4 : T(0));
    vb4 = -bc + nd4 + (act ? ub4 - sub4 / cnt : T(0));
  }
  (void)s4;
  // block 2 (Schatten prox): ubar2 = 2 J bbar - vbar2^{k+1}
  T jbh[L], jbv[L];
  T Ab11 = T(0), Ab12 = T(0), Ab22 = T(0);
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int dy = j / (2 * M + 1), dx = j % (2 * M + 1);
    const T w = a.omega[j];
    jbh[j] = bw[dy][dx + 1] - bw[dy][dx];             // unweighted S_j D bbar
    jbv[j] = bw[dy + 1][dx] - bw[dy][dx];
    T nh = T(0), nv = T(0);
    if (a.vn_2 && kok) {
      const auto q = ld_pair(a.vn_2 + e2 + (size_t)j * K * 2);
      nh = q.x;
      nv = q.y;
    }
    const T ubh = T(2) * w * jbh[j] - nh, ubv = T(2) * w * jbv[j] - nv;
    Ab11 += ubh * vh[j];
    Ab12 += ubh * vv[j] + ubv * vh[j];
    Ab22 += ubv * vv[j];
  }
  Ab11 = group_sum<G>(Ab11); Ab12 = group_sum<G>(Ab12); Ab22 = group_sum<G>(Ab22);
  T gbar4[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) gbar4[m] = Ab11 * A11.d[m] + Ab12 * A12.d[m] + Ab22 * A22.d[m];
  // per-thread terms of the parameter gradients, in the working precision (FP64 only from the
  // warp sums on: FP64 arithmetic is scarce on this part)
  T om_loc[L];
  T s_loc = T(0);
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int dy = j / (2 * M + 1), dx = j % (2 * M + 1);
    const T w = a.omega[j];
    T nh = T(0), nv = T(0);
    if (a.vn_2 && kok) {
      const auto q = ld_pair(a.vn_2 + e2 + (size_t)j * K * 2);
      nh = q.x;
      nv = q.y;
    }
    const T ubh = T(2) * w * jbh[j] - nh, ubv = T(2) * w * jbv[j] - nv;   // as in the loop above
    const T Vh = ubh * A11.v + ubv * A12.v + T(2) * gbar4[0] * vh[j] + gbar4[1] * vv[j];
    const T Vv = ubh * A12.v + ubv * A22.v + gbar4[1] * vh[j] + T(2) * gbar4[2] * vv[j];
    const T vbh = -w * jbh[j] + nh + Vh;
    const T vbv = -w * jbv[j] + nv + Vv;
    if (kok) st_pair(a.v_2 + e2 + (size_t)j * K * 2, vbh, vbv);
    // omega_j: v2 = omega_j S_j D z^k - d2 (first term); b = G^T w with w2 = 2 u2 - v2 (second)
    const T zdh = zw[dy][dx + 1] - zw[dy][dx], zdv = zw[dy + 1][dx] - zw[dy][dx];
    const T u2h = vh[j] * A11.v + vv[j] * A12.v, u2v = vh[j] * A12.v + vv[j] * A22.v;
    om_loc[j] = kok ? (vbh * zdh + vbv * zdv) +
                          (jbh[j] * (T(2) * u2h - vh[j]) + jbv[j] * (T(2) * u2v - vv[j]))
                    : T(0);
  }
  if (kok) {
    a.v_loc[el] = vb1;
    a.v_loc[el + K] = vb3;
    a.v_loc[el + 2 * K] = vb4;
    // S = <D bbar, D z^{k+1}> (A depends on omega through c = sum omega^2)
    const size_t qh = ((size_t)y * W + wrapi(x + 1, W)) * K + g;
    const size_t qv = ((size_t)wrapi(y + 1, H) * W + x) * K + g;
    const T z1 = a.zk1[e];
    s_loc = (a.bbar[qh] - bc) * (a.zk1[qh] - z1) + (a.bbar[qv] - bc) * (a.zk1[qv] - z1);
  }
  // block partial sums (tau once per pixel, from lane 0): warp shuffles in the working
  // precision, then the warps in a fixed order in FP64 (deterministic)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto wsum = [&](T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  {
    const T t0 = wsum((pok && g == 0) ? gbar4[3] : T(0));
    if (lane == 0) red[warp][0] = (double)t0;
  }
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const T t1 = wsum(om_loc[j]);
    if (lane == 0) red[warp][1 + j] = (double)t1;
  }
  {
    const T t2 = wsum(s_loc);
    if (lane == 0) red[warp][L + 1] = (double)t2;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < NP; j += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < NWARP; ++w) t += red[w][j];
    a.part[(size_t)j * gridDim.x + blockIdx.x] = t;
  }
}

// zbar^k = G^T vbar^k = vbar1 + J^T vbar2 + vbar3 + vbar4, one thread per (pixel, class).
template <typename T, int M>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_gt(AdjShape s, const T* v_loc, const T* v_2,
                                                        const T* omega, T* zbar) {
  constexpr int L = (2 * M + 1) * (2 * M + 1);
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)s.n * s.K) return;
  const int K = s.K;
  const int k = (int)(i % K);
  const int pix = (int)(i / K);
  const int y = pix / s.W, x = pix - y * s.W;
  const size_t el = (size_t)pix * 3 * K + k;
  T acc = v_loc[el] + v_loc[el + K] + v_loc[el + 2 * K];
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int sy = j / (2 * M + 1) - M, sx = j % (2 * M + 1) - M;
    // (J^T y)(x) = sum_j omega_j [y_h,j(x - s_j - e_h) - y_h,j(x - s_j)
    //                            + y_v,j(x - s_j - e_v) - y_v,j(x - s_j)]
    const int y0 = wrapi(y - sy, s.H), x0 = wrapi(x - sx, s.W);
    const int xm = wrapi(x0 - 1, s.W), ym = wrapi(y0 - 1, s.H);
    const size_t b0 = (((size_t)y0 * s.W + x0) * L + j) * K * 2 + 2 * k;
    const size_t bh = (((size_t)y0 * s.W + xm) * L + j) * K * 2 + 2 * k;
    const size_t bv = (((size_t)ym * s.W + x0) * L + j) * K * 2 + 2 * k;
    acc += omega[j] * (v_2[bh] - v_2[b0] + v_2[bv + 1] - v_2[b0 + 1]);
  }
  zbar[i] = acc;
}

// z^0 = p / 1^T p: glogp += z0 (zbar - <zbar, z0>) per pixel.
template <typename T, int G>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_init(AdjShape s, const T* p, const T* zbar,
                                                          T* glogp) {
  const int g = threadIdx.x & (G - 1);
  const int pix = blockIdx.x * (ADJ_THREADS / G) + threadIdx.x / G;
  const bool kok = pix < s.n && g < s.K;
  const size_t e = (size_t)pix * s.K + g;
  const T pk = kok ? p[e] : T(0);
  const T zb = kok ? zbar[e] : T(0);
  const T sp = group_sum<G>(pk);
  const T z0 = kok ? pk / sp : T(0);
  const T dot = group_sum<G>(zb * z0);
  if (kok) glogp[e] += z0 * (zb - dot);
}

// p = exp(log p - max_k log p) per pixel (the iterates do not see a per-pixel scale of p).
template <typename T, int G>
__global__ void __launch_bounds__(ADJ_THREADS) k_exp_logp(AdjShape s, const T* logp, T* p) {
  const int g = threadIdx.x & (G - 1);
  const int pix = blockIdx.x * (ADJ_THREADS / G) + threadIdx.x / G;
  const bool kok = pix < s.n && g < s.K;
  const size_t e = (size_t)pix * s.K + g;
  T v = kok ? logp[e] : T(-INFINITY);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o, G));
  if (kok) p[e] = exp(logp[e] - v);
}

template <typename T>
cudaError_t launch_adj_vjp(const AdjArgs<T>& a, int M, int G, int blocks, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_gt(AdjShape s, int M, const T* v_loc, const T* v_2, const T* omega,
                          T* zbar, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_init(AdjShape s, int G, const T* p, const T* zbar, T* glogp,
                            cudaStream_t st);
template <typename T>
cudaError_t launch_exp_logp(AdjShape s, int G, const T* logp, T* p, cudaStream_t st);
// acc[j] += sum over the `blocks` partials of column j of part ([np][blocks]), one block per
// column, in a fixed order.
cudaError_t launch_adj_sum(const double* part, int blocks, int np, double* acc, cudaStream_t st);

}  // namespace sgs
