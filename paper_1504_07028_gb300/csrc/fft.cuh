// z-update (12) of SegSALSA-STR: z = (3 I + J^T J)^{-1} rhs, periodic boundaries.
//
// J^T J = c (D_h^T D_h + D_v^T D_v) with c = sum_j omega_j^2 (periodic shifts are isometries),
// so G^T G is the 5-point operator 3 + c(2 - S_x - S_x^{-1}) + c(2 - S_y - S_y^{-1}), a cyclic
// convolution on each class image (Sec. 4). Three passes:
//   A  row pass:    real DFT along x of every row of every class (two classes per complex
//                   transform), reading rhs either densely or as the sum of the sweep's
//                   overlapping tile partials;
//   B  column pass: for every frequency kx the column system along y is the circulant
//                   tridiagonal (a_kx + 2c) - c (S_y + S_y^{-1}), a_kx = 3 + 4c sin^2(pi kx/W).
//                   It factors as (c/beta)(1 - beta S_y)(1 - beta S_y^{-1}) with
//                   beta + 1/beta = (a_kx + 2c)/c, so it is solved exactly by one causal and one
//                   anti-causal first-order recursion with periodic start values (the start
//                   value is a geometric sum truncated where beta^m is below rounding, or the
//                   exact periodic sum when the column is shorter);
//   C  row pass:    inverse real DFT along x, writing z.
// The 1D DFT is a shared-memory Stockham FFT (radix 8, 4, 2, 3, 5, 7); lengths with a prime
// factor above 7 go through Bluestein's chirp-z transform with a 7-smooth convolution length.
// Spectrum layout: S[y][kx][k] complex, kx in [0, W/2].
#pragma once

#include <algorithm>

#include "common.cuh"

namespace sgs {

constexpr int FFT_MAXST = 24;

// Shared-memory slot of complex element i of a transform buffer: one pad slot after every
// 128 bytes of elements (16 FP32 or 8 FP64 complex values). The first Stockham stage writes
// with a power-of-two stride (radix x sequences); without the pad those writes fall on a few
// banks, with it they spread over all of them. A pad per 128 bytes keeps every contiguous,
// 128-byte-aligned run of a warp's accesses (the stage loads, the later stages' stores) inside
// one set of 32 banks; a pad per 64 bytes (the first version) made all of those 2-way
// conflicted (half of the shared-memory wavefronts of the row passes were conflicts).
template <typename T>
struct PadShift {
  static constexpr int v = sizeof(T) == 4 ? 4 : 3;
};
template <typename T>
__host__ __device__ __forceinline__ int px(int i) { return i + (i >> PadShift<T>::v); }
template <typename T>
__host__ __device__ inline size_t padded_elems(size_t n) { return n + (n >> PadShift<T>::v) + 1; }

template <typename T>
struct FftPlan {
  int N;        // row length W
  int Mf;       // transform length run: N, or the Bluestein length
  int blue;     // 1 when Bluestein is used
  int nst;      // number of Stockham stages
  int radix[FFT_MAXST];
  int ns[FFT_MAXST];         // product of the radices before this stage
  uint32_t mg_ns[FFT_MAXST];   // ceil(2^32 / ns) (exact division of indices < 2^16)
  uint32_t mg_nsr[FFT_MAXST];  // ceil(2^32 / (ns * radix))
  const cplx<T>* tw;     // [Mf] exp(-2 pi i m / Mf)
  const cplx<T>* chirp;  // [N]  exp(i pi m^2 / N)          (Bluestein)
  const cplx<T>* bhat;   // [Mf] DFT of the chirp filter / Mf (Bluestein)
};

// ---------------------------------------------------------------- small DFT butterflies
template <int R, typename C> struct Dft;

template <typename C> struct Dft<2, C> {
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C> struct Dft<4, C> {
  __device__ __forceinline__ static void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <typename C> struct Dft<8, C> {
  __device__ __forceinline__ static void run(C* v) {
    using T = decltype(v[0].x);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, C>::run(e);
    Dft<4, C>::run(o);
    const T h = T(0.70710678118654752440);  // 1/sqrt(2)
    C o1; o1.x = h * (o[1].x + o[1].y); o1.y = h * (o[1].y - o[1].x);   // * exp(-i pi/4)
    C o2 = cmul_mi(o[2]);                                                 // * exp(-i pi/2)
    C o3; o3.x = h * (o[3].y - o[3].x); o3.y = -h * (o[3].x + o[3].y);   // * exp(-3i pi/4)
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
};

// Odd prime radix: direct DFT with the constant roots cos/sin(2 pi q / R), q in [0, R).
__host__ __device__ constexpr double root_cos(int R, int q) {
  return R == 3 ? (q == 0 ? 1.0 : -0.5)
       : R == 5 ? (q == 0 ? 1.0 : (q == 1 || q == 4) ? 0.30901699437494742410 : -0.80901699437494742410)
       : (q == 0 ? 1.0 : (q == 1 || q == 6) ? 0.62348980185873353053
                       : (q == 2 || q == 5) ? -0.22252093395631440429 : -0.90096886790241912624);
}
__host__ __device__ constexpr double root_sin(int R, int q) {
  return R == 3 ? (q == 0 ? 0.0 : q == 1 ? 0.86602540378443864676 : -0.86602540378443864676)
       : R == 5 ? (q == 0 ? 0.0 : q == 1 ? 0.95105651629515357212 : q == 2 ? 0.58778525229247312917
                  : q == 3 ? -0.58778525229247312917 : -0.95105651629515357212)
       : (q == 0 ? 0.0 : q == 1 ? 0.78183148246802980871 : q == 2 ? 0.97492791218182360702
                : q == 3 ? 0.43388373911755812048 : q == 4 ? -0.43388373911755812048
                : q == 5 ? -0.97492791218182360702 : -0.78183148246802980871);
}

// Output pairs m, R - m from the sums P_r = v_r + v_{R-r} and differences Q_r = v_r - v_{R-r},
// r = 1 .. (R-1)/2 (the roots of r and R - r are conjugate):
//   X_m = v_0 + sum_r P_r cos_rm + (sum_r Q_r.y sin_rm, -sum_r Q_r.x sin_rm),  X_{R-m} = ... -.
template <int R, typename C> struct DftOdd {
  __device__ __forceinline__ static void run(C* v) {
    using T = decltype(v[0].x);
    constexpr int H = (R - 1) / 2;
    C P[H + 1], Q[H + 1];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      P[r].x = v[r].x + v[R - r].x; P[r].y = v[r].y + v[R - r].y;
      Q[r].x = v[r].x - v[R - r].x; Q[r].y = v[r].y - v[R - r].y;
    }
    const C v0 = v[0];
    C x0 = v0;
#pragma unroll
    for (int r = 1; r <= H; ++r) { x0.x += P[r].x; x0.y += P[r].y; }
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      T ax = v0.x, ay = v0.y, bx = T(0), by = T(0);
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const int q = (r * m) % R;
        const T cr = T(root_cos(R, q)), sr = T(root_sin(R, q));
        ax += P[r].x * cr; ay += P[r].y * cr;
        bx += Q[r].y * sr; by -= Q[r].x * sr;
      }
      v[m].x = ax + bx; v[m].y = ay + by;
      v[R - m].x = ax - bx; v[R - m].y = ay - by;
    }
    v[0] = x0;
  }
};
template <typename C> struct Dft<3, C> : DftOdd<3, C> {};
template <typename C> struct Dft<5, C> : DftOdd<5, C> {};
template <typename C> struct Dft<7, C> : DftOdd<7, C> {};

// floor(t / d) for t < 2^16 with mg = ceil(2^32 / d) (mg = 0 encodes d = 1).
__device__ __forceinline__ int qdiv(int t, uint32_t mg) {
  return mg ? (int)__umulhi((uint32_t)t, mg) : t;
}

// One forward Stockham stage of radix R in {2,3,4,5,7,8} on B = 2^lgB interleaved sequences
// X[n * B + b], out of place: each work item is one radix-R butterfly reading Xin and writing
// Xout; the caller synchronises the block between stages.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ Xin, cplx<T>* __restrict__ Xout,
                                          int B, uint32_t mgB, int Mf, int Ns, uint32_t mg,
                                          const cplx<T>* tw, int S) {
  using C = cplx<T>;
  const int nb = Mf / R;
  const int items = nb * B;
  const int stride = nb / Ns;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int t = qdiv(it, mgB), b = it - t * B;
    const int g = qdiv(t, mg);
    const int j = t - g * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = Xin[px<T>((t + r * nb) * S + b)];
    // twiddles w^r, w = tw[j * stride]: w and (for R > 5) w^4 from the table, the other
    // powers by at most two products
    {
      const C w1 = tw[j * stride];
      v[1] = cmul(v[1], w1);
      if (R > 2) {
        const C w2 = cmul(w1, w1);
        v[2] = cmul(v[2], w2);
        if (R > 3) {
          const C w3 = cmul(w2, w1);
          v[3] = cmul(v[3], w3);
          if (R > 4) {
            const C w4 = (R > 5) ? tw[4 * j * stride] : cmul(w2, w2);
            v[4] = cmul(v[4], w4);
            if (R > 5) {
              v[5] = cmul(v[5], cmul(w4, w1));
              v[6] = cmul(v[6], cmul(w4, w2));
            }
            if (R > 7) v[7] = cmul(v[7], cmul(w4, w3));
          }
        }
      }
    }
    Dft<R, C>::run(v);
    const int base = (g * Ns * R + j) * S + b;
#pragma unroll
    for (int r = 0; r < R; ++r) Xout[px<T>(base + r * Ns * S)] = v[r];
  }
}

// A Stockham stage of prime radix R > 7: output o = g Ns R + m Ns + j of sequence b is
// X_m = sum_r y_r w^(r m nb), y_r = x_{t + r nb} w^(r j s), t = g Ns + j, s = nb / Ns, w the
// Mf-th root of unity (w^nb the R-th). The inter-stage twiddles are applied to the input in place
// first (only when Ns > 1). Then each work item computes one pair of outputs m and R - m from
// the symmetric and antisymmetric sums P_r = y_r + y_{R-r}, Q_r = y_r - y_{R-r}:
//   X_m = y_0 + sum_r P_r Re(w_rm) + i sum_r Q_r Im(w_rm),  X_{R-m} = same with - i ...,
// r = 1 .. (R-1)/2 (since w_{(R-r) m} = conj(w_rm)); m = 0 gives X_0 = y_0 + sum_r P_r alone.
// Xin is overwritten by the twiddled input; the output goes to Xout.
template <typename T>
__device__ __forceinline__ void fft_direct_stage(cplx<T>* __restrict__ Xin,
                                                 cplx<T>* __restrict__ Xout, int B, uint32_t mgB,
                                                 int Mf, int R, int Ns, uint32_t mg_ns,
                                                 uint32_t mg_nsr, const cplx<T>* tw, int S) {
  using C = cplx<T>;
  (void)mg_nsr;
  const int nb = Mf / R;
  const int s = nb / Ns;
  if (Ns > 1) {
    // element n = t + r nb of sequence b gets w^(r j s), j = t mod Ns; r j s < R nb = Mf
    for (int it = threadIdx.x; it < Mf * B; it += blockDim.x) {
      const int n = qdiv(it, mgB), b = it - n * B;
      const int r = n / nb, t = n - r * nb;
      const int jj = t - qdiv(t, mg_ns) * Ns;
      const int e = r * jj * s;
      if (e) {
        const int q = px<T>(n * S + b);
        Xin[q] = cmul(Xin[q], tw[e]);
      }
    }
    __syncthreads();
  }
  const int hm = (R + 1) / 2;
  const int items = nb * B * hm;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int rest = qdiv(it, mgB), b = it - rest * B;   // sequences fastest: shared loads
    const int t = rest / hm, m = rest - t * hm;
    const int src = t * S + b;
    const C y0 = Xin[px<T>(src)];
    const int step = m * nb;                               // < Mf
    int idx = 0;
    T ax = T(0), ay = T(0), bx = T(0), by = T(0);
    for (int r = 1; r < hm; ++r) {
      const C yr = Xin[px<T>(src + r * nb * S)];
      const C yq = Xin[px<T>(src + (R - r) * nb * S)];
      idx += step;
      idx -= (idx >= Mf) ? Mf : 0;
      const C w = tw[idx];
      ax += (yr.x + yq.x) * w.x;
      ay += (yr.y + yq.y) * w.x;
      bx += (yr.x - yq.x) * w.y;
      by += (yr.y - yq.y) * w.y;
    }
    const int g = qdiv(t, mg_ns), jj = t - g * Ns;
    const int ob = g * Ns * R + jj;
    // i (bx + i by) = -by + i bx
    Xout[px<T>((ob + m * Ns) * S + b)] = mkc<T>(y0.x + ax - by, y0.y + ay + bx);
    if (m > 0) Xout[px<T>((ob + (R - m) * Ns) * S + b)] = mkc<T>(y0.x + ax + by, y0.y + ay - bx);
  }
}

// Shared-memory copies of the transform tables, filled at kernel start.
template <typename T>
struct FftTables {
  const cplx<T>* tw;
  const cplx<T>* chirp;
  const cplx<T>* bhat;
};

// All stages of the plan, ping-ponging between X (holding the input; the caller has
// synchronised after filling it) and Y. Returns the buffer that holds the result; the block
// is synchronised on return.
template <typename T>
__device__ cplx<T>* fft_forward(cplx<T>* X, cplx<T>* Y, int B, uint32_t mgB, const FftPlan<T>& pl,
                                const cplx<T>* tw, int S = -1) {
  if (S < 0) S = B;  // element stride (sequences [0, B) interleaved at unit stride)
  cplx<T>* in = X;
  cplx<T>* out = Y;
  for (int s = 0; s < pl.nst; ++s) {
    const int Ns = pl.ns[s];
    const uint32_t mg = pl.mg_ns[s];
    switch (pl.radix[s]) {
      case 8: fft_stage<T, 8>(in, out, B, mgB, pl.Mf, Ns, mg, tw, S); break;
      case 4: fft_stage<T, 4>(in, out, B, mgB, pl.Mf, Ns, mg, tw, S); break;
      case 2: fft_stage<T, 2>(in, out, B, mgB, pl.Mf, Ns, mg, tw, S); break;
      case 3: fft_stage<T, 3>(in, out, B, mgB, pl.Mf, Ns, mg, tw, S); break;
      case 5: fft_stage<T, 5>(in, out, B, mgB, pl.Mf, Ns, mg, tw, S); break;
      case 7: fft_stage<T, 7>(in, out, B, mgB, pl.Mf, Ns, mg, tw, S); break;
      default:
        fft_direct_stage<T>(in, out, B, mgB, pl.Mf, pl.radix[s], Ns, mg, pl.mg_nsr[s], tw, S);
        break;
    }
    __syncthreads();
    cplx<T>* t = in; in = out; out = t;
  }
  return in;
}

// Bytes of shared memory for the tables of a plan (twiddles, and for Bluestein the chirp and
// the filter spectrum).
template <typename T>
__host__ __device__ inline size_t fft_table_bytes(int N, int Mf, int blue) {
  return sizeof(cplx<T>) * ((size_t)Mf + (blue ? (size_t)N + Mf : 0));
}

// Start the asynchronous copies of the tables into `tab` (caller commits and waits).
template <typename T>
__device__ inline FftTables<T> load_tables(const FftPlan<T>& pl, cplx<T>* tab) {
  constexpr int CB = sizeof(cplx<T>);
  for (int i = threadIdx.x; i < pl.Mf; i += blockDim.x) cp_async_zfill<CB>(tab + i, pl.tw + i, true);
  FftTables<T> t{tab, nullptr, nullptr};
  if (pl.blue) {
    cplx<T>* ch = tab + pl.Mf;
    cplx<T>* bh = ch + pl.N;
    for (int i = threadIdx.x; i < pl.N; i += blockDim.x) cp_async_zfill<CB>(ch + i, pl.chirp + i, true);
    for (int i = threadIdx.x; i < pl.Mf; i += blockDim.x) cp_async_zfill<CB>(bh + i, pl.bhat + i, true);
    t.chirp = ch;
    t.bhat = bh;
  }
  return t;
}

// Forward DFT of length N of the B sequences in X (slots [0, N) filled, Bluestein slots
// [N, Mf) need not be; the caller has synchronised). Y is the second buffer of the same
// size. Returns the buffer R with R[k*B + b], k < N, holding X_k for the mixed-radix path;
// for Bluestein the caller reads dft_out(R, k).
template <typename T>
__device__ cplx<T>* dft_rows(cplx<T>* X, cplx<T>* Y, int B, uint32_t mgB, const FftPlan<T>& pl,
                             const FftTables<T>& tb) {
  if (!pl.blue) return fft_forward<T>(X, Y, B, mgB, pl, tb.tw);
  // a_n = x_n conj(chirp_n), zero padded (each thread rewrites only its own elements)
  for (int i = threadIdx.x; i < pl.Mf * B; i += blockDim.x) {
    const int n = qdiv(i, mgB);
    X[px<T>(i)] = (n < pl.N) ? cmulc(X[px<T>(i)], tb.chirp[n]) : mkc<T>(T(0), T(0));
  }
  __syncthreads();
  cplx<T>* A = fft_forward<T>(X, Y, B, mgB, pl, tb.tw);
  for (int i = threadIdx.x; i < pl.Mf * B; i += blockDim.x)
    A[px<T>(i)] = cconj(cmul(A[px<T>(i)], tb.bhat[qdiv(i, mgB)]));
  __syncthreads();
  return fft_forward<T>(A, A == X ? Y : X, B, mgB, pl, tb.tw);  // = conj(cyclic convolution)
}

// Value X_k of sequence b after dft_rows (R is the buffer it returned).
template <typename T>
__device__ __forceinline__ cplx<T> dft_out(const cplx<T>* R, int B, int k, int b,
                                           const FftPlan<T>& pl, const FftTables<T>& tb) {
  const cplx<T> v = R[px<T>(k * B + b)];
  if (!pl.blue) return v;
  return cconj(cmul(tb.chirp[k], v));  // conj(chirp_k) * (a * b)_k
}

// ------------------------------------------------------------------- pass A (forward rows)
template <typename T>
struct RowArgs {
  int H, W, K, Wh;       // Wh = W/2 + 1 stored frequencies
  int QB;                // class pairs per CTA (a power of two)
  int lgB;               // log2(QB)
  uint32_t mgB;          // ceil(2^32 / QB)
  int smem_tables;       // 1: copy the transform tables (and the offsets of the partials) to shared memory
  FftPlan<T> pl;
  // source of rhs: dense [n][K] (src != null) or the sweep partials
  const T* src;
  const T* P;            // [tiles][EHmax][EWmax][K]
  int ntx, EHmax, EWmax;
  const int* covY;       // [H][2]: (tile row << 16 | ext row), -1 when absent
  const int* covX;       // [W][2]: (tile col << 16 | ext col)
  const int* offX;       // [W][2]: (tile col * EHmax * EWmax + ext col) * K, -1 when absent
  cplx<T>* S;            // [H][Wh][K]
  T* z;                  // pass C output [n][K]
  // persistent pipelined row passes (k_row_*_pipe): units (row, class block) in row-major
  // order, nq class blocks per row, and the vertical-cover slots of the forward stage (1 or 2)
  int nq, units, nslot;
};

// rhs(y, x, k) as the fixed-order sum of the (at most 2 x 2) tile partials covering (y, x);
// covY / covX entries are (tile << 16 | position in the tile + halo), -1 when absent.
template <typename T>
__device__ __forceinline__ T gather_rhs(const RowArgs<T>& a, int y, int x, int k) {
  if (a.src) return a.src[((size_t)y * a.W + x) * a.K + k];
  T v = T(0);
#pragma unroll
  for (int iy = 0; iy < 2; ++iy) {
    const int cy = a.covY[2 * y + iy];
    if (cy < 0) continue;
    const int ty = cy >> 16, ey = cy & 0xffff;
#pragma unroll
    for (int ix = 0; ix < 2; ++ix) {
      const int cx = a.covX[2 * x + ix];
      if (cx < 0) continue;
      const int tx = cx >> 16, ex = cx & 0xffff;
      const size_t t = (size_t)ty * a.ntx + tx;
      v += a.P[((t * a.EHmax + ey) * a.EWmax + ex) * a.K + k];
    }
  }
  return v;
}

// Same sum for a row whose two vertical covers start at P offsets rb0 / rb1 (-1 when absent),
// with the per-column offsets offX in shared memory. Same summation order as gather_rhs.
// Every row has a first vertical cover (rb0 >= 0) and every column a first horizontal one
// (o0 >= 0). The four loads are unconditional (an absent cover aliases the first one, whose
// value is then dropped by a select), so that the loads of all the elements a thread gathers
// can be in flight together.
template <typename T>
__device__ __forceinline__ T gather_row(const T* __restrict__ P, int rb0, int rb1, const int* oX,
                                        int x, int k) {
  const int o0 = oX[2 * x], o1r = oX[2 * x + 1];
  const bool hx = o1r >= 0, hy = rb1 >= 0;
  const int o1 = hx ? o1r : o0;
  const int r1 = hy ? rb1 : rb0;
  const T p00 = __ldg(P + rb0 + o0 + k), p01 = __ldg(P + rb0 + o1 + k);
  const T p10 = __ldg(P + r1 + o0 + k), p11 = __ldg(P + r1 + o1 + k);
  T v = p00;
  v += hx ? p01 : T(0);
  v += hy ? p10 : T(0);
  v += (hx && hy) ? p11 : T(0);
  return v;
}

// 16-byte vectors of the working precision (four FP32 or two FP64 classes of one pixel).
template <typename T> struct V16Of;
template <> struct V16Of<float> { using type = float4; };
template <> struct V16Of<double> { using type = double2; };
template <typename T> using v16 = typename V16Of<T>::type;
__device__ __forceinline__ float v16_at(const float4& v, int e) {
  return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ double v16_at(const double2& v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ float4 v16_add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 v16_add(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
template <typename T>
__device__ __forceinline__ v16<T> ldg16(const T* p) {
  return __ldg(reinterpret_cast<const v16<T>*>(p));
}

// gather_row for the 16 / sizeof(T) consecutive classes k, k + 1, ... (16-byte aligned), in the
// same summation order.
template <typename T>
__device__ __forceinline__ v16<T> gather_row16(const T* __restrict__ P, int rb0, int rb1,
                                               const int* oX, int x, int k) {
  const int o0 = oX[2 * x], o1r = oX[2 * x + 1];
  const bool hx = o1r >= 0, hy = rb1 >= 0;
  const int o1 = hx ? o1r : o0;
  const int r1 = hy ? rb1 : rb0;
  const v16<T> p00 = ldg16(P + rb0 + o0 + k), p01 = ldg16(P + rb0 + o1 + k);
  const v16<T> p10 = ldg16(P + r1 + o0 + k), p11 = ldg16(P + r1 + o1 + k);
  v16<T> v = p00;
  if (hx) v = v16_add(v, p01);
  if (hy) v = v16_add(v, p10);
  if (hx && hy) v = v16_add(v, p11);
  return v;
}

// P offset of the row start of vertical cover cy = (tile row << 16 | ext row), -1 if absent.
__device__ __forceinline__ int cover_row_base_raw(int cy, int ntx, int EHmax, int EWmax, int K) {
  if (cy < 0) return -1;
  return (((cy >> 16) * ntx * EHmax) + (cy & 0xffff)) * EWmax * K;
}
template <typename T>
__device__ __forceinline__ int cover_row_base(const RowArgs<T>& a, int cy) {
  return cover_row_base_raw(cy, a.ntx, a.EHmax, a.EWmax, a.K);
}
// ceil(2^32 / d) on the device (d >= 1; 0 encodes d = 1).
__device__ __forceinline__ uint32_t div_magic_dev(int d) {
  return d <= 1 ? 0u : (uint32_t)((0x100000000ULL + (unsigned long long)d - 1) / (unsigned long long)d);
}

// Shared memory of a row-pass CTA: two transform buffers and, when `tables`, copies of the
// transform tables and of the horizontal offset table of the tile partials.
template <typename T>
__host__ __device__ inline size_t row_smem_bytes(int N, int Mf, int blue, int QB, int tables) {
  return sizeof(cplx<T>) * 2 * padded_elems<T>((size_t)Mf * QB) +
         (tables ? fft_table_bytes<T>(N, Mf, blue) + sizeof(int) * 2 * (size_t)N : 0);
}
template <typename T>
__device__ inline FftTables<T> row_tables(const RowArgs<T>& a, cplx<T>* tab) {
  if (a.smem_tables) return load_tables<T>(a.pl, tab);
  return FftTables<T>{a.pl.tw, a.pl.chirp, a.pl.bhat};
}

// Two adjacent complex values as one 16-byte load (FP32) or two (FP64); src 16-byte aligned.
__device__ __forceinline__ void load_pair(const float2* src, float2& a, float2& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(src));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double2* src, double2& a, double2& b) {
  a = __ldg(src);
  b = __ldg(src + 1);
}

// Two adjacent complex values as 16-byte stores (dst 16-byte aligned).
__device__ __forceinline__ void store_pair(float2* dst, float2 a, float2 b) {
  *reinterpret_cast<float4*>(dst) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store_pair(double2* dst, double2 a, double2 b) {
  dst[0] = a;
  dst[1] = b;
}

// One unit of the forward row pass: row y, class pairs q0 .. q0 + QB - 1, on the calling CTA
// (any multiple of 32 threads; every loop strides by blockDim.x). OWN: the unit is the whole
// kernel (programmatic-dependency wait before reading the rhs, trigger after the transform);
// otherwise the caller has waited for the rhs already.
template <typename T, bool OWN>
__device__ __forceinline__ void row_forward_unit(const RowArgs<T>& a, int y, int q0,
                                                 unsigned char* smem_raw) {
  using C = cplx<T>;
  constexpr int U = 8;  // independent element loads in flight per thread
  C* X = reinterpret_cast<C*>(smem_raw);
  const int B = a.QB;
  const int N = a.pl.N;
  C* Y = X + padded_elems<T>((size_t)a.pl.Mf * B);  // second transform buffer
  C* tab = Y + padded_elems<T>((size_t)a.pl.Mf * B);
  // horizontal offsets of the partials: a shared-memory copy, or the global table (cached
  // loads) when the CTA's shared memory is kept to the transform buffers
  const int* cX = a.offX;
  const FftTables<T> tb = row_tables<T>(a, tab);
  if (a.smem_tables && !a.src) {
    int* cs = reinterpret_cast<int*>(tab + fft_table_bytes<T>(N, a.pl.Mf, a.pl.blue) / sizeof(C));
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) cp_async_zfill<4>(cs + i, a.offX + i, true);
    cX = cs;
  }
  cp_async_commit();
  if constexpr (OWN) pdl_wait();  // rhs / partials come from the previous kernel
  cp_async_wait_all();
  __syncthreads();
  T* Xf = reinterpret_cast<T*>(X);
  // load: two classes per complex sequence (real part class 2q, imaginary part class 2q+1)
  const int tot = N * B * 2;
  const int rb0 = a.src ? -1 : cover_row_base(a, a.covY[2 * y]);
  const int rb1 = a.src ? -1 : cover_row_base(a, a.covY[2 * y + 1]);
  // 16-byte reads of a pixel's classes when the CTA's classes are whole aligned vectors (a
  // caller's dense rhs may be only element-aligned)
  constexpr int VE = 16 / sizeof(T);
  const bool vec = a.K % VE == 0 && (2 * B) % VE == 0 && 2 * (q0 + B) <= a.K &&
                   (reinterpret_cast<uintptr_t>(a.src) & 15) == 0;
  if (vec) {
    constexpr int UV = 4;
    const int nv = 2 * B / VE;  // vectors per pixel (a power of two)
    const int lnv = __ffs(nv) - 1;
    const int totv = N * nv;
    for (int i0 = threadIdx.x; i0 < totv; i0 += UV * blockDim.x) {
      v16<T> v[UV];
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < totv) {
          const int x = i >> lnv, j = i & (nv - 1);
          const int k = 2 * q0 + j * VE;
          v[u] = a.src ? ldg16(a.src + ((size_t)y * a.W + x) * a.K + k)
                       : gather_row16<T>(a.P, rb0, rb1, cX, x, k);
        }
      }
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < totv) {
          const int x = i >> lnv, j = i & (nv - 1);
          // classes 2p, 2p + 1 of the vector form pair p (real, imaginary part)
#pragma unroll
          for (int pp = 0; pp < VE / 2; ++pp)
            X[px<T>(x * B + j * (VE / 2) + pp)] = mkc<T>(v16_at(v[u], 2 * pp), v16_at(v[u], 2 * pp + 1));
        }
      }
    }
  }
  for (int i0 = vec ? tot : threadIdx.x; i0 < tot; i0 += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = T(0);
      if (i < tot) {
        const int part = i & 1;
        const int qq = (i >> 1) & (B - 1);
        const int x = (i >> 1) >> a.lgB;
        const int k = 2 * (q0 + qq) + part;
        if (k < a.K)
          v[u] = a.src ? a.src[((size_t)y * a.W + x) * a.K + k] : gather_row<T>(a.P, rb0, rb1, cX, x, k);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < tot) Xf[2 * px<T>(i >> 1) + (i & 1)] = v[u];
    }
  }
  __syncthreads();
  const C* R = dft_rows<T>(X, Y, B, a.mgB, a.pl, tb);
  if constexpr (OWN) pdl_trigger();
  // unpack the two real spectra of each pair: A = (X_k + conj X_{N-k})/2,
  // B = (X_k - conj X_{N-k})/(2i); one thread per pair, stored together when K is even
  for (int i = threadIdx.x; i < a.Wh * B; i += blockDim.x) {
    const int qq = i & (B - 1);
    const int kx = i >> a.lgB;
    const int k = 2 * (q0 + qq);
    if (k >= a.K) continue;
    const C u = dft_out<T>(R, B, kx, qq, a.pl, tb);
    const C w = dft_out<T>(R, B, (kx == 0) ? 0 : N - kx, qq, a.pl, tb);
    C oa, ob;
    oa.x = T(0.5) * (u.x + w.x); oa.y = T(0.5) * (u.y - w.y);
    ob.x = T(0.5) * (u.y + w.y); ob.y = T(0.5) * (w.x - u.x);
    C* dst = a.S + ((size_t)y * a.Wh + kx) * a.K + k;
    if ((a.K & 1) == 0) {
      store_pair(dst, oa, ob);
    } else {
      dst[0] = oa;
      if (k + 1 < a.K) dst[1] = ob;
    }
  }
}

// grid (class blocks, rows): the class blocks of one row run side by side, so the 32-byte
// sectors they share are read from DRAM once
template <typename T>
__global__ void __launch_bounds__(1024) k_row_forward(const RowArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  row_forward_unit<T, true>(a, blockIdx.y, blockIdx.x * a.QB, smem_raw);
}

// Dense rhs [n][K] from the sweep partials (checkpoint read-out).
template <typename T>
__global__ void k_gather_dense(const RowArgs<T> a) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)a.H * a.W * a.K) return;
  const int k = (int)(i % a.K);
  const size_t pix = i / a.K;
  a.z[i] = gather_rhs(a, (int)(pix / a.W), (int)(pix % a.W), k);
}

// ------------------------------------------------------------------- pass C (inverse rows)
// One unit of the inverse row pass (row y, class pairs q0 .. q0 + QB - 1); OWN as for
// row_forward_unit.
template <typename T, bool OWN>
__device__ __forceinline__ void row_inverse_unit(const RowArgs<T>& a, int y, int q0,
                                                 unsigned char* smem_raw) {
  using C = cplx<T>;
  constexpr int U = 8;
  C* X = reinterpret_cast<C*>(smem_raw);
  const int B = a.QB;
  const int N = a.pl.N;
  C* Y = X + padded_elems<T>((size_t)a.pl.Mf * B);  // second transform buffer
  C* tab = Y + padded_elems<T>((size_t)a.pl.Mf * B);
  const FftTables<T> tb = row_tables<T>(a, tab);
  cp_async_commit();
  if constexpr (OWN) pdl_wait();  // the spectrum comes from the column pass
  // load conj(A + iB) over the full frequency range (Hermitian extension), inverse DFT by
  // conj(DFT(conj(.)))/N
  const int tot = N * B;
  for (int i0 = threadIdx.x; i0 < tot; i0 += U * blockDim.x) {
    C Av[U], Bv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      Av[u] = mkc<T>(T(0), T(0));
      Bv[u] = Av[u];
      if (i < tot) {
        const int qq = i & (B - 1);
        const int kx = i >> a.lgB;
        const int ka = 2 * (q0 + qq), kb = ka + 1;
        const int ks = kx < a.Wh ? kx : N - kx;
        const C* row = a.S + ((size_t)y * a.Wh + ks) * a.K;
        if (kb < a.K && (a.K & 1) == 0) {
          load_pair(row + ka, Av[u], Bv[u]);
        } else {
          if (ka < a.K) Av[u] = row[ka];
          if (kb < a.K) Bv[u] = row[kb];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < tot) {
        C A = Av[u], Bq = Bv[u];
        if ((i >> a.lgB) >= a.Wh) { A = cconj(A); Bq = cconj(Bq); }
        C xv; xv.x = A.x - Bq.y; xv.y = -(A.y + Bq.x);   // conj(A + i B)
        X[px<T>(i)] = xv;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const C* R = dft_rows<T>(X, Y, B, a.mgB, a.pl, tb);
  if constexpr (OWN) pdl_trigger();
  const T inv = T(1) / T(N);
  constexpr int VE = 16 / sizeof(T);
  const bool vec = a.K % VE == 0 && (2 * B) % VE == 0 && 2 * (q0 + B) <= a.K &&
                   (reinterpret_cast<uintptr_t>(a.z) & 15) == 0;  // z may be a caller's buffer
  if (vec) {
    // 16-byte stores of VE classes of one pixel (VE / 2 pairs)
    const int nv = 2 * B / VE;
    const int lnv = __ffs(nv) - 1;
    for (int i = threadIdx.x; i < N * nv; i += blockDim.x) {
      const int x = i >> lnv, j = i & (nv - 1);
      T o[VE];
#pragma unroll
      for (int e = 0; e < VE / 2; ++e) {
        const C v = dft_out<T>(R, B, x, j * (VE / 2) + e, a.pl, tb);  // conj(v) / N
        o[2 * e] = v.x * inv;
        o[2 * e + 1] = -v.y * inv;
      }
      T* dst = a.z + ((size_t)y * a.W + x) * a.K + 2 * q0 + j * VE;
      if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
      else
        *reinterpret_cast<double2*>(dst) = make_double2(o[0], o[1]);
    }
    return;
  }
  for (int i = threadIdx.x; i < N * B * 2; i += blockDim.x) {
    const int part = i & 1;
    const int qq = (i >> 1) & (B - 1);
    const int x = (i >> 1) >> a.lgB;
    const int k = 2 * (q0 + qq) + part;
    if (k >= a.K) continue;
    const C v = dft_out<T>(R, B, x, qq, a.pl, tb);     // DFT(conj X)_x ; result = conj(v)/N
    a.z[((size_t)y * a.W + x) * a.K + k] = (part == 0) ? v.x * inv : -v.y * inv;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_row_inverse(const RowArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  row_inverse_unit<T, true>(a, blockIdx.y, blockIdx.x * a.QB, smem_raw);
}

// ------------------------------------------------ pipelined row passes (persistent CTAs)
//
// The same transforms as k_row_forward / k_row_inverse, organised for long rows: a CTA stays
// resident and walks the units (row y, class block) u = blockIdx.x, blockIdx.x + gridDim.x, ...
// Each unit's input (the tile partials that cover row y, the dense rhs row, or the spectrum
// row) is brought into a shared-memory stage by asynchronous copies; the copies of the next
// unit are issued as soon as the current unit has left the stage, so they are in flight while
// the current unit's FFT and stores run. Every CTA thus keeps loads outstanding during its
// compute phases, instead of alternating between loading and computing. The summation order
// of the covers and the transforms are those of the one-unit-per-CTA kernels (bit-identical
// results).

// 16-byte asynchronous copy global -> shared that bypasses L1 (streamed data).
__device__ __forceinline__ void cp_async_cg16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}

// Shared memory of a pipelined row CTA: two transform buffers, then the stage.
template <typename T>
__host__ __device__ inline size_t rowpipe_fwd_stage_elems(int N, int ntx, int EWmax, int QB,
                                                          bool dense) {
  return dense ? (size_t)N * 2 * QB : (size_t)ntx * EWmax * 2 * QB;  // per slot, in T
}
template <typename T>
__host__ __device__ inline size_t rowpipe_smem_bytes(bool forward, int N, int Mf, int Wh, int QB,
                                                     int ntx, int EWmax, int nslot, bool dense) {
  const size_t xy = sizeof(cplx<T>) * 2 * padded_elems<T>((size_t)Mf * QB);
  if (forward)
    return xy + sizeof(T) * (dense ? 1 : nslot) *
                    rowpipe_fwd_stage_elems<T>(N, ntx, EWmax, QB, dense);
  return xy + sizeof(cplx<T>) * (size_t)Wh * 2 * QB;
}

// Issue the copies of the rhs of unit u into the stage: vertical covers [iy0, iy1) of row y
// (slot iy - iy0 each, laid out [tile column][ext column][class of the block]), or the dense
// rhs row ([x][class]). Classes past K are zero-filled.
template <typename T>
__device__ __forceinline__ void rowpipe_issue_fwd(const RowArgs<T>& a, int u, int iy0, int iy1,
                                                  T* stg, size_t slot) {
  const int y = u / a.nq, qb = u - y * a.nq;
  const int CW = 2 * a.QB;             // classes of the unit
  const int c0 = qb * CW;
  const int K = a.K;
  constexpr int VE = 16 / sizeof(T);
  const bool vec = CW % VE == 0 && K % VE == 0 && c0 + CW <= K;
  const int nv = CW / VE;
  if (a.src) {
    const T* row = a.src + (size_t)y * a.W * K + c0;
    if (vec && (reinterpret_cast<uintptr_t>(a.src) & 15) == 0) {
      for (int i = threadIdx.x; i < a.W * nv; i += blockDim.x) {
        const int x = i / nv, v = i - x * nv;
        cp_async_cg16(stg + (size_t)x * CW + v * VE, row + (size_t)x * K + v * VE);
      }
    } else {
      for (int i = threadIdx.x; i < a.W * CW; i += blockDim.x) {
        const int x = i / CW, c = i - x * CW;
        const bool ok = c0 + c < K;
        cp_async_zfill<sizeof(T)>(stg + i, ok ? row + (size_t)x * K + c : a.src, ok);
      }
    }
    return;
  }
  const size_t tstride = (size_t)a.EHmax * a.EWmax * K;  // P elements per tile
  const int R = a.ntx * a.EWmax;                          // stage rows per slot
  for (int iy = iy0; iy < iy1; ++iy) {
    const int cy = a.covY[2 * y + iy];
    if (cy < 0) continue;                                 // uniform over the CTA
    const T* base = a.P + cover_row_base(a, cy) + c0;
    T* dst = stg + (size_t)(iy - iy0) * slot;
    if (vec) {
      for (int i = threadIdx.x; i < R * nv; i += blockDim.x) {
        const int r = i / nv, v = i - r * nv;
        const int tx = r / a.EWmax, ex = r - tx * a.EWmax;
        cp_async_cg16(dst + (size_t)r * CW + v * VE, base + tx * tstride + (size_t)ex * K + v * VE);
      }
    } else {
      for (int i = threadIdx.x; i < R * CW; i += blockDim.x) {
        const int r = i / CW, c = i - r * CW;
        const int tx = r / a.EWmax, ex = r - tx * a.EWmax;
        const bool ok = c0 + c < K;
        cp_async_zfill<sizeof(T)>(dst + i, ok ? base + tx * tstride + (size_t)ex * K + c : a.P, ok);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_row_forward_pipe(const RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int B = a.QB, N = a.pl.N;
  const int CW = 2 * B;
  C* X = reinterpret_cast<C*>(smem_raw);
  C* Y = X + padded_elems<T>((size_t)a.pl.Mf * B);
  T* stg = reinterpret_cast<T*>(Y + padded_elems<T>((size_t)a.pl.Mf * B));
  const bool dense = a.src != nullptr;
  const size_t slot = rowpipe_fwd_stage_elems<T>(N, a.ntx, a.EWmax, B, dense);
  const FftTables<T> tb{a.pl.tw, a.pl.chirp, a.pl.bhat};
  pdl_wait();                              // the partials / rhs come from the previous kernel
  int u = blockIdx.x;
  if (u < a.units) rowpipe_issue_fwd<T>(a, u, 0, dense ? 1 : a.nslot, stg, slot);
  cp_async_commit();
  for (; u < a.units; u += gridDim.x) {
    const int y = u / a.nq, qb = u - y * a.nq;
    const int q0 = qb * B;
    const bool hy = !dense && a.covY[2 * y + 1] >= 0;
    cp_async_wait_all();
    __syncthreads();                       // stage of u landed; the previous unit is done
    // the stage holds classes (2q, 2q + 1) of a pixel next to each other: read them as the
    // complex value of pair q
    const C* sc = reinterpret_cast<const C*>(stg);
    const C zero = mkc<T>(T(0), T(0));
    if (dense) {
      for (int i = threadIdx.x; i < N * B; i += blockDim.x) X[px<T>(i)] = sc[i];
    } else {
      // v = p00 (+ p01) (+ p10) (+ p11): the order of gather_row; absent covers add +0
      const C* s1 = sc + slot / 2;
      const bool two = a.nslot == 2;
      for (int i = threadIdx.x; i < N * B; i += blockDim.x) {
        const int x = i >> a.lgB, q = i & (B - 1);
        const int2 cx = __ldg(reinterpret_cast<const int2*>(a.covX) + x);
        const int r0 = (cx.x >> 16) * a.EWmax + (cx.x & 0xffff);
        const bool hx = cx.y >= 0;
        const int r1 = hx ? (cx.y >> 16) * a.EWmax + (cx.y & 0xffff) : r0;
        C v = sc[r0 * B + q];
        v = cadd(v, hx ? sc[r1 * B + q] : zero);
        if (two) {
          v = cadd(v, hy ? s1[r0 * B + q] : zero);
          v = cadd(v, (hx && hy) ? s1[r1 * B + q] : zero);
        } else if (!hy) {
          v = cadd(v, zero);
          v = cadd(v, zero);
        }
        X[px<T>(i)] = v;
      }
      if (!two && hy) {
        // one slot: the second vertical cover goes through the stage after the first
        __syncthreads();
        rowpipe_issue_fwd<T>(a, u, 1, 2, stg, slot);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        for (int i = threadIdx.x; i < N * B; i += blockDim.x) {
          const int x = i >> a.lgB, q = i & (B - 1);
          const int2 cx = __ldg(reinterpret_cast<const int2*>(a.covX) + x);
          const int r0 = (cx.x >> 16) * a.EWmax + (cx.x & 0xffff);
          const bool hx = cx.y >= 0;
          const int r1 = hx ? (cx.y >> 16) * a.EWmax + (cx.y & 0xffff) : r0;
          C v = X[px<T>(i)];
          v = cadd(v, sc[r0 * B + q]);
          v = cadd(v, hx ? sc[r1 * B + q] : zero);
          X[px<T>(i)] = v;
        }
      }
    }
    __syncthreads();                       // the stage is free, X holds the unit's rows
    const int un = u + gridDim.x;
    if (un < a.units) rowpipe_issue_fwd<T>(a, un, 0, dense ? 1 : a.nslot, stg, slot);
    cp_async_commit();
    if (un >= a.units) pdl_trigger();
    const C* R = dft_rows<T>(X, Y, B, a.mgB, a.pl, tb);
    // unpack the two real spectra of each pair (as k_row_forward)
    for (int i = threadIdx.x; i < a.Wh * B; i += blockDim.x) {
      const int qq = i & (B - 1);
      const int kx = i >> a.lgB;
      const int k = 2 * (q0 + qq);
      if (k >= a.K) continue;
      const C uu = dft_out<T>(R, B, kx, qq, a.pl, tb);
      const C w = dft_out<T>(R, B, (kx == 0) ? 0 : N - kx, qq, a.pl, tb);
      C oa, ob;
      oa.x = T(0.5) * (uu.x + w.x); oa.y = T(0.5) * (uu.y - w.y);
      ob.x = T(0.5) * (uu.y + w.y); ob.y = T(0.5) * (w.x - uu.x);
      C* dst = a.S + ((size_t)y * a.Wh + kx) * a.K + k;
      if ((a.K & 1) == 0) {
        store_pair(dst, oa, ob);
      } else {
        dst[0] = oa;
        if (k + 1 < a.K) dst[1] = ob;
      }
    }
  }
  cp_async_wait_all();                     // nothing may be in flight when the CTA exits
}

// Issue the copies of the spectrum row of unit u: [kx][class of the block] complex, kx < Wh.
template <typename T>
__device__ __forceinline__ void rowpipe_issue_inv(const RowArgs<T>& a, int u, cplx<T>* stg) {
  using C = cplx<T>;
  const int y = u / a.nq, qb = u - y * a.nq;
  const int CW = 2 * a.QB;
  const int c0 = qb * CW;
  const C* row = a.S + (size_t)y * a.Wh * a.K + c0;
  constexpr int PE = 16 / sizeof(C);       // complex values per 16 bytes (2 FP32, 1 FP64)
  const bool vec = a.K % PE == 0 && c0 + CW <= a.K;
  if (vec) {
    const int nv = CW / PE;
    for (int i = threadIdx.x; i < a.Wh * nv; i += blockDim.x) {
      const int kx = i / nv, v = i - kx * nv;
      cp_async_cg16(stg + (size_t)kx * CW + v * PE, row + (size_t)kx * a.K + v * PE);
    }
  } else {
    for (int i = threadIdx.x; i < a.Wh * CW; i += blockDim.x) {
      const int kx = i / CW, c = i - kx * CW;
      const bool ok = c0 + c < a.K;
      cp_async_zfill<sizeof(C)>(stg + i, ok ? row + (size_t)kx * a.K + c : a.S, ok);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_row_inverse_pipe(const RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int B = a.QB, N = a.pl.N;
  const int CW = 2 * B;
  C* X = reinterpret_cast<C*>(smem_raw);
  C* Y = X + padded_elems<T>((size_t)a.pl.Mf * B);
  C* stg = Y + padded_elems<T>((size_t)a.pl.Mf * B);
  const FftTables<T> tb{a.pl.tw, a.pl.chirp, a.pl.bhat};
  pdl_wait();                              // the spectrum comes from the column pass
  int u = blockIdx.x;
  if (u < a.units) rowpipe_issue_inv<T>(a, u, stg);
  cp_async_commit();
  const T inv = T(1) / T(N);
  constexpr int VE = 16 / sizeof(T);
  for (; u < a.units; u += gridDim.x) {
    const int y = u / a.nq, qb = u - y * a.nq;
    const int q0 = qb * B;
    cp_async_wait_all();
    __syncthreads();
    // conj(A + iB) over the full frequency range (Hermitian extension), as k_row_inverse
    for (int i = threadIdx.x; i < N * B; i += blockDim.x) {
      const int qq = i & (B - 1);
      const int kx = i >> a.lgB;
      const int ks = kx < a.Wh ? kx : N - kx;
      C A = stg[(size_t)ks * CW + 2 * qq], Bq = stg[(size_t)ks * CW + 2 * qq + 1];
      if (kx >= a.Wh) { A = cconj(A); Bq = cconj(Bq); }
      C xv; xv.x = A.x - Bq.y; xv.y = -(A.y + Bq.x);
      X[px<T>(i)] = xv;
    }
    __syncthreads();
    const int un = u + gridDim.x;
    if (un < a.units) rowpipe_issue_inv<T>(a, un, stg);
    cp_async_commit();
    if (un >= a.units) pdl_trigger();
    const C* R = dft_rows<T>(X, Y, B, a.mgB, a.pl, tb);
    const bool vec = a.K % VE == 0 && (2 * B) % VE == 0 && 2 * (q0 + B) <= a.K &&
                     (reinterpret_cast<uintptr_t>(a.z) & 15) == 0;
    if (vec) {
      const int nv = 2 * B / VE;
      const int lnv = __ffs(nv) - 1;
      for (int i = threadIdx.x; i < N * nv; i += blockDim.x) {
        const int x = i >> lnv, j = i & (nv - 1);
        T o[VE];
#pragma unroll
        for (int e = 0; e < VE / 2; ++e) {
          const C v = dft_out<T>(R, B, x, j * (VE / 2) + e, a.pl, tb);
          o[2 * e] = v.x * inv;
          o[2 * e + 1] = -v.y * inv;
        }
        T* dst = a.z + ((size_t)y * a.W + x) * a.K + 2 * q0 + j * VE;
        if constexpr (sizeof(T) == 4)
          *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
        else
          *reinterpret_cast<double2*>(dst) = make_double2(o[0], o[1]);
      }
    } else {
      for (int i = threadIdx.x; i < N * B * 2; i += blockDim.x) {
        const int part = i & 1;
        const int qq = (i >> 1) & (B - 1);
        const int x = (i >> 1) >> a.lgB;
        const int k = 2 * (q0 + qq) + part;
        if (k >= a.K) continue;
        const C v = dft_out<T>(R, B, x, qq, a.pl, tb);
        a.z[((size_t)y * a.W + x) * a.K + k] = (part == 0) ? v.x * inv : -v.y * inv;
      }
    }
  }
  cp_async_wait_all();
}

// ------------------------------------------------------------------ pass B (column solve)
template <typename T>
struct ColArgs {
  int H, C;              // rows, complex columns per row (Wh*K)
  int K;
  int CB;                // complex columns per CTA
  int NSEG;              // segments along y
  int SL;                // rows per segment (segment i covers rows [i SL, min((i+1) SL, H)))
  const T* beta;         // [Wh]
  const T* gain;         // [Wh]
  const T* wfac;         // [Wh] 1 or 1/(1 - beta^H)
  const int* nwarm;      // [Wh]
  cplx<T>* S;            // [H][C]
};

// One unit of the column pass: complex columns blk * CB .. blk * CB + CB - 1 over all rows,
// on a CTA of at least 2 CB NSEG threads; OWN as for row_forward_unit.
template <typename T, bool OWN>
__device__ __forceinline__ void col_solve_unit(const ColArgs<T>& a, int blk, unsigned char* smem_raw) {
  T* buf = reinterpret_cast<T*>(smem_raw);  // [H][2*CB]
  const int c0 = blk * a.CB;
  const int nseq = 2 * a.CB;
  const int H = a.H;
  T* Sf = reinterpret_cast<T*>(a.S);
  // 16-byte moves when every row of the block starts on a 16-byte boundary and the block is full
  constexpr int V = 16 / sizeof(T);
  const bool vec = (2 * (size_t)a.C * sizeof(T)) % 16 == 0 && (nseq * sizeof(T)) % 16 == 0 &&
                   c0 + a.CB <= a.C;
  if constexpr (OWN) pdl_wait();  // the spectrum comes from the row pass
  if (vec) {
    const int per_row = nseq / V;
    for (int i = threadIdx.x; i < H * per_row; i += blockDim.x) {
      const int y = i / per_row, v = i - y * per_row;
      cp_async_zfill<16>(buf + y * nseq + v * V, Sf + (size_t)y * 2 * a.C + 2 * c0 + v * V, true);
    }
  } else {
    for (int i = threadIdx.x; i < H * nseq; i += blockDim.x) {
      const int y = i / nseq, s = i % nseq;
      const int col2 = 2 * c0 + s;
      const bool v = col2 < 2 * a.C;
      cp_async_zfill<sizeof(T)>(buf + i, v ? Sf + (size_t)y * 2 * a.C + col2 : Sf, v);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  const int s = threadIdx.x % nseq, seg = threadIdx.x / nseq;
  const bool act = seg < a.NSEG;
  const int c = c0 + s / 2;
  const int kx = (c < a.C) ? c / a.K : 0;
  const T beta = a.beta[kx], gain = a.gain[kx], wf = a.wfac[kx];
  const int nw = a.nwarm[kx];
  const int s0 = act ? min(seg * a.SL, H) : 0;
  const int s1 = act ? min(s0 + a.SL, H) : 0;
  // causal start value y_{s0-1} = sum_m beta^m r_{s0-1-m}
  T acc = T(0);
  if (act) {
    int n = s0 - nw;
    n += (n < 0) ? H : 0;
    for (int m = nw; m >= 1; --m) {
      acc = beta * acc + buf[n * nseq + s];
      n = (n + 1 == H) ? 0 : n + 1;
    }
    acc *= wf;
  }
  __syncthreads();
  if (act)
    for (int n = s0; n < s1; ++n) {
      acc = beta * acc + buf[n * nseq + s];
      buf[n * nseq + s] = acc;
    }
  __syncthreads();
  // anti-causal start value q_{s1} = sum_m beta^m y_{s1+m}
  T acc2 = T(0);
  if (act) {
    int n = s1 - 1 + nw;
    n -= (n >= H) ? H : 0;
    for (int m = nw; m >= 1; --m) {
      acc2 = beta * acc2 + buf[n * nseq + s];
      n = (n == 0) ? H - 1 : n - 1;
    }
    acc2 *= wf;
  }
  __syncthreads();
  if (act)
    for (int n = s1 - 1; n >= s0; --n) {
      acc2 = beta * acc2 + buf[n * nseq + s];
      buf[n * nseq + s] = gain * acc2;
    }
  if constexpr (OWN) pdl_trigger();
  __syncthreads();
  if (vec) {
    const int per_row = nseq / V;
    for (int i = threadIdx.x; i < H * per_row; i += blockDim.x) {
      const int y = i / per_row, v = i - y * per_row;
      *reinterpret_cast<float4*>(Sf + (size_t)y * 2 * a.C + 2 * c0 + v * V) =
          *reinterpret_cast<const float4*>(buf + y * nseq + v * V);
    }
  } else {
    for (int i = threadIdx.x; i < H * nseq; i += blockDim.x) {
      const int y = i / nseq, ss = i % nseq;
      const int col2 = 2 * c0 + ss;
      if (col2 < 2 * a.C) Sf[(size_t)y * 2 * a.C + col2] = buf[i];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_col_solve(const ColArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  col_solve_unit<T, true>(a, blockIdx.x, smem_raw);
}

// ---------------------------------------- the three passes in one launch (ordered tickets)
//
// The z-update as one launch of persistent CTAs. The work units of the three passes are
// numbered in pass order (forward (row, class block) units in row-major order, then the column
// blocks, then the inverse units) and handed out by an atomic ticket counter. A column unit
// starts once every forward unit has signalled completion, an inverse unit once every column
// unit has. A unit only ever waits for units with smaller tickets, and those were taken by
// CTAs that were already running and wait only for smaller tickets themselves, so the launch
// completes for any grid size and any number of co-resident CTAs: no cooperative launch is
// needed. The units run the bodies of k_row_forward / k_col_solve / k_row_inverse, so the
// results are bit-identical to the three launches. Each dependency wait is bounded (error
// flag, then the CTA stops taking tickets); the last CTA to finish returns the counters to 0
// for the next launch.
template <typename T>
struct ZseqArgs {
  RowArgs<T> f, i;       // forward and inverse row passes (their QB may differ)
  ColArgs<T> c;
  int nqf, nqi;          // class blocks per row of the forward / inverse pass
  int nf, nc, ni;        // units of each pass
  unsigned int* ctr;     // [4]: ticket, forward units done, column units done, CTAs done
  int* err;
  long long budget;      // clock cycles of one dependency wait
  int probe;             // 1: the column units wait for one forward unit more than exists
};

// Relaxed GPU-scope read of a counter (polling; an acquire fence follows the last read, so the
// polls themselves do not order, or invalidate, anything).
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;\n" ::: "memory"); }

constexpr int ZSEQ_MAX_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(ZSEQ_MAX_THREADS) k_zupdate_seq(const ZseqArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_ticket;
  pdl_wait();  // the rhs (partials or dense) comes from the previous kernel
  const int nfc = a.nf + a.nc, total = nfc + a.ni;
  bool triggered = false;
  for (;;) {
    if (threadIdx.x == 0) {
      int t = (int)atomicAdd(a.ctr, 1u);
      if (t >= a.nf && t < total) {
        const unsigned int* dep = t < nfc ? a.ctr + 1 : a.ctr + 2;
        const unsigned int need = t < nfc ? (unsigned)(a.nf + a.probe) : (unsigned)a.nc;
        if (ld_relaxed_u32(dep) < need) {
          const long long t0 = clock64();
          while (ld_relaxed_u32(dep) < need) {
            if (clock64() - t0 > a.budget) {
              atomicExch(a.err, 1);
              t = -1;
              break;
            }
            __nanosleep(128);
          }
        }
        fence_acq_rel_gpu();  // acquire: the producers' writes are visible to this CTA
      }
      s_ticket = t;
    }
    __syncthreads();
    const int t = s_ticket;
    if (t < 0 || t >= total) break;
    if (t < a.nf) {
      const int y = t / a.nqf, qb = t - y * a.nqf;
      row_forward_unit<T, false>(a.f, y, qb * a.f.QB, smem_raw);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.ctr + 1, 1u);
      }
    } else if (t < nfc) {
      col_solve_unit<T, false>(a.c, t - a.nf, smem_raw);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.ctr + 2, 1u);
      }
    } else {
      if (!triggered) {
        pdl_trigger();  // the next kernel may start its prologue once every CTA is here
        triggered = true;
      }
      const int u = t - nfc;
      const int y = u / a.nqi, qb = u - y * a.nqi;
      row_inverse_unit<T, false>(a.i, y, qb * a.i.QB, smem_raw);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.ctr + 3, 1u) == gridDim.x - 1) {
      // every CTA has taken its last ticket: nothing reads the counters any more
      atomicExch(a.ctr, 0u);
      atomicExch(a.ctr + 1, 0u);
      atomicExch(a.ctr + 2, 0u);
      atomicExch(a.ctr + 3, 0u);
    }
  }
}

// ------------------------------------------- power-of-two rows, compile-time Stockham plan
//
// Rows of N = 2^LOGN (256 <= N <= 4096) with B = QB class pairs per CTA whose 2B classes are
// whole 16- or 8-byte vectors: the plan of make_fft_plan (radix-8 stages, then one radix-4 or
// radix-2 stage) with every size, stride and twiddle step a compile-time constant, and the
// first radix-8 stage computed in registers straight from the loaded row (the gather of the
// rhs partials, or the Hermitian extension of the spectrum) instead of going through shared
// memory first. Same stages, same twiddles, same operation order as the generic kernels: the
// results are identical.

template <int LOGN>
struct P2Plan {
  static constexpr int N = 1 << LOGN;
};

// Butterfly it of a compile-time Stockham stage (radix R, Ns = NS, B interleaved sequences):
// p2_load reads its R inputs, p2_butterfly twiddles, transforms and writes them. A butterfly's
// R inputs (outputs) are NB * B (NS * B) elements apart: where that is a whole number of pad
// periods, the padded slots differ by a constant, so one padded base address and immediate
// offsets replace R index computations (same slots, same results).
template <typename T, int N, int B, int R>
__device__ __forceinline__ void p2_load(const cplx<T>* __restrict__ Xin, int it, cplx<T> (&v)[R]) {
  constexpr int NB = N / R;
  constexpr int PP = 1 << PadShift<T>::v;
  const int t = it / B, b = it - t * B;
  if constexpr ((NB * B) % PP == 0) {
    constexpr int SI = NB * B + NB * B / PP;
    const cplx<T>* xi = Xin + px<T>(t * B + b);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = xi[r * SI];
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = Xin[px<T>((t + r * NB) * B + b)];
  }
}
template <typename T, int N, int B, int R, int NS>
__device__ __forceinline__ void p2_twdft(int it, cplx<T> (&v)[R], const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int NB = N / R;
  constexpr int STRIDE = NB / NS;
  const int t = it / B;
  const int j = t - (t / NS) * NS;
  if constexpr (NS > 1) {
    const C w1 = tw[j * STRIDE];
    v[1] = cmul(v[1], w1);
    if constexpr (R > 2) {
      const C w2 = cmul(w1, w1);
      v[2] = cmul(v[2], w2);
      if constexpr (R > 3) {
        const C w3 = cmul(w2, w1);
        v[3] = cmul(v[3], w3);
        if constexpr (R > 4) {
          const C w4 = tw[4 * j * STRIDE];
          v[4] = cmul(v[4], w4);
          v[5] = cmul(v[5], cmul(w4, w1));
          v[6] = cmul(v[6], cmul(w4, w2));
          v[7] = cmul(v[7], cmul(w4, w3));
        }
      }
    }
  }
  Dft<R, C>::run(v);
}
template <typename T, int N, int B, int R, int NS>
__device__ __forceinline__ void p2_butterfly(cplx<T>* __restrict__ Xout, int it, cplx<T> (&v)[R],
                                             const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int PP = 1 << PadShift<T>::v;
  p2_twdft<T, N, B, R, NS>(it, v, tw);
  const int t = it / B, b = it - t * B;
  const int g = t / NS;
  const int j = t - g * NS;
  const int base = (g * NS * R + j) * B + b;
  if constexpr ((NS * B) % PP == 0) {
    constexpr int SO = NS * B + NS * B / PP;
    C* xo = Xout + px<T>(base);
#pragma unroll
    for (int r = 0; r < R; ++r) xo[r * SO] = v[r];
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) Xout[px<T>(base + r * NS * B)] = v[r];
  }
}

// One Stockham stage (generic fft_stage with compile-time arguments) on a CTA of TH threads,
// ITEMS / TH butterflies a thread, unrolled. Two buffers: each butterfly is read and written in
// turn. ONE (in place, Xout == Xin): every thread reads the inputs of all its butterflies, the
// CTA synchronises, then they are transformed and written.
template <typename T, int N, int B, int R, int NS, int TH, bool ONE>
__device__ __forceinline__ void p2_stage(const cplx<T>* Xin, cplx<T>* Xout, const cplx<T>* tw) {
  constexpr int ITEMS = N / R * B;
  static_assert(ITEMS % TH == 0, "whole butterflies per thread");
  constexpr int IPT = ITEMS / TH;
  if constexpr (ONE) {
    cplx<T> v[IPT][R];
#pragma unroll
    for (int u = 0; u < IPT; ++u) p2_load<T, N, B, R>(Xin, threadIdx.x + u * TH, v[u]);
    __syncthreads();  // every input read before any output lands on it
#pragma unroll
    for (int u = 0; u < IPT; ++u) p2_butterfly<T, N, B, R, NS>(Xout, threadIdx.x + u * TH, v[u], tw);
  } else {
    cplx<T> v[IPT][R];
#pragma unroll
    for (int u = 0; u < IPT; ++u) p2_load<T, N, B, R>(Xin, threadIdx.x + u * TH, v[u]);
#pragma unroll
    for (int u = 0; u < IPT; ++u) p2_butterfly<T, N, B, R, NS>(Xout, threadIdx.x + u * TH, v[u], tw);
  }
}

// Radix of the plan's stage with Ns = NS (radix 8 while it fits, then one radix-4 or radix-2
// stage), and of its last stage.
template <int N, int NS>
__host__ __device__ constexpr int p2_radix() {
  return (N / NS >= 8) ? 8 : (N / NS == 4 ? 4 : 2);
}
template <int N, int NS = 8>
__host__ __device__ constexpr int p2_last_radix() {
  if constexpr (NS * p2_radix<N, NS>() == N) return p2_radix<N, NS>();
  else return p2_last_radix<N, NS * p2_radix<N, NS>()>();
}

// The stages after the first (Ns = NS onwards), ping-ponging between two buffers, or in place
// in one (ONE); returns the result buffer. LAST: the last stage is left to the caller, and the
// buffer holding its input is returned.
template <typename T, int N, int B, int NS, int TH, bool ONE, bool LAST>
__device__ __forceinline__ cplx<T>* p2_rest(cplx<T>* in, cplx<T>* out, const cplx<T>* tw) {
  constexpr int R = p2_radix<N, NS>();
  if constexpr (NS == N || (LAST && NS * R == N)) {
    return in;
  } else {
    if constexpr (ONE) {
      p2_stage<T, N, B, R, NS, TH, true>(in, in, tw);
      __syncthreads();
      return p2_rest<T, N, B, NS * R, TH, true, LAST>(in, in, tw);
    } else {
      p2_stage<T, N, B, R, NS, TH, false>(in, out, tw);
      __syncthreads();
      return p2_rest<T, N, B, NS * R, TH, false, LAST>(out, in, tw);
    }
  }
}

// Forward last stage (radix R, Ns = N / R) fused with the unpack of the two real spectra of each
// pair: output r of butterfly j is bin k = j + r N/R, and its mirror N - k is output R - 1 - r of
// butterfly N/R - j (for j = 0, output (R - r) mod R of butterfly 0). The thread that transforms
// butterfly j also transforms N/R - j (butterflies 0 and N/(2R), their own mirrors, go
// together), so the unpack reads its two values from registers instead of the buffer. Needs
// two or more butterflies a thread (N/R B >= 2 TH).
template <typename T>
__device__ __forceinline__ void p2_emit_pair(cplx<T>* dst, cplx<T> u, cplx<T> w) {
  cplx<T> oa, ob;
  oa.x = T(0.5) * (u.x + w.x); oa.y = T(0.5) * (u.y - w.y);
  ob.x = T(0.5) * (u.y + w.y); ob.y = T(0.5) * (w.x - u.x);
  store_pair(dst, oa, ob);
}
template <typename T, int N, int B, int TH>
__device__ __forceinline__ void p2_last_unpack(const cplx<T>* __restrict__ X,
                                               const cplx<T>* __restrict__ tw,
                                               cplx<T>* __restrict__ dst, int K) {
  using C = cplx<T>;
  constexpr int R = p2_last_radix<N>();
  constexpr int NS = N / R;
  constexpr int UPT = NS * B / (2 * TH);
  static_assert(UPT >= 1 && NS * B % (2 * TH) == 0, "two or more butterflies a thread");
  const int b = threadIdx.x % B, p = threadIdx.x / B;
  dst += 2 * b;
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const int q = p + u * (TH / B);
    const int j1 = q, j2 = q == 0 ? NS / 2 : NS - q;
    C v1[R], v2[R];
    p2_load<T, N, B, R>(X, j1 * B + b, v1);
    p2_load<T, N, B, R>(X, j2 * B + b, v2);
    p2_twdft<T, N, B, R, NS>(j1 * B + b, v1, tw);
    p2_twdft<T, N, B, R, NS>(j2 * B + b, v2, tw);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k1 = j1 + r * NS, k2 = j2 + r * NS;
      if (k1 <= N / 2)
        p2_emit_pair<T>(dst + (size_t)k1 * K, v1[r], q == 0 ? v1[(R - r) % R] : v2[R - 1 - r]);
      if (k2 <= N / 2)
        p2_emit_pair<T>(dst + (size_t)k2 * K, v2[r], q == 0 ? v2[R - 1 - r] : v1[R - 1 - r]);
    }
  }
}

// Inverse last stage fused with the output: output r of butterfly (t, b) is pixel t + r N/R of
// pair b, written as conj(v) / N straight from registers.
template <typename T, int N, int B, int TH>
__device__ __forceinline__ void p2_last_store(const cplx<T>* __restrict__ X,
                                              const cplx<T>* __restrict__ tw,
                                              T* __restrict__ zrow, int K) {
  using C = cplx<T>;
  constexpr int R = p2_last_radix<N>();
  constexpr int NS = N / R;
  constexpr int IPT = NS * B / TH;
  static_assert(IPT >= 1 && NS * B % TH == 0, "whole butterflies per thread");
  const T inv = T(1) / T(N);
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int it = threadIdx.x + u * TH;
    const int t = it / B, b = it - t * B;
    C v[R];
    p2_load<T, N, B, R>(X, it, v);
    p2_twdft<T, N, B, R, NS>(it, v, tw);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T* d = zrow + (size_t)(t + r * NS) * K + 2 * b;
      if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float2*>(d) = make_float2(v[r].x * inv, -v[r].y * inv);
      else
        *reinterpret_cast<double2*>(d) = make_double2(v[r].x * inv, -v[r].y * inv);
    }
  }
}

// First stage (radix 8, Ns = 1, no twiddles) of sequence b of butterfly t from registers.
// With B <= 4 the residue of base = 8 B t + b modulo the pad period is at most b (or 8 for
// FP32, B = 1), so output r lies (r B) >> PadShift pad slots past base's: fixed offsets.
template <typename T, int N, int B>
__device__ __forceinline__ void p2_first(cplx<T> (&v)[8], int t, int b, cplx<T>* Xout) {
  static_assert(B == 1 || B == 2 || B == 4, "class pairs per CTA");
  Dft<8, cplx<T>>::run(v);
  cplx<T>* xo = Xout + px<T>(t * 8 * B + b);
#pragma unroll
  for (int r = 0; r < 8; ++r) xo[r * B + ((r * B) >> PadShift<T>::v)] = v[r];
}

// 2B consecutive values of type T (one class block of a pixel) as complex pairs.
template <typename T, int B>
__device__ __forceinline__ void p2_load_block(const T* __restrict__ src, cplx<T> (&c)[B]) {
  if constexpr (sizeof(T) * 2 * B >= 16) {
    constexpr int NV = sizeof(T) * 2 * B / 16;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(src) + v);
        c[2 * v] = mkc<T>(q.x, q.y);
        c[2 * v + 1] = mkc<T>(q.z, q.w);
      } else {
        const double2 q = __ldg(reinterpret_cast<const double2*>(src) + v);
        c[v] = mkc<T>(q.x, q.y);
      }
    }
  } else {  // FP32, B = 1: one 8-byte pair
    const float2 q = __ldg(reinterpret_cast<const float2*>(src));
    c[0] = mkc<T>(q.x, q.y);
  }
}

// One transform buffer, stages in place, for FP32 CTAs of N B / 8 = 1024 first-stage
// butterflies (2048-point rows with four class pairs, 4096-point rows with two): they take 512
// threads and half the shared memory, so that two CTAs share an SM and one CTA's loads overlap
// the other's transform. Other shapes ping-pong between two buffers.
template <typename T, int LOGN, int B>
__host__ __device__ constexpr bool p2_onebuf() {
  return sizeof(T) == 4 && (1 << LOGN) / 8 * B == 1024;
}
inline bool p2_onebuf_rt(size_t tsize, int N, int B) { return tsize == 4 && N / 8 * B == 1024; }

// Threads of a power-of-two row CTA: one first-stage butterfly of one sequence each (at most
// 1024; 512 with one buffer).
template <typename T, int LOGN, int B>
__host__ __device__ constexpr int p2_threads() {
  return p2_onebuf<T, LOGN, B>() ? 512
                                 : (((1 << LOGN) / 8 * B) > 1024 ? 1024 : ((1 << LOGN) / 8 * B));
}

template <typename T, int LOGN, int B>
__global__ void __launch_bounds__(p2_threads<T, LOGN, B>(), p2_onebuf<T, LOGN, B>() ? 2 : 0)
    k_row_forward_p2(const RowArgs<T> a) {
  using C = cplx<T>;
  constexpr int N = 1 << LOGN;
  constexpr int NB = N / 8;
  constexpr bool ONE = p2_onebuf<T, LOGN, B>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);
  C* Y = ONE ? X : X + padded_elems<T>((size_t)N * B);
  const int y = blockIdx.y;
  const int q0 = blockIdx.x * B;
  const int c0 = 2 * q0;
  const C* tw = a.pl.tw;
  pdl_wait();  // rhs / partials come from the previous kernel
  const int rb0 = a.src ? -1 : cover_row_base(a, a.covY[2 * y]);
  const int rb1 = a.src ? -1 : cover_row_base(a, a.covY[2 * y + 1]);
  const bool hy = rb1 >= 0;
  for (int it = threadIdx.x; it < NB * B; it += blockDim.x) {
    const int t = it / B, q = it - t * B;
    const int cq = c0 + 2 * q;              // the pair's classes cq, cq + 1
    C v[8];
    if (a.src) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        C c[1];
        p2_load_block<T, 1>(a.src + ((size_t)y * N + t + r * NB) * a.K + cq, c);
        v[r] = c[0];
      }
    } else if (!hy) {
      // a row with one vertical cover (most rows): p00 (+ p01) for all eight pixels, every
      // load issued before any sum, so that one memory latency covers the whole butterfly
      C c0[8], c1[8];
      bool hx[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int2 ox = __ldg(reinterpret_cast<const int2*>(a.offX) + t + r * NB);
        hx[r] = ox.y >= 0;
        const int o1 = hx[r] ? ox.y : ox.x;
        C e[1];
        p2_load_block<T, 1>(a.P + rb0 + ox.x + cq, e); c0[r] = e[0];
        p2_load_block<T, 1>(a.P + rb0 + o1 + cq, e);   c1[r] = e[0];
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = hx[r] ? cadd(c0[r], c1[r]) : c0[r];
    } else {
      // p00 (+ p01) (+ p10) (+ p11), the order of gather_row16. All loads of the butterfly
      // are issued before any sum (an absent cover aliases the first, its value is dropped),
      // so that they are in flight together.
      // (in two batches of four pixels, within 64 registers a thread)
      const int rb1a = rb1;
#pragma unroll
      for (int h = 0; h < 8; h += 4) {
        C c00[4], c01[4], c10[4], c11[4];
        bool hx[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int2 ox = __ldg(reinterpret_cast<const int2*>(a.offX) + t + (h + r) * NB);
          hx[r] = ox.y >= 0;
          const int o1 = hx[r] ? ox.y : ox.x;
          C e[1];
          p2_load_block<T, 1>(a.P + rb0 + ox.x + cq, e); c00[r] = e[0];
          p2_load_block<T, 1>(a.P + rb0 + o1 + cq, e);   c01[r] = e[0];
          p2_load_block<T, 1>(a.P + rb1a + ox.x + cq, e); c10[r] = e[0];
          p2_load_block<T, 1>(a.P + rb1a + o1 + cq, e);  c11[r] = e[0];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          C c = c00[r];
          if (hx[r]) c = cadd(c, c01[r]);
          if (hy) c = cadd(c, c10[r]);
          if (hy && hx[r]) c = cadd(c, c11[r]);
          v[h + r] = c;
        }
      }
    }
    p2_first<T, N, B>(v, t, q, Y);
  }
  __syncthreads();
  constexpr int TH = p2_threads<T, LOGN, B>();
  constexpr bool FUSE = N / p2_last_radix<N>() * B >= 2 * TH;
  const C* R = p2_rest<T, N, B, 8, TH, ONE, FUSE>(Y, X, tw);
  pdl_trigger();
  if constexpr (FUSE) {
    p2_last_unpack<T, N, B, TH>(R, tw, a.S + (size_t)y * a.Wh * a.K + 2 * q0, a.K);
  } else {
    // unpack the two real spectra of each pair (as k_row_forward)
    for (int i = threadIdx.x; i < (N / 2 + 1) * B; i += blockDim.x) {
      const int qq = i % B;
      const int kx = i / B;
      const C u = R[px<T>(kx * B + qq)];
      const C w = R[px<T>(((kx == 0) ? 0 : N - kx) * B + qq)];
      p2_emit_pair<T>(a.S + ((size_t)y * a.Wh + kx) * a.K + 2 * (q0 + qq), u, w);
    }
  }
}

template <typename T, int LOGN, int B>
__global__ void __launch_bounds__(p2_threads<T, LOGN, B>(), p2_onebuf<T, LOGN, B>() ? 2 : 0)
    k_row_inverse_p2(const RowArgs<T> a) {
  using C = cplx<T>;
  constexpr int N = 1 << LOGN;
  constexpr int NB = N / 8;
  constexpr int WH = N / 2 + 1;
  constexpr bool ONE = p2_onebuf<T, LOGN, B>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);
  C* Y = ONE ? X : X + padded_elems<T>((size_t)N * B);
  const int y = blockIdx.y;
  const int q0 = blockIdx.x * B;
  const C* tw = a.pl.tw;
  pdl_wait();  // the spectrum comes from the column pass
  const C* srow = a.S + (size_t)y * WH * a.K + 2 * q0;
  for (int it = threadIdx.x; it < NB * B; it += blockDim.x) {
    const int t = it / B, q = it - t * B;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      // bin kx = t + r N/8 of the full spectrum: stored for r < 4 (kx < N/2) and at kx = N/2
      // (r = 4, t = 0); the Hermitian mirror ks = N - kx (conjugated) for r > 4 and r = 4, t > 0
      const int ks = r < 4 ? t + r * NB : (r == 4 ? N / 2 - t : N - t - r * NB);
      const bool cj = r > 4 || (r == 4 && t > 0);
      C A, Bq;
      load_pair(srow + (size_t)ks * a.K + 2 * q, A, Bq);
      if (cj) { A = cconj(A); Bq = cconj(Bq); }
      C xv; xv.x = A.x - Bq.y; xv.y = -(A.y + Bq.x);   // conj(A + i B)
      v[r] = xv;
    }
    p2_first<T, N, B>(v, t, q, Y);
  }
  __syncthreads();
  constexpr int TH = p2_threads<T, LOGN, B>();
  const C* R = p2_rest<T, N, B, 8, TH, ONE, true>(Y, X, tw);
  pdl_trigger();
  p2_last_store<T, N, B, TH>(R, tw, a.z + (size_t)y * N * a.K + 2 * q0, a.K);
}

// Whether a row plan can run the power-of-two kernels: N = 2^LOGN with 256 <= N <= 4096, no
// Bluestein, B in {1, 2, 4}, every class block whole (K a multiple of 2B) and the caller's
// dense buffers (when used) aligned to the block's vector size.
inline int p2_log2(int N) {
  int l = 0;
  while ((1 << l) < N) ++l;
  return (1 << l) == N ? l : -1;
}
template <typename T>
inline bool p2_ok(int N, int blue, int QB, int K) {
  const int l = p2_log2(N);
  return !blue && l >= 8 && l <= 12 && (QB == 1 || QB == 2 || QB == 4) && K % (2 * QB) == 0;
}
template <typename T>
inline size_t p2_smem_bytes(int N, int QB) {
  return sizeof(cplx<T>) * (p2_onebuf_rt(sizeof(T), N, QB) ? 1 : 2) * padded_elems<T>((size_t)N * QB);
}

// ---------------------------------------------------------------- host-side launch helpers
struct RowLaunch {
  int threads;
  int tables;     // tables in shared memory
  size_t smem;
};

// Class pairs per CTA for a row transform of length Mf: a power of two, at most `max_elems`
// complex values a CTA (each of its two transform buffers); halved (down to 128 values a CTA)
// while the grid has fewer than eight CTAs per SM, so that small images spread over the GPU
// instead of running long per-CTA chains.
inline int row_pairs_per_cta(int Mf, int Q, int rows = 1 << 30, int max_elems = 4096,
                             bool trim = true) {
  int qb = 1;
  while (qb < Q && 2 * qb * Mf <= max_elems) qb *= 2;
  // at most a fifth of the pair slots of a row's CTAs empty (K = 9, five pairs: two a CTA, not
  // eight with three of them transformed for nothing; 610 x 340, 5x5: 326 -> 312 us per
  // iteration)
  while (trim && qb > 1 && (long long)((Q + qb - 1) / qb) * qb * 4 > 5LL * Q) qb /= 2;
  while (qb > 1 && (long long)rows * ((Q + qb - 1) / qb) < 2 * 152 && Mf * qb / 2 >= 128) qb /= 2;
  return qb;
}

inline uint32_t div_magic(int d) {
  return d <= 1 ? 0u : (uint32_t)(((1ULL << 32) + (unsigned long long)d - 1) / (unsigned long long)d);
}

// Column segments: rows per segment at least ceil(H / nseg), rounded up to 1 modulo the number
// of buffer rows that fill the 32 shared-memory banks, so that the segments one warp holds (32 /
// nseq of them, at the same step) sit in different banks; and the resulting segment count.
inline void col_segments(int H, int nseg, int nseq, int tbytes, int& SL, int& NSEG) {
  const int words = nseq * tbytes / 4;  // 4-byte words per buffer row
  const int q = words >= 32 ? 1 : 32 / words;
  int sl = (H + nseg - 1) / nseg;
  if (q > 1)
    while (sl % q != 1) ++sl;
  SL = sl;
  NSEG = (H + sl - 1) / sl;
}

// Largest prime factor handled by a direct Stockham stage; rows with a larger prime factor use
// Bluestein's transform. A direct stage costs about R / 2 multiply-adds per output; measured on
// one GB300 (z-update of 256 x W, K = 8, W = 2p), direct was faster up to p = 103 and
// Bluestein from p = 109 (p = 127: 45.0 vs 37.9 us).
constexpr int FFT_DIRECT_MAX = 103;

inline bool fft_smooth7(long n) {
  for (long r : {2L, 3L, 5L, 7L})
    while (n % r == 0) n /= r;
  return n == 1;
}

// Transform length and Stockham stages of a row of length N (direct prime stages first, then
// radices 8, 4, 2, 3, 5, 7); false when a stage table would overflow.
inline long largest_prime_factor(long n) {
  long best = 1;
  for (long p = 2; p * p <= n; ++p)
    while (n % p == 0) { best = p; n /= p; }
  return n > 1 ? (n > best ? n : best) : best;
}

template <typename T>
inline bool make_fft_plan(int N, FftPlan<T>& pl) {
  pl.N = N;
  if (largest_prime_factor(N) <= FFT_DIRECT_MAX) {
    pl.Mf = N;
    pl.blue = 0;
  } else {
    // Bluestein length: the 7-smooth length in [2N - 1, 4N] with the lowest modelled cost
    // (length x per-stage cost; radix-8 stages move the most data per barrier), which often
    // prefers a power of two over the shortest length (N = 202: 448 = 8 8 7 rather than
    // 405 = 3 3 3 3 5)
    auto cost = [](long m) {
      double c = 0.0;
      const long len = m;
      for (int r : {8, 4, 2, 3, 5, 7}) {
        const double cr = r == 8 ? 6.5 : r == 4 ? 4.0 : r == 2 ? 3.0 : r == 3 ? 5.0 : r == 5 ? 7.0 : 9.0;
        while (m % r == 0) { c += cr + 8.0; m /= r; }
      }
      return c * (double)len;
    };
    long best = 0;
    double bc = 0.0;
    for (long mm = 2L * N - 1; mm <= 4L * N; ++mm) {
      if (!fft_smooth7(mm)) continue;
      const double c = cost(mm);
      if (!best || c < bc) { best = mm; bc = c; }
    }
    pl.Mf = (int)best;
    pl.blue = 1;
  }
  int rest = pl.Mf, s = 0, ns = 1;
  auto push = [&](int r) {
    if (s >= FFT_MAXST) return;
    pl.radix[s] = r; pl.ns[s] = ns; pl.mg_ns[s] = div_magic(ns); pl.mg_nsr[s] = div_magic(ns * r);
    ns *= r; ++s; rest /= r;
  };
  // prime factors above 7 first: the first stage has Ns = 1, so a direct stage there needs no
  // inter-stage twiddles
  for (int p = 11; p <= FFT_DIRECT_MAX; p += 2)
    if (largest_prime_factor(p) == p)
      while (rest % p == 0) push(p);
  while (rest % 8 == 0) push(8);
  while (rest % 4 == 0) push(4);
  while (rest % 2 == 0) push(2);
  for (int p : {3, 5, 7})
    while (rest % p == 0) push(p);
  pl.nst = s;
  return rest == 1 && s <= FFT_MAXST;
}

template <typename T>
inline RowLaunch row_launch_config(int N, int Mf, int blue, int QB, int target_threads = 1024) {
  RowLaunch r{};
  // one radix-8 butterfly (eight values) per thread and stage; fewer threads loop. A direct
  // prime stage (prime factor 11 .. 103) sums (R - 1) / 2 terms per pair of outputs in
  // sequence: there, one thread per output pair keeps the chain short.
  const int elems = Mf * QB;
  const bool direct = !blue && largest_prime_factor(Mf) > 7;
  int t = ((direct ? elems / 2 : elems / 8) + 31) / 32 * 32;
  const int cap = std::min(target_threads, 1024);
  r.threads = t < 64 ? 64 : (t > cap ? cap : t);
  // tables in shared memory only while the CTA then stays within 72 KB: for long rows the
  // global (cached) tables let three CTAs share an SM (2048-long rows: 106 -> 74 KB, row
  // passes 14-16 % faster, measured)
  r.tables = row_smem_bytes<T>(N, Mf, blue, QB, 1) <= 72 * 1024;
  r.smem = row_smem_bytes<T>(N, Mf, blue, QB, r.tables);
  return r;
}

// Launchers of the row and column passes: defined (and instantiated for float and double) in
// fft_f32.cu / fft_f64.cu so that the many kernel variants compile in parallel. With
// pdl = false the row pass is an ordinary launch: it starts only after the previous kernel in
// the stream has completed (needed when that kernel wrote the transform tables, which the row
// pass copies before its programmatic-dependency wait).
template <typename T>
cudaError_t launch_row(bool forward, const RowArgs<T>& a, dim3 grid, const RowLaunch& rl,
                       cudaStream_t st, bool pdl = true);
template <typename T>
cudaError_t launch_col(const ColArgs<T>& a, int blocks, int threads, size_t smem, cudaStream_t st);
// Grant the dynamic shared memory of the row / column kernels of a plan before any launch.
template <typename T>
cudaError_t prepare_fft(const RowLaunch& rl, size_t col_smem);
// Pipelined row passes: launch on `grid` persistent CTAs of 256 threads, and the number of
// such CTAs one SM holds with `smem` bytes of dynamic shared memory (after granting it).
constexpr int ROWPIPE_THREADS = 256;
template <typename T>
cudaError_t launch_row_pipe(bool forward, const RowArgs<T>& a, int grid, size_t smem,
                            cudaStream_t st);
template <typename T>
cudaError_t row_pipe_blocks_per_sm(bool forward, size_t smem, int* blocks);
// The three passes in one launch (k_zupdate_seq) on `grid` CTAs; `grid` <= 0 only grants the
// shared memory and returns in *blocks the number of CTAs one SM holds.
template <typename T>
cudaError_t launch_zseq(const ZseqArgs<T>& a, int grid, int threads, size_t smem, cudaStream_t st,
                        int* blocks = nullptr);
// Power-of-two row passes (p2_ok): grid (class blocks, rows), N / 8 * QB threads (<= 1024).
template <typename T>
cudaError_t launch_row_p2(bool forward, const RowArgs<T>& a, dim3 grid, size_t smem,
                          cudaStream_t st);


#ifdef SGS_FFT_INSTANTIATE
template <typename T>
struct RowGrant {
  static SmemGrants f, i;
};
template <typename T> SmemGrants RowGrant<T>::f;
template <typename T> SmemGrants RowGrant<T>::i;
template <typename T>
struct ColGrant {
  static SmemGrants g;
};
template <typename T> SmemGrants ColGrant<T>::g;

template <typename T>
cudaError_t prepare_fft(const RowLaunch& rl, size_t col_smem) {
  cudaError_t e = grant_smem(k_row_forward<T>, rl.smem, RowGrant<T>::f);
  if (e != cudaSuccess) return e;
  if ((e = grant_smem(k_row_inverse<T>, rl.smem, RowGrant<T>::i)) != cudaSuccess) return e;
  return grant_smem(k_col_solve<T>, col_smem, ColGrant<T>::g);
}

template <typename T>
cudaError_t launch_row(bool forward, const RowArgs<T>& a, dim3 grid, const RowLaunch& rl,
                       cudaStream_t st, bool pdl) {
  cudaError_t e;
  if (forward) {
    if ((e = grant_smem(k_row_forward<T>, rl.smem, RowGrant<T>::f)) != cudaSuccess) return e;
    if (!pdl) {
      k_row_forward<T><<<grid, rl.threads, rl.smem, st>>>(a);
      return cudaGetLastError();
    }
    return launch_pdl(k_row_forward<T>, grid, dim3(rl.threads), rl.smem, st, a);
  }
  if ((e = grant_smem(k_row_inverse<T>, rl.smem, RowGrant<T>::i)) != cudaSuccess) return e;
  if (!pdl) {
    k_row_inverse<T><<<grid, rl.threads, rl.smem, st>>>(a);
    return cudaGetLastError();
  }
  return launch_pdl(k_row_inverse<T>, grid, dim3(rl.threads), rl.smem, st, a);
}

template <typename T>
struct ZseqGrant {
  static SmemGrants g;
};
template <typename T> SmemGrants ZseqGrant<T>::g;

template <typename T>
cudaError_t launch_zseq(const ZseqArgs<T>& a, int grid, int threads, size_t smem, cudaStream_t st,
                        int* blocks) {
  cudaError_t e = grant_smem(k_zupdate_seq<T>, smem, ZseqGrant<T>::g);
  if (e != cudaSuccess) return e;
  if (grid <= 0) {
    *blocks = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_zupdate_seq<T>, threads, smem);
  }
  return launch_pdl(k_zupdate_seq<T>, dim3(grid), dim3(threads), smem, st, a);
}

template <typename T>
struct RowPipeGrant {
  static SmemGrants f, i;
};
template <typename T> SmemGrants RowPipeGrant<T>::f;
template <typename T> SmemGrants RowPipeGrant<T>::i;

template <typename T>
cudaError_t launch_row_pipe(bool forward, const RowArgs<T>& a, int grid, size_t smem,
                            cudaStream_t st) {
  cudaError_t e;
  if (forward) {
    if ((e = grant_smem(k_row_forward_pipe<T>, smem, RowPipeGrant<T>::f)) != cudaSuccess) return e;
    return launch_pdl(k_row_forward_pipe<T>, dim3(grid), dim3(ROWPIPE_THREADS), smem, st, a);
  }
  if ((e = grant_smem(k_row_inverse_pipe<T>, smem, RowPipeGrant<T>::i)) != cudaSuccess) return e;
  return launch_pdl(k_row_inverse_pipe<T>, dim3(grid), dim3(ROWPIPE_THREADS), smem, st, a);
}

template <typename T>
cudaError_t row_pipe_blocks_per_sm(bool forward, size_t smem, int* blocks) {
  cudaError_t e;
  *blocks = 0;
  if (forward) {
    if ((e = grant_smem(k_row_forward_pipe<T>, smem, RowPipeGrant<T>::f)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_row_forward_pipe<T>,
                                                         ROWPIPE_THREADS, smem);
  }
  if ((e = grant_smem(k_row_inverse_pipe<T>, smem, RowPipeGrant<T>::i)) != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_row_inverse_pipe<T>,
                                                       ROWPIPE_THREADS, smem);
}

template <typename T, int LOGN, int B>
struct RowP2Grant {
  static SmemGrants f, i;
};
template <typename T, int LOGN, int B> SmemGrants RowP2Grant<T, LOGN, B>::f;
template <typename T, int LOGN, int B> SmemGrants RowP2Grant<T, LOGN, B>::i;

template <typename T, int LOGN, int B>
cudaError_t launch_row_p2_inst(bool forward, const RowArgs<T>& a, dim3 grid, size_t smem,
                               cudaStream_t st) {
  cudaError_t e;
  if (forward) {
    if ((e = grant_smem(k_row_forward_p2<T, LOGN, B>, smem, RowP2Grant<T, LOGN, B>::f)) != cudaSuccess)
      return e;
    return launch_pdl(k_row_forward_p2<T, LOGN, B>, grid, dim3(p2_threads<T, LOGN, B>()), smem, st, a);
  }
  if ((e = grant_smem(k_row_inverse_p2<T, LOGN, B>, smem, RowP2Grant<T, LOGN, B>::i)) != cudaSuccess)
    return e;
  return launch_pdl(k_row_inverse_p2<T, LOGN, B>, grid, dim3(p2_threads<T, LOGN, B>()), smem, st, a);
}

template <typename T, int LOGN>
cudaError_t launch_row_p2_b(bool forward, const RowArgs<T>& a, dim3 grid, size_t smem,
                            cudaStream_t st) {
  switch (a.QB) {
    case 1: return launch_row_p2_inst<T, LOGN, 1>(forward, a, grid, smem, st);
    case 2: return launch_row_p2_inst<T, LOGN, 2>(forward, a, grid, smem, st);
    case 4: return launch_row_p2_inst<T, LOGN, 4>(forward, a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_row_p2(bool forward, const RowArgs<T>& a, dim3 grid, size_t smem,
                          cudaStream_t st) {
  switch (p2_log2(a.pl.N)) {
    case 8: return launch_row_p2_b<T, 8>(forward, a, grid, smem, st);
    case 9: return launch_row_p2_b<T, 9>(forward, a, grid, smem, st);
    case 10: return launch_row_p2_b<T, 10>(forward, a, grid, smem, st);
    case 11: return launch_row_p2_b<T, 11>(forward, a, grid, smem, st);
    case 12: return launch_row_p2_b<T, 12>(forward, a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_col(const ColArgs<T>& a, int blocks, int threads, size_t smem,
                              cudaStream_t st) {
  cudaError_t e = grant_smem(k_col_solve<T>, smem, ColGrant<T>::g);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_col_solve<T>, dim3(blocks), dim3(threads), smem, st, a);
}

#else
extern template cudaError_t launch_row<float>(bool, const RowArgs<float>&, dim3, const RowLaunch&, cudaStream_t, bool);
extern template cudaError_t launch_row<double>(bool, const RowArgs<double>&, dim3, const RowLaunch&, cudaStream_t, bool);
extern template cudaError_t launch_col<float>(const ColArgs<float>&, int, int, size_t, cudaStream_t);
extern template cudaError_t launch_col<double>(const ColArgs<double>&, int, int, size_t, cudaStream_t);
extern template cudaError_t prepare_fft<float>(const RowLaunch&, size_t);
extern template cudaError_t prepare_fft<double>(const RowLaunch&, size_t);
extern template cudaError_t launch_row_pipe<float>(bool, const RowArgs<float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_row_pipe<double>(bool, const RowArgs<double>&, int, size_t, cudaStream_t);
extern template cudaError_t row_pipe_blocks_per_sm<float>(bool, size_t, int*);
extern template cudaError_t row_pipe_blocks_per_sm<double>(bool, size_t, int*);
extern template cudaError_t launch_row_p2<float>(bool, const RowArgs<float>&, dim3, size_t, cudaStream_t);
extern template cudaError_t launch_row_p2<double>(bool, const RowArgs<double>&, dim3, size_t, cudaStream_t);

#endif

}  // namespace sgs
