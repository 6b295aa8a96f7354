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

#include "common.cuh"

namespace sgs {

constexpr int FFT_MAXST = 24;
constexpr int FFT_MAXE = 16;  // complex values held per thread per stage

template <typename T>
struct FftPlan {
  int N;        // row length W
  int Mf;       // transform length run: N, or the Bluestein length
  int blue;     // 1 when Bluestein is used
  int nst;      // number of Stockham stages
  int radix[FFT_MAXST];
  int ns[FFT_MAXST];     // product of the radices before this stage
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

template <int R, typename C> struct DftOdd {
  __device__ __forceinline__ static void run(C* v) {
    using T = decltype(v[0].x);
    C in[R];
#pragma unroll
    for (int r = 0; r < R; ++r) in[r] = v[r];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      C acc = in[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int q = (r * m) % R;
        const T cr = T(root_cos(R, q)), sr = T(root_sin(R, q));
        // in[r] * exp(-2 pi i q / R)
        acc.x += in[r].x * cr + in[r].y * sr;
        acc.y += in[r].y * cr - in[r].x * sr;
      }
      v[m] = acc;
    }
  }
};
template <typename C> struct Dft<3, C> : DftOdd<3, C> {};
template <typename C> struct Dft<5, C> : DftOdd<5, C> {};
template <typename C> struct Dft<7, C> : DftOdd<7, C> {};

// One forward Stockham stage on B interleaved sequences X[n * B + b] (in place: every thread
// reads its inputs, the block synchronises, then writes).
template <typename T, int R>
__device__ __forceinline__ void fft_stage(cplx<T>* X, int B, int Mf, int Ns,
                                          const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int MI = (FFT_MAXE + R - 1) / R;
  const int nb = Mf / R;
  const int items = nb * B;
  const int stride = Mf / (Ns * R);
  C out[MI][R];
  int base[MI];
#pragma unroll
  for (int q = 0; q < MI; ++q) {
    const int it = threadIdx.x + q * blockDim.x;
    base[q] = -1;
    if (it < items) {
      const int b = it % B, t = it / B;
      const int j = t % Ns;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = X[(t + r * nb) * B + b];
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * j * stride]);
      Dft<R, C>::run(v);
#pragma unroll
      for (int r = 0; r < R; ++r) out[q][r] = v[r];
      base[q] = ((t / Ns) * Ns * R + j) * B + b;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MI; ++q) {
    if (base[q] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) X[base[q] + r * Ns * B] = out[q][r];
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void fft_forward(cplx<T>* X, int B, const FftPlan<T>& pl) {
  for (int s = 0; s < pl.nst; ++s) {
    const int Ns = pl.ns[s];
    switch (pl.radix[s]) {
      case 8: fft_stage<T, 8>(X, B, pl.Mf, Ns, pl.tw); break;
      case 4: fft_stage<T, 4>(X, B, pl.Mf, Ns, pl.tw); break;
      case 2: fft_stage<T, 2>(X, B, pl.Mf, Ns, pl.tw); break;
      case 3: fft_stage<T, 3>(X, B, pl.Mf, Ns, pl.tw); break;
      case 5: fft_stage<T, 5>(X, B, pl.Mf, Ns, pl.tw); break;
      case 7: fft_stage<T, 7>(X, B, pl.Mf, Ns, pl.tw); break;
    }
  }
}

// Forward DFT of length N of the B sequences in X (slots [0, N) filled, Bluestein slots
// [N, Mf) need not be). Afterwards X[k*B + b], k < N, holds X_k for the mixed-radix path; for
// Bluestein the caller reads bluestein_out(k).
template <typename T>
__device__ void dft_rows(cplx<T>* X, int B, const FftPlan<T>& pl) {
  using C = cplx<T>;
  if (!pl.blue) {
    fft_forward<T>(X, B, pl);
    return;
  }
  // a_n = x_n conj(chirp_n), zero padded
  for (int i = threadIdx.x; i < pl.Mf * B; i += blockDim.x) {
    const int n = i / B;
    X[i] = (n < pl.N) ? cmulc(X[i], pl.chirp[n]) : mkc<T>(T(0), T(0));
  }
  __syncthreads();
  fft_forward<T>(X, B, pl);
  for (int i = threadIdx.x; i < pl.Mf * B; i += blockDim.x)
    X[i] = cconj(cmul(X[i], pl.bhat[i / B]));
  __syncthreads();
  fft_forward<T>(X, B, pl);  // = conj(cyclic convolution)
}

// Value X_k after dft_rows.
template <typename T>
__device__ __forceinline__ cplx<T> dft_out(const cplx<T>* X, int B, int k, int b,
                                           const FftPlan<T>& pl) {
  const cplx<T> v = X[k * B + b];
  if (!pl.blue) return v;
  return cconj(cmul(pl.chirp[k], v));  // conj(chirp_k) * (a * b)_k
}

// ------------------------------------------------------------------- pass A (forward rows)
template <typename T>
struct RowArgs {
  int H, W, K, Wh;       // Wh = W/2 + 1 stored frequencies
  int QB;                // class pairs per CTA
  FftPlan<T> pl;
  // source of rhs: dense [n][K] (src != null) or the sweep partials
  const T* src;
  const T* P;            // [tiles][EHmax][EWmax][K]
  int ntx, EHmax, EWmax;
  const int* covY;       // [H][2]: (tile row << 16 | ext row), -1 when absent
  const int* covX;       // [W][2]: (tile col << 16 | ext col)
  cplx<T>* S;            // [H][Wh][K]
  T* z;                  // pass C output [n][K]
};

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

template <typename T>
__global__ void __launch_bounds__(512) k_row_forward(const RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);
  const int y = blockIdx.x;
  const int q0 = blockIdx.y * a.QB;
  const int B = a.QB;
  const int N = a.pl.N;
  T* Xf = reinterpret_cast<T*>(X);
  // load: two classes per complex sequence (real part class 2q, imaginary part class 2q+1)
  for (int i = threadIdx.x; i < N * B * 2; i += blockDim.x) {
    const int part = i & 1;
    const int qq = (i >> 1) % B;
    const int x = (i >> 1) / B;
    const int k = 2 * (q0 + qq) + part;
    Xf[i] = (k < a.K) ? gather_rhs(a, y, x, k) : T(0);
  }
  __syncthreads();
  dft_rows<T>(X, B, a.pl);
  // unpack the two real spectra: A = (X_k + conj X_{N-k})/2, B = (X_k - conj X_{N-k})/(2i)
  for (int i = threadIdx.x; i < a.Wh * B * 2; i += blockDim.x) {
    const int part = i & 1;
    const int qq = (i >> 1) % B;
    const int kx = (i >> 1) / B;
    const int k = 2 * (q0 + qq) + part;
    if (k >= a.K) continue;
    const C u = dft_out<T>(X, B, kx, qq, a.pl);
    const C w = dft_out<T>(X, B, (kx == 0) ? 0 : N - kx, qq, a.pl);
    C o;
    if (part == 0) { o.x = T(0.5) * (u.x + w.x); o.y = T(0.5) * (u.y - w.y); }
    else           { o.x = T(0.5) * (u.y + w.y); o.y = T(0.5) * (w.x - u.x); }
    a.S[((size_t)y * a.Wh + kx) * a.K + k] = o;
  }
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
template <typename T>
__global__ void __launch_bounds__(512) k_row_inverse(const RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);
  const int y = blockIdx.x;
  const int q0 = blockIdx.y * a.QB;
  const int B = a.QB;
  const int N = a.pl.N;
  // load conj(A + iB) over the full frequency range (Hermitian extension), inverse DFT by
  // conj(DFT(conj(.)))/N
  for (int i = threadIdx.x; i < N * B; i += blockDim.x) {
    const int qq = i % B;
    const int kx = i / B;
    const int ka = 2 * (q0 + qq), kb = ka + 1;
    const bool lo = kx < a.Wh;
    const int ks = lo ? kx : N - kx;
    const C* row = a.S + ((size_t)y * a.Wh + ks) * a.K;
    C A = (ka < a.K) ? row[ka] : mkc<T>(T(0), T(0));
    C Bv = (kb < a.K) ? row[kb] : mkc<T>(T(0), T(0));
    if (!lo) { A = cconj(A); Bv = cconj(Bv); }
    // X = A + i B; store conj(X)
    C xv; xv.x = A.x - Bv.y; xv.y = -(A.y + Bv.x);
    X[i] = xv;
  }
  __syncthreads();
  dft_rows<T>(X, B, a.pl);
  const T inv = T(1) / T(N);
  for (int i = threadIdx.x; i < N * B * 2; i += blockDim.x) {
    const int part = i & 1;
    const int qq = (i >> 1) % B;
    const int x = (i >> 1) / B;
    const int k = 2 * (q0 + qq) + part;
    if (k >= a.K) continue;
    const C v = dft_out<T>(X, B, x, qq, a.pl);     // DFT(conj X)_x ; result = conj(v)/N
    a.z[((size_t)y * a.W + x) * a.K + k] = (part == 0) ? v.x * inv : -v.y * inv;
  }
}

// ------------------------------------------------------------------ pass B (column solve)
template <typename T>
struct ColArgs {
  int H, C;              // rows, complex columns per row (Wh*K)
  int K;
  int CB;                // complex columns per CTA
  int NSEG;              // segments along y
  const T* beta;         // [Wh]
  const T* gain;         // [Wh]
  const T* wfac;         // [Wh] 1 or 1/(1 - beta^H)
  const int* nwarm;      // [Wh]
  cplx<T>* S;            // [H][C]
};

template <typename T>
__global__ void __launch_bounds__(1024) k_col_solve(const ColArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);  // [H][2*CB]
  const int c0 = blockIdx.x * a.CB;
  const int nseq = 2 * a.CB;
  const int H = a.H;
  T* Sf = reinterpret_cast<T*>(a.S);
  for (int i = threadIdx.x; i < H * nseq; i += blockDim.x) {
    const int y = i / nseq, s = i % nseq;
    const int col2 = 2 * c0 + s;
    buf[i] = (col2 < 2 * a.C) ? Sf[(size_t)y * 2 * a.C + col2] : T(0);
  }
  __syncthreads();
  const int s = threadIdx.x % nseq, seg = threadIdx.x / nseq;
  const bool act = seg < a.NSEG;
  const int c = c0 + s / 2;
  const int kx = (c < a.C) ? c / a.K : 0;
  const T beta = a.beta[kx], gain = a.gain[kx], wf = a.wfac[kx];
  const int nw = a.nwarm[kx];
  const int s0 = act ? (int)(((long long)seg * H) / a.NSEG) : 0;
  const int s1 = act ? (int)(((long long)(seg + 1) * H) / a.NSEG) : 0;
  // causal start value y_{s0-1} = sum_m beta^m r_{s0-1-m}
  T acc = T(0);
  if (act) {
    for (int m = nw; m >= 1; --m) acc = beta * acc + buf[wrap_idx(s0 - m, H) * nseq + s];
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
    for (int m = nw; m >= 1; --m) acc2 = beta * acc2 + buf[wrap_idx(s1 - 1 + m, H) * nseq + s];
    acc2 *= wf;
  }
  __syncthreads();
  if (act)
    for (int n = s1 - 1; n >= s0; --n) {
      acc2 = beta * acc2 + buf[n * nseq + s];
      buf[n * nseq + s] = gain * acc2;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < H * nseq; i += blockDim.x) {
    const int y = i / nseq, ss = i % nseq;
    const int col2 = 2 * c0 + ss;
    if (col2 < 2 * a.C) Sf[(size_t)y * 2 * a.C + col2] = buf[i];
  }
}

}  // namespace sgs
