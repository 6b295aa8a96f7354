// z-update (12) in one launch: passes A, B and C of fft.cuh fused over a thread-block cluster.
//
// A cluster of CS CTAs takes QG class pairs of the whole image; CTA r of the cluster owns the
// band of rows [floor(r H / CS), floor((r + 1) H / CS)). Each CTA
//   A  gathers rhs for its rows and transforms them along x (two classes per complex
//      sequence, all rows of the band and all pairs of the group in one batched transform),
//      keeping the half spectra in its own shared memory;
//   B  solves the column systems along y for every (kx, class) column with the causal and
//      anti-causal first-order recursions of fft.cuh, its band being one segment: the start
//      value of a segment is the geometric sum over the nwarm rows before it (after it, for
//      the anti-causal pass), read from the neighbouring CTAs' shared memory through the
//      cluster's distributed shared memory; four cluster barriers order the start-value reads
//      against the in-place recursions of the other bands;
//   C  transforms its rows back and writes z.
// The spectrum never leaves the SMs. The arithmetic of each element is that of the three-pass
// path (same transforms, same recursions, segments at the band boundaries).
// Measured on one GB300 it is slower than the three launches at every shape tried (64 x 64 to
// 256 x 256, K = 4..16): a cluster holds one class pair, so an image of Q pairs gives only
// Q x CS CTAs for the transforms, and the start-value reads through distributed shared memory
// cost several microseconds per pass. It is therefore selected only on request (zfuse).
#pragma once

#include <cooperative_groups.h>

#include "fft.cuh"

namespace sgs {

template <typename T>
struct ZfArgs {
  RowArgs<T> r;          // image shape, rhs source (dense or tile partials), FFT plan, z output
  const T* beta;         // [Wh] column recursion coefficients (as for k_col_solve)
  const T* gain;         // [Wh]
  const T* wfac;         // [Wh]
  const int* nwarm;      // [Wh]
  int CS;                // CTAs per cluster = row bands
  int QG;                // class pairs per cluster
  int RMAX;              // rows of the tallest band, ceil(H / CS)
  uint32_t mgB;          // ceil(2^32 / (RMAX QG))
};

// Shared memory of a fused CTA: two transform buffers, the tables, the horizontal offsets of the
// tile partials, the per-row vertical cover bases, the band's half spectra (as real sequences)
// and one start value per sequence.
template <typename T>
__host__ __device__ inline size_t zf_smem_bytes(int N, int Mf, int blue, int Wh, int RMAX, int QG,
                                                int tables) {
  const size_t B = (size_t)RMAX * QG;
  const size_t nseq = (size_t)Wh * 4 * QG;
  return sizeof(cplx<T>) * 2 * padded_elems<T>((size_t)Mf * B) +
         (tables ? fft_table_bytes<T>(N, Mf, blue) : 0) + sizeof(int) * 2 * (size_t)N +
         sizeof(int) * 2 * (size_t)RMAX + sizeof(T) * (RMAX + 1) * nseq;
}

// Band of row n: the largest r with floor(r H / CS) <= n.
__device__ __forceinline__ int zf_owner(int n, int H, int CS) { return ((n + 1) * CS - 1) / H; }

template <typename T>
__global__ void __launch_bounds__(512) k_zfused(const ZfArgs<T> a) {
  using C = cplx<T>;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RowArgs<T>& ra = a.r;
  const int H = ra.H, W = ra.W, K = ra.K, Wh = ra.Wh, N = ra.pl.N, Mf = ra.pl.Mf;
  const int CS = a.CS, QG = a.QG;
  const int rank = (int)cluster.block_rank();
  const int grp = blockIdx.x / CS;
  const int q0 = grp * QG;                        // first class pair of the group
  const int y0 = (int)(((long long)rank * H) / CS);
  const int y1 = (int)(((long long)(rank + 1) * H) / CS);
  const int R = y1 - y0;
  const int B = a.RMAX * QG;                      // sequences: b = row * QG + pair
  const int nseq = Wh * 4 * QG;                   // real sequences: (kx, class, re/im)
  C* X = reinterpret_cast<C*>(smem_raw);
  C* Y = X + padded_elems<T>((size_t)Mf * B);
  C* tab = Y + padded_elems<T>((size_t)Mf * B);
  int* cX = reinterpret_cast<int*>(
      tab + (ra.smem_tables ? fft_table_bytes<T>(N, Mf, ra.pl.blue) / sizeof(C) : 0));
  int* rbs = cX + 2 * N;                          // [RMAX][2] vertical cover bases
  T* Sp = reinterpret_cast<T*>(rbs + 2 * a.RMAX);  // [RMAX][nseq]
  T* start = Sp + (size_t)a.RMAX * nseq;          // [nseq]
  const FftTables<T> tb = row_tables<T>(ra, tab);
  if (!ra.src) {
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) cp_async_zfill<4>(cX + i, ra.offX + i, true);
    for (int i = threadIdx.x; i < 2 * a.RMAX; i += blockDim.x) {
      const int rr = i >> 1;
      rbs[i] = rr < R ? cover_row_base(ra, ra.covY[2 * (y0 + rr) + (i & 1)]) : -1;
    }
  }
  cp_async_commit();
  pdl_wait();  // rhs / partials come from the previous kernel
  cp_async_wait_all();
  __syncthreads();

  // ---- A: rhs of the band, forward transforms along x. Element order (row, x, pair, re/im):
  // consecutive threads read consecutive classes and pixels of one row.
  {
    constexpr int U = 8;
    T* Xf = reinterpret_cast<T*>(X);
    const int tot = R * N * QG * 2;
    for (int i0 = threadIdx.x; i0 < tot; i0 += U * blockDim.x) {
      T v[U];
      int dst[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * blockDim.x;
        v[u] = T(0);
        dst[u] = -1;
        if (i < tot) {
          const int part = i & 1;
          const int t = i >> 1;
          const int qq = t % QG, rx = t / QG;
          const int rr = rx / N, x = rx - rr * N;
          const int k = 2 * (q0 + qq) + part;
          dst[u] = 2 * px<T>(x * B + rr * QG + qq) + part;
          if (k < K)
            v[u] = ra.src ? ra.src[((size_t)(y0 + rr) * W + x) * K + k]
                          : gather_row<T>(ra.P, rbs[2 * rr], rbs[2 * rr + 1], cX, x, k);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dst[u] >= 0) Xf[dst[u]] = v[u];
    }
    // rows of a shorter band: zero sequences
    for (int i = threadIdx.x; i < (a.RMAX - R) * N * QG; i += blockDim.x) {
      const int qq = i % QG, rx = i / QG;
      const int rr = R + rx / N, x = rx % N;
      X[px<T>(x * B + rr * QG + qq)] = mkc<T>(T(0), T(0));
    }
  }
  __syncthreads();
  {
    const C* Rb = dft_rows<T>(X, Y, B, a.mgB, ra.pl, tb);
    // half spectra of the two classes of each sequence, column (kx, class c = 2 qq + part);
    // element order (row, pair, kx, re/im)
    for (int i = threadIdx.x; i < R * QG * Wh * 2; i += blockDim.x) {
      const int part = i & 1;
      const int t = i >> 1;
      const int kx = t % Wh, rq = t / Wh;
      const int qq = rq % QG, rr = rq / QG;
      const int b = rr * QG + qq;
      const C u = dft_out<T>(Rb, B, kx, b, ra.pl, tb);
      const C w = dft_out<T>(Rb, B, (kx == 0) ? 0 : N - kx, b, ra.pl, tb);
      C o;
      if (part == 0) { o.x = T(0.5) * (u.x + w.x); o.y = T(0.5) * (u.y - w.y); }
      else           { o.x = T(0.5) * (u.y + w.y); o.y = T(0.5) * (w.x - u.x); }
      const int sq = 2 * (kx * 2 * QG + 2 * qq + part);
      Sp[(size_t)rr * nseq + sq] = o.x;
      Sp[(size_t)rr * nseq + sq + 1] = o.y;
    }
  }
  cluster.sync();  // every band's spectrum is complete

  // ---- B: column recursions, one segment per band
  // sum over m = nw .. 1 of beta^(m-1) v(n_m) for the rows n_nw, n_nw + step, ... (mod H) of
  // sequence s, read from the bands that own them (eight loads in flight per thread)
  auto warm = [&](int n, int step, int nw, int s, T beta) -> T {
    constexpr int U = 8;
    T acc = T(0);
    for (int m0 = nw; m0 >= 1; m0 -= U) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        v[u] = T(0);
        if (m0 - u >= 1) {
          const int o = zf_owner(n, H, CS);
          const int oy0 = (int)(((long long)o * H) / CS);
          v[u] = cluster.map_shared_rank(Sp, o)[(size_t)(n - oy0) * nseq + s];
        }
        n += step;
        n += (n < 0) ? H : 0;
        n -= (n >= H) ? H : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (m0 - u >= 1) acc = beta * acc + v[u];
    }
    return acc;
  };
  for (int s = threadIdx.x; s < nseq; s += blockDim.x) {
    const int kx = s / (4 * QG);
    const int nw = a.nwarm[kx];
    // causal start value y_{y0-1} = sum_m beta^(m-1) r_{y0-m}, m = 1 .. nw
    int n = y0 - nw;
    n += (n < 0) ? H : 0;
    start[s] = warm(n, 1, nw, s, a.beta[kx]) * a.wfac[kx];
  }
  cluster.sync();  // all start values read before any band overwrites its rows
  for (int s = threadIdx.x; s < nseq; s += blockDim.x) {
    const T beta = a.beta[s / (4 * QG)];
    T acc = start[s];
    for (int rr = 0; rr < R; ++rr) {
      acc = beta * acc + Sp[(size_t)rr * nseq + s];
      Sp[(size_t)rr * nseq + s] = acc;
    }
  }
  cluster.sync();  // causal outputs complete in every band
  for (int s = threadIdx.x; s < nseq; s += blockDim.x) {
    const int kx = s / (4 * QG);
    const int nw = a.nwarm[kx];
    // anti-causal start value q_{y1} = sum_m beta^(m-1) y_{y1-1+m}, m = 1 .. nw
    int n = y1 - 1 + nw;
    n -= (n >= H) ? H : 0;
    start[s] = warm(n, -1, nw, s, a.beta[kx]) * a.wfac[kx];
  }
  cluster.sync();  // no band reads another band's shared memory after this point
  for (int s = threadIdx.x; s < nseq; s += blockDim.x) {
    const int kx = s / (4 * QG);
    const T beta = a.beta[kx], gain = a.gain[kx];
    T acc = start[s];
    for (int rr = R - 1; rr >= 0; --rr) {
      acc = beta * acc + Sp[(size_t)rr * nseq + s];
      Sp[(size_t)rr * nseq + s] = gain * acc;
    }
  }
  __syncthreads();

  // ---- C: inverse transforms of the band's rows, z. Loads in order (row, pair, kx).
  for (int e = threadIdx.x; e < a.RMAX * QG * N; e += blockDim.x) {
    const int kx = e % N, rq = e / N;
    const int qq = rq % QG, rr = rq / QG;
    const int ks = kx < Wh ? kx : N - kx;
    C A = mkc<T>(T(0), T(0)), Bq = A;
    if (rr < R) {
      const T* row = Sp + (size_t)rr * nseq + 2 * (ks * 2 * QG + 2 * qq);
      if (2 * (q0 + qq) < K) A = mkc<T>(row[0], row[1]);
      if (2 * (q0 + qq) + 1 < K) Bq = mkc<T>(row[2], row[3]);
    }
    if (kx >= Wh) { A = cconj(A); Bq = cconj(Bq); }
    C xv;
    xv.x = A.x - Bq.y;
    xv.y = -(A.y + Bq.x);  // conj(A + i B)
    X[px<T>(kx * B + rr * QG + qq)] = xv;
  }
  __syncthreads();
  const C* Rb = dft_rows<T>(X, Y, B, a.mgB, ra.pl, tb);
  pdl_trigger();
  // stores in order (row, x, pair, re/im): consecutive classes and pixels of one row
  const T inv = T(1) / T(N);
  for (int i = threadIdx.x; i < R * N * QG * 2; i += blockDim.x) {
    const int part = i & 1;
    const int t = i >> 1;
    const int qq = t % QG, rx = t / QG;
    const int rr = rx / N, x = rx - rr * N;
    const int k = 2 * (q0 + qq) + part;
    if (k >= K) continue;
    const C v = dft_out<T>(Rb, B, x, rr * QG + qq, ra.pl, tb);  // DFT(conj X)_x ; z = conj(v) / N
    ra.z[((size_t)(y0 + rr) * W + x) * K + k] = (part == 0) ? v.x * inv : -v.y * inv;
  }
}

// Launcher (clusters of a.CS CTAs, programmatic dependent launch; groups = class-pair groups)
// and the number of such clusters that can be resident at once (0: the shape cannot run).
// Defined and instantiated in fft_f32.cu / fft_f64.cu.
template <typename T>
cudaError_t launch_zfused(const ZfArgs<T>& a, int groups, int threads, size_t smem,
                          cudaStream_t st);
template <typename T>
int zfused_max_clusters(int CS, int threads, size_t smem);

#ifdef SGS_FFT_INSTANTIATE
template <typename T>
struct ZfGrant {
  static SmemGrants g;
};
template <typename T> SmemGrants ZfGrant<T>::g;

template <typename T>
static cudaError_t zfused_attrs(int CS, size_t smem) {
  cudaError_t e = grant_smem(k_zfused<T>, smem, ZfGrant<T>::g);
  if (e != cudaSuccess) return e;
  // clusters above the portable size of 8: set on every call (the attribute belongs to the
  // current device's context, and the fused form is an opt-in path)
  if (CS > 8)
    return cudaFuncSetAttribute(k_zfused<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_zfused(const ZfArgs<T>& a, int groups, int threads, size_t smem,
                          cudaStream_t st) {
  cudaError_t e = zfused_attrs<T>(a.CS, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(groups * a.CS);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = a.CS;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_zfused<T>, a);
}

template <typename T>
int zfused_max_clusters(int CS, int threads, size_t smem) {
  if (zfused_attrs<T>(CS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_zfused<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
#else
extern template cudaError_t launch_zfused<float>(const ZfArgs<float>&, int, int, size_t, cudaStream_t);
extern template cudaError_t launch_zfused<double>(const ZfArgs<double>&, int, int, size_t, cudaStream_t);
extern template int zfused_max_clusters<float>(int, int, size_t);
extern template int zfused_max_clusters<double>(int, int, size_t);
#endif

}  // namespace sgs
