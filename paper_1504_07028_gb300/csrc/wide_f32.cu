// FLOAT instantiations of the wide-patch sweep (k_wide_gram, k_wide_jt) and their launchers.
#include <algorithm>

#include "wide.cuh"

namespace sgs {

template <int G, bool DIAG, bool SIMP>
struct WideGramGrant { static SmemGrants g; };
template <int G, bool DIAG, bool SIMP> SmemGrants WideGramGrant<G, DIAG, SIMP>::g;

template <int G, bool DIAG>
struct WideJtGrant { static SmemGrants g; };
template <int G, bool DIAG> SmemGrants WideJtGrant<G, DIAG>::g;

template <int G, bool DIAG, bool SIMP>
static cudaError_t wide_g(const WideArgs<float>& a, cudaStream_t st) {
  const size_t s1 = wide_gram_smem<float>(a.M, G), s2 = wide_jt_smem<float>(a.M, G);
  cudaError_t e = grant_smem(k_wide_gram<float, G, DIAG, SIMP>, s1, WideGramGrant<G, DIAG, SIMP>::g);
  if (e != cudaSuccess) return e;
  if ((e = grant_smem(k_wide_jt<float, G, DIAG>, s2, WideJtGrant<G, DIAG>::g)) != cudaSuccess) return e;
  if (st == reinterpret_cast<cudaStream_t>(-1)) return cudaSuccess;  // grants only
  if ((e = launch_pdl(k_wide_gram<float, G, DIAG, SIMP>, dim3(a.ntiles1), dim3(256), s1, st, a)) != cudaSuccess)
    return e;
  if ((e = launch_pdl(k_wide_jt<float, G, DIAG>, dim3(a.nblk2), dim3(256), s2, st, a)) != cudaSuccess)
    return e;
  const size_t nK = (size_t)a.H * a.W * a.K;
  const int nb3 = (int)std::min<size_t>((nK + 255) / 256, 152 * 8);
  return launch_pdl(k_wide_diff<float, DIAG>, dim3(nb3), dim3(256), 0, st, a);
}

template <int G>
static cudaError_t wide_ds(const WideArgs<float>& a, bool diag, bool simplex, cudaStream_t st) {
  if (diag) return simplex ? wide_g<G, true, true>(a, st) : wide_g<G, true, false>(a, st);
  return simplex ? wide_g<G, false, true>(a, st) : wide_g<G, false, false>(a, st);
}

template <>
cudaError_t launch_wide<float>(const WideArgs<float>& a, int G, bool diag, bool simplex, cudaStream_t st) {
  switch (G) {
    case 4: return wide_ds<4>(a, diag, simplex, st);
    case 8: return wide_ds<8>(a, diag, simplex, st);
    case 16: return wide_ds<16>(a, diag, simplex, st);
    case 32: return wide_ds<32>(a, diag, simplex, st);
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t prepare_wide<float>(int M, int G) {
  WideArgs<float> a{};
  a.M = M;
  const cudaStream_t none = reinterpret_cast<cudaStream_t>(-1);
  for (int d = 0; d < 2; ++d)
    for (int s = 0; s < 2; ++s)
      if (cudaError_t e = launch_wide<float>(a, G, d, s, none)) return e;
  return cudaSuccess;
}

template <>
cudaError_t launch_wide_dual<float>(const float* V, const float* coef, float* d2, int n, int LK, cudaStream_t st) {
  const size_t tot = (size_t)n * LK;
  const int blocks = (int)std::min<size_t>((tot + 255) / 256, 152 * 16);
  k_wide_dual<float><<<blocks, 256, 0, st>>>(V, coef, d2, n, LK);
  return cudaGetLastError();
}

template <>
cudaError_t launch_wide_coef_identity<float>(float* coef, int n, cudaStream_t st) {
  const int blocks = std::min((n + 255) / 256, 152 * 16);
  k_wide_coef_identity<float><<<blocks, 256, 0, st>>>(coef, n);
  return cudaGetLastError();
}

}  // namespace sgs
