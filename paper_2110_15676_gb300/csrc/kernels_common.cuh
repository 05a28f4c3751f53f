// Small device helpers shared by the hot-path kernels.
#pragma once

#include "afc_internal.h"

namespace afc {

// m_ij and d_ij of the pair (i, i + o_k), k != Kup.  Stored once per pair at the
// row of the pair's lower node, offset index ku of the positive offset |o_k|.
__device__ __forceinline__ void pair_coef(const Offsets& of, int k, int64_t i, int64_t N,
                                          const double* __restrict__ m_up, const double* __restrict__ d_up,
                                          double& m, double& d) {
  int64_t q;
  if (k > of.Kup) q = (int64_t)(k - of.Kup - 1) * N + i;
  else q = (int64_t)(of.Kup - 1 - k) * N + i + of.o[k];
  m = m_up[q];
  d = d_up[q];
}

__device__ __forceinline__ double pair_d(const Offsets& of, int k, int64_t i, int64_t N,
                                         const double* __restrict__ d_up) {
  if (k > of.Kup) return d_up[(int64_t)(k - of.Kup - 1) * N + i];
  return d_up[(int64_t)(of.Kup - 1 - k) * N + i + of.o[k]];
}

// minmod of Eq. prelimiting: 0 unless both arguments have the same strict sign.
__device__ __forceinline__ double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return fmin(a, b);
  if (a < 0.0 && b < 0.0) return fmax(a, b);
  return 0.0;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum v over the block (fixed order) and store it in part[blockIdx.x].
// Every thread of the block must call it.
__device__ __forceinline__ void block_sum_to(double v, double* part) {
  __shared__ double sh[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) part[blockIdx.x] = t;
  }
  __syncthreads();
}

// Several sums at once (NV values per thread), stored at part[q * stride + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_sums_to(double (&v)[NV], double* part, int64_t stride) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double t = warp_sum(v[q]);
    if (lane == 0) sh[q][w] = t;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = lane < nw ? sh[q][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) part[q * stride + blockIdx.x] = t;
    }
  }
  __syncthreads();
}

// out[0] = sum of part[0..n) in a fixed order (one block).
void finalize_sum(afc_problem_s* p, const double* part, int n, double* out);

}  // namespace afc
