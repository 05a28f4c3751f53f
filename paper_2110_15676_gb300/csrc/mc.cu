// Monolithic convex limiter for the stationary problem (Sec. 2.2, Sec. 3.1):
// bounds u_i^max/min over N_i (Eq. u_max_min), fluxes r_ij = d_ij (u_j - u_i),
// bar states 2 d_ij ubar_ij = d_ij (u_i + u_j) + a_ij (u_j - u_i) with the
// convective entries a_ij = k_ij (Remark rem:assembling_mc), the clip of
// Eq. MClimiter, and the nonlinear residual f + F*(u) - AA u of Sec. 4.
//
// Formulation used on the device.  With D = u_j - u_i, A_i = u_i^max - u_i,
// B_i = u_i - u_i^min and d_ij <= 0, the bounds of Eq. MClimiter differ from r_ij by
//   2 d_ij (ubar_ij - u_i^max) - r_ij = a_ij D + 2|d_ij| A_i       (r_ij > 0)
//   2 d_ij (u_j^min - ubar_ji) - r_ij = a_ji D + 2|d_ij| B_j
// (and the mirrored pair for r_ij < 0), so the clipped amount c_ij = r_ij - r*_ij is
//   r_ij > 0:  c = max(0, -T_i, -T_j),  T_i = 2|d| A_i - a_ij |D|,  T_j = 2|d| B_j - a_ji |D|
//   r_ij < 0:  c = min(0,  T_i,  T_j),  T_i = 2|d| B_i - a_ij |D|,  T_j = 2|d| A_j - a_ji |D|
// and a side with a <= 0 can never clip.  Since D has zero row sums,
// F*_i = sum_j r*_ij = (D u)_i - sum_j c_ij, and the residual is
//   res = f - (K + eps S + c M_L) u - sum_j c_ij.
// On GB300 (2 FP64 operations per SM and cycle) this needs ~3 FP64 operations per
// pair instead of ~10 for the printed form; the result is the same up to rounding.
#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

namespace {

// u_max / u_min over N_i (which contains i) and A = u_max - u, B = u - u_min; clears
// the row's clip mask for the edge pass that follows.
template <int KT>
__global__ void k_mc_bounds(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                            const double* __restrict__ u, double* __restrict__ umax, double* __restrict__ umin,
                            double* __restrict__ bA, double* __restrict__ bB, float4* __restrict__ nf,
                            unsigned int* __restrict__ clip) {
  const int K = KT > 0 ? KT : of.K;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  const double ui = u[i];
  long long kmax = dkey(ui), kmin = kmax;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!((mk >> k) & 1ull)) continue;
    const long long kj = dkey(u[i + of.o[k]]);
    kmax = kj > kmax ? kj : kmax;
    kmin = kj < kmin ? kj : kmin;
  }
  const double hi = from_key(kmax), lo = from_key(kmin);
  if (umax) {
    umax[i] = hi;
    umin[i] = lo;
  }
  const double A = hi - ui, B = ui - lo;
  bA[i] = A;
  bB[i] = B;
  // rounded copies for the pre-test; w = 1 where the single copy of u is exact
  const float uf = __double2float_rn(ui);
  const bool exact = __double_as_longlong(widen_exact(uf)) == __double_as_longlong(ui);
  nf[i] = make_float4(uf, (float)A, (float)B, exact ? 1.f : 0.f);
  clip[i] = 0u;
}

// Clipped amount c_ij of every pair i < j (stored at row i, only where nonzero; the
// row's clip mask gets bit ku) for one thread per pair slot (ku, i): a block covers
// 32 consecutive rows (threadIdx.x) and all upper offsets (threadIdx.y).
//
// Exact pre-test.  A side T = 2|d| X - a |D| (a > 0) can only clip if T < 0.  The
// test first evaluates T from single-precision copies of 2|d|, a, u and X together
// with a strict bound E on its rounding error (every input and operation in single
// precision carries a relative error of at most 2^-24, the sum of all of them stays
// below 2^-22 (p1 + p2 + a (|u_i| + |u_j|)); E uses 2^-20, plus 2^-100 for values in
// the single subnormal range, and 2|d|, a, X must exceed 2^-100).  If T_single > E the exact T is
// positive and the pair is certainly not clipped: c = 0 without any FP64 work.  Only
// the remaining pairs evaluate T in FP64 as written above.
__device__ __forceinline__ bool side_certainly_unclipped(float d2f, float af, float xf, float uif, float ujf) {
  const float tiny = 7.9e-31f;                        // ~2^-100: far above the single subnormals
  if (af < tiny || d2f < tiny || xf < tiny) return false;
  const float Df = fabsf(ujf - uif);
  const float p1 = d2f * xf, p2 = af * Df;
  // 2^-20 (...) covers the relative errors; 2^-100 covers any absolute error of values
  // in the single subnormal range
  const float err = 9.5367431640625e-07f * (p1 + p2 + af * (fabsf(uif) + fabsf(ujf))) + tiny;
  return p1 - p2 > err;
}

template <int KT>
__global__ void k_mc_edges(int64_t N, Offsets of, const double* __restrict__ d2_up, const double* __restrict__ kij,
                           const double* __restrict__ kji, const float* __restrict__ pf,
                           const double* __restrict__ u, const double* __restrict__ bA,
                           const double* __restrict__ bB, const float4* __restrict__ nf, double* __restrict__ c_up,
                           unsigned int* __restrict__ clip) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int ku = threadIdx.y;
  const int64_t i = blockIdx.x * (int64_t)32 + threadIdx.x;
  if (i >= N) return;
  const int64_t q = (int64_t)ku * N + i;
  const int64_t j = i + of.o[Kup + 1 + ku];
  const int64_t KN = (int64_t)Kup * N;
  const float4 cf = make_float4(pf[q], pf[KN + q], pf[2 * KN + q], 0.f);   // 2|d|, a_ij, a_ji in single
  const bool side_i = cf.y > 0.f, side_j = cf.z > 0.f;
  if (!(cf.x > 0.f) || !(side_i || side_j)) return;   // d = 0, or no side can clip
  const float4 ni = nf[i], nj = nf[j];
  if (ni.x == nj.x && ni.w != 0.f && nj.w != 0.f) return;   // equal exact copies: u_i = u_j, r = 0
  if (ni.x != nj.x) {   // equal single copies need not mean equal values: decided in double below
    const bool rpos = nj.x < ni.x;
    const bool ok_i = !side_i || side_certainly_unclipped(cf.x, cf.y, rpos ? ni.y : ni.z, ni.x, nj.x);
    const bool ok_j = !side_j || side_certainly_unclipped(cf.x, cf.z, rpos ? nj.z : nj.y, ni.x, nj.x);
    if (ok_i && ok_j) return;
  }
  const double ui = u[i], uj = u[j];
  const long long ki = dkey(ui), kj = dkey(uj);
  if (ki == kj) return;
  const bool rpos = kj < ki;                          // r_ij = d (u_j - u_i) > 0  <=>  u_j < u_i
  const double absD = abs_bits(uj - ui);
  const double d2 = d2_up[q];                         // 2 |d_ij|
  double m = 0.0;
  if (side_i) m = imin(m, fma(-kij[q], absD, d2 * (rpos ? bA[i] : bB[i])));
  if (side_j) m = imin(m, fma(-kji[q], absD, d2 * (rpos ? bB[j] : bA[j])));
  if (!is0(m)) {
    c_up[q] = rpos ? neg_bits(m) : m;
    atomicOr(clip + i, 1u << ku);
  }
}

// res = f - AG u - sum_j c_ij on free rows (0 on Dirichlet rows), block partials of
// res^2.  The limiter modes: MC (as above), Galerkin (c = 0), none (res = f - AA u).
// With Fout, also F*_i = sum_j (d_ij (u_j - u_i) - c_ij) for inspection.
template <int KT>
__global__ void k_mc_residual(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const unsigned int* __restrict__ clip, const double* __restrict__ c_up,
                              const double* __restrict__ Mop,
                              const double* __restrict__ d_up, const double* __restrict__ u,
                              const double* __restrict__ f, const uint8_t* __restrict__ dir,
                              double* __restrict__ res, double* __restrict__ Fout, double* __restrict__ part) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (i < N) {
    double rv = 0.0;
    if (!dir[i]) {
      double y = f[i];                      // y = f - M u
#pragma unroll
      for (int k = 0; k < K; ++k) y = fma(-Mop[k * N + i], u[i + of.o[k]], y);
      double C = 0.0;
      if (limiter == AFC_LIM_MC) {
        // pairs with a nonzero clipped amount: bit k of `bits` for offset index k
        unsigned long long bits = (unsigned long long)clip[i] << (Kup + 1);
#pragma unroll
        for (int ku = 0; ku < Kup; ++ku)
          bits |= (unsigned long long)((clip[i - of.o[Kup + 1 + ku]] >> ku) & 1u) << (Kup - 1 - ku);
        while (bits) {
          const int k = __ffsll(bits) - 1;
          bits &= bits - 1;
          C += pair_flux(of, Kup, k, i, N, c_up);
        }
      }
      rv = y - C;
      if (Fout) {   // inspection only
        double F = 0.0;
        if (limiter != AFC_LIM_NONE) {
          const unsigned long long mk = mask[i];
          const double ui = u[i];
          for (int k = 0; k < K; ++k) {
            if (k == Kup || !((mk >> k) & 1ull)) continue;
            const double r = pair_d(of, k, i, N, d_up) * (u[i + of.o[k]] - ui);
            F += r;
          }
          F -= C;
        }
        Fout[i] = F;
      }
    } else if (Fout) {
      Fout[i] = 0.0;
    }
    res[i] = rv;
    r2 = rv * rv;
  }
  block_sum_to(r2, part);
}

}  // namespace

int mc_limited_residual(afc_problem_s* p, const double* u, int limiter, double* res, double* normsq_slot,
                        bool want_F) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  const double* Mop = limiter == AFC_LIM_NONE ? p->AA.p : p->AG.p;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    if (limiter == AFC_LIM_MC) {
      AFC_LAUNCH(p, "k_mc_bounds",
                 k_mc_bounds<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, u, want_F ? p->umax.p : nullptr,
                                                      p->umin.p, p->bA.p, p->bB.p, p->nodef.p, p->clip.p));
      AFC_LAUNCH(p, "k_mc_edges", k_mc_edges<KT><<<grid_for(N, 32), dim3(32, p->Kup), 0, s>>>(
                                      N, p->offs, p->d2_up.p, p->kij_up.p, p->kji_up.p, p->pairf.p, u, p->bA.p,
                                      p->bB.p, p->nodef.p, p->r_up.p, p->clip.p));
    }
    AFC_LAUNCH(p, "k_mc_residual",
               k_mc_residual<KT><<<g, kBlock, 0, s>>>(N, p->offs, limiter, p->mask.p, p->clip.p, p->r_up.p, Mop,
                                                      p->d_up.p, u,
                                                      p->f.p, p->dir.p, res, want_F ? p->Fs.p : nullptr,
                                                      p->part.p));
  });
  finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
