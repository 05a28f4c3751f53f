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
                            unsigned long long* __restrict__ clip) {
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
  clip[i] = 0ull;
}

// Clipped amount c_ij of every pair i < j (stored at row i, only where nonzero; the
// clip masks of rows i and j get the pair's offset bits) for one thread per pair slot
// (ku, i): a block covers 32 consecutive rows (threadIdx.x) and all upper offsets
// (threadIdx.y).
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
                           unsigned long long* __restrict__ clip) {
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
    // the pair's bit at both ends: offset index Kup + 1 + ku at row i, Kup - 1 - ku
    // (the offset -o back to i) at row j
    atomicOr(clip + i, 1ull << (Kup + 1 + ku));
    atomicOr(clip + j, 1ull << (Kup - 1 - ku));
  }
}

// res = f - AG u - sum_j c_ij on free rows (0 on Dirichlet rows), block partials of
// res^2.  The limiter modes: MC (as above), Galerkin (c = 0), none (res = f - AA u).
// With Fout, also F*_i = sum_j (d_ij (u_j - u_i) - c_ij) for inspection.
template <int KT>
__global__ void k_mc_residual(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const unsigned long long* __restrict__ clip, const double* __restrict__ c_up,
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
        unsigned long long bits = clip[i];
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

// ---- monolithic upwind (MU) limiter (Sec. 3, MU limiter) ------------------------
// Stationary fluxes r_ij = d_ij (u_j - u_i), convective a_ij = k_ij (Remark
// rem:assembling_mc).  The pair (i, j) belongs to i if a_ji < a_ij, and on a tie
// a_ij = a_ji to the smaller index; its owner's factor is its alpha on both sides.
// a_ij, a_ji are computed values: they tie when within 1e-12 (|a_ij| + |a_ji|), so an
// exact tie of the exact entries does not depend on rounding.

// a_ij and a_ji of the pair (i, i + o_k) as seen from row i
__device__ __forceinline__ void pair_conv(const Offsets& of, int k, int64_t i, int64_t N,
                                          const double* __restrict__ kij, const double* __restrict__ kji,
                                          double& aij, double& aji) {
  if (k > of.Kup) {
    const int64_t q = (int64_t)(k - of.Kup - 1) * N + i;
    aij = kij[q];
    aji = kji[q];
  } else {
    const int64_t q = (int64_t)(of.Kup - 1 - k) * N + i + of.o[k];   // stored at the lower row j
    aij = kji[q];
    aji = kij[q];
  }
}

__device__ __forceinline__ bool mu_owns(double aij, double aji, int k, int Kup) {
  if (fabs(aij - aji) <= 1e-12 * (fabs(aij) + fabs(aji))) return k > Kup;   // tie: the smaller index (k > Kup: j > i)
  return aji < aij;
}

// steps 1-3: P+/- over the owned pairs, Q+/- over all pairs, R+/-
template <int KT>
__global__ void k_mu_factors(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                             const double* __restrict__ d_up, const double* __restrict__ kij,
                             const double* __restrict__ kji, const double* __restrict__ u,
                             const uint8_t* __restrict__ dir, double* __restrict__ Rp, double* __restrict__ Rm) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (dir[i]) {
    Rp[i] = 1.0;
    Rm[i] = 1.0;
    return;
  }
  const unsigned long long mk = mask[i];
  const double ui = u[i];
  double Pp = 0.0, Pm = 0.0, Qp = 0.0, Qm = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (k == Kup || !((mk >> k) & 1ull)) continue;
    const double r = pair_d(of, k, i, N, d_up) * (u[i + of.o[k]] - ui);
    double aij, aji;
    pair_conv(of, k, i, N, kij, kji, aij, aji);
    const bool own = mu_owns(aij, aji, k, Kup);
    if (gt0(r)) {
      Qm -= r;
      if (own) Pp += r;
    } else if (!is0(r)) {
      Qp -= r;
      if (own) Pm += r;
    }
  }
  Rp[i] = zalesak_factor(Qp, Pp);
  Rm[i] = zalesak_factor(Qm, Pm);
}

// step 4 and the residual res = f + F* - AA u (0 on Dirichlet rows), block partials
// of res^2; F*_i = sum_j alpha_ij r_ij with the owner's factor
template <int KT>
__global__ void __launch_bounds__(256, 3) k_mu_residual(
    int64_t N, Offsets of, const unsigned long long* __restrict__ mask, const double* __restrict__ d_up,
    const double* __restrict__ kij, const double* __restrict__ kji, const double* __restrict__ AA,
    const double* __restrict__ u, const double* __restrict__ f, const uint8_t* __restrict__ dir,
    const double* __restrict__ Rp, const double* __restrict__ Rm, double* __restrict__ res,
    double* __restrict__ Fout, double* __restrict__ part) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (i < N) {
    double rv = 0.0, F = 0.0;
    if (!dir[i]) {
      const unsigned long long mk = mask[i];
      const double ui = u[i], rpi = Rp[i], rmi = Rm[i];
      double y = f[i];
#pragma unroll
      for (int k = 0; k < K; ++k) y = fma(-AA[k * N + i], u[i + of.o[k]], y);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k == Kup || !((mk >> k) & 1ull)) continue;
        const int64_t j = i + of.o[k];
        const double r = pair_d(of, k, i, N, d_up) * (u[j] - ui);
        if (is0(r)) continue;                         // alpha = 1, r = 0
        double aij, aji;
        pair_conv(of, k, i, N, kij, kji, aij, aji);
        double alpha;
        if (mu_owns(aij, aji, k, Kup)) alpha = gt0(r) ? rpi : rmi;
        else alpha = gt0(r) ? Rm[j] : Rp[j];          // r_ji = -r_ij
        F = fma(alpha, r, F);
      }
      rv = y + F;
    }
    res[i] = rv;
    if (Fout) Fout[i] = F;
    r2 = rv * rv;
  }
  block_sum_to(r2, part);
}

// ---- transient MC (Sec. 2.2): the SSP fluxes clipped by Eq. MClimiter ---------------
template <int KT>
__global__ void k_mcssp_bounds(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                               const double* __restrict__ u, double* __restrict__ umax, double* __restrict__ umin) {
  const int K = KT > 0 ? KT : of.K;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  long long kmax = dkey(u[i]), kmin = kmax;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!((mk >> k) & 1ull)) continue;
    const long long kj = dkey(u[i + of.o[k]]);
    kmax = kj > kmax ? kj : kmax;
    kmin = kj < kmin ? kj : kmin;
  }
  umax[i] = from_key(kmax);
  umin[i] = from_key(kmin);
}

// r*_ij of every pair i < j at row i: r_ij = m_ij (udot_i - udot_j) + d_ij (u_j - u_i)
// (Eq. defn_r_ij_SSP) clipped with the bar states 2 d ubar_ij = d (u_i + u_j) + a_ij (u_j - u_i)
// and the bounds of the stage input; r* = 0 where d_ij = 0 (A16)
template <int KT>
__global__ void k_mcssp_edges(int64_t N, Offsets of, const double* __restrict__ m_up, const double* __restrict__ d_up,
                              const double* __restrict__ kij, const double* __restrict__ kji,
                              const double* __restrict__ u, const double* __restrict__ udot,
                              const double* __restrict__ umax, const double* __restrict__ umin,
                              double* __restrict__ r_up) {
  const int Kup = (KT > 0 ? KT : of.K) / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double ui = u[i], udi = udot[i], mxi = umax[i], mni = umin[i];
#pragma unroll
  for (int ku = 0; ku < Kup; ++ku) {
    const int64_t q = (int64_t)ku * N + i;
    const int64_t j = i + of.o[Kup + 1 + ku];
    const double d = d_up[q];
    double rs = 0.0;
    if (!is0(d)) {
      const double uj = u[j];
      const double r = fma(m_up[q], udi - udot[j], d * (uj - ui));
      const double d2 = 2.0 * d;
      const double ubij = (d * (ui + uj) + kij[q] * (uj - ui)) / d2;
      const double ubji = (d * (uj + ui) + kji[q] * (ui - uj)) / d2;
      if (gt0(r)) rs = imin(r, imin(d2 * (ubij - mxi), d2 * (umin[j] - ubji)));
      else rs = imax(r, imax(d2 * (ubij - mni), d2 * (umax[j] - ubji)));
    }
    r_up[q] = rs;
  }
}

}  // namespace

int mc_ssp_fluxes(afc_problem_s* p, const double* u) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    AFC_LAUNCH(p, "k_mcssp_bounds",
               k_mcssp_bounds<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, u, p->umax.p, p->umin.p));
    AFC_LAUNCH(p, "k_mcssp_edges",
               k_mcssp_edges<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->m_up.p, p->d_up.p, p->kij_up.p, p->kji_up.p, u,
                                                      p->udot.p, p->umax.p, p->umin.p, p->r_up.p));
  });
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int mc_limited_residual(afc_problem_s* p, const double* u, int limiter, double* res, double* normsq_slot,
                        bool want_F, bool pair) {
  if (pair && p->precision == AFC_MIXED && !want_F && (limiter == AFC_LIM_MC || limiter == AFC_LIM_GALERKIN))
    return mc_pair_residual(p, u, limiter, res, normsq_slot);
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  const double* Mop = limiter == AFC_LIM_NONE ? p->AA.p : p->AG.p;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    if (limiter == AFC_LIM_MU) {
      AFC_LAUNCH(p, "k_mu_factors",
                 k_mu_factors<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->d_up.p, p->kij_up.p, p->kji_up.p,
                                                       u, p->dir.p, p->Rp.p, p->Rm.p));
      AFC_LAUNCH(p, "k_mu_residual",
                 k_mu_residual<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->d_up.p, p->kij_up.p, p->kji_up.p,
                                                        p->AA.p, u, p->f.p, p->dir.p, p->Rp.p, p->Rm.p, res,
                                                        want_F ? p->Fs.p : nullptr, p->part.p));
      return;
    }
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
  if (normsq_slot) finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
