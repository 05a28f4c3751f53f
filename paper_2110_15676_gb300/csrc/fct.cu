// Zalesak flux-corrected transport passes (Sec. 2.1): the explicit FE-SSP stage
// (Sec. 2.1.2) and the Crank-Nicolson residual (Sec. 2.1.1), both with Zalesak's
// limiter (Sec. 2.1.3).
//
// Structure.  Each pass of a stage is one kernel over the rows; a pair's flux
// r_ij is computed once, by the row of its lower node, and stored in r_up (the
// upper half of the pattern, r_ji = -r_ij).  The node passes that need all
// fluxes of a row (P+/-, then alpha and F*) read r_up at their own row and,
// shifted by the column offset, at the rows of their lower neighbours.  On
// GB300 the FP64 pipe, not HBM, bounds these passes, so each pair costs as few
// FP64 operations as the formulas allow and every comparison, min and max runs
// on the integer pipe (kernels_common.cuh).
#include "afc_internal.h"
#include "kernels_common.cuh"
#include "ssp_rows.cuh"

namespace afc {

namespace {

// ---- explicit stage (per-row arithmetic in ssp_rows.cuh) ------------------------

template <int KT, bool MIXED>
__global__ void k_ssp_rate(Offsets of, SspArrays a, const double* __restrict__ u, double dt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.N) ssp_rate_row<KT, MIXED>(of, a, i, u, dt);
}

template <int KT, bool MIXED>
__global__ void k_ssp_edges(Offsets of, SspArrays a, const double* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.N) ssp_edges_row<KT, MIXED>(of, a, i, u);
}

template <int KT, bool MIXED>
__global__ void k_ssp_factors(Offsets of, SspArrays a, double dt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.N) ssp_factors_row<KT, MIXED>(of, a, i, dt);
}

template <int KT, bool MIXED>
__global__ void k_ssp_correct(Offsets of, SspArrays a, int limiter, double dt, double ca,
                              const double* __restrict__ uA, double cb, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < a.N) ssp_correct_row<KT, MIXED>(of, a, i, limiter, dt, ca, uA, cb, out);
}

__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = __double2float_rn(x[i]);
}

// ---- Crank-Nicolson -------------------------------------------------------------

// Once per step: y = AA u_old, predictor u~ = u_old - (dt/2)(y - f)/m (Eq. forward_euler,
// u_D at Dirichlet nodes), b0 = (m/dt) u_old - y/2 + f (right-hand side of Eq. CNZal).
template <int KT>
__global__ void k_cn_predictor(int64_t N, Offsets of, const double* __restrict__ AA, const double* __restrict__ uo,
                               const double* __restrict__ f, const double* __restrict__ mL,
                               const uint8_t* __restrict__ dir, const double* __restrict__ udir, double dt,
                               double* __restrict__ ut, double* __restrict__ b0) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double y = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) y = fma(AA[k * N + i], uo[i + of.o[k]], y);
  const double m = mL[i];
  ut[i] = dir[i] ? udir[i] : uo[i] - 0.5 * dt * (y - f[i]) / m;
  b0[i] = (m / dt * uo[i] - 0.5 * y) + f[i];
}

// m_i Q+/- of the CN predictor over N_i (fixed for the whole step, so the product
// with the lumped mass is formed once per step rather than in every factors pass).
template <int KT>
__global__ void k_bounds_of(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                            const double* __restrict__ v, const double* __restrict__ mL, double* __restrict__ Qp,
                            double* __restrict__ Qm) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  const double vi = v[i];
  long long kmax = dkey(vi), kmin = kmax;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!((mk >> k) & 1ull)) continue;
    const long long kj = dkey(v[i + of.o[k]]);
    kmax = kj > kmax ? kj : kmax;
    kmin = kj < kmin ? kj : kmin;
  }
  const double m = mL[i];
  Qp[i] = m * (from_key(kmax) - vi);
  Qm[i] = m * (from_key(kmin) - vi);
}

// Node sums of the CN flux: a = u - u_old, s = u + u_old; optionally first
// u += omega * delta (the damped update of Sec. 4).
__global__ void k_cn_update(int64_t N, double omega, const double* __restrict__ delta, double* __restrict__ u,
                            const double* __restrict__ uo, double* __restrict__ a, double* __restrict__ s) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double ui = u[i];
  if (delta) {
    ui = ui + omega * delta[i];
    u[i] = ui;
  }
  const double uoi = uo[i];
  a[i] = ui - uoi;
  s[i] = ui + uoi;
}

// Eq. flux_002 for every pair i < j, prelimited by Eq. prelimiting (L = 2) against twice
// its diffusive part at the CN average:  q = d_ij (s_j - s_i) = 2 d_ij (ubar_j - ubar_i),
// r = (m_ij / dt)(a_i - a_j) + q / 2,  r <- minmod(r, q).
// One thread per pair slot: block = 32 rows (threadIdx.x) x all upper offsets (threadIdx.y).
template <int KT>
__global__ void k_cn_edges(int64_t N, Offsets of, const double* __restrict__ mdt_up, const double* __restrict__ d_up,
                           const double* __restrict__ a, const double* __restrict__ s, int prelimit,
                           double* __restrict__ r_up) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int ku = threadIdx.y;
  const int64_t i = blockIdx.x * (int64_t)32 + threadIdx.x;
  if (i >= N) return;
  const int64_t q = (int64_t)ku * N + i;
  const int64_t j = i + of.o[Kup + 1 + ku];
  pdl_trigger();
  const double dq = d_up[q], mq = mdt_up[q];   // no pass of the step writes them
  pdl_wait();
  const double lim = dq * (s[j] - s[i]);
  double r = fma(mq, a[i] - a[j], half_exact(lim));
  if (prelimit) r = minmod(r, lim);
  r_up[q] = r;
}

// Zalesak steps 1-3 for the CN fluxes (Q+/- precomputed from the predictor).
template <int KT>
__global__ void k_cn_factors(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                             const double* __restrict__ r_up, const double* __restrict__ mQp,
                             const double* __restrict__ mQm,
                             const uint8_t* __restrict__ dir, double dt, double* __restrict__ Rp,
                             double* __restrict__ Rm) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  // the mask, the Dirichlet flag and m Q+/- (formed once per step) before the wait for
  // the fluxes of the edge pass
  const bool isdir = dir[i];
  const unsigned long long mk = mask[i];
  const double qp = mQp[i], qm = mQm[i];
  pdl_wait();
  if (isdir) { Rp[i] = 1.0; Rm[i] = 1.0; return; }
  constexpr int KA = KT > 0 ? KT : kMaxOffsets;
  SignedFixedSums acc;
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    if (k >= K || k == Kup || !((mk >> k) & 1ull)) continue;
    acc.add((unsigned long long)__double_as_longlong(pair_flux(of, Kup, k, i, N, r_up)));
  }
  double Pp, Pm;
  acc.result(Pp, Pm);
  Rp[i] = zalesak_factor(qp, dt * Pp);
  Rm[i] = zalesak_factor(qm, dt * Pm);
}

// Zalesak step 4, F*, and the nonlinear residual of Eq. CNZal:
// res = b0 + F* - (m/dt u + AA u / 2) on free rows, 0 on Dirichlet rows;
// block partial sums of res^2 for the stopping test.
template <int KT>
__global__ void __launch_bounds__(256, 4) k_cn_residual(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const double* __restrict__ r_up, const double* __restrict__ AA,
                              const double* __restrict__ un, const double* __restrict__ Rp,
                              const double* __restrict__ Rm, const double* __restrict__ b0,
                              const double* __restrict__ mLdt, const uint8_t* __restrict__ dir,
                              double* __restrict__ res, double* __restrict__ Fout, double* __restrict__ part) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  // y = AA u from the matrix and the state, before the wait for the factors pass: no pass
  // of the limiter writes them (u is the solver's, complete before the edge pass started)
  const bool act = i < N && !dir[i];
  double y = 0.0;
  if (act) {
#pragma unroll
    for (int k = 0; k < K; ++k) y = fma(AA[k * N + i], un[i + of.o[k]], y);
  }
  pdl_wait();
  if (i < N) {
    double rv = 0.0, F = 0.0;
    if (act) {
      const unsigned long long mk = mask[i];
      if (limiter != AFC_LIM_NONE) {
        const double rpi = Rp[i], rmi = Rm[i];
      #pragma unroll
  for (int k = 0; k < K; ++k) {
          if (k == Kup || !((mk >> k) & 1ull)) continue;
          const double r = pair_flux(of, Kup, k, i, N, r_up);
          if (limiter == AFC_LIM_ZALESAK) {
            const int64_t j = i + of.o[k];
            const double alpha = gt0(r) ? imin_nn(rpi, Rm[j]) : imin_nn(rmi, Rp[j]);
            F = fma(alpha, r, F);
          } else {
            F += r;
          }
        }
      }
      rv = b0[i] + F - (mLdt[i] * un[i] + 0.5 * y);
    }
    res[i] = rv;
    if (Fout) Fout[i] = F;
    r2 = rv * rv;
  }
  block_sum_to(r2, part);
}

}  // namespace

SspArrays ssp_arrays(afc_problem_s* p) {
  SspArrays a;
  a.N = p->N;
  a.AA = p->AA.p;
  a.m_up = p->m_up.p;
  a.d_up = p->d_up.p;
  a.m32 = p->m32_up.p;
  a.d32 = p->d32_up.p;
  a.mL = p->mL.p;
  a.f = p->f.p;
  a.dir = p->dir.p;
  a.udir = p->udir.p;
  a.mask = p->mask.p;
  a.udot = p->udot.p;
  a.ut = p->ut.p;
  a.uf = p->uf.p;
  a.udf = p->udf.p;
  a.r_up = p->r_up.p;
  a.r32 = p->r32.p;
  a.Rp = p->Rp.p;
  a.Rm = p->Rm.p;
  a.Fs = p->Fs.p;
  return a;
}

int ensure_ssp_mixed(afc_problem_s* p) {
  if (p->ssp32_ready) return AFC_OK;
  const int64_t N = p->N, Kup = p->Kup;
  int st;
  if ((st = p->m32_up.alloc(Kup * N)) || (st = p->d32_up.alloc(Kup * N)) || (st = p->r32.alloc(Kup * N)) ||
      (st = p->uf.alloc(N, p->pad)) || (st = p->udf.alloc(N, p->pad)))
    return st;
  AFC_LAUNCH(p, "k_to_float", k_to_float<<<grid_for(Kup * N), kBlock, 0, p->stream>>>(Kup * N, p->m_up.p, p->m32_up.p));
  AFC_LAUNCH(p, "k_to_float", k_to_float<<<grid_for(Kup * N), kBlock, 0, p->stream>>>(Kup * N, p->d_up.p, p->d32_up.p));
  AFC_CUDA(cudaGetLastError());
  p->ssp32_ready = true;
  return AFC_OK;
}

int fe_stage(afc_problem_s* p, const double* uin, double dt, int limiter, double a, const double* uA, double b,
             double* out, bool mixed) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  if (mixed) {
    int st = ensure_ssp_mixed(p);
    if (st) return st;
  }
  const SspArrays arr = ssp_arrays(p);
  if (limiter == AFC_LIM_MC) {
    // transient MC (Sec. 2.2): rate, clipped fluxes, then the unweighted sum of r*
    int st = AFC_OK;
    with_K(p->K, [&](auto kc) {
      constexpr int KT = decltype(kc)::value;
      AFC_LAUNCH(p, "k_ssp_rate", k_ssp_rate<KT, false><<<g, kBlock, 0, s>>>(p->offs, arr, uin, dt));
      if ((st = mc_ssp_fluxes(p, uin))) return;
      AFC_LAUNCH(p, "k_ssp_correct", k_ssp_correct<KT, false><<<g, kBlock, 0, s>>>(p->offs, arr, AFC_LIM_GALERKIN, dt,
                                                                                  a, uA, b, out));
    });
    if (st) return st;
    AFC_CUDA(cudaGetLastError());
    return AFC_OK;
  }
  auto run = [&](auto kc, auto mc) {
    constexpr int KT = decltype(kc)::value;
    constexpr bool MX = decltype(mc)::value;
    AFC_LAUNCH(p, "k_ssp_rate", k_ssp_rate<KT, MX><<<g, kBlock, 0, s>>>(p->offs, arr, uin, dt));
    if (limiter != AFC_LIM_NONE)
      AFC_LAUNCH(p, "k_ssp_edges", k_ssp_edges<KT, MX><<<g, kBlock, 0, s>>>(p->offs, arr, uin));
    if (limiter == AFC_LIM_ZALESAK)
      AFC_LAUNCH(p, "k_ssp_factors", k_ssp_factors<KT, MX><<<g, kBlock, 0, s>>>(p->offs, arr, dt));
    AFC_LAUNCH(p, "k_ssp_correct",
               k_ssp_correct<KT, MX><<<g, kBlock, 0, s>>>(p->offs, arr, limiter, dt, a, uA, b, out));
  };
  with_K(p->K, [&](auto kc) {
    if (mixed) run(kc, std::true_type{});
    else run(kc, std::false_type{});
  });
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

namespace {
// linear Zal+CN: u = 2 u~ - u_old (the value u^n is replaced by in Eq. flux_002), u_D on Dirichlet rows
__global__ void k_cn_linear_guess(int64_t N, const uint8_t* __restrict__ dir, const double* __restrict__ udir,
                                  const double* __restrict__ ut, const double* __restrict__ u_old,
                                  double* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) u[i] = dir[i] ? udir[i] : 2.0 * ut[i] - u_old[i];
}
}  // namespace

int cn_linear_guess(afc_problem_s* p, const double* u_old, double* u) {
  AFC_LAUNCH(p, "k_cn_linear_guess", k_cn_linear_guess<<<grid_for(p->N), kBlock, 0, p->stream>>>(
                                         p->N, p->dir.p, p->udir.p, p->ut.p, u_old, u));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int cn_predictor(afc_problem_s* p, const double* u_old, double dt) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    AFC_LAUNCH(p, "k_cn_predictor", k_cn_predictor<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->AA.p, u_old, p->f.p,
                                                                             p->mL.p, p->dir.p, p->udir.p, dt, p->ut.p,
                                                                             p->b0.p));
    AFC_LAUNCH(p, "k_bounds_of",
               k_bounds_of<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->ut.p, p->mL.p, p->Qp.p,
                                                    p->Qm.p));
  });
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int cn_update(afc_problem_s* p, double omega, const double* delta, double* u, const double* u_old) {
  AFC_LAUNCH(p, "k_cn_update", k_cn_update<<<grid_for(p->N), kBlock, 0, p->stream>>>(p->N, omega, delta, u, u_old,
                                                                                       p->cn_a.p, p->cn_s.p));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

namespace {

// F*_i = sum_j r*_ij of the clipped fluxes stored once per pair (0 on Dirichlet rows)
template <int KT>
__global__ void k_pair_sum(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                           const double* __restrict__ r_up, const uint8_t* __restrict__ dir, double* __restrict__ F) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  if (!dir[i]) {
    const unsigned long long mk = mask[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k == Kup || !((mk >> k) & 1ull)) continue;
      s += pair_flux(of, Kup, k, i, N, r_up);
    }
  }
  F[i] = s;
}

// res = b0 + (F*(u) + Fold) / 2 - (m/dt u + AA u / 2) on free rows, block partials of res^2
template <int KT>
__global__ void __launch_bounds__(256, 3) k_mccn_residual(
    int64_t N, Offsets of, const unsigned long long* __restrict__ mask, const double* __restrict__ r_up,
    const double* __restrict__ AA, const double* __restrict__ u, const double* __restrict__ Fold,
    const double* __restrict__ b0, const double* __restrict__ mLdt, const uint8_t* __restrict__ dir,
    double* __restrict__ res, double* __restrict__ Fout, double* __restrict__ part) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (i < N) {
    double rv = 0.0, F = 0.0;
    if (!dir[i]) {
      const unsigned long long mk = mask[i];
      double y = 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k) y = fma(AA[k * N + i], u[i + of.o[k]], y);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k == Kup || !((mk >> k) & 1ull)) continue;
        F += pair_flux(of, Kup, k, i, N, r_up);
      }
      F = 0.5 * (F + Fold[i]);
      rv = b0[i] + F - (mLdt[i] * u[i] + 0.5 * y);
    }
    res[i] = rv;
    if (Fout) Fout[i] = F;
    r2 = rv * rv;
  }
  block_sum_to(r2, part);
}

}  // namespace

int mc_cn_old_flux(afc_problem_s* p, const double* u_old) {
  const int64_t N = p->N, g = grid_for(N);
  cudaStream_t s = p->stream;
  const SspArrays arr = ssp_arrays(p);
  int st = AFC_OK;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    AFC_LAUNCH(p, "k_ssp_rate", k_ssp_rate<KT, false><<<g, kBlock, 0, s>>>(p->offs, arr, u_old, 0.0));
    if ((st = mc_ssp_fluxes(p, u_old))) return;
    AFC_LAUNCH(p, "k_pair_sum", k_pair_sum<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->r_up.p, p->dir.p,
                                                                      p->Fold.p));
  });
  if (st) return st;
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int mc_cn_residual(afc_problem_s* p, const double* u, double* res, double* normsq_slot) {
  const int64_t N = p->N, g = grid_for(N);
  cudaStream_t s = p->stream;
  const SspArrays arr = ssp_arrays(p);
  int st = AFC_OK;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    AFC_LAUNCH(p, "k_ssp_rate", k_ssp_rate<KT, false><<<g, kBlock, 0, s>>>(p->offs, arr, u, 0.0));
    if ((st = mc_ssp_fluxes(p, u))) return;
    AFC_LAUNCH(p, "k_mccn_residual",
               k_mccn_residual<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->r_up.p, p->AA.p, u, p->Fold.p,
                                                        p->b0.p, p->mLdt.p, p->dir.p, res, p->Fs.p, p->part.p));
  });
  if (st) return st;
  if (normsq_slot) finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int cn_limited_residual(afc_problem_s* p, const double* u_new, double dt, int limiter, int prelimit, double* res,
                        double* normsq_slot) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    if (limiter != AFC_LIM_NONE)
      AFC_LAUNCH(p, "k_cn_edges", k_cn_edges<KT><<<grid_for(N, 32), dim3(32, p->Kup), 0, s>>>(N, p->offs, p->mdt_up.p, p->d_up.p, p->cn_a.p,
                                                                       p->cn_s.p, prelimit, p->r_up.p));
    // programmatic dependent launch down the limiter passes (the edge pass follows the
    // solver with a plain dependency)
    if (limiter == AFC_LIM_ZALESAK)
      AFC_LAUNCH(p, "k_cn_factors", launch_pass(limiter != AFC_LIM_NONE, k_cn_factors<KT>, dim3((unsigned)g),
                                                dim3(kBlock), s, N, p->offs, (const unsigned long long*)p->mask.p,
                                                (const double*)p->r_up.p, (const double*)p->Qp.p,
                                                (const double*)p->Qm.p, (const uint8_t*)p->dir.p, dt, p->Rp.p,
                                                p->Rm.p));
    AFC_LAUNCH(p, "k_cn_residual",
               launch_pass(limiter != AFC_LIM_NONE, k_cn_residual<KT>, dim3((unsigned)g), dim3(kBlock), s, N,
                           p->offs, limiter, (const unsigned long long*)p->mask.p, (const double*)p->r_up.p,
                           (const double*)p->AA.p, u_new, (const double*)p->Rp.p, (const double*)p->Rm.p,
                           (const double*)p->b0.p, (const double*)p->mLdt.p, (const uint8_t*)p->dir.p, res, p->Fs.p,
                           p->part.p));
  });
  if (normsq_slot) finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
