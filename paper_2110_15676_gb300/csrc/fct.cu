// Zalesak flux-corrected transport passes (Sec. 2.1): the explicit FE-SSP stage
// (Sec. 2.1.2) and the Crank-Nicolson residual (Sec. 2.1.1), both with Zalesak's
// limiter (Sec. 2.1.3).  One thread owns one row i and visits its neighbours j
// through the column offsets; the symmetric coefficients m_ij, d_ij of a pair
// are read from the row of its lower node, so each row sees the same numbers as
// its partner and r_ji = -r_ij, alpha_ji = alpha_ij hold by construction.
#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

namespace {

// ---- explicit stage -----------------------------------------------------------

// y = AA u;  udot^L = (f - y) / m (0 at Dirichlet nodes, whose data is constant);
// predictor u~ = u + dt (f - y) / m, u~ = u_D at Dirichlet nodes.
__global__ void k_ssp_rate(int64_t N, Offsets of, const double* __restrict__ AA, const double* __restrict__ u,
                           const double* __restrict__ f, const double* __restrict__ mL,
                           const uint8_t* __restrict__ dir, const double* __restrict__ udir, double dt,
                           double* __restrict__ udot, double* __restrict__ ut) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double y = 0.0;
#pragma unroll 4
  for (int k = 0; k < of.K; ++k) y = fma(AA[k * N + i], u[i + of.o[k]], y);
  if (dir[i]) {
    udot[i] = 0.0;
    ut[i] = udir[i];
  } else {
    const double fy = f[i] - y;
    udot[i] = fy / mL[i];
    ut[i] = u[i] + dt * fy / mL[i];
  }
}

// Zalesak steps 1-3: P+/-, Q+/- (neighbours of the predictor), R+/-.
__global__ void k_ssp_factors(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                              const double* __restrict__ m_up, const double* __restrict__ d_up,
                              const double* __restrict__ u, const double* __restrict__ udot,
                              const double* __restrict__ ut, const double* __restrict__ mL,
                              const uint8_t* __restrict__ dir, double dt, double* __restrict__ Rp,
                              double* __restrict__ Rm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (dir[i]) { Rp[i] = 1.0; Rm[i] = 1.0; return; }
  const unsigned long long mk = mask[i];
  const double ui = u[i], udi = udot[i], uti = ut[i];
  double Pp = 0.0, Pm = 0.0, tmax = uti, tmin = uti;
  for (int k = 0; k < of.K; ++k) {
    if (k == of.Kup || !((mk >> k) & 1ull)) continue;
    const int64_t j = i + of.o[k];
    double m, d;
    pair_coef(of, k, i, N, m_up, d_up, m, d);
    const double r = m * (udi - udot[j]) + d * (u[j] - ui);
    if (r > 0.0) Pp += r; else Pm += r;
    const double utj = ut[j];
    tmax = fmax(tmax, utj);
    tmin = fmin(tmin, utj);
  }
  const double Qp = tmax - uti, Qm = tmin - uti;     // >= 0 and <= 0: the max/min include i itself
  const double m = mL[i];
  Rp[i] = Pp != 0.0 ? fmin(1.0, m * Qp / (dt * Pp)) : 1.0;
  Rm[i] = Pm != 0.0 ? fmin(1.0, m * Qm / (dt * Pm)) : 1.0;
}

// Zalesak step 4 and the update: F*_i = sum_j alpha_ij r_ij,
// u_new = u~ + dt F* / m (= u + dt (f + F* - AA u) / m, Eq. FE-SSP), Dirichlet: u_D;
// out = a * uA + b * u_new (the SSP combination of the stage).
__global__ void k_ssp_correct(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const double* __restrict__ m_up, const double* __restrict__ d_up,
                              const double* __restrict__ u, const double* __restrict__ udot,
                              const double* __restrict__ ut, const double* __restrict__ Rp,
                              const double* __restrict__ Rm, const double* __restrict__ mL,
                              const uint8_t* __restrict__ dir, const double* __restrict__ udir, double dt, double a,
                              const double* __restrict__ uA, double b, double* __restrict__ out,
                              double* __restrict__ Fout) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double unew;
  double F = 0.0;
  if (dir[i]) {
    unew = udir[i];
  } else {
    const unsigned long long mk = mask[i];
    const double ui = u[i], udi = udot[i], rpi = Rp[i], rmi = Rm[i];
    if (limiter != AFC_LIM_NONE) {
      for (int k = 0; k < of.K; ++k) {
        if (k == of.Kup || !((mk >> k) & 1ull)) continue;
        const int64_t j = i + of.o[k];
        double m, d;
        pair_coef(of, k, i, N, m_up, d_up, m, d);
        const double r = m * (udi - udot[j]) + d * (u[j] - ui);
        double alpha = 1.0;
        if (limiter == AFC_LIM_ZALESAK) alpha = r > 0.0 ? fmin(rpi, Rm[j]) : fmin(rmi, Rp[j]);
        F = fma(alpha, r, F);
      }
    }
    unew = ut[i] + dt * F / mL[i];
  }
  if (Fout) Fout[i] = F;
  out[i] = a != 0.0 ? a * uA[i] + b * unew : b * unew;
}

// ---- Crank-Nicolson -------------------------------------------------------------

// Once per step: y = AA u_old, predictor u~ = u_old - (dt/2)(y - f)/m (Eq. forward_euler,
// u_D at Dirichlet nodes), b0 = (m/dt) u_old - y/2 + f (right-hand side of Eq. CNZal).
__global__ void k_cn_predictor(int64_t N, Offsets of, const double* __restrict__ AA, const double* __restrict__ uo,
                               const double* __restrict__ f, const double* __restrict__ mL,
                               const uint8_t* __restrict__ dir, const double* __restrict__ udir, double dt,
                               double* __restrict__ ut, double* __restrict__ b0) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double y = 0.0;
#pragma unroll 4
  for (int k = 0; k < of.K; ++k) y = fma(AA[k * N + i], uo[i + of.o[k]], y);
  const double m = mL[i];
  ut[i] = dir[i] ? udir[i] : uo[i] - 0.5 * dt * (y - f[i]) / m;
  b0[i] = (m / dt * uo[i] - 0.5 * y) + f[i];
}

// Q+/- of the CN predictor (fixed for the whole step).
__global__ void k_bounds_of(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                            const double* __restrict__ v, double* __restrict__ Qp, double* __restrict__ Qm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  const double vi = v[i];
  double tmax = vi, tmin = vi;
  for (int k = 0; k < of.K; ++k) {
    if (!((mk >> k) & 1ull)) continue;
    const double vj = v[i + of.o[k]];
    tmax = fmax(tmax, vj);
    tmin = fmin(tmin, vj);
  }
  Qp[i] = tmax - vi;
  Qm[i] = tmin - vi;
}

// CN flux Eq. flux_002 for the pair (i, j), prelimited by Eq. prelimiting (L = 2)
// against twice its diffusive part evaluated at the CN average.
__device__ __forceinline__ double cn_flux(double m, double d, double dt, double uni, double uoi, double unj,
                                          double uoj, int prelimit) {
  double r = (m / dt) * ((uni - uoi) - (unj - uoj)) + (0.5 * d) * ((unj + uoj) - (uni + uoi));
  if (prelimit) {
    const double lim = (2.0 * d) * (0.5 * (unj + uoj) - 0.5 * (uni + uoi));
    r = minmod(r, lim);
  }
  return r;
}

// Zalesak steps 1-3 for the CN fluxes (Q+/- precomputed from the predictor).
__global__ void k_cn_factors(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                             const double* __restrict__ m_up, const double* __restrict__ d_up,
                             const double* __restrict__ un, const double* __restrict__ uo,
                             const double* __restrict__ Qp, const double* __restrict__ Qm,
                             const double* __restrict__ mL, const uint8_t* __restrict__ dir, double dt, int prelimit,
                             double* __restrict__ Rp, double* __restrict__ Rm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (dir[i]) { Rp[i] = 1.0; Rm[i] = 1.0; return; }
  const unsigned long long mk = mask[i];
  const double uni = un[i], uoi = uo[i];
  double Pp = 0.0, Pm = 0.0;
  for (int k = 0; k < of.K; ++k) {
    if (k == of.Kup || !((mk >> k) & 1ull)) continue;
    const int64_t j = i + of.o[k];
    double m, d;
    pair_coef(of, k, i, N, m_up, d_up, m, d);
    const double r = cn_flux(m, d, dt, uni, uoi, un[j], uo[j], prelimit);
    if (r > 0.0) Pp += r; else Pm += r;
  }
  const double m = mL[i];
  Rp[i] = Pp != 0.0 ? fmin(1.0, m * Qp[i] / (dt * Pp)) : 1.0;
  Rm[i] = Pm != 0.0 ? fmin(1.0, m * Qm[i] / (dt * Pm)) : 1.0;
}

// Zalesak step 4, F*, and the nonlinear residual of Eq. CNZal:
// res = b0 + F* - (m/dt u + AA u / 2) on free rows, 0 on Dirichlet rows;
// block partial sums of res^2 for the stopping test.
__global__ void k_cn_residual(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const double* __restrict__ m_up, const double* __restrict__ d_up,
                              const double* __restrict__ AA, const double* __restrict__ un,
                              const double* __restrict__ uo, const double* __restrict__ Rp,
                              const double* __restrict__ Rm, const double* __restrict__ b0,
                              const double* __restrict__ mL, const uint8_t* __restrict__ dir, double dt, int prelimit,
                              double* __restrict__ res, double* __restrict__ Fout, double* __restrict__ part) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (i < N) {
    double rv = 0.0, F = 0.0;
    if (!dir[i]) {
      const unsigned long long mk = mask[i];
      const double uni = un[i], uoi = uo[i];
      double y = 0.0;
      for (int k = 0; k < of.K; ++k) {
        const int64_t j = i + of.o[k];
        y = fma(AA[k * N + i], un[j], y);
        if (limiter == AFC_LIM_NONE || k == of.Kup || !((mk >> k) & 1ull)) continue;
        double m, d;
        pair_coef(of, k, i, N, m_up, d_up, m, d);
        const double r = cn_flux(m, d, dt, uni, uoi, un[j], uo[j], prelimit);
        double alpha = 1.0;
        if (limiter == AFC_LIM_ZALESAK) alpha = r > 0.0 ? fmin(Rp[i], Rm[j]) : fmin(Rm[i], Rp[j]);
        F = fma(alpha, r, F);
      }
      rv = b0[i] + F - (mL[i] / dt * uni + 0.5 * y);
    }
    res[i] = rv;
    if (Fout) Fout[i] = F;
    r2 = rv * rv;
  }
  block_sum_to(r2, part);
}

}  // namespace

int fe_stage(afc_problem_s* p, const double* uin, double dt, int limiter, double a, const double* uA, double b,
             double* out) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  AFC_LAUNCH(p, "k_ssp_rate", k_ssp_rate<<<g, kBlock, 0, s>>>(N, p->offs, p->AA.p, uin, p->f.p, p->mL.p, p->dir.p, p->udir.p, dt, p->udot.p,
                                  p->ut.p));
  if (limiter == AFC_LIM_ZALESAK)
    AFC_LAUNCH(p, "k_ssp_factors", k_ssp_factors<<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->m_up.p, p->d_up.p, uin, p->udot.p, p->ut.p, p->mL.p,
                                       p->dir.p, dt, p->Rp.p, p->Rm.p));
  AFC_LAUNCH(p, "k_ssp_correct", k_ssp_correct<<<g, kBlock, 0, s>>>(N, p->offs, limiter, p->mask.p, p->m_up.p, p->d_up.p, uin, p->udot.p, p->ut.p,
                                     p->Rp.p, p->Rm.p, p->mL.p, p->dir.p, p->udir.p, dt, a, uA, b, out, p->Fs.p));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int cn_predictor(afc_problem_s* p, const double* u_old, double dt) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  AFC_LAUNCH(p, "k_cn_predictor", k_cn_predictor<<<g, kBlock, 0, s>>>(N, p->offs, p->AA.p, u_old, p->f.p, p->mL.p, p->dir.p, p->udir.p, dt, p->ut.p,
                                      p->b0.p));
  AFC_LAUNCH(p, "k_bounds_of", k_bounds_of<<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->ut.p, p->Qp.p, p->Qm.p));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int cn_limited_residual(afc_problem_s* p, const double* u_new, const double* u_old, double dt, int limiter,
                        int prelimit, double* res, double* normsq_slot) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  if (limiter == AFC_LIM_ZALESAK)
    AFC_LAUNCH(p, "k_cn_factors", k_cn_factors<<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->m_up.p, p->d_up.p, u_new, u_old, p->Qp.p, p->Qm.p,
                                      p->mL.p, p->dir.p, dt, prelimit, p->Rp.p, p->Rm.p));
  AFC_LAUNCH(p, "k_cn_residual", k_cn_residual<<<g, kBlock, 0, s>>>(N, p->offs, limiter, p->mask.p, p->m_up.p, p->d_up.p, p->AA.p, u_new, u_old,
                                     p->Rp.p, p->Rm.p, p->b0.p, p->mL.p, p->dir.p, dt, prelimit, res, p->Fs.p,
                                     p->part.p));
  finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
