// Monolithic convex limiter for the stationary problem (Sec. 2.2, Sec. 3.1):
// bounds u_i^max/min over N_i (Eq. u_max_min), fluxes r_ij = d_ij (u_j - u_i),
// bar states 2 d_ij ubar_ij = d_ij (u_i + u_j) + a_ij (u_j - u_i) with the
// convective entries a_ij = k_ij (Remark rem:assembling_mc), the clip of
// Eq. MClimiter, and the nonlinear residual f + F*(u) - AA u of Sec. 4.
#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

namespace {

// u_max / u_min over N_i, which contains i.
__global__ void k_mc_bounds(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                            const double* __restrict__ u, double* __restrict__ umax, double* __restrict__ umin) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  double hi = u[i], lo = hi;
  for (int k = 0; k < of.K; ++k) {
    if (!((mk >> k) & 1ull)) continue;
    const double v = u[i + of.o[k]];
    hi = fmax(hi, v);
    lo = fmin(lo, v);
  }
  umax[i] = hi;
  umin[i] = lo;
}

// r*_ij of Eq. MClimiter; an edge with d_ij = 0 carries no flux.
__device__ __forceinline__ double mc_flux(double d, double aij, double aji, double ui, double uj, double umax_i,
                                          double umin_i, double umax_j, double umin_j) {
  const double r = d * (uj - ui);
  if (d == 0.0) return 0.0;
  const double ubij = (d * (ui + uj) + aij * (uj - ui)) / (2.0 * d);
  const double ubji = (d * (uj + ui) + aji * (ui - uj)) / (2.0 * d);
  if (r > 0.0) return fmin(r, fmin(2.0 * d * (ubij - umax_i), 2.0 * d * (umin_j - ubji)));
  return fmax(r, fmax(2.0 * d * (ubij - umin_i), 2.0 * d * (umax_j - ubji)));
}

// res = f + F*(u) - AA u on free rows (0 on Dirichlet rows), block partials of res^2.
__global__ void k_mc_residual(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const double* __restrict__ d_up, const double* __restrict__ Kf,
                              const double* __restrict__ AA, const double* __restrict__ u,
                              const double* __restrict__ umax, const double* __restrict__ umin,
                              const double* __restrict__ f, const uint8_t* __restrict__ dir,
                              double* __restrict__ res, double* __restrict__ Fout, double* __restrict__ part) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (i < N) {
    double rv = 0.0, F = 0.0;
    if (!dir[i]) {
      const unsigned long long mk = mask[i];
      const double ui = u[i];
      const double mxi = umax[i], mni = umin[i];
      double y = 0.0;
      for (int k = 0; k < of.K; ++k) {
        const int64_t j = i + of.o[k];
        const double uj = u[j];
        y = fma(AA[k * N + i], uj, y);
        if (limiter == AFC_LIM_NONE || k == of.Kup || !((mk >> k) & 1ull)) continue;
        const double d = pair_d(of, k, i, N, d_up);
        double rs;
        if (limiter == AFC_LIM_GALERKIN) {
          rs = d * (uj - ui);
        } else {
          const double aij = Kf[k * N + i];
          const double aji = Kf[(int64_t)(of.K - 1 - k) * N + j];
          rs = mc_flux(d, aij, aji, ui, uj, mxi, mni, umax[j], umin[j]);
        }
        F += rs;
      }
      rv = f[i] + F - y;
    }
    res[i] = rv;
    if (Fout) Fout[i] = F;
    r2 = rv * rv;
  }
  block_sum_to(r2, part);
}

}  // namespace

int mc_limited_residual(afc_problem_s* p, const double* u, int limiter, double* res, double* normsq_slot) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  if (limiter == AFC_LIM_MC)
    AFC_LAUNCH(p, "k_mc_bounds", k_mc_bounds<<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, u, p->umax.p, p->umin.p));
  AFC_LAUNCH(p, "k_mc_residual", k_mc_residual<<<g, kBlock, 0, s>>>(N, p->offs, limiter, p->mask.p, p->d_up.p, p->Kfull.p, p->AA.p, u, p->umax.p,
                                     p->umin.p, p->f.p, p->dir.p, res, p->Fs.p, p->part.p));
  finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
