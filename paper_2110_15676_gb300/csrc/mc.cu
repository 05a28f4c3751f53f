// Monolithic convex limiter for the stationary problem (Sec. 2.2, Sec. 3.1):
// bounds u_i^max/min over N_i (Eq. u_max_min), fluxes r_ij = d_ij (u_j - u_i),
// bar states 2 d_ij ubar_ij = d_ij (u_i + u_j) + a_ij (u_j - u_i) with the
// convective entries a_ij = k_ij (Remark rem:assembling_mc), the clip of
// Eq. MClimiter, and the nonlinear residual f + F*(u) - AA u of Sec. 4.
//
// r*_ji = -r*_ij, so each pair is limited once, by the row of its lower node, and
// stored in r_up; the residual pass sums the stored fluxes of a row.  The clip
// bounds 2 d_ij (ubar_ij - u_i^max) etc. are formed as 2 d_ij ubar_ij - 2 d_ij u_i^max
// without the division by 2 d_ij, and every min / max runs on the integer pipe.
#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

namespace {

// u_max / u_min over N_i, which contains i.
template <int KT>
__global__ void k_mc_bounds(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                            const double* __restrict__ u, double* __restrict__ umax, double* __restrict__ umin) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  double hi = u[i], lo = hi;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!((mk >> k) & 1ull)) continue;
    const double v = u[i + of.o[k]];
    hi = imax(hi, v);
    lo = imin(lo, v);
  }
  umax[i] = hi;
  umin[i] = lo;
}

// r*_ij of Eq. MClimiter for every pair i < j (r_ij itself for the Galerkin mode);
// a pair with d_ij = 0, or outside the pattern, carries no flux.
template <int KT>
__global__ void k_mc_edges(int64_t N, Offsets of, int limiter, const double* __restrict__ d_up,
                           const double* __restrict__ Kf, const double* __restrict__ u,
                           const double* __restrict__ umax, const double* __restrict__ umin,
                           double* __restrict__ r_up) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double ui = u[i], mxi = umax[i], mni = umin[i];
#pragma unroll
  for (int ku = 0; ku < Kup; ++ku) {
    const int64_t q = (int64_t)ku * N + i;
    const int k = Kup + 1 + ku;
    const int64_t j = i + of.o[k];
    const double d = d_up[q];
    double out = 0.0;
    if (!is0(d)) {
      const double uj = u[j];
      const double D = uj - ui;
      const double r = d * D;
      if (limiter == AFC_LIM_GALERKIN) {
        out = r;
      } else {
        const double aij = Kf[(int64_t)k * N + i];
        const double aji = Kf[(int64_t)(Kup - 1 - ku) * N + j];
        const double dS = d * (ui + uj);
        const double tij = fma(aij, D, dS);     // 2 d_ij ubar_ij
        const double tji = fma(-aji, D, dS);    // 2 d_ij ubar_ji
        const double d2 = twice_exact(d);
        if (gt0(r)) {
          const double c1 = fma(-d2, mxi, tij), c2 = fma(d2, umin[j], -tji);
          out = imin(r, imin(c1, c2));
        } else {
          const double c1 = fma(-d2, mni, tij), c2 = fma(d2, umax[j], -tji);
          out = imax(r, imax(c1, c2));
        }
      }
    }
    r_up[q] = out;
  }
}

// res = f + F*(u) - AA u on free rows (0 on Dirichlet rows), block partials of res^2.
template <int KT>
__global__ void k_mc_residual(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                              const double* __restrict__ r_up, const double* __restrict__ AA,
                              const double* __restrict__ u, const double* __restrict__ f,
                              const uint8_t* __restrict__ dir, double* __restrict__ res, double* __restrict__ Fout,
                              double* __restrict__ part) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (i < N) {
    double rv = 0.0, F = 0.0;
    if (!dir[i]) {
      double y = 0.0;
    #pragma unroll
  for (int k = 0; k < K; ++k) y = fma(AA[k * N + i], u[i + of.o[k]], y);
      if (limiter != AFC_LIM_NONE) {
        const unsigned long long mk = mask[i];
      #pragma unroll
  for (int k = 0; k < K; ++k) {
          if (k == Kup || !((mk >> k) & 1ull)) continue;
          const double r = pair_flux(of, Kup, k, i, N, r_up);
          if (!is0(r)) F += r;
        }
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
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    if (limiter == AFC_LIM_MC)
      AFC_LAUNCH(p, "k_mc_bounds",
                 k_mc_bounds<KT><<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, u, p->umax.p, p->umin.p));
    if (limiter != AFC_LIM_NONE)
      AFC_LAUNCH(p, "k_mc_edges", k_mc_edges<KT><<<g, kBlock, 0, s>>>(N, p->offs, limiter, p->d_up.p, p->Kfull.p, u,
                                                                       p->umax.p, p->umin.p, p->r_up.p));
    AFC_LAUNCH(p, "k_mc_residual",
               k_mc_residual<KT><<<g, kBlock, 0, s>>>(N, p->offs, limiter, p->mask.p, p->r_up.p, p->AA.p, u, p->f.p,
                                                      p->dir.p, res, p->Fs.p, p->part.p));
  });
  finalize_sum(p, p->part.p, (int)g, normsq_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
