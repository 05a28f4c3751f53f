// Per-row arithmetic of the explicit FE-SSP stage with Zalesak's limiter
// (Sec. 2.1.2, Sec. 2.1.3), shared by the one-problem kernels (fct.cu) and the
// batched kernels (batch.cu) so that an instance gives the same bits alone and
// in a batch.
//
// The stage has four passes, each needing the previous one on the neighbours:
//   rate     y = AA u, udot^L = (f - y) / m, predictor u~ = u + dt udot^L
//   edges    r_ij of every pair, once per pair at its lower row (Eq. defn_r_ij_SSP)
//   factors  P+/-, Q+/- over N_i, R+/- (Zalesak steps 1-3)
//   correct  alpha_ij, F*_i = sum_j alpha_ij r_ij, u_new = u~ + dt F* / m, and the
//            SSP combination out = a uA + b u_new
//
// Mixed precision (MIXED = true): the raw flux r_ij of a pair is formed in single
// precision, from single-precision copies of m_ij, d_ij, u and udot^L, and stored
// as a float; P+/-, Q+/-, R+/-, alpha, F* and the lumped-mass update stay in
// double and use the float fluxes widened exactly, so the limiter's local bounds
// hold for the fluxes that are actually applied.
#pragma once

#include "kernels_common.cuh"

namespace afc {

// Flux of the pair (i, i + o_k) seen from row i, stored once per pair as a float.
__device__ __forceinline__ double pair_flux32(const Offsets& of, int Kup, int k, int64_t i, int64_t N,
                                              const float* r32) {
  if (k > Kup) return widen_exact(r32[(int64_t)(k - Kup - 1) * N + i]);
  return neg_bits(widen_exact(r32[(int64_t)(Kup - 1 - k) * N + i + of.o[k]]));
}

// Pointers of one instance for the stage passes.  Node vectors carry the halo.
// No pointer here or in the row functions is __restrict__: a persistent batched
// launch writes, in one pass, arrays that later passes of the same launch read,
// so their loads must not take the read-only (non-coherent) cache path.
struct SspArrays {
  int64_t N;
  const double* AA;                 // K * N low-order operator
  const double* m_up;               // Kup * N
  const double* d_up;               // Kup * N
  const float* m32;                 // Kup * N (mixed)
  const float* d32;                 // Kup * N (mixed)
  const double* mL;
  const double* f;
  const uint8_t* dir;
  const double* udir;
  const unsigned long long* mask;
  double* udot;
  double* ut;
  float* uf;                        // mixed: u rounded to single (halo)
  float* udf;                       // mixed: udot^L rounded to single (halo)
  double* r_up;                     // Kup * N
  float* r32;                       // Kup * N (mixed)
  double* Rp;
  double* Rm;
  double* Fs;                       // F* of the stage (may be null)
};

// rate pass at row i (udot^L = 0 at Dirichlet nodes, whose data is constant in time)
template <int KT, bool MIXED>
__device__ __forceinline__ void ssp_rate_row(const Offsets& of, const SspArrays& a, int64_t i,
                                             const double* u, double dt) {
  const int K = KT > 0 ? KT : of.K;
  const int64_t N = a.N;
  double y = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) y = fma(a.AA[k * N + i], u[i + of.o[k]], y);
  const double ui = u[i];
  double ud, uti;
  if (a.dir[i]) {
    ud = 0.0;
    uti = a.udir[i];
  } else {
    ud = (a.f[i] - y) / a.mL[i];
    uti = fma(dt, ud, ui);
  }
  a.udot[i] = ud;
  a.ut[i] = uti;
  if (MIXED) {
    a.uf[i] = __double2float_rn(ui);
    a.udf[i] = __double2float_rn(ud);
  }
}

// edges pass: the Kup pairs (i, i + o) with o > 0 stored at row i
template <int KT, bool MIXED>
__device__ __forceinline__ void ssp_edges_row(const Offsets& of, const SspArrays& a, int64_t i,
                                              const double* u) {
  const int Kup = (KT > 0 ? KT : of.K) / 2;
  const int64_t N = a.N;
  if (MIXED) {
    const float ui = a.uf[i], udi = a.udf[i];
#pragma unroll
    for (int ku = 0; ku < Kup; ++ku) {
      const int64_t q = (int64_t)ku * N + i;
      const int64_t j = i + of.o[Kup + 1 + ku];
      a.r32[q] = fmaf(a.m32[q], udi - a.udf[j], a.d32[q] * (a.uf[j] - ui));
    }
  } else {
    const double ui = u[i], udi = a.udot[i];
#pragma unroll
    for (int ku = 0; ku < Kup; ++ku) {
      const int64_t q = (int64_t)ku * N + i;
      const int64_t j = i + of.o[Kup + 1 + ku];
      a.r_up[q] = fma(a.m_up[q], udi - a.udot[j], a.d_up[q] * (u[j] - ui));
    }
  }
}

template <int KT, bool MIXED>
__device__ __forceinline__ double ssp_flux(const Offsets& of, const SspArrays& a, int k, int64_t i) {
  const int Kup = (KT > 0 ? KT : of.K) / 2;
  if (MIXED) return pair_flux32(of, Kup, k, i, a.N, a.r32);
  return pair_flux(of, Kup, k, i, a.N, a.r_up);
}

// factors pass: P+/- from the stored fluxes, Q+/- from the predictor over N_i, R+/-
template <int KT, bool MIXED>
__device__ __forceinline__ void ssp_factors_row(const Offsets& of, const SspArrays& a, int64_t i, double dt) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  if (a.dir[i]) {
    a.Rp[i] = 1.0;
    a.Rm[i] = 1.0;
    return;
  }
  const unsigned long long mk = a.mask[i];
  const double uti = a.ut[i];
  double Pp = 0.0, Pm = 0.0;
  long long kmax = dkey(uti), kmin = kmax;
  if (MIXED) {
    // The fluxes are floats: P+ and P- are summed exactly in 64-bit fixed point scaled
    // to the row's largest flux (its 24-bit mantissa at bits 33..56, so 62 pairs cannot
    // overflow), then rounded once to double.  This is at least as accurate as a double
    // sum and runs on the integer pipe instead of two FP64 adds per pair.
    constexpr int KA = KT > 0 ? KT : kMaxOffsets;
    unsigned fb[KA];
    unsigned emax = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      fb[k] = 0u;
      if (k == Kup || !((mk >> k) & 1ull)) continue;
      unsigned b;
      if (k > Kup) b = __float_as_uint(a.r32[(int64_t)(k - Kup - 1) * a.N + i]);
      else b = __float_as_uint(a.r32[(int64_t)(Kup - 1 - k) * a.N + i + of.o[k]]) ^ 0x80000000u;   // r_ij = -r_ji
      fb[k] = b;
      const unsigned e = (b >> 23) & 0xffu;
      emax = e > emax ? e : emax;
      const long long kj = dkey(a.ut[i + of.o[k]]);
      kmax = kj > kmax ? kj : kmax;
      kmin = kj < kmin ? kj : kmin;
    }
    if (emax > 0u) {
      long long sp = 0, sm = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const unsigned b = fb[k];
        const int e = (int)((b >> 23) & 0xffu);
        if (e == 0) continue;                       // zero or subnormal: widened to 0 as well
        const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
        const int sh = e - (int)emax + 33;
        const long long v = sh >= 0 ? (m << sh) : (sh > -24 ? (m >> -sh) : 0LL);
        if (b & 0x80000000u) sm += v;
        else sp += v;
      }
      const double scale = __longlong_as_double((long long)((int)emax - 127 - 56 + 1023) << 52);   // 2^(emax-183)
      Pp = (double)sp * scale;
      Pm = -((double)sm * scale);
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k == Kup || !((mk >> k) & 1ull)) continue;
      const double r = ssp_flux<KT, MIXED>(of, a, k, i);
      if (gt0(r)) Pp += r;
      else if (!is0(r)) Pm += r;
      const long long kj = dkey(a.ut[i + of.o[k]]);
      kmax = kj > kmax ? kj : kmax;
      kmin = kj < kmin ? kj : kmin;
    }
  }
  // >= 0 and <= 0: the max / min include i itself
  const double Qp = from_key(kmax) - uti, Qm = from_key(kmin) - uti;
  const double m = a.mL[i];
  a.Rp[i] = zalesak_factor(m * Qp, dt * Pp);
  a.Rm[i] = zalesak_factor(m * Qm, dt * Pm);
}

// correct pass and the SSP combination; returns the new value written to out[i]
template <int KT, bool MIXED>
__device__ __forceinline__ void ssp_correct_row(const Offsets& of, const SspArrays& a, int64_t i, int limiter,
                                                double dt, double ca, const double* uA, double cb,
                                                double* out) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  double unew;
  double F = 0.0;
  if (a.dir[i]) {
    unew = a.udir[i];
  } else {
    if (limiter != AFC_LIM_NONE) {
      const unsigned long long mk = a.mask[i];
      const double rpi = a.Rp[i], rmi = a.Rm[i];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k == Kup || !((mk >> k) & 1ull)) continue;
        const double r = ssp_flux<KT, MIXED>(of, a, k, i);
        if (limiter == AFC_LIM_ZALESAK) {
          const int64_t j = i + of.o[k];
          const double alpha = gt0(r) ? imin_nn(rpi, a.Rm[j]) : imin_nn(rmi, a.Rp[j]);
          F = fma(alpha, r, F);
        } else {
          F += r;
        }
      }
    }
    unew = a.ut[i] + dt * F / a.mL[i];
  }
  if (a.Fs) a.Fs[i] = F;
  out[i] = ca != 0.0 ? ca * uA[i] + cb * unew : cb * unew;
}

}  // namespace afc
