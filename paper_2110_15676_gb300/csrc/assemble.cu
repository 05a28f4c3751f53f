// Device assembly of the Galerkin and low-order matrices (Sec. 2):
//   m_ij = (phi_j, phi_i),  s_ij = (grad phi_j, grad phi_i),  k_ij = (b . grad phi_j, phi_i),
//   M_L = diag(sum_j m_ij),  d_ij = -max{a_ij, 0, a_ji} (i != j),  d_ii = -sum_{j != i} d_ij,
//   AA = A + D  (Eq. low_order_disc).
// One thread owns one matrix row and visits the cells incident to its node, so
// every entry is summed in a fixed order without atomics.
#include <cmath>

#include "afc_internal.h"

namespace afc {

namespace {

__device__ __forceinline__ int find_offset(const Offsets& of, int o) {
  int lo = 0, hi = of.K - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (of.o[mid] < o) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void inv3(const double J[3][3], double Ji[3][3], double& det) {
  det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
        J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double id = 1.0 / det;
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
}

// Row `a` of the element matrices of a tetrahedron with vertices X[4][3] and
// nodal velocity B[4][3] (linear basis lambda_k, exact integrals):
//   M_ab = V (1 + delta_ab) / 20,  S_ab = V grad l_a . grad l_b,
//   C_ab = sum_k (1 + delta_ak) V / 20 * (b_k . grad l_b).
__device__ void p1_row(const double X[4][3], const double B[4][3], int a, double* M, double* S, double* C) {
  double J[3][3], Ji[3][3], det;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) J[r][q] = X[q + 1][r] - X[0][r];   // columns are edge vectors
  inv3(J, Ji, det);
  const double V = fabs(det) / 6.0;
  double G[4][3];
  for (int d = 0; d < 3; ++d) {
    G[1][d] = Ji[0][d];
    G[2][d] = Ji[1][d];
    G[3][d] = Ji[2][d];
    G[0][d] = -(Ji[0][d] + Ji[1][d] + Ji[2][d]);
  }
  for (int b = 0; b < 4; ++b) {
    M[b] = V * (a == b ? 2.0 : 1.0) / 20.0;
    S[b] = V * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
    double cb = 0.0;
    for (int k = 0; k < 4; ++k) {
      double w = V * (a == k ? 2.0 : 1.0) / 20.0;
      cb += w * (B[k][0] * G[b][0] + B[k][1] * G[b][1] + B[k][2] * G[b][2]);
    }
    C[b] = cb;
  }
}

// Row `a` of the reaction matrix (c_h phi_b, phi_a) of a tetrahedron for the linear
// interpolant c_h of the nodal reaction Cn: int l_a l_b l_k = V (1 + d_ab + d_ak + d_bk
// + 2 d_abk) / 120 (the integral of a product of barycentric coordinates).
__device__ void p1_row_reaction(const double X[4][3], const double Cn[4], int a, double* R) {
  double J[3][3], Ji[3][3], det;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) J[r][q] = X[q + 1][r] - X[0][r];
  inv3(J, Ji, det);
  const double V = fabs(det) / 6.0;
  for (int b = 0; b < 4; ++b) {
    double s = 0.0;
    for (int k = 0; k < 4; ++k) {
      const double t = 1.0 + (a == b) + (a == k) + (b == k) + 2.0 * (a == b && b == k);
      s += t * Cn[k];
    }
    R[b] = V * s / 120.0;
  }
}

// Row `a` of the trilinear reaction matrix, 2x2x2 Gauss points (exact on
// parallelepipeds: degree 3 per reference coordinate).
__device__ void q1_row_reaction(const double X[8][3], const double Cn[8], int a, double* R) {
  const double g0 = 0.5 - 0.5 / sqrt(3.0), g1 = 0.5 + 0.5 / sqrt(3.0);
  for (int b = 0; b < 8; ++b) R[b] = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double xi[3] = {(q & 4) ? g1 : g0, (q & 2) ? g1 : g0, (q & 1) ? g1 : g0};
    double phi[8], dr[8][3];
    for (int k = 0; k < 8; ++k) {
      double f[3], df[3];
      for (int d = 0; d < 3; ++d) {
        bool bit = (k >> d) & 1;
        f[d] = bit ? xi[d] : 1.0 - xi[d];
        df[d] = bit ? 1.0 : -1.0;
      }
      phi[k] = f[0] * f[1] * f[2];
      dr[k][0] = df[0] * f[1] * f[2];
      dr[k][1] = f[0] * df[1] * f[2];
      dr[k][2] = f[0] * f[1] * df[2];
    }
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Ji[3][3], det;
    for (int k = 0; k < 8; ++k)
      for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) J[r][d] += X[k][r] * dr[k][d];
    inv3(J, Ji, det);
    double cq = 0.0;
    for (int k = 0; k < 8; ++k) cq += phi[k] * Cn[k];
    const double wd = 0.125 * fabs(det) * cq;
    for (int b = 0; b < 8; ++b) R[b] += wd * phi[a] * phi[b];
  }
}

// Row `a` of the trilinear element matrices, 2x2x2 Gauss points on [0,1]^3.
__device__ void q1_row(const double X[8][3], const double B[8][3], int a, double* M, double* S, double* C) {
  const double g0 = 0.5 - 0.5 / sqrt(3.0), g1 = 0.5 + 0.5 / sqrt(3.0);
  for (int b = 0; b < 8; ++b) M[b] = S[b] = C[b] = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double xi[3] = {(q & 4) ? g1 : g0, (q & 2) ? g1 : g0, (q & 1) ? g1 : g0};
    double phi[8], dr[8][3];
    for (int k = 0; k < 8; ++k) {
      double f[3], df[3];
      for (int d = 0; d < 3; ++d) {
        bool bit = (k >> d) & 1;
        f[d] = bit ? xi[d] : 1.0 - xi[d];
        df[d] = bit ? 1.0 : -1.0;
      }
      phi[k] = f[0] * f[1] * f[2];
      dr[k][0] = df[0] * f[1] * f[2];
      dr[k][1] = f[0] * df[1] * f[2];
      dr[k][2] = f[0] * f[1] * df[2];
    }
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Ji[3][3], det;
    for (int k = 0; k < 8; ++k)
      for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) J[r][d] += X[k][r] * dr[k][d];
    inv3(J, Ji, det);
    const double wd = 0.125 * fabs(det);
    double g[8][3], bq[3] = {0, 0, 0};
    for (int k = 0; k < 8; ++k) {
      for (int r = 0; r < 3; ++r) g[k][r] = dr[k][0] * Ji[0][r] + dr[k][1] * Ji[1][r] + dr[k][2] * Ji[2][r];
      for (int r = 0; r < 3; ++r) bq[r] += phi[k] * B[k][r];
    }
    for (int b = 0; b < 8; ++b) {
      M[b] += wd * phi[a] * phi[b];
      S[b] += wd * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
      C[b] += wd * phi[a] * (bq[0] * g[b][0] + bq[1] * g[b][1] + bq[2] * g[b][2]);
    }
  }
}

template <int NL>
__global__ void k_assemble_rows(int64_t N, Offsets of, const double* __restrict__ xyz, const double* __restrict__ bn,
                                const int32_t* __restrict__ conn, const int32_t* __restrict__ inc_ptr,
                                const int32_t* __restrict__ inc, double* __restrict__ Mf, double* __restrict__ Sf,
                                double* __restrict__ Kf, const double* __restrict__ cn, double* __restrict__ Rf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double am[kMaxOffsets], as[kMaxOffsets], ak[kMaxOffsets], ar[kMaxOffsets];
  for (int k = 0; k < of.K; ++k) am[k] = as[k] = ak[k] = ar[k] = 0.0;
  for (int t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
    const int code = inc[t];
    const int64_t e = code >> 3;
    const int a = code & 7;
    double X[NL][3], B[NL][3];
    int v[NL];
    for (int k = 0; k < NL; ++k) {
      v[k] = conn[e * NL + k];
      for (int d = 0; d < 3; ++d) {
        X[k][d] = xyz[3 * (int64_t)v[k] + d];
        B[k][d] = bn[3 * (int64_t)v[k] + d];
      }
    }
    double M[NL], S[NL], C[NL], R[NL];
    if (NL == 4) p1_row((const double(*)[3])X, (const double(*)[3])B, a, M, S, C);
    else q1_row((const double(*)[3])X, (const double(*)[3])B, a, M, S, C);
    if (cn) {   // nodal reaction: its Galerkin matrix
      double Cn[NL];
      for (int k = 0; k < NL; ++k) Cn[k] = cn[v[k]];
      if (NL == 4) p1_row_reaction((const double(*)[3])X, Cn, a, R);
      else q1_row_reaction((const double(*)[3])X, Cn, a, R);
    }
    for (int b = 0; b < NL; ++b) {
      int k = find_offset(of, v[b] - (int)i);
      am[k] += M[b];
      as[k] += S[b];
      ak[k] += C[b];
      if (cn) ar[k] += R[b];
    }
  }
  for (int k = 0; k < of.K; ++k) {
    Mf[k * N + i] = am[k];
    Sf[k * N + i] = as[k];
    Kf[k * N + i] = ak[k];
    if (cn) Rf[k * N + i] = ar[k];
  }
}

// mL, f = M_L f_nodal, the lumped reaction rl (c m_i, or the row sums of the nodal
// reaction's matrix Rf), and the matrix whose off-diagonals define D.
__global__ void k_lumped_and_A(int64_t N, Offsets of, int family, double eps, double c, const double* __restrict__ Mf,
                               const double* __restrict__ Sf, const double* __restrict__ Kf,
                               const double* __restrict__ Rf, const double* __restrict__ fn,
                               double* __restrict__ mL, double* __restrict__ f, double* __restrict__ rl,
                               double* __restrict__ Af) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0, sr = 0.0;
  for (int k = 0; k < of.K; ++k) s += Mf[k * N + i];
  if (Rf)
    for (int k = 0; k < of.K; ++k) sr += Rf[k * N + i];
  mL[i] = s;
  f[i] = s * fn[i];
  rl[i] = Rf ? sr : c * s;
  for (int k = 0; k < of.K; ++k) {
    size_t q = k * N + i;
    Af[q] = family == AFC_FAMILY_FCT ? (eps * Sf[q] + Kf[q]) + (Rf ? Rf[q] : c * Mf[q]) : Kf[q];
  }
}

// d_ij for the pair (i, i + o) with o > 0, stored at row i.
__global__ void k_upwind_edges(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                               const double* __restrict__ Af, double* __restrict__ dup) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  for (int ku = 0; ku < of.Kup; ++ku) {
    const int k = of.Kup + 1 + ku;        // offset index of +o
    const int km = of.Kup - 1 - ku;       // offset index of -o
    double d = 0.0;
    if ((mk >> k) & 1ull) {
      const double aij = Af[k * N + i];
      const double aji = Af[km * N + i + of.o[k]];
      d = -fmax(fmax(aij, 0.0), aji);
    }
    dup[ku * N + i] = d;
  }
}

// AA = A + D (FCT) or K + D + eps S + (lumped reaction) (MC), full rows.
__global__ void k_low_order(int64_t N, Offsets of, int family, double eps, const double* __restrict__ rl,
                            const unsigned long long* __restrict__ mask, const double* __restrict__ Af,
                            const double* __restrict__ Sf,
                            const double* __restrict__ dup, double* __restrict__ AAf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  double dsum = 0.0;
  for (int k = 0; k < of.K; ++k) {
    if (k == of.Kup) continue;
    double d = 0.0;
    if ((mk >> k) & 1ull) {
      if (k > of.Kup) d = dup[(k - of.Kup - 1) * N + i];
      else d = dup[(of.Kup - 1 - k) * N + i + of.o[k]];   // pair (i + o, i) is stored at its lower row
    }
    dsum += d;
    double v = Af[k * N + i] + d;
    if (family == AFC_FAMILY_MC) v = v + eps * Sf[k * N + i];
    AAf[k * N + i] = v;
  }
  double dv = Af[of.Kup * N + i] + (-dsum);
  if (family == AFC_FAMILY_MC) dv = (dv + eps * Sf[of.Kup * N + i]) + rl[i];
  AAf[of.Kup * N + i] = dv;
}

// MC family: the convective entries of each pair i < j at row i (k_ij, k_ji) and the
// unlimited operator AG = K + eps S + c M_L (AA without D) of the residual.
__global__ void k_mc_extras(int64_t N, Offsets of, double eps, const double* __restrict__ rl,
                            const unsigned long long* __restrict__ mask,
                            const double* __restrict__ Kf, const double* __restrict__ Sf, const double* __restrict__ dup,
                            double* __restrict__ kij, double* __restrict__ kji, double* __restrict__ d2,
                            float* __restrict__ pairf, double* __restrict__ AG) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long mk = mask[i];
  for (int ku = 0; ku < of.Kup; ++ku) {
    const int k = of.Kup + 1 + ku;
    const bool present = (mk >> k) & 1ull;
    kij[ku * N + i] = present ? Kf[k * N + i] : 0.0;
    kji[ku * N + i] = present ? Kf[(of.Kup - 1 - ku) * N + i + of.o[k]] : 0.0;
    d2[ku * N + i] = -2.0 * dup[ku * N + i];
    const int64_t KN = (int64_t)of.Kup * N;
    pairf[ku * N + i] = (float)d2[ku * N + i];
    pairf[KN + ku * N + i] = (float)kij[ku * N + i];
    pairf[2 * KN + ku * N + i] = (float)kji[ku * N + i];
  }
  for (int k = 0; k < of.K; ++k) {
    double v = Kf[k * N + i] + eps * Sf[k * N + i];
    if (k == of.Kup) v = v + rl[i];
    AG[k * N + i] = v;
  }
}

// System matrix: scale * AA, plus m_i / dt on the diagonal if dt > 0; Dirichlet rows -> identity.
template <class T>
__global__ void k_system(int64_t N, Offsets of, const double* __restrict__ AAf, const double* __restrict__ mL,
                         const uint8_t* __restrict__ dir, double scale, double dt, T* __restrict__ B,
                         T* __restrict__ dinv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool isd = dir[i] != 0;
  double diag = 1.0;
  for (int k = 0; k < of.K; ++k) {
    double v;
    if (isd) v = (k == of.Kup) ? 1.0 : 0.0;
    else {
      v = scale * AAf[k * N + i];
      if (k == of.Kup && dt > 0.0) v = mL[i] / dt + v;
    }
    if (k == of.Kup) diag = v;
    B[k * N + i] = (T)v;
  }
  dinv[i] = (T)(1.0 / diag);
}

}  // namespace

int assemble_device(afc_problem_s* p, int family, int precision) {
  const int64_t N = p->N;
  const int K = p->K, Kup = p->Kup;
  cudaStream_t s = p->stream;
  int st;
  if ((st = p->Mfull.alloc(K * N)) || (st = p->Sfull.alloc(K * N)) || (st = p->Kfull.alloc(K * N)) ||
      (st = p->Afull.alloc(K * N)) || (st = p->AA.alloc(K * N)) || (st = p->m_up.alloc(Kup * N)) ||
      (st = p->d_up.alloc(Kup * N)) || (st = p->mL.alloc(N, p->pad)) || (st = p->f.alloc(N, p->pad)) ||
      (st = p->Bst.alloc(K * N)) || (st = p->dinv_st.alloc(N, p->pad)) || (st = p->r_up.alloc(Kup * N)) ||
      (st = p->rl.alloc(N, p->pad)))
    return st;
  const bool nodal_c = p->c_nodal;
  if (nodal_c && (st = p->Rfull.alloc(K * N))) return st;
  const double* cn = nodal_c ? p->cnod.p : nullptr;
  double* Rf = nodal_c ? p->Rfull.p : nullptr;
  const int64_t g = grid_for(N);
  if (p->mesh.nl == 4)
    AFC_LAUNCH(p, "k_assemble_rows", k_assemble_rows<4><<<g, kBlock, 0, s>>>(N, p->offs, p->xyz.p, p->bnod.p, p->conn.p, p->inc_ptr.p, p->inc.p,
                                             p->Mfull.p, p->Sfull.p, p->Kfull.p, cn, Rf));
  else
    AFC_LAUNCH(p, "k_assemble_rows", k_assemble_rows<8><<<grid_for(N, 128), 128, 0, s>>>(N, p->offs, p->xyz.p, p->bnod.p, p->conn.p, p->inc_ptr.p,
                                                         p->inc.p, p->Mfull.p, p->Sfull.p, p->Kfull.p, cn, Rf));
  AFC_CUDA(cudaGetLastError());
  AFC_LAUNCH(p, "k_lumped_and_A", k_lumped_and_A<<<g, kBlock, 0, s>>>(N, p->offs, family, p->eps, p->c, p->Mfull.p, p->Sfull.p, p->Kfull.p, Rf,
                                      p->fnod.p, p->mL.p, p->f.p, p->rl.p, p->Afull.p));
  AFC_LAUNCH(p, "k_upwind_edges", k_upwind_edges<<<g, kBlock, 0, s>>>(N, p->offs, p->mask.p, p->Afull.p, p->d_up.p));
  AFC_LAUNCH(p, "k_low_order", k_low_order<<<g, kBlock, 0, s>>>(N, p->offs, family, p->eps, p->rl.p, p->mask.p, p->Afull.p, p->Sfull.p,
                                   p->d_up.p, p->AA.p));
  if (family == AFC_FAMILY_MC) {
    if ((st = p->kij_up.alloc(Kup * N)) || (st = p->kji_up.alloc(Kup * N)) || (st = p->d2_up.alloc(Kup * N)) ||
        (st = p->AG.alloc(K * N)) || (st = p->clip.alloc(N, p->pad)) || (st = p->pairf.alloc(3 * Kup * N)) ||
        (st = p->nodef.alloc(N, p->pad)))
      return st;
    AFC_LAUNCH(p, "k_mc_extras", k_mc_extras<<<g, kBlock, 0, s>>>(N, p->offs, p->eps, p->rl.p, p->mask.p, p->Kfull.p,
                                                                   p->Sfull.p, p->d_up.p, p->kij_up.p,
                                                                   p->kji_up.p, p->d2_up.p, p->pairf.p, p->AG.p));
    if (precision == AFC_MIXED && (st = mc_pair_setup(p))) return st;
  }
  // symmetric mass data of the upper half: m_up[ku][i] = m_{i, i + o}
  for (int ku = 0; ku < Kup; ++ku)
    AFC_CUDA(cudaMemcpyAsync(p->m_up.p + ku * N, p->Mfull.p + (Kup + 1 + ku) * N, N * sizeof(double),
                             cudaMemcpyDeviceToDevice, s));
  AFC_LAUNCH(p, "k_system", k_system<double><<<g, kBlock, 0, s>>>(N, p->offs, p->AA.p, p->mL.p, p->dir.p, 1.0, 0.0, p->Bst.p, p->dinv_st.p));
  if (precision == AFC_MIXED) {
    if ((st = p->Bst32.alloc(K * N)) || (st = p->dinv_st32.alloc(N, p->pad))) return st;
    AFC_LAUNCH(p, "k_system", k_system<float><<<g, kBlock, 0, s>>>(N, p->offs, p->AA.p, p->mL.p, p->dir.p, 1.0, 0.0, p->Bst32.p,
                                         p->dinv_st32.p));
  }
  AFC_CUDA(cudaGetLastError());
  AFC_CUDA(cudaStreamSynchronize(s));
  p->family = family;
  p->precision = precision;
  p->cn_dt = -1.0;
  p->ssp32_ready = false;
  p->assembled = true;
  return AFC_OK;
}

namespace {
// m_ij / dt for the pairs and m_i / dt for the nodes of the CN step
__global__ void k_scale_by_dt(int64_t n, const double* __restrict__ x, double dt, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] / dt;
}
}  // namespace

int build_cn_system(afc_problem_s* p, double dt) {
  if (p->cn_dt == dt) return AFC_OK;
  const int64_t N = p->N;
  int st;
  if ((st = p->Bcn.alloc(p->K * N)) || (st = p->dinv_cn.alloc(N, p->pad)) || (st = p->mdt_up.alloc(p->Kup * N)) ||
      (st = p->mLdt.alloc(N, p->pad)))
    return st;
  const int64_t g = grid_for(N);
  AFC_LAUNCH(p, "k_scale_by_dt", k_scale_by_dt<<<grid_for(p->Kup * N), kBlock, 0, p->stream>>>(p->Kup * N, p->m_up.p,
                                                                                              dt, p->mdt_up.p));
  AFC_LAUNCH(p, "k_scale_by_dt", k_scale_by_dt<<<g, kBlock, 0, p->stream>>>(N, p->mL.p, dt, p->mLdt.p));
  AFC_LAUNCH(p, "k_system", k_system<double><<<g, kBlock, 0, p->stream>>>(N, p->offs, p->AA.p, p->mL.p, p->dir.p, 0.5, dt, p->Bcn.p,
                                                p->dinv_cn.p));
  if (p->precision == AFC_MIXED) {
    if ((st = p->Bcn32.alloc(p->K * N)) || (st = p->dinv_cn32.alloc(N, p->pad))) return st;
    AFC_LAUNCH(p, "k_system", k_system<float><<<g, kBlock, 0, p->stream>>>(N, p->offs, p->AA.p, p->mL.p, p->dir.p, 0.5, dt, p->Bcn32.p,
                                                 p->dinv_cn32.p));
  }
  AFC_CUDA(cudaGetLastError());
  p->cn_dt = dt;
  return AFC_OK;
}

}  // namespace afc
