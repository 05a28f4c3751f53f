// Jacobi-preconditioned Krylov solvers for the constant M-matrix systems of the
// fixed-point iteration (Sec. 4; Tables 1 and 3: BiCGStab, GMRES, Jacobi), run
// entirely on the device.  Solver scalars (rho, alpha, omega, Hessenberg
// columns, Givens rotations) live in device memory and are finalised by
// one-block kernels, so the host only polls a status word every few iterations
// (BiCGStab) or once per restart cycle (GMRES).  All reductions are two-stage
// with a fixed order, so results do not depend on scheduling.
//
// Vector type T is double (FP64) or float (the FP32 inner solve of the mixed
// mode, with FP32 matrix values).  Partial sums are always double.
#include <cmath>
#include <cstring>

#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

int64_t grid_for(int64_t n, int block) { return (n + block - 1) / block; }

template <class T>
int DBuf<T>::alloc(int64_t n_, int64_t pad_) {
  if (base && n == n_ && pad == pad_) return AFC_OK;
  free_();
  size_t bytes = (size_t)(n_ + 2 * pad_) * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  cudaError_t e = cudaMalloc((void**)&base, bytes);
  if (e != cudaSuccess) {
    base = nullptr;
    cudaGetLastError();
    set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    return AFC_E_OOM;
  }
  e = cudaMemset(base, 0, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  n = n_;
  pad = pad_;
  p = base + pad_;
  return AFC_OK;
}

template <class T>
void DBuf<T>::free_() {
  if (base) cudaFree(base);
  base = p = nullptr;
  n = pad = 0;
}

template struct DBuf<double>;
template struct DBuf<float>;
template struct DBuf<int32_t>;
template struct DBuf<uint8_t>;
template struct DBuf<unsigned long long>;

namespace {

__global__ void k_finalize_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v += part[q];
  block_sum_to(v, out);   // one block: out[0]
}

}  // namespace

void finalize_sum(afc_problem_s* p, const double* part, int n, double* out) {
  AFC_LAUNCH(p, "k_finalize_sum", k_finalize_sum<<<1, 1024, 0, p->stream>>>(part, n, out));
}

// ---------------------------------------------------------------------------
// BLAS-1 helpers on double vectors (outer loop)
// ---------------------------------------------------------------------------
namespace {

__global__ void k_dot(int64_t N, const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ part) {
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v = fma(x[i], y[i], v);
  block_sum_to(v, part);
}

__global__ void k_axpy(int64_t N, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] + a * x[i];
}

__global__ void k_minmax(int64_t N, const double* __restrict__ x, double* __restrict__ part) {
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    mn = fmin(mn, x[i]);
    mx = fmax(mx, x[i]);
  }
  __shared__ double smn[kBlock], smx[kBlock];
  smn[threadIdx.x] = mn;
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + s]);
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = smn[0];
    part[2 * blockIdx.x + 1] = smx[0];
  }
}

__global__ void k_minmax_fin(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double mn = INFINITY, mx = -INFINITY;
  for (int q = 0; q < n; ++q) {
    mn = fmin(mn, part[2 * q]);
    mx = fmax(mx, part[2 * q + 1]);
  }
  out[0] = mn;
  out[1] = mx;
}

template <class T, class TV>
__global__ void k_spmv(int64_t N, Offsets of, const T* __restrict__ A, const TV* __restrict__ x, TV* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  TV s = 0;
#pragma unroll 4
  for (int k = 0; k < of.K; ++k) s = fma((TV)A[k * N + i], x[i + of.o[k]], s);
  y[i] = s;
}

}  // namespace

int dot_device(afc_problem_s* p, const double* x, const double* y, double* out_slot) {
  AFC_LAUNCH(p, "k_dot", k_dot<<<kRedBlocks, kBlock, 0, p->stream>>>(p->N, x, y, p->part.p));
  finalize_sum(p, p->part.p, kRedBlocks, out_slot);
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int axpy_device(afc_problem_s* p, double a, const double* x, double* y) {
  AFC_LAUNCH(p, "k_axpy", k_axpy<<<kRedBlocks, kBlock, 0, p->stream>>>(p->N, a, x, y));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

int minmax_device(afc_problem_s* p, const double* x, double* mn, double* mx) {
  AFC_LAUNCH(p, "k_minmax", k_minmax<<<kRedBlocks, kBlock, 0, p->stream>>>(p->N, x, p->part.p));
  AFC_LAUNCH(p, "k_minmax_fin", k_minmax_fin<<<1, 32, 0, p->stream>>>(p->part.p, kRedBlocks, p->scal.p + 60));
  AFC_CUDA(cudaGetLastError());
  AFC_CUDA(cudaMemcpyAsync(p->host_scal + 60, p->scal.p + 60, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  AFC_CUDA(cudaStreamSynchronize(p->stream));
  *mn = p->host_scal[60];
  *mx = p->host_scal[61];
  return AFC_OK;
}

int dia_spmv(afc_problem_s* p, const double* A, const double* x, double* y) {
  AFC_LAUNCH(p, "k_spmv", k_spmv<double, double><<<grid_for(p->N), kBlock, 0, p->stream>>>(p->N, p->offs, A, x, y));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

// ---------------------------------------------------------------------------
// Solver workspace
// ---------------------------------------------------------------------------
constexpr int kMaxRestart = 64;

// device scalar slots
enum : int {
  S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_TOL, S_NRES, S_N0, S_ITS, S_DONE, S_MAXIT,
  S_BETA, S_K_USED, S_INVH, S_CYCLE_DONE, S_FIRST,
  S_CS = 16, S_SN = S_CS + kMaxRestart, S_G = S_SN + kMaxRestart, S_Y = S_G + kMaxRestart + 1,
  S_H1 = S_Y + kMaxRestart, S_H2 = S_H1 + kMaxRestart + 1, S_HCOL = S_H2 + kMaxRestart + 1,
  S_END = S_HCOL + (kMaxRestart + 1) * kMaxRestart
};
// S_DONE: 0 running, 1 converged, 2 breakdown / non-finite, 3 converged at s (x update pending), 4 maxit

struct KrylovWork {
  int64_t N = 0;
  int pad = 0, m = 0, fp32 = -1;
  DBuf<char> vec;       // all vectors (with halos)
  DBuf<double> sc, part;
  double* hsc = nullptr;
  size_t vstride = 0;   // elements per vector incl. halo
  void* vptr(int q) { return vec.base + q * vstride * (fp32 ? sizeof(float) : sizeof(double)); }
};

template struct DBuf<char>;

namespace {

// ---- BiCGStab ----
template <class T>
__global__ void k_bicg_init(int64_t N, const double* __restrict__ rhs, T* x, T* r, T* rh, T* p, T* v,
                            double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = (T)rhs[i];
    x[i] = 0;
    r[i] = ri;
    rh[i] = ri;
    p[i] = 0;
    v[i] = 0;
    acc += (double)ri * (double)ri;
  }
  block_sum_to(acc, part);
}

__global__ void k_bicg_init_fin(const double* __restrict__ part, int n, double* sc, double atol, double rtol,
                                int maxit) {
  __shared__ double tot;
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v += part[q];
  block_sum_to(v, sc + S_END);   // scratch slot past the named ones
  if (threadIdx.x == 0) {
    tot = sc[S_END];
    const double n0 = sqrt(tot);
    sc[S_N0] = n0;
    sc[S_NRES] = n0;
    sc[S_RHO] = tot;
    sc[S_RHO_OLD] = 1.0;
    sc[S_ALPHA] = 1.0;
    sc[S_OMEGA] = 1.0;
    sc[S_TOL] = fmax(atol, rtol * n0);
    sc[S_ITS] = 0.0;
    sc[S_MAXIT] = (double)maxit;
    sc[S_DONE] = !isfinite(n0) ? 2.0 : (n0 < sc[S_TOL] ? 1.0 : (maxit <= 0 ? 4.0 : 0.0));
  }
}

template <class T>
__global__ void k_bicg_p(int64_t N, const double* __restrict__ sc, const T* __restrict__ r, T* p,
                         const T* __restrict__ v, const T* __restrict__ dinv, T* __restrict__ ph) {
  if (sc[S_DONE] != 0.0) return;
  const T beta = (T)((sc[S_RHO] / sc[S_RHO_OLD]) * (sc[S_ALPHA] / sc[S_OMEGA]));
  const T om = (T)sc[S_OMEGA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T pi = r[i] + beta * (p[i] - om * v[i]);
    p[i] = pi;
    ph[i] = dinv[i] * pi;
  }
}

// y = B x (row i), plus block partials of sum(a * y) (one dot) or of (y.s, y.y) (two dots)
template <class T, int NDOT>
__global__ void k_bicg_spmv(int64_t N, Offsets of, const double* __restrict__ sc, const T* __restrict__ B,
                            const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ a,
                            double* __restrict__ part, int64_t pstride) {
  if (sc[S_DONE] != 0.0) return;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc[NDOT];
#pragma unroll
  for (int q = 0; q < NDOT; ++q) acc[q] = 0.0;
  if (i < N) {
    T s = 0;
#pragma unroll 4
    for (int k = 0; k < of.K; ++k) s = fma(B[k * N + i], x[i + of.o[k]], s);
    y[i] = s;
    if (NDOT == 1) {
      acc[0] = (double)a[i] * (double)s;
    } else {
      acc[0] = (double)s * (double)a[i];
      acc[NDOT - 1] = (double)s * (double)s;
    }
  }
  block_sums_to<NDOT>(acc, part, pstride);
}

__global__ void k_bicg_fin_alpha(const double* __restrict__ part, int n, double* sc) {
  if (sc[S_DONE] != 0.0) return;
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v += part[q];
  block_sum_to(v, sc + S_END);
  if (threadIdx.x == 0) {
    const double rv = sc[S_END];
    const double al = sc[S_RHO] / rv;
    if (!isfinite(al) || rv == 0.0) sc[S_DONE] = 2.0;
    else sc[S_ALPHA] = al;
  }
}

template <class T>
__global__ void k_bicg_s(int64_t N, const double* __restrict__ sc, const T* __restrict__ r, const T* __restrict__ v,
                         const T* __restrict__ dinv, T* __restrict__ s, T* __restrict__ sh, double* __restrict__ part) {
  if (sc[S_DONE] != 0.0) return;
  const T al = (T)sc[S_ALPHA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T si = r[i] - al * v[i];
    s[i] = si;
    sh[i] = dinv[i] * si;
    acc += (double)si * (double)si;
  }
  block_sum_to(acc, part);
}

__global__ void k_bicg_fin_s(const double* __restrict__ part, int n, double* sc) {
  if (sc[S_DONE] != 0.0) return;
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v += part[q];
  block_sum_to(v, sc + S_END);
  if (threadIdx.x == 0) {
    const double ns = sqrt(sc[S_END]);
    if (!isfinite(ns)) { sc[S_DONE] = 2.0; return; }
    if (ns < sc[S_TOL]) {
      sc[S_NRES] = ns;
      sc[S_ITS] += 1.0;
      sc[S_DONE] = 3.0;     // converged at s: x += alpha phat still to do
    }
  }
}

// x += alpha phat once, when the solve converged at s
template <class T>
__global__ void k_bicg_early_x(int64_t N, const double* __restrict__ sc, T* __restrict__ x, const T* __restrict__ ph) {
  if (sc[S_DONE] != 3.0) return;
  const T al = (T)sc[S_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = x[i] + al * ph[i];
}

__global__ void k_bicg_fin_omega(const double* __restrict__ part, int n, int64_t pstride, double* sc) {
  if (sc[S_DONE] == 3.0) {
    if (threadIdx.x == 0) sc[S_DONE] = 1.0;
    return;
  }
  if (sc[S_DONE] != 0.0) return;
  double v0 = 0.0, v1 = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    v0 += part[q];
    v1 += part[pstride + q];
  }
  double vv[2] = {v0, v1};
  block_sums_to<2>(vv, sc + S_END, 1);
  if (threadIdx.x == 0) {
    const double ts = sc[S_END], tt = sc[S_END + 1];
    const double om = ts / tt;
    if (!isfinite(om) || tt == 0.0) sc[S_DONE] = 2.0;
    else sc[S_OMEGA] = om;
  }
}

template <class T>
__global__ void k_bicg_xr(int64_t N, const double* __restrict__ sc, T* __restrict__ x, const T* __restrict__ ph,
                          const T* __restrict__ sh, const T* __restrict__ s, const T* __restrict__ t,
                          T* __restrict__ r, const T* __restrict__ rh, double* __restrict__ part, int64_t pstride) {
  if (sc[S_DONE] != 0.0) return;
  const T al = (T)sc[S_ALPHA], om = (T)sc[S_OMEGA];
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = x[i] + al * ph[i] + om * sh[i];
    const T ri = s[i] - om * t[i];
    r[i] = ri;
    acc[0] += (double)ri * (double)ri;
    acc[1] += (double)rh[i] * (double)ri;
  }
  block_sums_to<2>(acc, part, pstride);
}

__global__ void k_bicg_fin_r(const double* __restrict__ part, int n, int64_t pstride, double* sc) {
  if (sc[S_DONE] != 0.0) return;
  double v0 = 0.0, v1 = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    v0 += part[q];
    v1 += part[pstride + q];
  }
  double vv[2] = {v0, v1};
  block_sums_to<2>(vv, sc + S_END, 1);
  if (threadIdx.x == 0) {
    const double nr = sqrt(sc[S_END]);
    sc[S_NRES] = nr;
    sc[S_RHO_OLD] = sc[S_RHO];
    sc[S_RHO] = sc[S_END + 1];
    sc[S_ITS] += 1.0;
    if (!isfinite(nr)) sc[S_DONE] = 2.0;
    else if (nr < sc[S_TOL]) sc[S_DONE] = 1.0;
    else if (sc[S_ITS] >= sc[S_MAXIT]) sc[S_DONE] = 4.0;
  }
}

template <class T>
__global__ void k_to_double(int64_t N, const T* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// ---- GMRES(m), right Jacobi preconditioning, classical Gram-Schmidt with one
// re-orthogonalisation pass ----

// w = rhs - B x  (x = 0 on the first cycle), partial ||w||^2
template <class T>
__global__ void k_gm_residual(int64_t N, Offsets of, const double* __restrict__ sc, const T* __restrict__ B,
                              const T* __restrict__ x, const double* __restrict__ rhs, T* __restrict__ w,
                              double* __restrict__ part) {
  if (sc[S_DONE] != 0.0) return;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < N) {
    T s = 0;
    if (sc[S_FIRST] == 0.0) {
#pragma unroll 4
      for (int k = 0; k < of.K; ++k) s = fma(B[k * N + i], x[i + of.o[k]], s);
    }
    const T wi = (T)rhs[i] - s;
    w[i] = wi;
    acc = (double)wi * (double)wi;
  }
  block_sum_to(acc, part);
}

// beta = ||r||; stop test on the true residual; start a new cycle
__global__ void k_gm_start(const double* __restrict__ part, int n, double* sc, double atol, double rtol, int maxit) {
  if (sc[S_DONE] != 0.0) return;
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v += part[q];
  block_sum_to(v, sc + S_END);
  if (threadIdx.x == 0) {
    const double beta = sqrt(sc[S_END]);
    if (sc[S_FIRST] != 0.0) {
      sc[S_N0] = beta;
      sc[S_TOL] = fmax(atol, rtol * beta);
      sc[S_ITS] = 0.0;
      sc[S_MAXIT] = (double)maxit;
      sc[S_FIRST] = 0.0;
    }
    sc[S_NRES] = beta;
    sc[S_BETA] = beta;
    sc[S_K_USED] = 0.0;
    sc[S_CYCLE_DONE] = 0.0;
    if (!isfinite(beta)) sc[S_DONE] = 2.0;
    else if (beta < sc[S_TOL]) sc[S_DONE] = 1.0;
    else if (sc[S_ITS] >= sc[S_MAXIT]) sc[S_DONE] = 4.0;
    for (int q = 0; q <= kMaxRestart; ++q) sc[S_G + q] = 0.0;
    sc[S_G] = beta;
    sc[S_INVH] = 1.0 / beta;
  }
}

// v_k = w * invh; z = dinv * v_k
template <class T>
__global__ void k_gm_normalize(int64_t N, const double* __restrict__ sc, const T* __restrict__ w, T* __restrict__ vk,
                               const T* __restrict__ dinv, T* __restrict__ z) {
  if (sc[S_DONE] != 0.0 || sc[S_CYCLE_DONE] != 0.0) return;
  const T ih = (T)sc[S_INVH];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T vi = w[i] * ih;
    vk[i] = vi;
    z[i] = dinv[i] * vi;
  }
}

template <class T>
__global__ void k_gm_spmv(int64_t N, Offsets of, const double* __restrict__ sc, const T* __restrict__ B,
                          const T* __restrict__ z, T* __restrict__ w) {
  if (sc[S_DONE] != 0.0 || sc[S_CYCLE_DONE] != 0.0) return;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  T s = 0;
#pragma unroll 4
  for (int k = 0; k < of.K; ++k) s = fma(B[k * N + i], z[i + of.o[k]], s);
  w[i] = s;
}

// optionally w -= sum_q h[q] V_q (h from sc + hslot), then partials of (w, V_q), q <= k
template <class T>
__global__ void k_gm_orth(int64_t N, const double* __restrict__ sc, int k, int hslot, T* __restrict__ w,
                          const T* __restrict__ V, size_t vstride, double* __restrict__ part, int64_t pstride,
                          int want_norm) {
  if (sc[S_DONE] != 0.0 || sc[S_CYCLE_DONE] != 0.0) return;
  __shared__ double hs[kMaxRestart + 1];
  for (int q = threadIdx.x; q <= k; q += blockDim.x) hs[q] = hslot >= 0 ? sc[hslot + q] : 0.0;
  __syncthreads();
  double acc[kMaxRestart + 1];
  for (int q = 0; q <= k; ++q) acc[q] = 0.0;
  double nrm = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    T wi = w[i];
    if (hslot >= 0) {
      for (int q = 0; q <= k; ++q) wi -= (T)hs[q] * V[q * vstride + i];
      w[i] = wi;
    }
    if (want_norm) {
      nrm += (double)wi * (double)wi;
    } else {
      for (int q = 0; q <= k; ++q) acc[q] += (double)wi * (double)V[q * vstride + i];
    }
  }
  // block reduction of k+1 (or 1) values
  __shared__ double red[kBlock / 32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nq = want_norm ? 1 : k + 1;
  for (int q = 0; q < nq; ++q) {
    double t = warp_sum(want_norm ? nrm : acc[q]);
    if (lane == 0) red[wp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int u = 0; u < (int)(blockDim.x >> 5); ++u) s += red[u];
      part[q * pstride + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// h[q] = sum of the partials of dot q, stored at sc + hslot + q
__global__ void k_gm_fin_dots(const double* __restrict__ part, int n, int64_t pstride, int nq, double* sc, int hslot) {
  if (sc[S_DONE] != 0.0 || sc[S_CYCLE_DONE] != 0.0) return;
  for (int q = 0; q < nq; ++q) {
    double v = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) v += part[q * pstride + b];
    block_sum_to(v, sc + S_END);
    if (threadIdx.x == 0) sc[hslot + q] = sc[S_END];
    __syncthreads();
  }
}

// Hessenberg column k = h1 + h2, subdiagonal = ||w||; Givens rotations; residual estimate
__global__ void k_gm_column(const double* __restrict__ part, int n, double* sc, int k, int m) {
  if (sc[S_DONE] != 0.0 || sc[S_CYCLE_DONE] != 0.0) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) v += part[b];
  block_sum_to(v, sc + S_END);
  if (threadIdx.x != 0) return;
  const double hk1 = sqrt(sc[S_END]);
  double* H = sc + S_HCOL;   // H[row * kMaxRestart + col]
  for (int q = 0; q <= k; ++q) H[q * kMaxRestart + k] = sc[S_H1 + q] + sc[S_H2 + q];
  H[(k + 1) * kMaxRestart + k] = hk1;
  double* cs = sc + S_CS;
  double* sn = sc + S_SN;
  double* g = sc + S_G;
  for (int q = 0; q < k; ++q) {
    const double a = H[q * kMaxRestart + k], b = H[(q + 1) * kMaxRestart + k];
    H[q * kMaxRestart + k] = cs[q] * a + sn[q] * b;
    H[(q + 1) * kMaxRestart + k] = -sn[q] * a + cs[q] * b;
  }
  const double a = H[k * kMaxRestart + k], b = H[(k + 1) * kMaxRestart + k];
  const double den = hypot(a, b);
  cs[k] = a / den;
  sn[k] = b / den;
  H[k * kMaxRestart + k] = den;
  H[(k + 1) * kMaxRestart + k] = 0.0;
  g[k + 1] = -sn[k] * g[k];
  g[k] = cs[k] * g[k];
  sc[S_ITS] += 1.0;
  sc[S_K_USED] = (double)(k + 1);
  sc[S_NRES] = fabs(g[k + 1]);
  sc[S_INVH] = 1.0 / hk1;
  if (!isfinite(den) || den == 0.0) { sc[S_DONE] = 2.0; return; }
  if (fabs(g[k + 1]) < sc[S_TOL] || sc[S_ITS] >= sc[S_MAXIT] || k + 1 == m || hk1 == 0.0) sc[S_CYCLE_DONE] = 1.0;
}

// back substitution H y = g for the k_used leading columns
__global__ void k_gm_solve(double* sc) {
  if (threadIdx.x != 0 || sc[S_DONE] == 2.0) return;
  const int ku = (int)sc[S_K_USED];
  const double* H = sc + S_HCOL;
  double* y = sc + S_Y;
  for (int q = ku - 1; q >= 0; --q) {
    double s = sc[S_G + q];
    for (int c = q + 1; c < ku; ++c) s -= H[q * kMaxRestart + c] * y[c];
    y[q] = s / H[q * kMaxRestart + q];
  }
}

// x += dinv * sum_q y_q V_q
template <class T>
__global__ void k_gm_update(int64_t N, const double* __restrict__ sc, T* __restrict__ x, const T* __restrict__ V,
                            size_t vstride, const T* __restrict__ dinv) {
  if (sc[S_DONE] == 2.0) return;
  const int ku = (int)sc[S_K_USED];
  if (ku == 0) return;
  __shared__ double ys[kMaxRestart];
  for (int q = threadIdx.x; q < ku; q += blockDim.x) ys[q] = sc[S_Y + q];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int q = 0; q < ku; ++q) s += (T)ys[q] * V[q * vstride + i];
    x[i] = x[i] + dinv[i] * s;
  }
}

__global__ void k_gm_reset(double* sc) {
  if (threadIdx.x == 0) {
    sc[S_DONE] = 0.0;
    sc[S_FIRST] = 1.0;
    sc[S_K_USED] = 0.0;
  }
}

}  // namespace

void krylov_free(afc_problem_s* p) {
  if (!p->kw) return;
  p->kw->vec.free_();
  p->kw->sc.free_();
  p->kw->part.free_();
  if (p->kw->hsc) cudaFreeHost(p->kw->hsc);
  delete p->kw;
  p->kw = nullptr;
}

namespace {

int ensure_work(afc_problem_s* p, int nvec, bool fp32) {
  if (!p->kw) p->kw = new KrylovWork();
  KrylovWork& w = *p->kw;
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  const size_t vstride = (size_t)(p->N + 2 * p->pad + 32) & ~(size_t)31;
  const int64_t bytes = (int64_t)(nvec * vstride * esz);
  if (w.vec.base == nullptr || w.vec.n < bytes) {
    int st = w.vec.alloc(bytes);   // zero-filled
    if (st) return st;
  } else if (w.vstride != vstride || w.fp32 != (int)fp32) {
    // halos are read by the SpMV (times zero coefficients): keep them zero
    AFC_CUDA(cudaMemsetAsync(w.vec.base, 0, (size_t)w.vec.n, p->stream));
  }
  w.vstride = vstride;
  w.fp32 = fp32;
  w.N = p->N;
  w.pad = p->pad;
  if (!w.sc.base) {
    int st = w.sc.alloc(S_END + 8);
    if (st) return st;
    if (cudaMallocHost((void**)&w.hsc, (S_END + 8) * sizeof(double)) != cudaSuccess) {
      set_error("cudaMallocHost failed");
      return AFC_E_OOM;
    }
  }
  const int64_t need_part = (int64_t)(kMaxRestart + 2) * std::max<int64_t>(kRedBlocks, grid_for(p->N));
  if (w.part.n < need_part) {
    int st = w.part.alloc(need_part);
    if (st) return st;
  }
  return AFC_OK;
}

template <class T>
T* vec_at(KrylovWork& w, int q) {
  return reinterpret_cast<T*>(w.vec.base) + q * w.vstride + w.pad;
}

template <class T>
int bicgstab_impl(afc_problem_s* p, const T* B, const T* dinv, const afc_opts* o, const double* rhs, double* xout,
                  int* its, double* res) {
  int st = ensure_work(p, 9, sizeof(T) == 4);
  if (st) return st;
  KrylovWork& w = *p->kw;
  const int64_t N = p->N;
  cudaStream_t s = p->stream;
  T *x = vec_at<T>(w, 0), *r = vec_at<T>(w, 1), *rh = vec_at<T>(w, 2), *pp = vec_at<T>(w, 3), *v = vec_at<T>(w, 4),
    *sv = vec_at<T>(w, 5), *t = vec_at<T>(w, 6), *ph = vec_at<T>(w, 7), *sh = vec_at<T>(w, 8);
  double* sc = w.sc.p;
  double* part = w.part.p;
  const int G = kRedBlocks;
  const int64_t gr = grid_for(N);
  const int64_t pst = std::max<int64_t>(G, gr);
  AFC_LAUNCH(p, "k_bicg_init", k_bicg_init<T><<<G, kBlock, 0, s>>>(N, rhs, x, r, rh, pp, v, part));
  AFC_LAUNCH(p, "k_bicg_init_fin", k_bicg_init_fin<<<1, 1024, 0, s>>>(part, G, sc, o->ksp_atol, o->ksp_rtol, o->ksp_maxit));
  AFC_CUDA(cudaGetLastError());
  int chunk = 2;
  int launched = 0;
  for (;;) {
    AFC_CUDA(cudaMemcpyAsync(w.hsc, sc, (S_MAXIT + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (w.hsc[S_DONE] != 0.0 || launched >= o->ksp_maxit) break;
    for (int c = 0; c < chunk && launched < o->ksp_maxit; ++c, ++launched) {
      AFC_LAUNCH(p, "k_bicg_p", k_bicg_p<T><<<G, kBlock, 0, s>>>(N, sc, r, pp, v, dinv, ph));
      AFC_LAUNCH(p, "k_bicg_spmv", k_bicg_spmv<T, 1><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, ph, v, rh, part, pst));
      AFC_LAUNCH(p, "k_bicg_fin_alpha", k_bicg_fin_alpha<<<1, 1024, 0, s>>>(part, (int)gr, sc));
      AFC_LAUNCH(p, "k_bicg_s", k_bicg_s<T><<<G, kBlock, 0, s>>>(N, sc, r, v, dinv, sv, sh, part));
      AFC_LAUNCH(p, "k_bicg_fin_s", k_bicg_fin_s<<<1, 1024, 0, s>>>(part, G, sc));
      AFC_LAUNCH(p, "k_bicg_early_x", k_bicg_early_x<T><<<G, kBlock, 0, s>>>(N, sc, x, ph));
      AFC_LAUNCH(p, "k_bicg_spmv", k_bicg_spmv<T, 2><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, sh, t, sv, part, pst));
      AFC_LAUNCH(p, "k_bicg_fin_omega", k_bicg_fin_omega<<<1, 1024, 0, s>>>(part, (int)gr, pst, sc));
      AFC_LAUNCH(p, "k_bicg_xr", k_bicg_xr<T><<<G, kBlock, 0, s>>>(N, sc, x, ph, sh, sv, t, r, rh, part, pst));
      AFC_LAUNCH(p, "k_bicg_fin_r", k_bicg_fin_r<<<1, 1024, 0, s>>>(part, G, pst, sc));
    }
    AFC_CUDA(cudaGetLastError());
    chunk = std::min(chunk * 2, 16);
  }
  AFC_LAUNCH(p, "k_to_double", k_to_double<T><<<G, kBlock, 0, s>>>(N, x, xout));
  AFC_CUDA(cudaGetLastError());
  if (its) *its = (int)w.hsc[S_ITS];
  if (res) *res = w.hsc[S_NRES];
  const double done = w.hsc[S_DONE];
  if (done == 2.0) { set_error("BiCGStab breakdown or non-finite value"); return AFC_E_NAN; }
  return done == 1.0 ? AFC_OK : AFC_NOT_CONVERGED;
}

template <class T>
int gmres_impl(afc_problem_s* p, const T* B, const T* dinv, const afc_opts* o, const double* rhs, double* xout,
               int* its, double* res) {
  const int m = o->gmres_restart;
  if (m < 1 || m > kMaxRestart) { set_error("gmres_restart must be in 1..64"); return AFC_E_INVALID; }
  // vectors: x, w, z, V_0..V_m
  int st = ensure_work(p, 3 + m + 1, sizeof(T) == 4);
  if (st) return st;
  KrylovWork& w = *p->kw;
  const int64_t N = p->N;
  cudaStream_t s = p->stream;
  T *x = vec_at<T>(w, 0), *wv = vec_at<T>(w, 1), *z = vec_at<T>(w, 2), *V = vec_at<T>(w, 3);
  const size_t vs = w.vstride;
  double* sc = w.sc.p;
  double* part = w.part.p;
  const int G = kRedBlocks;
  const int64_t gr = grid_for(N);
  const int64_t pst = std::max<int64_t>(G, gr);
  AFC_CUDA(cudaMemsetAsync(x - p->pad, 0, vs * sizeof(T), s));
  AFC_LAUNCH(p, "k_gm_reset", k_gm_reset<<<1, 32, 0, s>>>(sc));
  for (;;) {
    // true residual, stop test, new cycle
    AFC_LAUNCH(p, "k_gm_residual", k_gm_residual<T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, x, rhs, wv, part));
    AFC_LAUNCH(p, "k_gm_start", k_gm_start<<<1, 1024, 0, s>>>(part, (int)gr, sc, o->ksp_atol, o->ksp_rtol, o->ksp_maxit));
    AFC_CUDA(cudaGetLastError());
    AFC_CUDA(cudaMemcpyAsync(w.hsc, sc, S_CS * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (w.hsc[S_DONE] != 0.0) break;
    AFC_LAUNCH(p, "k_gm_normalize", k_gm_normalize<T><<<G, kBlock, 0, s>>>(N, sc, wv, V, dinv, z));
    for (int k = 0; k < m; ++k) {
      AFC_LAUNCH(p, "k_gm_spmv", k_gm_spmv<T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, z, wv));
      AFC_LAUNCH(p, "k_gm_orth", k_gm_orth<T><<<G, kBlock, 0, s>>>(N, sc, k, -1, wv, V, vs, part, G, 0));
      AFC_LAUNCH(p, "k_gm_fin_dots", k_gm_fin_dots<<<1, 1024, 0, s>>>(part, G, G, k + 1, sc, S_H1));
      AFC_LAUNCH(p, "k_gm_orth", k_gm_orth<T><<<G, kBlock, 0, s>>>(N, sc, k, S_H1, wv, V, vs, part, G, 0));
      AFC_LAUNCH(p, "k_gm_fin_dots", k_gm_fin_dots<<<1, 1024, 0, s>>>(part, G, G, k + 1, sc, S_H2));
      AFC_LAUNCH(p, "k_gm_orth", k_gm_orth<T><<<G, kBlock, 0, s>>>(N, sc, k, S_H2, wv, V, vs, part, G, 1));
      AFC_LAUNCH(p, "k_gm_column", k_gm_column<<<1, 1024, 0, s>>>(part, G, sc, k, m));
      AFC_LAUNCH(p, "k_gm_normalize", k_gm_normalize<T><<<G, kBlock, 0, s>>>(N, sc, wv, V + (k + 1) * vs, dinv, z));
    }
    AFC_LAUNCH(p, "k_gm_solve", k_gm_solve<<<1, 32, 0, s>>>(sc));
    AFC_LAUNCH(p, "k_gm_update", k_gm_update<T><<<G, kBlock, 0, s>>>(N, sc, x, V, vs, dinv));
    AFC_CUDA(cudaGetLastError());
  }
  AFC_LAUNCH(p, "k_to_double", k_to_double<T><<<G, kBlock, 0, s>>>(N, x, xout));
  AFC_CUDA(cudaGetLastError());
  if (its) *its = (int)w.hsc[S_ITS];
  if (res) *res = w.hsc[S_NRES];
  const double done = w.hsc[S_DONE];
  if (done == 2.0) { set_error("GMRES breakdown or non-finite value"); return AFC_E_NAN; }
  return done == 1.0 ? AFC_OK : AFC_NOT_CONVERGED;
}

}  // namespace

int krylov_solve(afc_problem_s* p, int system, const afc_opts* o, const double* rhs, double* x, int* its,
                 double* res) {
  const bool mixed = o->precision == AFC_MIXED;
  if (mixed && p->precision != AFC_MIXED) {
    set_error("mixed-precision solve needs afc_assemble(..., AFC_MIXED)");
    return AFC_E_STATE;
  }
  if (system == 1 && p->cn_dt < 0.0) { set_error("CN system not built"); return AFC_E_STATE; }
  const bool gm = o->ksp == AFC_KSP_GMRES;
  if (mixed) {
    const float* B = system == 0 ? p->Bst32.p : p->Bcn32.p;
    const float* di = system == 0 ? p->dinv_st32.p : p->dinv_cn32.p;
    return gm ? gmres_impl<float>(p, B, di, o, rhs, x, its, res) : bicgstab_impl<float>(p, B, di, o, rhs, x, its, res);
  }
  const double* B = system == 0 ? p->Bst.p : p->Bcn.p;
  const double* di = system == 0 ? p->dinv_st.p : p->dinv_cn.p;
  return gm ? gmres_impl<double>(p, B, di, o, rhs, x, its, res) : bicgstab_impl<double>(p, B, di, o, rhs, x, its, res);
}

}  // namespace afc
