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
#include "graph_util.h"
#include "kernels_common.cuh"
#include "grid_sync.cuh"

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
  // zero-fill and wait for it here: a plain cudaMemset runs on the legacy default
  // stream, which is not ordered with the non-blocking streams a problem may use
  e = cudaMemsetAsync(base, 0, bytes, cudaStreamPerThread);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
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
template struct DBuf<float4>;
template struct DBuf<float2>;

namespace {

__global__ void k_finalize_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  block_sum_to(strided_sum_1024(part, n, threadIdx.x), out);   // one block of 1024: out[0]
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
  __shared__ double smn[kBlock], smx[kBlock];
  double mn = INFINITY, mx = -INFINITY;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    mn = fmin(mn, part[2 * q]);
    mx = fmax(mx, part[2 * q + 1]);
  }
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
    out[0] = smn[0];
    out[1] = smx[0];
  }
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
  AFC_LAUNCH(p, "k_minmax_fin", k_minmax_fin<<<1, kBlock, 0, p->stream>>>(p->part.p, kRedBlocks, p->scal.p + 60));
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
constexpr int kMaxRestart = 32;   // GMRES(m), m <= 32: the Gram-Schmidt kernel keeps m dots in registers

// device scalar slots
enum : int {
  S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_TOL, S_NRES, S_N0, S_ITS, S_DONE, S_MAXIT,
  S_BETA, S_K_USED, S_INVH, S_CYCLE_DONE, S_FIRST, S_ATOL, S_RTOL, S_NO_REORTH,
  S_CS = 20, S_SN = S_CS + kMaxRestart, S_G = S_SN + kMaxRestart, S_Y = S_G + kMaxRestart + 1,
  S_H1 = S_Y + kMaxRestart, S_H2 = S_H1 + kMaxRestart + 1, S_HCOL = S_H2 + kMaxRestart + 1,
  S_END = S_HCOL + (kMaxRestart + 1) * kMaxRestart
};
// S_DONE: 0 running, 1 converged, 2 breakdown / non-finite, 3 converged at s (x update pending), 4 maxit
static_assert(S_ITS == kKrylovItsSlot && S_DONE == kKrylovDoneSlot, "slot numbers shared with graph.cu");
constexpr int S_CYCLES = 18;   // GMRES restart cycles begun (true-residual evaluations)
constexpr int S_BERR = 19;     // persistent BiCGStab: a grid barrier gave up waiting
static_assert(S_CYCLES > S_NO_REORTH && S_BERR > S_CYCLES && S_BERR < S_CS, "slot range");
static_assert(S_BERR == kKrylovBarrierErrSlot, "slot number shared with graph.cu");

// A solver flag (a double slot holding 0 or a positive code) tested on its bit pattern:
// a compare of doubles issues on GB300's FP64 pipe, where every warp instruction
// costs 16 cycles, and the kernels below test their flags in every thread.
__device__ __forceinline__ bool flag_set(const double* sc, int slot) {
  return (__double_as_longlong(sc[slot]) << 1) != 0;
}
// float -> double without the FP64 pipe (exact; the FP64 instance passes through)
__device__ __forceinline__ double to_dbl(float x) { return widen_exact(x); }
__device__ __forceinline__ double to_dbl(double x) { return x; }

struct KrylovWork {
  int64_t N = 0;
  int pad = 0, m = 0, fp32 = -1;
  DBuf<char> vec;       // all vectors (with halos)
  DBuf<double> sc, part;
  DBuf<unsigned int> counter;
  DBuf<unsigned int> barrier;   // GridBar of the persistent BiCGStab launch
  int coop = -1;                // device supports cooperative launches (-1: not asked yet)
  int nsm = 0;
  double* hsc = nullptr;
  size_t vstride = 0;   // elements per vector incl. halo
};

template struct DBuf<char>;
template struct DBuf<unsigned int>;
template struct DBuf<uint16_t>;

namespace {

// ---- "last block" reductions ------------------------------------------------
// A producer kernel writes one partial per block and counts finished blocks; the
// block that finishes last sums all partials in block order (deterministic) and
// updates the solver scalars.  Every block reads the scalars it needs before it
// counts itself, and only the last block writes them, so no block of a kernel
// sees a scalar that the same kernel changes.
// Sum v over the block in a fixed order; every thread receives the total.
__device__ __forceinline__ double block_allsum(double v) {
  __shared__ double total;
  if (blockDim.x > kBlock) {
    __shared__ double sw[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sw[w] = v;
    __syncthreads();
    if (w == 0) {
      const int nw = (blockDim.x + 31) >> 5;
      double t = lane < nw ? sw[lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) total = t;
    }
  } else {
    __shared__ double sh[kBlock];
    sh[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      const double t = warp0_column_sum(sh);
      if (threadIdx.x == 0) total = t;
    }
  }
  __syncthreads();
  const double r = total;
  __syncthreads();
  return r;
}

template <int NV>
__device__ __forceinline__ bool last_block_sums(double (&v)[NV], double* part, int64_t pstride,
                                                unsigned int* counter, double (&tot)[NV]) {
  block_sums_to<NV>(v, part, pstride);
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(counter, 1u);
    am_last = done == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const int n = gridDim.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    // thread t adds partials t, t + blockDim.x, ... in turn, the loads eight at a time
    double s = 0.0;
    for (int b0 = threadIdx.x; b0 < n; b0 += 8 * blockDim.x) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = b0 + u * blockDim.x;
        x[u] = b < n ? __ldcg(part + q * pstride + b) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) s += x[u];
    }
    tot[q] = block_allsum(s);
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ bool stop_test(double nr, const double* sc) { return nr < sc[S_TOL]; }

// ---- BiCGStab (van der Vorst 1992), Jacobi preconditioner on the directions ----
template <class T>
__global__ void k_bicg_init(int64_t N, const double* __restrict__ rhs, T* x, T* r, T* rh, T* p, T* v,
                            double* __restrict__ part, unsigned int* counter, double* sc) {
  T a0 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = (T)rhs[i];
    x[i] = 0;
    r[i] = ri;
    rh[i] = ri;
    p[i] = 0;
    v[i] = 0;
    a0 = fma(ri, ri, a0);
  }
  double acc[1] = {(double)a0};
  double tot[1];
  if (!last_block_sums<1>(acc, part, gridDim.x, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double n0 = sqrt(tot[0]);
    sc[S_N0] = n0;
    sc[S_NRES] = n0;
    sc[S_RHO] = tot[0];
    sc[S_RHO_OLD] = 1.0;
    sc[S_ALPHA] = 1.0;
    sc[S_OMEGA] = 1.0;
    sc[S_BETA] = (tot[0] / 1.0) * (1.0 / 1.0);
    sc[S_TOL] = fmax(sc[S_ATOL], sc[S_RTOL] * n0);
    sc[S_ITS] = 0.0;
    sc[S_DONE] = !isfinite(n0) ? 2.0 : (n0 < sc[S_TOL] ? 1.0 : (sc[S_MAXIT] <= 0.0 ? 4.0 : 0.0));
  }
}

// p = r + beta (p - omega v), phat = D^{-1} p
template <class T>
__global__ void k_bicg_p(int64_t N, const double* __restrict__ sc, const T* __restrict__ r, T* p,
                         const T* __restrict__ v, const T* __restrict__ dinv, T* __restrict__ ph) {
  if (flag_set(sc, S_DONE)) return;
  const T beta = (T)sc[S_BETA];       // (rho / rho_old)(alpha / omega), formed once by the previous kernel
  const T om = (T)sc[S_OMEGA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T pi = r[i] + beta * (p[i] - om * v[i]);
    p[i] = pi;
    ph[i] = dinv[i] * pi;
  }
}

// v = B phat and (rhat, v); the last block sets alpha = rho / (rhat, v)
template <int KT, class T>
__global__ void k_bicg_spmv1(int64_t N, Offsets of, double* sc, const T* __restrict__ B, const T* __restrict__ x,
                             T* __restrict__ y, const T* __restrict__ a, double* __restrict__ part,
                             unsigned int* counter) {
  if (flag_set(sc, S_DONE)) return;
  const int K = KT > 0 ? KT : of.K;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (i < N) {
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) s = fma(B[k * N + i], x[i + of.o[k]], s);
    y[i] = s;
    acc[0] = (double)(a[i] * s);
  }
  double tot[1];
  if (!last_block_sums<1>(acc, part, gridDim.x, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double al = sc[S_RHO] / tot[0];
    if (!isfinite(al) || tot[0] == 0.0) sc[S_DONE] = 2.0;
    else sc[S_ALPHA] = al;
  }
}

// s = r - alpha v, shat = D^{-1} s, ||s||; the last block tests convergence at s
template <class T>
__global__ void k_bicg_s(int64_t N, double* sc, const T* __restrict__ r, const T* __restrict__ v,
                         const T* __restrict__ dinv, T* __restrict__ s, T* __restrict__ sh, double* __restrict__ part,
                         unsigned int* counter) {
  if (flag_set(sc, S_DONE)) return;
  const T al = (T)sc[S_ALPHA];
  T a0 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T si = r[i] - al * v[i];
    s[i] = si;
    sh[i] = dinv[i] * si;
    a0 = fma(si, si, a0);
  }
  double acc[1] = {(double)a0};
  double tot[1];
  if (!last_block_sums<1>(acc, part, gridDim.x, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double ns = sqrt(tot[0]);
    if (!isfinite(ns)) { sc[S_DONE] = 2.0; return; }
    if (stop_test(ns, sc)) {
      sc[S_NRES] = ns;
      sc[S_ITS] += 1.0;
      sc[S_DONE] = 3.0;     // converged at s: x += alpha phat in the next kernel
    }
  }
}

// t = B shat, (t, s), (t, t); the last block sets omega.  When the solve converged at
// s, this kernel instead finishes x += alpha phat.
template <int KT, class T>
__global__ void k_bicg_spmv2(int64_t N, Offsets of, double* sc, const T* __restrict__ B, const T* __restrict__ sh,
                             T* __restrict__ t, const T* __restrict__ s, T* __restrict__ x,
                             const T* __restrict__ ph, double* __restrict__ part, unsigned int* counter) {
  const double done = sc[S_DONE];
  if (done != 0.0 && done != 3.0) return;
  const int K = KT > 0 ? KT : of.K;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (done == 3.0) {
    if (i < N) x[i] = x[i] + (T)sc[S_ALPHA] * ph[i];
  } else if (i < N) {
    T v = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) v = fma(B[k * N + i], sh[i + of.o[k]], v);
    t[i] = v;
    acc[0] = (double)(v * s[i]);
    acc[1] = (double)(v * v);
  }
  double tot[2];
  if (!last_block_sums<2>(acc, part, gridDim.x, counter, tot)) return;
  if (threadIdx.x == 0) {
    if (done == 3.0) { sc[S_DONE] = 1.0; return; }
    const double om = tot[0] / tot[1];
    if (!isfinite(om) || tot[1] == 0.0) sc[S_DONE] = 2.0;
    else sc[S_OMEGA] = om;
  }
}

// x += alpha phat + omega shat, r = s - omega t, ||r||, (rhat, r); the last block tests
// convergence and rotates rho
template <class T>
__global__ void k_bicg_xr(int64_t N, double* sc, T* __restrict__ x, const T* __restrict__ ph,
                          const T* __restrict__ sh, const T* __restrict__ s, const T* __restrict__ t,
                          T* __restrict__ r, const T* __restrict__ rh, double* __restrict__ part,
                          unsigned int* counter, GraphCond cond) {
  if (flag_set(sc, S_DONE)) {
    if (cond.use && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond.h, 0u);
    return;
  }
  const T al = (T)sc[S_ALPHA], om = (T)sc[S_OMEGA];
  T a0 = 0, a1 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = x[i] + al * ph[i] + om * sh[i];
    const T ri = s[i] - om * t[i];
    r[i] = ri;
    a0 = fma(ri, ri, a0);
    a1 = fma(rh[i], ri, a1);
  }
  double acc[2] = {(double)a0, (double)a1};
  double tot[2];
  if (!last_block_sums<2>(acc, part, gridDim.x, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double nr = sqrt(tot[0]);
    sc[S_NRES] = nr;
    sc[S_RHO_OLD] = sc[S_RHO];
    sc[S_RHO] = tot[1];
    sc[S_BETA] = (sc[S_RHO] / sc[S_RHO_OLD]) * (sc[S_ALPHA] / sc[S_OMEGA]);
    sc[S_ITS] += 1.0;
    if (!isfinite(nr)) sc[S_DONE] = 2.0;
    else if (stop_test(nr, sc)) sc[S_DONE] = 1.0;
    else if (sc[S_ITS] >= sc[S_MAXIT]) sc[S_DONE] = 4.0;
    if (cond.use) cudaGraphSetConditional(cond.h, sc[S_DONE] == 0.0 ? 1u : 0u);
  }
}

// ---- BiCGStab as one persistent cooperative launch ----------------------------
// The five phases of an iteration (p update, v = B phat, s update, t = B shat, x / r
// update) run in one launch, separated by grid barriers; nothing returns to the
// host or the graph between iterations.  A grid-wide sum: every block stores its
// partials, waits at the barrier, then sums all blocks' partials in block order.
// The order is the same in every block, so every block obtains the same totals
// bit for bit and takes the same branches.  Partials alternate between two buffers
// (a block can run at most one reduction ahead of another).
// Shape of the persistent launch: one block of 512 threads per SM.  Every barrier
// and grid-wide sum costs more with more blocks.  On GB300 (Q1 65^3, 27 offsets,
// per BiCGStab iteration) 512 x 1 per SM took 62.4 us, 256 x 2 66.0 us, 1024 x 1
// 65.9 us, 256 x 1 72.1 us, 128 x 4 77.0 us; earlier, 256 x 3 and 256 x 4 were
// 8 % and 14 % slower than 256 x 2.  Block b owns the contiguous rows
// [N b / G, N (b + 1) / G), which balances the blocks to one row.
constexpr int kFusedBlock = 512;
constexpr int kFusedBlocksPerSM = 1;

// Grid-wide sums of NV <= 2 values per thread.  Warp q forms the block's sum of
// value q (a column sum in the order of warp0_column_sum) and stores it at
// part[q * G + block]; after the barrier warp q of every block reads the G partials
// of value q, lane l summing blocks l, l + 32, ... in turn before a butterfly over
// the lanes.  Every block runs the same operations on the same partials, so all
// obtain the same totals bit for bit.  The two sums of NV = 2 run in two warps at
// once, and the only block-wide meeting after the barrier is the one that hands
// the totals on (the totals alternate between two shared slots, like the partials,
// so a later call cannot overwrite a slot that a thread still reads).
// grid_sums_begin stores the partials and arrives; grid_sums_end waits and sums, so
// that work no other block needs can run in between.
template <int NV>
__device__ __forceinline__ unsigned int grid_sums_begin(double (&v)[NV], double* part, int buf, GridBar* bar) {
  static_assert(NV >= 1 && NV <= 2, "two partial buffers of 2 G values");
  __shared__ double col[NV][kFusedBlock];
  const int G = gridDim.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* pb = part + (size_t)buf * 2 * G;
#pragma unroll
  for (int q = 0; q < NV; ++q) col[q][threadIdx.x] = v[q];
  __syncthreads();
  if (w < NV) {
    double t = col[w][lane];
    for (int j = lane + 32; j < kFusedBlock; j += 32) t += col[w][j];
    t = warp_sum(t);
    if (lane == 0) pb[w * G + blockIdx.x] = t;
  }
  return grid_arrive(bar);   // begins with __syncthreads: col is free again after it
}

template <int NV>
__device__ __forceinline__ void grid_sums_end(double* part, int& buf, GridBar* bar, unsigned int old,
                                              double (&tot)[NV], unsigned long long wait_ns) {
  __shared__ double shtot[2][NV];
  const int G = gridDim.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* pb = part + (size_t)buf * 2 * G;
  grid_wait(bar, old, wait_ns);
  if (w < NV) {
    // lane l adds partials l, l + 32, ... in turn, the loads eight at a time (one round
    // trip for up to 256 blocks)
    double t = 0.0;
    for (int b0 = lane; b0 < G; b0 += 256) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = b0 + 32 * u < G ? __ldcg(pb + w * G + b0 + 32 * u) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) t += x[u];
    }
    t = warp_sum(t);
    if (lane == 0) shtot[buf][w] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = shtot[buf][q];
  buf ^= 1;
}

template <int NV>
__device__ __forceinline__ void grid_sums(double (&v)[NV], double* part, int& buf, GridBar* bar,
                                          double (&tot)[NV], unsigned long long wait_ns) {
  const unsigned int old = grid_sums_begin<NV>(v, part, buf, bar);
  grid_sums_end<NV>(part, buf, bar, old, tot, wait_ns);
}

template <int KT, class T>
__global__ void __launch_bounds__(kFusedBlock, 1024 / kFusedBlock) k_bicg_fused(int64_t N, Offsets of, double* sc, const T* __restrict__ B,
                                                   const T* __restrict__ dinv, const double* __restrict__ rhs,
                                                   double* xout, T* x, T* r, T* rh, T* pv, T* v, T* s, T* t, T* ph,
                                                   T* sh, double* part, GridBar* bar, double atol, double rtol,
                                                   int maxit, KrylovEpilogue ep, unsigned long long wait_ns) {
  const int K = KT > 0 ? KT : of.K;
  const int64_t G = gridDim.x;
  const int64_t stride = kFusedBlock;
  const int64_t i0 = N * blockIdx.x / G + threadIdx.x, iend = N * (blockIdx.x + 1) / G;
  volatile int* berr = &bar->err;
  int buf = 0;
  double a1[1], t1[1], a2[2], t2[2];
  // r = rhs, rhat = r, x = v = 0, rho = (r, r); and the first iteration's p update
  // (beta = 0 and p = v = 0 before it: p = r + 0, phat = D^{-1} p), so that
  // iteration needs no pass and no barrier of its own before its product
  T a0 = 0;
  for (int64_t i = i0; i < iend; i += stride) {
    const T ri = (T)rhs[i];
    x[i] = 0;
    r[i] = ri;
    rh[i] = ri;
    v[i] = 0;
    const T pi = ri + (T)0;   // as r + 0 * (0 - 1 * 0) rounds: -0 becomes +0
    pv[i] = pi;
    ph[i] = dinv[i] * pi;
    a0 = fma(ri, ri, a0);
  }
  a1[0] = (double)a0;
  grid_sums<1>(a1, part, buf, bar, t1, wait_ns);
  double rho = t1[0];
  const double n0 = sqrt(rho);
  const double tol = fmax(atol, rtol * n0);
  double alpha = 1.0, omega = 1.0, beta = 0.0, nres = n0;
  int its = 0;
  int done = !isfinite(n0) ? 2 : (n0 < tol ? 1 : (maxit <= 0 ? 4 : 0));
  bool first = true;
  while (done == 0) {
    // p = r + beta (p - omega v), phat = D^{-1} p (the first iteration's came with r)
    if (!first) {
      const T tb = (T)beta, to = (T)omega;
      for (int64_t i = i0; i < iend; i += stride) {
        const T pi = r[i] + tb * (pv[i] - to * v[i]);
        pv[i] = pi;
        ph[i] = dinv[i] * pi;
      }
      grid_barrier(bar, wait_ns);
    }
    first = false;
    // v = B phat, alpha = rho / (rhat, v)
    a0 = 0;
    for (int64_t i = i0; i < iend; i += stride) {
      T y = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) y = fma(B[k * N + i], ph[i + of.o[k]], y);
      v[i] = y;
      a0 = fma(rh[i], y, a0);
    }
    a1[0] = (double)a0;
    grid_sums<1>(a1, part, buf, bar, t1, wait_ns);
    alpha = rho / t1[0];
    if (!isfinite(alpha) || t1[0] == 0.0 || *berr) { done = 2; break; }
    // s = r - alpha v, shat = D^{-1} s, ||s||
    const T ta = (T)alpha;
    a0 = 0;
    for (int64_t i = i0; i < iend; i += stride) {
      const T si = r[i] - ta * v[i];
      s[i] = si;
      sh[i] = dinv[i] * si;
      a0 = fma(si, si, a0);
    }
    a1[0] = (double)a0;
    grid_sums<1>(a1, part, buf, bar, t1, wait_ns);
    const double ns = sqrt(t1[0]);
    if (!isfinite(ns) || *berr) { done = 2; break; }
    if (ns < tol) {   // converged at s: x += alpha phat
      for (int64_t i = i0; i < iend; i += stride) x[i] = x[i] + ta * ph[i];
      nres = ns;
      ++its;
      done = 1;
      break;
    }
    // t = B shat, omega = (t, s) / (t, t)
    T b0 = 0, b1 = 0;
    for (int64_t i = i0; i < iend; i += stride) {
      T y = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) y = fma(B[k * N + i], sh[i + of.o[k]], y);
      t[i] = y;
      b0 = fma(y, s[i], b0);
      b1 = fma(y, y, b1);
    }
    a2[0] = (double)b0;
    a2[1] = (double)b1;
    grid_sums<2>(a2, part, buf, bar, t2, wait_ns);
    omega = t2[0] / t2[1];
    if (!isfinite(omega) || t2[1] == 0.0 || *berr) { done = 2; break; }
    // r = s - omega t, ||r||, (rhat, r); x += alpha phat + omega shat while the sums
    // complete (no other block reads x)
    const T tom = (T)omega;
    b0 = 0;
    b1 = 0;
    for (int64_t i = i0; i < iend; i += stride) {
      const T ri = s[i] - tom * t[i];
      r[i] = ri;
      b0 = fma(ri, ri, b0);
      b1 = fma(rh[i], ri, b1);
    }
    a2[0] = (double)b0;
    a2[1] = (double)b1;
    const unsigned int arrived = grid_sums_begin<2>(a2, part, buf, bar);
    for (int64_t i = i0; i < iend; i += stride) x[i] = x[i] + ta * ph[i] + tom * sh[i];
    grid_sums_end<2>(part, buf, bar, arrived, t2, wait_ns);
    nres = sqrt(t2[0]);
    const double rho_old = rho;
    rho = t2[1];
    beta = (rho / rho_old) * (alpha / omega);
    ++its;
    if (!isfinite(nres) || *berr) done = 2;
    else if (nres < tol) done = 1;
    else if (its >= maxit) done = 4;
  }
  if (ep.u != nullptr && done != 2) {
    const double om = ep.omega;
    for (int64_t i = i0; i < iend; i += stride) {
      const double xi = (double)x[i];
      xout[i] = xi;
      const double ui = ep.u[i] + om * xi;
      ep.u[i] = ui;
      const double uoi = ep.uo[i];
      ep.a[i] = ui - uoi;
      ep.s[i] = ui + uoi;
    }
  } else {
    for (int64_t i = i0; i < iend; i += stride) xout[i] = (double)x[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {   // the solver scalars, as the kernel-per-phase form leaves them
    sc[S_ATOL] = atol;
    sc[S_RTOL] = rtol;
    sc[S_MAXIT] = (double)maxit;
    sc[S_FIRST] = 1.0;
    sc[S_K_USED] = 0.0;
    sc[S_CYCLE_DONE] = 0.0;
    sc[S_TOL] = tol;
    sc[S_N0] = n0;
    sc[S_NRES] = nres;
    sc[S_ITS] = (double)its;
    sc[S_ALPHA] = alpha;
    sc[S_OMEGA] = omega;
    sc[S_RHO] = rho;
    sc[S_DONE] = *berr ? 2.0 : (double)done;
    sc[S_BERR] = *berr ? 1.0 : 0.0;
    if (ep.fp_sc) {   // the fixed-point loop's count of this correction (the after-solve node's work)
      double* f = ep.fp_sc;
      f[F_CORR] += 1.0;
      f[F_INNER] += (double)its;
      f[F_KBODY] += (double)its;
      if (*berr || done == 2) f[F_STATUS] = 2.0;
      if (*berr) f[F_TIMEOUT] = 1.0;
    }
  }
}

// arm a solver loop: condition = (solver still running)
__global__ void k_cond_running(const double* __restrict__ sc, GraphCond cond) {
  if (threadIdx.x == 0 && cond.use) cudaGraphSetConditional(cond.h, sc[S_DONE] == 0.0 ? 1u : 0u);
}

template <class T>
__global__ void k_to_double(int64_t N, const T* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// ---- GMRES(m), right Jacobi preconditioning, classical Gram-Schmidt with one
// re-orthogonalisation pass ----

// w = rhs - B x (x = 0 on the first cycle) and ||w||; the last block runs the stop test
// on this true residual and starts a cycle: g = (beta, 0, ...), invh = 1 / beta
template <int KT, class T>
__global__ void k_gm_residual(int64_t N, Offsets of, double* sc, const T* __restrict__ B, const T* __restrict__ x,
                              const double* __restrict__ rhs, T* __restrict__ w, double* __restrict__ part,
                              unsigned int* counter) {
  if (flag_set(sc, S_DONE)) return;
  const int K = KT > 0 ? KT : of.K;
  const bool first = flag_set(sc, S_FIRST);
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (i < N) {
    T s = 0;
    if (!first) {
#pragma unroll
      for (int k = 0; k < K; ++k) s = fma(B[k * N + i], x[i + of.o[k]], s);
    }
    const T wi = (T)rhs[i] - s;
    w[i] = wi;
    acc[0] = (double)(wi * wi);
  }
  double tot[1];
  if (!last_block_sums<1>(acc, part, gridDim.x, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double beta = sqrt(tot[0]);
    if (first) {
      sc[S_N0] = beta;
      sc[S_TOL] = fmax(sc[S_ATOL], sc[S_RTOL] * beta);
      sc[S_ITS] = 0.0;
      sc[S_FIRST] = 0.0;
      sc[S_CYCLES] = 0.0;
    }
    sc[S_CYCLES] += 1.0;
    sc[S_NRES] = beta;
    sc[S_BETA] = beta;
    sc[S_K_USED] = 0.0;
    sc[S_CYCLE_DONE] = 0.0;
    if (!isfinite(beta)) sc[S_DONE] = 2.0;
    else if (stop_test(beta, sc)) sc[S_DONE] = 1.0;
    else if (sc[S_ITS] >= sc[S_MAXIT]) sc[S_DONE] = 4.0;
    for (int q = 0; q <= kMaxRestart; ++q) sc[S_G + q] = 0.0;
    sc[S_G] = beta;
    sc[S_INVH] = 1.0 / beta;
  }
}

// v_k = w * invh; z = D^{-1} v_k
template <class T>
__global__ void k_gm_normalize(int64_t N, const double* __restrict__ sc, const T* __restrict__ w, T* __restrict__ vk,
                               const T* __restrict__ dinv, T* __restrict__ z) {
  if (flag_set(sc, S_DONE) || flag_set(sc, S_CYCLE_DONE)) return;
  __shared__ T ihs;   // one conversion per block instead of one per thread
  if (threadIdx.x == 0) ihs = (T)sc[S_INVH];
  __syncthreads();
  const T ih = ihs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const T vi = w[i] * ih;
    vk[i] = vi;
    z[i] = dinv[i] * vi;
  }
}

template <int KT, class T>
__global__ void k_gm_spmv(int64_t N, Offsets of, const double* __restrict__ sc, const T* __restrict__ B,
                          const T* __restrict__ z, T* __restrict__ w) {
  if (flag_set(sc, S_DONE) || flag_set(sc, S_CYCLE_DONE)) return;
  const int K = KT > 0 ? KT : of.K;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  T s = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) s = fma(B[k * N + i], z[i + of.o[k]], s);
  w[i] = s;
}

// Gram-Schmidt pass: optionally w -= sum_q h[q] V_q (h at sc + hslot), then the dots
// (w, V_q), q <= k (pass 1, 2) or ||w|| (pass 3).  The last block stores the dots at
// sc + outslot (passes 1, 2) or completes Hessenberg column k (pass 3): H[0..k][k] =
// h1 + h2, H[k+1][k] = ||w||, earlier Givens rotations, a new rotation, the residual
// estimate |g[k+1]|, the end-of-cycle test and invh = 1 / ||w||.
// A thread owns elements and holds all k + 1 running dots in registers (QMAX is the
// compile-time bound on k + 1, the loops over q are unrolled and predicated), so each
// element's k + 1 basis values are independent loads in flight together.
//
// Three launches per Arnoldi step: (1) h1 = V^T w and ||w||^2; (2) w -= V h1 and
// h2 = V^T w (the re-orthogonalisation); (3) w -= V h2, ||w||, and the Hessenberg
// column.  The last block of (1) applies the DGKS test: if ||w - V h1|| >= ||w|| / sqrt(2)
// (with ||w - V h1||^2 = ||w||^2 - ||h1||^2 for orthonormal V) little of w lay in the
// basis, the second projection would change nothing worth keeping, and (2) takes the
// role of (3) directly (h2 = 0) while (3) does nothing.
template <class T, int QMAX>
__global__ void __launch_bounds__(256) k_gm_orth(int64_t N, double* sc, int k, int m, int hslot, int outslot,
                                                 T* __restrict__ w, const T* __restrict__ V, size_t vstride,
                                                 double* __restrict__ part, int64_t pstride, unsigned int* counter) {
  if (flag_set(sc, S_DONE) || flag_set(sc, S_CYCLE_DONE)) return;
  const bool first = hslot < 0;                               // launch (1)
  const bool no_reorth = !first && flag_set(sc, S_NO_REORTH);
  if (no_reorth && outslot < 0) return;                       // launch (3) has nothing to do
  const bool want_norm = outslot < 0 || no_reorth;
  if (want_norm && no_reorth) outslot = -1;
  __shared__ T hs[QMAX];
  for (int q = threadIdx.x; q < QMAX; q += blockDim.x) hs[q] = (hslot >= 0 && q <= k) ? (T)sc[hslot + q] : (T)0;
  __syncthreads();
  // running sums in the vector type (a thread sees a handful of elements); widened to
  // double for the sums across warps and blocks
  T acc[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) acc[q] = (T)0;
  T nrm = (T)0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    T v[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) v[q] = q <= k ? V[q * vstride + i] : (T)0;
    T wi = w[i];
    if (hslot >= 0) {
#pragma unroll
      for (int q = 0; q < QMAX; ++q) wi -= hs[q] * v[q];
      w[i] = wi;
    }
    if (want_norm) {
      nrm = fma(wi, wi, nrm);
    } else {
#pragma unroll
      for (int q = 0; q < QMAX; ++q)
        if (q <= k) acc[q] = fma(wi, v[q], acc[q]);
      if (first) nrm = fma(wi, wi, nrm);
    }
  }
  // sums: the k + 1 dots (and ||w||^2 as sum k + 1 in launch (1)), or the norm alone
  const int nq = want_norm ? 1 : (first ? k + 2 : k + 1);
  if (want_norm) {
    const double t = block_allsum(to_dbl(nrm));
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  } else {
    // a block's warp sums meet in the vector type (for the single-precision instance: no
    // FP64 instruction per warp and sum) and are widened once per block
    __shared__ T red[kBlock / 32][QMAX + 1];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      if (q > k) break;
      const T t = warp_sum(acc[q]);
      if (lane == 0) red[wp][q] = t;
    }
    if (first) {
      const T t = warp_sum(nrm);
      if (lane == 0) red[wp][k + 1] = t;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      T s = 0;
      for (int u = 0; u < (int)(blockDim.x >> 5); ++u) s += red[u][q];
      part[q * pstride + blockIdx.x] = to_dbl(s);
    }
  }
  __threadfence();   // every thread that wrote a partial makes it visible before the count
  __syncthreads();
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // totals of the nq sums: warp q' takes q = q', q' + 8, ... (block order, fixed)
  __shared__ double tot[QMAX + 1];
  {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // lane l adds partials l, l + 32, ... in turn, the loads eight at a time
    const int n = gridDim.x;
    for (int q = wp; q < nq; q += nwarp) {
      double s = 0.0;
      for (int b0 = lane; b0 < n; b0 += 256) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = b0 + 32 * u < n ? __ldcg(part + q * pstride + b0 + 32 * u) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += x[u];
      }
      s = warp_sum(s);
      if (lane == 0) tot[q] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  *counter = 0u;
  if (!want_norm) {
    for (int q = 0; q <= k; ++q) sc[outslot + q] = tot[q];
    if (first) {   // DGKS test: re-orthogonalise only if ||w - V h1||^2 < ||w||^2 / 2
      double proj = 0.0;
      for (int q = 0; q <= k; ++q) proj += tot[q] * tot[q];
      const double ww = tot[k + 1], rest = ww - proj;
      const bool skip = rest >= 0.5 * ww && ww > 0.0;
      sc[S_NO_REORTH] = skip ? 1.0 : 0.0;
      if (skip)
        for (int q = 0; q <= k; ++q) sc[S_H2 + q] = 0.0;
    }
    return;
  }
  const double hk1 = sqrt(tot[0]);
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
  if (stop_test(fabs(g[k + 1]), sc) || sc[S_ITS] >= sc[S_MAXIT] || k + 1 == m || hk1 == 0.0) sc[S_CYCLE_DONE] = 1.0;
}

// Launch a Gram-Schmidt pass with the smallest register footprint that holds k + 1 dots,
// on as many blocks as are resident at once (one wave), at most G.
template <class T, int Q>
int orth_grid(int G) {
  static const int nb = [] {
    int b = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gm_orth<T, Q>, kBlock, 0) != cudaSuccess) {
      cudaGetLastError();
      b = 0;
    }
    return b * nsm;
  }();
  return nb > 0 ? std::min(G, nb) : G;
}

template <class T>
void orth_launch(afc_problem_s* p, int G, int64_t N, double* sc, int k, int m, int hslot, int outslot, T* w,
                 const T* V, size_t vs, double* part, int64_t pst, unsigned int* cnt) {
  cudaStream_t s = p->stream;
#define AFC_ORTH(Q) AFC_LAUNCH(p, "k_gm_orth", k_gm_orth<T, Q><<<orth_grid<T, Q>(G), kBlock, 0, s>>>(N, sc, k, m, hslot, outslot, w, V, vs, part, pst, cnt))
  if (k + 1 <= 4) AFC_ORTH(4);
  else if (k + 1 <= 8) AFC_ORTH(8);
  else if (k + 1 <= 12) AFC_ORTH(12);
  else if (k + 1 <= 16) AFC_ORTH(16);
  else if (k + 1 <= 20) AFC_ORTH(20);
  else if (k + 1 <= 24) AFC_ORTH(24);
  else AFC_ORTH(32);
#undef AFC_ORTH
}

// back substitution H y = g for the k_used leading columns, then x += D^{-1} sum_q y_q V_q
// (every block solves the small triangular system itself)
template <class T>
__global__ void k_gm_update(int64_t N, const double* __restrict__ sc, T* __restrict__ x, const T* __restrict__ V,
                            size_t vstride, const T* __restrict__ dinv, GraphCond cond) {
  // another restart cycle only while the solve is running (set before any early return)
  if (cond.use && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond.h, sc[S_DONE] == 0.0 ? 1u : 0u);
  if (sc[S_DONE] == 2.0) return;
  const int ku = (int)sc[S_K_USED];
  if (ku == 0) return;
  __shared__ double ys[kMaxRestart];
  __shared__ T yt[kMaxRestart];
  // the leading ku x ku block of H and g, staged by the whole block (one round of loads
  // instead of one dependent load per entry for the thread that solves)
  __shared__ double hs[kMaxRestart * kMaxRestart];
  __shared__ double gs[kMaxRestart];
  for (int e = threadIdx.x; e < ku * ku; e += blockDim.x) {
    const int q = e / ku, c = e - q * ku;
    hs[q * kMaxRestart + c] = sc[S_HCOL + q * kMaxRestart + c];
  }
  for (int q = threadIdx.x; q < ku; q += blockDim.x) gs[q] = sc[S_G + q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = ku - 1; q >= 0; --q) {
      double s = gs[q];
      for (int c = q + 1; c < ku; ++c) s -= hs[q * kMaxRestart + c] * ys[c];
      ys[q] = s / hs[q * kMaxRestart + q];
    }
    for (int q = 0; q < ku; ++q) yt[q] = (T)ys[q];
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int q = 0; q < ku; ++q) s = fma(yt[q], V[q * vstride + i], s);
    x[i] = x[i] + dinv[i] * s;
  }
}

__global__ void k_solver_reset(double* sc, double atol, double rtol, int maxit) {
  if (threadIdx.x == 0) {
    sc[S_DONE] = 0.0;
    sc[S_BERR] = 0.0;
    sc[S_FIRST] = 1.0;
    sc[S_K_USED] = 0.0;
    sc[S_CYCLE_DONE] = 0.0;
    sc[S_ATOL] = atol;
    sc[S_RTOL] = rtol;
    sc[S_MAXIT] = (double)maxit;
  }
}

}  // namespace

void krylov_free(afc_problem_s* p) {
  if (!p->kw) return;
  p->kw->vec.free_();
  p->kw->sc.free_();
  p->kw->part.free_();
  p->kw->counter.free_();
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
    if ((st = w.counter.alloc(4))) return st;
    if ((st = w.barrier.alloc(4))) return st;
    if (cudaMallocHost((void**)&w.hsc, (S_END + 8) * sizeof(double)) != cudaSuccess) {
      set_error("cudaMallocHost failed");
      return AFC_E_OOM;
    }
  }
  const int64_t need_part = (int64_t)(kMaxRestart + 4) * std::max<int64_t>(kRedBlocks, grid_for(p->N));
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

// The persistent BiCGStab launch on stream s (no synchronisation); *ok = false when
// the device cannot run cooperative launches (the caller then takes the
// kernel-per-phase path).
template <class T>
int bicg_fused_launch(afc_problem_s* p, cudaStream_t s, const T* B, const T* dinv, const afc_opts* o,
                      const double* rhs, double* xout, bool* ok, const KrylovEpilogue* epi) {
  KrylovWork& w = *p->kw;
  if (w.coop < 0) {
    int c = 0;
    AFC_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, p->device));
    AFC_CUDA(cudaDeviceGetAttribute(&w.nsm, cudaDevAttrMultiProcessorCount, p->device));
    w.coop = c;
  }
  *ok = w.coop > 0;
  if (!*ok) return AFC_OK;
  const int64_t N = p->N;
  T *x = vec_at<T>(w, 0), *r = vec_at<T>(w, 1), *rh = vec_at<T>(w, 2), *pp = vec_at<T>(w, 3), *v = vec_at<T>(w, 4),
    *sv = vec_at<T>(w, 5), *t = vec_at<T>(w, 6), *ph = vec_at<T>(w, 7), *sh = vec_at<T>(w, 8);
  double* sc = w.sc.p;
  GridBar* bar = reinterpret_cast<GridBar*>(w.barrier.p);
  int st = AFC_OK;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicg_fused<KT, T>, kFusedBlock, 0);
    if (e != cudaSuccess || nb < 1) {
      st = cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidConfiguration, "occupancy of k_bicg_fused");
      return;
    }
    const int64_t want = (N + kFusedBlock - 1) / kFusedBlock;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::min(nb, kFusedBlocksPerSM) * w.nsm));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kFusedBlock);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaEvent_t ev = prof_start(p);
    e = cudaLaunchKernelEx(&cfg, k_bicg_fused<KT, T>, N, p->offs, sc, B, dinv, rhs, xout, x, r, rh, pp, v, sv, t, ph,
                           sh, w.part.p, bar, o->ksp_atol, o->ksp_rtol, o->ksp_maxit,
                           epi ? *epi : KrylovEpilogue{}, (unsigned long long)p->grid_wait_ns);
    prof_stop(p, "k_bicg_fused", ev);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaLaunchKernelEx(k_bicg_fused)");
  });
  return st;
}

template <class T>
int bicgstab_impl(afc_problem_s* p, const T* B, const T* dinv, const afc_opts* o, const double* rhs, double* xout,
                  int* its, double* res, const KrylovEpilogue* epi, bool* epi_done) {
  int st = ensure_work(p, 9, sizeof(T) == 4);
  if (st) return st;
  KrylovWork& w = *p->kw;
  const int64_t N = p->N;
  cudaStream_t s = p->stream;
  T *x = vec_at<T>(w, 0), *r = vec_at<T>(w, 1), *rh = vec_at<T>(w, 2), *pp = vec_at<T>(w, 3), *v = vec_at<T>(w, 4),
    *sv = vec_at<T>(w, 5), *t = vec_at<T>(w, 6), *ph = vec_at<T>(w, 7), *sh = vec_at<T>(w, 8);
  double* sc = w.sc.p;
  double* part = w.part.p;
  unsigned int* cnt = w.counter.p;
  const int G = kRedBlocks;
  const int64_t gr = grid_for(N);
  bool fused = false;
  if ((st = bicg_fused_launch<T>(p, s, B, dinv, o, rhs, xout, &fused, epi))) return st;
  if (epi_done) *epi_done = fused && epi != nullptr;
  if (fused) {
    AFC_CUDA(cudaMemcpyAsync(w.hsc, sc, (S_MAXIT + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    unsigned int* hbar = reinterpret_cast<unsigned int*>(w.hsc + S_END);
    AFC_CUDA(cudaMemcpyAsync(hbar, w.barrier.p, 4 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (its) *its = (int)w.hsc[S_ITS];
    if (res) *res = w.hsc[S_NRES];
    if (hbar[2] != 0u) {
      AFC_CUDA(cudaMemsetAsync(w.barrier.p, 0, 4 * sizeof(unsigned int), s));
      AFC_CUDA(cudaStreamSynchronize(s));
      set_error("a grid barrier of the BiCGStab launch gave up waiting");
      return AFC_E_TIMEOUT;
    }
    const double done = w.hsc[S_DONE];
    if (done == 2.0) { set_error("BiCGStab breakdown or non-finite value"); return AFC_E_NAN; }
    return done == 1.0 ? AFC_OK : AFC_NOT_CONVERGED;
  }
  AFC_LAUNCH(p, "k_solver_reset", k_solver_reset<<<1, 32, 0, s>>>(sc, o->ksp_atol, o->ksp_rtol, o->ksp_maxit));
  AFC_LAUNCH(p, "k_bicg_init", k_bicg_init<T><<<G, kBlock, 0, s>>>(N, rhs, x, r, rh, pp, v, part, cnt, sc));
  AFC_CUDA(cudaGetLastError());
  int chunk = 2;
  int launched = 0;
  for (;;) {
    AFC_CUDA(cudaMemcpyAsync(w.hsc, sc, (S_MAXIT + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (w.hsc[S_DONE] != 0.0 || launched >= o->ksp_maxit) break;
    with_K(p->K, [&](auto kc) {
      constexpr int KT = decltype(kc)::value;
      for (int c = 0; c < chunk && launched < o->ksp_maxit; ++c, ++launched) {
        AFC_LAUNCH(p, "k_bicg_p", k_bicg_p<T><<<G, kBlock, 0, s>>>(N, sc, r, pp, v, dinv, ph));
        AFC_LAUNCH(p, "k_bicg_spmv1",
                   k_bicg_spmv1<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, ph, v, rh, part, cnt));
        AFC_LAUNCH(p, "k_bicg_s", k_bicg_s<T><<<G, kBlock, 0, s>>>(N, sc, r, v, dinv, sv, sh, part, cnt));
        AFC_LAUNCH(p, "k_bicg_spmv2",
                   k_bicg_spmv2<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, sh, t, sv, x, ph, part, cnt));
        AFC_LAUNCH(p, "k_bicg_xr", k_bicg_xr<T><<<G, kBlock, 0, s>>>(N, sc, x, ph, sh, sv, t, r, rh, part, cnt,
                                                                     GraphCond{}));
      }
    });
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
  if (m < 1 || m > kMaxRestart) { set_error("gmres_restart must be in 1..32"); return AFC_E_INVALID; }
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
  unsigned int* cnt = w.counter.p;
  const int G = kRedBlocks;
  const int64_t gr = grid_for(N);
  AFC_CUDA(cudaMemsetAsync(x - p->pad, 0, vs * sizeof(T), s));
  AFC_LAUNCH(p, "k_solver_reset", k_solver_reset<<<1, 32, 0, s>>>(sc, o->ksp_atol, o->ksp_rtol, o->ksp_maxit));
  for (;;) {
    with_K(p->K, [&](auto kc) {
      constexpr int KT = decltype(kc)::value;
      AFC_LAUNCH(p, "k_gm_residual",
                 k_gm_residual<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, x, rhs, wv, part, cnt));
    });
    AFC_CUDA(cudaGetLastError());
    AFC_CUDA(cudaMemcpyAsync(w.hsc, sc, S_CS * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFC_CUDA(cudaStreamSynchronize(s));
    if (w.hsc[S_DONE] != 0.0) break;
    AFC_LAUNCH(p, "k_gm_normalize", k_gm_normalize<T><<<G, kBlock, 0, s>>>(N, sc, wv, V, dinv, z));
    for (int k = 0; k < m; ++k) {
      with_K(p->K, [&](auto kc) {
        constexpr int KT = decltype(kc)::value;
        AFC_LAUNCH(p, "k_gm_spmv", k_gm_spmv<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, z, wv));
      });
      orth_launch<T>(p, G, N, sc, k, m, -1, S_H1, wv, V, vs, part, G, cnt);
      orth_launch<T>(p, G, N, sc, k, m, S_H1, S_H2, wv, V, vs, part, G, cnt);
      orth_launch<T>(p, G, N, sc, k, m, S_H2, -1, wv, V, vs, part, G, cnt);
      AFC_LAUNCH(p, "k_gm_normalize", k_gm_normalize<T><<<G, kBlock, 0, s>>>(N, sc, wv, V + (k + 1) * vs, dinv, z));
    }
    AFC_LAUNCH(p, "k_gm_update", k_gm_update<T><<<G, kBlock, 0, s>>>(N, sc, x, V, vs, dinv, GraphCond{}));
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

namespace {

template <class T>
int bicgstab_graph(afc_problem_s* p, const T* B, const T* dinv, const afc_opts* o, const double* rhs, double* xout,
                   cudaStream_t cs, cudaGraph_t g, std::vector<cudaGraphNode_t>& frontier,
                   const KrylovEpilogue* epi, bool* epi_done) {
  int st = ensure_work(p, 9, sizeof(T) == 4);
  if (st) return st;
  KrylovWork& w = *p->kw;
  const int64_t N = p->N;
  T *x = vec_at<T>(w, 0), *r = vec_at<T>(w, 1), *rh = vec_at<T>(w, 2), *pp = vec_at<T>(w, 3), *v = vec_at<T>(w, 4),
    *sv = vec_at<T>(w, 5), *t = vec_at<T>(w, 6), *ph = vec_at<T>(w, 7), *sh = vec_at<T>(w, 8);
  double* sc = w.sc.p;
  double* part = w.part.p;
  unsigned int* cnt = w.counter.p;
  const int G = kRedBlocks;
  const int64_t gr = grid_for(N);
  if (w.coop < 0) {
    int c = 0;
    AFC_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, p->device));
    AFC_CUDA(cudaDeviceGetAttribute(&w.nsm, cudaDevAttrMultiProcessorCount, p->device));
    w.coop = c;
  }
  if (w.coop > 0) {   // the whole solve is one persistent launch: no loop node needed
    if (epi_done) *epi_done = epi != nullptr;
    return capture_into(p, cs, g, frontier, [&]() -> int {
      bool ok = false;
      int s2 = bicg_fused_launch<T>(p, p->stream, B, dinv, o, rhs, xout, &ok, epi);
      if (s2) return s2;
      AFC_CUDA(cudaGetLastError());
      return AFC_OK;
    }, frontier);
  }
  GraphCond cond;
  cond.use = true;
  AFC_CUDA(cudaGraphConditionalHandleCreate(&cond.h, g, 0, 0));
  if ((st = capture_into(p, cs, g, frontier, [&]() -> int {
         AFC_LAUNCH(p, "k_solver_reset",
                    k_solver_reset<<<1, 32, 0, p->stream>>>(sc, o->ksp_atol, o->ksp_rtol, o->ksp_maxit));
         AFC_LAUNCH(p, "k_bicg_init", k_bicg_init<T><<<G, kBlock, 0, p->stream>>>(N, rhs, x, r, rh, pp, v, part, cnt, sc));
         AFC_LAUNCH(p, "k_cond_running", k_cond_running<<<1, 32, 0, p->stream>>>(sc, cond));
         AFC_CUDA(cudaGetLastError());
         return AFC_OK;
       }, frontier)))
    return st;
  cudaGraph_t body;
  cudaGraphNode_t loop;
  if ((st = add_conditional(g, frontier, cond.h, cudaGraphCondTypeWhile, &body, &loop))) return st;
  std::vector<cudaGraphNode_t> inner;
  if ((st = capture_into(p, cs, body, {}, [&]() -> int {
         with_K(p->K, [&](auto kc) {
           constexpr int KT = decltype(kc)::value;
           cudaStream_t s = p->stream;
           AFC_LAUNCH(p, "k_bicg_p", k_bicg_p<T><<<G, kBlock, 0, s>>>(N, sc, r, pp, v, dinv, ph));
           AFC_LAUNCH(p, "k_bicg_spmv1",
                      k_bicg_spmv1<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, ph, v, rh, part, cnt));
           AFC_LAUNCH(p, "k_bicg_s", k_bicg_s<T><<<G, kBlock, 0, s>>>(N, sc, r, v, dinv, sv, sh, part, cnt));
           AFC_LAUNCH(p, "k_bicg_spmv2",
                      k_bicg_spmv2<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, sh, t, sv, x, ph, part, cnt));
           AFC_LAUNCH(p, "k_bicg_xr",
                      k_bicg_xr<T><<<G, kBlock, 0, s>>>(N, sc, x, ph, sh, sv, t, r, rh, part, cnt, cond));
         });
         AFC_CUDA(cudaGetLastError());
         return AFC_OK;
       }, inner)))
    return st;
  frontier.assign(1, loop);
  return capture_into(p, cs, g, frontier, [&]() -> int {
    AFC_LAUNCH(p, "k_to_double", k_to_double<T><<<G, kBlock, 0, p->stream>>>(N, x, xout));
    AFC_CUDA(cudaGetLastError());
    return AFC_OK;
  }, frontier);
}

template <class T>
int gmres_graph(afc_problem_s* p, const T* B, const T* dinv, const afc_opts* o, const double* rhs, double* xout,
                cudaStream_t cs, cudaGraph_t g, std::vector<cudaGraphNode_t>& frontier) {
  const int m = o->gmres_restart;
  if (m < 1 || m > kMaxRestart) { set_error("gmres_restart must be in 1..32"); return AFC_E_INVALID; }
  int st = ensure_work(p, 3 + m + 1, sizeof(T) == 4);
  if (st) return st;
  KrylovWork& w = *p->kw;
  const int64_t N = p->N;
  T *x = vec_at<T>(w, 0), *wv = vec_at<T>(w, 1), *z = vec_at<T>(w, 2), *V = vec_at<T>(w, 3);
  const size_t vs = w.vstride;
  double* sc = w.sc.p;
  double* part = w.part.p;
  unsigned int* cnt = w.counter.p;
  const int G = kRedBlocks;
  const int64_t gr = grid_for(N);
  GraphCond cond;
  cond.use = true;
  AFC_CUDA(cudaGraphConditionalHandleCreate(&cond.h, g, 0, 0));
  if ((st = capture_into(p, cs, g, frontier, [&]() -> int {
         AFC_CUDA(cudaMemsetAsync(x - p->pad, 0, vs * sizeof(T), p->stream));
         AFC_LAUNCH(p, "k_solver_reset",
                    k_solver_reset<<<1, 32, 0, p->stream>>>(sc, o->ksp_atol, o->ksp_rtol, o->ksp_maxit));
         AFC_LAUNCH(p, "k_cond_running", k_cond_running<<<1, 32, 0, p->stream>>>(sc, cond));
         AFC_CUDA(cudaGetLastError());
         return AFC_OK;
       }, frontier)))
    return st;
  cudaGraph_t body;
  cudaGraphNode_t loop;
  if ((st = add_conditional(g, frontier, cond.h, cudaGraphCondTypeWhile, &body, &loop))) return st;
  std::vector<cudaGraphNode_t> inner;
  if ((st = capture_into(p, cs, body, {}, [&]() -> int {
         cudaStream_t s = p->stream;
         with_K(p->K, [&](auto kc) {
           constexpr int KT = decltype(kc)::value;
           AFC_LAUNCH(p, "k_gm_residual",
                      k_gm_residual<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, x, rhs, wv, part, cnt));
           AFC_LAUNCH(p, "k_gm_normalize", k_gm_normalize<T><<<G, kBlock, 0, s>>>(N, sc, wv, V, dinv, z));
           for (int k = 0; k < m; ++k) {
             AFC_LAUNCH(p, "k_gm_spmv", k_gm_spmv<KT, T><<<gr, kBlock, 0, s>>>(N, p->offs, sc, B, z, wv));
             orth_launch<T>(p, G, N, sc, k, m, -1, S_H1, wv, V, vs, part, G, cnt);
             orth_launch<T>(p, G, N, sc, k, m, S_H1, S_H2, wv, V, vs, part, G, cnt);
             orth_launch<T>(p, G, N, sc, k, m, S_H2, -1, wv, V, vs, part, G, cnt);
             AFC_LAUNCH(p, "k_gm_normalize",
                        k_gm_normalize<T><<<G, kBlock, 0, s>>>(N, sc, wv, V + (k + 1) * vs, dinv, z));
           }
           AFC_LAUNCH(p, "k_gm_update", k_gm_update<T><<<G, kBlock, 0, s>>>(N, sc, x, V, vs, dinv, cond));
         });
         AFC_CUDA(cudaGetLastError());
         return AFC_OK;
       }, inner)))
    return st;
  frontier.assign(1, loop);
  return capture_into(p, cs, g, frontier, [&]() -> int {
    AFC_LAUNCH(p, "k_to_double", k_to_double<T><<<G, kBlock, 0, p->stream>>>(N, x, xout));
    AFC_CUDA(cudaGetLastError());
    return AFC_OK;
  }, frontier);
}

}  // namespace

int krylov_graph(afc_problem_s* p, int system, const afc_opts* o, const double* rhs, double* x, cudaStream_t cs,
                 cudaGraph_t g, std::vector<cudaGraphNode_t>& frontier, const KrylovEpilogue* epi,
                 bool* epi_done) {
  if (epi_done) *epi_done = false;
  const bool mixed = o->precision == AFC_MIXED;
  if (mixed && p->precision != AFC_MIXED) {
    set_error("mixed-precision solve needs afc_assemble(..., AFC_MIXED)");
    return AFC_E_STATE;
  }
  const bool gm = o->ksp == AFC_KSP_GMRES;
  if (mixed) {
    const float* B = system == 0 ? p->Bst32.p : p->Bcn32.p;
    const float* di = system == 0 ? p->dinv_st32.p : p->dinv_cn32.p;
    return gm ? gmres_graph<float>(p, B, di, o, rhs, x, cs, g, frontier)
              : bicgstab_graph<float>(p, B, di, o, rhs, x, cs, g, frontier, epi, epi_done);
  }
  const double* B = system == 0 ? p->Bst.p : p->Bcn.p;
  const double* di = system == 0 ? p->dinv_st.p : p->dinv_cn.p;
  return gm ? gmres_graph<double>(p, B, di, o, rhs, x, cs, g, frontier)
            : bicgstab_graph<double>(p, B, di, o, rhs, x, cs, g, frontier, epi, epi_done);
}

const double* krylov_scalars(afc_problem_s* p) { return p->kw ? p->kw->sc.p : nullptr; }
int krylov_cycles_slot() { return S_CYCLES; }

int krylov_reset_barrier(afc_problem_s* p) {
  if (!p->kw || !p->kw->barrier.p) return AFC_OK;
  AFC_CUDA(cudaMemsetAsync(p->kw->barrier.p, 0, 4 * sizeof(unsigned int), p->stream));
  AFC_CUDA(cudaStreamSynchronize(p->stream));
  return AFC_OK;
}
const void* krylov_key(afc_problem_s* p) { return p->kw ? (const void*)p->kw->vec.base : nullptr; }

int krylov_solve(afc_problem_s* p, int system, const afc_opts* o, const double* rhs, double* x, int* its,
                 double* res, const KrylovEpilogue* epi, bool* epi_done) {
  if (epi_done) *epi_done = false;
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
    return gm ? gmres_impl<float>(p, B, di, o, rhs, x, its, res)
              : bicgstab_impl<float>(p, B, di, o, rhs, x, its, res, epi, epi_done);
  }
  const double* B = system == 0 ? p->Bst.p : p->Bcn.p;
  const double* di = system == 0 ? p->dinv_st.p : p->dinv_cn.p;
  return gm ? gmres_impl<double>(p, B, di, o, rhs, x, its, res)
            : bicgstab_impl<double>(p, B, di, o, rhs, x, its, res, epi, epi_done);
}

}  // namespace afc
