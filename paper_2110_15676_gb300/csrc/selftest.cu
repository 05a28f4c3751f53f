// Self-test of the bounded grid wait (the failure-detection path of the persistent
// kernels' barriers), exercised without a fault: block 1 of a two-block launch never
// arrives, so block 0's wait runs out after the given limit, records the error in
// the barrier state and the launch ends.  The host then reads the flag as the
// solvers do and checks that the device still runs kernels.
#include <chrono>

#include "grid_sync.cuh"
#include "kernels_common.cuh"
#include "pair_float.cuh"

namespace afc {
namespace {

__global__ void k_grid_wait_selftest(GridBar* gb, unsigned long long limit_ns) {
  if (blockIdx.x != 0) return;   // the block that never arrives
  const unsigned int old = grid_arrive(gb);
  grid_wait(gb, old, limit_ns);
}

__global__ void k_selftest_touch(int* x) {
  if (threadIdx.x == 0) *x = 7;
}

// The float-pair split and the exact widening of the mixed MC sweep, element by element.
__global__ void k_selftest_split(int64_t n, const double* __restrict__ x, float* __restrict__ hi,
                                 float* __restrict__ lo, double* __restrict__ back) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 p = split_pair(x[i]);
  hi[i] = p.x;
  lo[i] = p.y;
  back[i] = widen_exact(p.x);
}

}  // namespace
}  // namespace afc

using namespace afc;

extern "C" int afc_selftest_grid_wait(int device, double limit_ms, int* observed, double* waited_ms) {
  if (!(limit_ms > 0.0) || limit_ms > 4000.0 || !observed) {
    set_error("afc_selftest_grid_wait: need 0 < limit_ms <= 4000 and an output pointer");
    return AFC_E_INVALID;
  }
  AFC_CUDA(cudaSetDevice(device));
  GridBar* gb = nullptr;
  int* flag = nullptr;
  AFC_CUDA(cudaMalloc((void**)&gb, sizeof(GridBar) + sizeof(int)));
  flag = reinterpret_cast<int*>(gb + 1);
  int st = AFC_OK;
  do {
    cudaError_t e;
    if ((e = cudaMemset(gb, 0, sizeof(GridBar) + sizeof(int))) != cudaSuccess) { st = cuda_fail(e, "cudaMemset"); break; }
    const auto t0 = std::chrono::steady_clock::now();
    k_grid_wait_selftest<<<2, 64>>>(gb, (unsigned long long)(limit_ms * 1e6));
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
      st = cuda_fail(e, "k_grid_wait_selftest");
      break;
    }
    const auto t1 = std::chrono::steady_clock::now();
    if (waited_ms) *waited_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    GridBar h{};
    if ((e = cudaMemcpy(&h, gb, sizeof(GridBar), cudaMemcpyDeviceToHost)) != cudaSuccess) {
      st = cuda_fail(e, "cudaMemcpy");
      break;
    }
    *observed = h.err != 0 ? AFC_E_TIMEOUT : AFC_OK;
    // the context is still usable: a later launch runs and its result arrives
    k_selftest_touch<<<1, 32>>>(flag);
    int hf = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
      st = cuda_fail(e, "launch after the expired wait");
      break;
    }
    if (hf != 7) {
      set_error("a launch after the expired wait did not run");
      st = AFC_E_CUDA;
    }
  } while (false);
  cudaFree(gb);
  return st;
}

extern "C" int afc_selftest_split(int device, const double* x, int64_t n, float* hi, float* lo, double* hi_widened) {
  if (n < 0 || (n > 0 && (!x || !hi || !lo || !hi_widened)) || n > ((int64_t)1 << 26)) {
    set_error("afc_selftest_split: need 0 <= n <= 2^26 and host arrays of n values");
    return AFC_E_INVALID;
  }
  if (n == 0) return AFC_OK;
  AFC_CUDA(cudaSetDevice(device));
  char* buf = nullptr;
  const size_t bx = (size_t)n * sizeof(double), bf = (size_t)n * sizeof(float);
  AFC_CUDA(cudaMalloc((void**)&buf, 2 * bx + 2 * bf));
  double* dx = reinterpret_cast<double*>(buf);
  double* db = reinterpret_cast<double*>(buf + bx);
  float* dh = reinterpret_cast<float*>(buf + 2 * bx);
  float* dl = reinterpret_cast<float*>(buf + 2 * bx + bf);
  int st = AFC_OK;
  cudaError_t e;
  if ((e = cudaMemcpy(dx, x, bx, cudaMemcpyHostToDevice)) != cudaSuccess) {
    st = cuda_fail(e, "cudaMemcpy");
  } else {
    k_selftest_split<<<(unsigned)((n + 255) / 256), 256>>>(n, dx, dh, dl, db);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess ||
        (e = cudaMemcpy(hi, dh, bf, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(lo, dl, bf, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(hi_widened, db, bx, cudaMemcpyDeviceToHost)) != cudaSuccess)
      st = cuda_fail(e, "k_selftest_split");
  }
  cudaFree(buf);
  return st;
}
