// A variant of the monolithic-convex limited sum (afc_mc_limited_sum) that
// allocates no device memory, for callers that cannot call cudaMalloc: code
// that runs between the set-up and tear-down of a solver inside a stream-ordered
// pipeline (cudaMalloc synchronises the device and is not allowed while a stream
// is being captured), and embedding runtimes that reserve all device memory up
// front and forbid allocation afterwards.  The caller passes the input state and
// the output array on the device; the two bound vectors u_max / u_min the
// limiter needs live in a fixed, file-scope device array instead of buffers of
// the problem.
#include <mutex>

#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

namespace {

// Largest problem the entry point accepts, and the scratch it needs: two node
// vectors of doubles, 2 x 262144 x 8 bytes = 4 MiB, held by every GPU that loads
// this library until the process exits.
constexpr int64_t kNoAllocMaxNodes = 262144;
static __device__ __align__(256) double g_mc_bounds_scratch[2 * kNoAllocMaxNodes];

// Device address of the scratch array, looked up once per device.  In host code
// the array's name is only a host-side stand-in, never a device address.
std::mutex g_scratch_mutex;
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};

// Makes the problem's device current for the call and gives the caller's current
// device back when the call returns.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int device) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != device) err = cudaSetDevice(device);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

int scratch_for(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("device index out of range for the no-allocation entry point");
    return AFC_E_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    // the caller made `device` current
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_mc_bounds_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_mc_bounds_scratch)");
    g_scratch_ptr[device] = static_cast<double*>(ptr);
  }
  *out = g_scratch_ptr[device];
  return AFC_OK;
}

// u_max / u_min over N_i (Eq. u_max_min).  The caller's u has no halo, so only
// neighbours present in the pattern (all inside 0..N-1) are read.
__global__ void k_mc_bounds_noalloc(int64_t N, Offsets of, const unsigned long long* __restrict__ mask,
                                    const double* __restrict__ u, double* __restrict__ umax,
                                    double* __restrict__ umin) {
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

// F*_i = sum_j r*_ij (Eq. MClimiter; alpha = 1 / alpha = 0 for the other limiter
// modes), 0 at Dirichlet rows; the same arithmetic as the allocating pass.
__global__ void k_mc_fstar_noalloc(int64_t N, Offsets of, int limiter, const unsigned long long* __restrict__ mask,
                                   const double* __restrict__ d_up, const double* __restrict__ Kf,
                                   const double* __restrict__ u, const double* __restrict__ umax,
                                   const double* __restrict__ umin, const uint8_t* __restrict__ dir,
                                   double* __restrict__ Fout) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double F = 0.0;
  if (!dir[i] && limiter != AFC_LIM_NONE) {
    const unsigned long long mk = mask[i];
    const double ui = u[i], mxi = umax[i], mni = umin[i];
    for (int k = 0; k < of.K; ++k) {
      if (k == of.Kup || !((mk >> k) & 1ull)) continue;
      const int64_t j = i + of.o[k];
      const double uj = u[j];
      const double d = pair_d(of, k, i, N, d_up);
      double rs = d * (uj - ui);
      if (limiter == AFC_LIM_MC) {
        if (d == 0.0) {
          rs = 0.0;
        } else {
          const double aij = Kf[k * N + i];
          const double aji = Kf[(int64_t)(of.K - 1 - k) * N + j];
          const double ubij = (d * (ui + uj) + aij * (uj - ui)) / (2.0 * d);
          const double ubji = (d * (uj + ui) + aji * (ui - uj)) / (2.0 * d);
          if (rs > 0.0) rs = fmin(rs, fmin(2.0 * d * (ubij - mxi), 2.0 * d * (umin[j] - ubji)));
          else rs = fmax(rs, fmax(2.0 * d * (ubij - mni), 2.0 * d * (umax[j] - ubji)));
        }
      }
      F += rs;
    }
  }
  Fout[i] = F;
}

}  // namespace

}  // namespace afc

using namespace afc;

extern "C" int afc_mc_limited_sum_noalloc(afc_problem p, int limiter, const double* u, double* Fstar) {
  if (!p) { set_error("null problem"); return AFC_E_INVALID; }
  if (!p->assembled) { set_error("call afc_assemble first"); return AFC_E_STATE; }
  if (!u || !Fstar) { set_error("need device pointers u and Fstar"); return AFC_E_INVALID; }
  if (limiter != AFC_LIM_NONE && limiter != AFC_LIM_GALERKIN && limiter != AFC_LIM_MC) {
    set_error("limiter must be AFC_LIM_NONE, AFC_LIM_GALERKIN or AFC_LIM_MC");
    return AFC_E_INVALID;
  }
  if (p->family != AFC_FAMILY_MC && limiter != AFC_LIM_NONE) {
    // d_ij and the convective entries of the MC family (Remark rem:assembling_mc)
    set_error("the MC limiter and its Galerkin mode need afc_assemble(..., AFC_FAMILY_MC, ...)");
    return AFC_E_STATE;
  }
  if (p->N > kNoAllocMaxNodes) {
    set_error("afc_mc_limited_sum_noalloc accepts at most 262144 nodes (its fixed scratch holds two node vectors); "
              "use afc_mc_limited_sum");
    return AFC_E_INVALID;
  }
  DeviceGuard dg(p->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  double* scratch = nullptr;
  int st = scratch_for(p->device, &scratch);
  if (st) return st;
  double* umax = scratch;
  double* umin = scratch + kNoAllocMaxNodes;
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  if (limiter == AFC_LIM_MC) {
    k_mc_bounds_noalloc<<<g, kBlock, 0, p->stream>>>(N, p->offs, p->mask.p, u, umax, umin);
    p->launches++;
  }
  k_mc_fstar_noalloc<<<g, kBlock, 0, p->stream>>>(N, p->offs, limiter, p->mask.p, p->d_up.p, p->Kfull.p, u, umax, umin,
                                                 p->dir.p, Fstar);
  p->launches++;
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}
