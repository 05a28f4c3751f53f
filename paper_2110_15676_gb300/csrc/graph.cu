// One time step or one stationary solve as a single CUDA graph launch.
//
// The damped fixed point of Sec. 4 is a while node: its body evaluates the
// limited residual and a one-thread control kernel decides on the device whether
// to stop (Eq. tol_formula, the iteration limit, or a fixed count) and whether
// the body's if node runs the linear solve (itself a while node over the Krylov
// iterations) and the update.  The host launches the graph and synchronises once;
// no scalar travels to the host inside the step.  The explicit SSP step is a
// plain captured graph.  Graphs are built on first use and rebuilt when the
// options or the problem's buffers change.
#include <cmath>
#include <cstring>
#include <vector>

#include "graph_util.h"
#include "kernels_common.cuh"

namespace afc {

namespace {


__global__ void k_fp_init(double* sc, double thresh, int fixed, int maxit) {
  if (threadIdx.x != 0) return;
  sc[F_CORR] = 0.0;
  sc[F_INNER] = 0.0;
  sc[F_STATUS] = 0.0;
  sc[F_THRESH] = thresh;
  sc[F_FIXED] = (double)fixed;
  sc[F_MAXIT] = (double)maxit;
  sc[F_KBODY] = 0.0;
  sc[F_REVAL] = 0.0;
  sc[F_TIMEOUT] = 0.0;
}

// After a residual evaluation: R = ||res||; stop or solve.  The residual pass leaves
// its block partials of res^2 in part[0 .. npart); one block of 1024 threads sums them
// (the order of finalize_sum) before the decision, so the sum needs no launch of its own.
__global__ void k_fp_control(double* sc, const double* __restrict__ part, int npart,
                             cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_solve) {
  pdl_wait();   // the residual pass's partials (a no-op when launched without the attribute)
  block_sum_to(strided_sum_1024(part, npart, threadIdx.x), sc + F_NORMSQ);   // one block of 1024
  if (threadIdx.x != 0) return;
  const double R = sqrt(sc[F_NORMSQ]);
  const double it = sc[F_CORR];
  if (sc[F_REVAL] == 0.0) sc[F_RES0] = R;
  sc[F_RESF] = R;
  sc[F_REVAL] += 1.0;
  bool stop = false;
  if (!isfinite(R) || sc[F_STATUS] == 2.0) {
    stop = true;
    sc[F_STATUS] = 2.0;
  } else if (sc[F_FIXED] > 0.0) {
    if (it >= sc[F_FIXED]) { stop = true; sc[F_STATUS] = 1.0; }
  } else if (R < sc[F_THRESH]) {
    stop = true;
    sc[F_STATUS] = 1.0;
  } else if (it >= sc[F_MAXIT]) {
    stop = true;
    sc[F_STATUS] = 3.0;
  }
  cudaGraphSetConditional(h_loop, stop ? 0u : 1u);
  cudaGraphSetConditional(h_solve, stop ? 0u : 1u);
}

// After a linear solve: count it, its Krylov iterations and loop-body executions;
// a solver breakdown ends the fixed point at the next control.
__global__ void k_fp_after_solve(double* sc, const double* __restrict__ ksc, int gmres, int cycles_slot) {
  if (threadIdx.x != 0) return;
  sc[F_CORR] += 1.0;
  sc[F_INNER] += ksc[kKrylovItsSlot];
  sc[F_KBODY] += gmres ? ksc[cycles_slot] : ksc[kKrylovItsSlot];
  if (ksc[kKrylovDoneSlot] == 2.0) sc[F_STATUS] = 2.0;
  if (!gmres && ksc[kKrylovBarrierErrSlot] != 0.0) {
    sc[F_STATUS] = 2.0;
    sc[F_TIMEOUT] = 1.0;
  }
}

__global__ void k_copy(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i];
}

__global__ void k_apply_dirichlet_g(int64_t N, const uint8_t* __restrict__ dir, const double* __restrict__ udir,
                                    double* __restrict__ u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N && dir[i]) u[i] = udir[i];
}

__global__ void k_minmax_g(int64_t N, const double* __restrict__ x, double* __restrict__ part) {
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

__global__ void k_minmax_fin_g(const double* __restrict__ part, int n, double* __restrict__ out) {
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

// solution extremes into scal[60..61], then all scalars to the pinned host mirror
int enqueue_stats(afc_problem_s* p) {
  AFC_LAUNCH(p, "k_minmax", k_minmax_g<<<kRedBlocks, kBlock, 0, p->stream>>>(p->N, p->u.p, p->part.p));
  AFC_LAUNCH(p, "k_minmax_fin", k_minmax_fin_g<<<1, kBlock, 0, p->stream>>>(p->part.p, kRedBlocks, p->scal.p + 60));
  AFC_CUDA(cudaGetLastError());
  AFC_CUDA(cudaMemcpyAsync(p->host_scal, p->scal.p, 64 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  return AFC_OK;
}

}  // namespace

// Cached executable graph and the kernel count of each of its sections (for the
// launch accounting of afc_profile_read).
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;
  int64_t k_pro = 0, k_outer = 0, k_solve = 0, k_body = 0, k_epi = 0;
  int kind = 0;   // 1 fixed point, 2 explicit SSP
};

namespace {

std::vector<unsigned char> make_key(afc_problem_s* p, const afc_opts* o, int what) {
  std::vector<unsigned char> k(sizeof(afc_opts) + 64);
  std::memcpy(k.data(), o, sizeof(afc_opts));
  double cdt = p->cn_dt;
  uintptr_t cdt_bits;
  std::memcpy(&cdt_bits, &cdt, sizeof(cdt_bits));
  uintptr_t extra[7] = {(uintptr_t)what, (uintptr_t)p->stream, (uintptr_t)krylov_key(p), (uintptr_t)p->AA.p,
                        (uintptr_t)p->Bcn.p, cdt_bits, (uintptr_t)p->grid_wait_ns};
  std::memcpy(k.data() + sizeof(afc_opts), extra, sizeof(extra));
  return k;
}

void drop(StepGraph*& g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  g = nullptr;
}

struct ProfOff {   // no event records inside captured graphs; captured launches are not executions
  afc_problem_s* p;
  bool was = false;
  int64_t launches = 0;
  explicit ProfOff(afc_problem_s* p_) : p(p_), launches(p_->launches) { was = prof_set_enabled(p, false); }
  ~ProfOff() {
    prof_set_enabled(p, was);
    p->launches = launches;
  }
};

// Build the fixed-point graph: prologue, while(outer){ residual; control; if(solve){ Krylov; update; count } },
// epilogue.  `system` 1: CN step, 0: stationary.
template <class Pro, class Res, class Upd>
int build_fixed_point(afc_problem_s* p, const afc_opts* o, int system, Pro prologue, Res residual, Upd update,
                      StepGraph& sg, const KrylovEpilogue* epi = nullptr) {
  if (!p->cap_stream) AFC_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = p->cap_stream;
  ProfOff po(p);
  cudaGraph_t g = nullptr;
  AFC_CUDA(cudaGraphCreate(&g, 0));
  int st = AFC_OK;
  std::vector<cudaGraphNode_t> fr;
  cudaGraphConditionalHandle h_loop, h_solve;
  const double thresh = std::sqrt((double)p->N) * o->fp_tol;
  auto count = [&](auto&& f) {
    const int64_t l0 = p->launches;
    int s = f();
    return std::make_pair(s, p->launches - l0);
  };
  do {
    auto r1 = count([&]() -> int {
      return capture_into(p, cs, g, fr, [&]() -> int {
        AFC_LAUNCH(p, "k_fp_init", k_fp_init<<<1, 32, 0, p->stream>>>(p->scal.p, thresh, o->fp_fixed_its,
                                                                       o->fp_maxit));
        return prologue();
      }, fr);
    });
    if ((st = r1.first)) break;
    sg.k_pro = r1.second;
    if (cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "cudaGraphConditionalHandleCreate");
      break;
    }
    cudaGraph_t body;
    cudaGraphNode_t loop;
    if ((st = add_conditional(g, fr, h_loop, cudaGraphCondTypeWhile, &body, &loop))) break;
    if (cudaGraphConditionalHandleCreate(&h_solve, body, 0, 0) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "cudaGraphConditionalHandleCreate");
      break;
    }
    std::vector<cudaGraphNode_t> bf;
    auto r2 = count([&]() -> int {
      return capture_into(p, cs, body, {}, [&]() -> int {
        int s = residual();
        if (s) return s;
        // programmatic dependency on the Zalesak CN residual pass, which ends the body's residual
        // (the other residuals end with other work and keep a plain one)
        const bool pdl = system == 1 && o->limiter == AFC_LIM_ZALESAK;
        AFC_LAUNCH(p, "k_fp_control", launch_pass(pdl, k_fp_control, dim3(1), dim3(1024), p->stream,
                                                  p->scal.p, (const double*)p->part.p, (int)grid_for(p->N), h_loop,
                                                  h_solve));
        AFC_CUDA(cudaGetLastError());
        return AFC_OK;
      }, bf);
    });
    if ((st = r2.first)) break;
    sg.k_outer = r2.second;
    cudaGraph_t sbody;
    cudaGraphNode_t ifnode;
    if ((st = add_conditional(body, bf, h_solve, cudaGraphCondTypeIf, &sbody, &ifnode))) break;
    // Krylov solve (its while node counts separately), update and counters
    std::vector<cudaGraphNode_t> sf;
    const int64_t l0 = p->launches;
    bool applied = false;   // the persistent BiCGStab applies the update itself
    // ... and then also counts the correction in the fixed-point scalars (no after-solve node)
    KrylovEpilogue epc;
    if (epi) {
      epc = *epi;
      epc.fp_sc = p->scal.p;
    }
    if ((st = krylov_graph(p, system, o, p->res.p, p->delta.p, cs, sbody, sf, epi ? &epc : nullptr, &applied)))
      break;
    const int64_t lk = p->launches - l0;
    const int64_t body_k = o->ksp == AFC_KSP_GMRES ? 3 + 5 * (int64_t)o->gmres_restart : 5;
    auto r3 = count([&]() -> int {
      return capture_into(p, cs, sbody, sf, [&]() -> int {
        if (applied) return AFC_OK;   // the fused solve updated u and counted the correction
        int s = update();
        if (s) return s;
        AFC_LAUNCH(p, "k_fp_after_solve",
                   k_fp_after_solve<<<1, 32, 0, p->stream>>>(p->scal.p, krylov_scalars(p),
                                                             o->ksp == AFC_KSP_GMRES ? 1 : 0, krylov_cycles_slot()));
        AFC_CUDA(cudaGetLastError());
        return AFC_OK;
      }, sf);
    });
    if ((st = r3.first)) break;
    sg.k_body = body_k;
    sg.k_solve = lk - body_k + r3.second;
    fr.assign(1, loop);
    auto r4 = count([&]() -> int { return capture_into(p, cs, g, fr, [&]() -> int { return enqueue_stats(p); }, fr); });
    if ((st = r4.first)) break;
    sg.k_epi = r4.second;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphInstantiate"); break; }
    sg.exec = ex;
    sg.kind = 1;
  } while (false);
  cudaGraphDestroy(g);
  return st;
}

int run_fixed_point_graph(afc_problem_s* p, StepGraph& sg, afc_stats* stt) {
  AFC_CUDA(cudaGraphLaunch(sg.exec, p->stream));
  AFC_CUDA(cudaStreamSynchronize(p->stream));
  const double* h = p->host_scal;
  const int64_t reval = (int64_t)h[F_REVAL], corr = (int64_t)h[F_CORR], kbody = (int64_t)h[F_KBODY];
  p->launches += sg.k_pro + reval * sg.k_outer + corr * sg.k_solve + kbody * sg.k_body + sg.k_epi;
  int status = h[F_STATUS] == 1.0 ? AFC_OK : h[F_STATUS] == 2.0 ? AFC_E_NAN : AFC_NOT_CONVERGED;
  if (h[F_TIMEOUT] != 0.0) {
    // the barrier counter is inconsistent after blocks skipped barriers: clear it so
    // that the next persistent launch starts from a clean state
    const int rs = krylov_reset_barrier(p);
    if (rs) return rs;
    status = AFC_E_TIMEOUT;
    set_error("a grid barrier of the persistent BiCGStab launch gave up waiting");
  } else if (status == AFC_E_NAN) {
    set_error("non-finite nonlinear residual or Krylov breakdown");
  }
  if (stt) {
    stt->outer_its = (int)corr;
    stt->inner_its = (int)h[F_INNER];
    stt->res0 = h[F_RES0];
    stt->res_final = h[F_RESF];
    stt->umin = h[60];
    stt->umax = h[61];
    stt->status = status;
  }
  return status;
}

}  // namespace

void graph_free(afc_problem_s* p) {
  drop(p->g_step);
  drop(p->g_stat);
  if (p->cap_stream) {
    cudaStreamDestroy(p->cap_stream);
    p->cap_stream = nullptr;
  }
}

int cn_step_graph(afc_problem_s* p, const afc_opts* o, afc_stats* stt) {
  const auto key = make_key(p, o, 1);
  if (!p->g_step || p->g_step->key != key) {
    drop(p->g_step);
    p->g_step = new StepGraph();
    const int lim = o->limiter;
    const double dt = o->dt;
    KrylovEpilogue epi;
    epi.omega = o->omega;
    epi.u = p->u.p;
    epi.uo = p->u0.p;
    epi.a = p->cn_a.p;
    epi.s = p->cn_s.p;
    int st = build_fixed_point(
        p, o, 1,
        [&]() -> int {
          const int64_t N = p->N;
          AFC_LAUNCH(p, "k_copy", k_copy<<<grid_for(N), kBlock, 0, p->stream>>>(N, p->u.p, p->u0.p));
          int s = cn_predictor(p, p->u0.p, dt);
          if (s) return s;
          if (lim == AFC_LIM_MC) {
            AFC_LAUNCH(p, "k_apply_dirichlet",
                       k_apply_dirichlet_g<<<grid_for(N), kBlock, 0, p->stream>>>(N, p->dir.p, p->udir.p, p->u.p));
            return mc_cn_old_flux(p, p->u0.p);
          }
          if (o->scheme == AFC_CN_LINEAR) {
            if ((s = cn_linear_guess(p, p->u0.p, p->u.p))) return s;
          } else {
            AFC_LAUNCH(p, "k_apply_dirichlet",
                       k_apply_dirichlet_g<<<grid_for(N), kBlock, 0, p->stream>>>(N, p->dir.p, p->udir.p, p->u.p));
          }
          return cn_update(p, 0.0, nullptr, p->u.p, p->u0.p);
        },
        [&]() -> int {
          if (lim == AFC_LIM_MC) return mc_cn_residual(p, p->u.p, p->res.p, nullptr);
          return cn_limited_residual(p, p->u.p, dt, lim, o->prelimit, p->res.p, nullptr);
        },
        [&]() -> int {
          if (lim == AFC_LIM_MC) return axpy_device(p, o->omega, p->delta.p, p->u.p);
          return cn_update(p, o->omega, p->delta.p, p->u.p, p->u0.p);
        }, *p->g_step, lim == AFC_LIM_MC ? nullptr : &epi);
    if (st) {
      drop(p->g_step);
      return st;
    }
    p->g_step->key = key;
  }
  return run_fixed_point_graph(p, *p->g_step, stt);
}

int stationary_graph(afc_problem_s* p, const afc_opts* o, afc_stats* stt) {
  const auto key = make_key(p, o, 2);
  if (!p->g_stat || p->g_stat->key != key) {
    drop(p->g_stat);
    p->g_stat = new StepGraph();
    const int lim = o->limiter;
    int st = build_fixed_point(
        p, o, 0,
        [&]() -> int {
          AFC_LAUNCH(p, "k_apply_dirichlet", k_apply_dirichlet_g<<<grid_for(p->N), kBlock, 0, p->stream>>>(
                                                 p->N, p->dir.p, p->udir.p, p->u.p));
          AFC_CUDA(cudaGetLastError());
          return AFC_OK;
        },
        [&]() -> int {
          return mc_limited_residual(p, p->u.p, lim, p->res.p, nullptr, false, o->precision == AFC_MIXED);
        },
        [&]() -> int { return axpy_device(p, o->omega, p->delta.p, p->u.p); }, *p->g_stat);
    if (st) {
      drop(p->g_stat);
      return st;
    }
    p->g_stat->key = key;
  }
  return run_fixed_point_graph(p, *p->g_stat, stt);
}

int ssp_step_graph(afc_problem_s* p, const afc_opts* o, afc_stats* stt) {
  const bool mixed = o->precision == AFC_MIXED;
  if (mixed) {
    int s0 = ensure_ssp_mixed(p);   // allocation and conversion stay outside the capture
    if (s0) return s0;
  }
  const auto key = make_key(p, o, 3);
  if (!p->g_step || p->g_step->key != key) {
    drop(p->g_step);
    p->g_step = new StepGraph();
    if (!p->cap_stream) AFC_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    ProfOff po(p);
    cudaGraph_t g = nullptr;
    AFC_CUDA(cudaGraphCreate(&g, 0));
    std::vector<cudaGraphNode_t> fr;
    const int64_t l0 = p->launches;
    const int lim = o->limiter;
    const double dt = o->dt;
    int st = capture_into(p, p->cap_stream, g, fr, [&]() -> int {
      const int64_t N = p->N;
      AFC_LAUNCH(p, "k_copy", k_copy<<<grid_for(N), kBlock, 0, p->stream>>>(N, p->u.p, p->u0.p));
      int s;
      if (o->scheme == AFC_SSP2) {
        if ((s = fe_stage(p, p->u0.p, dt, lim, 0.0, nullptr, 1.0, p->ustage.p, mixed))) return s;
        if ((s = fe_stage(p, p->ustage.p, dt, lim, 0.5, p->u0.p, 0.5, p->u.p, mixed))) return s;
      } else {
        if ((s = fe_stage(p, p->u0.p, dt, lim, 0.0, nullptr, 1.0, p->ustage.p, mixed))) return s;
        if ((s = fe_stage(p, p->ustage.p, dt, lim, 0.75, p->u0.p, 0.25, p->tmp.p, mixed))) return s;
        if ((s = fe_stage(p, p->tmp.p, dt, lim, 1.0 / 3.0, p->u0.p, 2.0 / 3.0, p->u.p, mixed))) return s;
      }
      return enqueue_stats(p);
    }, fr);
    if (!st) {
      cudaGraphExec_t ex = nullptr;
      cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
      else p->g_step->exec = ex;
    }
    cudaGraphDestroy(g);
    if (st) {
      drop(p->g_step);
      return st;
    }
    p->g_step->k_pro = p->launches - l0;
    p->g_step->kind = 2;
    p->g_step->key = key;
  }
  AFC_CUDA(cudaGraphLaunch(p->g_step->exec, p->stream));
  AFC_CUDA(cudaStreamSynchronize(p->stream));
  p->launches += p->g_step->k_pro;
  if (stt) {
    stt->stages = o->scheme == AFC_SSP2 ? 2 : 3;
    stt->umin = p->host_scal[60];
    stt->umax = p->host_scal[61];
    stt->status = AFC_OK;
  }
  return AFC_OK;
}

}  // namespace afc
