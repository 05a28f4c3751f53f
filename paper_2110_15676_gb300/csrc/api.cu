// C ABI of libafc (declared in include/afc.h): problem lifetime, data transfer,
// and the drivers of the hot path (explicit SSP stages, the Crank-Nicolson and
// stationary fixed-point loops of Sec. 4).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "afc_internal.h"
#include "kernels_common.cuh"

namespace afc {

namespace {
thread_local std::string g_error;

template <class T>
int64_t bytes_of(const DBuf<T>& b) {
  return b.base ? (int64_t)((b.n + 2 * b.pad) * sizeof(T)) : 0;
}

__global__ void k_apply_dirichlet(int64_t N, const uint8_t* __restrict__ dir, const double* __restrict__ udir,
                                  double* __restrict__ u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N && dir[i]) u[i] = udir[i];
}

__global__ void k_cfl_ratio(int64_t N, Offsets of, const double* __restrict__ AA, const double* __restrict__ mL,
                            const uint8_t* __restrict__ dir, double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  out[i] = dir[i] ? INFINITY : mL[i] / AA[(int64_t)of.Kup * N + i];
}

int check(afc_problem_s* p, bool need_assembled) {
  if (!p) { set_error("null problem"); return AFC_E_INVALID; }
  if (need_assembled && !p->assembled) { set_error("call afc_assemble first"); return AFC_E_STATE; }
  if (cudaSetDevice(p->device) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  return AFC_OK;
}

int to_device(afc_problem_s* p, double* dst, const double* src, int64_t n) {
  AFC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  return AFC_OK;
}

int to_host(afc_problem_s* p, double* dst, const double* src, int64_t n) {
  if (!dst) return AFC_OK;
  AFC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  return AFC_OK;
}

int sync(afc_problem_s* p) {
  AFC_CUDA(cudaStreamSynchronize(p->stream));
  return AFC_OK;
}

// read one device scalar slot (synchronises the stream)
int read_scal(afc_problem_s* p, int slot, double* out) {
  AFC_CUDA(cudaMemcpyAsync(p->host_scal + slot, p->scal.p + slot, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  AFC_CUDA(cudaStreamSynchronize(p->stream));
  *out = p->host_scal[slot];
  return AFC_OK;
}

int create_common(afc_problem_s* p) {
  const int64_t N = p->N;
  const auto& m = p->mesh;
  p->K = (int)m.offsets.size();
  p->Kup = p->K / 2;
  p->offs.K = p->K;
  p->offs.Kup = p->Kup;
  for (int k = 0; k < p->K; ++k) p->offs.o[k] = m.offsets[k];
  p->pad = std::max(std::abs(m.offsets.front()), std::abs(m.offsets.back()));
  if (p->K % 2 != 1 || m.offsets[p->Kup] != 0) { set_error("offset set is not symmetric"); return AFC_E_INVALID; }
  int st;
  if ((st = p->xyz.alloc(3 * N)) || (st = p->conn.alloc(m.nl * m.ncells)) || (st = p->inc_ptr.alloc(N + 1)) ||
      (st = p->inc.alloc((int64_t)m.inc.size())) || (st = p->mask.alloc(N)) || (st = p->bnod.alloc(3 * N)) ||
      (st = p->fnod.alloc(N)) || (st = p->dir.alloc(N)) || (st = p->udir.alloc(N)))
    return st;
  DBuf<double>* vecs[] = {&p->u,  &p->u0,  &p->ustage, &p->udot, &p->ut,   &p->Rp,  &p->Rm,
                          &p->Fs, &p->Qp,  &p->Qm,     &p->b0,   &p->res,  &p->delta, &p->umax,
                          &p->umin, &p->tmp, &p->cn_a, &p->cn_s, &p->bA, &p->bB, &p->Fold};
  for (auto* v : vecs)
    if ((st = v->alloc(N, p->pad))) return st;
  if ((st = p->scal.alloc(64)) || (st = p->part.alloc(4 * std::max<int64_t>(kRedBlocks, grid_for(N))))) return st;
  if (cudaMallocHost((void**)&p->host_scal, 64 * sizeof(double)) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    return AFC_E_OOM;
  }
  cudaStream_t s = p->stream;
  AFC_CUDA(cudaMemcpyAsync(p->xyz.p, m.xyz.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, s));
  AFC_CUDA(cudaMemcpyAsync(p->conn.p, m.conn.data(), m.conn.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AFC_CUDA(cudaMemcpyAsync(p->inc_ptr.p, m.inc_ptr.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AFC_CUDA(cudaMemcpyAsync(p->inc.p, m.inc.data(), m.inc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  AFC_CUDA(cudaMemcpyAsync(p->mask.p, m.mask.data(), N * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  return sync(p);
}

void destroy_all(afc_problem_s* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  graph_free(p);
  prof_free(p);
  krylov_free(p);
  DBuf<double>* dv[] = {&p->xyz, &p->bnod, &p->fnod, &p->udir, &p->Mfull, &p->Sfull, &p->Kfull, &p->Afull,
                        &p->AA, &p->m_up, &p->d_up, &p->mL, &p->f, &p->Bst, &p->dinv_st, &p->Bcn, &p->dinv_cn,
                        &p->u, &p->u0, &p->ustage, &p->udot, &p->ut, &p->Rp, &p->Rm, &p->Fs, &p->Qp, &p->Qm,
                        &p->b0, &p->res, &p->delta, &p->umax, &p->umin, &p->tmp, &p->cn_a, &p->cn_s,
                        &p->scal, &p->part, &p->r_up, &p->mdt_up, &p->mLdt, &p->kij_up, &p->kji_up,
                        &p->AG, &p->bA, &p->bB, &p->d2_up, &p->Fold, &p->cnod, &p->Rfull, &p->rl};
  for (auto* b : dv) b->free_();
  p->Bst32.free_(); p->dinv_st32.free_(); p->Bcn32.free_(); p->dinv_cn32.free_();
  p->conn.free_(); p->inc_ptr.free_(); p->inc.free_(); p->mask.free_(); p->dir.free_(); p->clip.free_();
  p->pairf.free_(); p->nodef.free_();
  p->AGp.free_(); p->fp2.free_(); p->pk_hi.free_(); p->pk_lo.free_(); p->up2.free_(); p->yp2.free_(); p->abh2.free_(); p->abl2.free_();
  p->cp_up.free_(); p->mask32.free_(); p->clip32.free_(); p->mask16.free_(); p->clip16.free_();
  p->m32_up.free_(); p->d32_up.free_(); p->r32.free_(); p->uf.free_(); p->udf.free_();
  if (p->host_scal) cudaFreeHost(p->host_scal);
  delete p;
}

int finish_stats(afc_problem_s* p, afc_stats* st, int status) {
  if (!st) return status;
  double mn = 0, mx = 0;
  int e = minmax_device(p, p->u.p, &mn, &mx);
  if (e) return e;
  st->umin = mn;
  st->umax = mx;
  st->status = status;
  return status;
}

// Damped fixed point of Sec. 4 in defect form: res = residual(u); stop if
// ||res|| < sqrt(N) tol; solve B delta = res; u += omega delta.
// With `epi`, a persistent BiCGStab applies the update in its last pass and update()
// only runs where the solve did not.
template <class Residual, class Update>
int fixed_point(afc_problem_s* p, const afc_opts* o, int system, afc_stats* st, Residual residual, Update update,
                const KrylovEpilogue* epi = nullptr) {
  const double thresh = std::sqrt((double)p->N) * o->fp_tol;
  int status = AFC_NOT_CONVERGED;
  for (int it = 0;; ++it) {
    int e = residual();
    if (e) return e;
    double r2;
    if ((e = read_scal(p, 0, &r2))) return e;
    const double R = std::sqrt(r2);
    if (!std::isfinite(R)) { set_error("non-finite nonlinear residual"); return AFC_E_NAN; }
    if (st) {
      if (it == 0) st->res0 = R;
      st->res_final = R;
    }
    if (o->fp_fixed_its > 0) {
      if (it == o->fp_fixed_its) { status = AFC_OK; break; }
    } else {
      if (R < thresh) { status = AFC_OK; break; }
      if (it >= o->fp_maxit) break;
    }
    int its = 0;
    double kres = 0;
    bool applied = false;
    e = krylov_solve(p, system, o, p->res.p, p->delta.p, &its, &kres, epi, &applied);
    if (e < 0) return e;
    if (st) {
      st->inner_its += its;
      st->outer_its += 1;
    }
    if (!applied && (e = update())) return e;
  }
  return status;
}

}  // namespace

void set_error(const std::string& msg) { g_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  g_error = std::string(what) + ": " + cudaGetErrorString(e);
  return AFC_E_CUDA;
}

}  // namespace afc

using namespace afc;

extern "C" {

const char* afc_last_error(void) { return g_error.c_str(); }

const char* afc_status_str(int s) {
  switch (s) {
    case AFC_OK: return "ok";
    case AFC_NOT_CONVERGED: return "not converged (last iterate returned)";
    case AFC_E_INVALID: return "invalid argument";
    case AFC_E_OOM: return "out of device memory";
    case AFC_E_CUDA: return "CUDA error";
    case AFC_E_NAN: return "NaN or Inf encountered";
    case AFC_E_TIMEOUT: return "bounded device wait expired";
    case AFC_E_STATE: return "call out of order";
    default: return "unknown status";
  }
}

void afc_default_opts(afc_opts* o) {
  if (!o) return;
  o->scheme = AFC_SSP3;
  o->limiter = AFC_LIM_ZALESAK;
  o->dt = 0.0;
  o->fp_tol = 1e-10;
  o->fp_maxit = 100;
  o->fp_fixed_its = 0;
  o->omega = 1.0;
  o->ksp = AFC_KSP_BICGSTAB;
  o->ksp_maxit = 1000;
  o->ksp_atol = 1e-12;
  o->ksp_rtol = 0.0;
  o->gmres_restart = 20;
  o->precision = AFC_FP64;
  o->prelimit = 1;
  o->graph = 1;
}

static int create_with(afc_problem_s* p, int /*device*/, void* /*stream*/, afc_problem* out) {
  int st = create_common(p);
  if (st) { destroy_all(p); return st; }
  *out = p;
  return AFC_OK;
}

int afc_create_structured(int elem, int nx, int ny, int nz, const double lo[3], const double hi[3], int device,
                          void* stream, afc_problem* out) {
  if (!out || !lo || !hi) { set_error("null argument"); return AFC_E_INVALID; }
  *out = nullptr;
  afc_problem_s* p = new afc_problem_s();
  p->device = device;
  p->stream = (cudaStream_t)stream;
  int st = build_structured(elem, nx, ny, nz, lo, hi, p->mesh);   // host-only validation first
  if (st) { delete p; return st; }
  p->N = p->mesh.N;
  if (cudaSetDevice(device) != cudaSuccess) { delete p; return cuda_fail(cudaGetLastError(), "cudaSetDevice"); }
  return create_with(p, device, stream, out);
}

int afc_create_from_elements(int elem, int64_t n_nodes, const double* xyz, int64_t n_cells, const int32_t* conn,
                             int device, void* stream, afc_problem* out) {
  if (!out) { set_error("null argument"); return AFC_E_INVALID; }
  *out = nullptr;
  afc_problem_s* p = new afc_problem_s();
  p->device = device;
  p->stream = (cudaStream_t)stream;
  int st = build_from_elements(elem, n_nodes, xyz, n_cells, conn, p->mesh);   // host-only validation first
  if (st) { delete p; return st; }
  p->N = p->mesh.N;
  if (cudaSetDevice(device) != cudaSuccess) { delete p; return cuda_fail(cudaGetLastError(), "cudaSetDevice"); }
  return create_with(p, device, stream, out);
}

int afc_destroy(afc_problem p) {
  if (!p) return AFC_OK;
  destroy_all(p);
  return AFC_OK;
}

int afc_set_coefficients(afc_problem p, double eps, const double* b_nodal, const double b_const[3],
                         const double* c_nodal, double c_const, const double* f_nodal) {
  int st = check(p, false);
  if (st) return st;
  if ((!b_nodal && !b_const) || !(eps >= 0.0) || !std::isfinite(eps) ||
      (!c_nodal && (!(c_const >= 0.0) || !std::isfinite(c_const)))) {
    set_error("need b_nodal or b_const, eps >= 0 and c_const >= 0 (or c_nodal)");
    return AFC_E_INVALID;
  }
  if (c_nodal)
    for (int64_t i = 0; i < p->N; ++i)
      if (!(c_nodal[i] >= 0.0) || !std::isfinite(c_nodal[i])) {
        set_error("c_nodal must be finite and >= 0 at every node");
        return AFC_E_INVALID;
      }
  std::vector<double> bc;
  if (!b_nodal) {   // a constant velocity at every node
    bc.resize(3 * p->N);
    for (int64_t i = 0; i < p->N; ++i)
      for (int d = 0; d < 3; ++d) bc[3 * i + d] = b_const[d];
    b_nodal = bc.data();
  }
  p->eps = eps;
  p->c = c_nodal ? 0.0 : c_const;
  p->c_nodal = c_nodal != nullptr;
  if (c_nodal) {
    if ((st = p->cnod.alloc(p->N))) return st;
    if ((st = to_device(p, p->cnod.p, c_nodal, p->N))) return st;
  }
  if ((st = to_device(p, p->bnod.p, b_nodal, 3 * p->N))) return st;
  if (f_nodal) {
    if ((st = to_device(p, p->fnod.p, f_nodal, p->N))) return st;
  } else {
    AFC_CUDA(cudaMemsetAsync(p->fnod.p, 0, p->N * sizeof(double), p->stream));
  }
  p->coef_set = true;
  p->assembled = false;
  return sync(p);
}

int afc_set_dirichlet(afc_problem p, const uint8_t* mask, const double* values) {
  int st = check(p, false);
  if (st) return st;
  if (!mask || !values) { set_error("need mask and values"); return AFC_E_INVALID; }
  std::vector<uint8_t> m(mask, mask + p->N);
  for (auto& v : m) v = v ? 1 : 0;
  p->dir_lo = 1e308;
  p->dir_hi = -1e308;
  for (int64_t i = 0; i < p->N; ++i)
    if (m[i]) {
      p->dir_lo = std::min(p->dir_lo, values[i]);
      p->dir_hi = std::max(p->dir_hi, values[i]);
    }
  AFC_CUDA(cudaMemcpyAsync(p->dir.p, m.data(), p->N, cudaMemcpyHostToDevice, p->stream));
  if ((st = to_device(p, p->udir.p, values, p->N))) return st;
  if ((st = sync(p))) return st;
  if (p->assembled) return assemble_device(p, p->family, p->precision);   // system rows depend on the set
  return AFC_OK;
}

int afc_assemble(afc_problem p, int family, int precision) {
  int st = check(p, false);
  if (st) return st;
  if (!p->coef_set) { set_error("call afc_set_coefficients first"); return AFC_E_STATE; }
  if ((family != AFC_FAMILY_FCT && family != AFC_FAMILY_MC) || (precision != AFC_FP64 && precision != AFC_MIXED)) {
    set_error("bad family or precision");
    return AFC_E_INVALID;
  }
  return assemble_device(p, family, precision);
}

int afc_get_info(afc_problem p, afc_info* out) {
  int st = check(p, false);
  if (st) return st;
  if (!out) { set_error("null argument"); return AFC_E_INVALID; }
  out->n_nodes = p->N;
  out->nnz = p->mesh.nnz;
  out->n_edges = p->mesh.n_edges;
  out->n_offsets = p->K;
  out->max_offset = p->pad;
  int64_t b = 0;
  b += bytes_of(p->xyz) + bytes_of(p->conn) + bytes_of(p->inc_ptr) + bytes_of(p->inc) + bytes_of(p->mask);
  b += bytes_of(p->bnod) + bytes_of(p->fnod) + bytes_of(p->dir) + bytes_of(p->udir);
  b += bytes_of(p->Mfull) + bytes_of(p->Sfull) + bytes_of(p->Kfull) + bytes_of(p->Afull) + bytes_of(p->AA);
  b += bytes_of(p->m_up) + bytes_of(p->d_up) + bytes_of(p->mL) + bytes_of(p->f) + bytes_of(p->Bst) +
       bytes_of(p->Bst32) + bytes_of(p->Bcn) + bytes_of(p->Bcn32);
  b += 16 * bytes_of(p->u);
  out->device_bytes = b;
  out->assembled = p->assembled ? 1 : 0;
  out->family = p->family;
  return AFC_OK;
}

int afc_export_csr(afc_problem p, int which, int32_t* rowptr, int32_t* col, double* val) {
  int st = check(p, true);
  if (st) return st;
  if (!rowptr || !col || !val) { set_error("null argument"); return AFC_E_INVALID; }
  const int64_t N = p->N;
  const int K = p->K, Kup = p->Kup;
  std::vector<double> full((size_t)K * N, 0.0);
  const double* src = nullptr;
  switch (which) {
    case AFC_MAT_MC: src = p->Mfull.p; break;
    case AFC_MAT_A: src = p->Afull.p; break;
    case AFC_MAT_LOW: src = p->AA.p; break;
    case AFC_MAT_K: src = p->Kfull.p; break;
    case AFC_MAT_S: src = p->Sfull.p; break;
    case AFC_MAT_D: break;
    default: set_error("unknown matrix"); return AFC_E_INVALID;
  }
  if (src) {
    AFC_CUDA(cudaMemcpyAsync(full.data(), src, full.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  } else {
    std::vector<double> dup((size_t)Kup * N);
    AFC_CUDA(cudaMemcpyAsync(dup.data(), p->d_up.p, dup.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    if ((st = sync(p))) return st;
    const auto& mask = p->mesh.mask;
    for (int64_t i = 0; i < N; ++i) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) {
        if (k == Kup || !((mask[i] >> k) & 1ull)) continue;
        double d = k > Kup ? dup[(size_t)(k - Kup - 1) * N + i] : dup[(size_t)(Kup - 1 - k) * N + i + p->offs.o[k]];
        full[(size_t)k * N + i] = d;
        s += d;
      }
      full[(size_t)Kup * N + i] = -s;
    }
  }
  if ((st = sync(p))) return st;
  int64_t q = 0;
  rowptr[0] = 0;
  const auto& mask = p->mesh.mask;
  for (int64_t i = 0; i < N; ++i) {
    for (int k = 0; k < K; ++k) {
      if (!((mask[i] >> k) & 1ull)) continue;
      col[q] = (int32_t)(i + p->offs.o[k]);
      val[q] = full[(size_t)k * N + i];
      ++q;
    }
    rowptr[i + 1] = (int32_t)q;
  }
  return AFC_OK;
}

int afc_export_lumped_mass(afc_problem p, double* mL) {
  int st = check(p, true);
  if (st) return st;
  if ((st = to_host(p, mL, p->mL.p, p->N))) return st;
  return sync(p);
}

int afc_set_solution(afc_problem p, const double* u, int is_device) {
  int st = check(p, false);
  if (st) return st;
  if (!u) { set_error("null argument"); return AFC_E_INVALID; }
  AFC_CUDA(cudaMemcpyAsync(p->u.p, u, p->N * sizeof(double),
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
  p->u_range_valid = false;   // measured on the device by the next step or solve
  return sync(p);
}

int afc_get_solution(afc_problem p, double* u, int is_device) {
  int st = check(p, false);
  if (st) return st;
  if (!u) { set_error("null argument"); return AFC_E_INVALID; }
  AFC_CUDA(cudaMemcpyAsync(u, p->u.p, p->N * sizeof(double),
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
  return sync(p);
}

int afc_cfl_timestep(afc_problem p, double cfl, double* dt) {
  int st = check(p, true);
  if (st) return st;
  if (!dt || !(cfl > 0.0)) { set_error("need cfl > 0"); return AFC_E_INVALID; }
  AFC_LAUNCH(p, "k_cfl_ratio", k_cfl_ratio<<<grid_for(p->N), kBlock, 0, p->stream>>>(p->N, p->offs, p->AA.p, p->mL.p, p->dir.p, p->tmp.p));
  AFC_CUDA(cudaGetLastError());
  double mn, mx;
  if ((st = minmax_device(p, p->tmp.p, &mn, &mx))) return st;
  if (!std::isfinite(mn)) { set_error("no free nodes"); return AFC_E_INVALID; }
  *dt = cfl * mn;
  return AFC_OK;
}

namespace {
int step_impl(afc_problem p, const afc_opts* o, afc_stats* stt) {
  int st = check(p, true);
  if (st) return st;
  if (!o || !(o->dt > 0.0)) { set_error("need options with dt > 0"); return AFC_E_INVALID; }
  if (stt) std::memset(stt, 0, sizeof(*stt));
  const int64_t N = p->N;
  const int lim = o->limiter;
  const bool ssp = o->scheme == AFC_SSP2 || o->scheme == AFC_SSP3;
  if (lim == AFC_LIM_MC && (ssp || o->scheme == AFC_CN_NONLINEAR)) {
    // transient MC (Sec. 2.2): the SSP schemes (FP64) or nonlinear CN with the MC limiter
    if (p->family != AFC_FAMILY_MC) { set_error("transient MC needs the MC family assembly"); return AFC_E_STATE; }
    if (ssp && o->precision != AFC_FP64) { set_error("transient MC with SSP runs in FP64 only"); return AFC_E_INVALID; }
  } else if (lim != AFC_LIM_NONE && lim != AFC_LIM_GALERKIN && lim != AFC_LIM_ZALESAK) {
    set_error("afc_step supports limiters NONE, GALERKIN, ZALESAK (and MC with SSP2, SSP3, CN_NONLINEAR)");
    return AFC_E_INVALID;
  }
  const int cn_family = lim == AFC_LIM_MC ? AFC_FAMILY_MC : AFC_FAMILY_FCT;
  cudaStream_t s = p->stream;
  const bool mixed = o->precision == AFC_MIXED;
  const bool graph = o->graph != 0;   // captured on a private stream, launched on the problem's stream
  if (graph && (o->scheme == AFC_SSP2 || o->scheme == AFC_SSP3)) return ssp_step_graph(p, o, stt);
  // linear Zal+CN: one undamped correction from 2 u~ - u_old solves its linear system
  afc_opts olin;
  if (o->scheme == AFC_CN_LINEAR) {
    olin = *o;
    olin.fp_fixed_its = 1;
    olin.omega = 1.0;
    o = &olin;
  }
  const bool cn = o->scheme == AFC_CN_NONLINEAR || o->scheme == AFC_CN_LINEAR;
  if (graph && cn) {
    if (p->family != cn_family) { set_error("CN FCT needs the FCT family"); return AFC_E_STATE; }
    if ((st = build_cn_system(p, o->dt))) return st;
    return cn_step_graph(p, o, stt);
  }
  AFC_CUDA(cudaMemcpyAsync(p->u0.p, p->u.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (o->scheme == AFC_SSP2) {
    if ((st = fe_stage(p, p->u0.p, o->dt, lim, 0.0, nullptr, 1.0, p->ustage.p, mixed))) return st;
    if ((st = fe_stage(p, p->ustage.p, o->dt, lim, 0.5, p->u0.p, 0.5, p->u.p, mixed))) return st;
    if (stt) stt->stages = 2;
    return finish_stats(p, stt, AFC_OK);
  }
  if (o->scheme == AFC_SSP3) {
    if ((st = fe_stage(p, p->u0.p, o->dt, lim, 0.0, nullptr, 1.0, p->ustage.p, mixed))) return st;
    if ((st = fe_stage(p, p->ustage.p, o->dt, lim, 0.75, p->u0.p, 0.25, p->tmp.p, mixed))) return st;
    if ((st = fe_stage(p, p->tmp.p, o->dt, lim, 1.0 / 3.0, p->u0.p, 2.0 / 3.0, p->u.p, mixed))) return st;
    if (stt) stt->stages = 3;
    return finish_stats(p, stt, AFC_OK);
  }
  if (!cn) { set_error("unknown scheme"); return AFC_E_INVALID; }
  if (p->family != cn_family) { set_error("CN FCT needs the FCT family"); return AFC_E_STATE; }
  if ((st = build_cn_system(p, o->dt))) return st;
  if ((st = cn_predictor(p, p->u0.p, o->dt))) return st;
  if (lim == AFC_LIM_MC) {
    // CN with the MC limiter: F* = (F*(u) + F*(u_old)) / 2, plain damped updates
    AFC_LAUNCH(p, "k_apply_dirichlet", k_apply_dirichlet<<<grid_for(N), kBlock, 0, s>>>(N, p->dir.p, p->udir.p, p->u.p));
    AFC_CUDA(cudaGetLastError());
    if ((st = mc_cn_old_flux(p, p->u0.p))) return st;
    st = fixed_point(
        p, o, 1, stt, [&]() { return mc_cn_residual(p, p->u.p, p->res.p, p->scal.p); },
        [&]() { return axpy_device(p, o->omega, p->delta.p, p->u.p); });
    if (st < 0) return st;
    return finish_stats(p, stt, st);
  }
  if (o->scheme == AFC_CN_LINEAR) {
    if ((st = cn_linear_guess(p, p->u0.p, p->u.p))) return st;
  } else {
    AFC_LAUNCH(p, "k_apply_dirichlet", k_apply_dirichlet<<<grid_for(N), kBlock, 0, s>>>(N, p->dir.p, p->udir.p, p->u.p));
    AFC_CUDA(cudaGetLastError());
  }
  if ((st = cn_update(p, 0.0, nullptr, p->u.p, p->u0.p))) return st;
  const double dt = o->dt;
  KrylovEpilogue epi;
  epi.omega = o->omega;
  epi.u = p->u.p;
  epi.uo = p->u0.p;
  epi.a = p->cn_a.p;
  epi.s = p->cn_s.p;
  st = fixed_point(
      p, o, 1, stt, [&]() { return cn_limited_residual(p, p->u.p, dt, lim, o->prelimit, p->res.p, p->scal.p); },
      [&]() { return cn_update(p, o->omega, p->delta.p, p->u.p, p->u0.p); }, &epi);
  if (st < 0) return st;
  return finish_stats(p, stt, st);
}

int stationary_impl(afc_problem p, const afc_opts* o, afc_stats* stt) {
  int st = check(p, true);
  if (st) return st;
  if (!o) { set_error("null options"); return AFC_E_INVALID; }
  if (stt) std::memset(stt, 0, sizeof(*stt));
  const int lim = o->limiter;
  if (lim != AFC_LIM_NONE && lim != AFC_LIM_GALERKIN && lim != AFC_LIM_MC && lim != AFC_LIM_MU) {
    set_error("afc_solve_stationary supports limiters NONE, GALERKIN, MC, MU");
    return AFC_E_INVALID;
  }
  if (lim != AFC_LIM_NONE && p->family != AFC_FAMILY_MC) {
    set_error("the stationary MC limiter and its Galerkin mode need the MC family");
    return AFC_E_STATE;
  }
  if (o->graph != 0) return stationary_graph(p, o, stt);
  AFC_LAUNCH(p, "k_apply_dirichlet", k_apply_dirichlet<<<grid_for(p->N), kBlock, 0, p->stream>>>(p->N, p->dir.p, p->udir.p, p->u.p));
  AFC_CUDA(cudaGetLastError());
  st = fixed_point(
      p, o, 0, stt, [&]() {
        return mc_limited_residual(p, p->u.p, lim, p->res.p, p->scal.p, false, o->precision == AFC_MIXED);
      },
      [&]() { return axpy_device(p, o->omega, p->delta.p, p->u.p); });
  if (st < 0) return st;
  return finish_stats(p, stt, st);
}

// Range of the stored solution before a call (computed on the device only when no
// earlier call left it known).
int input_range(afc_problem_s* p, double* lo, double* hi) {
  if (!p->u_range_valid) {
    int st = minmax_device(p, p->u.p, &p->u_lo, &p->u_hi);
    if (st) return st;
    p->u_range_valid = true;
  }
  *lo = std::min(p->u_lo, p->dir_lo);
  *hi = std::max(p->u_hi, p->dir_hi);
  return AFC_OK;
}

// dmp_violation and t_ms of a step or solve; the returned solution's range becomes the
// next call's input range (not after an error: the state may then not be an iterate)
int finish_call(afc_problem_s* p, afc_stats* stt, int status, double lo, double hi,
                std::chrono::steady_clock::time_point t0) {
  if (status < 0) {
    p->u_range_valid = false;
    return status;
  }
  stt->dmp_violation = std::max(0.0, std::max(lo - stt->umin, stt->umax - hi));
  stt->t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  p->u_lo = stt->umin;
  p->u_hi = stt->umax;
  p->u_range_valid = true;
  return status;
}
}  // namespace

int afc_step(afc_problem p, const afc_opts* o, afc_stats* stt) {
  const auto t0 = std::chrono::steady_clock::now();
  int st = check(p, true);
  if (st) return st;
  double lo, hi;
  if ((st = input_range(p, &lo, &hi))) return st;
  afc_stats local;
  afc_stats* s = stt ? stt : &local;
  return finish_call(p, s, step_impl(p, o, s), lo, hi, t0);
}

int afc_solve_stationary(afc_problem p, const afc_opts* o, afc_stats* stt) {
  const auto t0 = std::chrono::steady_clock::now();
  int st = check(p, true);
  if (st) return st;
  double lo, hi;
  if ((st = input_range(p, &lo, &hi))) return st;
  afc_stats local;
  afc_stats* s = stt ? stt : &local;
  return finish_call(p, s, stationary_impl(p, o, s), lo, hi, t0);
}

int afc_fe_stage(afc_problem p, double dt, int limiter, double* u_tilde, double* Rp, double* Rm, double* Fstar,
                 double* u_new) {
  int st = check(p, true);
  if (st) return st;
  if (!(dt > 0.0)) { set_error("need dt > 0"); return AFC_E_INVALID; }
  if ((st = fe_stage(p, p->u.p, dt, limiter, 0.0, nullptr, 1.0, p->tmp.p))) return st;
  if ((st = to_host(p, u_tilde, p->ut.p, p->N)) || (st = to_host(p, Rp, p->Rp.p, p->N)) ||
      (st = to_host(p, Rm, p->Rm.p, p->N)) || (st = to_host(p, Fstar, p->Fs.p, p->N)) ||
      (st = to_host(p, u_new, p->tmp.p, p->N)))
    return st;
  return sync(p);
}

int afc_cn_limited_sum(afc_problem p, double dt, int limiter, int prelimit, const double* u_new, const double* u_old,
                       double* u_tilde, double* Rp, double* Rm, double* Fstar) {
  int st = check(p, true);
  if (st) return st;
  if (!(dt > 0.0) || !u_new || !u_old) { set_error("need dt > 0, u_new, u_old"); return AFC_E_INVALID; }
  if ((st = to_device(p, p->ustage.p, u_new, p->N)) || (st = to_device(p, p->u0.p, u_old, p->N))) return st;
  if ((st = build_cn_system(p, dt))) return st;
  if ((st = cn_predictor(p, p->u0.p, dt))) return st;
  if ((st = cn_update(p, 0.0, nullptr, p->ustage.p, p->u0.p))) return st;
  if ((st = cn_limited_residual(p, p->ustage.p, dt, limiter, prelimit, p->res.p, p->scal.p))) return st;
  if ((st = to_host(p, u_tilde, p->ut.p, p->N)) || (st = to_host(p, Rp, p->Rp.p, p->N)) ||
      (st = to_host(p, Rm, p->Rm.p, p->N)) || (st = to_host(p, Fstar, p->Fs.p, p->N)))
    return st;
  return sync(p);
}

int afc_mc_limited_sum(afc_problem p, int limiter, const double* u, double* umax, double* umin, double* Fstar) {
  int st = check(p, true);
  if (st) return st;
  if (!u) { set_error("null argument"); return AFC_E_INVALID; }
  if ((st = to_device(p, p->ustage.p, u, p->N))) return st;
  if (limiter != AFC_LIM_NONE && limiter != AFC_LIM_GALERKIN && limiter != AFC_LIM_MC && limiter != AFC_LIM_MU) {
    set_error("limiter must be NONE, GALERKIN, MC or MU");
    return AFC_E_INVALID;
  }
  if (p->family != AFC_FAMILY_MC && limiter != AFC_LIM_NONE) {
    set_error("the MC limiter and its Galerkin mode need afc_assemble(..., AFC_FAMILY_MC, ...)");
    return AFC_E_STATE;
  }
  if ((st = mc_limited_residual(p, p->ustage.p, limiter, p->res.p, p->scal.p, true))) return st;
  if ((st = to_host(p, umax, p->umax.p, p->N)) || (st = to_host(p, umin, p->umin.p, p->N)) ||
      (st = to_host(p, Fstar, p->Fs.p, p->N)))
    return st;
  return sync(p);
}

int afc_mc_residual_sweep(afc_problem p, int limiter) {
  int st = check(p, true);
  if (st) return st;
  if (limiter != AFC_LIM_NONE && limiter != AFC_LIM_GALERKIN && limiter != AFC_LIM_MC && limiter != AFC_LIM_MU) {
    set_error("limiter must be NONE, GALERKIN, MC or MU");
    return AFC_E_INVALID;
  }
  if (p->family != AFC_FAMILY_MC && limiter != AFC_LIM_NONE) { set_error("needs the MC family"); return AFC_E_STATE; }
  return mc_limited_residual(p, p->u.p, limiter, p->res.p, p->scal.p, false, true);
}

int afc_get_residual(afc_problem p, double* res) {
  int st = check(p, true);
  if (st) return st;
  if (!res) { set_error("null argument"); return AFC_E_INVALID; }
  if ((st = to_host(p, res, p->res.p, p->N))) return st;
  return sync(p);
}

int afc_apply(afc_problem p, int which, const double* x, double* y) {
  int st = check(p, true);
  if (st) return st;
  if (!x || !y) { set_error("null argument"); return AFC_E_INVALID; }
  const double* A = which == AFC_MAT_LOW ? p->AA.p : which == AFC_MAT_MC ? p->Mfull.p : nullptr;
  if (!A) { set_error("afc_apply supports AFC_MAT_LOW and AFC_MAT_MC"); return AFC_E_INVALID; }
  if ((st = to_device(p, p->ustage.p, x, p->N))) return st;
  if ((st = dia_spmv(p, A, p->ustage.p, p->tmp.p))) return st;
  if ((st = to_host(p, y, p->tmp.p, p->N))) return st;
  return sync(p);
}

int afc_linear_solve(afc_problem p, int system, double dt, const afc_opts* o, const double* rhs, double* x, int* its,
                     double* res) {
  int st = check(p, true);
  if (st) return st;
  if (!o || !rhs || !x || (system != 0 && system != 1)) { set_error("bad arguments"); return AFC_E_INVALID; }
  if (system == 1) {
    if (!(dt > 0.0)) { set_error("need dt > 0"); return AFC_E_INVALID; }
    if ((st = build_cn_system(p, dt))) return st;
  }
  if ((st = to_device(p, p->res.p, rhs, p->N))) return st;
  int status = krylov_solve(p, system, o, p->res.p, p->delta.p, its, res);
  if (status < 0) return status;
  if ((st = to_host(p, x, p->delta.p, p->N))) return st;
  if ((st = sync(p))) return st;
  return status;
}

int afc_set_grid_wait_limit(afc_problem p, double limit_ms) {
  int st = check(p, false);
  if (st) return st;
  if (!(limit_ms >= 0.0 && limit_ms <= 4000.0)) {
    set_error("afc_set_grid_wait_limit: need 0 <= limit_ms <= 4000");
    return AFC_E_INVALID;
  }
  p->grid_wait_ns = (unsigned long long)(limit_ms * 1e6);
  return AFC_OK;
}

}  // extern "C"
