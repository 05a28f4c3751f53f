// Batches of independent problems: the explicit FE-SSP step (Sec. 2.1.2 with
// Zalesak's limiter, Sec. 2.1.3) of many instances of different sizes at once.
//
// Work list.  The rows of every instance are cut into tiles of `block` rows
// (one row per thread); the instance table holds each instance's first tile, so
// tile t belongs to the instance whose range contains it.  Each pass (rate,
// edges, factors, correct) walks all tiles of all instances, so a pass over 256
// small instances is one launch that fills the GPU instead of 256 launches that
// each fill a few SMs.
//
// Launch shapes.  PER_PASS: one ordinary launch per pass, one tile per block.
// PER_STAGE / PER_STEP: one persistent cooperative launch per stage / per time
// step; each block takes a contiguous range of tiles (neighbouring rows, few
// instance switches) and the passes are separated by a grid-wide barrier.  The
// barrier wait is bounded (a few seconds of the global timer): on expiry the
// block records an error that the host reports as AFC_E_TIMEOUT, and every later
// barrier of the launch passes at once, so a launch always ends.  Cooperative
// launch guarantees that all blocks are resident, so the bound is a safety net.
//
// Each time step is captured once as a CUDA graph and replayed.  An instance's
// arithmetic is the one of the single-problem kernels (ssp_rows.cuh), so its
// result does not depend on the batch, the tile size or the launch shape.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "afc_internal.h"
#include "kernels_common.cuh"
#include "ssp_rows.cuh"
#include "grid_sync.cuh"

namespace afc {
namespace {

struct __align__(16) BInst {
  Offsets of;
  SspArrays a;
  double* vec[3];       // stored solution u, stage vectors ustage and tmp
  double dt;
  int64_t tile0;        // first tile of the instance
  int64_t ntiles;
};
static_assert(sizeof(BInst) % 4 == 0, "BInst is copied as 32-bit words");

// up to three stages in one launch: out = ca * vec[uA] + cb * FE(vec[in])
struct StageArgs {
  int nst;
  int in[3], uA[3], out[3];
  double ca[3], cb[3];
};

template <int KT, bool MIXED>
__device__ __forceinline__ void batch_row(const BInst& in, int phase, int st, const StageArgs& sa, int limiter,
                                          int64_t i) {
  const double dt = in.dt;
  switch (phase) {
    case 0:
      ssp_rate_row<KT, MIXED>(in.of, in.a, i, in.vec[sa.in[st]], dt);
      break;
    case 1:
      ssp_edges_row<KT, MIXED>(in.of, in.a, i, in.vec[sa.in[st]]);
      break;
    case 2:
      ssp_factors_row<KT, MIXED>(in.of, in.a, i, dt);
      break;
    default: {
      const double* uA = sa.uA[st] >= 0 ? in.vec[sa.uA[st]] : nullptr;
      ssp_correct_row<KT, MIXED>(in.of, in.a, i, limiter, dt, sa.ca[st], uA, sa.cb[st], in.vec[sa.out[st]]);
    }
  }
}

// One pass over the tiles [t0, t1).  `sh` caches the table entry of the current
// instance; sh_lo / sh_hi is its tile range (empty at the start).
template <bool MIXED>
__device__ void batch_pass(const BInst* __restrict__ tab, int ninst, int64_t t0, int64_t t1, int phase, int st,
                           const StageArgs& sa, int limiter, BInst& sh, int64_t& sh_lo, int64_t& sh_hi) {
  __shared__ int sh_idx;
  for (int64_t t = t0; t < t1; ++t) {
    if (t < sh_lo || t >= sh_hi) {
      __syncthreads();   // everyone is done with the previous entry
      if (threadIdx.x == 0) {
        int lo = 0, hi = ninst - 1;   // last instance with tile0 <= t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (tab[mid].tile0 <= t) lo = mid;
          else hi = mid - 1;
        }
        sh_idx = lo;
      }
      __syncthreads();
      const unsigned int* src = reinterpret_cast<const unsigned int*>(tab + sh_idx);
      unsigned int* dst = reinterpret_cast<unsigned int*>(&sh);
      for (int w = threadIdx.x; w < (int)(sizeof(BInst) / 4); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) {
        sh_lo = sh.tile0;
        sh_hi = sh.tile0 + sh.ntiles;
      }
      __syncthreads();
    }
    const int64_t i = (t - sh_lo) * (int64_t)blockDim.x + threadIdx.x;
    if (i < sh.a.N) {
      const int K = sh.of.K;
      if (K == 27) batch_row<27, MIXED>(sh, phase, st, sa, limiter, i);
      else if (K == 15) batch_row<15, MIXED>(sh, phase, st, sa, limiter, i);
      else batch_row<0, MIXED>(sh, phase, st, sa, limiter, i);
    }
  }
}

__device__ __forceinline__ bool pass_needed(int phase, int limiter) {
  if (phase == 1) return limiter != AFC_LIM_NONE;
  if (phase == 2) return limiter == AFC_LIM_ZALESAK;
  return true;
}

// Passes ph_lo..ph_hi of the stages in `sa`, over all tiles.  With a barrier
// (persistent launches) block b takes the contiguous tile range b; without one
// (ph_lo == ph_hi, one stage) the grid has a block per tile.
template <bool MIXED>
__global__ void __launch_bounds__(512) k_batch_ssp(const BInst* __restrict__ tab, int ninst, int64_t ntiles,
                                                  StageArgs sa, int limiter, int ph_lo, int ph_hi, GridBar* bar) {
  __shared__ BInst sh;
  __shared__ int64_t sh_lo, sh_hi;
  if (threadIdx.x == 0) {
    sh_lo = 0;
    sh_hi = 0;
  }
  __syncthreads();
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t t0 = ntiles * b / G, t1 = ntiles * (b + 1) / G;
  bool first = true;
  for (int st = 0; st < sa.nst; ++st) {
    for (int ph = ph_lo; ph <= ph_hi; ++ph) {
      if (!pass_needed(ph, limiter)) continue;
      if (!first) grid_barrier(bar);
      first = false;
      batch_pass<MIXED>(tab, ninst, t0, t1, ph, st, sa, limiter, sh, sh_lo, sh_hi);
    }
  }
}

// per instance: min and max of the stored solution
__global__ void k_batch_minmax(const BInst* __restrict__ tab, double* __restrict__ out) {
  const BInst& in = tab[blockIdx.x];
  const double* u = in.vec[0];
  long long kmx = LLONG_MIN, kmn = LLONG_MAX;
  for (int64_t i = threadIdx.x; i < in.a.N; i += blockDim.x) {
    const long long k = dkey(u[i]);
    kmx = k > kmx ? k : kmx;
    kmn = k < kmn ? k : kmn;
  }
  __shared__ long long smx[32], smn[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long a = __shfl_xor_sync(0xffffffffu, kmx, o), c = __shfl_xor_sync(0xffffffffu, kmn, o);
    kmx = a > kmx ? a : kmx;
    kmn = c < kmn ? c : kmn;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    smx[w] = kmx;
    smn[w] = kmn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      kmx = smx[q] > kmx ? smx[q] : kmx;
      kmn = smn[q] < kmn ? smn[q] : kmn;
    }
    out[2 * blockIdx.x] = from_key(kmn);
    out[2 * blockIdx.x + 1] = from_key(kmx);
  }
}

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;   // null: enqueue the step's launches directly
  int launches = 0;                 // kernels per step
  int grid = 0;                     // persistent launches: blocks
};

std::mutex g_tune_mutex;
std::map<std::string, afc_batch_tuning> g_tune_cache;   // size class -> fastest launch shape

}  // namespace
}  // namespace afc

struct afc_batch_s {
  std::vector<afc_problem_s*> list;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int nsm = 0;
  int64_t total_nodes = 0;
  afc::BInst* tab_h = nullptr;          // pinned
  afc::BInst* tab_d = nullptr;
  int tab_block = 0;                    // rows per tile the table was built for
  std::vector<double> tab_dt;           // time steps in the table
  int64_t ntiles = 0;
  afc::GridBar* bar = nullptr;
  double* mm_d = nullptr;               // 2 * count min/max
  double* mm_h = nullptr;               // pinned: 2 * count + bar error
  afc_batch_tuning tuning{};
  bool fixed = false;                   // tuning set explicitly or by afc_batch_tune
  std::map<std::string, afc::GraphEntry> graphs;
  int64_t launches = 0;
  double* backup = nullptr;             // saved solutions during tuning
};

namespace afc {
namespace {

std::string size_class(afc_batch_s* b, const afc_opts* o) {
  bool p1 = false, q1 = false, other = false;
  for (auto* p : b->list) {
    if (p->K == 15) p1 = true;
    else if (p->K == 27) q1 = true;
    else other = true;
  }
  const int lt = (int)std::floor(std::log2((double)std::max<int64_t>(b->total_nodes, 1)));
  const int lm = (int)std::floor(std::log2((double)std::max<int64_t>(b->total_nodes / (int64_t)b->list.size(), 1)));
  char buf[128];
  std::snprintf(buf, sizeof buf, "%d%d%d/%d/%d/%d/%d/%d", (int)p1, (int)q1, (int)other, lt, lm, o->precision,
                o->limiter, o->scheme);
  return buf;
}

int max_blocks_per_sm(bool mixed, int block, int* out) {
  int nb = 0;
  cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_ssp<true>, block, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_ssp<false>, block, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  *out = nb;
  return AFC_OK;
}

int valid_tuning(const afc_batch_tuning& t) {
  if (t.mode < AFC_BATCH_PER_PASS || t.mode > AFC_BATCH_PER_STEP || (t.block != 128 && t.block != 256 &&
                                                                      t.block != 512) ||
      t.blocks_per_sm < 0) {
    set_error("batch tuning: mode PER_PASS/PER_STAGE/PER_STEP, block 128/256/512, blocks_per_sm >= 0");
    return AFC_E_INVALID;
  }
  return AFC_OK;
}

afc_batch_tuning effective_tuning(afc_batch_s* b, const afc_opts* o) {
  if (b->fixed) return b->tuning;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find(size_class(b, o));
    if (it != g_tune_cache.end()) return it->second;
  }
  afc_batch_tuning t{};
  t.mode = AFC_BATCH_PER_STAGE;
  t.block = 256;
  t.blocks_per_sm = 0;
  return t;
}

// Instance table for `block` rows per tile and the given time steps (host + device).
int build_table(afc_batch_s* b, int block, const double* dt, double dt_all, bool mixed) {
  const size_t n = b->list.size();
  std::vector<double> dts(n);
  for (size_t q = 0; q < n; ++q) dts[q] = dt ? dt[q] : dt_all;
  if (mixed)
    for (auto* p : b->list) {
      // the single-precision copies are made on the instance's own stream: wait for
      // them there before the batch's stream reads them
      const bool ready = p->ssp32_ready;
      int st = ensure_ssp_mixed(p);   // no-op once the copies match the assembly
      if (st) return st;
      if (!ready && p->stream != b->stream) AFC_CUDA(cudaStreamSynchronize(p->stream));
    }
  if (b->tab_block == block && b->tab_dt == dts) return AFC_OK;
  // the previous upload may still be reading the pinned table
  AFC_CUDA(cudaStreamSynchronize(b->stream));
  int64_t tile = 0;
  for (size_t q = 0; q < b->list.size(); ++q) {
    afc_problem_s* p = b->list[q];
    BInst& e = b->tab_h[q];
    std::memset(&e, 0, sizeof(e));
    e.of = p->offs;
    e.a = ssp_arrays(p);
    e.a.Fs = nullptr;   // F* is not kept in a batch
    e.vec[0] = p->u.p;
    e.vec[1] = p->ustage.p;
    e.vec[2] = p->tmp.p;
    e.dt = dts[q];
    e.tile0 = tile;
    e.ntiles = (p->N + block - 1) / block;
    tile += e.ntiles;
  }
  b->ntiles = tile;
  b->tab_block = block;
  b->tab_dt = dts;
  AFC_CUDA(cudaMemcpyAsync(b->tab_d, b->tab_h, b->list.size() * sizeof(BInst), cudaMemcpyHostToDevice, b->stream));
  return AFC_OK;
}

StageArgs stage_args(int scheme, int s) {
  // vec: 0 = u (stored solution, u^n during the step), 1 = ustage, 2 = tmp
  StageArgs a{};
  a.nst = 1;
  if (scheme == AFC_SSP2) {
    if (s == 0) { a.in[0] = 0; a.uA[0] = -1; a.out[0] = 1; a.ca[0] = 0.0; a.cb[0] = 1.0; }
    else        { a.in[0] = 1; a.uA[0] = 0;  a.out[0] = 0; a.ca[0] = 0.5; a.cb[0] = 0.5; }
  } else {
    if (s == 0)      { a.in[0] = 0; a.uA[0] = -1; a.out[0] = 1; a.ca[0] = 0.0;       a.cb[0] = 1.0; }
    else if (s == 1) { a.in[0] = 1; a.uA[0] = 0;  a.out[0] = 2; a.ca[0] = 0.75;      a.cb[0] = 0.25; }
    else             { a.in[0] = 2; a.uA[0] = 0;  a.out[0] = 0; a.ca[0] = 1.0 / 3.0; a.cb[0] = 2.0 / 3.0; }
  }
  return a;
}

StageArgs step_args(int scheme) {
  StageArgs all{};
  const int ns = scheme == AFC_SSP2 ? 2 : 3;
  all.nst = ns;
  for (int s = 0; s < ns; ++s) {
    StageArgs one = stage_args(scheme, s);
    all.in[s] = one.in[0];
    all.uA[s] = one.uA[0];
    all.out[s] = one.out[0];
    all.ca[s] = one.ca[0];
    all.cb[s] = one.cb[0];
  }
  return all;
}

int launch_batch(afc_batch_s* b, cudaStream_t s, bool mixed, bool coop, int grid, int block, StageArgs sa,
                 int limiter, int lo, int hi) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = coop ? at : nullptr;
  cfg.numAttrs = coop ? 1 : 0;
  const int ninst = (int)b->list.size();
  cudaError_t e = mixed ? cudaLaunchKernelEx(&cfg, k_batch_ssp<true>, (const BInst*)b->tab_d, ninst, b->ntiles, sa,
                                             limiter, lo, hi, b->bar)
                        : cudaLaunchKernelEx(&cfg, k_batch_ssp<false>, (const BInst*)b->tab_d, ninst, b->ntiles, sa,
                                             limiter, lo, hi, b->bar);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernelEx(k_batch_ssp)");
  return AFC_OK;
}

// Grid of the persistent launches: resident blocks per SM x SMs, at most one block per tile.
int coop_grid(afc_batch_s* b, bool mixed, const afc_batch_tuning& t, int* grid) {
  int mb = 0;
  int st = max_blocks_per_sm(mixed, t.block, &mb);
  if (st) return st;
  if (mb < 1) { set_error("batch kernel does not fit on an SM at this block size"); return AFC_E_INVALID; }
  const int bps = t.blocks_per_sm > 0 ? std::min(t.blocks_per_sm, mb) : mb;
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->ntiles, (int64_t)bps * b->nsm));
  return AFC_OK;
}

// Enqueue the launches of one time step on stream s; *nl receives their count.
int enqueue_step(afc_batch_s* b, cudaStream_t s, const afc_opts* o, const afc_batch_tuning& t, int grid, int* nl) {
  const bool mixed = o->precision == AFC_MIXED;
  const int ns = o->scheme == AFC_SSP2 ? 2 : 3;
  int st;
  *nl = 0;
  if (t.mode == AFC_BATCH_PER_PASS) {
    if (b->ntiles > 0x7fffffff) { set_error("batch too large for one launch per pass"); return AFC_E_INVALID; }
    for (int sidx = 0; sidx < ns; ++sidx) {
      const StageArgs sa = stage_args(o->scheme, sidx);
      for (int ph = 0; ph < 4; ++ph) {
        if (ph == 1 && o->limiter == AFC_LIM_NONE) continue;
        if (ph == 2 && o->limiter != AFC_LIM_ZALESAK) continue;
        if ((st = launch_batch(b, s, mixed, false, (int)b->ntiles, t.block, sa, o->limiter, ph, ph))) return st;
        ++*nl;
      }
    }
    return AFC_OK;
  }
  if (t.mode == AFC_BATCH_PER_STAGE) {
    for (int sidx = 0; sidx < ns; ++sidx) {
      if ((st = launch_batch(b, s, mixed, true, grid, t.block, stage_args(o->scheme, sidx), o->limiter, 0, 3)))
        return st;
      ++*nl;
    }
  } else {
    if ((st = launch_batch(b, s, mixed, true, grid, t.block, step_args(o->scheme), o->limiter, 0, 3))) return st;
    ++*nl;
  }
  return AFC_OK;
}

std::string graph_key(const afc_opts* o, const afc_batch_tuning& t) {
  char buf[96];
  std::snprintf(buf, sizeof buf, "%d/%d/%d/%d/%d/%d", o->scheme, o->limiter, o->precision, t.mode, t.block,
                t.blocks_per_sm);
  return buf;
}

// The graph of one step for this shape (built on first use).  If the runtime
// cannot capture the launches, the entry has no graph and the step is enqueued
// directly.
int step_graph(afc_batch_s* b, const afc_opts* o, const afc_batch_tuning& t, GraphEntry** out) {
  const std::string key = graph_key(o, t) + "/" + std::to_string(b->ntiles);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = &it->second;
    return AFC_OK;
  }
  GraphEntry ge;
  int st = t.mode == AFC_BATCH_PER_PASS ? AFC_OK : coop_grid(b, o->precision == AFC_MIXED, t, &ge.grid);
  if (st) return st;
  if (!b->cap_stream) AFC_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  AFC_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  int nl = 0;
  st = enqueue_step(b, b->cap_stream, o, t, ge.grid, &nl);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  if (st && st != AFC_E_CUDA) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (!st && e == cudaSuccess && g) {
    e = cudaGraphInstantiate(&ge.exec, g, 0);
    if (e != cudaSuccess) ge.exec = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();   // a failed capture leaves no sticky error; direct launches follow
  ge.launches = nl;
  auto res = b->graphs.emplace(key, ge);
  *out = &res.first->second;
  return AFC_OK;
}

int check_opts(const afc_opts* o) {
  if (!o) { set_error("null options"); return AFC_E_INVALID; }
  if (o->scheme != AFC_SSP2 && o->scheme != AFC_SSP3) {
    set_error("batched steps support AFC_SSP2 and AFC_SSP3");
    return AFC_E_INVALID;
  }
  if (o->limiter != AFC_LIM_NONE && o->limiter != AFC_LIM_GALERKIN && o->limiter != AFC_LIM_ZALESAK) {
    set_error("batched steps support limiters NONE, GALERKIN, ZALESAK");
    return AFC_E_INVALID;
  }
  if (o->precision != AFC_FP64 && o->precision != AFC_MIXED) { set_error("bad precision"); return AFC_E_INVALID; }
  return AFC_OK;
}

int check_dt(afc_batch_s* b, const afc_opts* o, const double* dt) {
  if (dt) {
    for (size_t q = 0; q < b->list.size(); ++q)
      if (!(dt[q] > 0.0) || !std::isfinite(dt[q])) { set_error("every dt must be finite and > 0"); return AFC_E_INVALID; }
  } else if (!(o->dt > 0.0)) {
    set_error("need dt > 0 (opts->dt or the dt array)");
    return AFC_E_INVALID;
  }
  return AFC_OK;
}

// Work the caller enqueued on an instance's own stream (set_solution, ...) must be
// done before the batch's stream reads the instance.
int join_instance_streams(afc_batch_s* b) {
  for (auto* p : b->list)
    if (p->stream != b->stream) AFC_CUDA(cudaStreamSynchronize(p->stream));
  return AFC_OK;
}

// nsteps steps with tuning t; no synchronisation
int run_steps(afc_batch_s* b, const afc_opts* o, const double* dt, int nsteps, const afc_batch_tuning& t) {
  int st;
  if ((st = join_instance_streams(b))) return st;
  if ((st = build_table(b, t.block, dt, o->dt, o->precision == AFC_MIXED))) return st;
  GraphEntry* ge = nullptr;
  if ((st = step_graph(b, o, t, &ge))) return st;
  for (int k = 0; k < nsteps; ++k) {
    if (ge->exec) {
      AFC_CUDA(cudaGraphLaunch(ge->exec, b->stream));
    } else {
      int nl = 0;
      if ((st = enqueue_step(b, b->stream, o, t, ge->grid, &nl))) return st;
    }
  }
  b->launches += (int64_t)ge->launches * nsteps;
  return AFC_OK;
}

// Extremes of every instance's stored solution (one launch), into b->mm_h.
int batch_minmax(afc_batch_s* b) {
  const int n = (int)b->list.size();
  k_batch_minmax<<<n, 256, 0, b->stream>>>(b->tab_d, b->mm_d);
  b->launches++;
  AFC_CUDA(cudaGetLastError());
  AFC_CUDA(cudaMemcpyAsync(b->mm_h, b->mm_d, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  return AFC_OK;
}

// The instances' input ranges for afc_stats.dmp_violation: measured once for all when
// any instance's range is not known from an earlier call.  k_batch_minmax reads the
// instance table, so the table of this call's launch shape is built first (the
// device table is uninitialised until the first build).
int batch_input_ranges(afc_batch_s* b, int block, const double* dt, const afc_opts* o) {
  bool all = true;
  for (auto* p : b->list) all = all && p->u_range_valid;
  if (all) return AFC_OK;
  int st = build_table(b, block, dt, o->dt, o->precision == AFC_MIXED);
  if (st) return st;
  if ((st = batch_minmax(b))) return st;
  AFC_CUDA(cudaStreamSynchronize(b->stream));
  for (size_t q = 0; q < b->list.size(); ++q) {
    b->list[q]->u_lo = b->mm_h[2 * q];
    b->list[q]->u_hi = b->mm_h[2 * q + 1];
    b->list[q]->u_range_valid = true;
  }
  return AFC_OK;
}

int batch_status(afc_batch_s* b, afc_stats* stats, int stages) {
  const int n = (int)b->list.size();
  int st0 = batch_minmax(b);
  if (st0) return st0;
  AFC_CUDA(cudaMemcpyAsync(b->mm_h + 2 * n, &b->bar->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  AFC_CUDA(cudaStreamSynchronize(b->stream));
  int err = 0;
  std::memcpy(&err, b->mm_h + 2 * n, sizeof(int));
  const int status = err ? AFC_E_TIMEOUT : AFC_OK;
  for (int q = 0; q < n; ++q) {
    afc_problem_s* p = b->list[q];
    const double mn = b->mm_h[2 * q], mx = b->mm_h[2 * q + 1];
    if (stats) {
      const double lo = std::min(p->u_lo, p->dir_lo), hi = std::max(p->u_hi, p->dir_hi);
      std::memset(&stats[q], 0, sizeof(afc_stats));
      stats[q].stages = stages;
      stats[q].umin = mn;
      stats[q].umax = mx;
      stats[q].dmp_violation = std::max(0.0, std::max(lo - mn, mx - hi));
      stats[q].status = status;
    }
    p->u_lo = mn;
    p->u_hi = mx;
    p->u_range_valid = !err;
  }
  if (err) {
    AFC_CUDA(cudaMemsetAsync(b->bar, 0, sizeof(GridBar), b->stream));
    AFC_CUDA(cudaStreamSynchronize(b->stream));
    set_error("a grid barrier of the batched step gave up waiting");
    return AFC_E_TIMEOUT;
  }
  return AFC_OK;
}

void batch_free(afc_batch_s* b) {
  for (auto& kv : b->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  b->graphs.clear();
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->tab_h) cudaFreeHost(b->tab_h);
  if (b->mm_h) cudaFreeHost(b->mm_h);
  if (b->tab_d) cudaFree(b->tab_d);
  if (b->bar) cudaFree(b->bar);
  if (b->mm_d) cudaFree(b->mm_d);
  if (b->backup) cudaFree(b->backup);
  delete b;
}

}  // namespace
}  // namespace afc

using namespace afc;

namespace afc {

// A batch enqueued on `stream` instead of the first problem's.
int batch_create_on_stream(const afc_problem* list, int count, cudaStream_t stream, afc_batch* out);

}  // namespace afc

extern "C" int afc_batch_create(const afc_problem* list, int count, afc_batch* out) {
  if (!out || !list) { set_error("null argument"); return AFC_E_INVALID; }
  if (count < 1 || !list[0]) { set_error("batch size must be 1..65536"); return AFC_E_INVALID; }
  return afc::batch_create_on_stream(list, count, list[0]->stream, out);
}

int afc::batch_create_on_stream(const afc_problem* list, int count, cudaStream_t stream, afc_batch* out) {
  if (!out || !list) { set_error("null argument"); return AFC_E_INVALID; }
  *out = nullptr;
  if (count < 1 || count > 65536) { set_error("batch size must be 1..65536"); return AFC_E_INVALID; }
  for (int q = 0; q < count; ++q) {
    if (!list[q]) { set_error("null problem in the batch"); return AFC_E_INVALID; }
    if (!list[q]->assembled) { set_error("every problem of a batch must be assembled"); return AFC_E_STATE; }
    if (list[q]->device != list[0]->device) { set_error("the problems of a batch must share a device"); return AFC_E_INVALID; }
    for (int r = 0; r < q; ++r)
      if (list[r] == list[q]) { set_error("a problem appears twice in the batch"); return AFC_E_INVALID; }
  }
  afc_batch_s* b = new afc_batch_s();
  b->list.assign(list, list + count);
  b->device = list[0]->device;
  b->stream = stream;
  for (auto* p : b->list) b->total_nodes += p->N;
  auto fail = [&](int st) {
    batch_free(b);
    return st;
  };
  if (cudaSetDevice(b->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaSetDevice"));
  cudaError_t e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
  int coop = 0;
  e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
  if (!coop) {
    set_error("device does not support cooperative launches");
    return fail(AFC_E_CUDA);
  }
  if ((e = cudaMallocHost((void**)&b->tab_h, count * sizeof(BInst))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->mm_h, (2 * count + 1) * sizeof(double))) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMallocHost"));
  if ((e = cudaMalloc((void**)&b->tab_d, count * sizeof(BInst))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->bar, sizeof(GridBar))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->mm_d, 2 * count * sizeof(double))) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of the batch tables failed");
    return fail(AFC_E_OOM);
  }
  if ((e = cudaMemsetAsync(b->bar, 0, sizeof(GridBar), b->stream)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMemsetAsync"));
  *out = b;
  return AFC_OK;
}

extern "C" int afc_batch_destroy(afc_batch b) {
  if (!b) return AFC_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return AFC_OK;
}

extern "C" int afc_batch_step(afc_batch b, const afc_opts* o, const double* dt, int nsteps, afc_stats* stats) {
  if (!b) { set_error("null batch"); return AFC_E_INVALID; }
  int st;
  if ((st = check_opts(o)) || (st = check_dt(b, o, dt))) return st;
  if (nsteps < 0) { set_error("nsteps must be >= 0"); return AFC_E_INVALID; }
  if (cudaSetDevice(b->device) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  const afc_batch_tuning t = effective_tuning(b, o);
  if ((st = batch_input_ranges(b, t.block, dt, o))) return st;
  if ((st = run_steps(b, o, dt, nsteps, t))) return st;
  return batch_status(b, stats, nsteps * (o->scheme == AFC_SSP2 ? 2 : 3));
}

extern "C" int afc_batch_set_tuning(afc_batch b, const afc_batch_tuning* t) {
  if (!b || !t) { set_error("null argument"); return AFC_E_INVALID; }
  if (t->mode == AFC_BATCH_AUTO) {
    b->fixed = false;
    return AFC_OK;
  }
  int st = valid_tuning(*t);
  if (st) return st;
  b->tuning = *t;
  b->fixed = true;
  return AFC_OK;
}

extern "C" int afc_batch_get_tuning(afc_batch b, afc_batch_tuning* t) {
  if (!b || !t) { set_error("null argument"); return AFC_E_INVALID; }
  if (b->fixed) {
    *t = b->tuning;
  } else {
    afc_opts o;
    afc_default_opts(&o);
    *t = effective_tuning(b, &o);
    t->mode = AFC_BATCH_AUTO;
  }
  return AFC_OK;
}

extern "C" int afc_batch_tune(afc_batch b, const afc_opts* o, const double* dt, afc_batch_tuning* best) {
  if (!b) { set_error("null batch"); return AFC_E_INVALID; }
  int st;
  if ((st = check_opts(o)) || (st = check_dt(b, o, dt))) return st;
  if (cudaSetDevice(b->device) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  cudaStream_t s = b->stream;
  if (!b->backup) {
    cudaError_t e = cudaMalloc((void**)&b->backup, b->total_nodes * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of the tuning backup failed");
      return AFC_E_OOM;
    }
  }
  auto copy_all = [&](bool save) -> int {
    int64_t off = 0;
    for (auto* p : b->list) {
      if (save)
        AFC_CUDA(cudaMemcpyAsync(b->backup + off, p->u.p, p->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      else
        AFC_CUDA(cudaMemcpyAsync(p->u.p, b->backup + off, p->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      off += p->N;
    }
    return AFC_OK;
  };
  if ((st = copy_all(true))) return st;
  std::vector<afc_batch_tuning> cand;
  const int blocks[3] = {128, 256, 512};
  for (int blk : blocks) {
    cand.push_back({AFC_BATCH_PER_PASS, blk, 0, 0.0});
    cand.push_back({AFC_BATCH_PER_STAGE, blk, 0, 0.0});
    cand.push_back({AFC_BATCH_PER_STEP, blk, 0, 0.0});
    int mb = 0;
    if ((st = max_blocks_per_sm(o->precision == AFC_MIXED, blk, &mb))) return st;
    if (mb >= 2) cand.push_back({AFC_BATCH_PER_STAGE, blk, mb / 2, 0.0});
  }
  cudaEvent_t e0, e1;
  AFC_CUDA(cudaEventCreate(&e0));
  AFC_CUDA(cudaEventCreate(&e1));
  afc_batch_tuning win{};
  win.ms_per_step = 1e300;
  const int reps = 3;
  for (auto& c : cand) {
    if ((st = run_steps(b, o, dt, 1, c))) break;   // warm-up (and graph build)
    cudaEventRecord(e0, s);
    if ((st = run_steps(b, o, dt, reps, c))) break;
    cudaEventRecord(e1, s);
    if ((st = batch_status(b, nullptr, 0))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c.ms_per_step = ms / reps;
    if (c.ms_per_step < win.ms_per_step) win = c;
    if ((st = copy_all(false))) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int st2 = copy_all(false);
  for (auto* p : b->list) p->u_range_valid = false;   // the trials' ranges are not the restored states'
  if (st) return st;
  if (st2) return st2;
  AFC_CUDA(cudaStreamSynchronize(s));
  b->tuning = win;
  b->fixed = true;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tune_cache[size_class(b, o)] = win;
  }
  if (best) *best = win;
  return AFC_OK;
}

extern "C" int afc_batch_info(afc_batch b, int64_t* total_nodes, int64_t* launches) {
  if (!b) { set_error("null batch"); return AFC_E_INVALID; }
  if (total_nodes) *total_nodes = b->total_nodes;
  if (launches) *launches = b->launches;
  return AFC_OK;
}
