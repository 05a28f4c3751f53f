// Internal declarations of libafc (not part of the C ABI).
//
// Storage: every matrix lives in diagonal-offset form ("DIA").  The pattern of
// a mesh (pairs i, j with m_ij != 0) is described by K distinct column offsets
// o_0 < ... < o_{K-1} (o = j - i; symmetric set, o_{Kup} = 0).  A full matrix X
// is stored row-indexed, offset-major: X[k * N + i] = x_{i, i + o_k} (0 where the
// pair is not in the pattern).  A symmetric edge quantity (m_ij, d_ij) is stored
// once per pair i < j in the upper half: E[k * N + i] = e_{i, i + o_{Kup+1+k}},
// k = 0..Kup-1.  Consecutive threads (rows) read consecutive addresses for every
// k, with no column-index traffic.  Node vectors carry a zero halo of `pad`
// entries on both sides so that i + o_k is always a valid address.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/afc.h"

namespace afc {

constexpr int kMaxOffsets = 63;       // K <= 63 so that a row's presence mask fits 64 bits
constexpr int kBlock = 256;           // threads per block of the row kernels
constexpr int kRedBlocks = 1216;      // blocks of the reduction kernels (8 x 152 SMs)

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define AFC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return afc::cuda_fail(e__, #call); \
  } while (0)

// A CUDA-graph condition a kernel may set (use = false outside graphs).
struct GraphCond {
  bool use = false;
  cudaGraphConditionalHandle h = 0;
};

// Offsets passed by value to kernels (constant bank, unrolled loops).
struct Offsets {
  int K;          // number of offsets (odd)
  int Kup;        // number of positive offsets; index of offset 0 is Kup
  int o[kMaxOffsets];
};

// Host-side mesh structure (integer only).
struct MeshStructure {
  int elem = 0;                       // AFC_P1 / AFC_Q1
  int nl = 0;                         // vertices per cell
  int64_t N = 0, ncells = 0;
  std::vector<double> xyz;            // 3N
  std::vector<int32_t> conn;          // nl * ncells
  std::vector<int32_t> offsets;       // K sorted offsets
  std::vector<uint64_t> mask;         // N: bit k set iff (i, i + o_k) is in the pattern
  std::vector<int32_t> inc_ptr;       // N + 1: cells incident to a node
  std::vector<int32_t> inc;           // (cell << 3) | local vertex
  int64_t nnz = 0, n_edges = 0;
};

int build_structured(int elem, int nx, int ny, int nz, const double lo[3], const double hi[3], MeshStructure& m);
int build_from_elements(int elem, int64_t n_nodes, const double* xyz, int64_t n_cells, const int32_t* conn,
                        MeshStructure& m);

// Device buffer helpers.
template <class T>
struct DBuf {
  T* base = nullptr;   // allocation
  T* p = nullptr;      // logical start (after the halo)
  int64_t n = 0, pad = 0;
  int alloc(int64_t n_, int64_t pad_ = 0);
  void free_();
};

struct KrylovWork;   // defined in krylov.cu
struct Profiler;     // defined in prof.cpp
struct StepGraph;    // defined in graph.cu

}  // namespace afc

struct afc_problem_s;

namespace afc {

// Kernel launches of the library go through AFC_LAUNCH: it counts launches and,
// while profiling is on, brackets each launch with two events on the stream.
cudaEvent_t prof_start(afc_problem_s* p);
void prof_stop(afc_problem_s* p, const char* name, cudaEvent_t start);
void prof_free(afc_problem_s* p);
bool prof_set_enabled(afc_problem_s* p, bool on);   // returns the previous state

#define AFC_LAUNCH(p, name, ...)                       \
  do {                                                 \
    cudaEvent_t ev0__ = afc::prof_start(p);            \
    __VA_ARGS__;                                       \
    afc::prof_stop(p, name, ev0__);                    \
  } while (0)

}  // namespace afc

struct afc_problem_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  afc::MeshStructure mesh;
  afc::Offsets offs{};
  int64_t N = 0;
  int K = 0, Kup = 0, pad = 0;

  // mesh on device
  afc::DBuf<double> xyz;
  afc::DBuf<int32_t> conn, inc_ptr, inc;
  afc::DBuf<unsigned long long> mask;

  // coefficients and boundary data
  bool coef_set = false;
  double eps = 0.0, c = 0.0;
  afc::DBuf<double> bnod, fnod;
  afc::DBuf<double> cnod;                         // N: nodal reaction (when c_nodal)
  bool c_nodal = false;
  afc::DBuf<uint8_t> dir;
  afc::DBuf<double> udir;

  // matrices (see the storage note at the top)
  bool assembled = false;
  int family = 0, precision = 0;
  afc::DBuf<double> Mfull, Sfull, Kfull, Afull;   // K * N each
  afc::DBuf<double> AA;                           // K * N, low-order operator
  afc::DBuf<double> Rfull;                        // K * N, (c_h phi_j, phi_i) for a nodal reaction
  afc::DBuf<double> rl;                           // N: lumped reaction (c m_i or row sums of Rfull)
  afc::DBuf<double> m_up, d_up;                   // Kup * N, symmetric edge data
  afc::DBuf<double> kij_up, kji_up;               // Kup * N, MC: convective k_ij and k_ji of each pair i < j
  afc::DBuf<double> d2_up;                        // Kup * N, MC: 2 |d_ij|
  afc::DBuf<float> pairf;                         // 3 * Kup * N, MC: 2|d_ij|, k_ij, k_ji rounded to single
  afc::DBuf<double> AG;                           // K * N, MC: unlimited operator K + eps S + c M_L
  afc::DBuf<double> mL, f;                        // N
  afc::DBuf<double> Bst;                          // K * N, stationary system (Dirichlet rows = identity)
  afc::DBuf<float> Bst32;
  afc::DBuf<double> dinv_st;
  afc::DBuf<float> dinv_st32;
  double cn_dt = -1.0;                            // dt the CN system was built for
  afc::DBuf<double> Bcn;                          // K * N, M_L/dt + AA/2 (Dirichlet rows = identity)
  afc::DBuf<double> mdt_up;                       // Kup * N, m_ij / dt of the CN step
  afc::DBuf<double> mLdt;                         // N, m_i / dt
  afc::DBuf<float> Bcn32;
  afc::DBuf<double> dinv_cn;
  afc::DBuf<float> dinv_cn32;

  // state and work vectors (node vectors carry the halo)
  afc::DBuf<double> u, u0, ustage, udot, ut, Rp, Rm, Fs, Qp, Qm, b0, res, delta, umax, umin, tmp, cn_a, cn_s;
  afc::DBuf<double> bA, bB;         // MC: u_max - u and u - u_min
  afc::DBuf<double> Fold;           // CN with the MC limiter: F*(u^{n-1})
  afc::DBuf<unsigned long long> clip;   // MC: per row, bit k set if the pair of offset k was clipped
  afc::DBuf<float4> nodef;          // MC: (u, u_max - u, u - u_min) rounded to single
  // MC, mixed precision: the sweep in float pairs (mc_pair.cu)
  afc::DBuf<float2> AGp, fp2;       // K * N and N: AG and f as pairs
  afc::DBuf<float2> pk_hi, pk_lo;   // Kup * N: (k_ij, k_ji) of each pair, high parts and low parts
  afc::DBuf<float2> up2, yp2;       // node vectors: u and y = f - AG u as pairs
  afc::DBuf<float2> abh2, abl2;     // node vectors: high and low parts of (A, B) = (u_max - u, u - u_min)
  afc::DBuf<float2> cp_up;          // Kup * N: clipped amount of each pair, at its lower row
  afc::DBuf<unsigned> mask32, clip32;   // node vectors, 16 < K <= 32: presence and clip masks in 32 bits
  afc::DBuf<uint16_t> mask16, clip16;   // K <= 16: the same in 16 bits (clip16: N + 1 entries, no halo)
  afc::DBuf<double> r_up;           // Kup * N: antidiffusive flux of each pair, at its lower row
  // mixed-precision explicit stage: m_ij, d_ij, r_ij (Kup * N) and u, udot^L (node vectors) in single
  afc::DBuf<float> m32_up, d32_up, r32, uf, udf;
  bool ssp32_ready = false;         // m32_up / d32_up match the assembled m_up / d_up
  afc::DBuf<double> scal;           // small device scalars (norms, dt, ...)
  afc::DBuf<double> part;           // reduction partials
  double* host_scal = nullptr;      // pinned host mirror of scal

  afc::KrylovWork* kw = nullptr;
  afc::Profiler* prof = nullptr;
  afc::StepGraph* g_step = nullptr;   // cached graph of afc_step
  afc::StepGraph* g_stat = nullptr;   // cached graph of afc_solve_stationary
  cudaStream_t cap_stream = nullptr;  // private stream used to capture graphs
  int64_t launches = 0;             // kernel launches issued on this problem
  // range of the stored solution (known after afc_set_solution, a step or a solve)
  // and of the Dirichlet values: the reference of afc_stats.dmp_violation
  bool u_range_valid = false;
  double u_lo = 0.0, u_hi = 0.0;
  double dir_lo = 1e308, dir_hi = -1e308;
  // bounded-wait limit of the grid barriers in this problem's persistent launches
  unsigned long long grid_wait_ns = 4000000000ull;
  int64_t device_bytes = 0;
};

namespace afc {

// ---- assembly (assemble.cu) ----
int assemble_device(afc_problem_s* p, int family, int precision);
int build_cn_system(afc_problem_s* p, double dt);

// ---- kernels of the hot path (fct.cu, mc.cu) ----
// SSP forward-Euler stage: out = a * uA + b * FE(uin) (Eq. FE-SSP with Zalesak).
int fe_stage(afc_problem_s* p, const double* uin, double dt, int limiter, double a, const double* uA, double b,
             double* out, bool mixed = false);
int ensure_ssp_mixed(afc_problem_s* p);   // single-precision copies of m_ij, d_ij for the mixed stage
struct SspArrays;
SspArrays ssp_arrays(afc_problem_s* p);
// The residual functions below store ||res||^2 at *normsq_slot; with a null slot they
// leave the grid_for(N) block partials of res^2 in p->part for the caller to sum.
// CN helpers
int cn_predictor(afc_problem_s* p, const double* u_old, double dt);   // ut, b0, Qp = m Q+, Qm = m Q-
int cn_linear_guess(afc_problem_s* p, const double* u_old, double* u);             // u = 2 ut - u_old (after cn_predictor)
// CN with the MC limiter (Sec. 2.2): Fold = F*(u_old), then res = b0 + (F*(u) + Fold)/2 - (M_L/dt + AA/2) u
int mc_cn_old_flux(afc_problem_s* p, const double* u_old);
int mc_cn_residual(afc_problem_s* p, const double* u, double* res, double* normsq_slot);
// a = u - u_old, s = u + u_old after u += omega * delta (delta may be null)
int cn_update(afc_problem_s* p, double omega, const double* delta, double* u, const double* u_old);
int cn_limited_residual(afc_problem_s* p, const double* u_new, double dt, int limiter, int prelimit, double* res,
                        double* normsq_slot);                                      // needs cn_update first
// MC
// transient MC stage: bounds of u and the clipped SSP fluxes r*_ij into r_up (after the rate pass)
int mc_ssp_fluxes(afc_problem_s* p, const double* u);
// pair = true: the MC and Galerkin modes of a mixed-precision assembly evaluate the
// residual in float pairs (mc_pair.cu); F* for inspection and the other modes stay FP64
int mc_limited_residual(afc_problem_s* p, const double* u, int limiter, double* res, double* normsq_slot,
                        bool want_F = false, bool pair = false);
// the same residual (MC or Galerkin) in float-pair arithmetic, for mixed-precision MC
// problems (mc_pair.cu); mc_pair_setup builds its pair copies at assembly
int mc_pair_setup(afc_problem_s* p);
int mc_pair_residual(afc_problem_s* p, const double* u, int limiter, double* res, double* normsq_slot);

// ---- reductions and BLAS-1 (krylov.cu) ----
int dot_device(afc_problem_s* p, const double* x, const double* y, double* out_slot);
// An update that the persistent BiCGStab applies to the solution x in its last pass,
// unless the solve broke down: u += omega x, then a = u - uo and s = u + uo (the
// damped CN correction and the node sums of the next flux pass, bit for bit what
// cn_update computes).  u == nullptr: none.
struct KrylovEpilogue {
  double omega = 0.0;
  double* u = nullptr;
  const double* uo = nullptr;
  double* a = nullptr;
  double* s = nullptr;
  double* fp_sc = nullptr;   // graph form: the fixed-point scalars, where the solve counts itself
};
// *epi_done (if given) tells whether the solve applied *epi; when it did not, the
// caller applies the update itself.
int krylov_solve(afc_problem_s* p, int system, const afc_opts* o, const double* rhs, double* x, int* its,
                 double* res, const KrylovEpilogue* epi = nullptr, bool* epi_done = nullptr);
int dia_spmv(afc_problem_s* p, const double* A, const double* x, double* y);
int axpy_device(afc_problem_s* p, double a, const double* x, double* y);   // y += a x
int minmax_device(afc_problem_s* p, const double* x, double* mn, double* mx);
void krylov_free(afc_problem_s* p);
const void* krylov_key(afc_problem_s* p);   // changes when the solver workspace is reallocated

// ---- whole steps as CUDA graphs (graph.cu) ----
int cn_step_graph(afc_problem_s* p, const afc_opts* o, afc_stats* st);
int ssp_step_graph(afc_problem_s* p, const afc_opts* o, afc_stats* st);
int stationary_graph(afc_problem_s* p, const afc_opts* o, afc_stats* st);
void graph_free(afc_problem_s* p);

int64_t grid_for(int64_t n, int block = kBlock);

}  // namespace afc
