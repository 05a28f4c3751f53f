// Mixed-precision sweep of the stationary MC limiter (Sec. 3.1, Eq. MClimiter with the
// bounds of Eq. u_max_min) and the nonlinear residual res = f + F*(u) - AA u of Sec. 4,
// in float-pair arithmetic (pair_float.cuh) instead of FP64.
//
// The formulation is that of mc.cu: with the clipped amounts c_ij (r_ij - r*_ij),
//   res = f - AG u - sum_j c_ij,   AG = K + eps S + c M_L,
// and c_ij = max(0, -T_i, -T_j) (r_ij > 0) or min(0, T_i, T_j) (r_ij < 0) with
// T = 2|d_ij| X - a |u_j - u_i|, X the room of the side in its bounds.  The matrix AG,
// f, k_ij and k_ji are stored as float pairs (8 bytes per value, as many as a double;
// (k_ij, k_ji) interleaved per pair, high parts and low parts apart; 2|d_ij| =
// 2 max(0, k_ij, k_ji) is formed from them), and the state is split into pairs once
// per sweep, so that the sweep
// issues no FP64 instruction per matrix entry or per pair: on GB300 one FP64 warp
// instruction per pair of the P1 129^3 grid alone costs ~23 us, which is what
// bounded the FP64 form.
//
// Passes (one launch each):
//  1. k_mcp_split:   u -> pairs (integer pipe);
//  2. k_mcp_rows:    per row, y = f - AG u and the bounds u_max, u_min over N_i in
//                    one pass over the row's neighbours (the same state loads serve
//                    both), A = u_max - u, B = u - u_min; clears the clip mask;
//  3. k_mcp_edges:   per pair i < j, the exact single-precision pre-test of mc.cu on
//                    the high parts, and for the pairs it cannot clear, T_i, T_j and
//                    c_ij in pair arithmetic (stored at row i, its bit set in the masks
//                    of rows i and j);
//  4. k_mcp_residual: res = y - sum_j c_ij on free rows (0 on Dirichlet rows), in
//                    pairs, rounded to double once; block partials of res^2 (in pairs
//                    while |res| < 2^60), summed by k_mcp_finalize when the caller
//                    wants the norm (a separate one-block launch: a last-block sum
//                    in the pass, with a fence and an atomic per block, was slower).
// Accuracy: every value carries a relative error of at most 2^-48 and every product
// and sum an error of that order relative to the magnitudes summed, so res agrees
// with its FP64 evaluation to ~1e-14 of sum_j |AG_ij u_j| + sum_j |c_ij|, and the
// bounds are exact up to pairs that tie within 2^-48.
#include <type_traits>

#include "afc_internal.h"
#include "kernels_common.cuh"
#include "pair_float.cuh"

namespace afc {

namespace {

// Word of the per-row presence and clip masks (bit k: offset k), as narrow as the
// number of offsets known at compile time allows: 16 bits for P1 (15 offsets), 32
// for Q1 (27), 64 otherwise; narrower masks mean less traffic in the rows and
// residual passes.  16-bit clip masks are set by 32-bit atomics on the aligned word
// that holds two rows' masks (row i in the half (i & 1) of word i >> 1).
template <int KT>
using MaskWord = std::conditional_t<(KT > 0 && KT <= 16), uint16_t,
                                    std::conditional_t<(KT > 0 && KT <= 32), unsigned, unsigned long long>>;

// The presence masks in a narrower word (once, at assembly).
template <class M>
__global__ void k_mcp_mask_narrow(int64_t N, const unsigned long long* __restrict__ mask, M* __restrict__ m) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) m[i] = (M)mask[i];
}

// Sets bit b of row r's clip mask.
template <class M>
__device__ __forceinline__ void clip_set(M* clip, int64_t r, int b) {
  if constexpr (sizeof(M) == 2) {
    atomicOr(reinterpret_cast<unsigned*>(clip) + (r >> 1), (1u << b) << (16 * (int)(r & 1)));
  } else {
    atomicOr(clip + r, (M)1 << b);
  }
}

__global__ void k_mcp_split(int64_t N, const double* __restrict__ u, float2* __restrict__ up) {
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) up[i] = split_pair(u[i]);
}

template <int KT>
__global__ void __launch_bounds__(kBlock) k_mcp_rows(int64_t N, Offsets of, const MaskWord<KT>* __restrict__ mask,
                                                     const float2* __restrict__ up, const float2* __restrict__ AGp,
                                                     const float2* __restrict__ fp, float2* __restrict__ yp,
                                                     float2* __restrict__ abh, float2* __restrict__ abl,
                                                     MaskWord<KT>* __restrict__ clip) {
  const int K = KT > 0 ? KT : of.K;
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  // the row's matrix entries, mask and source first (no pass writes them), then, once
  // the split is done, its states: all loads of the row in flight together
  const MaskWord<KT> mk = __ldcs(mask + i);
  const float2 f = __ldcs(fp + i);
  constexpr int KL = KT > 0 ? KT : 1;
  float2 vv[KL], aa[KL];
  if (KT > 0) {
#pragma unroll
    for (int k = 0; k < KL; ++k) aa[k] = __ldcs(AGp + (int64_t)k * N + i);   // read once per sweep: past L2
  }
  pdl_wait();
  const float2 ui = up[i];
  float mxh = ui.x, mxl = ui.y, mnh = ui.x, mnl = ui.y;
  float sh = f.x, sl = f.y;   // y = f - sum_k AG_ik u_{i + o_k}: running high sum, summed errors
  if (KT > 0) {
#pragma unroll
    for (int k = 0; k < KL; ++k) vv[k] = up[i + of.o[k]];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 v = KT > 0 ? vv[KT > 0 ? k : 0] : up[i + of.o[k]];
    const float2 a = KT > 0 ? aa[KT > 0 ? k : 0] : __ldcs(AGp + (int64_t)k * N + i);
    float ph, pl, s, e;
    pair_mul(a.x, a.y, v.x, v.y, ph, pl);
    two_sum(sh, -ph, s, e);
    sh = s;
    sl = __fadd_rn(sl, __fsub_rn(e, pl));
    if ((mk >> k) & 1u) {
      if (pair_gt(v.x, v.y, mxh, mxl)) {
        mxh = v.x;
        mxl = v.y;
      }
      if (pair_gt(mnh, mnl, v.x, v.y)) {
        mnh = v.x;
        mnl = v.y;
      }
    }
  }
  float yh, yl;
  two_sum(sh, sl, yh, yl);
  yp[i] = make_float2(yh, yl);
  float Ah, Al, Bh, Bl;
  pair_sub(mxh, mxl, ui.x, ui.y, Ah, Al);
  pair_sub(ui.x, ui.y, mnh, mnl, Bh, Bl);
  if (Ah < 0.f) Ah = Al = 0.f;   // u_max >= u_i: only a tie within 2^-48 can give a negative room
  if (Bh < 0.f) Bh = Bl = 0.f;
  abh[i] = make_float2(Ah, Bh);
  abl[i] = make_float2(Al, Bl);
  clip[i] = 0;
}

// The pre-test of mc.cu (k_mc_edges), on the high parts: T = 2|d| X - a |D| is
// certainly positive when its single-precision estimate exceeds a strict bound on the
// estimate's error.  The high parts are the roundings of the values (2|d|, a, u) or,
// for X, the high part of a pair within 2^-48 of it, so each input still carries a
// relative error of at most 2^-24 (1 + 2^-24) and the bound 2^-20 (...) of mc.cu holds.
__device__ __forceinline__ bool side_clear(float d2f, float af, float xf, float uif, float ujf) {
  const float tiny = 7.9e-31f;
  if (af < tiny || d2f < tiny || xf < tiny) return false;
  const float Df = fabsf(ujf - uif);
  const float p1 = d2f * xf, p2 = af * Df;
  const float err = 9.5367431640625e-07f * (p1 + p2 + af * (fabsf(uif) + fabsf(ujf))) + tiny;
  return p1 - p2 > err;
}

// T = d2 X - a |D| in pairs, normalised.
__device__ __forceinline__ void side_value(float d2h, float d2l, float xh, float xl, float ah, float al, float Dh,
                                           float Dl, float& th, float& tl) {
  float p1h, p1l, p2h, p2l, s, e;
  pair_mul(d2h, d2l, xh, xl, p1h, p1l);
  pair_mul(ah, al, Dh, Dl, p2h, p2l);
  two_sum(p1h, -p2h, s, e);
  e = __fadd_rn(e, __fsub_rn(p1l, p2l));
  two_sum(s, e, th, tl);
}

// One pair (i, j = i + o) of row i given its loaded data; returns true and the clipped
// amount c_ij (c = -min(0, T_i, T_j) for r_ij > 0, min(0, T_i, T_j) for r_ij < 0) when
// the pair is clipped.  The low parts of a_ij, a_ji (and so of 2|d|) are loaded only here,
// for the pairs the pre-test cannot clear.
__device__ __forceinline__ bool pair_clip(int64_t q, const float2* __restrict__ pkl,
                                          const float2* __restrict__ abl, int64_t i, int64_t j, float d2h, float aih,
                                          float ajh, float2 ui, float2 uj, float2 bi, float2 bj, float2& c) {
  const bool side_i = aih > 0.f, side_j = ajh > 0.f;
  if (!(d2h > 0.f) || !(side_i || side_j)) return false;   // d = 0, or no side can clip
  if (ui.x == uj.x && ui.y == uj.y) return false;           // u_i = u_j: r = 0
  const bool rpos = pair_gt(ui.x, ui.y, uj.x, uj.y);        // r_ij = d (u_j - u_i) > 0  <=>  u_j < u_i
  // room of each side: r > 0 uses A_i = u_i^max - u_i and B_j; r < 0 uses B_i and A_j
  const float xih = rpos ? bi.x : bi.y, xjh = rpos ? bj.y : bj.x;
  if (ui.x != uj.x) {
    const bool ok_i = !side_i || side_clear(d2h, aih, xih, ui.x, uj.x);
    const bool ok_j = !side_j || side_clear(d2h, ajh, xjh, ui.x, uj.x);
    if (ok_i && ok_j) return false;
  }
  const float2 kl = __ldcs(pkl + q);
  const float ail = kl.x, ajl = kl.y;
  // low part of 2|d| = 2 max(0, k_ij, k_ji) (see k_mcp_edges): that of the larger of k_ij,
  // k_ji, whose pairs are ordered as the doubles are
  const float d2l = 2.f * (aih > ajh ? ail : ajh > aih ? ajl : fmaxf(ail, ajl));
  const float2 li = abl[i], lj = abl[j];
  const float xil = rpos ? li.x : li.y, xjl = rpos ? lj.y : lj.x;
  float Dh, Dl;   // |u_j - u_i|
  if (rpos) pair_sub(ui.x, ui.y, uj.x, uj.y, Dh, Dl);
  else pair_sub(uj.x, uj.y, ui.x, ui.y, Dh, Dl);
  float mh = 0.f, ml = 0.f;   // min(0, T_i, T_j)
  if (side_i) {
    float th, tl;
    side_value(d2h, d2l, xih, xil, aih, ail, Dh, Dl, th, tl);
    if (pair_gt(mh, ml, th, tl)) {
      mh = th;
      ml = tl;
    }
  }
  if (side_j) {
    float th, tl;
    side_value(d2h, d2l, xjh, xjl, ajh, ajl, Dh, Dl, th, tl);
    if (pair_gt(mh, ml, th, tl)) {
      mh = th;
      ml = tl;
    }
  }
  if (mh == 0.f && ml == 0.f) return false;
  c = rpos ? make_float2(-mh, -ml) : make_float2(mh, ml);
  return true;
}

// Clipped amount c_ij of every pair i < j (stored at row i, only where nonzero; the
// clip masks of rows i and j get the pair's offset bits, so that the residual pass
// finds a row's clipped pairs in its own mask), one thread per pair slot (ku, i): a
// block covers 32 consecutive rows (threadIdx.x) and all upper offsets (threadIdx.y).
// Every load a pair needs for its pre-test is issued at once (one round trip to
// memory); only the pairs the pre-test cannot clear load the low parts.
template <int KT>
__global__ void k_mcp_edges(int64_t N, Offsets of, const float2* __restrict__ pkh, const float2* __restrict__ pkl,
                            const float2* __restrict__ up, const float2* __restrict__ abh,
                            const float2* __restrict__ abl, float2* __restrict__ c_up,
                            MaskWord<KT>* __restrict__ clip) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  pdl_trigger();
  const int ku = threadIdx.y;
  const int64_t i = blockIdx.x * (int64_t)32 + threadIdx.x;
  if (i >= N) return;
  const int64_t q = (int64_t)ku * N + i;
  const int64_t j = i + of.o[Kup + 1 + ku];
  // a_ij = k_ij, a_ji = k_ji (high parts, one 8-byte load), streamed past L2 so that the
  // node arrays stay there; no pass writes them, so they load before the wait for the rows
  // pass
  const float2 kh = __ldcs(pkh + q);
  const float aih = kh.x, ajh = kh.y;
  // In the MC family D is the discrete upwinding of K: d_ij = -max(k_ij, 0, k_ji), so
  // 2|d_ij| = 2 max(0, k_ij, k_ji) and its high part, twice the larger high part, is exact
  // (rounding to float is monotone), and no copy of it is read.
  const float d2h = 2.f * fmaxf(fmaxf(aih, 0.f), ajh);
  pdl_wait();
  const float2 ui = up[i], uj = up[j];
  const float2 bi = abh[i], bj = abh[j];
  float2 c;
  if (pair_clip(q, pkl, abl, i, j, d2h, aih, ajh, ui, uj, bi, bj, c)) {
    c_up[q] = c;
    // the pair's bit at both ends: offset index Kup + 1 + ku at row i, Kup - 1 - ku
    // (the offset -o back to i) at row j
    clip_set(clip, i, Kup + 1 + ku);
    clip_set(clip, j, Kup - 1 - ku);
  }
}

// ||res||^2 from the residual pass's block partials in k_finalize_sum's order (one
// block of 1024 threads, so the graph's control kernel, which sums the same partials
// the same way, stops alike), launched as the pass's dependent: it waits for the pass.
__global__ void k_mcp_finalize(const double* __restrict__ part, int n, double* __restrict__ out) {
  pdl_wait();
  block_sum_to(strided_sum_1024(part, n, threadIdx.x), out);
}

// At 32 registers (8 blocks of 256 per SM) the 15-offset pass runs without spills and
// 25 % faster than at 48; the 27-offset pass would spill there and keeps its registers.
template <int KT>
__global__ void __launch_bounds__(kBlock, KT == 27 ? 1 : 8) k_mcp_residual(int64_t N, Offsets of, int limiter,
                                                         const MaskWord<KT>* __restrict__ clip,
                                                         const float2* __restrict__ c_up,
                                                         const float2* __restrict__ yp, const uint8_t* __restrict__ dir,
                                                         double* __restrict__ res, double* __restrict__ part) {
  const int K = KT > 0 ? KT : of.K, Kup = K / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool isdir = i < N && dir[i];
  pdl_wait();
  float qh = 0.f, ql = 0.f;   // res^2 as an unnormalised pair
  bool big = false;           // |res| >= 2^60: the block sums res^2 in double
  double rv = 0.0;
  if (i < N) {
    if (!isdir) {
      const float2 y = __ldcs(yp + i);
      float sh = y.x, sl = y.y;
      if (limiter == AFC_LIM_MC) {
        // pairs with a clipped amount: bit k of `bits` for offset index k
        unsigned long long bits = clip[i];
        if (KT > 0) {
          // every clipped amount of the row loaded at once (predicated), then summed in
          // offset order: res -= c_ij, with c_ij the stored amount of an upper pair
          // (k > Kup) and the negative of a lower one's (stored at its lower row i + o_k)
          constexpr int KL = KT > 0 ? KT : 1;
          float2 cv[KL];
#pragma unroll
          for (int k = 0; k < KL; ++k) {
            cv[k] = make_float2(0.f, 0.f);
            if (k != Kup && ((bits >> k) & 1ull))
              cv[k] = k > Kup ? __ldcs(c_up + (int64_t)(k - Kup - 1) * N + i)
                              : __ldcs(c_up + (int64_t)(Kup - 1 - k) * N + i + of.o[k]);
          }
#pragma unroll
          for (int k = 0; k < KL; ++k) {
            if (k == Kup || !((bits >> k) & 1ull)) continue;
            const float ch = k > Kup ? -cv[k].x : cv[k].x, cl = k > Kup ? -cv[k].y : cv[k].y;
            float s, e;
            two_sum(sh, ch, s, e);
            sh = s;
            sl = __fadd_rn(sl, __fadd_rn(e, cl));
          }
        } else {
          while (bits) {
            const int k = __ffsll(bits) - 1;
            bits &= bits - 1;
            float2 c;
            if (k > Kup) {
              c = c_up[(int64_t)(k - Kup - 1) * N + i];
              c.x = -c.x;
              c.y = -c.y;
            } else {
              c = c_up[(int64_t)(Kup - 1 - k) * N + i + of.o[k]];
            }
            float s, e;
            two_sum(sh, c.x, s, e);
            sh = s;
            sl = __fadd_rn(sl, __fadd_rn(e, c.y));
          }
        }
      }
      float h, l;
      two_sum(sh, sl, h, l);
      rv = widen_exact(h) + widen_exact(l);
      big = !(fabsf(h) < 1.152921504606846976e18f);   // 2^60 (and NaN)
      float e;
      two_prod(h, h, qh, e);
      ql = __fmaf_rn(__fadd_rn(h, h), l, e);
    }
    res[i] = rv;
  }
  // the block's sum of res^2 in pairs: the threads' pairs by columns in warp 0, as
  // block_sum_to does in double; with a |res| >= 2^60 in the block (res^2 near the
  // float range), in double by block_sum_to
  __shared__ float2 sq[kBlock];
  sq[threadIdx.x] = make_float2(qh, ql);
  if (__syncthreads_or(big)) {
    block_sum_to(rv * rv, part);
  } else if (threadIdx.x < 32) {
    float th = 0.f, tl = 0.f;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) {
      const float2 v = sq[threadIdx.x + 32 * w];
      float s, e;
      two_sum(th, v.x, s, e);
      th = s;
      tl = __fadd_rn(tl, __fadd_rn(e, v.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, th, o), ol = __shfl_down_sync(0xffffffffu, tl, o);
      float s, e;
      two_sum(th, oh, s, e);
      th = s;
      tl = __fadd_rn(tl, __fadd_rn(e, ol));
    }
    if (threadIdx.x == 0) {
      float h, l;
      two_sum(th, tl, h, l);
      part[blockIdx.x] = widen_exact(h) + widen_exact(l);
    }
  }
}

// Pair copies of the stationary operator data (once, at assembly): AG, f and, per pair,
// (k_ij, k_ji) as high parts and as low parts.
__global__ void k_mcp_setup(int64_t N, Offsets of, const double* __restrict__ AG, const double* __restrict__ f,
                            const double* __restrict__ kij, const double* __restrict__ kji,
                            float2* __restrict__ AGp, float2* __restrict__ fp, float2* __restrict__ pkh,
                            float2* __restrict__ pkl) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int k = 0; k < of.K; ++k) AGp[(int64_t)k * N + i] = split_pair(AG[(int64_t)k * N + i]);
  fp[i] = split_pair(f[i]);
  for (int ku = 0; ku < of.Kup; ++ku) {
    const int64_t q = (int64_t)ku * N + i;
    const float2 a = split_pair(kij[q]), b = split_pair(kji[q]);
    pkh[q] = make_float2(a.x, b.x);
    pkl[q] = make_float2(a.y, b.y);
  }
}

}  // namespace

int mc_pair_setup(afc_problem_s* p) {
  const int64_t N = p->N;
  int st;
  if ((st = p->AGp.alloc(p->K * N)) || (st = p->fp2.alloc(N, p->pad)) || (st = p->pk_hi.alloc(p->Kup * N)) ||
      (st = p->pk_lo.alloc(p->Kup * N)) ||
      (st = p->up2.alloc(N, p->pad)) || (st = p->abh2.alloc(N, p->pad)) || (st = p->abl2.alloc(N, p->pad)) ||
      (st = p->yp2.alloc(N, p->pad)) ||
      (st = p->cp_up.alloc(p->Kup * N)))
    return st;
  if (p->K <= 16) {
    // clip16 without a halo and with one entry more, so that it starts 4-byte aligned and
    // the word holding row N - 1 lies inside it
    if ((st = p->mask16.alloc(N)) || (st = p->clip16.alloc(N + 1))) return st;
    AFC_LAUNCH(p, "k_mcp_mask_narrow",
               k_mcp_mask_narrow<<<grid_for(N), kBlock, 0, p->stream>>>(N, p->mask.p, p->mask16.p));
  } else if (p->K <= 32) {
    if ((st = p->mask32.alloc(N)) || (st = p->clip32.alloc(N, p->pad))) return st;
    AFC_LAUNCH(p, "k_mcp_mask_narrow",
               k_mcp_mask_narrow<<<grid_for(N), kBlock, 0, p->stream>>>(N, p->mask.p, p->mask32.p));
  }
  AFC_LAUNCH(p, "k_mcp_setup", k_mcp_setup<<<grid_for(N), kBlock, 0, p->stream>>>(
                                   N, p->offs, p->AG.p, p->f.p, p->kij_up.p, p->kji_up.p, p->AGp.p, p->fp2.p,
                                   p->pk_hi.p, p->pk_lo.p));
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}


int mc_pair_residual(afc_problem_s* p, const double* u, int limiter, double* res, double* normsq_slot) {
  const int64_t N = p->N;
  const int64_t g = grid_for(N);
  cudaStream_t s = p->stream;
  // programmatic dependent launch between the passes, except while a graph is being
  // captured (the solve's graphs keep plain launches)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  AFC_CUDA(cudaStreamIsCapturing(s, &cap));
  const bool pdl = cap == cudaStreamCaptureStatusNone;
  AFC_LAUNCH(p, "k_mcp_split", k_mcp_split<<<g, kBlock, 0, s>>>(N, u, p->up2.p));
  AFC_CUDA(cudaGetLastError());
  int st = AFC_OK;
  with_K(p->K, [&](auto kc) {
    constexpr int KT = decltype(kc)::value;
    using M = MaskWord<KT>;
    const M* mask;
    M* clip;
    if constexpr (std::is_same_v<M, uint16_t>) {
      mask = p->mask16.p;
      clip = p->clip16.p;
    } else if constexpr (std::is_same_v<M, unsigned>) {
      mask = p->mask32.p;
      clip = p->clip32.p;
    } else {
      mask = p->mask.p;
      clip = p->clip.p;
    }
    cudaError_t e;
    AFC_LAUNCH(p, "k_mcp_rows", e = launch_pass(pdl, k_mcp_rows<KT>, dim3((unsigned)g), dim3(kBlock), s, N, p->offs,
                                                mask, (const float2*)p->up2.p,
                                                (const float2*)p->AGp.p, (const float2*)p->fp2.p, p->yp2.p, p->abh2.p,
                                                p->abl2.p, clip));
    if (e != cudaSuccess) { st = cuda_fail(e, "launch k_mcp_rows"); return; }
    if (limiter == AFC_LIM_MC) {
      AFC_LAUNCH(p, "k_mcp_edges",
                 e = launch_pass(pdl, k_mcp_edges<KT>, dim3((unsigned)grid_for(N, 32)), dim3(32, p->Kup), s, N, p->offs,
                                 (const float2*)p->pk_hi.p, (const float2*)p->pk_lo.p, (const float2*)p->up2.p,
                                 (const float2*)p->abh2.p, (const float2*)p->abl2.p, p->cp_up.p, clip));
      if (e != cudaSuccess) { st = cuda_fail(e, "launch k_mcp_edges"); return; }
    }
    AFC_LAUNCH(p, "k_mcp_residual",
               e = launch_pass(pdl, k_mcp_residual<KT>, dim3((unsigned)g), dim3(kBlock), s, N, p->offs, limiter,
                               (const M*)clip, (const float2*)p->cp_up.p, (const float2*)p->yp2.p,
                               (const uint8_t*)p->dir.p, res, p->part.p));
    if (e != cudaSuccess) { st = cuda_fail(e, "launch k_mcp_residual"); return; }
    if (normsq_slot) {
      AFC_LAUNCH(p, "k_mcp_finalize", e = launch_pass(pdl, k_mcp_finalize, dim3(1), dim3(1024), s,
                                                      (const double*)p->part.p, (int)g, normsq_slot));
      if (e != cudaSuccess) st = cuda_fail(e, "launch k_mcp_finalize");
    }
  });
  if (st) return st;
  AFC_CUDA(cudaGetLastError());
  return AFC_OK;
}

}  // namespace afc
