// Small device helpers shared by the hot-path kernels.
#pragma once

#include <type_traits>

#include "afc_internal.h"

namespace afc {

// m_ij and d_ij of the pair (i, i + o_k), k != Kup.  Stored once per pair at the
// row of the pair's lower node, offset index ku of the positive offset |o_k|.
__device__ __forceinline__ void pair_coef(const Offsets& of, int k, int64_t i, int64_t N,
                                          const double* __restrict__ m_up, const double* __restrict__ d_up,
                                          double& m, double& d) {
  int64_t q;
  if (k > of.Kup) q = (int64_t)(k - of.Kup - 1) * N + i;
  else q = (int64_t)(of.Kup - 1 - k) * N + i + of.o[k];
  m = m_up[q];
  d = d_up[q];
}

__device__ __forceinline__ double pair_d(const Offsets& of, int k, int64_t i, int64_t N,
                                         const double* __restrict__ d_up) {
  if (k > of.Kup) return d_up[(int64_t)(k - of.Kup - 1) * N + i];
  return d_up[(int64_t)(of.Kup - 1 - k) * N + i + of.o[k]];
}

// ---- comparisons on the integer pipe ----------------------------------------
// GB300 runs FP64 compares, min/max and arithmetic on a pipe that issues 2 thread
// operations per SM and cycle.  Comparisons of finite doubles are done here on
// their bit patterns instead: key() maps a double to an int64 with the same
// order (-0 sorts just below +0), so every decision below is exact.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }      // x > 0
__device__ __forceinline__ bool lt0(double x) { return dkey(x) < -1; }                      // x < 0
__device__ __forceinline__ bool is0(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ double imin(double a, double b) { return dkey(a) <= dkey(b) ? a : b; }
__device__ __forceinline__ double imax(double a, double b) { return dkey(a) >= dkey(b) ? a : b; }
// keys are their own inverse: key(key(x)) = x
__device__ __forceinline__ double from_key(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// Exact float -> double on the integer pipe (every user of a flux widens it the same
// way, so P+/- and F* see the same values).  A subnormal float m * 2^-149 becomes the
// normal double 2^(p - 149) (m / 2^p), p the position of m's leading bit.
__device__ __forceinline__ double widen_exact(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  const unsigned long long s = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u) {
    if (m == 0u) return __longlong_as_double((long long)s);
    const unsigned p = 31u - (unsigned)__clz(m);   // 0 .. 22
    return __longlong_as_double(
        (long long)(s | ((unsigned long long)(p + 874u) << 52) | ((unsigned long long)(m ^ (1u << p)) << (52u - p))));
  }
  const unsigned long long de = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(s | (de << 52) | ((unsigned long long)m << 29)));
}

// Sums of the positive and of the negative values of a row's pair fluxes, exact:
// every mantissa is placed in a 128-bit fixed point scaled to the largest exponent
// (its mantissa at bits 64..116, so up to 2^10 terms cannot overflow), the words are
// added with carry on the integer pipe, and each total is rounded to double once.
// Subnormal inputs count as zero.  On GB300 this replaces two FP64 adds per value (an
// FP64 warp instruction occupies the pipe for 16 cycles) with about a dozen integer
// instructions, and is more accurate.  The values are taken one at a time, so that
// none has to be kept: the totals are held scaled to the largest exponent seen so
// far, and a value with a larger exponent first shifts both totals right (the bits
// that leave the 128-bit range are below 2^-64 of the new largest value's last
// bit).  A row of 26 pair fluxes then needs no 52 registers to hold its bit
// patterns until its largest exponent is known.
struct SignedFixedSums {
  unsigned emax = 0u;
  unsigned long long ph = 0ull, pl = 0ull, nh = 0ull, nl = 0ull;

  __device__ static __forceinline__ void shr128(unsigned long long& h, unsigned long long& l, unsigned d) {
    if (d >= 128u) {
      h = 0ull;
      l = 0ull;
    } else if (d >= 64u) {
      l = h >> (d - 64u);
      h = 0ull;
    } else {
      l = (l >> d) | (h << (64u - d));
      h >>= d;
    }
  }
  __device__ __forceinline__ void add(unsigned long long b) {
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    if (e == 0u) return;
    if (e > emax) {
      if (emax != 0u) {
        shr128(ph, pl, e - emax);
        shr128(nh, nl, e - emax);
      }
      emax = e;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = (int)e - (int)emax + 64;   // <= 64
    unsigned long long lo, hi;
    if (sh >= 64) {
      lo = 0ull;
      hi = m;
    } else if (sh > 0) {
      lo = m << sh;
      hi = m >> (64 - sh);
    } else if (sh > -64) {
      lo = m >> (-sh);
      hi = 0ull;
    } else {
      lo = 0ull;
      hi = 0ull;
    }
    if (b >> 63) {
      nl += lo;
      nh += hi + (nl < lo ? 1ull : 0ull);
    } else {
      pl += lo;
      ph += hi + (pl < lo ? 1ull : 0ull);
    }
  }
  // The totals rounded to double (nearest, ties to even) on the integer pipe; value
  // = (h:l) * 2^(emax - 1139).  Totals whose double would be subnormal or overflow
  // take the FP64 route in a separate function.
  __device__ __forceinline__ void result(double& pos, double& neg) const {
    if (emax == 0u) {
      pos = 0.0;
      neg = 0.0;
      return;
    }
    const int ex = (int)emax - 1139;
    pos = to_double(ph, pl, ex);
    neg = neg_bits(to_double(nh, nl, ex));
  }
  __device__ static __noinline__ double to_double_fp64(unsigned long long h, unsigned long long l, int ex) {
    const double two64 = 18446744073709551616.0;
    return scalbn(fma(__ull2double_rn(h), two64, __ull2double_rn(l)), ex);
  }
  __device__ static __forceinline__ double to_double(unsigned long long h, unsigned long long l, int ex) {
    if ((h | l) == 0ull) return 0.0;
    const int lz = h != 0ull ? __clzll((long long)h) : 64 + __clzll((long long)l);
    unsigned long long nh, nl;   // normalised: bit 127 set
    if (lz >= 64) {
      nh = l << (lz - 64);
      nl = 0ull;
    } else if (lz > 0) {
      nh = (h << lz) | (l >> (64 - lz));
      nl = l << lz;
    } else {
      nh = h;
      nl = l;
    }
    unsigned long long m = nh >> 11;   // 53 bits, the leading one at bit 52
    const bool half = (nh >> 10) & 1ull;
    const bool sticky = ((nh & 0x3FFull) | nl) != 0ull;
    if (half && (sticky || (m & 1ull))) ++m;
    int e2 = 127 + ex - lz;            // exponent of the leading bit
    if (m >> 53) {
      m >>= 1;
      ++e2;
    }
    const int be = e2 + 1023;
    if (be <= 0 || be >= 2047) return to_double_fp64(h, l, ex);
    return __longlong_as_double((long long)(((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
  }
};

// min / max of two values known to be >= 0 (correction factors, bounds): plain int compare
__device__ __forceinline__ double imin_nn(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b) ? a : b;
}
// Exact 0.5 * x (IEEE, ties to even) on the integer pipe.  Normal numbers above the
// smallest binade move their exponent; zeros, subnormals and the smallest binade
// halve the 53-bit significand with round-half-even; Inf and NaN pass through.  No
// branch issues an FP64 instruction, so none costs the FP64 pipe even when the
// compiler evaluates both sides of a branch.
__device__ __forceinline__ double half_exact(double x) {
  const long long b = __double_as_longlong(x);
  const long long e = (b >> 52) & 0x7ff;
  if (e > 1 && e < 0x7ff) return __longlong_as_double(b - (1LL << 52));
  if (e == 0x7ff) return x;
  const long long sign = b & (long long)0x8000000000000000ULL;
  const unsigned long long M = (unsigned long long)(b & 0x000FFFFFFFFFFFFFLL) | (e == 1 ? (1ULL << 52) : 0ULL);
  unsigned long long h = M >> 1;
  if ((M & 1ULL) && (h & 1ULL)) ++h;   // exactly half-way: to even (may carry into the exponent)
  return __longlong_as_double(sign | (long long)h);
}

// R = min{1, num / den} of Zalesak's step 3 for num = m_i Q, den = dt P of the same sign,
// R = 1 if P = 0.  For same-sign num, den the rounded quotient reaches 1 exactly when
// |num| >= |den|, so the division is only done where R < 1 (same result bit for bit).
__device__ __forceinline__ double zalesak_factor(double num, double den) {
  if (is0(den)) return 1.0;
  const long long an = __double_as_longlong(num) & 0x7fffffffffffffffLL;
  const long long ad = __double_as_longlong(den) & 0x7fffffffffffffffLL;
  if (an >= ad) return 1.0;
  return num / den;
}

// minmod of Eq. prelimiting: 0 unless both arguments have the same strict sign.
__device__ __forceinline__ double minmod(double a, double b) {
  if (gt0(a) && gt0(b)) return imin(a, b);
  if (lt0(a) && lt0(b)) return imax(a, b);
  return 0.0;
}

// The antidiffusive flux of the pair (i, i + o_k) seen from row i, for a flux
// stored once per pair at the pair's lower row: r_ij = r_e (k > Kup) or -r_e.
__device__ __forceinline__ double pair_flux(const Offsets& of, int Kup, int k, int64_t i, int64_t N,
                                            const double* __restrict__ r_up) {
  if (k > Kup) return r_up[(int64_t)(k - Kup - 1) * N + i];
  return neg_bits(r_up[(int64_t)(Kup - 1 - k) * N + i + of.o[k]]);   // -r_e, sign bit on the integer pipe
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums in a fixed order.  On GB300 every FP64 warp instruction costs the
// FP64 pipe 16 cycles whatever its active lanes, so a shuffle tree in every warp
// (5 adds per warp) is the expensive way to sum a block.  Instead every thread
// stores its value in shared memory and warp 0 alone sums them: each lane adds
// blockDim/32 values, then one shuffle tree (blockDim/32 - 1 + 5 adds per block
// instead of 5 per warp).  Blocks of more than kBlock threads take the shuffle
// route.  Every thread of the block must call these.
__device__ __forceinline__ double warp0_column_sum(const double* col) {
  const int lane = threadIdx.x;   // < 32
  double t = col[lane];
  for (int w = lane + 32; w < (int)blockDim.x; w += 32) t += col[w];
  return warp_sum(t);
}

// The final sums over a pass's block partials run as 1024 threads: thread t adds
// part[t], part[t + 1024], part[t + 2048], ... (q < n) from left to right, then the
// block sums the threads (block_sum_to).  This is thread t's sum; its loads go out
// eight at a time instead of one round trip each.  A slot past n adds +0.0, which
// leaves the sum unchanged (it starts at +0.0, so it is never -0.0).  The loads go
// through L2 (partials of other blocks of the same grid are read this way too).
__device__ __forceinline__ double strided_sum_1024(const double* part, int n, int t) {
  double v = 0.0;
  for (int q0 = t; q0 < n; q0 += 8 * 1024) {
    double x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = q0 + 1024 * m < n ? __ldcg(part + q0 + 1024 * m) : 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m) v += x[m];
  }
  return v;
}

// Sum v over the block and store it in part[blockIdx.x].
__device__ __forceinline__ void block_sum_to(double v, double* part) {
  __shared__ double sh[kBlock];
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
      if (lane == 0) part[blockIdx.x] = t;
    }
    __syncthreads();
    return;
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double t = warp0_column_sum(sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
  __syncthreads();
}

// Several sums at once (NV values per thread), stored at part[q * stride + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_sums_to(double (&v)[NV], double* part, int64_t stride) {
  if (blockDim.x > kBlock) {
#pragma unroll
    for (int q = 0; q < NV; ++q) block_sum_to(v[q], part + q * stride);
    return;
  }
  __shared__ double sh[NV][kBlock];
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double t = warp0_column_sum(sh[q]);
      if (threadIdx.x == 0) part[q * stride + blockIdx.x] = t;
    }
  }
  __syncthreads();
}

// Run f(std::integral_constant<int, K>) with K fixed at compile time for the two
// structured patterns (15 offsets: Kuhn P1, 27: Q1) so that the per-row loops
// unroll completely and all loads of a row are in flight together; 0 = any K.
template <class F>
inline void with_K(int K, F&& f) {
  if (K == 15) f(std::integral_constant<int, 15>{});
  else if (K == 27) f(std::integral_constant<int, 27>{});
  else f(std::integral_constant<int, 0>{});
}

// Programmatic dependent launch between consecutive passes: a pass lets the next one
// launch as soon as all of its blocks run (griddepcontrol.launch_dependents), and the
// next pass issues the loads of data no earlier pass writes before it waits for its
// predecessor's results (griddepcontrol.wait), so those loads overlap the predecessor's
// last wave.  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch kernel k with programmatic dependent launch on `pdl`.
template <class... KArgs, class... Args>
inline cudaError_t launch_pass(bool pdl, void (*k)(KArgs...), dim3 g, dim3 b, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// out[0] = sum of part[0..n) in a fixed order (one block).
void finalize_sum(afc_problem_s* p, const double* part, int n, double* out);

}  // namespace afc
