// Device helpers shared by the kernels of the EREM library: warp and block
// reductions, deterministic cross-block partial sums, vector loads and
// stores of the padded layout, exact float -> double conversion, the Leja
// stopping test and the control-block bookkeeping of one Leja substep.
//
// Included by kernels.cu (one translation unit); everything sits in an
// anonymous namespace inside erem.
#pragma once

#include "erem_internal.h"

namespace erem {
namespace {

constexpr int NT = kThreads;

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reduction over BS threads with linear index tid; the result is
// valid in tid 0.  OP 0 = sum, 1 = min, 2 = max.  Safe to call repeatedly
// (syncs before reusing smem).
template <int OP, int BS>
__device__ double block_reduce_t(double v, double* sh, int tid) {
  v = OP == 0 ? warp_sum(v) : (OP == 1 ? warp_min(v) : warp_max(v));
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    double w = tid < (BS / 32) ? sh[tid] : (OP == 0 ? 0.0 : (OP == 1 ? INFINITY : -INFINITY));
    w = OP == 0 ? warp_sum(w) : (OP == 1 ? warp_min(w) : warp_max(w));
    v = w;
  }
  return v;
}
template <int OP>
__device__ double block_reduce(double v, double* sh) {
  return block_reduce_t<OP, NT>(v, sh, threadIdx.x);
}

// Publish this block's partials (block bid of nblocks); returns true in every
// thread of the last block to arrive.  part has kRedSlots doubles per block.
__device__ bool publish_partials_t(double* part, unsigned* cnt, const double* vals, int nv,
                                   int tid, int bid, int nblocks) {
  __shared__ int s_last;
  if (tid == 0) {
    for (int k = 0; k < nv; ++k) part[bid * kRedSlots + k] = vals[k];
    __threadfence();
    const unsigned t = atomicAdd(cnt, 1u);
    s_last = (t == (unsigned)nblocks - 1u);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}
__device__ bool publish_partials(double* part, unsigned* cnt, const double* vals, int nv) {
  return publish_partials_t(part, cnt, vals, nv, threadIdx.x, blockIdx.x, gridDim.x);
}

// Sum (or min/max) of partial k over all blocks, in block order; tid 0.
template <int OP, int BS>
__device__ double gather_partials_t(const double* part, int k, double* sh, int tid, int nblocks) {
  double v = OP == 0 ? 0.0 : (OP == 1 ? INFINITY : -INFINITY);
  for (int b = tid; b < nblocks; b += BS) {
    const double x = __ldcg(part + b * kRedSlots + k);
    v = OP == 0 ? v + x : (OP == 1 ? fmin(v, x) : fmax(v, x));
  }
  return block_reduce_t<OP, BS>(v, sh, tid);
}
template <int OP>
__device__ double gather_partials(const double* part, int k, double* sh) {
  return gather_partials_t<OP, NT>(part, k, sh, threadIdx.x, gridDim.x);
}

// Arm the control block for a new Leja substep.
__device__ __forceinline__ void arm_ctrl(Ctrl* c, const StopParams& sp) {
  c->done = 0;
  c->degree = 0;
  c->fail = 0;
  c->nonfinite = 0;
  c->m_last = 0;
  c->stop_m = 0x3fffffff;
  c->err = 0.0;
  c->sp = sp;
}

// ---------------------------------------------------------------------------
// vector access to the padded layout
// ---------------------------------------------------------------------------
template <typename Tq, int VEC> struct VecT;
template <> struct VecT<float, 4> { using V = float4; };
template <> struct VecT<float, 2> { using V = float2; };
template <> struct VecT<double, 2> { using V = double2; };

template <typename Tq, int VEC>
__device__ __forceinline__ void ldv(Tq (&r)[VEC], const Tq* p) {
  using V = typename VecT<Tq, VEC>::V;
  const V v = *reinterpret_cast<const V*>(p);
  const Tq* s = reinterpret_cast<const Tq*>(&v);
#pragma unroll
  for (int k = 0; k < VEC; ++k) r[k] = s[k];
}
template <typename Tq, int VEC>
__device__ __forceinline__ void ldv_stream(Tq (&r)[VEC], const Tq* p) {
  using V = typename VecT<Tq, VEC>::V;
  const V v = __ldcs(reinterpret_cast<const V*>(p));
  const Tq* s = reinterpret_cast<const Tq*>(&v);
#pragma unroll
  for (int k = 0; k < VEC; ++k) r[k] = s[k];
}
template <typename Tq, int VEC>
__device__ __forceinline__ void stv(Tq* p, const Tq (&r)[VEC]) {
  using V = typename VecT<Tq, VEC>::V;
  V v;
  Tq* d = reinterpret_cast<Tq*>(&v);
#pragma unroll
  for (int k = 0; k < VEC; ++k) d[k] = r[k];
  *reinterpret_cast<V*>(p) = v;
}
// VEC doubles of P, streamed (read once, written once per term)
template <int VEC>
__device__ __forceinline__ void ldP(double (&r)[VEC], const double* p) {
#pragma unroll
  for (int k = 0; k < VEC; k += 2) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p + k));
    r[k] = v.x;
    r[k + 1] = v.y;
  }
}
template <int VEC>
__device__ __forceinline__ void stP(double* p, const double (&r)[VEC]) {
#pragma unroll
  for (int k = 0; k < VEC; k += 2) __stcs(reinterpret_cast<double2*>(p + k), make_double2(r[k], r[k + 1]));
}

// float -> double, exact, from the bit fields with integer instructions
// only (the FP64 pipe of GB300 is the scarce unit in the FP32-bulk sweep, and
// a hardware conversion kept for rare inputs is if-converted into one that
// every call executes): normal numbers, infinities and NaNs by widening the
// fields, zeros by their sign, and a subnormal f through 2^24 f (an exact
// FP32 product, and a normal number) with 24 taken off the exponent.
__device__ __forceinline__ double f2d_fast(float f) {
  const unsigned e0 = (__float_as_uint(f) >> 23) & 0xffu;
  const float g = e0 == 0u ? f * 16777216.0f : f;
  const unsigned u = __float_as_uint(g);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned E = e == 0xffu ? 0x7ffu : e + (e0 == 0u ? 872u : 896u);
  const unsigned hi = e == 0u ? (u & 0x80000000u)
                              : (u & 0x80000000u) | (E << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lo = e == 0u ? 0u : u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// |x| as ordered bits (for |x| the order of the bits is the order of the
// values) and a finiteness test on them: integer operations only.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ bool bits_finite(unsigned long long b) {
  return (b >> 52) != 0x7ffULL;
}

// The Leja copy of J is interleaved per warp tile of T = 32 VEC cells: the
// tile's NC coefficient arrays D W E S N (B T) follow one another, T values
// each.  A warp whose lanes own 32 consecutive VEC-cell vectors reads each
// coefficient as one contiguous 512-byte run, and the NC runs of a tile are
// adjacent in memory (one stream instead of NC).  c[k] points at coefficient
// k of tile 0; the vector starting at cell i reads c[k] + leja_off(i).
template <typename Tq>
struct LejaCoef {
  const Tq* c[7];
  int nc;
  // diagonal-free copy (c[0] unused): the row sum of each x = 0 cell, one per
  // (y, z) row; every other row of J sums to zero (a uniform temperature is
  // transported nowhere in the interior)
  const Tq* r0;
};
template <int T>
__device__ __forceinline__ size_t leja_off(int i, int nc) {
  return (size_t)i + (size_t)(i / T) * (size_t)(nc - 1) * T;
}

// Stopping test of §4.2 on the estimate of term m (thread 0 of the last block).
__device__ void stop_test(Ctrl* c, int m, double dm, double S) {
  const StopParams sp = c->sp;
  const double scal = sp.tol_a + sp.tol_r * c->yinf;
  const double e = fabs(sp.delta * dm) / scal * sqrt(S / sp.ncells);
  c->e[m] = e;
  c->m_last = m;
  if (!isfinite(e)) {
    c->nonfinite = 1;
    c->done = 1;
    return;
  }
  const int lo = max(1, m - sp.window + 1);
  double mean = 0.0;
  for (int k = lo; k <= m; ++k) mean += c->e[k];
  mean /= (double)(m - lo + 1);
  c->err = mean;
  if (sp.replay) return;
  if (sp.pow10 * mean < 1.0) {
    c->done = 1;
    c->degree = m;
  } else if (m >= sp.m_max) {
    c->fail = 1;
    c->done = 1;
  }
}

template <typename Tq>
__device__ __forceinline__ double to_f64_fast(Tq v) {
  if constexpr (sizeof(Tq) == 4) return f2d_fast(v);
  else return v;
}

}  // namespace
}  // namespace erem
