// The batched ensemble kernel: every member of an ensemble of independent 2D
// problems is run, step after step, by one thread-block cluster.
//
// A persistent grid of clusters takes members from a queue (heaviest first,
// the order the host writes) and runs each one through all the steps of the
// run as the state machine of erem_internal.h: G(T^n), the Leja terms with
// the stopping test of §4.2, the substep bookkeeping and T^{n+1}.  Every
// pass over the member's cells ends at the cluster barrier; the pass's
// reduced value (the sum of q_m^2, or ||T^n||_inf) travels through
// distributed shared memory, and every CTA of the cluster sums the CTAs'
// partials in rank order, so every CTA holds the same bits and takes the same
// decision.  Nothing waits on another cluster: clusters share only the queue
// counter.
//
// A member's Leja working set (its Leja copy of J, q_{m-1}, q_m and P: 36 B
// a cell in FP32-bulk) stays in L2 while its cluster works on it.  Values
// another CTA of the cluster wrote in an earlier pass (q, T, w at neighbour
// cells) are loaded past L1 (ld.global.cg); values a thread wrote itself (P,
// G, w and T at its own cells) and the read-only coefficients use ordinary
// loads.
#include <cooperative_groups.h>

#include "erem_internal.h"
#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace erem {
namespace {

constexpr int kEnsThreads = 512;  // threads per CTA

template <typename Tq, int VEC>
__device__ __forceinline__ void ldv_l2(Tq (&r)[VEC], const Tq* p) {
  using V = typename VecT<Tq, VEC>::V;
  const V v = __ldcg(reinterpret_cast<const V*>(p));
  const Tq* s = reinterpret_cast<const Tq*>(&v);
#pragma unroll
  for (int k = 0; k < VEC; ++k) r[k] = s[k];
}
template <int VEC>
__device__ __forceinline__ void ld2(double (&r)[VEC], const double* p) {
#pragma unroll
  for (int k = 0; k < VEC; k += 2) {
    const double2 v = *reinterpret_cast<const double2*>(p + k);
    r[k] = v.x;
    r[k + 1] = v.y;
  }
}
template <int VEC>
__device__ __forceinline__ void ld2_l2(double (&r)[VEC], const double* p) {
#pragma unroll
  for (int k = 0; k < VEC; k += 2) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p + k));
    r[k] = v.x;
    r[k + 1] = v.y;
  }
}
template <int VEC>
__device__ __forceinline__ void st2(double* p, const double (&r)[VEC]) {
#pragma unroll
  for (int k = 0; k < VEC; k += 2) *reinterpret_cast<double2*>(p + k) = make_double2(r[k], r[k + 1]);
}

// a = J x at the VEC cells from i (FP64 cell form D W E S N; x at the
// neighbours written by other CTAs, so loaded past L1)
template <int VEC>
__device__ __forceinline__ void ens_apply_J(const EnsMember& M, const double* x, int i, int row,
                                            int ix, double (&a)[VEC]) {
  double xc[VEC], xs[VEC], xn[VEC], c[5][VEC];
  ld2_l2<VEC>(xc, x + i);
  ld2_l2<VEC>(xs, x + i - (row > 0 ? M.px : 0));
  ld2_l2<VEC>(xn, x + i + (row < M.ny - 1 ? M.px : 0));
  const double xl = ix > 0 ? __ldcg(x + i - 1) : 0.0;
  const double xr = ix + VEC < M.px ? __ldcg(x + i + VEC) : 0.0;
#pragma unroll
  for (int k = 0; k < 5; ++k) ld2<VEC>(c[k], M.jc[k] + i);
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const double west = v == 0 ? xl : xc[v - 1];
    const double east = v == VEC - 1 ? xr : xc[v + 1];
    double y = c[0][v] * xc[v];
    y = fma(c[1][v], west, y);
    y = fma(c[2][v], east, y);
    y = fma(c[3][v], xs[v], y);
    y = fma(c[4][v], xn[v], y);
    a[v] = y;
  }
}

// INIT / SUBSTART at the two cells i, i + 1: INIT G = J T^n + b (with
// ||T^n||_inf and the non-finite check), SUBSTART q_0 = G + J w; then
// P = d_0 q_0 and q_0 in the Leja precision.
template <typename Tq>
__device__ __forceinline__ void ens_start_pair(const EnsMember& M, const double* x, int i, int row,
                                               int ix, bool init, double d0,
                                               unsigned long long& tmax, bool& bad) {
  double a[2];
  ens_apply_J<2>(M, x, i, row, ix, a);
  if (init) {
    if (ix == 0) a[0] += M.b0[row];
    double tc[2];
    ld2_l2<2>(tc, M.T + i);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const unsigned long long tb = abs_bits(tc[k]);
      tmax = tmax > tb ? tmax : tb;
      bad |= !bits_finite(tb) | !bits_finite(abs_bits(a[k]));
    }
    st2<2>(M.G + i, a);
  } else {
    double g[2];
    ld2<2>(g, M.G + i);
    a[0] += g[0];
    a[1] += g[1];
  }
  const double p[2] = {d0 * a[0], d0 * a[1]};
  const Tq o[2] = {(Tq)a[0], (Tq)a[1]};
  st2<2>(M.P + i, p);
  stv<Tq, 2>((Tq*)M.q[0] + i, o);
}

// What the compute warps do in one pass (written by the control warp one
// pass ahead, double-buffered by pass parity).
struct PassDesc {
  int phase;      // ENS_*; ENS_DONE or ENS_FAILED end the member
  int m;          // ENS_TERM: the term computed, q_m from q_{m-1}
  int sub;        // ENS_ACCUM / ENS_FINAL: the substep just finished (w is added when > 0)
  int level;      // the substep level of the pass
  double shift;   // ENS_TERM: c/gamma + xi_{m-1}
  double dprev;   // ENS_TERM, m >= 2: d_{m-1} (P += d_{m-1} q_{m-1}, one term behind)
  double dm;      // ENS_TERM: d_m, for the estimate e_m
  double d0, delta;  // d_0 and dt / 2^level of the level
};

// The member's state machine, kept by lane 0 of the control warp of every
// CTA (identical copies).
struct EnsCtl {
  int level, sub, step, target, status, terms, attempts, last_S;
  int junk;       // the pass in flight is a term past a decided stop or failure
  int pad;
  long long n_pass, pass_bound;  // passes issued, and their bound
  double yinf;                   // ||T^n||_inf of the step
  int cur_deg[64], last_deg[64];
  double e[kEnsWin];             // error estimates e_m, ring of kEnsWin
};

constexpr int kEnsWarps = kEnsThreads / 32;  // warps per CTA
constexpr int kEnsTab = 1280;  // doubles of divided differences and Leja points kept in shared memory
constexpr int kEnsWork = kEnsThreads - 32;   // threads of the compute warps (all but the last)

// The descriptor of a pass of phase `phase` (TERM: term m) at the state's
// level.
__device__ PassDesc ens_desc(const EnsCtl& c, const EnsMember& M, const double* dd_all,
                             const double* xi, int mmax, int phase, int m) {
  PassDesc d;
  const double* dd = dd_all + (size_t)c.level * (mmax + 1);
  d.phase = phase;
  d.m = m;
  d.sub = c.sub;
  d.level = c.level;
  d.d0 = dd[0];
  d.delta = M.dt * (1.0 / (double)(1 << c.level));  // exact: a power of two
  d.shift = 0.0;
  d.dprev = 0.0;
  d.dm = 0.0;
  if (phase == ENS_TERM) {
    d.shift = M.cg + xi[m - 1];
    d.dprev = m >= 2 ? dd[m - 1] : 0.0;
    d.dm = m <= mmax ? dd[m] : 0.0;  // m = m_max + 1 is only ever a term past the decision
  }
  return d;
}

// Control step, taken by lane 0 of the control warp while the compute warps
// run pass j (descriptor cur): the outcome of pass j - 1 (descriptor prev,
// reduced value v0 and non-finite flag bad) is known; decide the pass
// j + 1.  A term's pass is issued before the stopping test of the term
// before it has run (the test runs here, one pass later); the pass that
// follows a stop at term m adds d_m q_m to P and its own q_{m+1} is not
// used.
__device__ PassDesc ens_control(EnsCtl& c, const EnsMember& M, const EnsRun R, const double* dd_all,
                                const double* xi, const PassDesc& cur, const PassDesc* prev, double v0,
                                bool bad) {
  int next = -1;  // phase decided by the outcome of prev
  const int S = 1 << c.level;
  const bool prev_junk = c.junk != 0;
  c.junk = 0;
  if (prev && prev->phase == ENS_INIT) {
    if (bad) {
      c.status = ENS_NONFINITE;
      next = ENS_FAILED;
      c.junk = 1;
    } else {
      c.yinf = v0;
    }
  } else if (prev && prev->phase == ENS_TERM && !prev_junk) {
    // stopping test of §4.2 on the estimate of term m
    const StopParams& sp = M.sp;
    const int m = prev->m;
    c.terms += 1;
    const double scal = sp.tol_a + sp.tol_r * c.yinf;
    const double e = fabs(prev->delta * prev->dm) / scal * sqrt(v0 / sp.ncells);
    c.e[m % kEnsWin] = e;
    bool failed = false;
    if (!isfinite(e)) {
      failed = true;  // the Newton vectors left the range of the Leja precision
    } else {
      const int lo = max(1, m - sp.window + 1);
      double mean = 0.0;
      for (int k = lo; k <= m; ++k) mean += c.e[k % kEnsWin];
      mean /= (double)(m - lo + 1);
      if (sp.pow10 * mean < 1.0) {
        c.cur_deg[c.sub] = m;
        next = c.sub == S - 1 ? ENS_FINAL : ENS_ACCUM;
        c.junk = 1;  // pass j completes P with d_m q_m; its q_{m+1} is not used
      } else if (m >= sp.m_max) {
        failed = true;
      }
    }
    if (failed) {
      // the attempt failed: the whole step again at twice the substeps
      c.attempts += 1;
      c.junk = 1;
      if (c.level + 1 < R.nlev) {
        c.level += 1;
        next = ENS_RESTART;
      } else {
        c.status = isfinite(e) ? ENS_NOTCONV : ENS_NONFINITE;
        next = ENS_FAILED;
      }
    }
  }
  int m_next = 0;
  if (next < 0) {
    // no decision from prev: the successor of the pass in flight
    switch (cur.phase) {
      case ENS_TERM:
        next = ENS_TERM;
        m_next = cur.m + 1;
        break;
      case ENS_INIT:
      case ENS_SUBSTART:
      case ENS_RESTART:
        next = ENS_TERM;
        m_next = 1;
        break;
      case ENS_ACCUM:
        next = ENS_SUBSTART;
        c.sub += 1;
        break;
      case ENS_FINAL:
        if (c.step >= c.target) {
          next = ENS_DONE;
        } else {
          if (R.restart) c.level = 0;
          next = ENS_INIT;
        }
        break;
      default:
        next = ENS_FAILED;
        break;
    }
  }
  if (next == ENS_RESTART) c.sub = 0;
  if (next == ENS_INIT) c.sub = 0;
  if (next == ENS_FINAL) {
    const int Sl = 1 << c.level;
    c.last_S = Sl;
    for (int k = 0; k < 64; ++k) c.last_deg[k] = k < Sl ? c.cur_deg[k] : 0;
    c.step += 1;
  }
  if (next != ENS_DONE && next != ENS_FAILED) {
    if (c.n_pass >= c.pass_bound) {
      c.status = ENS_TIMEOUT;
      next = ENS_FAILED;
    } else {
      c.n_pass += 1;
    }
  }
  return ens_desc(c, M, dd_all, xi, R.mmax, next, m_next);
}

// One Leja term over the thread's vectors: q_m = ((J_l - shift) q_{m-1}) and,
// from m = 2, P += d_{m-1} q_{m-1}; returns the thread's sum of q_m^2.  Kept
// out of line so that the hot loop has the register budget to itself.
template <typename Tq, int VEC, bool ND>
__device__ __noinline__ double ens_term_pass(const EnsMember& M, const PassDesc& d, int g0, int G) {
  double r0 = 0.0;
  const int nvec = M.Np / VEC;
  const int vrow = M.px / VEC;
  const int m = d.m;
  const bool addP = m >= 2;
  const double dprev = d.dprev;
  const Tq shm = (Tq)d.shift;
  const Tq* __restrict__ qi = (const Tq*)M.q[(m - 1) & 1];
  Tq* __restrict__ qo = (Tq*)M.q[m & 1];
  const Tq* __restrict__ jl = (const Tq*)M.jl;
  double* __restrict__ P = M.P;
  for (int v = g0; v < nvec; v += G) {
    const int row = v / vrow;
    const int i = v * VEC;
    const int ix = i - row * M.px;
    Tq qc[VEC], qs[VEC], qn[VEC];
    ldv_l2<Tq, VEC>(qc, qi + i);
    ldv_l2<Tq, VEC>(qs, qi + i - (row > 0 ? M.px : 0));
    ldv_l2<Tq, VEC>(qn, qi + i + (row < M.ny - 1 ? M.px : 0));
    const Tq ql = ix > 0 ? __ldcg(qi + i - 1) : Tq(0);
    const Tq qr = ix + VEC < M.px ? __ldcg(qi + i + VEC) : Tq(0);
    // the Leja copy: D W E S N, or (ND) W E S N with the diagonal implied by
    // the row sums, zero off the x = 0 column
    Tq c[5][VEC];
    Tq rsum = Tq(0);  // ND: the row sum of an x = 0 cell
    if constexpr (ND) {
      const size_t off = leja_off<32 * VEC>(i, 4);
#pragma unroll
      for (int k = 1; k < 5; ++k) ldv<Tq, VEC>(c[k], jl + (k - 1) * 32 * VEC + off);
      if (ix == 0) rsum = (Tq)M.r0[row];
    } else {
      const size_t off = leja_off<32 * VEC>(i, 5);
#pragma unroll
      for (int k = 0; k < 5; ++k) ldv<Tq, VEC>(c[k], jl + k * 32 * VEC + off);
    }
    double p[VEC];
    if (addP) ld2<VEC>(p, P + i);
    Tq out[VEC];
    Tq sq = Tq(0);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const Tq west = k == 0 ? ql : qc[k - 1];
      const Tq east = k == VEC - 1 ? qr : qc[k + 1];
      Tq a;
      if constexpr (ND) {  // sum_j J_ij (q_j - q_i) + (r_i - shift) q_i
        a = ((k == 0 ? rsum : Tq(0)) - shm) * qc[k];
        a = fma(c[1][k], west - qc[k], a);
        a = fma(c[2][k], east - qc[k], a);
        a = fma(c[3][k], qs[k] - qc[k], a);
        a = fma(c[4][k], qn[k] - qc[k], a);
      } else {
        a = (c[0][k] - shm) * qc[k];
        a = fma(c[1][k], west, a);
        a = fma(c[2][k], east, a);
        a = fma(c[3][k], qs[k], a);
        a = fma(c[4][k], qn[k], a);
      }
      out[k] = a;
    }
    stv<Tq, VEC>(qo + i, out);
    if (addP) {  // the running sum, one term behind: P += d_{m-1} q_{m-1}
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        if constexpr (sizeof(Tq) == 4) p[k] = fma(dprev, f2d_fast(qc[k]), p[k]);
        else p[k] = fma(dprev, qc[k], p[k]);
      }
      st2<VEC>(P + i, p);
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      if constexpr (sizeof(Tq) == 4) sq = fmaf(out[k], out[k], sq);
      else r0 = fma(out[k], out[k], r0);
    }
    if constexpr (sizeof(Tq) == 4) r0 += (double)sq;
  }
  return r0;
}

template <typename Tq, int VEC>
__global__ void __launch_bounds__(kEnsThreads, 2) k_ens_cluster(EnsRun R) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const unsigned csize = cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool control = wid == kEnsWarps - 1;
  __shared__ __align__(16) EnsMember s_M;
  __shared__ EnsCtl s_c;
  __shared__ PassDesc s_d[2];
  __shared__ double s_red[2][kEnsWarps - 1][2];  // [pass parity][compute warp][value, non-finite]
  __shared__ double s_cta[2][2];                   // [pass parity][CTA value, non-finite]
  __shared__ unsigned s_cnt[2];                    // compute warps done, per pass parity
  __shared__ double s_tab[kEnsTab];                // the member's d tables and Leja points
  __shared__ int s_q;
  static_assert(sizeof(EnsMember) % 8 == 0 && sizeof(EnsMember) / 8 <= kEnsThreads, "EnsMember copy");

  const int G = (int)csize * kEnsWork;
  const int g0 = (int)rank * kEnsWork + tid;
  for (;;) {
    // the next member of the queue, drawn by CTA 0 and read by every CTA
    if (rank == 0 && tid == 0) s_q = (int)atomicAdd(R.next, 1u);
    cl.sync();
    const int q = *cl.map_shared_rank(&s_q, 0);
    cl.sync();  // CTA 0 neither rewrites s_q nor exits while it is read
    if (q >= R.n) return;
    const int e = R.order[q];
    if (tid < (int)(sizeof(EnsMember) / 8))
      reinterpret_cast<unsigned long long*>(&s_M)[tid] =
          reinterpret_cast<const unsigned long long*>(R.mem + e)[tid];
    if (tid < 2) s_cnt[tid] = 0u;
    __syncthreads();
    // the member's divided differences of every level and the Leja points in
    // shared memory when they fit (m_max up to 150 at 7 levels)
    const int ntab = R.nlev * (R.mmax + 1);
    const bool staged = ntab + R.mmax + 1 <= kEnsTab;
    if (staged) {
      for (int k = tid; k < ntab; k += kEnsThreads) s_tab[k] = s_M.dd[k];
      for (int k = tid; k <= R.mmax; k += kEnsThreads) s_tab[ntab + k] = R.xi[k];
    }
    const double* dd_all = staged ? s_tab : s_M.dd;
    const double* xi_tab = staged ? s_tab + ntab : R.xi;
    __syncthreads();
    if (control && lane == 0) {
      const EnsState& st = R.st[e];
      EnsCtl& c = s_c;
      c.level = st.level;
      c.target = st.target;
      c.sub = c.step = c.status = c.terms = c.attempts = c.last_S = c.junk = 0;
      c.n_pass = 1;
      c.pass_bound = (long long)st.target * R.passes_per_step;
      c.yinf = 0.0;
      for (int k = 0; k < 64; ++k) c.cur_deg[k] = c.last_deg[k] = 0;
      s_d[0] = ens_desc(c, s_M, dd_all, xi_tab, R.mmax, ENS_INIT, 0);
    }
    __syncthreads();
    const EnsMember& M = s_M;
    const int nvec = M.Np / VEC;
    const int vrow = M.px / VEC;

    for (int j = 0;; ++j) {
      const int par = j & 1;
      const PassDesc d = s_d[par];
      if (d.phase == ENS_DONE || d.phase == ENS_FAILED) break;
      if (!control) {
        double r0 = 0.0;
        bool bad = false;
        if (d.phase == ENS_TERM) {
          r0 = M.r0 ? ens_term_pass<Tq, VEC, true>(M, d, g0, G)
                    : ens_term_pass<Tq, VEC, false>(M, d, g0, G);
        } else if (d.phase == ENS_INIT || d.phase == ENS_SUBSTART) {
          // INIT: G = J T^n + b, q_0 = G, P = d_0 G.  SUBSTART: q_0 = G + J w.
          const double* x = d.phase == ENS_INIT ? M.T : M.w;
          unsigned long long tmax = 0ULL;
          for (int v = g0; v < nvec; v += G) {
            const int row = v / vrow;
            const int i = v * VEC;
            const int ix = i - row * M.px;
            // two cells at a time (the FP64 stencil of four cells would not fit
            // the register budget)
#pragma unroll 1
            for (int h = 0; h < VEC; h += 2)
              ens_start_pair<Tq>(M, x, i + h, row, ix + h, d.phase == ENS_INIT, d.d0, tmax, bad);
          }
          if (d.phase == ENS_INIT) r0 = __longlong_as_double((long long)tmax);
        } else {
          // cell-local passes (own cells only)
          for (int v = g0; v < nvec; v += G) {
            const int i = v * VEC;
            if (d.phase == ENS_RESTART) {
              double g[VEC], p[VEC];
              Tq o[VEC];
              ld2<VEC>(g, M.G + i);
#pragma unroll
              for (int k = 0; k < VEC; ++k) {
                p[k] = d.d0 * g[k];
                o[k] = (Tq)g[k];
              }
              st2<VEC>(M.P + i, p);
              stv<Tq, VEC>((Tq*)M.q[0] + i, o);
            } else {  // ACCUM: w = w + delta P; FINAL: T = T + w + delta P
              double p[VEC], w[VEC], base[VEC];
              ld2<VEC>(p, M.P + i);
              if (d.sub > 0) ld2<VEC>(w, M.w + i);
              if (d.phase == ENS_FINAL) ld2_l2<VEC>(base, M.T + i);
#pragma unroll
              for (int k = 0; k < VEC; ++k) {
                double y = d.delta * p[k];
                if (d.sub > 0) y += w[k];
                if (d.phase == ENS_FINAL) y += base[k];
                p[k] = y;
              }
              st2<VEC>((d.phase == ENS_ACCUM ? M.w : M.T) + i, p);
            }
          }
        }
        // warp partial (sum for TERM, max of ordered bits for INIT) and the
        // non-finite flag, in a fixed order
        const bool is_max = d.phase == ENS_INIT;
        double x = r0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(0xffffffffu, x, o);
          x = is_max ? fmax(x, y) : x + y;
        }
        const unsigned badw = __ballot_sync(0xffffffffu, bad);
        if (lane == 0) {
          s_red[par][wid][0] = x;
          s_red[par][wid][1] = badw ? 1.0 : 0.0;
          __threadfence_block();
          // the last compute warp to finish combines the warps' partials in
          // warp order into the CTA's partial
          if (atomicAdd(&s_cnt[par], 1u) == (unsigned)(kEnsWarps - 2)) {
            __threadfence_block();
            const volatile double* rv = &s_red[par][0][0];
            double a = rv[0], b = rv[1];
            for (int w = 1; w < kEnsWarps - 1; ++w) {
              a = is_max ? fmax(a, rv[2 * w]) : a + rv[2 * w];
              b = fmax(b, rv[2 * w + 1]);
            }
            s_cta[par][0] = a;
            s_cta[par][1] = b;
            s_cnt[par] = 0u;
          }
        }
      } else {
        // control warp: the outcome of pass j - 1 (its partials were complete
        // at the last barrier), then the descriptor of pass j + 1
        const bool has_prev = j > 0;
        PassDesc pv;
        double tot = 0.0, flag = 0.0;
        if (has_prev) {
          pv = s_d[par ^ 1];
          const bool is_max = pv.phase == ENS_INIT;
          if (pv.phase == ENS_INIT || pv.phase == ENS_TERM) {
            // the CTAs' partials, one per lane, combined by a tree of fixed
            // shape: the same bits in every CTA of the cluster
            double a = 0.0, b = 0.0;
            if (lane < (int)csize) {
              const double* rp = cl.map_shared_rank(&s_cta[par ^ 1][0], (unsigned)lane);
              a = rp[0];
              b = rp[1];
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
              const double ao = __shfl_down_sync(0xffffffffu, a, o);
              const double bo = __shfl_down_sync(0xffffffffu, b, o);
              a = is_max ? fmax(a, ao) : a + ao;
              b = fmax(b, bo);
            }
            tot = a;
            flag = b;
          }
        }
        if (lane == 0) {
          const PassDesc nx =
              ens_control(s_c, M, R, dd_all, xi_tab, d, has_prev ? &pv : nullptr, tot, flag != 0.0);
          s_d[par ^ 1] = nx;
          if (rank == 0 && (nx.phase == ENS_DONE || nx.phase == ENS_FAILED)) {
            const EnsCtl& c = s_c;
            EnsState& st = R.st[e];
            st.phase = nx.phase;
            st.level = c.level;
            st.sub = c.sub;
            st.step = c.step;
            st.status = c.status;
            st.terms = c.terms;
            st.attempts = c.attempts;
            st.last_S = c.last_S;
            st.passes = (int)(c.n_pass - c.terms);
            for (int k = 0; k < 64; ++k) {
              st.last_deg[k] = c.last_deg[k];
              st.cur_deg[k] = c.cur_deg[k];
            }
          }
        }
      }
      // pass j is complete in every CTA of the cluster, and the descriptor of
      // pass j + 1 is written
      cl.sync();
    }
  }
}

template <typename Tq, int VEC>
cudaError_t ens_cluster_config(int cs, int* max_clusters) {
  auto kern = k_ens_cluster<Tq, VEC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)cs);
  cfg.blockDim = dim3(kEnsThreads);
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(max_clusters, (void*)kern, &cfg);
}

template <typename Tq, int VEC>
cudaError_t ens_cluster_launch(const EnsRun& R, int cs, int clusters, cudaStream_t s) {
  auto kern = k_ens_cluster<Tq, VEC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(cs * clusters));
  cfg.blockDim = dim3(kEnsThreads);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, R);
}

}  // namespace

int ens_cta_threads() { return kEnsThreads; }

cudaError_t ens_max_clusters(int prec, int cs, int* n) {
  *n = 0;
  return prec == EREM_FP32_BULK ? ens_cluster_config<float, 4>(cs, n)
                                : ens_cluster_config<double, 2>(cs, n);
}

cudaError_t launch_ens_cluster(const EnsRun& R, int prec, int cs, int clusters, cudaStream_t s) {
  return prec == EREM_FP32_BULK ? ens_cluster_launch<float, 4>(R, cs, clusters, s)
                                : ens_cluster_launch<double, 2>(R, cs, clusters, s);
}

}  // namespace erem
