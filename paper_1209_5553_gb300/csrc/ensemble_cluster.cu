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

// The member's state machine, kept by thread 0 of every CTA (identical
// copies), with the parameters of the next pass that every thread reads.
struct EnsCtl {
  int phase, level, sub, m;   // m: the term the next ENS_TERM pass computes
  int step, target, status, terms;
  int attempts, last_S, passes, pad;
  long long n_pass, pass_bound;
  double yinf;                // ||T^n||_inf of the step
  double dm, shm, d0, delta;  // next pass: d_m, c/gamma + xi_{m-1}, d_0, dt / 2^level
  int cur_deg[64], last_deg[64];
  double e[kEnsWin];          // error estimates e_m, ring of kEnsWin
};

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

// Arm a new Leja substep at the state's level: the next pass computes q_1.
__device__ void ens_arm(EnsCtl& c) { c.m = 1; }

// Pass parameters of the state's next pass.
__device__ void ens_params(EnsCtl& c, const EnsMember& M, const double* xi, int mmax) {
  const double* dd = M.dd + (size_t)c.level * (mmax + 1);
  c.d0 = dd[0];
  c.delta = M.dt / (double)(1 << c.level);
  if (c.phase == ENS_TERM) {
    c.dm = dd[c.m];
    c.shm = M.cg + xi[c.m - 1];
  }
}

// Advance the state after a complete pass of phase c.phase; v0 is the
// pass's reduced value (sum of q_m^2 after ENS_TERM, ||T^n||_inf after
// ENS_INIT), bad its non-finite flag (ENS_INIT).
__device__ void ens_advance(EnsCtl& c, const EnsMember& M, int nlev, int restart, double v0,
                            bool bad) {
  c.n_pass += 1;
  if (c.phase != ENS_TERM) c.passes += 1;
  const int S = 1 << c.level;
  switch (c.phase) {
    case ENS_INIT:
      if (bad) {
        c.status = ENS_NONFINITE;
        c.phase = ENS_FAILED;
        break;
      }
      c.yinf = v0;
      c.sub = 0;
      ens_arm(c);
      c.phase = ENS_TERM;
      break;
    case ENS_TERM: {
      // stopping test of §4.2 on the estimate of term m
      const StopParams& sp = M.sp;
      const int m = c.m;
      c.terms += 1;
      const double scal = sp.tol_a + sp.tol_r * c.yinf;
      const double e = fabs(c.delta * c.dm) / scal * sqrt(v0 / sp.ncells);
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
          c.phase = c.sub == S - 1 ? ENS_FINAL : ENS_ACCUM;
        } else if (m >= sp.m_max) {
          failed = true;
        } else {
          c.m = m + 1;
        }
      }
      if (failed) {
        // the attempt failed: the whole step again at twice the substeps
        c.attempts += 1;
        if (c.level + 1 < nlev) {
          c.level += 1;
          c.phase = ENS_RESTART;
        } else {
          c.status = isfinite(e) ? ENS_NOTCONV : ENS_NONFINITE;
          c.phase = ENS_FAILED;
        }
      }
      break;
    }
    case ENS_ACCUM:
      c.phase = ENS_SUBSTART;
      break;
    case ENS_SUBSTART:
      c.sub += 1;
      ens_arm(c);
      c.phase = ENS_TERM;
      break;
    case ENS_RESTART:
      c.sub = 0;
      ens_arm(c);
      c.phase = ENS_TERM;
      break;
    case ENS_FINAL:
      c.last_S = S;
      for (int k = 0; k < 64; ++k) c.last_deg[k] = k < S ? c.cur_deg[k] : 0;
      c.step += 1;
      if (c.step >= c.target) {
        c.phase = ENS_DONE;
        break;
      }
      if (restart) c.level = 0;
      c.phase = ENS_INIT;
      break;
    default:
      break;
  }
  if (c.phase != ENS_DONE && c.phase != ENS_FAILED && c.n_pass >= c.pass_bound) {
    c.status = ENS_TIMEOUT;
    c.phase = ENS_FAILED;
  }
}

template <typename Tq, int VEC>
__global__ void __launch_bounds__(kEnsThreads, 2) k_ens_cluster(EnsRun R) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const unsigned csize = cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ __align__(16) EnsMember s_M;
  __shared__ EnsCtl s_c;
  __shared__ double s_red[2][kEnsThreads / 32];
  __shared__ double s_part[2][2];  // [pass parity][sum or max, non-finite flag]
  __shared__ int s_q;
  static_assert(sizeof(EnsMember) % 8 == 0 && sizeof(EnsMember) / 8 <= kEnsThreads, "EnsMember copy");

  const int G = (int)csize * kEnsThreads;
  const int g0 = (int)rank * kEnsThreads + tid;
  int par = 0;
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
    if (tid == 0) {
      const EnsState& st = R.st[e];
      EnsCtl& c = s_c;
      c.phase = ENS_INIT;
      c.level = st.level;
      c.target = st.target;
      c.sub = c.m = c.step = c.status = c.terms = c.attempts = c.last_S = c.passes = 0;
      c.n_pass = 0;
      c.pass_bound = (long long)st.target * R.passes_per_step;
      c.yinf = c.dm = c.shm = 0.0;
      for (int k = 0; k < 64; ++k) c.cur_deg[k] = c.last_deg[k] = 0;
    }
    __syncthreads();
    if (tid == 0) ens_params(s_c, s_M, R.xi, R.mmax);
    __syncthreads();
    const EnsMember& M = s_M;
    const int nvec = M.Np / VEC;
    const int vrow = M.px / VEC;

    for (;;) {
      const int phase = s_c.phase;
      if (phase == ENS_DONE || phase == ENS_FAILED) break;
      double r0 = 0.0;
      bool bad = false;
      if (phase == ENS_TERM) {
        const int m = s_c.m;
        const double dm = s_c.dm;
        const Tq shm = (Tq)s_c.shm;
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
          Tq c[5][VEC];
          const size_t off = leja_off<32 * VEC>(i, 5);
#pragma unroll
          for (int k = 0; k < 5; ++k) ldv<Tq, VEC>(c[k], jl + k * 32 * VEC + off);
          Tq out[VEC];
          Tq sq = Tq(0);
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            const Tq west = k == 0 ? ql : qc[k - 1];
            const Tq east = k == VEC - 1 ? qr : qc[k + 1];
            Tq a = (c[0][k] - shm) * qc[k];
            a = fma(c[1][k], west, a);
            a = fma(c[2][k], east, a);
            a = fma(c[3][k], qs[k], a);
            a = fma(c[4][k], qn[k], a);
            out[k] = a;
          }
          stv<Tq, VEC>(qo + i, out);
          double p[VEC];
          ld2<VEC>(p, P + i);
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            if constexpr (sizeof(Tq) == 4) {
              p[k] = fma(dm, f2d_fast(out[k]), p[k]);
              sq = fmaf(out[k], out[k], sq);
            } else {
              p[k] = fma(dm, out[k], p[k]);
              r0 = fma(out[k], out[k], r0);
            }
          }
          if constexpr (sizeof(Tq) == 4) r0 += (double)sq;
          st2<VEC>(P + i, p);
        }
      } else if (phase == ENS_INIT || phase == ENS_SUBSTART) {
        // INIT: G = J T^n + b, q_0 = G, P = d_0 G.  SUBSTART: q_0 = G + J w.
        const double d0 = s_c.d0;
        const double* x = phase == ENS_INIT ? M.T : M.w;
        unsigned long long tmax = 0ULL;
        for (int v = g0; v < nvec; v += G) {
          const int row = v / vrow;
          const int i = v * VEC;
          const int ix = i - row * M.px;
          // two cells at a time (the FP64 stencil of four cells would not fit
          // the register budget)
#pragma unroll 1
          for (int h = 0; h < VEC; h += 2)
            ens_start_pair<Tq>(M, x, i + h, row, ix + h, phase == ENS_INIT, d0, tmax, bad);
        }
        if (phase == ENS_INIT) r0 = __longlong_as_double((long long)tmax);
      } else {
        // cell-local passes (own cells only)
        const double d0 = s_c.d0, delta = s_c.delta;
        const int sub = s_c.sub;
        for (int v = g0; v < nvec; v += G) {
          const int i = v * VEC;
          if (phase == ENS_RESTART) {
            double g[VEC], p[VEC];
            Tq o[VEC];
            ld2<VEC>(g, M.G + i);
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
              p[k] = d0 * g[k];
              o[k] = (Tq)g[k];
            }
            st2<VEC>(M.P + i, p);
            stv<Tq, VEC>((Tq*)M.q[0] + i, o);
          } else {  // ACCUM: w = w + delta P; FINAL: T = T + w + delta P
            double p[VEC], w[VEC], base[VEC];
            ld2<VEC>(p, M.P + i);
            if (sub > 0) ld2<VEC>(w, M.w + i);
            if (phase == ENS_FINAL) ld2_l2<VEC>(base, M.T + i);
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
              double y = delta * p[k];
              if (sub > 0) y += w[k];
              if (phase == ENS_FINAL) y += base[k];
              p[k] = y;
            }
            st2<VEC>((phase == ENS_ACCUM ? M.w : M.T) + i, p);
          }
        }
      }

      // CTA reduction (sum for TERM, max of ordered bits for INIT) and the
      // non-finite flag, in a fixed order
      const bool is_max = phase == ENS_INIT;
      double x = r0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, x, o);
        x = is_max ? fmax(x, y) : x + y;
      }
      const unsigned badw = __ballot_sync(0xffffffffu, bad);
      if (lane == 0) {
        s_red[0][wid] = x;
        s_red[1][wid] = badw ? 1.0 : 0.0;
      }
      __syncthreads();
      if (wid == 0) {
        double a = lane < kEnsThreads / 32 ? s_red[0][lane] : 0.0;
        double b = lane < kEnsThreads / 32 ? s_red[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(0xffffffffu, a, o);
          a = is_max ? fmax(a, y) : a + y;
          b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
          s_part[par][0] = a;
          s_part[par][1] = b;
        }
      }
      // every CTA's pass (and its partial) is complete past this barrier
      cl.sync();
      if (wid == 0) {
        double a = 0.0, b = 0.0;
        if (lane < (int)csize) {
          const double* rp = cl.map_shared_rank(&s_part[par][0], (unsigned)lane);
          a = rp[0];
          b = rp[1];
        }
        // lane 0 combines the CTAs' partials in rank order: the same bits in
        // every CTA of the cluster
        double tot = 0.0, flag = 0.0;
        for (int r = 0; r < (int)csize; ++r) {
          const double ar = __shfl_sync(0xffffffffu, a, r);
          const double br = __shfl_sync(0xffffffffu, b, r);
          tot = is_max ? fmax(tot, ar) : tot + ar;
          flag = fmax(flag, br);
        }
        if (lane == 0) {
          ens_advance(s_c, M, R.nlev, R.restart, tot, flag != 0.0);
          ens_params(s_c, M, R.xi, R.mmax);
          if (rank == 0 && (s_c.phase == ENS_DONE || s_c.phase == ENS_FAILED)) {
            EnsState& st = R.st[e];
            const EnsCtl& c = s_c;
            st.phase = c.phase;
            st.level = c.level;
            st.sub = c.sub;
            st.step = c.step;
            st.status = c.status;
            st.terms = c.terms;
            st.attempts = c.attempts;
            st.last_S = c.last_S;
            st.passes = c.passes;
            for (int k = 0; k < 64; ++k) {
              st.last_deg[k] = c.last_deg[k];
              st.cur_deg[k] = c.cur_deg[k];
            }
          }
        }
      }
      __syncthreads();
      par ^= 1;
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
