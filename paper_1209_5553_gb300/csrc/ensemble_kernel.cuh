// The batched ensemble kernel (k_ens_iter) and its device helpers: one
// launch advances every active member of an ensemble of independent 2D
// problems by one pass of its own EREM state machine (erem_internal.h).
//
// Included by kernels.cu (one translation unit).
#pragma once

#include "device_common.cuh"

namespace erem {
namespace {

// ---------------------------------------------------------------------------
// Batched ensemble of independent 2D members: one launch is one iteration of
// every active member's state machine (erem_internal.h).  Work items are
// (member, tile) pairs of the active members, a tile being U thread-vectors
// per thread (U NT VEC cells, row-major over the padded grid); blocks walk
// them grid-stride.  The phase is uniform over a tile.  Per member, the block
// that completes the member's last tile (ticket) reduces the tile partials in
// tile order and advances the state, so results do not depend on which block
// took which tile.
// ---------------------------------------------------------------------------
template <int VEC>
__device__ __forceinline__ void ens_stencil(const EnsMember& M, const double* __restrict__ x,
                                            int i, int row, int ix, double (&a)[VEC]) {
  double xc[VEC], xs[VEC], xn[VEC], c[5][VEC];
  ldP<VEC>(xc, x + i);
  ldP<VEC>(xs, x + i - (row > 0 ? M.px : 0));
  ldP<VEC>(xn, x + i + (row < M.ny - 1 ? M.px : 0));
  const double xl = ix > 0 ? x[i - 1] : 0.0;
  const double xr = ix + VEC < M.px ? x[i + VEC] : 0.0;
#pragma unroll
  for (int k = 0; k < 5; ++k) ldP<VEC>(c[k], M.jc[k] + i);
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

template <typename Tq, int VEC>
__device__ __forceinline__ void ens_store_q(Tq* q, int i, const double (&a)[VEC]) {
  Tq o[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) o[v] = (Tq)a[v];
  stv<Tq, VEC>(q + i, o);
}

// Arm the stopping test for a new Leja substep at the state's level.
__device__ void ens_arm(const EnsMember& M, const EnsState* st) {
  Ctrl* c = M.ctrl;
  c->done = 0;
  c->degree = 0;
  c->fail = 0;
  c->nonfinite = 0;
  c->m_last = 0;
  c->err = 0.0;
  StopParams sp = M.sp;
  sp.delta = M.dt / (double)(1 << st->level);
  c->sp = sp;
}

// Advance member M after a complete pass of phase `phase` (thread 0 of the
// member's last block).  r: the reduced value (||T^n||_inf after ENS_INIT,
// sum of q_m^2 after ENS_TERM).  Returns 1 when the member left the active
// set.
__device__ int ens_advance(const EnsMember& M, const EnsLaunch& L, int phase, int m, double dm,
                           double r) {
  EnsState* st = M.st;
  Ctrl* c = M.ctrl;
  if (phase != ENS_TERM) st->passes += 1;
  switch (phase) {
    case ENS_INIT:
      c->yinf = r;
      if (__ldcg(&c->flags) & FLAG_NONFINITE) {  // raised by this pass's blocks
        st->status = ENS_NONFINITE;
        st->phase = ENS_FAILED;
        return 1;
      }
      st->sub = 0;
      ens_arm(M, st);
      st->phase = ENS_TERM;
      return 0;
    case ENS_TERM:
      stop_test(c, m, dm, r);
      st->terms += 1;
      if (c->nonfinite) {
        st->status = ENS_NONFINITE;
        st->phase = ENS_FAILED;
        return 1;
      }
      if (!c->done) return 0;
      if (!c->fail) {
        st->cur_deg[st->sub] = c->degree;
        st->phase = st->sub == (1 << st->level) - 1 ? ENS_FINAL : ENS_ACCUM;
        return 0;
      }
      st->attempts += 1;
      if (st->level + 1 < L.nlev) {
        st->level += 1;
        st->phase = ENS_RESTART;
        return 0;
      }
      st->status = ENS_NOTCONV;
      st->phase = ENS_FAILED;
      return 1;
    case ENS_ACCUM:
      st->phase = ENS_SUBSTART;
      return 0;
    case ENS_SUBSTART:
      st->sub += 1;
      ens_arm(M, st);
      st->phase = ENS_TERM;
      return 0;
    case ENS_RESTART:
      st->sub = 0;
      ens_arm(M, st);
      st->phase = ENS_TERM;
      return 0;
    case ENS_FINAL: {
      const int S = 1 << st->level;
      st->last_S = S;
      for (int k = 0; k < 64; ++k) st->last_deg[k] = k < S ? st->cur_deg[k] : 0;
      st->step += 1;
      if (st->step >= st->target) {
        st->phase = ENS_DONE;
        return 1;
      }
      if (L.restart) st->level = 0;
      st->phase = ENS_INIT;
      return 0;
    }
    default:
      return 0;
  }
}

// Block-wide exclusive scan of one int per thread; *total gets the sum.
__device__ int block_exscan(int v, int* sm, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < NT / 32; ++k) {
      const int t = sm[k];
      sm[k] = acc;
      acc += t;
    }
    sm[NT / 32] = acc;
  }
  __syncthreads();
  *total = sm[NT / 32];
  return sm[wid] + x - v;
}

template <typename Tq, int VEC, int U>
__global__ void __launch_bounds__(NT, 4)
k_ens_iter(EnsLaunch L, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh[NT / 32];
  __shared__ int s_last;
  __shared__ int s_scan[NT / 32 + 1];
  const int n_act = L.act[0];
  const int n_tiles = L.act[1];
  const int* act_member = L.act + 4;
  const int* act_start = L.act + 4 + L.n_members;
  for (int gt = blockIdx.x; gt < n_tiles; gt += gridDim.x) {
    // the active member owning work item gt: last k with act_start[k] <= gt
    // (the list was written by an earlier launch: plain cached loads)
    int lo = 0, hi = n_act - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (act_start[mid] <= gt) lo = mid;
      else hi = mid - 1;
    }
    const EnsMember& M = L.mem[act_member[lo]];
    const int t = gt - act_start[lo];
    EnsState* st = M.st;
    const int phase = st->phase;
    const int level = st->level;
    const int sub = st->sub;
    const double* dd = M.dd + (size_t)level * (L.mmax + 1);
    const double delta = M.dt / (double)(1 << level);
    const int nvec = M.Np / VEC;
    const int vrow = M.px / VEC;
    int m = 0;
    double dm = 0.0;
    double acc = 0.0;                 // ENS_TERM: sum of q_m^2
    unsigned long long tmax = 0ULL;   // ENS_INIT: ||T^n||_inf as bits
    bool bad = false;
    if (phase == ENS_TERM) {
      m = M.ctrl->m_last + 1;
      dm = dd[m];
      const Tq shm = (Tq)(M.cg + L.xi[m - 1]);
      const Tq* qi = (const Tq*)M.q[(m - 1) & 1];
      Tq* qo = (Tq*)M.q[m & 1];
      const Tq* jl = (const Tq*)M.jl;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int v = (t * U + j) * NT + threadIdx.x;
        if (v >= nvec) continue;
        const int row = v / vrow;
        const int i = v * VEC;
        const int ix = i - row * M.px;
        Tq qc[VEC], qs[VEC], qn[VEC];
        ldv<Tq, VEC>(qc, qi + i);
        ldv<Tq, VEC>(qs, qi + i - (row > 0 ? M.px : 0));
        ldv<Tq, VEC>(qn, qi + i + (row < M.ny - 1 ? M.px : 0));
        const Tq ql = ix > 0 ? qi[i - 1] : Tq(0);
        const Tq qr = ix + VEC < M.px ? qi[i + VEC] : Tq(0);
        Tq c[5][VEC];
        const size_t off = leja_off<32 * VEC>(i, 5);
#pragma unroll
        for (int k = 0; k < 5; ++k) ldv_stream<Tq, VEC>(c[k], jl + k * 32 * VEC + off);
        double p[VEC];
        ldP<VEC>(p, M.P + i);
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
          if constexpr (sizeof(Tq) == 4) {
            p[k] = fma(dm, f2d_exact(a), p[k]);
            sq = fmaf(a, a, sq);
          } else {
            p[k] = fma(dm, a, p[k]);
            acc = fma(a, a, acc);
          }
        }
        if constexpr (sizeof(Tq) == 4) acc += (double)sq;
        stv<Tq, VEC>(qo + i, out);
        stP<VEC>(M.P + i, p);
      }
    } else if (phase == ENS_INIT || phase == ENS_SUBSTART) {
      // INIT: G = J T^n + b, q_0 = G, P = d_0 G.  SUBSTART: q_0 = G + J w.
      const double d0 = dd[0];
      const double* x = phase == ENS_INIT ? M.T : M.w;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int v = (t * U + j) * NT + threadIdx.x;
        if (v >= nvec) continue;
        const int row = v / vrow;
        const int i = v * VEC;
        const int ix = i - row * M.px;
        double a[VEC];
        ens_stencil<VEC>(M, x, i, row, ix, a);
        if (phase == ENS_INIT) {
          if (ix == 0) a[0] += M.b0[row];
          double tc[VEC];
          ldP<VEC>(tc, M.T + i);
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            const unsigned long long tb = abs_bits(tc[k]);
            tmax = tmax > tb ? tmax : tb;
            bad |= !bits_finite(tb) | !bits_finite(abs_bits(a[k]));
          }
          stP<VEC>(M.G + i, a);
        } else {
          double g[VEC];
          ldP<VEC>(g, M.G + i);
#pragma unroll
          for (int k = 0; k < VEC; ++k) a[k] += g[k];
        }
        double p[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) p[k] = d0 * a[k];
        stP<VEC>(M.P + i, p);
        ens_store_q<Tq, VEC>((Tq*)M.q[0], i, a);
      }
    } else {
      // cell-local phases
      const double d0 = dd[0];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int v = (t * U + j) * NT + threadIdx.x;
        if (v >= nvec) continue;
        const int i = v * VEC;
        if (phase == ENS_RESTART) {
          double g[VEC], p[VEC];
          ldP<VEC>(g, M.G + i);
#pragma unroll
          for (int k = 0; k < VEC; ++k) p[k] = d0 * g[k];
          stP<VEC>(M.P + i, p);
          ens_store_q<Tq, VEC>((Tq*)M.q[0], i, g);
        } else {
          double p[VEC], w[VEC];
          ldP<VEC>(p, M.P + i);
          if (sub > 0) ldP<VEC>(w, M.w + i);
          double* dst = phase == ENS_ACCUM ? M.w : M.T;
          double base[VEC];
          if (phase == ENS_FINAL) ldP<VEC>(base, M.T + i);
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            double y = delta * p[k];
            if (sub > 0) y += w[k];
            if (phase == ENS_FINAL) y += base[k];
            p[k] = y;
          }
          stP<VEC>(dst + i, p);
        }
      }
    }
    double bv = 0.0;
    if (phase == ENS_INIT) bv = block_reduce<2>(__longlong_as_double((long long)tmax), sh);
    else if (phase == ENS_TERM) bv = block_reduce<0>(acc, sh);
    if (bad) atomicOr(&M.ctrl->flags, FLAG_NONFINITE);
    __syncthreads();
    if (threadIdx.x == 0) {
      M.part[(size_t)t * kRedSlots] = bv;
      __threadfence();
      s_last = atomicInc(M.cnt, (unsigned)M.tiles - 1u) == (unsigned)M.tiles - 1u;
    }
    __syncthreads();
    if (s_last) {  // every tile of this member's pass is done
      __threadfence();
      double r = 0.0;
      if (phase == ENS_INIT) r = gather_partials_t<2, NT>(M.part, 0, sh, threadIdx.x, M.tiles);
      else if (phase == ENS_TERM) r = gather_partials_t<0, NT>(M.part, 0, sh, threadIdx.x, M.tiles);
      if (threadIdx.x == 0) {
        if (ens_advance(M, L, phase, m, dm, r)) atomicExch(&L.act[2], 1);
        __threadfence();
      }
    }
    __syncthreads();
  }

  // The last block of the launch: rebuild the active list when a member
  // left it, count the iteration and decide whether the loop goes on.
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicInc(L.gcnt, gridDim.x - 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int* act = L.act;
  if (*(volatile int*)&act[2]) {
    int n_off = 0, t_off = 0;
    for (int base = 0; base < L.n_members; base += NT) {
      const int e = base + threadIdx.x;
      int on = 0, tl = 0;
      if (e < L.n_members) {
        const int ph = *(volatile int*)&L.mem[e].st->phase;
        on = ph != ENS_DONE && ph != ENS_FAILED;
        tl = on ? L.mem[e].tiles : 0;
      }
      int n_tot, t_tot;
      const int pos = block_exscan(on, s_scan, &n_tot) + n_off;
      const int tpos = block_exscan(tl, s_scan, &t_tot) + t_off;
      if (on) {
        act[4 + pos] = e;
        act[4 + L.n_members + pos] = tpos;
      }
      n_off += n_tot;
      t_off += t_tot;
    }
    if (threadIdx.x == 0) {
      act[4 + L.n_members + n_off] = t_off;
      act[0] = n_off;
      act[1] = t_off;
      act[2] = 0;
    }
  }
  if (threadIdx.x == 0) {
    const unsigned it = *(volatile unsigned*)L.iters + (n_act > 0 ? 1u : 0u);
    *L.iters = it;
    const int more = *(volatile int*)&act[0] > 0 && (long long)it < (long long)L.max_iters;
    act[3] = more;
    __threadfence();
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

}  // namespace
}  // namespace erem
