// Batched ensembles of independent 2D EREM problems (declared in
// include/erem.h): member contexts, the batch tables the kernel reads, the
// divided-difference tables of every substep level, the CUDA graph of a run
// and the tile-size autotuner.
//
// Each member is a full context (erem_create / erem_set_state build its
// Jacobian, its Leja copy of J and its spectral interval exactly as for a
// single problem); the batched kernel k_ens_iter then drives all members'
// buffers at once.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "erem_internal.h"

using namespace erem;

struct erem_ens {
  int n = 0;
  erem_precision prec = EREM_FP64;
  std::vector<erem_ctx*> ctx;
  std::vector<char> ready;
  std::vector<double> dt;
  std::string err;
  int sm_count = 1;

  // Leja options and batching configuration
  double tol_a = 1e-6, tol_r = 1e-6;
  int p_order = 2, m_max = 150, max_doublings = 6, avg_window = 5;
  erem_ens_config cfg{EREM_ENS_KEEP_SUBSTEPS, 0, 0, 1};
  int tuned_U = 0;

  // divided differences of every member and level (host copy, reused by
  // rebuilds until a member or the options change)
  std::vector<double> dd_host;
  bool dd_valid = false;

  // batch tables (valid while built)
  bool built = false;
  int U = 2, grid = 1, nlev = 7, total_tiles = 0;
  std::vector<int> tiles, tile0;
  std::vector<int> level_start;     // KEEP policy: first level of each member's next step
  std::vector<char> clear_flags;    // members whose non-finite flag must be cleared
  EnsMember* mem_d = nullptr;
  EnsState* st_d = nullptr;
  EnsState* st_h = nullptr;         // pinned
  double* part_d = nullptr;
  unsigned* cnt_d = nullptr;
  double* dd_d = nullptr;
  int* act_d = nullptr;
  int* act_h = nullptr;             // pinned
  unsigned* ctr_d = nullptr;        // [0] launch ticket, [1] iterations
  unsigned* ctr_h = nullptr;        // pinned
  double* xi_d = nullptr;
  double* snap_d = nullptr;         // autotuner: saved temperatures
  double* stage_d = nullptr;        // host-pointer staging (largest member)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_iters = -1;             // iteration bound baked into the graph
  cudaEvent_t ev[2] = {nullptr, nullptr};
  EnsLaunch L{};

  // statistics of the last run
  erem_ens_run_stats rs{};
  std::vector<EnsState> last;
};

namespace {

erem_status efail(erem_ens* E, erem_status st, const std::string& m) {
  if (E) E->err = m;
  return st;
}

#define ENS_CUDA(E, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return efail((E), EREM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define ENS_TRY(expr)               \
  do {                              \
    erem_status st_ = (expr);       \
    if (st_ != EREM_OK) return st_; \
  } while (0)

template <typename T>
erem_status ens_alloc(erem_ens* E, T** p, size_t count) {
  if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return efail(E, EREM_ENOMEM, "cudaMalloc of the ensemble tables failed");
  }
  ENS_CUDA(E, cudaMemset(*p, 0, std::max<size_t>(count, 1) * sizeof(T)));
  return EREM_OK;
}

void release_tables(erem_ens* E) {
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  E->exec = nullptr;
  E->graph = nullptr;
  void* dp[] = {E->mem_d, E->st_d, E->part_d, E->cnt_d, E->dd_d, E->act_d, E->ctr_d, E->xi_d};
  for (void* p : dp)
    if (p) cudaFree(p);
  E->mem_d = nullptr;
  E->st_d = nullptr;
  E->part_d = nullptr;
  E->cnt_d = nullptr;
  E->dd_d = nullptr;
  E->act_d = nullptr;
  E->ctr_d = nullptr;
  E->xi_d = nullptr;
  if (E->st_h) cudaFreeHost(E->st_h);
  if (E->act_h) cudaFreeHost(E->act_h);
  if (E->ctr_h) cudaFreeHost(E->ctr_h);
  E->st_h = nullptr;
  E->act_h = nullptr;
  E->ctr_h = nullptr;
  E->built = false;
}

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Divided differences of every member and substep level, on host threads:
// table (e, l) holds d_0..d_mmax for the interval of dt J / 2^l.
erem_status build_dd(erem_ens* E, const std::vector<double>& xi, std::vector<double>* dd) {
  const int M = E->m_max, nl = kEnsMaxLevels;
  dd->assign((size_t)E->n * nl * (M + 1), 0.0);
  std::atomic<int> next{0}, bad{-1};
  auto work = [&]() {
    for (int job = next++; job < E->n * E->nlev; job = next++) {
      const int e = job / E->nlev, l = job % E->nlev;
      const erem_ctx* c = E->ctx[e];
      const double S = (double)(1 << l);
      double* d = dd->data() + ((size_t)e * nl + l) * (M + 1);
      if (divided_differences(M, xi.data(), c->cfoc / S, c->gam / S, d) != 0) {
        bad = e;
        continue;
      }
      for (int k = 0; k <= M; ++k)
        if (!std::isfinite(d[k])) bad = e;
    }
  };
  const int nt = std::max(1, std::min<int>(32, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  if (bad >= 0)
    return efail(E, EREM_ENONFINITE,
                 "divided differences of member " + std::to_string(bad.load()) + " are not finite");
  return EREM_OK;
}

long long iteration_bound(const erem_ens* E, int steps) {
  long long per_step = 2;
  for (int l = 0; l < E->nlev; ++l) per_step += (1LL << l) * (E->m_max + 2) + 2;
  const long long b = (long long)steps * per_step + 16;
  return std::min<long long>(b, 2000000000LL);
}

// Member table, tile layout, divided differences, active list and graph for
// tile size U.
erem_status build(erem_ens* E, int U) {
  for (int e = 0; e < E->n; ++e)
    if (!E->ready[e])
      return efail(E, EREM_EINVAL, "member " + std::to_string(e) + " has no state (erem_ensemble_set_member)");
  release_tables(E);
  E->U = U;
  E->nlev = E->max_doublings + 1;
  const int tile_cells = ens_tile_cells(E->prec, U);
  E->tiles.assign(E->n, 0);
  E->tile0.assign(E->n, 0);
  long long tot = 0;
  for (int e = 0; e < E->n; ++e) {
    E->tile0[e] = (int)tot;
    E->tiles[e] = (int)((E->ctx[e]->Np + tile_cells - 1) / tile_cells);
    tot += E->tiles[e];
  }
  if (tot >= (1LL << 30)) return efail(E, EREM_EINVAL, "ensemble too large");
  E->total_tiles = (int)tot;

  const int M = E->m_max;
  std::vector<double> xi;
  leja_table(M, &xi);
  if (!E->dd_valid) {
    ENS_TRY(build_dd(E, xi, &E->dd_host));
    E->dd_valid = true;
  }
  const std::vector<double>& dd = E->dd_host;

  ENS_TRY(ens_alloc(E, &E->mem_d, (size_t)E->n));
  ENS_TRY(ens_alloc(E, &E->st_d, (size_t)E->n));
  ENS_TRY(ens_alloc(E, &E->part_d, (size_t)E->total_tiles * kRedSlots));
  ENS_TRY(ens_alloc(E, &E->cnt_d, (size_t)E->n));
  ENS_TRY(ens_alloc(E, &E->dd_d, dd.size()));
  ENS_TRY(ens_alloc(E, &E->act_d, (size_t)2 * E->n + 5));
  ENS_TRY(ens_alloc(E, &E->ctr_d, (size_t)2));
  ENS_TRY(ens_alloc(E, &E->xi_d, (size_t)M + 1));
  if (cudaMallocHost((void**)&E->st_h, sizeof(EnsState) * E->n) != cudaSuccess ||
      cudaMallocHost((void**)&E->act_h, sizeof(int) * (2 * E->n + 5)) != cudaSuccess ||
      cudaMallocHost((void**)&E->ctr_h, sizeof(unsigned) * 2) != cudaSuccess)
    return efail(E, EREM_ENOMEM, "cudaMallocHost of the ensemble tables failed");
  std::memset(E->st_h, 0, sizeof(EnsState) * E->n);

  std::vector<EnsMember> mem(E->n);
  for (int e = 0; e < E->n; ++e) {
    const erem_ctx* c = E->ctx[e];
    EnsMember& m = mem[e];
    std::memset(&m, 0, sizeof(m));
    m.nx = c->nx;
    m.ny = c->ny;
    m.px = c->px;
    m.Np = (int)c->Np;
    m.tiles = E->tiles[e];
    for (int k = 0; k < 5; ++k) m.jc[k] = c->jc[k];
    m.b0 = c->b0;
    m.jl = c->jl_all;
    m.T = c->Tn;
    m.G = c->vrhs;
    m.w = c->w;
    m.P = c->P;
    m.q[0] = c->q[0];
    m.q[1] = c->q[1];
    m.part = E->part_d + (size_t)E->tile0[e] * kRedSlots;
    m.cnt = E->cnt_d + e;
    m.ctrl = c->ctrl;
    m.st = E->st_d + e;
    m.dd = E->dd_d + (size_t)e * kEnsMaxLevels * (M + 1);
    m.sp.delta = E->dt[e];
    m.sp.ncells = (double)c->N;
    m.sp.pow10 = std::pow(10.0, E->p_order);
    m.sp.tol_a = E->tol_a;
    m.sp.tol_r = E->tol_r;
    m.sp.window = E->avg_window;
    m.sp.m_max = E->m_max;
    m.sp.replay = 0;
    m.dt = E->dt[e];
    m.cg = c->cfoc / c->gam;
  }
  ENS_CUDA(E, cudaMemcpy(E->mem_d, mem.data(), sizeof(EnsMember) * E->n, cudaMemcpyHostToDevice));
  ENS_CUDA(E, cudaMemcpy(E->dd_d, dd.data(), sizeof(double) * dd.size(), cudaMemcpyHostToDevice));
  ENS_CUDA(E, cudaMemcpy(E->xi_d, xi.data(), sizeof(double) * (M + 1), cudaMemcpyHostToDevice));

  int bps = E->cfg.blocks_per_sm > 0 ? E->cfg.blocks_per_sm : ens_blocks_per_sm(E->prec, U);
  E->grid = std::max(1, std::min(E->total_tiles, bps * E->sm_count));
  EnsLaunch& L = E->L;
  L.prec = E->prec;
  L.U = U;
  L.grid = E->grid;
  L.n_members = E->n;
  L.nlev = E->nlev;
  L.mmax = M;
  L.restart = E->cfg.substep_policy == EREM_ENS_RESTART_SUBSTEPS ? 1 : 0;
  L.max_iters = 0;  // set per run (the graph reads it from the table below)
  L.mem = E->mem_d;
  L.xi = E->xi_d;
  L.act = E->act_d;
  L.gcnt = E->ctr_d;
  L.iters = E->ctr_d + 1;
  E->built = true;
  return EREM_OK;
}

// The graph bakes in the launch parameters, max_iters included; it is
// rebuilt when the run length changes.
erem_status ensure_graph(erem_ens* E, int max_iters) {
  if (E->exec && E->graph_iters == max_iters) return EREM_OK;
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  E->exec = nullptr;
  E->graph = nullptr;
  E->L.max_iters = max_iters;
  ENS_CUDA(E, build_ens_graph(E->L, &E->graph, &E->exec));
  E->graph_iters = max_iters;
  return EREM_OK;
}

// One pass of the batched loop over the members in `list` (their states in
// st_h set by the caller; the states of the other members are not touched by
// the kernel).  Adds the pass's device time and iterations to *ms, *iters.
erem_status run_pass(erem_ens* E, const std::vector<int>& list, long long bound, cudaStream_t s,
                     double* ms, long long* iters) {
  int* a = E->act_h;
  int tiles = 0;
  for (size_t k = 0; k < list.size(); ++k) {
    a[4 + k] = list[k];
    a[4 + E->n + k] = tiles;
    tiles += E->tiles[list[k]];
  }
  a[0] = (int)list.size();
  a[1] = tiles;
  a[2] = 0;
  a[3] = 1;
  a[4 + E->n + list.size()] = tiles;
  ENS_CUDA(E, cudaMemcpyAsync(E->st_d, E->st_h, sizeof(EnsState) * E->n, cudaMemcpyHostToDevice, s));
  ENS_CUDA(E, cudaMemcpyAsync(E->act_d, a, sizeof(int) * (2 * E->n + 5), cudaMemcpyHostToDevice, s));
  ENS_CUDA(E, cudaMemsetAsync(E->ctr_d, 0, 2 * sizeof(unsigned), s));
  ENS_CUDA(E, cudaMemsetAsync(E->cnt_d, 0, sizeof(unsigned) * E->n, s));
  ENS_CUDA(E, cudaEventRecord(E->ev[0], s));
  if (E->cfg.use_graph) {
    ENS_CUDA(E, cudaGraphLaunch(E->exec, s));
  } else {
    // host-driven: batches of launches, then the loop flag act[3]
    long long done = 0;
    while (true) {
      const int batch = 32;
      for (int k = 0; k < batch; ++k) launch_ens_iter(E->L, s);
      ENS_CUDA(E, cudaGetLastError());
      done += batch;
      ENS_CUDA(E, cudaMemcpyAsync(E->act_h + 3, E->act_d + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
      ENS_CUDA(E, cudaStreamSynchronize(s));
      if (!E->act_h[3] || done > bound + batch) break;
    }
  }
  ENS_CUDA(E, cudaEventRecord(E->ev[1], s));
  ENS_CUDA(E, cudaMemcpyAsync(E->st_h, E->st_d, sizeof(EnsState) * E->n, cudaMemcpyDeviceToHost, s));
  ENS_CUDA(E, cudaMemcpyAsync(E->ctr_h, E->ctr_d, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  ENS_CUDA(E, cudaMemcpyAsync(E->act_h, E->act_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  ENS_CUDA(E, cudaStreamSynchronize(s));
  float t = 0.f;
  ENS_CUDA(E, cudaEventElapsedTime(&t, E->ev[0], E->ev[1]));
  *ms += t;
  *iters += E->ctr_h[1];
  if (E->act_h[0] != 0)
    return efail(E, EREM_ETIMEOUT, "the batched loop reached its iteration bound");
  return EREM_OK;
}

// One run: every member advances `steps` steps.  A member whose Leja error
// estimate became non-finite (the Newton vectors or their squares left the
// range of the Leja precision; a bad state is flagged separately by the first
// pass of its step) stops at the start of that step; it is run again, alone
// with the other such members, from that step at the next substep level, as
// erem_step splits a step whose interpolation failed.
erem_status run(erem_ens* E, int steps, cudaStream_t s) {
  const long long bound = iteration_bound(E, steps);
  E->L.max_iters = (int)bound;
  if (E->cfg.use_graph) ENS_TRY(ensure_graph(E, (int)bound));
  const bool keep = E->cfg.substep_policy == EREM_ENS_KEEP_SUBSTEPS;
  std::vector<EnsState> tot(E->n);
  std::vector<int> list(E->n);
  for (int e = 0; e < E->n; ++e) {
    EnsState& st = E->st_h[e];
    std::memset(&st, 0, sizeof(st));
    st.phase = ENS_INIT;
    st.level = std::min(keep ? E->level_start[e] : 0, E->nlev - 1);
    st.target = steps;
    std::memset(&tot[e], 0, sizeof(EnsState));
    list[e] = e;
    if (E->clear_flags[e]) {
      ENS_CUDA(E, cudaMemsetAsync(&E->ctx[e]->ctrl->flags, 0, sizeof(int), s));
      E->clear_flags[e] = 0;
    }
  }
  double ms = 0.0;
  long long iters = 0;
  while (!list.empty()) {
    ENS_TRY(run_pass(E, list, bound, s, &ms, &iters));
    std::vector<int> retry;
    for (int e : list) {
      const EnsState& st = E->st_h[e];
      EnsState& t = tot[e];
      t.step += st.step;
      t.terms += st.terms;
      t.passes += st.passes;
      t.attempts += st.attempts;
      if (st.last_S > 0) {
        t.last_S = st.last_S;
        std::memcpy(t.last_deg, st.last_deg, sizeof(t.last_deg));
      }
      t.phase = st.phase;
      t.status = st.status;
      t.level = st.level;
      if (st.phase == ENS_FAILED && st.status == ENS_NONFINITE && st.level + 1 < E->nlev) {
        int flags = 0;
        ENS_CUDA(E, cudaMemcpy(&flags, &E->ctx[e]->ctrl->flags, sizeof(int), cudaMemcpyDeviceToHost));
        if (!(flags & FLAG_NONFINITE)) retry.push_back(e);
      }
    }
    for (int e : retry) {
      EnsState& st = E->st_h[e];
      const int level = st.level + 1;
      const int left = steps - tot[e].step;
      std::memset(&st, 0, sizeof(st));
      st.phase = ENS_INIT;
      st.level = level;
      st.target = left;
      tot[e].attempts += 1;
    }
    list.swap(retry);
  }

  erem_ens_run_stats& r = E->rs;
  std::memset(&r, 0, sizeof(r));
  r.t_ms = ms;
  r.iterations = iters;
  r.tile_vecs = E->U;
  r.grid = E->grid;
  r.use_graph = E->cfg.use_graph;
  E->last = tot;
  int first_fail = -1;
  for (int e = 0; e < E->n; ++e) {
    const EnsState& st = tot[e];
    const long long N = E->ctx[e]->N;
    r.cells += N;
    r.cell_terms += N * st.terms;
    r.cell_passes += N * st.passes;
    if (st.phase == ENS_FAILED) {
      ++r.members_failed;
      if (first_fail < 0) first_fail = e;
      if (st.status == ENS_NONFINITE) E->clear_flags[e] = 1;
    } else if (st.last_S > 0) {
      int l = 0;
      while ((1 << l) < st.last_S) ++l;
      E->level_start[e] = l;
    }
  }
  if (first_fail >= 0) {
    const EnsState& st = tot[first_fail];
    const std::string who = "member " + std::to_string(first_fail);
    if (st.status == ENS_NONFINITE)
      return efail(E, EREM_ENONFINITE, who + ": non-finite value in the state or the Leja estimate");
    return efail(E, EREM_ENOTCONV,
                 who + ": Leja interpolation did not meet the stopping test within m_max terms after " +
                     std::to_string(E->max_doublings) + " substep doublings");
  }
  return EREM_OK;
}

erem_status check_member(erem_ens* E, int e) {
  if (e < 0 || e >= E->n) return efail(E, EREM_EINVAL, "member index out of range");
  return EREM_OK;
}

}  // namespace

extern "C" {

erem_status erem_ensemble_create(int n_members, const erem_grid* grids, const erem_physics* phys,
                                 erem_precision prec, erem_ens** out) {
  if (!out) return EREM_EINVAL;
  *out = nullptr;
  if (n_members < 1 || !grids || !phys) return EREM_EINVAL;
  if (prec != EREM_FP64 && prec != EREM_FP32_BULK) return EREM_EINVAL;
  for (int e = 0; e < n_members; ++e)
    if (grids[e].dim != 2 || phys[e].fluid_model != 0) return EREM_EINVAL;
  erem_ens* E = new erem_ens();
  E->n = n_members;
  E->prec = prec;
  E->ctx.assign(n_members, nullptr);
  E->ready.assign(n_members, 0);
  E->dt.assign(n_members, 0.0);
  E->level_start.assign(n_members, 0);
  E->clear_flags.assign(n_members, 0);
  auto bail = [&](erem_status st) {
    erem_ensemble_destroy(E);
    return st;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&E->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bail(EREM_ECUDA);
  long long maxN = 1;
  for (int e = 0; e < n_members; ++e) {
    const erem_status st = erem_create(&grids[e], &phys[e], prec, &E->ctx[e]);
    if (st != EREM_OK) return bail(st);
    maxN = std::max(maxN, E->ctx[e]->N);
  }
  if (cudaMalloc((void**)&E->stage_d, sizeof(double) * maxN) != cudaSuccess) return bail(EREM_ENOMEM);
  if (cudaEventCreate(&E->ev[0]) != cudaSuccess || cudaEventCreate(&E->ev[1]) != cudaSuccess)
    return bail(EREM_ECUDA);
  *out = E;
  return EREM_OK;
}

erem_status erem_ensemble_destroy(erem_ens* E) {
  if (!E) return EREM_OK;
  release_tables(E);
  for (erem_ctx* c : E->ctx)
    if (c) erem_destroy(c);
  if (E->snap_d) cudaFree(E->snap_d);
  if (E->stage_d) cudaFree(E->stage_d);
  for (cudaEvent_t ev : E->ev)
    if (ev) cudaEventDestroy(ev);
  delete E;
  return EREM_OK;
}

erem_status erem_ensemble_set_member(erem_ens* E, int e, const double* T, const double* p,
                                     const double* lnk, const double* phi, const double* lam,
                                     double dt, void* stream) {
  if (!E) return EREM_EINVAL;
  ENS_TRY(check_member(E, e));
  E->ready[e] = 0;
  E->built = false;
  E->dd_valid = false;
  const erem_status st = erem_set_state(E->ctx[e], T, p, lnk, phi, lam, dt, stream);
  if (st != EREM_OK) return efail(E, st, "member " + std::to_string(e) + ": " + E->ctx[e]->err);
  E->ready[e] = 1;
  E->dt[e] = dt;
  E->level_start[e] = 0;
  E->clear_flags[e] = 0;
  return EREM_OK;
}

erem_status erem_ensemble_set_temperature(erem_ens* E, int e, const double* T, void* stream) {
  if (!E) return EREM_EINVAL;
  ENS_TRY(check_member(E, e));
  if (!T) return efail(E, EREM_EINVAL, "T is NULL");
  if (!E->ready[e]) return efail(E, EREM_EINVAL, "member has no state");
  cudaStream_t s = (cudaStream_t)stream;
  const erem_ctx* c = E->ctx[e];
  const double* src = T;
  if (!is_device(T)) {
    ENS_CUDA(E, cudaMemcpyAsync(E->stage_d, T, sizeof(double) * c->N, cudaMemcpyHostToDevice, s));
    src = E->stage_d;
  }
  launch_pack(c, src, c->Tn, s);
  ENS_CUDA(E, cudaGetLastError());
  if (src != T) ENS_CUDA(E, cudaStreamSynchronize(s));  // the staging buffer is reused
  return EREM_OK;
}

erem_status erem_ensemble_get_member(erem_ens* E, int e, double* T, void* stream) {
  if (!E) return EREM_EINVAL;
  ENS_TRY(check_member(E, e));
  if (!T) return efail(E, EREM_EINVAL, "T is NULL");
  if (!E->ready[e]) return efail(E, EREM_EINVAL, "member has no state");
  cudaStream_t s = (cudaStream_t)stream;
  const erem_ctx* c = E->ctx[e];
  if (is_device(T)) {
    launch_unpack(c, c->Tn, T, s);
    ENS_CUDA(E, cudaGetLastError());
    return EREM_OK;
  }
  launch_unpack(c, c->Tn, E->stage_d, s);
  ENS_CUDA(E, cudaGetLastError());
  ENS_CUDA(E, cudaMemcpyAsync(T, E->stage_d, sizeof(double) * c->N, cudaMemcpyDeviceToHost, s));
  ENS_CUDA(E, cudaStreamSynchronize(s));
  return EREM_OK;
}

erem_status erem_ensemble_configure(erem_ens* E, const erem_leja_opts* o, const erem_ens_config* cfg) {
  if (!E) return EREM_EINVAL;
  double tol_a = 1e-6, tol_r = 1e-6;
  int p_order = 2, m_max = 150, max_doublings = 6, avg_window = 5;
  if (o) {
    if (o->replay || o->time_terms) return efail(E, EREM_EINVAL, "replay and time_terms are not batched");
    if (o->tol_a != 0.0) tol_a = o->tol_a;
    if (o->tol_r != 0.0) tol_r = o->tol_r;
    if (o->p_order != 0) p_order = o->p_order;
    if (o->m_max != 0) m_max = o->m_max;
    max_doublings = o->max_doublings;
    if (o->avg_window != 0) avg_window = o->avg_window;
  }
  if (!(tol_a >= 0.0) || !(tol_r >= 0.0) || tol_a + tol_r <= 0.0)
    return efail(E, EREM_EINVAL, "tolerances must be >= 0 with tol_a + tol_r > 0");
  if (m_max < 1 || m_max > kMaxTerms || avg_window < 1 || p_order < 0 || p_order > 30 ||
      max_doublings < 0 || max_doublings > kEnsMaxLevels - 1)
    return efail(E, EREM_EINVAL, "bad m_max, avg_window, p_order or max_doublings (0..6)");
  erem_ens_config c = E->cfg;
  if (cfg) {
    c = *cfg;
    if (c.substep_policy != EREM_ENS_KEEP_SUBSTEPS && c.substep_policy != EREM_ENS_RESTART_SUBSTEPS)
      return efail(E, EREM_EINVAL, "unknown substep policy");
    if (c.tile_vecs != 0 && c.tile_vecs != 1 && c.tile_vecs != 2 && c.tile_vecs != 4)
      return efail(E, EREM_EINVAL, "tile_vecs must be 0, 1, 2 or 4");
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 32) return efail(E, EREM_EINVAL, "blocks_per_sm 0..32");
    if (c.use_graph != 0 && c.use_graph != 1) return efail(E, EREM_EINVAL, "use_graph must be 0 or 1");
  }
  E->tol_a = tol_a;
  E->tol_r = tol_r;
  E->p_order = p_order;
  E->m_max = m_max;
  E->max_doublings = max_doublings;
  E->avg_window = avg_window;
  E->cfg = c;
  E->built = false;
  E->dd_valid = false;
  std::fill(E->level_start.begin(), E->level_start.end(), 0);
  return EREM_OK;
}

erem_status erem_ensemble_run(erem_ens* E, int steps, void* stream) {
  if (!E) return EREM_EINVAL;
  if (steps < 1) return efail(E, EREM_EINVAL, "steps must be >= 1");
  const int U = E->cfg.tile_vecs ? E->cfg.tile_vecs : (E->tuned_U ? E->tuned_U : 2);
  if (!E->built || E->U != U) ENS_TRY(build(E, U));
  return run(E, steps, (cudaStream_t)stream);
}

erem_status erem_ensemble_autotune(erem_ens* E, int probe_steps, void* stream) {
  if (!E) return EREM_EINVAL;
  if (probe_steps < 1) return efail(E, EREM_EINVAL, "probe_steps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  long long tot = 0;
  for (int e = 0; e < E->n; ++e) tot += E->ctx[e]->Np;
  if (!E->snap_d && cudaMalloc((void**)&E->snap_d, sizeof(double) * tot) != cudaSuccess) {
    cudaGetLastError();
    E->snap_d = nullptr;
    return efail(E, EREM_ENOMEM, "cudaMalloc of the autotuner snapshot failed");
  }
  auto copy_all = [&](bool save) -> erem_status {
    long long off = 0;
    for (int e = 0; e < E->n; ++e) {
      const erem_ctx* c = E->ctx[e];
      double* a = E->snap_d + off;
      ENS_CUDA(E, cudaMemcpyAsync(save ? a : c->Tn, save ? c->Tn : a, sizeof(double) * c->Np,
                                  cudaMemcpyDeviceToDevice, s));
      off += c->Np;
    }
    return EREM_OK;
  };
  // A first probe from the current starting levels learns each member's
  // substep level (reached by doubling, as erem_step would); then every
  // tile size is timed on that schedule.
  const std::vector<int> levels0 = E->level_start;
  const erem_ens_config keep = E->cfg;
  const bool keep_policy = keep.substep_policy == EREM_ENS_KEEP_SUBSTEPS;
  auto restore = [&](erem_status st) {
    E->cfg = keep;
    E->level_start = levels0;
    E->built = false;
    copy_all(false);
    cudaStreamSynchronize(s);
    return st;
  };
  ENS_TRY(copy_all(true));
  const int U0 = keep.tile_vecs ? keep.tile_vecs : 2;
  erem_status st = build(E, U0);
  if (st == EREM_OK) st = run(E, probe_steps, s);
  if (st != EREM_OK) return restore(st);
  const std::vector<int> learned = E->level_start;
  if (copy_all(false) != EREM_OK) return restore(EREM_ECUDA);
  const int cand[3] = {1, 2, 4};
  double best = 1e300;
  int bestU = U0;
  for (int U : cand) {
    E->cfg.tile_vecs = U;
    E->level_start = keep_policy ? learned : levels0;
    st = build(E, U);
    if (st == EREM_OK) st = run(E, probe_steps, s);
    if (st != EREM_OK) return restore(st);
    if (E->rs.t_ms < best) {
      best = E->rs.t_ms;
      bestU = U;
    }
    if (copy_all(false) != EREM_OK) return restore(EREM_ECUDA);
  }
  ENS_CUDA(E, cudaStreamSynchronize(s));
  E->cfg = keep;
  E->tuned_U = bestU;
  E->level_start = keep_policy ? learned : levels0;
  E->built = false;
  return EREM_OK;
}

erem_status erem_ensemble_member_stats(const erem_ens* E, int e, erem_ens_member_stats* out) {
  if (!E || !out || e < 0 || e >= E->n) return EREM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->alpha = E->ctx[e]->alpha;
  out->beta = E->ctx[e]->beta;
  if (E->last.empty()) return EREM_OK;
  const EnsState& st = E->last[e];
  out->status = st.phase != ENS_FAILED ? EREM_OK
                                       : (st.status == ENS_NONFINITE ? EREM_ENONFINITE : EREM_ENOTCONV);
  out->steps_done = st.step;
  out->substeps = st.last_S;
  for (int k = 0; k < 64; ++k) {
    out->degrees[k] = st.last_deg[k];
    out->degree_total += st.last_deg[k];
  }
  out->terms = st.terms;
  out->passes = st.passes;
  out->attempts = st.attempts;
  return EREM_OK;
}

erem_status erem_ensemble_run_stats(const erem_ens* E, erem_ens_run_stats* out) {
  if (!E || !out) return EREM_EINVAL;
  *out = E->rs;
  return EREM_OK;
}

const char* erem_ensemble_last_error(const erem_ens* E) {
  return E ? E->err.c_str() : "erem: NULL ensemble";
}

}  // extern "C"
