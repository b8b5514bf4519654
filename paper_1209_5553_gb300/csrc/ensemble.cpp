// Batched ensembles of independent 2D EREM problems (declared in
// include/erem.h): member contexts, the member table the batched kernel
// reads, the divided-difference tables of every substep level, the queue
// order of a run and the cluster-size autotuner.
//
// Each member is a full context (erem_create / erem_set_state build its
// Jacobian, its Leja copy of J and its spectral interval exactly as for a
// single problem); the batched kernel (ensemble_cluster.cu) then runs every
// member on one thread-block cluster, using the member's own buffers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
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

  // Leja options and batching configuration
  double tol_a = 1e-6, tol_r = 1e-6;
  int p_order = 2, m_max = 150, max_doublings = 6, avg_window = 5;
  erem_ens_config cfg{EREM_ENS_KEEP_SUBSTEPS, 0, 0, 0};
  int tuned_cs = 0;

  // divided differences of every member and level (host copy, reused by
  // rebuilds until a member or the options change)
  std::vector<double> dd_host;
  bool dd_valid = false;

  // batch tables (valid while built)
  bool built = false;
  int nlev = 7;
  std::vector<int> level_start;     // KEEP policy: first level of each member's next step
  std::vector<double> pass_rate;    // passes per step of each member's last run (0: none yet)
  EnsMember* mem_d = nullptr;
  EnsState* st_d = nullptr;
  EnsState* st_h = nullptr;         // pinned
  double* dd_d = nullptr;
  double* xi_d = nullptr;
  int* order_d = nullptr;
  int* order_h = nullptr;           // pinned
  unsigned* next_d = nullptr;       // queue position
  double* snap_d = nullptr;         // autotuner: saved temperatures
  double* stage_d = nullptr;        // host-pointer staging (largest member)
  cudaEvent_t ev[2] = {nullptr, nullptr};

  // the run as a CUDA graph (state and queue upload, the persistent launch,
  // state read-back), captured once per run descriptor and cluster shape
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t run_exec = nullptr;
  EnsRun run_key{};
  int key_cs = 0, key_clusters = 0;
  bool graph_ok = true;             // false after a failed capture: direct launches

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

void drop_graph(erem_ens* E) {
  if (E->run_exec) cudaGraphExecDestroy(E->run_exec);
  E->run_exec = nullptr;
}

void release_tables(erem_ens* E) {
  drop_graph(E);
  void* dp[] = {E->mem_d, E->st_d, E->dd_d, E->xi_d, E->order_d, E->next_d};
  for (void* p : dp)
    if (p) cudaFree(p);
  E->mem_d = nullptr;
  E->st_d = nullptr;
  E->dd_d = nullptr;
  E->xi_d = nullptr;
  E->order_d = nullptr;
  E->next_d = nullptr;
  if (E->st_h) cudaFreeHost(E->st_h);
  if (E->order_h) cudaFreeHost(E->order_h);
  E->st_h = nullptr;
  E->order_h = nullptr;
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

// Passes one step of a member may take at most: every level's substeps,
// each with m_max terms, the term pass that follows the decision, and its
// start and bookkeeping passes.
long long passes_per_step(const erem_ens* E) {
  long long per_step = 2;
  for (int l = 0; l < E->nlev; ++l) per_step += (1LL << l) * (E->m_max + 3) + 2;
  return per_step;
}

// Member table, divided differences and queue for the current options.
erem_status build(erem_ens* E) {
  for (int e = 0; e < E->n; ++e)
    if (!E->ready[e])
      return efail(E, EREM_EINVAL, "member " + std::to_string(e) + " has no state (erem_ensemble_set_member)");
  release_tables(E);
  E->nlev = E->max_doublings + 1;
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
  ENS_TRY(ens_alloc(E, &E->dd_d, dd.size()));
  ENS_TRY(ens_alloc(E, &E->xi_d, (size_t)M + 1));
  ENS_TRY(ens_alloc(E, &E->order_d, (size_t)E->n));
  ENS_TRY(ens_alloc(E, &E->next_d, (size_t)1));
  if (cudaMallocHost((void**)&E->st_h, sizeof(EnsState) * E->n) != cudaSuccess ||
      cudaMallocHost((void**)&E->order_h, sizeof(int) * E->n) != cudaSuccess)
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
    for (int k = 0; k < 5; ++k) m.jc[k] = c->jc[k];
    m.b0 = c->b0;
    m.jl = c->jl_all;
    m.r0 = c->jl_nodiag ? c->jl_r0 : nullptr;
    m.T = c->Tn;
    m.G = c->vrhs;
    m.w = c->w;
    m.P = c->P;
    m.q[0] = c->q[0];
    m.q[1] = c->q[1];
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
  E->built = true;
  return EREM_OK;
}

// Cluster size of the next run and the clusters that fit at once.
erem_status cluster_shape(erem_ens* E, int* cs, int* clusters) {
  *cs = E->cfg.cluster_ctas ? E->cfg.cluster_ctas : (E->tuned_cs ? E->tuned_cs : 8);
  int fit = 0;
  ENS_CUDA(E, ens_max_clusters(E->prec, *cs, &fit));
  if (fit < 1)
    return efail(E, EREM_ECUDA, "a cluster of " + std::to_string(*cs) + " CTAs does not fit the device");
  if (E->cfg.max_clusters > 0) fit = std::min(fit, E->cfg.max_clusters);
  *clusters = std::min(fit, E->n);
  return EREM_OK;
}

// Work estimate of member e for the queue order: its passes per step (from
// its last run, else the width of its spectral interval as a proxy for the
// Leja degree) times its cells plus a latency term of a pass.
double member_weight(const erem_ens* E, int e) {
  const erem_ctx* c = E->ctx[e];
  const double rate = E->pass_rate[e] > 0.0 ? E->pass_rate[e] : 1.0 + c->gam;
  return rate * ((double)c->Np + 16384.0);
}

bool same_run(const EnsRun& a, const EnsRun& b) {
  return a.mem == b.mem && a.st == b.st && a.order == b.order && a.next == b.next && a.xi == b.xi &&
         a.n == b.n && a.nlev == b.nlev && a.mmax == b.mmax && a.restart == b.restart &&
         a.passes_per_step == b.passes_per_step;
}

// The device work of a run, in stream order: the member states and the queue
// order up from pinned host memory, the queue position reset, the persistent
// launch, the states back.  The copies read and write the pinned buffers when
// they execute, so one capture serves every run with the same descriptor.
cudaError_t enqueue_run(erem_ens* E, const EnsRun& R, int cs, int clusters, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(E->st_d, E->st_h, sizeof(EnsState) * E->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(E->order_d, E->order_h, sizeof(int) * E->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E->next_d, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_ens_cluster(R, E->prec, cs, clusters, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(E->st_h, E->st_d, sizeof(EnsState) * E->n, cudaMemcpyDeviceToHost, s);
  return e;
}

// Capture the run on the ensemble's own stream (a legacy default stream
// cannot be captured) and instantiate it; on any failure the ensemble keeps
// to direct launches.
void capture_run(erem_ens* E, const EnsRun& R, int cs, int clusters) {
  if (!E->cap_stream && cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    E->cap_stream = nullptr;
    E->graph_ok = false;
    return;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    E->graph_ok = false;
    return;
  }
  const cudaError_t e = enqueue_run(E, R, cs, clusters, E->cap_stream);
  const cudaError_t ee = cudaStreamEndCapture(E->cap_stream, &g);
  cudaGraphExec_t x = nullptr;
  if (e != cudaSuccess || ee != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    E->graph_ok = false;
    return;
  }
  cudaGraphDestroy(g);
  E->run_exec = x;
  E->run_key = R;
  E->key_cs = cs;
  E->key_clusters = clusters;
}

// One run: every member advances `steps` steps, one launch of the batched
// kernel.  A member whose Leja estimate became non-finite (the Newton
// vectors or their squares left the range of the Leja precision) or whose
// interpolation did not meet the test within m_max terms takes the step again
// at twice the substeps, as erem_step splits a step whose interpolation
// failed.
erem_status run(erem_ens* E, int steps, cudaStream_t s) {
  int cs = 0, clusters = 0;
  ENS_TRY(cluster_shape(E, &cs, &clusters));
  const bool keep = E->cfg.substep_policy == EREM_ENS_KEEP_SUBSTEPS;
  for (int e = 0; e < E->n; ++e) {
    EnsState& st = E->st_h[e];
    std::memset(&st, 0, sizeof(st));
    st.phase = ENS_INIT;
    st.level = std::min(keep ? E->level_start[e] : 0, E->nlev - 1);
    st.target = steps;
  }
  std::vector<std::pair<double, int>> w(E->n);
  for (int e = 0; e < E->n; ++e) w[e] = {member_weight(E, e), e};
  std::stable_sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  for (int k = 0; k < E->n; ++k) E->order_h[k] = w[k].second;

  EnsRun R{};
  R.mem = E->mem_d;
  R.st = E->st_d;
  R.order = E->order_d;
  R.next = E->next_d;
  R.xi = E->xi_d;
  R.n = E->n;
  R.nlev = E->nlev;
  R.mmax = E->m_max;
  R.restart = keep ? 0 : 1;
  R.passes_per_step = passes_per_step(E);
  if (const char* v = std::getenv("EREM_ENS_PASSES_PER_STEP")) {  // test hook: a small bound
    const long long b = std::atoll(v);
    if (b >= 1) R.passes_per_step = b;
  }
  if (E->graph_ok) {
    if (E->run_exec && !(same_run(R, E->run_key) && cs == E->key_cs && clusters == E->key_clusters))
      drop_graph(E);
    if (!E->run_exec) capture_run(E, R, cs, clusters);
  }
  // the events bracket the whole run: copies, queue reset and the launch
  ENS_CUDA(E, cudaEventRecord(E->ev[0], s));
  if (E->run_exec)
    ENS_CUDA(E, cudaGraphLaunch(E->run_exec, s));
  else
    ENS_CUDA(E, enqueue_run(E, R, cs, clusters, s));
  ENS_CUDA(E, cudaEventRecord(E->ev[1], s));
  ENS_CUDA(E, cudaStreamSynchronize(s));
  float t = 0.f;
  ENS_CUDA(E, cudaEventElapsedTime(&t, E->ev[0], E->ev[1]));

  erem_ens_run_stats& r = E->rs;
  std::memset(&r, 0, sizeof(r));
  r.t_ms = t;
  r.cluster_ctas = cs;
  r.clusters = clusters;
  r.cta_threads = ens_cta_threads();
  r.graph = E->run_exec ? 1 : 0;
  E->last.assign(E->st_h, E->st_h + E->n);
  int first_fail = -1;
  for (int e = 0; e < E->n; ++e) {
    const EnsState& st = E->last[e];
    const long long N = E->ctx[e]->N;
    r.passes += st.terms + st.passes;
    r.cells += N;
    r.cell_terms += N * st.terms;
    r.cell_passes += N * st.passes;
    if (st.step > 0) E->pass_rate[e] = (double)(st.terms + st.passes) / st.step;
    if (st.phase == ENS_FAILED) {
      ++r.members_failed;
      if (first_fail < 0) first_fail = e;
    } else if (st.last_S > 0) {
      int l = 0;
      while ((1 << l) < st.last_S) ++l;
      E->level_start[e] = l;
    }
  }
  if (first_fail >= 0) {
    const EnsState& st = E->last[first_fail];
    const std::string who = "member " + std::to_string(first_fail);
    if (st.status == ENS_NONFINITE)
      return efail(E, EREM_ENONFINITE, who + ": non-finite value in the state or the Leja estimate");
    if (st.status == ENS_TIMEOUT)
      return efail(E, EREM_ETIMEOUT, who + ": the member reached its bound on passes");
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
  E->pass_rate.assign(n_members, 0.0);
  auto bail = [&](erem_status st) {
    erem_ensemble_destroy(E);
    return st;
  };
  long long maxN = 1;
  for (int e = 0; e < n_members; ++e) {
    const erem_status st = erem_create(&grids[e], &phys[e], prec, &E->ctx[e]);
    if (st != EREM_OK) return bail(st);
    maxN = std::max(maxN, E->ctx[e]->N);
  }
  if (cudaMalloc((void**)&E->stage_d, sizeof(double) * maxN) != cudaSuccess) return bail(EREM_ENOMEM);
  if (cudaEventCreate(&E->ev[0]) != cudaSuccess || cudaEventCreate(&E->ev[1]) != cudaSuccess)
    return bail(EREM_ECUDA);
  if (const char* v = std::getenv("EREM_ENS_GRAPH")) E->graph_ok = std::atoi(v) != 0;  // 0: direct launches
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
  if (E->cap_stream) cudaStreamDestroy(E->cap_stream);
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
  E->pass_rate[e] = 0.0;
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
  if (m_max < 1 || m_max > kMaxTerms || avg_window < 1 || avg_window > kEnsWin || p_order < 0 ||
      p_order > 30 || max_doublings < 0 || max_doublings > kEnsMaxLevels - 1)
    return efail(E, EREM_EINVAL, "bad m_max, avg_window (1..64), p_order or max_doublings (0..6)");
  erem_ens_config c = E->cfg;
  if (cfg) {
    c = *cfg;
    if (c.substep_policy != EREM_ENS_KEEP_SUBSTEPS && c.substep_policy != EREM_ENS_RESTART_SUBSTEPS)
      return efail(E, EREM_EINVAL, "unknown substep policy");
    if (c.cluster_ctas != 0 && c.cluster_ctas != 2 && c.cluster_ctas != 4 && c.cluster_ctas != 8 &&
        c.cluster_ctas != 16)
      return efail(E, EREM_EINVAL, "cluster_ctas must be 0, 2, 4, 8 or 16");
    if (c.max_clusters < 0) return efail(E, EREM_EINVAL, "max_clusters must be >= 0");
    if (c.reserved != 0) return efail(E, EREM_EINVAL, "reserved must be 0");
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
  std::fill(E->pass_rate.begin(), E->pass_rate.end(), 0.0);
  return EREM_OK;
}

erem_status erem_ensemble_run(erem_ens* E, int steps, void* stream) {
  if (!E) return EREM_EINVAL;
  if (steps < 1) return efail(E, EREM_EINVAL, "steps must be >= 1");
  if (!E->built) ENS_TRY(build(E));
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
  // substep level (reached by doubling, as erem_step would) and its passes
  // per step (the queue order); then every cluster size that fits is timed
  // on that schedule.
  const std::vector<int> levels0 = E->level_start;
  const std::vector<double> rates0 = E->pass_rate;
  const erem_ens_config keep = E->cfg;
  const bool keep_policy = keep.substep_policy == EREM_ENS_KEEP_SUBSTEPS;
  auto restore = [&](erem_status st) {
    E->cfg = keep;
    E->level_start = levels0;
    E->pass_rate = rates0;
    copy_all(false);
    cudaStreamSynchronize(s);
    return st;
  };
  ENS_TRY(copy_all(true));
  erem_status st = E->built ? EREM_OK : build(E);
  if (st == EREM_OK) st = run(E, probe_steps, s);
  if (st != EREM_OK) return restore(st);
  const std::vector<int> learned = E->level_start;
  const std::vector<double> rates = E->pass_rate;
  if (copy_all(false) != EREM_OK) return restore(EREM_ECUDA);
  const int cand[4] = {2, 4, 8, 16};
  double best = 1e300;
  int best_cs = 0;
  for (int cs : cand) {
    int fit = 0;
    if (ens_max_clusters(E->prec, cs, &fit) != cudaSuccess || fit < 1) {
      cudaGetLastError();
      continue;
    }
    E->cfg.cluster_ctas = cs;
    E->level_start = keep_policy ? learned : levels0;
    E->pass_rate = rates;
    st = run(E, probe_steps, s);
    if (st != EREM_OK) return restore(st);
    if (E->rs.t_ms < best) {
      best = E->rs.t_ms;
      best_cs = cs;
    }
    if (copy_all(false) != EREM_OK) return restore(EREM_ECUDA);
  }
  ENS_CUDA(E, cudaStreamSynchronize(s));
  if (best_cs == 0) return restore(efail(E, EREM_ECUDA, "no cluster size fits the device"));
  E->cfg = keep;
  E->tuned_cs = best_cs;
  E->level_start = keep_policy ? learned : levels0;
  E->pass_rate = rates;
  return EREM_OK;
}

erem_status erem_ensemble_member_stats(const erem_ens* E, int e, erem_ens_member_stats* out) {
  if (!E || !out || e < 0 || e >= E->n) return EREM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->alpha = E->ctx[e]->alpha;
  out->beta = E->ctx[e]->beta;
  out->leja_coefficients = erem_leja_coefficients(E->ctx[e]);
  if (E->last.empty()) return EREM_OK;
  const EnsState& st = E->last[e];
  out->status = st.phase != ENS_FAILED       ? EREM_OK
                : st.status == ENS_NONFINITE ? EREM_ENONFINITE
                : st.status == ENS_TIMEOUT   ? EREM_ETIMEOUT
                                             : EREM_ENOTCONV;
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
