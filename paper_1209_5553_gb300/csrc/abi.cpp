// C ABI of the EREM library (declared in include/erem.h): contexts, pointer
// staging, and the host loops that drive the device kernels.
//
// The Leja loop (§4.2) runs without a host round trip per term: each term
// kernel's last block evaluates the stopping test on the device and raises
// `done`; later term kernels of the same chunk see it and return at once.
// The host launches a chunk of terms (sized from the previous degree), then
// reads the control block once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <string>

#include "erem_internal.h"

using namespace erem;

namespace {

const char* const kNullCtxMsg = "erem: NULL context";

erem_status fail(erem_ctx* c, erem_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define EREM_CUDA(ctx, call)                                                         \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      return fail((ctx), EREM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                \
  } while (0)

#define EREM_TRY(expr)              \
  do {                              \
    erem_status st_ = (expr);       \
    if (st_ != EREM_OK) return st_; \
  } while (0)

erem_status check_launch(erem_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, EREM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return EREM_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory that the GPU can reach
// directly (mapped under unified addressing; over NVLink-C2C on Grace
// systems), or nullptr.
double* host_mapped(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<double*>(a.devicePointer);
}

erem_status dalloc(erem_ctx* c, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, EREM_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  if (cudaMemset(*p, 0, bytes) != cudaSuccess) return fail(c, EREM_ECUDA, "cudaMemset failed");
  return EREM_OK;
}

template <typename T>
erem_status dalloc_t(erem_ctx* c, T** p, size_t count) {
  return dalloc(c, reinterpret_cast<void**>(p), count * sizeof(T));
}

// Device pointer for a caller array of N doubles: the pointer itself when it
// is device memory, else a context staging buffer (filled when copy_in).
erem_status resolve(erem_ctx* c, int slot, const double* ptr, bool copy_in, cudaStream_t s,
                    double** out) {
  if (!ptr) return fail(c, EREM_EINVAL, "NULL array argument");
  if ((slot == 0 && c->zc_active) || is_device_ptr(ptr)) {
    *out = const_cast<double*>(ptr);
    return EREM_OK;
  }
  if (!c->stage[slot]) EREM_TRY(dalloc_t(c, &c->stage[slot], (size_t)c->N));
  if (copy_in)
    EREM_CUDA(c, cudaMemcpyAsync(c->stage[slot], ptr, (size_t)c->N * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
  *out = c->stage[slot];
  return EREM_OK;
}

erem_status ensure_krylov(erem_ctx* c) {
  if (c->kv[0]) return EREM_OK;
  for (int k = 0; k < 12; ++k) EREM_TRY(dalloc_t(c, &c->kv[k], (size_t)c->Np));
  return EREM_OK;
}

erem_status read_ctrl(erem_ctx* c, cudaStream_t s) {
  EREM_CUDA(c, cudaMemcpyAsync(c->ctrl_h, c->ctrl, offsetof(Ctrl, e), cudaMemcpyDeviceToHost, s));
  EREM_CUDA(c, cudaStreamSynchronize(s));
  return EREM_OK;
}

erem_status check_flags(erem_ctx* c) {
  if (c->ctrl_h->flags & FLAG_NONFINITE)
    return fail(c, EREM_ENONFINITE, "non-finite value in an input field or its derived coefficients");
  if (c->ctrl_h->flags & FLAG_BAD_INPUT)
    return fail(c, EREM_EINVAL, "negative conductivity, porosity outside [0,1] or non-positive capacity");
  return EREM_OK;
}

erem_status ensure_pc(erem_ctx* c) {
  if (c->pc[0]) return EREM_OK;
  for (int k = 0; k < 8; ++k) EREM_TRY(dalloc_t(c, &c->pc[k], (size_t)c->Np));
  return EREM_OK;
}

// Chebyshev iteration on [2/deg^2, 2] (the spectrum of D^-1 A lies in
// (0, 2]; the lower end trades the compression of the upper spectrum against
// the reach towards 0, deg^2 measured best on the channel reservoirs):
// theta, delta = centre and half-width, sigma = theta/delta, rho_0 = 1/sigma,
// rho_j = 1/(2 sigma - rho_{j-1}); step j >= 1 adds rho_j rho_{j-1} times the
// previous increment and 2 rho_j / delta times the scaled residual.
PcPoly pc_poly(int deg, double lo = -1.0) {
  PcPoly P;
  P.deg = deg;
  const double hi = 2.0;
  if (lo < 0.0) lo = 2.0 / ((double)deg * deg);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  P.c2[0] = 1.0 / theta;
  for (int j = 1; j < deg; ++j) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    P.c1[j] = rn * rho;
    P.c2[j] = 2.0 * rn / delta;
    rho = rn;
  }
  return P;
}

// Levels of the pressure multigrid: halve every dimension > 1 (rounding up)
// until at most kMgCoarsest cells remain (at least one coarse level).  A small
// coarsest level keeps its one-block solve short (a few dozen barriers).
erem_status ensure_mg(erem_ctx* c) {
  if (!c->pc_diag) EREM_TRY(dalloc_t(c, &c->pc_diag, (size_t)c->Np));
  if (!c->mg.empty()) return EREM_OK;
  int nx = c->nx, ny = c->ny, nz = c->nz;
  while (c->mg.empty() || (long long)nx * ny * nz > kMgCoarsest) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = c->dim == 3 ? (nz + 1) / 2 : 1;
    if (!c->mg.empty() && cx == nx && cy == ny && cz == nz) break;
    nx = cx;
    ny = cy;
    nz = cz;
    MgLevel m;
    m.nx = nx;
    m.ny = ny;
    m.nz = nz;
    const size_t n = (size_t)nx * ny * nz;
    c->mg.push_back(m);
    MgLevel& L = c->mg.back();
    for (float** a : {&L.diag, &L.dinv, &L.Ux, &L.Uy, &L.rhs, &L.x[0], &L.x[1], &L.x[2], &L.x[3]})
      EREM_TRY(dalloc_t(c, a, n));
    if (c->dim == 3) EREM_TRY(dalloc_t(c, &L.Uz, n));
  }
  MgLevel& last = c->mg.back();  // at most 512 cells: its inverse, at most 1 MB
  const size_t nc = (size_t)last.nx * last.ny * last.nz;
  if (nc <= (size_t)kMgCoarsest) EREM_TRY(dalloc_t(c, &last.inv, nc * nc));
  return EREM_OK;
}

// The graph of two preconditioned iterations (their kernels' arguments are
// fixed for the context and preconditioner; the scalars live on the device).
// Captured on a stream of the context's own, so any caller stream may replay
// it.  Returns false when capture is not available (the caller then launches
// the kernels itself).
bool ensure_pcg_graph(erem_ctx* c, const PcPoly& P, const float* z) {
  const long long key = ((long long)c->pc_deg << 40) ^ ((long long)c->mg_nu << 32) ^
                        (long long)(c->mg_omega * 1e6f);
  if (c->pcg_exec && c->pcg_key == key) return true;
  if (c->bicg_exec) cudaGraphExecDestroy(c->bicg_exec);
  if (c->bicg_graph) cudaGraphDestroy(c->bicg_graph);
  if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
  if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
  c->pcg_exec = nullptr;
  c->pcg_graph = nullptr;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    return false;
  }
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const long long before = c->launches;
  launch_pcg_iter(c, P, z, 0, c->cap_stream);
  launch_pcg_iter(c, P, z, 1, c->cap_stream);
  c->pcg_kernels = (int)(c->launches - before);
  c->launches = before;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(c->cap_stream, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return false;
  }
  if (cudaGraphInstantiate(&c->pcg_exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    c->pcg_exec = nullptr;
    return false;
  }
  c->pcg_graph = g;
  c->pcg_key = key;
  return true;
}

// CG on the pressure system whose matrix and right-hand side the caller has
// assembled into kv (initial guess in kv[0]): Jacobi-preconditioned for
// pc_deg = 1, else flexible CG with the FP32 polynomial preconditioner
// (pc_deg >= 2) or the multigrid V-cycle (pc_deg = 0).
erem_status run_pressure_cg(erem_ctx* c, double tol, int maxit, cudaStream_t s) {
  const bool prec = c->pc_deg != 1;
  const bool mg = c->pc_deg == 0;
  PcPoly P;
  const float* z = nullptr;
  launch_cg_init(c, tol, s);
  EREM_TRY(check_launch(c, "pressure CG set-up"));
  EREM_TRY(read_ctrl(c, s));
  EREM_TRY(check_flags(c));
  if (prec && !c->ctrl_h->lin_done) {  // nothing to precondition when the guess solves it
    EREM_TRY(ensure_pc(c));
    if (mg) EREM_TRY(ensure_mg(c));
    // the multigrid smoother damps the upper part [1/4, 2] of the spectrum
    P = mg ? pc_poly(c->mg_nu, 0.25) : pc_poly(c->pc_deg);
    launch_pc_setup(c, s);
    if (mg) launch_mg_setup(c, s);
    z = launch_pc_apply(c, P, s);
    EREM_TRY(check_launch(c, "pressure preconditioner set-up"));
    EREM_TRY(read_ctrl(c, s));
  }
  int chunk = mg ? 2 : (prec ? std::max(2, 64 / c->pc_deg) : 32);
  const bool graph = prec && !c->ctrl_h->lin_done && ensure_pcg_graph(c, P, z);
  if (graph) chunk = (chunk + 1) / 2 * 2;  // whole even/odd pairs
  int k = 0;
  while (!c->ctrl_h->lin_done && k < maxit) {
    const int n = std::min(chunk, maxit - k);
    if (graph && n % 2 == 0) {
      for (int j = 0; j < n; j += 2) {
        EREM_CUDA(c, cudaGraphLaunch(c->pcg_exec, s));
        c->launches += c->pcg_kernels;
      }
    } else {
      for (int j = 0; j < n; ++j) {
        if (prec) launch_pcg_iter(c, P, z, k + j, s);
        else launch_cg_iter(c, k + j, s);
      }
    }
    EREM_TRY(check_launch(c, "cg"));
    k += n;
    EREM_TRY(read_ctrl(c, s));
  }
  return EREM_OK;
}

erem_status ensure_leja(erem_ctx* c, int M) {
  if (M <= c->xi_cap) return EREM_OK;
  if (M > kMaxTerms) return fail(c, EREM_EINVAL, "m_max above " + std::to_string(kMaxTerms));
  int cap = std::max(M, 2 * c->xi_cap);
  cap = std::min(cap, kMaxTerms);
  if (c->leja_kind == EREM_LEJA_FAST) fast_leja_table(cap, &c->xi_host);
  else leja_table(cap, &c->xi_host);
  if (c->xi_dev) cudaFree(c->xi_dev);
  c->xi_dev = nullptr;
  EREM_TRY(dalloc_t(c, &c->xi_dev, (size_t)cap + 1));
  EREM_CUDA(c, cudaMemcpy(c->xi_dev, c->xi_host.data(), (cap + 1) * sizeof(double),
                          cudaMemcpyHostToDevice));
  c->xi_cap = cap;
  return EREM_OK;
}

// [alpha, beta] = dt times the held bounds, else dt times the Gershgorin
// bounds of the last assembly.
void set_interval(erem_ctx* c) {
  c->alpha = c->dt * (c->hold_iv ? c->hold_lo : c->ctrl_h->gmin);
  c->beta = c->dt * (c->hold_iv ? c->hold_hi : c->ctrl_h->gmax);
}

void focal_map(erem_ctx* c) {
  c->cfoc = 0.5 * (c->alpha + c->beta);
  double g = 0.25 * (c->beta - c->alpha);
  const double floor = 1e-8 * std::max(1.0, std::fabs(c->cfoc));
  c->gam = std::max(g, floor);
}

// Divided differences of level S (interval / S) with at least M+1 entries
// (of phi_1, or phi_2 for phi = 2), on the device in dd_dev.
int dd_key(int S, int phi) { return 8 * S + phi; }
DDEntry& dd_entry(erem_ctx* c, int S, int phi = 1) { return c->dd_cache[dd_key(S, phi)]; }

erem_status prepare_dd(erem_ctx* c, int S, int M, cudaStream_t s, int phi = 1,
                       bool take_spec = true) {
  DDEntry& e = dd_entry(c, S, phi);
  const int key = dd_key(S, phi);
  const double cc = c->cfoc / S, gg = c->gam / S;
  if (e.M < M || e.c != cc || e.gamma != gg) {
    e.c = cc;
    e.gamma = gg;
    erem_ctx::DDSpec* sp = nullptr;
    for (auto& x : c->dd_spec)
      if (take_spec && x.f.valid() && x.key == key && x.kind == c->leja_kind && x.M >= M &&
          x.c == cc && x.g == gg)
        sp = &x;
    if (sp) {
      // computed ahead on host threads (the same function of the same inputs)
      e.d = sp->f.get();
      e.M = sp->M;
    } else {
      e.M = M;
      e.d.assign(M + 1, 0.0);
      if (divided_differences_phi(phi, M, c->xi_host.data(), cc, gg, e.d.data(), kDdThreads) != 0)
        e.d.clear();
    }
    if (e.d.empty()) {
      e.M = -1;
      return fail(c, EREM_EINVAL, "divided differences: bad interval");
    }
    for (double v : e.d)
      if (!std::isfinite(v)) {
        e.M = -1;  // not cached: a later call with this interval fails the same way
        return fail(c, EREM_ENONFINITE, "non-finite divided difference");
      }
    c->dd_tag_S = -1;
  }
  if (c->dd_tag_S != key || c->dd_tag_M != e.M) {
    std::memcpy(c->dd_h, e.d.data(), (e.M + 1) * sizeof(double));
    EREM_CUDA(c, cudaMemcpyAsync(c->dd_dev, c->dd_h, (e.M + 1) * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    c->dd_tag_S = key;
    c->dd_tag_M = e.M;
  }
  return EREM_OK;
}

// Start the phi_1 table of substep level S (M + 1 entries) on host threads;
// prepare_dd takes it if that level is reached with the same interval.  Two
// tables may be under way; a third waits for the older one.
void speculate_dd(erem_ctx* c, int S, int M) {
  const int key = dd_key(S, 1);
  const double cc = c->cfoc / S, gg = c->gam / S;
  const DDEntry& e = dd_entry(c, S, 1);
  if (e.M >= M && e.c == cc && e.gamma == gg) return;  // cached
  for (auto& x : c->dd_spec)
    if (x.f.valid() && x.key == key && x.kind == c->leja_kind && x.M >= M && x.c == cc && x.g == gg)
      return;  // already under way
  erem_ctx::DDSpec* slot = nullptr;
  for (auto& x : c->dd_spec)
    if (!x.f.valid()) slot = &x;
  if (!slot) {  // both busy: reuse the older one
    slot = &c->dd_spec[0];
    slot->f.wait();
    std::swap(c->dd_spec[0], c->dd_spec[1]);
    slot = &c->dd_spec[1];
  }
  std::vector<double> xi(c->xi_host.begin(), c->xi_host.begin() + M + 1);
  try {
    slot->f = std::async(std::launch::async, [xi = std::move(xi), M, cc, gg]() {
      std::vector<double> d(M + 1, 0.0);
      if (divided_differences_phi(1, M, xi.data(), cc, gg, d.data(), kDdThreads) != 0) d.clear();
      return d;
    });
  } catch (...) {  // no thread: prepare_dd computes the table itself
    slot->f = std::future<std::vector<double>>();
    return;
  }
  slot->key = key;
  slot->kind = c->leja_kind;
  slot->M = M;
  slot->c = cc;
  slot->g = gg;
}

struct Opts {
  double tol_a = 1e-6, tol_r = 1e-6;
  int p_order = 2, m_max = 150, max_doublings = 6, avg_window = 5;
  std::vector<int> replay;
  bool time_terms = false;
};

erem_status parse_opts(erem_ctx* c, const erem_leja_opts* o, Opts* out) {
  Opts r;
  if (o) {
    if (o->tol_a != 0.0) r.tol_a = o->tol_a;
    if (o->tol_r != 0.0) r.tol_r = o->tol_r;
    if (o->p_order != 0) r.p_order = o->p_order;
    if (o->m_max != 0) r.m_max = o->m_max;
    r.max_doublings = o->max_doublings;
    if (o->avg_window != 0) r.avg_window = o->avg_window;
    r.time_terms = o->time_terms != 0;
    if (o->replay) {
      if (o->n_replay < 2) return fail(c, EREM_EINVAL, "replay needs [s, m_1..m_s]");
      const int S = o->replay[0];
      if (S < 1 || S > 64 || o->n_replay != 1 + S)
        return fail(c, EREM_EINVAL, "replay: s must be 1..64 and n_replay = 1 + s");
      for (int k = 1; k <= S; ++k)
        if (o->replay[k] < 1 || o->replay[k] > kMaxTerms)
          return fail(c, EREM_EINVAL, "replay degree out of range");
      r.replay.assign(o->replay, o->replay + o->n_replay);
    }
  }
  if (!(r.tol_a >= 0.0) || !(r.tol_r >= 0.0) || r.tol_a + r.tol_r <= 0.0)
    return fail(c, EREM_EINVAL, "tolerances must be >= 0 with tol_a + tol_r > 0");
  if (r.m_max < 1 || r.m_max > kMaxTerms) return fail(c, EREM_EINVAL, "m_max out of range");
  if (r.avg_window < 1 || r.p_order < 0 || r.p_order > 30 || r.max_doublings < 0 ||
      r.max_doublings > 6)
    return fail(c, EREM_EINVAL, "bad avg_window, p_order or max_doublings (0..6)");
  *out = r;
  return EREM_OK;
}

erem_status ensure_events(erem_ctx* c, int n) {
  while ((int)c->ev.size() < 2 * n) {
    cudaEvent_t e;
    EREM_CUDA(c, cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  return EREM_OK;
}

// out (unpadded, device) = base + dt phi_1(dt J) src, with src and base padded
// device vectors (base may be null).  J, dt, alpha, beta and the Leja copy of
// J must be current.  With fused_T (linear fluid model) the first substep is
// started by the fused kernel that computes src = J T + b and base = T^n from
// the caller's T itself.
// Device time of the Leja launches of a call (time_terms).
struct TermTiming {
  double ms = 0.0;
  int terms = 0, launches = 0;
};

// One Newton interpolation (§4.2) at substep level S with the table of phi
// (prepared in dd_dev): q_0 = u (or, for the fused first kernel, G(T) from
// fused_T), P = sum_m d_m q_m, the terms launched in chunks and stopped by
// the device test (StopParams sp) or at the forced degree.  *degree gets m;
// *failed is set when m_max terms do not meet the test, *nonfinite when the
// estimate left the range of the Leja precision.  The term kernel adds the
// products d_m q_m to P in pairs (at odd m): when the degree is even, the
// last one is still to be added.  With fix, the caller's consumer of P adds
// it (fix->q = q_M, or null when P is complete); without, it is added here.
erem_status leja_interp(erem_ctx* c, const double* u, const double* fused_T, int S, int phi,
                        int* M_avail, int mcap, const StopParams& sp, int forced, const Opts& o,
                        TermTiming* tt, int* degree, bool* failed, bool* nonfinite,
                        cudaStream_t s, PFixHost* fix = nullptr) {
  const double cg = c->cfoc / c->gam;  // the same for every substep level
  *failed = *nonfinite = false;
  if (fix) *fix = PFixHost{};
  if (fused_T)  // also writes vrhs = G(T)
    launch_step_init(c, fused_T, sp, s);
  else
    launch_leja_init(c, u, sp, s);
  // taping (phi_1 of erem_step): the terms write q_m straight into the tape,
  // slot m of this interpolation, when the arena has room for every term
  const size_t qbytes = (size_t)c->Np * (c->prec == EREM_FP32_BULK ? sizeof(float) : sizeof(double));
  char* slot0 = nullptr;
  if (c->rec_ok && phi == 1) {
    const size_t need = (size_t)(forced ? forced : *M_avail) + 1;
    if (c->tape_used + need * qbytes <= c->tape_cap) {
      slot0 = c->tape + c->tape_used;
      c->rec.q_off.push_back(c->tape_used);
      EREM_CUDA(c, cudaMemcpyAsync(slot0, c->q[0], qbytes, cudaMemcpyDeviceToDevice, s));
    } else {
      c->rec_ok = false;
    }
  }
  // small grids, untaped: each launch takes the stopping test of the term
  // before it (k_leja_term_lag), so the launch after the stopping term is
  // needed too: it completes P
  const int lag = (c->term_lag && !slot0) ? 1 : 0;
  if (lag) c->last_lag = true;
  int m = 1, qin = 0;
  int chunk = forced ? forced + lag : std::max(4, c->last_degree + 2 + lag);
  // the terms [first, last] of every chunk of launches, in order; with
  // time_terms a pair of events brackets each chunk (not each launch: an
  // event between two terms would stop the next one from being scheduled
  // while the previous one ends)
  std::vector<std::pair<int, int>> chunks;
  while (true) {
    const int end = forced ? forced + lag : std::min(*M_avail + lag, m + chunk - 1);
    if (o.time_terms) cudaEventRecord(c->ev[2 * chunks.size()], s);
    for (int mm = m; mm <= end; ++mm) {
      if (slot0)
        launch_leja_term_ptr(c, mm, slot0 + (size_t)(mm - 1) * qbytes, slot0 + (size_t)mm * qbytes,
                             cg, s);
      else if (lag) launch_leja_term_lag(c, mm, qin, cg, s);
      else launch_leja_term(c, mm, qin, cg, s);
      qin ^= 1;
    }
    if (o.time_terms) cudaEventRecord(c->ev[2 * chunks.size() + 1], s);
    chunks.emplace_back(m, end);
    EREM_TRY(check_launch(c, "leja term"));
    EREM_TRY(read_ctrl(c, s));
    EREM_TRY(check_flags(c));
    const Ctrl& h = *c->ctrl_h;
    if (h.nonfinite) {
      // the Newton vectors (or their squares) left the range of the Leja
      // precision: the interpolation at this substep length failed
      if (forced) return fail(c, EREM_ENONFINITE, "non-finite Leja error estimate");
      *nonfinite = *failed = true;
      return EREM_OK;
    }
    if (forced) {
      *degree = forced;
      break;
    }
    if (h.done && !h.fail) {
      *degree = h.degree;
      break;
    }
    if (h.fail || end >= o.m_max + lag) {
      *failed = true;
      return EREM_OK;
    }
    if (end >= *M_avail + lag) {  // table exhausted below m_max: extend it
      *M_avail = mcap;
      EREM_TRY(prepare_dd(c, S, *M_avail, s, phi));
      if (slot0 && c->tape_used + ((size_t)mcap + 1) * qbytes > c->tape_cap) {
        // the tape cannot hold the longer interpolation: go on untaped (the
        // remaining terms continue from the last taped slot)
        EREM_CUDA(c, cudaMemcpyAsync(c->q[qin], slot0 + (size_t)(end)*qbytes, qbytes,
                                     cudaMemcpyDeviceToDevice, s));
        slot0 = nullptr;
        c->rec_ok = false;
      }
    }
    m = end + 1;
    chunk = 8;
  }
  if (o.time_terms && tt) {
    // a chunk's time includes its launches after the stop (they return at
    // once) and the gaps between launches: per computed term it is an upper
    // bound of the term kernel's own time
    for (size_t j = 0; j < chunks.size(); ++j) {
      const int first = chunks[j].first, last = chunks[j].second;
      if (first > *degree) break;  // every launch returned at once
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[2 * j], c->ev[2 * j + 1]) == cudaSuccess) {
        tt->ms += ms;
        tt->terms += std::min(last, *degree) - first + 1;
        tt->launches += last - first + 1;
      }
    }
  }
  c->last_degree = *degree;
  if (!lag && *degree % 2 == 0) {  // q_M: the tape slot, or the ping-pong buffer of m's parity
    const void* qM = slot0 ? (const void*)(slot0 + (size_t)*degree * qbytes) : c->q[*degree & 1];
    if (fix) *fix = PFixHost{qM, *degree};
    else launch_pfix(c, qM, *degree, s);
  }
  if (slot0) c->tape_used += ((size_t)*degree + 1) * qbytes;
  return EREM_OK;
}

StopParams stop_params(const erem_ctx* c, const Opts& o, double scale, int m_max, bool replay) {
  StopParams sp{};
  sp.delta = scale;
  sp.ncells = (double)c->N;
  sp.pow10 = std::pow(10.0, o.p_order);
  sp.tol_a = o.tol_a;
  sp.tol_r = o.tol_r;
  sp.window = o.avg_window;
  sp.m_max = m_max;
  sp.replay = replay ? 1 : 0;
  return sp;
}

// out = base + dt phi_1(dt J) src (T^n + the EREM increment when base = T^n),
// with substep doubling (§4.2) or the replayed schedule.
erem_status run_phi1(erem_ctx* c, const double* src, const double* base, double* out,
                     const Opts& o, erem_stats* st, cudaStream_t s,
                     const double* fused_T = nullptr) {
  const bool replay = !o.replay.empty();
  int mcap = o.m_max;
  if (replay)
    for (size_t k = 1; k < o.replay.size(); ++k) mcap = std::max(mcap, o.replay[k]);
  EREM_TRY(ensure_leja(c, mcap));
  int n_attempts = replay ? 1 : o.max_doublings + 1;
  // the first attempt: one substep, or the last step's count (at most 2^max_doublings)
  int a0 = 0;
  if (!replay && c->substep_start == EREM_SUBSTEPS_FROM_LAST)
    while (a0 < o.max_doublings && (1 << a0) < c->last_S) ++a0;
  bool nonfinite_attempt = false;  // the last failed attempt had a non-finite estimate
  int degrees[64];
  TermTiming tt;
  PFixHost fix;  // the last product of the substep just interpolated, if P lacks it
  if (o.time_terms) EREM_TRY(ensure_events(c, mcap + 1));
  for (int a = a0; a < n_attempts; ++a) {
    const int S = replay ? o.replay[0] : (1 << a);
    const double delta = c->dt / S;
    if (c->rec_try) {  // a new attempt tapes from the start of the record
      c->tape_used = c->rec.begin;
      c->rec.q_off.clear();
      c->rec.w_off.clear();
      c->rec_ok = true;
    }
    // a short table first; the full one when a substep needs more terms.  A
    // table not cached yet starts at kDdShort terms, computed here, while
    // host threads compute the full one (m_max terms) for the chunk loop to
    // take when the substep runs past the short one
    int M_avail = replay ? mcap : std::min(mcap, std::max(kDdShort, 2 * c->last_degree + 8));
    bool short_first = false;
    if (!replay && M_avail > kDdShort) {
      const DDEntry& e = dd_entry(c, S, 1);
      if (!(e.M >= M_avail && e.c == c->cfoc / S && e.gamma == c->gam / S)) {
        speculate_dd(c, S, mcap);
        M_avail = kDdShort;
        short_first = true;
      }
    }
    EREM_TRY(prepare_dd(c, S, M_avail, s, 1, !short_first));
    // the last step needed more substeps: the next level's table is computed
    // on the host while this level's terms run
    if (!replay && a + 1 < n_attempts && c->last_S > S) speculate_dd(c, 2 * S, mcap);
    bool ok = true;
    for (int k = 0; k < S; ++k) {
      const double* u = src;
      if (k > 0) {
        launch_japply_add(c, c->w, src, c->u, s);
        u = c->u;
      }
      const int forced = replay ? o.replay[1 + k] : 0;
      const StopParams sp = stop_params(c, o, delta, replay ? forced : o.m_max, replay);
      int degree = 0;
      bool failed = false, nonfinite = false;
      EREM_TRY(leja_interp(c, u, (fused_T && a == a0 && k == 0) ? fused_T : nullptr, S, 1, &M_avail,
                           mcap, sp, forced, o, &tt, &degree, &failed, &nonfinite, s, &fix));
      if (failed) {
        nonfinite_attempt = nonfinite;
        ok = false;
        break;
      }
      degrees[k] = degree;
      if (st) st->err_est = c->ctrl_h->err;
      if (k + 1 < S) {
        launch_axpy(c, c->w, c->P, delta, k == 0 ? 1 : 0, s, &fix);
        if (c->rec_ok) {  // the start of substep k+1 for the adjoint
          const size_t wb = (size_t)c->Np * sizeof(double);
          if (c->tape_used + wb <= c->tape_cap) {
            EREM_CUDA(c, cudaMemcpyAsync(c->tape + c->tape_used, c->w, wb, cudaMemcpyDeviceToDevice, s));
            c->rec.w_off.push_back(c->tape_used);
            c->tape_used += wb;
          } else {
            c->rec_ok = false;
          }
        }
      }
    }
    if (!ok) continue;
    c->last_S = S;
    if (c->rec_try) {
      if (c->rec_ok) {
        c->rec.sched.assign(1, S);
        for (int k = 0; k < S; ++k) c->rec.sched.push_back(degrees[k]);
        c->tape_recs.push_back(c->rec);
      } else {
        // a step that does not fit ends the tape: records are matched to
        // steps by order, so a gap would pair a later step with a wrong one
        c->tape_recs.clear();
        c->tape_used = 0;
        c->tape_on = false;
        c->rec_count0 = 0;
      }
    }
    // fused start: T^n is the caller's array itself, updated in place; a host
    // T (c->zc_out) is written once from T^n in Tn, where the fused kernel read it
    if (c->zc_out)
      launch_finish(c, c->zc_out, c->Tn, S > 1 ? c->w : nullptr, c->P, delta, s, 0, &fix);
    else
      launch_finish(c, out, fused_T ? nullptr : base, S > 1 ? c->w : nullptr, c->P, delta, s,
                    fused_T ? 1 : 0, &fix);
    EREM_TRY(check_launch(c, "finish"));
    if (st) {
      st->substeps = S;
      st->degree_total = 0;
      for (int k = 0; k < 64; ++k) st->degrees[k] = k < S ? degrees[k] : 0;
      for (int k = 0; k < S; ++k) st->degree_total += degrees[k];
      st->t_terms_ms = tt.ms;
      st->n_terms_timed = tt.terms;
      st->n_launches_timed = tt.launches;
    }
    return EREM_OK;
  }
  if (nonfinite_attempt)
    return fail(c, EREM_ENONFINITE, "non-finite Leja error estimate at every substep level");
  return fail(c, EREM_ENOTCONV,
              "Leja interpolation did not meet the stopping test within m_max terms after " +
                  std::to_string(o.max_doublings) + " substep doublings");
}

// out = T^n + dt phi_1(dt J) vrhs + dt^2 phi_2(dt J) fin_w (eq. nEERMg) with
// substep doubling; m2_forced is the replayed phi_2 degree (with o.replay).
erem_status run_forced(erem_ctx* c, double* out, const Opts& o, int m2_forced, erem_stats* st,
                       cudaStream_t s) {
  const bool replay = !o.replay.empty();
  int mcap = o.m_max;
  if (replay) {
    for (size_t k = 1; k < o.replay.size(); ++k) mcap = std::max(mcap, o.replay[k]);
    mcap = std::max(mcap, m2_forced);
  }
  EREM_TRY(ensure_leja(c, mcap));
  const int n_attempts = replay ? 1 : o.max_doublings + 1;
  bool nonfinite_attempt = false;
  int degrees[64];
  TermTiming tt;
  if (o.time_terms) EREM_TRY(ensure_events(c, mcap + 1));
  for (int a = 0; a < n_attempts; ++a) {
    const int S = replay ? o.replay[0] : (1 << a);
    const double delta = c->dt / S;
    int M1 = replay ? mcap : std::min(mcap, std::max(48, 2 * c->last_degree + 8));
    int M2 = M1;
    // phi_2 part, the same for every piece: fin_p2 = delta^2 phi_2(delta J) w
    EREM_TRY(prepare_dd(c, S, M2, s, 2));
    int deg2 = 0;
    bool failed = false, nonfinite = false;
    {
      const StopParams sp = stop_params(c, o, delta * delta, replay ? m2_forced : o.m_max, replay);
      EREM_TRY(leja_interp(c, c->fin_w, nullptr, S, 2, &M2, mcap, sp, replay ? m2_forced : 0, o,
                           &tt, &deg2, &failed, &nonfinite, s));
    }
    if (failed) {
      nonfinite_attempt = nonfinite;
      continue;
    }
    launch_lincomb(c, c->fin_p2, 0.0, c->P, delta * delta, c->P, s);
    EREM_TRY(prepare_dd(c, S, M1, s, 1));
    bool ok = true;
    for (int k = 0; k < S; ++k) {
      const double* u = c->vrhs;
      if (k > 0) {  // J y_k + G + k delta w
        launch_japply_add(c, c->w, c->vrhs, c->u, s);
        launch_lincomb(c, c->u, 1.0, c->u, k * delta, c->fin_w, s);
        u = c->u;
      }
      const int forced = replay ? o.replay[1 + k] : 0;
      const StopParams sp = stop_params(c, o, delta, replay ? forced : o.m_max, replay);
      int degree = 0;
      EREM_TRY(leja_interp(c, u, nullptr, S, 1, &M1, mcap, sp, forced, o, &tt, &degree, &failed,
                           &nonfinite, s));
      if (failed) {
        nonfinite_attempt = nonfinite;
        ok = false;
        break;
      }
      degrees[k] = degree;
      if (st) st->err_est = c->ctrl_h->err;
      if (k + 1 < S) {  // y_{k+1} = y_k + delta P + the phi_2 increment
        launch_axpy(c, c->w, c->P, delta, k == 0 ? 1 : 0, s);
        launch_lincomb(c, c->w, 1.0, c->w, 1.0, c->fin_p2, s);
      }
    }
    if (!ok) continue;
    // the last piece's phi_2 increment, then out = T^n + y + delta P
    if (S == 1) launch_lincomb(c, c->w, 0.0, c->fin_p2, 1.0, c->fin_p2, s);
    else launch_lincomb(c, c->w, 1.0, c->w, 1.0, c->fin_p2, s);
    launch_finish(c, out, c->Tn, c->w, c->P, delta, s, 0);
    EREM_TRY(check_launch(c, "forced finish"));
    if (st) {
      st->substeps = S;
      st->degree_total = deg2;
      for (int k = 0; k < 64; ++k) st->degrees[k] = k < S ? degrees[k] : 0;
      for (int k = 0; k < S; ++k) st->degree_total += degrees[k];
      st->degree_phi2 = deg2;
      st->t_terms_ms = tt.ms;
      st->n_terms_timed = tt.terms;
      st->n_launches_timed = tt.launches;
    }
    return EREM_OK;
  }
  if (nonfinite_attempt)
    return fail(c, EREM_ENONFINITE, "non-finite Leja error estimate at every substep level");
  return fail(c, EREM_ENOTCONV,
              "Leja interpolation did not meet the stopping test within m_max terms after " +
                  std::to_string(o.max_doublings) + " substep doublings");
}

// Assemble face fluxes (if fields changed or the fluid laws depend on T),
// the cell form of J, G(T^n) and ||T^n||_inf; read alpha, beta back.
erem_status assemble(erem_ctx* c, bool faces, bool rhs, cudaStream_t s) {
  if (faces) launch_faces(c, s);
  launch_cellJ(c, s);
  if (rhs) launch_rhs(c, c->Tn, c->vrhs, 1, s);
  EREM_TRY(check_launch(c, "assembly"));
  EREM_TRY(read_ctrl(c, s));
  EREM_TRY(check_flags(c));
  // FP32-bulk: where every row of J off the inflow plane sums to zero (a
  // uniform temperature is transported nowhere; the discrete flux is
  // divergence-free to far below FP32 rounding), the Leja copy keeps the
  // couplings only and the term kernel forms sum_j J_ij (q_j - q_i) + r_i q_i
  // with r_i stored for the x = 0 cells (EREM_LEJA_DIAG=1 keeps the diagonal)
  {
    const char* e = std::getenv("EREM_LEJA_DIAG");
    const bool keep_diag = e && std::atoi(e) != 0;
    c->jl_nodiag = c->jl_r0 && !keep_diag && c->ctrl_h->rowsum <= kRowSumNoDiag;
  }
  set_interval(c);
  if (!std::isfinite(c->alpha) || !std::isfinite(c->beta))
    return fail(c, EREM_ENONFINITE, "non-finite spectral interval");
  focal_map(c);
  return EREM_OK;
}

erem_status clear_flags(erem_ctx* c, cudaStream_t s) {
  EREM_CUDA(c, cudaMemsetAsync(&c->ctrl->flags, 0, sizeof(int), s));
  return EREM_OK;
}

erem_status load_fields(erem_ctx* c, const double* p, const double* lnk, const double* phi,
                        const double* lam, cudaStream_t s) {
  double *dp, *dk, *dphi, *dl;
  EREM_TRY(resolve(c, 1, p, true, s, &dp));
  EREM_TRY(resolve(c, 2, lnk, true, s, &dk));
  EREM_TRY(resolve(c, 3, phi, true, s, &dphi));
  EREM_TRY(resolve(c, 4, lam, true, s, &dl));
  launch_pack(c, dp, c->p, s);
  launch_pack(c, dk, c->lnk, s);
  launch_pack(c, dphi, c->phi, s);
  launch_pack(c, dl, c->lam, s);
  return check_launch(c, "pack fields");
}

// The Leja copy of J scaled by dt / gamma of the current interval; cached
// divided differences and the adjoint's transposed copy are stale after it.
erem_status rescale_jl(erem_ctx* c, cudaStream_t s) {
  c->jlT_valid = false;
  c->jl_sc = c->dt / c->gam;
  launch_scale_jl(c, c->jl_sc, s);
  EREM_TRY(check_launch(c, "scale"));
  c->jl_valid = true;
  c->dd_cache.clear();
  c->dd_tag_S = -1;
  return EREM_OK;
}

// Shared front half of erem_step / rosm_step: T^n into the context, fields,
// assembly when needed, G(T^n) into vrhs.  *Tdev receives T's device view.
erem_status prepare_step(erem_ctx* c, double* T, const double* p, const double* lnk,
                         const double* phi, const double* lam, double dt, bool need_interval,
                         cudaStream_t s, double** Tdev, bool fused = false) {
  if (!T) return fail(c, EREM_EINVAL, "T is NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, EREM_EINVAL, "dt must be finite and > 0");
  const int nnull = (p == nullptr) + (lnk == nullptr) + (phi == nullptr) + (lam == nullptr);
  if (nnull != 0 && nnull != 4)
    return fail(c, EREM_EINVAL, "pass all of p, lnk, phi, lambda or none of them");
  const bool fields = nnull == 0;
  if (!fields && !c->have_state)
    return fail(c, EREM_EINVAL, "no stored fields: pass p, lnk, phi, lambda (or call erem_set_state)");
  EREM_TRY(clear_flags(c, s));
  EREM_TRY(resolve(c, 0, T, true, s, Tdev));
  const bool tdep = c->phys.fluid_model != 0;
  // the fused first kernel of run_phi1 computes G(T) and T^n itself
  const bool rhs_here = !(fused && !tdep);
  const bool assemble_now = fields || tdep || !c->have_state;
  if (rhs_here || assemble_now) launch_pack(c, *Tdev, c->Tn, s);
  if (fields) EREM_TRY(load_fields(c, p, lnk, phi, lam, s));
  const double old_dt = c->dt;
  c->dt = dt;
  if (assemble_now) {
    EREM_TRY(assemble(c, fields || tdep, rhs_here, s));
    c->jl_valid = false;
    c->have_state = true;
  } else {
    if (rhs_here) launch_rhs(c, c->Tn, c->vrhs, 1, s);
    EREM_TRY(check_launch(c, "rhs"));
    if (dt != old_dt) {
      set_interval(c);
      focal_map(c);
      c->jl_valid = false;
    }
  }
  if (need_interval && !c->jl_valid) EREM_TRY(rescale_jl(c, s));
  return EREM_OK;
}

// A host output is copied back and complete on return; a device output is
// complete in stream order (its last kernel may still be running).
erem_status finish_staged(erem_ctx* c, double* host_T, const double* dev_T, cudaStream_t s) {
  if (dev_T != host_T) {
    EREM_CUDA(c, cudaMemcpyAsync(host_T, dev_T, (size_t)c->N * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
    EREM_CUDA(c, cudaStreamSynchronize(s));
  }
  return EREM_OK;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

void fill_interval(const erem_ctx* c, erem_stats* st) {
  if (!st) return;
  st->alpha = c->alpha;
  st->beta = c->beta;
}

// BiCGSTAB solve of (sigma I - J) x = b (b padded); x in kv[0].
// Levels of the stage multigrid: the fine level, then halve every dimension
// > 1 until at most kMgCoarsest cells remain (at least one coarse level).
erem_status ensure_smg(erem_ctx* c) {
  if (!c->smg.empty()) return EREM_OK;
  int nx = c->nx, ny = c->ny, nz = c->nz;
  const int nk = c->dim == 3 ? 6 : 4;
  auto add = [&](int ax, int ay, int az, size_t n) -> erem_status {
    SmgLevel m;
    m.nx = ax;
    m.ny = ay;
    m.nz = az;
    c->smg.push_back(m);
    SmgLevel& L = c->smg.back();
    for (float** a : {&L.D, &L.Dinv, &L.rhs, &L.x[0], &L.x[1], &L.x[2]}) EREM_TRY(dalloc_t(c, a, n));
    for (int q = 0; q < nk; ++q) EREM_TRY(dalloc_t(c, &L.c[q], n));
    return EREM_OK;
  };
  EREM_TRY(add(nx, ny, nz, (size_t)c->Np));
  while (c->smg.size() < 2 || (long long)nx * ny * nz > kMgCoarsest) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = c->dim == 3 ? (nz + 1) / 2 : 1;
    if (c->smg.size() >= 2 && cx == nx && cy == ny && cz == nz) break;
    nx = cx;
    ny = cy;
    nz = cz;
    EREM_TRY(add(nx, ny, nz, (size_t)nx * ny * nz));
  }
  return EREM_OK;
}

// Two multigrid-preconditioned BiCGSTAB iterations as one graph (their
// arguments are fixed for the context and sigma); false when capture is not
// available.
bool ensure_bicg_graph(erem_ctx* c, double sigma) {
  if (c->bicg_exec && c->bicg_sigma == sigma) return true;
  if (c->bicg_exec) cudaGraphExecDestroy(c->bicg_exec);
  if (c->bicg_graph) cudaGraphDestroy(c->bicg_graph);
  c->bicg_exec = nullptr;
  c->bicg_graph = nullptr;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    return false;
  }
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const long long before = c->launches;
  launch_bicg_iter_mg(c, sigma, c->cap_stream);
  launch_bicg_iter_mg(c, sigma, c->cap_stream);
  c->bicg_kernels = (int)(c->launches - before);
  c->launches = before;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(c->cap_stream, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return false;
  }
  if (cudaGraphInstantiate(&c->bicg_exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    c->bicg_exec = nullptr;
    return false;
  }
  c->bicg_graph = g;
  c->bicg_sigma = sigma;
  return true;
}

erem_status bicg_solve(erem_ctx* c, const double* b, double sigma, double tol, int maxit,
                       cudaStream_t s, int* iters, double* resid) {
  const bool mg = c->stage_precond == 1;
  if (mg) {
    EREM_TRY(ensure_smg(c));
    launch_smg_setup(c, sigma, s);
  }
  launch_bicg_init(c, b, sigma, tol, s);
  const bool graph = mg && ensure_bicg_graph(c, sigma);
  int it = 0;
  while (true) {
    EREM_TRY(read_ctrl(c, s));
    if (c->ctrl_h->lin_done || it >= maxit) break;
    const int n = std::min(mg ? 2 : 8, maxit - it);
    if (graph && n == 2) {
      EREM_CUDA(c, cudaGraphLaunch(c->bicg_exec, s));
      c->launches += c->bicg_kernels;
    } else {
      for (int k = 0; k < n; ++k) {
        if (mg) launch_bicg_iter_mg(c, sigma, s);
        else launch_bicg_iter(c, sigma, s);
      }
    }
    EREM_TRY(check_launch(c, "bicgstab"));
    it += n;
  }
  const Ctrl& h = *c->ctrl_h;
  *iters = h.lin_it;
  *resid = h.lin[K_BB] > 0 ? std::sqrt(h.lin[K_RR] / h.lin[K_BB]) : 0.0;
  if (h.lin_break && !(h.lin[K_RR] <= h.lin[K_TOL2]))
    return fail(c, EREM_ENOTCONV, "BiCGSTAB breakdown");
  if (!h.lin_done) return fail(c, EREM_ENOTCONV, "BiCGSTAB did not converge within maxit");
  return EREM_OK;
}

// ---------------------------------------------------------------------------
// Krylov phi_1 (§4.1): the basis is built on the device (kernels.cu); the
// substep control and the small exponentials run here, one read-back of the
// Arnoldi scalars per substep.
// ---------------------------------------------------------------------------
struct KrOpts {
  double tol_a = 1e-6, tol_r = 1e-6;
  int m = 10, max_substeps = 1000;
  std::vector<double> replay;
};

erem_status parse_kr_opts(erem_ctx* c, const erem_krylov_opts* o, KrOpts* out) {
  KrOpts r;
  if (o) {
    if (o->tol_a != 0.0) r.tol_a = o->tol_a;
    if (o->tol_r != 0.0) r.tol_r = o->tol_r;
    if (o->m != 0) r.m = o->m;
    if (o->max_substeps != 0) r.max_substeps = o->max_substeps;
    if (o->replay) {
      if (o->n_replay < 1) return fail(c, EREM_EINVAL, "replay needs at least one substep length");
      for (int k = 0; k < o->n_replay; ++k)
        if (!(o->replay[k] > 0.0) || !std::isfinite(o->replay[k]))
          return fail(c, EREM_EINVAL, "replayed substep lengths must be finite and > 0");
      r.replay.assign(o->replay, o->replay + o->n_replay);
    }
  }
  if (!(r.tol_a >= 0.0) || !(r.tol_r >= 0.0) || r.tol_a + r.tol_r <= 0.0)
    return fail(c, EREM_EINVAL, "tolerances must be >= 0 with tol_a + tol_r > 0");
  if (r.m < 1 || r.m > kKrMax) return fail(c, EREM_EINVAL, "Krylov dimension m must be 1..32");
  if (r.max_substeps < 1) return fail(c, EREM_EINVAL, "max_substeps must be >= 1");
  *out = r;
  return EREM_OK;
}

erem_status ensure_kr(erem_ctx* c, int m) {
  if (!c->kr_dev) {
    EREM_TRY(dalloc(c, (void**)&c->kr_dev, sizeof(KrDev)));
    if (cudaMallocHost((void**)&c->kr_host, sizeof(KrDev)) != cudaSuccess) {
      cudaGetLastError();
      c->kr_host = nullptr;
      return fail(c, EREM_ENOMEM, "cudaMallocHost of the Krylov scalars failed");
    }
    for (int k = 0; k < 2; ++k) EREM_TRY(dalloc_t(c, &c->kr_w[k], (size_t)c->Np));
    EREM_TRY(dalloc_t(c, &c->kr_r, (size_t)c->Np));
    EREM_TRY(dalloc_t(c, &c->kr_y, (size_t)c->Np));
  }
  while (c->kr_cap < m + 1) {
    EREM_TRY(dalloc_t(c, &c->kr_V[c->kr_cap], (size_t)c->Np));
    ++c->kr_cap;
  }
  return EREM_OK;
}

// [phi_1, phi_2, phi_3](delta H) e_1 for the k x k Hessenberg H (row-major
// from KrDev): the exponential of H augmented by e_1 and a shift chain.
void kr_phis(const KrDev& K, int k, double delta, std::vector<double>* out) {
  const int n = k + 3;
  std::vector<double> A((size_t)n * n, 0.0), E((size_t)n * n);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) A[(size_t)i * n + j] = delta * K.H[i * kKrMax + j];
  A[k] = 1.0;                                   // (0, k)
  A[(size_t)k * n + k + 1] = 1.0;
  A[(size_t)(k + 1) * n + k + 2] = 1.0;
  expm_small(n, A.data(), E.data());
  out->assign((size_t)3 * k, 0.0);
  for (int q = 0; q < 3; ++q)
    for (int i = 0; i < k; ++i) (*out)[(size_t)q * k + i] = E[(size_t)i * n + k + q];
}

// phi_1(delta Hbar_{k+1}) e_1 (eq. approphi) from the exponential of the
// (k + 2) augmented matrix; k + 1 entries.
void kr_phi1_hbar(const KrDev& K, int k, double delta, std::vector<double>* out) {
  const int n = k + 2;
  std::vector<double> A((size_t)n * n, 0.0), E((size_t)n * n);
  for (int i = 0; i <= k; ++i)
    for (int j = 0; j < k; ++j) A[(size_t)i * n + j] = delta * K.H[i * kKrMax + j];
  A[k + 1] = 1.0;                               // (0, k + 1)
  expm_small(n, A.data(), E.data());
  out->assign(k + 1, 0.0);
  for (int i = 0; i <= k; ++i) (*out)[i] = E[(size_t)i * n + k + 1];
}

// c->kr_y (padded) = dt phi_1(dt J) src (padded); J, dt and ||T^n||_inf
// (in the control block) must be current.
erem_status run_krylov(erem_ctx* c, const double* src, const KrOpts& o, erem_krylov_stats* st,
                       cudaStream_t s) {
  EREM_TRY(ensure_kr(c, o.m));
  c->kr_pass = 0;  // the same sweep directions on every call
  EREM_TRY(read_ctrl(c, s));
  EREM_TRY(check_flags(c));
  const double tau = c->dt;
  const int m = (int)std::min<long long>(o.m, c->N);
  const double jnorm = std::max(std::fabs(c->alpha), std::fabs(c->beta)) / tau;
  const double btol = 1e-12 * std::max(jnorm, 1e-300);
  const double tol = (o.tol_a + o.tol_r * c->ctrl_h->yinf) * std::sqrt((double)c->N);
  const bool replay = !o.replay.empty();
  EREM_CUDA(c, cudaMemsetAsync(c->kr_y, 0, sizeof(double) * c->Np, s));
  double t = 0.0, delta = tau;
  int nsub = 0, rej_total = 0;
  std::vector<double> phis, coef;
  while (replay ? nsub < (int)o.replay.size() : t < tau * (1.0 - 1e-15)) {
    if (nsub >= o.max_substeps) return fail(c, EREM_ENOTCONV, "Krylov: substep limit reached");
    const double* r = src;
    if (nsub > 0) {
      launch_japply_add(c, c->kr_y, src, c->kr_r, s);
      r = c->kr_r;
    }
    launch_kr_norm0(c, r, btol, s);
    const double* w_in = r;
    int cur = 0;
    for (int j = 0; j < m; ++j) {
      launch_kr_matvec(c, w_in, c->kr_V[j], c->kr_w[cur], j, 0, s);
      for (int i = 1; i <= j; ++i) launch_kr_orth(c, c->kr_w[cur], c->kr_V[i - 1], c->kr_V[i], i, j, 0, s);
      launch_kr_orth(c, c->kr_w[cur], c->kr_V[j], c->kr_V[j], j + 1, j, 1, s);
      w_in = c->kr_w[cur];
      cur ^= 1;
    }
    launch_kr_matvec(c, w_in, c->kr_V[m], c->kr_w[cur], m, 1, s);  // v_{m+1}, ||J v_{m+1}||
    EREM_TRY(check_launch(c, "arnoldi"));
    EREM_CUDA(c, cudaMemcpyAsync(c->kr_host, c->kr_dev, sizeof(KrDev), cudaMemcpyDeviceToHost, s));
    EREM_CUDA(c, cudaStreamSynchronize(s));
    const KrDev& K = *c->kr_host;
    if (!(K.beta > 0.0)) {
      if (!std::isfinite(K.beta)) return fail(c, EREM_ENONFINITE, "Krylov: non-finite start vector");
      break;  // J y + v = 0: y is the exact solution from here on
    }
    const bool happy = K.breakdown >= 0;
    const int k = happy ? K.breakdown + 1 : m;
    const double hnext = K.H[k * kKrMax + (k - 1)];
    if (replay) delta = o.replay[nsub];
    else delta = std::min(delta, tau - t);
    int rej = 0;
    double err = 0.0;
    while (true) {
      if (!happy) {
        kr_phis(K, k, delta, &phis);
        const double p1 = K.beta * hnext * delta * delta * std::fabs(phis[(size_t)1 * k + k - 1]);
        const double p2 =
            K.beta * hnext * delta * delta * delta * std::fabs(phis[(size_t)2 * k + k - 1]) * K.avnorm;
        err = p1 > 10.0 * p2 ? p2 : (p1 > p2 ? p1 * p2 / (p1 - p2) : p1);
        if (!std::isfinite(err)) return fail(c, EREM_ENONFINITE, "Krylov: non-finite error estimate");
      }
      if (replay || happy || err <= 1.2 * tol * delta / tau) break;
      if (++rej > 50) return fail(c, EREM_ENOTCONV, "Krylov: rejection limit reached");
      delta = 0.9 * delta * std::pow(tol * delta / (tau * err), 1.0 / k);
    }
    kr_phi1_hbar(K, k, delta, &coef);
    KrComb cb{};
    cb.n = happy ? k : k + 1;
    for (int i = 0; i < cb.n; ++i) {
      cb.v[i] = c->kr_V[i];
      cb.coef[i] = delta * K.beta * coef[i];
      if (!std::isfinite(cb.coef[i])) return fail(c, EREM_ENONFINITE, "Krylov: non-finite coefficient");
    }
    launch_kr_combine(c, c->kr_y, cb, s);
    EREM_TRY(check_launch(c, "krylov combine"));
    if (st && nsub < 64) {
      st->dims[nsub] = k;
      st->deltas[nsub] = delta;
      st->err[nsub] = err;
    }
    rej_total += rej;
    ++nsub;
    t += delta;
    delta = (happy || err == 0.0) ? tau - t : 0.9 * delta * std::pow(tol * delta / (tau * err), 1.0 / k);
  }
  if (st) {
    st->substeps = nsub;
    st->rejections = rej_total;
  }
  return EREM_OK;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
erem_status ensure_adj(erem_ctx* c, int M, int S) {
  const size_t np = (size_t)c->Np;
  const size_t esz = c->prec == EREM_FP32_BULK ? sizeof(float) : sizeof(double);
  const int nc = c->dim == 3 ? 7 : 5;
  if (!c->jlT_all) {
    if (c->prec == EREM_FP32_BULK) choose_adj_vec(c);
    EREM_TRY(dalloc(c, &c->jlT_all, (np + 128) / 128 * 128 * nc * esz));
    for (int k = 0; k < 2; ++k) EREM_TRY(dalloc(c, &c->adj_s[k], np * esz));
    EREM_TRY(dalloc_t(c, &c->adj_mu, np));
    EREM_TRY(dalloc_t(c, &c->adj_z, np));
    EREM_TRY(dalloc_t(c, &c->adj_G, np));
    EREM_TRY(dalloc_t(c, &c->adj_lam, np));
    EREM_TRY(dalloc_t(c, &c->adj_gx, np));
    EREM_TRY(dalloc_t(c, &c->adj_gy, np));
    if (c->dim == 3) EREM_TRY(dalloc_t(c, &c->adj_gz, np));
    EREM_TRY(dalloc_t(c, &c->adj_g0, (size_t)c->ny * c->nz));
    if (c->prec == EREM_FP32_BULK) {
      EREM_TRY(dalloc_t(c, &c->adj_up, np));
      EREM_TRY(dalloc_t(c, &c->adj_icap32, np));
      EREM_TRY(dalloc_t(c, &c->adj_mu32, np));
      for (int k = 0; k < (c->dim == 3 ? 3 : 2); ++k) {
        EREM_TRY(dalloc_t(c, &c->adj_g32[k], np));
        EREM_CUDA(c, cudaMemset(c->adj_g32[k], 0, np * sizeof(float)));
      }
    }
  }
  if (M > c->adj_store_cap) {
    if (c->adj_store) cudaFree(c->adj_store);
    c->adj_store = nullptr;
    c->adj_store_cap = 0;
    EREM_TRY(dalloc(c, &c->adj_store, (size_t)M * np * esz));
    c->adj_store_cap = M;
  }
  while ((int)c->adj_w.size() < S) {
    double* w = nullptr;
    EREM_TRY(dalloc_t(c, &w, np));
    c->adj_w.push_back(w);
  }
  return EREM_OK;
}

erem_status adj_clear_faces(erem_ctx* c, cudaStream_t s) {
  const size_t np = (size_t)c->Np;
  EREM_CUDA(c, cudaMemsetAsync(c->adj_gx, 0, np * sizeof(double), s));
  EREM_CUDA(c, cudaMemsetAsync(c->adj_gy, 0, np * sizeof(double), s));
  if (c->adj_gz) EREM_CUDA(c, cudaMemsetAsync(c->adj_gz, 0, np * sizeof(double), s));
  EREM_CUDA(c, cudaMemsetAsync(c->adj_g0, 0, (size_t)c->ny * c->nz * sizeof(double), s));
  for (float* g : c->adj_g32)
    if (g) EREM_CUDA(c, cudaMemsetAsync(g, 0, np * sizeof(float), s));
  return EREM_OK;
}

erem_status adj_check(erem_ctx* c) {
  if (!c->have_state || !c->jl_valid) return fail(c, EREM_EINVAL, "adjoint before erem_set_state");
  if (c->phys.fluid_model != 0) return fail(c, EREM_EINVAL, "the adjoint needs fluid_model = 0");
  return EREM_OK;
}

}  // namespace

extern "C" {

void erem_default_leja_opts(erem_leja_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol_a = 1e-6;
  o->tol_r = 1e-6;
  o->p_order = 2;
  o->m_max = 150;
  o->max_doublings = 6;
  o->avg_window = 5;
}

erem_status erem_create(const erem_grid* grid, const erem_physics* phys, erem_precision prec,
                        erem_ctx** out) {
  if (!out) return EREM_EINVAL;
  *out = nullptr;
  if (!grid || !phys) return EREM_EINVAL;
  const erem_grid g = *grid;
  if ((g.dim != 2 && g.dim != 3) || g.nx < 1 || g.ny < 1 || g.nz < 1 || (g.dim == 2 && g.nz != 1))
    return EREM_EINVAL;
  if (!(g.lx > 0) || !(g.ly > 0) || (g.dim == 3 && !(g.lz > 0))) return EREM_EINVAL;
  if (prec != EREM_FP64 && prec != EREM_FP32_BULK) return EREM_EINVAL;
  if (!(phys->rhoc_f >= 0) || !(phys->rhoc_s >= 0) || !std::isfinite(phys->head_left) ||
      !std::isfinite(phys->head_right) || !std::isfinite(phys->T_inflow) ||
      (phys->fluid_model != 0 && phys->fluid_model != 1))
    return EREM_EINVAL;
  const long long px = ((long long)g.nx + 3) / 4 * 4;
  const long long Np = px * g.ny * g.nz;
  if (Np >= (1LL << 31) - 1024) return EREM_EINVAL;
  erem_ctx* c = new erem_ctx();
  c->grid = g;
  c->phys = *phys;
  c->prec = prec;
  c->dim = g.dim;
  c->nx = g.nx;
  c->ny = g.ny;
  c->nz = g.nz;
  c->px = (int)px;
  c->N = (long long)g.nx * g.ny * g.nz;
  c->Np = Np;
  c->hx = g.lx / g.nx;
  c->hy = g.ly / g.ny;
  c->hz = g.dim == 3 ? g.lz / g.nz : 1.0;
  c->vol = c->hx * c->hy * c->hz;
  c->ax = c->hy * c->hz;
  c->ay = c->hx * c->hz;
  c->az = c->hx * c->hy;
  auto bail = [&](erem_status st) {
    erem_destroy(c);
    return st;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(EREM_ECUDA);
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return bail(EREM_ECUDA);
  c->red_blocks = c->sm_count * 8;
  int term_waves = 1;  // the one-term grid is one resident wave
  if (const char* e = std::getenv("EREM_TERM_WAVES")) {  // tuning override
    const int w = std::atoi(e);
    if (w >= 1) term_waves = w;
  }
  c->term_grid = std::min(c->red_blocks, term_waves * c->sm_count * leja_term_blocks_per_sm(c));
  if (const char* e = std::getenv("EREM_TERM_PDL")) c->pdl = std::atoi(e) != 0;  // tuning override
  c->term_lag = Np <= kLagCells;
  if (const char* e = std::getenv("EREM_TERM_LAG")) c->term_lag = std::atoi(e) != 0;  // override
  const size_t np = (size_t)Np, nf = (size_t)g.ny * g.nz;
  const size_t esz = prec == EREM_FP32_BULK ? sizeof(float) : sizeof(double);
  erem_status st = EREM_OK;
  auto A = [&](double** p, size_t n) {
    if (st == EREM_OK) st = dalloc_t(c, p, n);
  };
  A(&c->lnk, np); A(&c->phi, np); A(&c->lam, np); A(&c->p, np);
  A(&c->Lx, np); A(&c->Ly, np); A(&c->Fx, np); A(&c->Fy, np); A(&c->icap, np);
  A(&c->LD0, nf); A(&c->F0, nf); A(&c->b0, nf);
  if (g.dim == 3) { A(&c->Lz, np); A(&c->Fz, np); }
  const int nc = g.dim == 3 ? 7 : 5;
  for (int k = 0; k < nc; ++k) A(&c->jc[k], np);
  if (st == EREM_OK) st = dalloc(c, &c->jl_all, (np + 128) / 128 * 128 * nc * esz);
  if (st == EREM_OK && prec == EREM_FP32_BULK) st = dalloc(c, (void**)&c->jrow, np * sizeof(float2));
  if (st == EREM_OK && prec == EREM_FP32_BULK)
    st = dalloc(c, (void**)&c->jl_r0, nf * sizeof(float));
  A(&c->Tn, np); A(&c->vrhs, np); A(&c->vin, np); A(&c->w, np); A(&c->u, np); A(&c->P, np);
  for (int k = 0; k < 2; ++k)
    if (st == EREM_OK) st = dalloc(c, &c->q[k], np * esz);
  A(&c->red_part, (size_t)c->red_blocks * kRedSlots);
  A(&c->dd_dev, (size_t)kMaxTerms + 2);
  if (st == EREM_OK) st = dalloc(c, (void**)&c->red_cnt, sizeof(unsigned) * 4);
  if (st == EREM_OK) st = dalloc(c, (void**)&c->ctrl, sizeof(Ctrl));
  if (st != EREM_OK) return bail(st);
  if (cudaMallocHost((void**)&c->ctrl_h, sizeof(Ctrl)) != cudaSuccess ||
      cudaMallocHost((void**)&c->dd_h, sizeof(double) * (kMaxTerms + 2)) != cudaSuccess)
    return bail(EREM_ENOMEM);
  std::memset(c->ctrl_h, 0, sizeof(Ctrl));
  if (ensure_leja(c, 160) != EREM_OK) return bail(EREM_ECUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(EREM_ECUDA);
  *out = c;
  return EREM_OK;
}

erem_status erem_destroy(erem_ctx* c) {
  if (!c) return EREM_OK;
  double* dp[] = {c->lnk, c->phi, c->lam, c->p, c->Lx, c->Ly, c->Lz, c->Fx, c->Fy, c->Fz,
                  c->icap, c->LD0, c->F0, c->b0, c->Tn, c->vrhs, c->vin, c->w, c->u, c->P,
                  c->red_part, c->xi_dev, c->dd_dev};
  for (double* p : dp)
    if (p) cudaFree(p);
  for (int k = 0; k < 7; ++k)
    if (c->jc[k]) cudaFree(c->jc[k]);
  if (c->jl_all) cudaFree(c->jl_all);
  if (c->jrow) cudaFree(c->jrow);
  if (c->jl_r0) cudaFree(c->jl_r0);
  for (int k = 0; k < 2; ++k)
    if (c->q[k]) cudaFree(c->q[k]);
  for (double* p : c->kv)
    if (p) cudaFree(p);
  for (double* p : c->stage)
    if (p) cudaFree(p);
  for (double* p : c->kr_V)
    if (p) cudaFree(p);
  for (double* p : c->kr_w)
    if (p) cudaFree(p);
  if (c->kr_r) cudaFree(c->kr_r);
  if (c->kr_y) cudaFree(c->kr_y);
  if (c->kr_dev) cudaFree(c->kr_dev);
  void* adj[] = {c->jlT_all, c->adj_store, c->adj_s[0], c->adj_s[1], c->adj_mu, c->adj_z, c->adj_G,
                 c->adj_lam, c->adj_gx, c->adj_gy, c->adj_gz, c->adj_g0};
  for (void* p : adj)
    if (p) cudaFree(p);
  for (double* p : c->adj_w)
    if (p) cudaFree(p);
  if (c->tape) cudaFree(c->tape);
  for (double* p : {c->fin_b, c->fin_w, c->fin_p2, c->ada_save})
    if (p) cudaFree(p);
  void* adj32[] = {c->adj_up, c->adj_icap32, c->adj_mu32, c->adj_g32[0], c->adj_g32[1],
                   c->adj_g32[2]};
  for (void* p : adj32)
    if (p) cudaFree(p);
  for (float* p : c->pc)
    if (p) cudaFree(p);
  if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
  if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->pc_diag) cudaFree(c->pc_diag);
  for (SmgLevel& m : c->smg) {
    for (float* p : {m.D, m.Dinv, m.rhs, m.x[0], m.x[1], m.x[2]})
      if (p) cudaFree(p);
    for (float* p : m.c)
      if (p) cudaFree(p);
  }
  for (MgLevel& m : c->mg)
    for (float* p : {m.diag, m.dinv, m.Ux, m.Uy, m.Uz, m.rhs, m.x[0], m.x[1], m.x[2], m.x[3], m.inv})
      if (p) cudaFree(p);
  if (c->kr_host) cudaFreeHost(c->kr_host);
  if (c->red_cnt) cudaFree(c->red_cnt);
  if (c->ctrl) cudaFree(c->ctrl);
  if (c->ctrl_h) cudaFreeHost(c->ctrl_h);
  if (c->dd_h) cudaFreeHost(c->dd_h);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  delete c;
  return EREM_OK;
}

erem_status erem_set_physics(erem_ctx* c, const erem_physics* phys) {
  if (!c) return EREM_EINVAL;
  if (!phys || !(phys->rhoc_f >= 0) || !(phys->rhoc_s >= 0) ||
      (phys->fluid_model != 0 && phys->fluid_model != 1))
    return fail(c, EREM_EINVAL, "bad physics");
  c->phys = *phys;
  c->have_state = false;  // the stored J no longer matches
  return EREM_OK;
}

int erem_leja_coefficients(const erem_ctx* c) {
  if (!c || !c->have_state) return 0;
  return (c->dim == 3 ? 7 : 5) - (c->jl_nodiag ? 1 : 0);
}

const char* erem_last_error(const erem_ctx* c) { return c ? c->err.c_str() : kNullCtxMsg; }

erem_status pressure_solve(erem_ctx* c, const double* lnk, const double* T, double* p, double tol,
                           int maxit, erem_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  if (!lnk || !p) return fail(c, EREM_EINVAL, "lnk and p must not be NULL");
  if (!(tol > 0.0) || maxit < 0) return fail(c, EREM_EINVAL, "tol must be > 0 and maxit >= 0");
  EREM_TRY(ensure_krylov(c));
  EREM_TRY(clear_flags(c, s));
  double *dk, *dT = nullptr, *dp;
  EREM_TRY(resolve(c, 5, lnk, true, s, &dk));
  if (T) EREM_TRY(resolve(c, 6, T, true, s, &dT));
  EREM_TRY(resolve(c, 7, p, true, s, &dp));
  launch_pres_faces(c, dk, dT, s);
  launch_pack(c, dp, c->kv[0], s);
  EREM_TRY(run_pressure_cg(c, tol, maxit, s));
  const Ctrl h = *c->ctrl_h;
  const double resid = h.lin[K_BB] > 0 ? std::sqrt(h.lin[K_RR] / h.lin[K_BB]) : 0.0;
  launch_finish(c, dp, c->kv[0], nullptr, c->kv[0], 0.0, s);
  launch_pres_post(c, dk, dT, s);
  EREM_TRY(check_launch(c, "pressure post"));
  EREM_TRY(finish_staged(c, p, dp, s));
  EREM_TRY(read_ctrl(c, s));
  if (st) {
    st->lin_iters = h.lin_it;
    st->lin_resid = resid;
    st->flux_in = c->ctrl_h->flux_in;
    st->vmax = c->ctrl_h->vmax;
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
    st->terms_lagged = c->last_lag ? 1 : 0;
  }
  if (h.lin_break && !(h.lin[K_RR] <= h.lin[K_TOL2]))
    return fail(c, EREM_ENOTCONV, "CG breakdown (matrix not positive definite?)");
  if (!h.lin_done) return fail(c, EREM_ENOTCONV, "CG did not converge within maxit");
  return EREM_OK;
}

erem_status erem_set_state(erem_ctx* c, const double* T, const double* p, const double* lnk,
                           const double* phi, const double* lam, double dt, void* stream) {
  if (!c) return EREM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!T || !p || !lnk || !phi || !lam) return fail(c, EREM_EINVAL, "NULL field");
  double* Td;
  c->have_state = false;
  c->last_S = 1;  // a new run starts from one substep
  EREM_TRY(prepare_step(c, const_cast<double*>(T), p, lnk, phi, lam, dt, true, s, &Td));
  EREM_CUDA(c, cudaStreamSynchronize(s));
  return EREM_OK;
}

erem_status phi1_apply(erem_ctx* c, const double* v, double* out, const erem_leja_opts* opts,
                       erem_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->have_state || !c->jl_valid) return fail(c, EREM_EINVAL, "phi1_apply before erem_set_state");
  if (!v || !out) return fail(c, EREM_EINVAL, "NULL vector");
  Opts o;
  EREM_TRY(parse_opts(c, opts, &o));
  EREM_TRY(clear_flags(c, s));
  double *dv, *dout;
  EREM_TRY(resolve(c, 5, v, true, s, &dv));
  launch_pack(c, dv, c->vin, s);
  EREM_TRY(resolve(c, 6, out, false, s, &dout));
  EREM_TRY(run_phi1(c, c->vin, nullptr, dout, o, st, s));
  EREM_TRY(finish_staged(c, out, dout, s));
  fill_interval(c, st);
  if (st) {
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
    st->terms_lagged = c->last_lag ? 1 : 0;
  }
  return EREM_OK;
}

erem_status erem_step(erem_ctx* c, double* T, const double* p, const double* lnk,
                      const double* phi, const double* lam, double dt, const erem_leja_opts* opts,
                      erem_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  Opts o;
  EREM_TRY(parse_opts(c, opts, &o));
  double* Td = nullptr;
  const bool fused = c->phys.fluid_model == 0;
  // adjoint tape: record this step (erem_adjoint_tape); a failed step leaves
  // the tape as it was
  struct RecScope {
    erem_ctx* c;
    ~RecScope() {
      if (c->rec_try && c->tape_on && c->tape_recs.size() == c->rec_count0)
        c->tape_used = c->rec.begin;
      c->rec_try = false;
      c->rec_ok = false;
    }
  } rec_scope{c};
  c->rec_try = c->tape_on && c->phys.fluid_model == 0;
  c->rec = erem_ctx::TapeRec{};
  c->rec.begin = c->tape_used;
  c->rec_count0 = c->tape_recs.size();
  // a page-locked host T (unpadded rows) is read once by a streaming kernel
  // into Tn and written once by the last kernel (one pass each way over the
  // link) instead of being staged by copies
  double* Tz = (fused && c->host_access == 1 && c->px == c->nx && T && !is_device_ptr(T))
                   ? host_mapped(T) : nullptr;
  struct ZcScope {
    erem_ctx* c;
    ~ZcScope() {
      c->zc_active = false;
      c->zc_out = nullptr;
    }
  } zc_scope{c};
  if (Tz) {
    c->zc_active = true;
    EREM_TRY(prepare_step(c, Tz, p, lnk, phi, lam, dt, true, s, &Td, fused));
    launch_pack(c, Tz, c->Tn, s);
    c->zc_out = Tz;
    EREM_TRY(run_phi1(c, c->vrhs, c->Tn, c->Tn, o, st, s, c->Tn));
    EREM_CUDA(c, cudaStreamSynchronize(s));
  } else {
    EREM_TRY(prepare_step(c, T, p, lnk, phi, lam, dt, true, s, &Td, fused));
    EREM_TRY(run_phi1(c, c->vrhs, c->Tn, Td, o, st, s, fused ? Td : nullptr));
    EREM_TRY(finish_staged(c, T, Td, s));
  }
  fill_interval(c, st);
  if (st) {
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
    st->terms_lagged = c->last_lag ? 1 : 0;
  }
  return EREM_OK;
}

erem_status erem_step_forced(erem_ctx* c, double* T, double dt, double T_in, double T_in_rate,
                             const double* p, const double* lnk, const double* phi,
                             const double* lam, const erem_leja_opts* opts, erem_stats* st,
                             void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  if (c->phys.fluid_model != 0)
    return fail(c, EREM_EINVAL, "erem_step_forced needs fluid_model 0 (G affine in T_in)");
  if (!std::isfinite(T_in) || !std::isfinite(T_in_rate))
    return fail(c, EREM_EINVAL, "T_in and T_in_rate must be finite");
  // replay [s, m_1..m_s, m_phi2]: the phi_1 part is parsed as for erem_step
  erem_leja_opts o1{};
  const erem_leja_opts* op = opts;
  int m2 = 0;
  if (opts && opts->replay) {
    const int S = opts->n_replay >= 1 ? opts->replay[0] : 0;
    if (S < 1 || S > 64 || opts->n_replay != S + 2)
      return fail(c, EREM_EINVAL, "replay must be [s, m_1..m_s, m_phi2] with n_replay = s + 2");
    m2 = opts->replay[S + 1];
    if (m2 < 1 || m2 > kMaxTerms) return fail(c, EREM_EINVAL, "replay degree out of range");
    o1 = *opts;
    o1.n_replay = S + 1;
    op = &o1;
  }
  Opts o;
  EREM_TRY(parse_opts(c, op, &o));
  if (!c->fin_b) {
    EREM_TRY(dalloc_t(c, &c->fin_b, (size_t)c->Np));
    EREM_TRY(dalloc_t(c, &c->fin_w, (size_t)c->Np));
    EREM_TRY(dalloc_t(c, &c->fin_p2, (size_t)c->Np));
  }
  double* Td = nullptr;
  EREM_TRY(prepare_step(c, T, p, lnk, phi, lam, dt, true, s, &Td, false));
  launch_inflow_forced(c, T_in, T_in_rate, c->fin_b, c->fin_w, s);
  launch_japply_add(c, c->Tn, c->fin_b, c->vrhs, s);  // G(T^n, t_n) = J T^n + b(T_in)
  EREM_TRY(check_launch(c, "forced right-hand side"));
  EREM_TRY(run_forced(c, Td, o, m2, st, s));
  EREM_TRY(finish_staged(c, T, Td, s));
  fill_interval(c, st);
  if (st) {
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
    st->terms_lagged = c->last_lag ? 1 : 0;
  }
  return EREM_OK;
}

erem_status rosm_step(erem_ctx* c, double* T, const double* p, const double* lnk,
                      const double* phi, const double* lam, double dt, erem_rosm_scheme scheme,
                      double lin_tol, int maxit, erem_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  if (scheme != EREM_ROSM1 && scheme != EREM_ROSM_HALF && scheme != EREM_ROS2 &&
      scheme != EREM_ROS3P)
    return fail(c, EREM_EINVAL, "unknown Rosenbrock scheme");
  if (!(lin_tol > 0.0) || maxit < 1) return fail(c, EREM_EINVAL, "lin_tol > 0 and maxit >= 1");
  EREM_TRY(ensure_krylov(c));
  double* Td = nullptr;
  EREM_TRY(prepare_step(c, T, p, lnk, phi, lam, dt, false, s, &Td));
  int it_total = 0, it = 0;
  double res = 0.0, r = 0.0;
  bool embedded = false;
  if (scheme == EREM_ROS2) {
    // ROS2(1), Table ros2: gamma = 1 + 1/sqrt(2), a21 = 1/gamma, c21 = 2/gamma,
    // b = (3/(2 gamma), 1/(2 gamma)); stage matrix I/(dt gamma) - J.
    const double gam = 1.0 + 1.0 / std::sqrt(2.0);
    const double a21 = 1.0 / gam, c21 = 2.0 / gam, b1 = 3.0 / (2.0 * gam), b2 = 1.0 / (2.0 * gam);
    const double sigma = 1.0 / (dt * gam);
    double* k1 = c->kv[10];
    double* Y = c->kv[11];
    EREM_TRY(bicg_solve(c, c->vrhs, sigma, lin_tol, maxit, s, &it, &r));
    it_total += it;
    res = std::max(res, r);
    launch_lincomb(c, k1, 1.0, c->kv[0], 0.0, c->kv[0], s);
    launch_lincomb(c, Y, 1.0, c->Tn, a21, k1, s);
    launch_rhs(c, Y, c->vin, 0, s);
    launch_lincomb(c, c->vin, 1.0, c->vin, -c21 / dt, k1, s);
    EREM_TRY(check_launch(c, "ros2 stage"));
    EREM_TRY(bicg_solve(c, c->vin, sigma, lin_tol, maxit, s, &it, &r));
    it_total += it;
    res = std::max(res, r);
    // T^{n+1} = T^n + b1 k1 + b2 k2; embedded y_hat = T^n + k1 / gamma
    launch_lincomb(c, c->u, b1, k1, b2, c->kv[0], s);
    launch_finish(c, Td, c->Tn, nullptr, c->u, 1.0, s);
    launch_lincomb(c, c->vin, b1 - 1.0 / gam, k1, b2, c->kv[0], s);
    launch_sumsq(c, c->vin, s);
    embedded = true;
  } else if (scheme == EREM_ROS3P) {
    // ROS3p, Table ros3: gamma = (3 + sqrt 3)/6, a21 = a31 = 1/gamma, a32 = 0,
    // c21 = 1/gamma^2, c31 = 2 sqrt 3, c32 = sqrt 3, b = (2, 1/sqrt 3,
    // 1 - 1/sqrt 3); embedded weights as printed
    const double r3 = std::sqrt(3.0);
    const double gam = (3.0 + r3) / 6.0;
    const double a21 = 1.0 / gam, a31 = 1.0 / gam, c21 = 1.0 / (gam * gam), c31 = 2.0 * r3,
                 c32 = r3;
    const double b[3] = {2.0, 1.0 / r3, 1.0 - 1.0 / r3};
    const double bh[3] = {2.113248654051871, 1.0, 0.4226497308103742};
    const double sigma = 1.0 / (dt * gam);
    double* k1 = c->kv[10];
    double* k2 = c->w;
    double* Y = c->kv[11];
    EREM_TRY(bicg_solve(c, c->vrhs, sigma, lin_tol, maxit, s, &it, &r));
    it_total += it;
    res = std::max(res, r);
    launch_lincomb(c, k1, 1.0, c->kv[0], 0.0, c->kv[0], s);
    launch_lincomb(c, Y, 1.0, c->Tn, a21, k1, s);
    launch_rhs(c, Y, c->vin, 0, s);
    launch_lincomb(c, c->vin, 1.0, c->vin, -c21 / dt, k1, s);
    EREM_TRY(check_launch(c, "ros3p stage 2"));
    EREM_TRY(bicg_solve(c, c->vin, sigma, lin_tol, maxit, s, &it, &r));
    it_total += it;
    res = std::max(res, r);
    launch_lincomb(c, k2, 1.0, c->kv[0], 0.0, c->kv[0], s);
    launch_lincomb(c, Y, 1.0, c->Tn, a31, k1, s);  // a32 = 0
    launch_rhs(c, Y, c->vin, 0, s);
    launch_lincomb(c, c->vin, 1.0, c->vin, -c31 / dt, k1, s);
    launch_lincomb(c, c->vin, 1.0, c->vin, -c32 / dt, k2, s);
    EREM_TRY(check_launch(c, "ros3p stage 3"));
    EREM_TRY(bicg_solve(c, c->vin, sigma, lin_tol, maxit, s, &it, &r));
    it_total += it;
    res = std::max(res, r);
    // T^{n+1} = T^n + sum b_i k_i (k3 in kv[0]); y - y_hat = sum (b_i - bh_i) k_i
    launch_lincomb(c, c->u, b[0], k1, b[1], k2, s);
    launch_lincomb(c, c->u, 1.0, c->u, b[2], c->kv[0], s);
    launch_finish(c, Td, c->Tn, nullptr, c->u, 1.0, s);
    launch_lincomb(c, c->vin, b[0] - bh[0], k1, b[1] - bh[1], k2, s);
    launch_lincomb(c, c->vin, 1.0, c->vin, b[2] - bh[2], c->kv[0], s);
    launch_sumsq(c, c->vin, s);
    embedded = true;
  } else {
    // ROSM(gamma), eq. ROS: (I/(dt gamma) - J) k = G, T^{n+1} = T^n + k / gamma
    const double gam = scheme == EREM_ROSM1 ? 1.0 : 0.5;
    EREM_TRY(bicg_solve(c, c->vrhs, 1.0 / (dt * gam), lin_tol, maxit, s, &it, &r));
    it_total += it;
    res = r;
    launch_finish(c, Td, c->Tn, nullptr, c->kv[0], 1.0 / gam, s);
  }
  EREM_TRY(check_launch(c, "rosm finish"));
  EREM_TRY(read_ctrl(c, s));
  EREM_TRY(check_flags(c));
  EREM_TRY(finish_staged(c, T, Td, s));
  if (st) {
    fill_interval(c, st);
    st->lin_iters = it_total;
    st->lin_resid = res;
    st->substeps = 0;
    st->degree_total = 0;
    st->err_est = embedded ? std::sqrt(c->ctrl_h->lin[K_EMB] / (double)c->N) : 0.0;
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
    st->terms_lagged = c->last_lag ? 1 : 0;
  }
  return EREM_OK;
}

erem_status coupled_step(erem_ctx* c, double* T, double* p, double* T_p, const double* lnk,
                         const double* phi, const double* lam, double dt, erem_splitting split,
                         double ptol, int pmaxit, const erem_leja_opts* opts, erem_stats* st,
                         erem_stats* pst, void* stream) {
  if (!c) return EREM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (split != EREM_SPLIT_TROTTER && split != EREM_SPLIT_STRANG)
    return fail(c, EREM_EINVAL, "splitting must be EREM_SPLIT_TROTTER or EREM_SPLIT_STRANG");
  if (!T || !p || !lnk || !phi || !lam) return fail(c, EREM_EINVAL, "NULL array argument");
  if (T_p == T || T_p == p) return fail(c, EREM_EINVAL, "T_p must be an array of its own");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, EREM_EINVAL, "dt must be finite and > 0");
  // T_p <- the temperature the pressure was just solved at
  auto keep_Tp = [&]() -> erem_status {
    if (T_p)
      EREM_CUDA(c, cudaMemcpyAsync(T_p, T, (size_t)c->N * sizeof(double), cudaMemcpyDefault, s));
    return EREM_OK;
  };
  if (split == EREM_SPLIT_TROTTER) {
    EREM_TRY(pressure_solve(c, lnk, T, p, ptol, pmaxit, pst, stream));
    EREM_TRY(keep_Tp());
    return erem_step(c, T, p, lnk, phi, lam, dt, opts, st, stream);
  }
  // first half: the fluxes of the last solve, the viscosity at T_p
  if (T_p) {
    double* dTp;
    EREM_TRY(resolve(c, 6, T_p, true, s, &dTp));
    launch_pack(c, dTp, c->u, s);
    EREM_TRY(check_launch(c, "pack T_p"));
    c->visc_u = true;
  }
  const erem_status e1 = erem_step(c, T, p, lnk, phi, lam, 0.5 * dt, opts, st, stream);
  c->visc_u = false;
  EREM_TRY(e1);
  EREM_TRY(pressure_solve(c, lnk, T, p, ptol, pmaxit, pst, stream));
  EREM_TRY(keep_Tp());
  return erem_step(c, T, p, lnk, phi, lam, 0.5 * dt, opts ? opts + 1 : nullptr,
                   st ? st + 1 : nullptr, stream);
}

erem_status rosm_integrate(erem_ctx* c, double* T, double t_end, double dt0,
                           erem_rosm_scheme scheme, double tol_a, double tol_r, double lin_tol,
                           int maxit, int max_attempts, double* dts, erem_adapt_stats* ast,
                           void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  cudaStream_t s = (cudaStream_t)stream;
  if (scheme != EREM_ROS2 && scheme != EREM_ROS3P)
    return fail(c, EREM_EINVAL, "rosm_integrate needs EREM_ROS2 or EREM_ROS3P");
  if (!T) return fail(c, EREM_EINVAL, "T is NULL");
  if (!(t_end > 0.0) || !std::isfinite(t_end) || !(dt0 > 0.0) || !std::isfinite(dt0))
    return fail(c, EREM_EINVAL, "t_end and dt0 must be finite and > 0");
  if (!(tol_a >= 0.0) || !(tol_r >= 0.0) || tol_a + tol_r <= 0.0)
    return fail(c, EREM_EINVAL, "tolerances must be >= 0 with tol_a + tol_r > 0");
  if (max_attempts < 1) return fail(c, EREM_EINVAL, "max_attempts must be >= 1");
  if (!c->have_state) return fail(c, EREM_EINVAL, "no stored state: call erem_set_state first");
  if (!c->ada_save) EREM_TRY(dalloc_t(c, &c->ada_save, (size_t)c->N));
  const double order = scheme == EREM_ROS2 ? 2.0 : 3.0;
  const size_t bytes = (size_t)c->N * sizeof(double);
  erem_adapt_stats a{};
  a.dt_min = INFINITY;
  a.dt_max = 0.0;
  int launches = 0;
  double t = 0.0, dt = dt0, facmax = 5.0;
  while (t < t_end && a.accepted + a.rejected < max_attempts) {
    const bool last = dt >= t_end - t;
    const double h = last ? t_end - t : dt;
    EREM_CUDA(c, cudaMemcpyAsync(c->ada_save, T, bytes, cudaMemcpyDefault, s));
    erem_stats st{};
    EREM_TRY(rosm_step(c, T, nullptr, nullptr, nullptr, nullptr, h, scheme, lin_tol, maxit, &st,
                       stream));
    launches += st.launches + 1;
    a.lin_iters += st.lin_iters;
    const double sc = tol_a + tol_r * c->ctrl_h->yinf;  // ||T^n||_inf of this attempt
    const double err = st.err_est / sc;
    const double pred = err == 0.0 ? INFINITY : 0.9 * std::pow(err, -1.0 / order);
    double grow;
    if (err <= 1.0) {
      if (dts) dts[a.accepted] = h;
      ++a.accepted;
      t = last ? t_end : t + h;
      a.dt_min = std::min(a.dt_min, h);
      a.dt_max = std::max(a.dt_max, h);
      grow = std::min(facmax, std::max(0.2, pred));
      facmax = 5.0;
    } else {
      ++a.rejected;
      EREM_CUDA(c, cudaMemcpyAsync(T, c->ada_save, bytes, cudaMemcpyDefault, s));
      ++launches;
      grow = std::min(1.0, std::max(0.2, pred));
      facmax = 1.0;
    }
    dt = h * grow;
  }
  EREM_CUDA(c, cudaStreamSynchronize(s));
  a.t_reached = t;
  a.launches = launches;
  a.t_ms = now_ms() - t0;
  if (ast) *ast = a;
  if (t < t_end)
    return fail(c, EREM_ENOTCONV, "rosm_integrate: max_attempts reached before t_end");
  return EREM_OK;
}

void erem_default_krylov_opts(erem_krylov_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol_a = 1e-6;
  o->tol_r = 1e-6;
  o->m = 10;
  o->max_substeps = 1000;
}

erem_status phi1_apply_krylov(erem_ctx* c, const double* v, double* out, const erem_krylov_opts* opts,
                              erem_krylov_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->have_state) return fail(c, EREM_EINVAL, "phi1_apply_krylov before erem_set_state");
  if (!v || !out) return fail(c, EREM_EINVAL, "NULL vector");
  KrOpts o;
  EREM_TRY(parse_kr_opts(c, opts, &o));
  if (st) std::memset(st, 0, sizeof(*st));
  EREM_TRY(clear_flags(c, s));
  double *dv, *dout;
  EREM_TRY(resolve(c, 5, v, true, s, &dv));
  launch_pack(c, dv, c->vin, s);
  EREM_TRY(resolve(c, 6, out, false, s, &dout));
  EREM_TRY(run_krylov(c, c->vin, o, st, s));
  launch_finish(c, dout, nullptr, nullptr, c->kr_y, 1.0, s);
  EREM_TRY(check_launch(c, "krylov finish"));
  EREM_TRY(finish_staged(c, out, dout, s));
  if (st) {
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
  }
  return EREM_OK;
}

erem_status erem_step_krylov(erem_ctx* c, double* T, const double* p, const double* lnk,
                             const double* phi, const double* lam, double dt,
                             const erem_krylov_opts* opts, erem_krylov_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  const double t0 = now_ms();
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  KrOpts o;
  EREM_TRY(parse_kr_opts(c, opts, &o));
  if (st) std::memset(st, 0, sizeof(*st));
  double* Td = nullptr;
  EREM_TRY(prepare_step(c, T, p, lnk, phi, lam, dt, false, s, &Td));
  EREM_TRY(run_krylov(c, c->vrhs, o, st, s));
  launch_finish(c, Td, c->Tn, nullptr, c->kr_y, 1.0, s);
  EREM_TRY(check_launch(c, "krylov finish"));
  EREM_TRY(finish_staged(c, T, Td, s));
  if (st) {
    st->t_ms = now_ms() - t0;
    st->launches = (int)c->launches;
  }
  return EREM_OK;
}

erem_status erem_set_leja_points(erem_ctx* c, int kind) {
  if (!c) return EREM_EINVAL;
  if (kind != EREM_LEJA_EXACT && kind != EREM_LEJA_FAST)
    return fail(c, EREM_EINVAL, "Leja point kind must be EREM_LEJA_EXACT or EREM_LEJA_FAST");
  if (kind == c->leja_kind) return EREM_OK;
  const int cap = c->xi_cap;
  c->leja_kind = kind;
  c->xi_cap = 0;            // rebuilt for the new kind
  c->dd_cache.clear();      // divided differences belong to the points
  c->dd_tag_S = -1;
  return cap > 0 ? ensure_leja(c, cap) : EREM_OK;
}

erem_status erem_set_substep_start(erem_ctx* c, int mode) {
  if (!c) return EREM_EINVAL;
  if (mode != EREM_SUBSTEPS_FROM_ONE && mode != EREM_SUBSTEPS_FROM_LAST)
    return fail(c, EREM_EINVAL, "substep start must be EREM_SUBSTEPS_FROM_ONE or EREM_SUBSTEPS_FROM_LAST");
  c->substep_start = mode;
  return EREM_OK;
}

erem_status erem_set_pressure_precond(erem_ctx* c, int degree) {
  if (!c) return EREM_EINVAL;
  if (degree < 0 || degree > kMaxPcDeg)
    return fail(c, EREM_EINVAL, "preconditioner degree must be in 0.." + std::to_string(kMaxPcDeg));
  c->pc_deg = degree;
  return EREM_OK;
}

erem_status erem_set_host_access(erem_ctx* c, int mode) {
  if (!c) return EREM_EINVAL;
  if (mode != 0 && mode != 1) return fail(c, EREM_EINVAL, "host access: 0 (staged) or 1 (in place)");
  c->host_access = mode;
  return EREM_OK;
}

erem_status erem_set_stage_precond(erem_ctx* c, int kind) {
  if (!c) return EREM_EINVAL;
  if (kind != 0 && kind != 1)
    return fail(c, EREM_EINVAL, "stage preconditioner: 0 (Jacobi) or 1 (multigrid)");
  c->stage_precond = kind;
  return EREM_OK;
}

erem_status erem_set_pressure_multigrid(erem_ctx* c, int nu, double omega) {
  if (!c) return EREM_EINVAL;
  if (nu < 1 || nu > 16 || !(omega > 0.0 && omega < 2.0))
    return fail(c, EREM_EINVAL, "multigrid: nu in 1..16 and omega in (0, 2)");
  c->mg_nu = nu;
  c->mg_omega = (float)omega;
  return EREM_OK;
}

erem_status erem_hold_interval(erem_ctx* c, int hold, double lo, double hi) {
  if (!c) return EREM_EINVAL;
  if (hold && !(std::isfinite(lo) && std::isfinite(hi) && lo <= hi))
    return fail(c, EREM_EINVAL, "held interval must be finite with lo <= hi");
  c->hold_iv = hold != 0;
  c->hold_lo = hold ? lo : 0.0;
  c->hold_hi = hold ? hi : 0.0;
  if (!c->have_state) return EREM_OK;
  // the stored state takes the new interval at once (phi1_apply uses it)
  set_interval(c);
  focal_map(c);
  EREM_TRY(rescale_jl(c, nullptr));
  EREM_CUDA(c, cudaStreamSynchronize(nullptr));
  return EREM_OK;
}

erem_status erem_adjoint_tape(erem_ctx* c, size_t bytes, int record) {
  if (!c) return EREM_EINVAL;
  c->tape_recs.clear();
  c->tape_used = 0;
  c->tape_on = false;
  if (!record) return EREM_OK;
  if (bytes > c->tape_cap) {
    if (c->tape) cudaFree(c->tape);
    c->tape = nullptr;
    c->tape_cap = 0;
    if (cudaMalloc(reinterpret_cast<void**>(&c->tape), bytes) != cudaSuccess) {
      cudaGetLastError();
      c->tape = nullptr;
      return fail(c, EREM_ENOMEM, "adjoint tape: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->tape_cap = bytes;
  }
  c->tape_on = true;
  return EREM_OK;
}

erem_status erem_adjoint_begin(erem_ctx* c, void* stream) {
  if (!c) return EREM_EINVAL;
  EREM_TRY(adj_check(c));
  EREM_TRY(ensure_adj(c, 1, 1));
  return adj_clear_faces(c, (cudaStream_t)stream);
}

erem_status erem_adjoint_step(erem_ctx* c, const double* T, double* lam, const int* sched,
                              int ns, void* stream) {
  if (!c) return EREM_EINVAL;
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  EREM_TRY(adj_check(c));
  if (!T || !lam || !sched) return fail(c, EREM_EINVAL, "NULL argument");
  const int S = ns >= 2 ? sched[0] : 0;
  if (S < 1 || S > 64 || ns != 1 + S) return fail(c, EREM_EINVAL, "schedule must be [s, m_1..m_s], 1 <= s <= 64");
  int M = 0;
  for (int k = 1; k <= S; ++k) {
    if (sched[k] < 1 || sched[k] > kMaxTerms) return fail(c, EREM_EINVAL, "schedule degree out of range");
    M = std::max(M, sched[k]);
  }
  EREM_TRY(ensure_leja(c, M));
  EREM_TRY(ensure_adj(c, M, S));
  if (!c->jlT_valid) {
    launch_adj_scale_jlT(c, c->dt / c->gam, s);
    if (c->prec == EREM_FP32_BULK) launch_adj_aux32(c, s);
    c->jlT_valid = true;
  }
  double *Td, *lamd;
  EREM_TRY(resolve(c, 6, T, true, s, &Td));
  EREM_TRY(resolve(c, 7, lam, true, s, &lamd));
  launch_pack(c, Td, c->Tn, s);
  launch_pack(c, lamd, c->adj_lam, s);
  EREM_TRY(prepare_dd(c, S, M, s));
  const std::vector<double>& d = dd_entry(c, S).d;
  const double delta = c->dt / S;
  const double cg = c->cfoc / c->gam;
  const double scale = delta * delta / (c->gam / S);
  const size_t qbytes = (size_t)c->Np * (c->prec == EREM_FP32_BULK ? sizeof(float) : sizeof(double));
  char* store = (char*)c->adj_store;
  StopParams sp{};
  sp.delta = delta;
  sp.ncells = (double)c->N;
  sp.pow10 = 1.0;
  sp.tol_a = 1.0;
  sp.tol_r = 0.0;
  sp.window = 1;
  sp.m_max = kMaxTerms;
  sp.replay = 1;
  // the last taped record, if it is this step's: its substep starts and Newton
  // vectors replace the recomputation below (the values are the same bits)
  const erem_ctx::TapeRec* rec = nullptr;
  if (!c->tape_recs.empty()) {
    const erem_ctx::TapeRec& r = c->tape_recs.back();
    if ((int)r.sched.size() == ns && std::equal(r.sched.begin(), r.sched.end(), sched)) rec = &r;
  }
  std::vector<const double*> wk(S, nullptr);  // w_k, k >= 1
  if (rec) {
    for (int k = 1; k < S; ++k) wk[k] = (const double*)(c->tape + rec->w_off[k - 1]);
  } else {
    // G = J T^n + b (the step's first kernel), then the w_k of the substeps
    launch_step_init(c, Td, sp, s);
    for (int k = 0; k + 1 < S; ++k) {
      const double* u = c->vrhs;
      if (k > 0) {
        launch_japply_add(c, c->adj_w[k], c->vrhs, c->u, s);
        u = c->u;
      }
      launch_leja_init(c, u, sp, s);
      int qin = 0;
      for (int m = 1; m <= sched[1 + k]; ++m) {
        launch_leja_term(c, m, qin, cg, s);
        qin ^= 1;
      }
      if (sched[1 + k] % 2 == 0)  // the last product, as erem_step's consumer adds it
        launch_pfix(c, c->q[sched[1 + k] & 1], sched[1 + k], s);
      // the forward's own update w += delta P (k_axpy), so that these are the
      // bits erem_step produced (and an adjoint tape recorded)
      if (k > 0)
        EREM_CUDA(c, cudaMemcpyAsync(c->adj_w[k + 1], c->adj_w[k], sizeof(double) * c->Np,
                                     cudaMemcpyDeviceToDevice, s));
      launch_axpy(c, c->adj_w[k + 1], c->P, delta, k == 0 ? 1 : 0, s);
    }
    for (int k = 1; k < S; ++k) wk[k] = c->adj_w[k];
  }
  // backwards through the substeps
  launch_lincomb(c, c->adj_mu, 1.0, c->adj_lam, 0.0, c->adj_lam, s);
  EREM_CUDA(c, cudaMemsetAsync(c->adj_G, 0, sizeof(double) * c->Np, s));
  for (int k = S - 1; k >= 0; --k) {
    const int mk = sched[1 + k];
    const char* qk = store;
    if (rec) {
      qk = c->tape + rec->q_off[k];
    } else {
      const double* u = c->vrhs;
      if (k > 0) {
        launch_japply_add(c, c->adj_w[k], c->vrhs, c->u, s);
        u = c->u;
      }
      launch_leja_init(c, u, sp, s);
      EREM_CUDA(c, cudaMemcpyAsync(store, c->q[0], qbytes, cudaMemcpyDeviceToDevice, s));
      for (int m = 1; m < mk; ++m)
        launch_leja_term_ptr(c, m, store + (size_t)(m - 1) * qbytes, store + (size_t)m * qbytes, cg, s);
    }
    launch_adj_start(c, c->adj_mu, d[mk], c->adj_s[0], s);
    int cur = 0;
    for (int j = mk - 1; j >= 0; --j) {
      launch_adj_horner(c, c->adj_s[cur], c->adj_s[cur ^ 1], c->adj_mu, qk + (size_t)j * qbytes, d[j],
                        cg + c->xi_host[j], scale, 1, s);
      cur ^= 1;
    }
    launch_adj_z(c, c->adj_s[cur], delta, c->adj_z, c->adj_G, s);
    if (k > 0) launch_adj_face_pair(c, c->adj_z, wk[k], 1.0, s);
    launch_adj_jT_apply(c, c->adj_z, c->adj_mu, c->adj_mu, s);
  }
  if (rec) {  // consumed: the tape shrinks back to the record's start
    c->tape_used = rec->begin;
    c->tape_recs.pop_back();
  }
  if (c->prec == EREM_FP32_BULK) launch_adj_flush32(c, s);
  launch_adj_face_pair(c, c->adj_G, c->Tn, 1.0, s);
  launch_adj_b_use(c, c->adj_G, s);
  launch_adj_jT_apply(c, c->adj_G, c->adj_lam, c->adj_lam, s);
  launch_unpack(c, c->adj_lam, lamd, s);
  EREM_TRY(check_launch(c, "adjoint step"));
  EREM_TRY(finish_staged(c, lam, lamd, s));
  return EREM_OK;
}

erem_status erem_adjoint_lnk(erem_ctx* c, const double* lnk, double* glnk, double tol, int maxit,
                             erem_stats* st, void* stream) {
  if (!c) return EREM_EINVAL;
  c->launches = 0;
  c->last_lag = false;
  cudaStream_t s = (cudaStream_t)stream;
  EREM_TRY(adj_check(c));
  if (!c->adj_gx) return fail(c, EREM_EINVAL, "erem_adjoint_lnk before erem_adjoint_begin");
  if (!lnk || !glnk) return fail(c, EREM_EINVAL, "NULL argument");
  if (!(tol > 0.0) || maxit < 0) return fail(c, EREM_EINVAL, "tol must be > 0 and maxit >= 0");
  EREM_TRY(ensure_krylov(c));
  double *dk, *dout;
  EREM_TRY(resolve(c, 5, lnk, true, s, &dk));
  launch_pres_faces(c, dk, nullptr, s);
  launch_adj_dLdp(c, s);
  EREM_TRY(check_launch(c, "adjoint pressure set-up"));
  EREM_TRY(run_pressure_cg(c, tol, maxit, s));
  const Ctrl h = *c->ctrl_h;
  EREM_TRY(resolve(c, 6, glnk, false, s, &dout));
  launch_adj_lnk(c, dout, s);
  EREM_TRY(check_launch(c, "adjoint lnk"));
  EREM_TRY(finish_staged(c, glnk, dout, s));
  if (st) {
    st->lin_iters = h.lin_it;
    st->lin_resid = h.lin[K_BB] > 0 ? std::sqrt(h.lin[K_RR] / h.lin[K_BB]) : 0.0;
    st->launches = (int)c->launches;
    st->terms_lagged = c->last_lag ? 1 : 0;
  }
  if (h.lin_break && !(h.lin[K_RR] <= h.lin[K_TOL2]))
    return fail(c, EREM_ENOTCONV, "adjoint pressure CG breakdown");
  if (!h.lin_done) return fail(c, EREM_ENOTCONV, "adjoint pressure CG did not converge within maxit");
  return EREM_OK;
}

}  // extern "C"
