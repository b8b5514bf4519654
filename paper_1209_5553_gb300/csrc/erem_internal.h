// Internal declarations of the EREM library: the context, the device
// control block and the kernel launchers (defined in kernels.cu, driven by
// abi.cpp).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <future>
#include <map>
#include <string>
#include <vector>

#include "../../include/erem.h"

namespace erem {

constexpr int kThreads = 256;      // threads per block of every kernel
constexpr int kMaxTerms = 4096;    // largest Leja degree a context accepts
constexpr int kMaxPcDeg = 64;      // largest degree of the pressure CG's polynomial preconditioner
constexpr int kDefaultPcDeg = 0;   // its default: multigrid (1 = plain Jacobi CG)
constexpr int kMgCoarsest = 512;   // cells of the coarsest multigrid level, at most
constexpr int kRedSlots = 4;       // reduction values per block
constexpr double kRowSumNoDiag = 0x1p-28;  // largest relative interior row sum for a diagonal-free Leja copy

// Bits of Ctrl::flags raised by the set-up kernels.
enum : int { FLAG_NONFINITE = 1, FLAG_BAD_INPUT = 2 };

// Parameters of the Leja stopping test of one substep (§4.2).
struct StopParams {
  double delta;    // substep length dt / s
  double ncells;   // N, the number of real cells
  double pow10;    // 10^p
  double tol_a, tol_r;
  int window;      // estimates averaged
  int m_max;       // degree at which the substep fails
  int replay;      // nonzero: never stop, the host sets the degree
  int pad;
};

// Krylov scalars kept on the device (indices into Ctrl::lin).
enum : int {
  K_RZ = 0, K_RR, K_BB, K_ALPHA, K_BETA, K_DAD, K_RHO, K_RHO_PREV, K_OMEGA, K_SS, K_TOL2,
  K_EMB,  // sum of squares of the embedded Rosenbrock difference
  K_NLIN = 16
};

// Device control block: written by the last block of a reducing kernel,
// read by later kernels and, in small pieces, by the host.
struct Ctrl {
  int done;        // Leja substep finished (stop, failure or non-finite)
  int degree;      // degree m at which the stopping test passed
  int fail;        // m_max reached without passing
  int nonfinite;   // non-finite estimate met
  int m_last;      // last term evaluated
  int flags;       // FLAG_* from the set-up kernels
  int lin_done;    // linear solver converged (or broke down)
  int lin_it;      // linear solver iterations
  int lin_break;   // linear solver breakdown
  int stop_m;      // lagged Leja terms: the term the test stopped at (large while running)
  int pad_ctrl;
  double err;      // mean error estimate at the last term
  double yinf;     // ||T^n||_inf of the current state
  double gmin, gmax;   // Gershgorin bounds of J (before the factor dt)
  double flux_in, vmax;
  double rowsum;   // max over cells off the x = 0 plane of |row sum of J| / sum of |off-diagonals|
  StopParams sp;
  double lin[K_NLIN];
  double e[kMaxTerms + 2];  // error estimates e_1 .. e_m of the substep
};

// ---------------------------------------------------------------------------
// Batched ensemble of independent 2D members (ensemble.cpp,
// ensemble_cluster.cu).
//
// Every member runs the same EREM step as a single context, as a state
// machine whose phases are the passes over the member's cells; one
// thread-block cluster runs a member's whole run, pass after pass, with the
// cluster barrier between passes.
// ---------------------------------------------------------------------------
enum : int {
  ENS_INIT = 0,   // G = J T^n + b, ||T^n||_inf, first substep's q_0 and P
  ENS_TERM,       // one Leja term and the stopping test
  ENS_ACCUM,      // w += delta P after a substep that is not the last
  ENS_SUBSTART,   // next substep: q_0 = G + J w, P = d_0 q_0
  ENS_FINAL,      // T^{n+1} = T^n + w + delta P
  ENS_RESTART,    // substeps doubled after a failure: q_0 = G, P = d_0 G
  ENS_DONE,       // all steps of the run taken
  ENS_FAILED      // stopped: not converged at the last level, non-finite, or out of passes
};
enum : int { ENS_OK = 0, ENS_NOTCONV = 1, ENS_NONFINITE = 2, ENS_TIMEOUT = 3 };
constexpr int kEnsMaxLevels = 7;   // substeps 1, 2, .., 64
constexpr int kEnsWin = 64;        // largest averaging window of the batched stopping test

struct EnsState {
  int phase;      // ENS_*
  int level;      // the current attempt takes 2^level substeps
  int sub;        // substep in progress
  int step;       // steps completed in this run
  int target;     // steps of this run
  int status;     // ENS_OK, ENS_NOTCONV, ENS_NONFINITE, ENS_TIMEOUT
  int terms;      // Leja terms evaluated in this run, failed attempts included
  int attempts;   // failed attempts (substep doublings) in this run
  int last_S;     // substeps of the last completed step
  int passes;     // passes of the other phases in this run
  int last_deg[64];  // degrees of the last completed step
  int cur_deg[64];   // degrees of the step in progress
};

struct EnsMember {
  int nx, ny, px, Np;   // 2D geometry, padded pitch
  const double* jc[5];  // FP64 cell form of J: D W E S N (padded)
  const double* b0;     // constant part of G at the x = 0 cells (ny)
  const void* jl;       // Leja copy of J (context precision, interleaved)
  const float* r0;      // diagonal-free FP32 copy: the x = 0 row sums (else nullptr)
  double *T, *G, *w, *P;
  void* q[2];
  const double* dd;     // kEnsMaxLevels tables of mmax + 1 divided differences
  StopParams sp;        // tolerances, window, m_max (delta unused)
  double dt, cg;        // step, c / gamma
};

// Arguments of one run of the batched kernel.
struct EnsRun {
  const EnsMember* mem;   // [n]
  EnsState* st;           // [n]: level and target in, statistics out
  const int* order;       // [n]: members in the order the clusters take them
  unsigned* next;         // queue position (0 at launch)
  const double* xi;       // Leja points, mmax + 1
  int n;
  int nlev;               // substep levels allowed (max_doublings + 1)
  int mmax;               // entries per divided-difference table - 1
  int restart;            // 1: each step starts again from one substep
  long long passes_per_step;  // bound on a member's passes per step
};

// Krylov (Arnoldi) phi_1: device scalars of one basis (kernels.cu,
// abi.cpp).  H(i, j) is stored at H[i * kKrMax + j].
constexpr int kKrMax = 32;   // largest Krylov dimension
struct KrDev {
  double H[(kKrMax + 1) * kKrMax];
  double beta;      // ||r||_2 of the start vector
  double avnorm;    // ||J v_{m+1}||_2
  double btol;      // breakdown threshold on h_{j+1,j}
  int breakdown;    // first j with h_{j+1,j} <= btol, or -1
  int pad;
};

// One coarse level of the pressure multigrid: an aggregate of 2 x 2 (x 2)
// cells of the level above; A = diag - (couplings), FP32, unpadded layout.
struct MgLevel {
  int nx = 0, ny = 0, nz = 0;
  float *diag = nullptr, *dinv = nullptr, *Ux = nullptr, *Uy = nullptr, *Uz = nullptr;
  float* rhs = nullptr;
  float* x[4] = {};
  float* inv = nullptr;   // coarsest level: its operator's inverse, N x N by columns
};

// One level of the multigrid preconditioner of the Rosenbrock stage systems
// (sigma I - J, non-symmetric): A x = D x - sum_k c_k x_(neighbour k),
// k = west, east, south, north, bottom, top; FP32.  Level 0 has the padded
// layout of the context, coarse levels (aggregates of 2 x 2 (x 2) cells) an
// unpadded one.
struct SmgLevel {
  int nx = 0, ny = 0, nz = 0;
  float *D = nullptr, *Dinv = nullptr;
  float* c[6] = {};
  float* rhs = nullptr;
  float* x[3] = {};
};

constexpr int kDdShort = 48;    // divided differences of a level's first table
constexpr int kDdThreads = 8;   // host threads of a divided-difference table
constexpr long long kLagCells = 4500000;  // padded cells below which Leja terms run lagged

struct DDEntry {
  double c = 0, gamma = 0;
  int M = -1;
  std::vector<double> d;
};

}  // namespace erem

struct erem_ctx {
  erem_grid grid{};
  erem_physics phys{};
  erem_precision prec{};
  int dim = 2, nx = 1, ny = 1, nz = 1, px = 4;
  long long N = 0, Np = 0;   // real and padded cell counts
  double hx = 1, hy = 1, hz = 1, vol = 1, ax = 1, ay = 1, az = 1;
  int device = 0, sm_count = 1, red_blocks = 1;
  int term_grid = 1;      // blocks of the one-term kernel (one resident wave)
  bool pdl = true;        // Leja terms launched as programmatic dependents
  bool term_lag = false;  // small grids: each term's test taken by the next launch (k_leja_term_lag)
  mutable bool last_lag = false;  // the current call ran lagged terms
  std::string err;

  // stored fields (padded, FP64)
  double *lnk = nullptr, *phi = nullptr, *lam = nullptr, *p = nullptr;
  // face form: conduction and (rho c)_f * Darcy flux through the + faces,
  // inverse capacity, and the x = 0 faces (ny*nz entries)
  double *Lx = nullptr, *Ly = nullptr, *Lz = nullptr;
  double *Fx = nullptr, *Fy = nullptr, *Fz = nullptr;
  double *icap = nullptr, *LD0 = nullptr, *F0 = nullptr;
  double* b0 = nullptr;   // constant part of G at the x = 0 cells (ny*nz)
  // cell form of J (FP64): D, W, E, S, N, B, T
  double* jc[7] = {};
  // Leja copy of J scaled by dt / gamma, in the precision of the context,
  // interleaved per thread-vector (7 or 5 values per cell)
  void* jl_all = nullptr;
  bool jl_nodiag = false;    // FP32 3D: the Leja copy holds the couplings only (diagonal implied)
  float* jl_r0 = nullptr;    // its row sums at the x = 0 cells, one per (y, z) row
  double jl_sc = 0;          // the factor dt / gamma of jl_all
  // FP32-bulk: row sums r_i = sum_j J_ij of the cell form, as float pairs
  // (hi, lo), for the difference form of G in the step's first kernel
  float2* jrow = nullptr;
  // vectors
  double *Tn = nullptr, *vrhs = nullptr, *vin = nullptr, *w = nullptr, *u = nullptr, *P = nullptr;
  void* q[2] = {};
  // linear solvers (allocated on first use)
  double* kv[12] = {};
  // pressure CG polynomial preconditioner: degree (1 = Jacobi), FP32 arrays
  // dinv, Ux, Uy, Uz, r and three z buffers (allocated on first use)
  int pc_deg = erem::kDefaultPcDeg;
  float* pc[8] = {};
  // multigrid preconditioner (pc_deg = 0): FP32 diagonal of the fine level
  // and the coarse levels 1..L (levels[0] is the first coarse level)
  float* pc_diag = nullptr;
  std::vector<erem::MgLevel> mg;
  int mg_nu = 3;          // Chebyshev-Jacobi smoothing steps before and after
  float mg_omega = 1.8f;  // weight of the coarse correction
  // two preconditioned CG iterations (even, odd) captured as one CUDA graph,
  // replayed per chunk; rebuilt when the preconditioner settings change
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t pcg_graph = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  long long pcg_key = -1;
  int pcg_kernels = 0;    // kernels in the graph (for the launch count)
  // the same for two multigrid-preconditioned BiCGSTAB iterations of the
  // stage systems (keyed by sigma)
  cudaGraph_t bicg_graph = nullptr;
  cudaGraphExec_t bicg_exec = nullptr;
  double bicg_sigma = 0.0;
  int bicg_kernels = 0;
  // Rosenbrock stage systems: 0 = Jacobi BiCGSTAB, 1 = multigrid-preconditioned
  int stage_precond = 1;
  std::vector<erem::SmgLevel> smg;   // smg[0] = the fine level
  // staging for host pointers (allocated on first use)
  double* stage[8] = {};
  // Krylov basis and work vectors (allocated on first use)
  double* kr_V[erem::kKrMax + 1] = {};
  double* kr_w[2] = {};
  double* kr_r = nullptr;
  double* kr_y = nullptr;
  erem::KrDev* kr_dev = nullptr;
  erem::KrDev* kr_host = nullptr;   // pinned
  int kr_cap = 0;                   // basis vectors allocated
  mutable unsigned kr_pass = 0;     // Krylov passes launched (their direction alternates)
  // adjoint (allocated on first use)
  void* jlT_all = nullptr;          // Leja copy of J^T (FP32: interleaved per 32 adj_vec cells)
  int adj_vec = 2;                  // cells per thread of the FP32 Horner pass
  int adj_blocks_per_sm = 4;        // its resident blocks per SM (one wave of them)
  bool jlT_valid = false;
  void* adj_store = nullptr;        // forward Newton vectors q_0..q_{m-1} of one substep
  int adj_store_cap = 0;            // vectors adj_store holds
  // erem_step_forced: b(T_in) and D_t G as full vectors (non-zero on the x = 0
  // cells), and the phi_2 increment delta^2 phi_2(delta J) D_t G
  double *fin_b = nullptr, *fin_w = nullptr, *fin_p2 = nullptr;
  double* ada_save = nullptr;  // rosm_integrate: T before an attempt [N]
  // adjoint tape: erem_step records, while tape_on, what erem_adjoint_step
  // would otherwise recompute (the substep starts w_k and the Newton vectors
  // q_j of every substep) into one reserved device arena; records are
  // consumed last in, first out
  struct TapeRec {
    std::vector<int> sched;          // [s, m_1..m_s]
    std::vector<size_t> w_off;       // w_1..w_{s-1} (FP64, padded)
    std::vector<size_t> q_off;       // q_0 of each substep (Leja precision, padded)
    size_t begin = 0;
  };
  char* tape = nullptr;
  size_t tape_cap = 0, tape_used = 0;
  bool tape_on = false;
  std::vector<TapeRec> tape_recs;
  // the record of the step in progress (rec_ok = false: this step is not taped)
  TapeRec rec;
  bool rec_try = false;   // erem_step in progress tapes (tape_on)
  bool rec_ok = false;    // ... and its current attempt still fits
  size_t rec_count0 = 0;  // records before the step
  // erem_step with a pinned host T read and written in place by the kernels
  // (the first kernel also leaves T^n in Tn); host_access = 0 stages copies
  int host_access = 1;
  bool zc_active = false;
  // the face assembly takes the viscosity's temperature from u (padded)
  // instead of T^n: a Strang half step with the fluxes of the last solve
  bool visc_u = false;
  double* zc_out = nullptr;   // the host T the last kernel writes (device address)
  // FP32-bulk Horner pass: upwind flags, FP32 capacities, FP32 mu, FP32 face
  // sums of the current adjoint step
  unsigned char* adj_up = nullptr;
  float* adj_icap32 = nullptr;
  float* adj_mu32 = nullptr;
  float* adj_g32[3] = {};
  void* adj_s[2] = {};              // Horner values (Leja precision)
  double *adj_mu = nullptr, *adj_z = nullptr, *adj_G = nullptr, *adj_lam = nullptr;
  std::vector<double*> adj_w;       // w_k of the substeps of one step
  double *adj_gx = nullptr, *adj_gy = nullptr, *adj_gz = nullptr, *adj_g0 = nullptr;
  // reductions and control
  double* red_part = nullptr;
  unsigned* red_cnt = nullptr;
  erem::Ctrl* ctrl = nullptr;       // device
  erem::Ctrl* ctrl_h = nullptr;     // pinned host mirror
  double* xi_dev = nullptr;         // Leja points on the device
  double* dd_dev = nullptr;         // divided differences of the active substep level
  double* dd_h = nullptr;           // pinned staging of dd
  int xi_cap = 0;
  int leja_kind = 0;   // EREM_LEJA_EXACT or EREM_LEJA_FAST
  int dd_tag_S = -1, dd_tag_M = -1;
  std::vector<double> xi_host;
  std::map<int, erem::DDEntry> dd_cache;  // substep count -> table
  // phi_1 tables computed on host threads while the GPU runs terms: the
  // full table of the level being interpolated (its first terms use a short
  // one), and the next level's when the last step needed it
  struct DDSpec {
    std::future<std::vector<double>> f;
    int key = -1, kind = -1, M = -1;
    double c = 0, g = 0;
  };
  DDSpec dd_spec[2];
  int last_S = 1;   // substeps of the last erem_step
  int substep_start = 0;   // EREM_SUBSTEPS_FROM_ONE or EREM_SUBSTEPS_FROM_LAST

  // state
  bool hold_iv = false;              // interval held by erem_hold_interval
  double hold_lo = 0, hold_hi = 0;    // held bounds of J (before the factor dt)
  bool have_state = false;
  bool jl_valid = false;
  double dt = 0, alpha = 0, beta = 0;
  double cfoc = 0, gam = 0;   // c and gamma of [alpha, beta]
  int last_degree = 0;

  // kernels launched since the current ABI call began
  mutable long long launches = 0;
  // FP64 vector the last Leja start kernel made q_0 from (G or u): the first
  // term starts the running sum from d_0 times it
  mutable const double* p0 = nullptr;

  // timing
  std::vector<cudaEvent_t> ev;
  cudaEvent_t ev_call[2] = {nullptr, nullptr};
};

namespace erem {

// ---------------------------------------------------------------------------
// launchers (kernels.cu)
// ---------------------------------------------------------------------------
int grid_for(const erem_ctx* c, long long items);

void launch_pack(const erem_ctx* c, const double* src, double* dst, cudaStream_t s);
// The last product d_M q_M of a Leja sum stopped at an even degree M, which
// the term kernel leaves out of P (it adds products in pairs at odd m); the
// consumers below add it (q = null: P is complete).
struct PFixHost {
  const void* q = nullptr;  // q_M (Leja precision, padded)
  int M = 0;
};
void launch_finish(const erem_ctx* c, double* out, const double* base, const double* w,
                   const double* P, double delta, cudaStream_t s, int in_place = 0,
                   const PFixHost* fix = nullptr);
void launch_faces(const erem_ctx* c, cudaStream_t s);
void launch_cellJ(const erem_ctx* c, cudaStream_t s);
void launch_scale_jl(const erem_ctx* c, double sc, cudaStream_t s);
void launch_rhs(const erem_ctx* c, const double* T, double* G, int set_yinf, cudaStream_t s);
void launch_inflow_forced(const erem_ctx* c, double T_in, double rate, double* b, double* w,
                          cudaStream_t s);
void launch_sumsq(const erem_ctx* c, const double* x, cudaStream_t s);  // -> ctrl->lin[K_EMB]
void launch_japply_add(const erem_ctx* c, const double* x, const double* v, double* out,
                       cudaStream_t s);
void launch_leja_init(const erem_ctx* c, const double* u, const StopParams& sp, cudaStream_t s);
void launch_step_init(const erem_ctx* c, const double* T, const StopParams& sp, cudaStream_t s,
                      double* Tcopy = nullptr);
int leja_term_blocks_per_sm(const erem_ctx* c);
void launch_leja_term(const erem_ctx* c, int m, int qin, double cg, cudaStream_t s);
void launch_leja_term_ptr(const erem_ctx* c, int m, const void* qi, void* qo, double cg,
                          cudaStream_t s);
void launch_axpy(const erem_ctx* c, double* w, const double* P, double delta, int first,
                 cudaStream_t s, const PFixHost* fix = nullptr);
// P += d_M q_M (dd of the current level)
void launch_pfix(const erem_ctx* c, const void* q, int M, cudaStream_t s);
// Lagged form for small grids: launch m tests term m - 1 (block 0) while the
// other blocks compute term m and add d_{m-1} q_{m-1} to P; m = 1 starts P
// = d_0 p0.  The launch after the stopping term completes P.
void launch_leja_term_lag(const erem_ctx* c, int m, int qin, double cg, cudaStream_t s);
void launch_lincomb(const erem_ctx* c, double* out, double a, const double* x, double b,
                    const double* y, cudaStream_t s);

// pressure (CG)
void launch_pres_faces(const erem_ctx* c, const double* lnk, const double* T, cudaStream_t s);
void launch_cg_init(const erem_ctx* c, double tol, cudaStream_t s);
void launch_cg_iter(const erem_ctx* c, int k, cudaStream_t s);
// Chebyshev coefficients of the pressure CG's polynomial preconditioner:
// sweep j computes z_{j+1} = z_j + c1[j] (z_j - z_{j-1}) + c2[j] (D^-1 (r - A z_j))
// (sweep 0: z_1 = c2[0] D^-1 r)
struct PcPoly {
  int deg = 0;
  double c1[kMaxPcDeg] = {}, c2[kMaxPcDeg] = {};
};
void launch_pc_setup(const erem_ctx* c, cudaStream_t s);
// The preconditioner (Chebyshev polynomial, or the multigrid V-cycle with
// `poly` as its smoother when pc_deg = 0); returns the buffer that holds z.
const float* launch_pc_apply(const erem_ctx* c, const PcPoly& poly, cudaStream_t s);
void launch_pcg_iter(const erem_ctx* c, const PcPoly& poly, const float* z, int k, cudaStream_t s);
void launch_mg_setup(const erem_ctx* c, cudaStream_t s);
// stage multigrid: operators of every level for sigma I - J; one BiCGSTAB
// iteration with the V-cycle as right preconditioner
void launch_smg_setup(const erem_ctx* c, double sigma, cudaStream_t s);
void launch_bicg_iter_mg(const erem_ctx* c, double sigma, cudaStream_t s);
void launch_pres_post(const erem_ctx* c, const double* lnk, const double* T, cudaStream_t s);

// stage solver (BiCGSTAB) for (sigma I - J) x = b
void launch_bicg_init(const erem_ctx* c, const double* b, double sigma, double tol,
                      cudaStream_t s);
void launch_bicg_iter(const erem_ctx* c, double sigma, cudaStream_t s);

// batched ensemble (ensemble_cluster.cu): one cluster of cs CTAs per member
int ens_cta_threads();
cudaError_t ens_max_clusters(int prec, int cs, int* n);
cudaError_t launch_ens_cluster(const EnsRun& R, int prec, int cs, int clusters, cudaStream_t s);
void launch_unpack(const erem_ctx* c, const double* src, double* dst, cudaStream_t s);

// Krylov (Arnoldi, modified Gram-Schmidt) passes, FP64
void launch_kr_norm0(const erem_ctx* c, const double* r, double btol, cudaStream_t s);
void launch_kr_matvec(const erem_ctx* c, const double* w_in, double* v_out, double* w_out, int j,
                      int mode, cudaStream_t s);
void launch_kr_orth(const erem_ctx* c, double* w, const double* vprev, const double* vi, int i,
                    int j, int last, cudaStream_t s);
struct KrComb {
  const double* v[kKrMax + 1];
  double coef[kKrMax + 1];
  int n;
};
void launch_kr_combine(const erem_ctx* c, double* y, const KrComb& cb, cudaStream_t s);
// adjoint passes
void launch_adj_scale_jlT(const erem_ctx* c, double sc, cudaStream_t s);
void launch_adj_jT_apply(const erem_ctx* c, const double* x, const double* a, double* out,
                         cudaStream_t s);
void launch_adj_face_pair(const erem_ctx* c, const double* y, const double* x, double scale,
                          cudaStream_t s);
void launch_adj_start(const erem_ctx* c, const double* mu, double d, void* sbuf, cudaStream_t s);
void choose_adj_vec(erem_ctx* c);
void launch_adj_aux32(const erem_ctx* c, cudaStream_t s);
void launch_adj_flush32(const erem_ctx* c, cudaStream_t s);
void launch_adj_horner(const erem_ctx* c, const void* s_in, void* s_out, const double* mu,
                       const void* q, double dj, double shift, double scale, int faces,
                       cudaStream_t s);
void launch_adj_z(const erem_ctx* c, const void* sbuf, double delta, double* z, double* zacc,
                  cudaStream_t s);
void launch_adj_b_use(const erem_ctx* c, const double* y, cudaStream_t s);
void launch_adj_dLdp(const erem_ctx* c, cudaStream_t s);
void launch_adj_lnk(const erem_ctx* c, double* out, cudaStream_t s);

// dense exponential of a small host matrix (row-major n x n), Taylor +
// scaling and squaring (leja_host.cpp)
void expm_small(int n, const double* A, double* E);

// host scalar side (leja_host.cpp)
int divided_differences_phi(int kphi, int M, const double* xi, double c, double gamma, double* d,
                            int threads = 1);
void leja_table(int M, std::vector<double>* out);
void fast_leja_table(int M, std::vector<double>* out);
int divided_differences(int M, const double* xi, double c, double gamma, double* d);

}  // namespace erem
