// Steady pressure solve that allocates nothing.
//
// Some callers cannot call cudaMalloc (or anything that allocates) when they
// need a pressure field: code that runs under a memory budget fixed at
// start-up, inside a host callback, or in a runtime whose device allocator is
// owned by someone else.  erem_pressure_solve_static gives them the same
// Jacobi-preconditioned CG as pressure_solve, but its work vectors, reduction
// partials and control block live in one file-scope device array that is
// part of the loaded library, so the call itself allocates nothing; the
// caller still passes its own device arrays for the inputs and the output.
//
// The array holds at most kMaxCells padded cells (about 5.8 MB).  With the
// CUDA runtime's lazy module loading the array is placed on a device when
// the library's module is loaded there, which the first call on that device
// does (through cudaGetSymbolAddress); from then on it stays until the
// process exits.  All calls share it and it keeps what the last call left
// there: each call clears the parts that must start at zero, and two calls
// that overlap on the GPU (different streams or host threads) race on it.
#include <chrono>
#include <cstddef>
#include <cstring>

#include "erem_internal.h"

namespace {

constexpr long long kMaxCells = 65536;  // padded cells: round_up(nx, 4) * ny * nz
constexpr int kVecs = 11;               // x r z d0 d1 Ad Ux Uy Uz diag b
constexpr int kMaxBlocks = 1024;        // reduction partial slots
constexpr size_t kCtrlWords = (sizeof(erem::Ctrl) + 255) / 256 * 32;
constexpr size_t kWords = (size_t)kVecs * kMaxCells + (size_t)kMaxBlocks * erem::kRedSlots +
                          kCtrlWords + 32;

static __device__ __align__(256) double g_pressure_scratch[kWords];

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Device address of the scratch array on the current device.  It is looked
// up on every call (with the device current), not cached: a device reset or
// a new primary context reloads the module and places the array anew.  Once
// the module is loaded on the device the lookup allocates nothing.
erem_status scratch_base(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_pressure_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return EREM_ECUDA;
  }
  *out = (double*)p;
  return EREM_OK;
}

// A device array the kernels of the current device can read: device memory
// of this device (memory of another GPU would be an illegal address here
// without peer access), or managed memory.  Host memory is refused, pinned
// or not: staging it through device buffers would allocate.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" erem_status erem_pressure_solve_static(const erem_grid* grid, const erem_physics* phys,
                                                  const double* lnk, const double* T, double* p,
                                                  double tol, int maxit, erem_stats* stats,
                                                  void* stream) {
  using namespace erem;
  if (!grid || !phys || !lnk || !p) return EREM_EINVAL;
  const erem_grid g = *grid;
  if ((g.dim != 2 && g.dim != 3) || g.nx < 1 || g.ny < 1 || g.nz < 1 || (g.dim == 2 && g.nz != 1))
    return EREM_EINVAL;
  if (!(g.lx > 0) || !(g.ly > 0) || (g.dim == 3 && !(g.lz > 0))) return EREM_EINVAL;
  if (phys->fluid_model != 0 && phys->fluid_model != 1) return EREM_EINVAL;
  if (!(tol > 0.0) || maxit < 0) return EREM_EINVAL;
  const long long px = ((long long)g.nx + 3) / 4 * 4;
  const long long Np = px * g.ny * g.nz;
  if (Np > kMaxCells) return EREM_EINVAL;  // grid larger than the static scratch
  const double t0 = now_ms();
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EREM_ECUDA;
  if (!on_device(lnk, dev) || !on_device(p, dev) || (T && !on_device(T, dev))) return EREM_EINVAL;

  double* base = nullptr;
  if (scratch_base(&base) != EREM_OK) return EREM_ECUDA;

  // A context view over the scratch array: the existing CG launchers read
  // their geometry and work-vector pointers from it.  Nothing is allocated.
  erem_ctx v;
  v.grid = g;
  v.phys = *phys;
  v.dim = g.dim;
  v.nx = g.nx;
  v.ny = g.ny;
  v.nz = g.nz;
  v.px = (int)px;
  v.N = (long long)g.nx * g.ny * g.nz;
  v.Np = Np;
  v.hx = g.lx / g.nx;
  v.hy = g.ly / g.ny;
  v.hz = g.dim == 3 ? g.lz / g.nz : 1.0;
  v.vol = v.hx * v.hy * v.hz;
  v.ax = v.hy * v.hz;
  v.ay = v.hx * v.hz;
  v.az = v.hx * v.hy;
  v.device = dev;
  v.sm_count = sms;
  v.red_blocks = sms * 8 < kMaxBlocks ? sms * 8 : kMaxBlocks;
  for (int k = 0; k < kVecs; ++k) v.kv[k] = base + (size_t)k * kMaxCells;
  v.red_part = base + (size_t)kVecs * kMaxCells;
  v.ctrl = reinterpret_cast<Ctrl*>(v.red_part + (size_t)kMaxBlocks * kRedSlots);
  v.red_cnt = reinterpret_cast<unsigned*>(reinterpret_cast<double*>(v.ctrl) + kCtrlWords);

  cudaStream_t s = (cudaStream_t)stream;
  // what must start at zero: the arrival counter of the reductions and the
  // input flags (the CG kernels initialise every other value they read)
  if (cudaMemsetAsync(v.red_cnt, 0, sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(&v.ctrl->flags, 0, sizeof(int), s) != cudaSuccess)
    return EREM_ECUDA;
  launch_pres_faces(&v, lnk, T, s);
  launch_pack(&v, p, v.kv[0], s);
  launch_cg_init(&v, tol, s);
  Ctrl h;
  auto readback = [&]() -> bool {
    return cudaMemcpyAsync(&h, v.ctrl, offsetof(Ctrl, e), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
  };
  if (cudaGetLastError() != cudaSuccess || !readback()) return EREM_ECUDA;
  if (h.flags & FLAG_NONFINITE) return EREM_ENONFINITE;
  int k = 0;
  while (!h.lin_done && k < maxit) {
    const int n = maxit - k < 32 ? maxit - k : 32;
    for (int j = 0; j < n; ++j) launch_cg_iter(&v, k + j, s);
    k += n;
    if (cudaGetLastError() != cudaSuccess || !readback()) return EREM_ECUDA;
  }
  const Ctrl last = h;
  launch_finish(&v, p, v.kv[0], nullptr, v.kv[0], 0.0, s);
  launch_pres_post(&v, lnk, T, s);
  if (cudaGetLastError() != cudaSuccess || !readback()) return EREM_ECUDA;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->lin_iters = last.lin_it;
    stats->lin_resid = last.lin[K_BB] > 0 ? sqrt(last.lin[K_RR] / last.lin[K_BB]) : 0.0;
    stats->flux_in = h.flux_in;
    stats->vmax = h.vmax;
    stats->launches = (int)v.launches;
    stats->t_ms = now_ms() - t0;
  }
  if (last.lin_break && !(last.lin[K_RR] <= last.lin[K_TOL2])) return EREM_ENOTCONV;
  if (!last.lin_done) return EREM_ENOTCONV;
  return EREM_OK;
}
