// Device kernels of the EREM library for sm_103a (GB300).
//
// Data layout: every cell-centred device array is padded along x to a pitch
// px (a multiple of 4 cells), index ip = ix + px*(iy + ny*iz).  Pad cells
// hold 0 in every array and 0 coefficients, so the Leja sweep can load and
// store whole 128-bit vectors without a ragged-edge branch; they stay 0
// through every kernel.  Arrays that come straight from the caller (ABI
// inputs) are unpadded, index i = ix + nx*(iy + ny*iz).
//
// Reductions are deterministic: each block writes one partial per value,
// the last block to finish (atomic ticket) sums the partials in block order
// and writes the result into the control block.  Min/max reductions are
// exact in any order.
#include <algorithm>
#include <cstdint>

#include "erem_internal.h"
#include "device_common.cuh"

namespace erem {
namespace {

struct Geo {
  int nx, ny, nz, px, dim;
  int N, Np;
  int plane;  // px * ny
};

__device__ __forceinline__ void cell_of(int i, const Geo& g, int& ix, int& iy, int& iz, int& ip) {
  const int r = i / g.nx;
  ix = i - r * g.nx;
  iy = r % g.ny;
  iz = r / g.ny;
  ip = ix + g.px * r;
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// Fluid laws (fluid_model = 1): rho/rho0 = 1 - 3e-4 (T - 20),
// mu/mu0 = exp(-0.02 (T - 20)); X = rho/rho0 * T and its T-derivative.
__device__ __forceinline__ double rho_rel(double T, int fm) { return fm ? 1.0 - 3e-4 * (T - 20.0) : 1.0; }
__device__ __forceinline__ double mu_rel(double T, int fm) { return fm ? exp(-0.02 * (T - 20.0)) : 1.0; }
__device__ __forceinline__ double Xof(double T, int fm) { return rho_rel(T, fm) * T; }
__device__ __forceinline__ double dXof(double T, int fm) { return fm ? rho_rel(T, fm) - 3e-4 * T : 1.0; }

// two-point harmonic transmissibility |s| ki kj / (ki d + kj d), uniform d
__device__ __forceinline__ double harm(double area, double d, double ki, double kj) {
  const double den = ki * d + kj * d;
  return den != 0.0 ? area * ki * kj / den : 0.0;
}

struct Phys {
  double rhoc_f, rhoc_s, head_left, head_right, T_in;
  int fm;
  double hx, hy, hz, vol, ax, ay, az;
};

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------
__global__ void k_pack(const double* __restrict__ src, double* __restrict__ dst, Geo g,
                       int* flags) {
  int bad = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double v = src[i];
    bad |= !finite(v);
    dst[ip] = v;
  }
  if (bad && flags) atomicOr(flags, FLAG_NONFINITE);
}

// The last product d_M q_M of a Leja sum that stopped at an even degree M
// (the term kernel adds products in pairs at odd m; see k_leja_term): the
// consumers of P add it on the fly.  q = null: P is complete.
struct PFix {
  const void* q;      // q_M in the Leja precision, padded layout
  int q32;            // q is FP32
  const double* dd;   // divided differences of the substep level
  int M;
};
__device__ __forceinline__ double p_full(const double* __restrict__ P, const PFix& f, int ip) {
  double p = P[ip];
  if (f.q) {
    const double q = f.q32 ? f2d_fast(static_cast<const float*>(f.q)[ip])
                           : static_cast<const double*>(f.q)[ip];
    p = fma(f.dd[f.M], q, p);
  }
  return p;
}

// out[i] = (delta * P[ip] + w[ip]) + base[ip]  (base, w may be null); with
// in_place the base is out[i] itself (the caller's unpadded array).  Every
// operation is rounded on its own (no contraction into an FMA), so the
// result has the same bits whichever of base or in_place supplies T^n.
__global__ void k_finish(double* out, const double* __restrict__ base,
                         const double* __restrict__ w, const double* __restrict__ P, PFix f,
                         double delta, int in_place, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    double v = __dmul_rn(delta, p_full(P, f, ip));
    if (w) v = __dadd_rn(v, w[ip]);
    if (base) v = __dadd_rn(v, base[ip]);
    else if (in_place) v = __dadd_rn(v, out[i]);
    out[i] = v;
  }
}

// w = (first ? 0 : w) + delta * P over padded arrays
__global__ void k_axpy(double* __restrict__ w, const double* __restrict__ P, PFix f, double delta,
                       int first, int Np) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) {
    const double p = p_full(P, f, i);
    w[i] = first ? delta * p : w[i] + delta * p;
  }
}

__global__ void k_lincomb(double* __restrict__ out, double a, const double* __restrict__ x,
                          double b, const double* __restrict__ y, int Np) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT)
    out[i] = a * x[i] + b * y[i];
}

// ---------------------------------------------------------------------------
// face form of the heat operator (§3.1): conduction transmissibilities and
// (rho c)_f * Darcy fluxes through the + faces of every cell, the x = 0
// faces, and 1 / (C |Omega|).
// ---------------------------------------------------------------------------
struct FaceOut {
  double *Lx, *Ly, *Lz, *Fx, *Fy, *Fz, *icap, *LD0, *F0;
};
struct FieldIn {
  const double *lnk, *phi, *lam, *p, *T;  // padded
};

// Cell mobility, once per cell into m (padded): K rho(T)/mu(T) for the
// pressure matrix (darcy = 0), K/mu(T) for the Darcy fluxes (darcy = 1).  The
// face kernels below take their harmonic means from it instead of evaluating
// the fluid laws (two FP64 exponentials) again for every face of every cell.
__global__ void k_mobility(const double* __restrict__ lnk, const double* __restrict__ T,
                           double* __restrict__ m, Geo g, Phys ph, int darcy, int in_padded,
                           int* flags) {
  int bad = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const int j = in_padded ? ip : i;  // lnk and T in the padded or the caller's layout
    const double Ti = T ? T[j] : 20.0;
    const double mi = darcy ? exp(lnk[j]) / mu_rel(Ti, ph.fm)
                            : exp(lnk[j]) * rho_rel(Ti, ph.fm) / mu_rel(Ti, ph.fm);
    bad |= !finite(mi);
    m[ip] = mi;
  }
  if (bad && flags) atomicOr(flags, FLAG_NONFINITE);
}

__global__ void k_faces(FieldIn in, const double* __restrict__ m, FaceOut o, Geo g, Phys ph,
                        int* flags) {
  int bad = 0, inval = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double Ti = in.T[ip];
    const double mi = m[ip];  // K / mu(T), k_mobility
    const double li = in.lam[ip];
    const double pi = in.p[ip];
    const double phi = in.phi[ip];
    bad |= !finite(mi) | !finite(li) | !finite(pi) | !finite(phi) | !finite(Ti);
    inval |= (li < 0.0) | (phi < 0.0) | (phi > 1.0);
    // + x face
    if (ix < g.nx - 1) {
      const int j = ip + 1;
      const double mj = m[j];
      o.Lx[ip] = harm(ph.ax, 0.5 * ph.hx, li, in.lam[j]);
      o.Fx[ip] = ph.rhoc_f * harm(ph.ax, 0.5 * ph.hx, mi, mj) * (pi - in.p[j]);
    } else {  // x = 1: Dirichlet pressure, outflow face without conduction
      o.Lx[ip] = 0.0;
      o.Fx[ip] = ph.rhoc_f * (ph.ax * mi / (0.5 * ph.hx)) * (pi - ph.head_right);
    }
    // + y face
    if (iy < g.ny - 1) {
      const int j = ip + g.px;
      const double mj = m[j];
      o.Ly[ip] = harm(ph.ay, 0.5 * ph.hy, li, in.lam[j]);
      o.Fy[ip] = ph.rhoc_f * harm(ph.ay, 0.5 * ph.hy, mi, mj) * (pi - in.p[j]);
    } else {
      o.Ly[ip] = 0.0;
      o.Fy[ip] = 0.0;
    }
    if (g.dim == 3) {
      if (iz < g.nz - 1) {
        const int j = ip + g.plane;
        const double mj = m[j];
        o.Lz[ip] = harm(ph.az, 0.5 * ph.hz, li, in.lam[j]);
        o.Fz[ip] = ph.rhoc_f * harm(ph.az, 0.5 * ph.hz, mi, mj) * (pi - in.p[j]);
      } else {
        o.Lz[ip] = 0.0;
        o.Fz[ip] = 0.0;
      }
    }
    if (ix == 0) {  // x = 0: Dirichlet pressure and temperature
      const int r = iy + g.ny * iz;
      o.LD0[r] = ph.ax * li / (0.5 * ph.hx);
      o.F0[r] = ph.rhoc_f * (ph.ax * mi / (0.5 * ph.hx)) * (ph.head_left - pi);
    }
    const double C = phi * ph.rhoc_f + (1.0 - phi) * ph.rhoc_s;
    inval |= !(C > 0.0);
    o.icap[ip] = 1.0 / (C * ph.vol);
  }
  if (bad) atomicOr(flags, FLAG_NONFINITE);
  if (inval) atomicOr(flags, FLAG_BAD_INPUT);
}

// ---------------------------------------------------------------------------
// cell form of J = D_T G (eq. linear): per cell the diagonal and the six
// neighbour couplings, from the derivative of every face flux; plus the
// Gershgorin bounds min(J_ii - R_i), max(J_ii + R_i) (§4.2).
// ---------------------------------------------------------------------------
struct FaceIn {
  const double *Lx, *Ly, *Lz, *Fx, *Fy, *Fz, *icap, *LD0, *F0;
};
struct JOut {
  double* c[7];  // D W E S N B T
  double* b0;    // constant part of G at the x = 0 cells (linear fluid model)
};

__global__ void k_cellJ(FaceIn f, const double* __restrict__ T, JOut o, Geo g, Phys ph,
                        double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  double gmin = INFINITY, gmax = -INFINITY, rmax = 0.0;
  int bad = 0;
  const int fm = ph.fm;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double dXi = dXof(T[ip], fm);
    double D = 0.0, W = 0.0, E = 0.0, S = 0.0, Nn = 0.0, B = 0.0, Tt = 0.0;
    // + x face
    {
      const double F = f.Fx[ip];
      if (ix < g.nx - 1) {
        D -= f.Lx[ip] + (F >= 0.0 ? F * dXi : 0.0);
        E = f.Lx[ip] + (F < 0.0 ? -F * dXof(T[ip + 1], fm) : 0.0);
      } else {
        D -= F * dXi;  // outflow face carries X_i for either sign
      }
    }
    // - x face
    if (ix > 0) {
      const double F = f.Fx[ip - 1];
      D -= f.Lx[ip - 1] + (F < 0.0 ? -F * dXi : 0.0);
      W = f.Lx[ip - 1] + (F >= 0.0 ? F * dXof(T[ip - 1], fm) : 0.0);
    } else {
      const int r = iy + g.ny * iz;
      const double F = f.F0[r];
      D -= f.LD0[r] + (F > 0.0 ? 0.0 : -F * dXi);
      if (o.b0)
        o.b0[r] = f.icap[ip] * (f.LD0[r] * ph.T_in + (F > 0.0 ? F * Xof(ph.T_in, fm) : 0.0));
    }
    // +- y faces
    if (iy < g.ny - 1) {
      const double F = f.Fy[ip];
      D -= f.Ly[ip] + (F >= 0.0 ? F * dXi : 0.0);
      Nn = f.Ly[ip] + (F < 0.0 ? -F * dXof(T[ip + g.px], fm) : 0.0);
    }
    if (iy > 0) {
      const double F = f.Fy[ip - g.px];
      D -= f.Ly[ip - g.px] + (F < 0.0 ? -F * dXi : 0.0);
      S = f.Ly[ip - g.px] + (F >= 0.0 ? F * dXof(T[ip - g.px], fm) : 0.0);
    }
    if (g.dim == 3) {
      if (iz < g.nz - 1) {
        const double F = f.Fz[ip];
        D -= f.Lz[ip] + (F >= 0.0 ? F * dXi : 0.0);
        Tt = f.Lz[ip] + (F < 0.0 ? -F * dXof(T[ip + g.plane], fm) : 0.0);
      }
      if (iz > 0) {
        const double F = f.Fz[ip - g.plane];
        D -= f.Lz[ip - g.plane] + (F < 0.0 ? -F * dXi : 0.0);
        B = f.Lz[ip - g.plane] + (F >= 0.0 ? F * dXof(T[ip - g.plane], fm) : 0.0);
      }
    }
    const double ic = f.icap[ip];
    D *= ic; W *= ic; E *= ic; S *= ic; Nn *= ic; B *= ic; Tt *= ic;
    o.c[0][ip] = D; o.c[1][ip] = W; o.c[2][ip] = E; o.c[3][ip] = S; o.c[4][ip] = Nn;
    if (g.dim == 3) { o.c[5][ip] = B; o.c[6][ip] = Tt; }
    const double R = fabs(W) + fabs(E) + fabs(S) + fabs(Nn) + fabs(B) + fabs(Tt);
    bad |= !finite(D) | !finite(R);
    gmin = fmin(gmin, D - R);
    gmax = fmax(gmax, D + R);
    if (ix > 0) {  // the row sum relative to the couplings, off the Dirichlet inflow plane
      const double rs = fabs(D + W + E + S + Nn + B + Tt);
      rmax = fmax(rmax, R > 0.0 ? rs / R : (rs > 0.0 ? INFINITY : 0.0));
    }
  }
  if (bad) atomicOr(&ctrl->flags, FLAG_NONFINITE);
  const double bmin = block_reduce<1>(gmin, sh);
  const double bmax = block_reduce<2>(gmax, sh);
  const double brs = block_reduce<2>(rmax, sh);
  double vals[3] = {bmin, bmax, brs};
  if (publish_partials(part, cnt, vals, 3)) {
    const double a = gather_partials<1>(part, 0, sh);
    const double b = gather_partials<2>(part, 1, sh);
    const double r = gather_partials<2>(part, 2, sh);
    if (threadIdx.x == 0) {
      ctrl->gmin = a;
      ctrl->gmax = b;
      ctrl->rowsum = r;
      *cnt = 0;
    }
  }
}

// Leja copy of J: (Tq)(sc * jc_k) for every padded cell, in the warp-tile
// interleaved layout of LejaCoef (tile of T cells).  skip = 1: the couplings
// only (the diagonal is implied by the row sums, zero off the x = 0 plane),
// and r0[row] = (Tq)(sc * row sum) at the x = 0 cells.
template <typename Tq, int T>
__global__ void k_scale_jl(JOut jc, Tq* __restrict__ out, double sc, int Np, int nc,
                           float2* __restrict__ rsum, int skip, Tq* __restrict__ r0, int px) {
  const int nout = nc - skip;
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) {
    const size_t base = (size_t)(i / T) * nout * T + (i % T);
    for (int k = skip; k < nc; ++k) out[base + (size_t)(k - skip) * T] = (Tq)(sc * jc.c[k][i]);
    if (rsum || skip) {
      double r = 0.0;  // row sum r_i of J (FP64)
      for (int k = 0; k < nc; ++k) r += jc.c[k][i];
      if (rsum) {  // as a float pair hi + lo
        const float hi = (float)r;
        rsum[i] = make_float2(hi, (float)(r - (double)hi));
      }
      if (skip && i % px == 0) r0[i / px] = (Tq)(sc * r);
    }
  }
}

// ---------------------------------------------------------------------------
// heat right-hand side G(T) (eq. spaceheat2): conductive and upwind
// advective fluxes into each cell (§3.1) over its capacity.
// ---------------------------------------------------------------------------
__global__ void k_rhs(FaceIn f, const double* __restrict__ T, double* __restrict__ G, Geo g,
                      Phys ph, int set_yinf, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  const int fm = ph.fm;
  double tmax = 0.0;
  int bad = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double Ti = T[ip];
    const double Xi = Xof(Ti, fm);
    double in = 0.0;
    {  // + x face
      const double F = f.Fx[ip];
      if (ix < g.nx - 1) {
        const double Tj = T[ip + 1];
        in -= f.Lx[ip] * (Ti - Tj) + F * (F >= 0.0 ? Xi : Xof(Tj, fm));
      } else {
        in -= F * Xi;
      }
    }
    if (ix > 0) {  // - x face, flux in +x direction enters cell i
      const double F = f.Fx[ip - 1];
      const double Tj = T[ip - 1];
      in += f.Lx[ip - 1] * (Tj - Ti) + F * (F >= 0.0 ? Xof(Tj, fm) : Xi);
    } else {
      const int r = iy + g.ny * iz;
      const double F = f.F0[r];
      in += f.LD0[r] * (ph.T_in - Ti) + F * (F > 0.0 ? Xof(ph.T_in, fm) : Xi);
    }
    if (iy < g.ny - 1) {
      const double F = f.Fy[ip];
      const double Tj = T[ip + g.px];
      in -= f.Ly[ip] * (Ti - Tj) + F * (F >= 0.0 ? Xi : Xof(Tj, fm));
    }
    if (iy > 0) {
      const double F = f.Fy[ip - g.px];
      const double Tj = T[ip - g.px];
      in += f.Ly[ip - g.px] * (Tj - Ti) + F * (F >= 0.0 ? Xof(Tj, fm) : Xi);
    }
    if (g.dim == 3) {
      if (iz < g.nz - 1) {
        const double F = f.Fz[ip];
        const double Tj = T[ip + g.plane];
        in -= f.Lz[ip] * (Ti - Tj) + F * (F >= 0.0 ? Xi : Xof(Tj, fm));
      }
      if (iz > 0) {
        const double F = f.Fz[ip - g.plane];
        const double Tj = T[ip - g.plane];
        in += f.Lz[ip - g.plane] * (Tj - Ti) + F * (F >= 0.0 ? Xof(Tj, fm) : Xi);
      }
    }
    const double Gi = f.icap[ip] * in;
    G[ip] = Gi;
    bad |= !finite(Gi) | !finite(Ti);
    tmax = fmax(tmax, fabs(Ti));
  }
  if (bad) atomicOr(&ctrl->flags, FLAG_NONFINITE);
  if (!set_yinf) return;
  const double bmax = block_reduce<2>(tmax, sh);
  double vals[1] = {bmax};
  if (publish_partials(part, cnt, vals, 1)) {
    const double a = gather_partials<2>(part, 0, sh);
    if (threadIdx.x == 0) {
      ctrl->yinf = a;
      *cnt = 0;
    }
  }
}

// (J x)_i from the FP64 cell form, one cell
struct JIn {
  const double* c[7];
};
__device__ __forceinline__ double japply_cell(const JIn& J, const double* __restrict__ x, int ip,
                                              int ix, int iy, int iz, const Geo& g) {
  double a = J.c[0][ip] * x[ip];
  if (ix > 0) a += J.c[1][ip] * x[ip - 1];
  if (ix < g.nx - 1) a += J.c[2][ip] * x[ip + 1];
  if (iy > 0) a += J.c[3][ip] * x[ip - g.px];
  if (iy < g.ny - 1) a += J.c[4][ip] * x[ip + g.px];
  if (g.dim == 3) {
    if (iz > 0) a += J.c[5][ip] * x[ip - g.plane];
    if (iz < g.nz - 1) a += J.c[6][ip] * x[ip + g.plane];
  }
  return a;
}

// out = J x + v (the right-hand side J w_k + v of a later substep)
__global__ void k_japply_add(JIn J, const double* __restrict__ x, const double* __restrict__ v,
                             double* __restrict__ out, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    out[ip] = japply_cell(J, x, ip, ix, iy, iz, g) + v[ip];
  }
}

// Time-dependent inflow temperature, linear fluid model: the x = 0 cells'
// b(T_in) = (LD0 + F0^+) T_in / C and w = D_t G = T_in_rate (LD0 + F0^+) / C
// (Dirichlet conduction and inflowing advection of §3.1); the other cells of
// both vectors stay 0.
__global__ void k_inflow_forced(const double* __restrict__ icap, const double* __restrict__ LD0,
                                const double* __restrict__ F0, double T_in, double rate,
                                double* __restrict__ b, double* __restrict__ w, Geo g) {
  const int nf = g.ny * g.nz;
  for (int r = blockIdx.x * NT + threadIdx.x; r < nf; r += gridDim.x * NT) {
    const int ip = g.px * r;
    const double coef = icap[ip] * (LD0[r] + (F0[r] > 0.0 ? F0[r] : 0.0));
    b[ip] = coef * T_in;
    w[ip] = coef * rate;
  }
}

// First kernel of an EREM step with the linear fluid model, where G is
// affine in T: G = J T + b exactly (b non-zero only at the x = 0 cells).
// One pass reads the caller's T (unpadded, left in place for the final
// update), writes v = G(T^n) (FP64) and q_0 = v in the Leja precision,
// reduces ||T^n||_inf for the error scale, and arms the control block of the
// first substep (the first Leja term starts the running sum from v).  This
// replaces the face-form G (about 40 FP64 instructions per cell on GB300's
// slow FP64 pipe) by 7.
template <typename Tq>
__global__ void k_step_init(JIn J, const double* __restrict__ b0, const double* __restrict__ T,
                            double* __restrict__ Tcopy, double* __restrict__ G, Tq* __restrict__ q0,
                            Geo g, StopParams sp, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    arm_ctrl(ctrl, sp);
  }
  const int sx = 1, sy = g.nx, sz = g.nx * g.ny;
  double tmax = 0.0;
  int bad = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double Ti = T[i];
    double a = J.c[0][ip] * Ti;
    if (ix > 0) a = fma(J.c[1][ip], T[i - sx], a);
    if (ix < g.nx - 1) a = fma(J.c[2][ip], T[i + sx], a);
    if (iy > 0) a = fma(J.c[3][ip], T[i - sy], a);
    if (iy < g.ny - 1) a = fma(J.c[4][ip], T[i + sy], a);
    if (g.dim == 3) {
      if (iz > 0) a = fma(J.c[5][ip], T[i - sz], a);
      if (iz < g.nz - 1) a = fma(J.c[6][ip], T[i + sz], a);
    }
    if (ix == 0) a += b0[iy + g.ny * iz];
    G[ip] = a;
    q0[ip] = (Tq)a;
    if (Tcopy) Tcopy[ip] = Ti;
    bad |= !finite(a);
    tmax = fmax(tmax, fabs(Ti));
  }
  if (bad) atomicOr(&ctrl->flags, FLAG_NONFINITE);
  const double bmax = block_reduce<2>(tmax, sh);
  double vals[1] = {bmax};
  if (publish_partials(part, cnt, vals, 1)) {
    const double a = gather_partials<2>(part, 0, sh);
    if (threadIdx.x == 0) {
      ctrl->yinf = a;
      *cnt = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Newton-Leja recurrence (eq. newt)
// ---------------------------------------------------------------------------
// The same first kernel when nx is a multiple of 4 (the caller's T then has
// the padded layout): each thread owns four consecutive cells and moves them
// with 128-bit loads and stores.  ||T^n||_inf and the finiteness checks use
// integer operations on the bit patterns (for |x| the order of the bits is
// the order of the values), so the FP64 pipe only does the 8 FMAs of G.
template <typename Tq, int DIM>
__global__ void __launch_bounds__(NT)
k_step_init_vec(JIn J, const double* __restrict__ b0, const double* __restrict__ T,
                double* __restrict__ Tcopy, double* __restrict__ G, Tq* __restrict__ q0,
                Geo g, StopParams sp, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    arm_ctrl(ctrl, sp);
  }
  unsigned long long tmax = 0ULL;
  bool bad = false;
  const int nvec = g.Np / 4;
  const int vrow = g.px / 4;
  for (int t = blockIdx.x * NT + threadIdx.x; t < nvec; t += gridDim.x * NT) {
    const int row = t / vrow;
    const int ix = (t - row * vrow) * 4;
    const int iy = row % g.ny;
    const int iz = row / g.ny;
    const int i = row * g.px + ix;
    double tc[4], ts[4], tn[4], tb[4], tt[4];
    ldP<4>(tc, T + i);
    ldP<4>(ts, T + i - (iy > 0 ? g.px : 0));
    ldP<4>(tn, T + i + (iy < g.ny - 1 ? g.px : 0));
    if (DIM == 3) {
      ldP<4>(tb, T + i - (iz > 0 ? g.plane : 0));
      ldP<4>(tt, T + i + (iz < g.nz - 1 ? g.plane : 0));
    }
    const double tl = ix > 0 ? T[i - 1] : 0.0;
    const double tr = ix + 4 < g.px ? T[i + 4] : 0.0;
    constexpr int NC = DIM == 3 ? 7 : 5;
    double c[7][4];
#pragma unroll
    for (int k = 0; k < NC; ++k) ldP<4>(c[k], J.c[k] + i);
    double a[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double west = v == 0 ? tl : tc[v - 1];
      const double east = v == 3 ? tr : tc[v + 1];
      double x = c[0][v] * tc[v];
      x = fma(c[1][v], west, x);
      x = fma(c[2][v], east, x);
      x = fma(c[3][v], ts[v], x);
      x = fma(c[4][v], tn[v], x);
      if (DIM == 3) {
        x = fma(c[5][v], tb[v], x);
        x = fma(c[6][v], tt[v], x);
      }
      a[v] = x;
    }
    if (ix == 0) a[0] += b0[iy + g.ny * iz];
    Tq qv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qv[v] = (Tq)a[v];
      const unsigned long long tb_ = abs_bits(tc[v]);
      tmax = tmax > tb_ ? tmax : tb_;
      bad |= !bits_finite(tb_) | !bits_finite(abs_bits(a[v]));
    }
    stP<4>(G + i, a);
    if (Tcopy) stP<4>(Tcopy + i, tc);
    if constexpr (sizeof(Tq) == 4) {
      *reinterpret_cast<float4*>(q0 + i) = make_float4(qv[0], qv[1], qv[2], qv[3]);
    } else {
      *reinterpret_cast<double2*>(q0 + i) = make_double2(qv[0], qv[1]);
      *reinterpret_cast<double2*>(q0 + i + 2) = make_double2(qv[2], qv[3]);
    }
  }
  if (bad) atomicOr(&ctrl->flags, FLAG_NONFINITE);
  const double bmax = block_reduce<2>(__longlong_as_double((long long)tmax), sh);
  double vals[1] = {bmax};
  if (publish_partials(part, cnt, vals, 1)) {
    const double a = gather_partials<2>(part, 0, sh);
    if (threadIdx.x == 0) {
      ctrl->yinf = a;
      *cnt = 0;
    }
  }
}

// x = hi + lo with hi, lo floats, from the bit fields with integer
// instructions only (the FP64 pipe of GB300 is the scarce unit here): hi is
// x cut to its leading 24 significand bits, lo the next 23 bits, both exact,
// |x - hi - lo| <= 2^-46 |x|, for 2^-80 <= |x| < 2^128.  Below that lo is 0
// (hi still exact down to 2^-126, the smallest normal float), magnitudes
// under 2^-126 give hi = 0 (flushed, as FP32 arithmetic with flush-to-zero
// would), and magnitudes of 2^128 and more give an infinite hi (a NaN stays
// a NaN), which the caller's finiteness check reports.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned e = (h32 >> 20) & 0x7ffu;
  const unsigned sgn = h32 & 0x80000000u;
  unsigned hb;
  float l = 0.0f;
  if (e - 897u <= 1150u - 897u) {
    hb = sgn | ((e - 896u) << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    if (e >= 943u) {
      // bits 28..6 of the significand as an integer r < 2^23 (exactly,
      // through the float 2^23 + r), then r 2^(e - 1069), a product with a
      // power of 2
      const float r = __uint_as_float(0x4b000000u | ((l32 & 0x1fffffffu) >> 6)) - 8388608.0f;
      l = __uint_as_float(sgn | ((e - 942u) << 23)) * r;
    }
  } else if (e < 897u) {
    hb = sgn;
  } else {
    hb = sgn | ((e == 0x7ffu && ((h32 & 0xfffffu) | l32)) ? 0x7fc00000u : 0x7f800000u);
  }
  hi = __uint_as_float(hb);
  lo = l;
}

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// First kernel of an FP32-bulk EREM step (linear fluid model, nx a multiple
// of 4): G = J T + b on the FP32 pipe, in the form
//   G_i = sum_{j != i} J_ij (T_j - T_i) + (r_i T_i + b_i),   r_i = sum_j J_ij,
// which equals J T + b exactly.  In J T the products J_ii T_i and J_ij T_j
// nearly cancel wherever T is smooth, so G computed that way in FP32 carries
// an error of the size of T itself; here every product is of the size of
// the result.  Each T (FP64) is split into a float pair hi + lo by integer
// instructions; T_j - T_i = (hi_j - hi_i) + (lo_j - lo_i) (the hi difference
// is exact when the two are within a factor 2, i.e. wherever they nearly
// cancel); the couplings J_ij are the FP32 Leja copy tau J / gamma times
// gamma / tau; r_i T_i + b_i, which cancels at the Dirichlet inflow, is
// evaluated in float-pair arithmetic (two-product by fmaf, two-sum).  G
// keeps its float-pair value in FP64 (vrhs) and rounded to FP32 in q_0; the
// FP64 pipe carries one addition per cell.  Also: ||T^n||_inf and the
// finiteness checks on integer bit patterns, T^n copied when Tcopy is set,
// the control block armed for the first substep.
template <int DIM, bool ND = false>
__global__ void __launch_bounds__(NT)
k_step_init_df(LejaCoef<float> cf, float jinv, const float2* __restrict__ rsum,
               const double* __restrict__ b0, const double* __restrict__ T,
               double* __restrict__ Tcopy, double* __restrict__ G, float* __restrict__ q0, Geo g,
               StopParams sp, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    arm_ctrl(ctrl, sp);
  }
  unsigned long long tmax = 0ULL;
  bool bad = false;
  const int nvec = g.Np / 4;
  const int vrow = g.px / 4;
  for (int t = blockIdx.x * NT + threadIdx.x; t < nvec; t += gridDim.x * NT) {
    const int row = t / vrow;
    const int ix = (t - row * vrow) * 4;
    const int iy = row % g.ny;
    const int iz = row / g.ny;
    const int i = row * g.px + ix;
    double tc[4];
    ldP<4>(tc, T + i);
    if (Tcopy) stP<4>(Tcopy + i, tc);
    float h[4], l[4];  // the centre cells as float pairs
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const unsigned long long tb_ = abs_bits(tc[v]);
      tmax = tmax > tb_ ? tmax : tb_;
      bad |= !bits_finite(tb_);
      split_f64(tc[v], h[v], l[v]);
    }
    const size_t off = leja_off<128>(i, cf.nc);
    // sum_j J_ij (T_j - T_i) direction by direction, couplings of the scaled copy
    float S[4];
    {
      float wh, wl, eh, el, cW[4], cE[4];
      split_f64(ix > 0 ? T[i - 1] : 0.0, wh, wl);
      split_f64(ix + 4 < g.px ? T[i + 4] : 0.0, eh, el);
      ldv_stream<float, 4>(cW, cf.c[1] + off);
      ldv_stream<float, 4>(cE, cf.c[2] + off);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float xh = v == 0 ? wh : h[v - 1], xl = v == 0 ? wl : l[v - 1];
        const float yh = v == 3 ? eh : h[v + 1], yl = v == 3 ? el : l[v + 1];
        S[v] = fmaf(cE[v], (yh - h[v]) + (yl - l[v]), cW[v] * ((xh - h[v]) + (xl - l[v])));
      }
    }
    constexpr int NB = DIM == 3 ? 4 : 2;
#pragma unroll
    for (int k = 0; k < NB; ++k) {  // S, N (, B, T)
      const int step = k < 2 ? g.px : g.plane;
      const bool has = k == 0 ? iy > 0 : k == 1 ? iy < g.ny - 1 : k == 2 ? iz > 0 : iz < g.nz - 1;
      double tn[4];
      ldP<4>(tn, T + i + (has ? (k & 1 ? step : -step) : 0));
      float cN[4];
      ldv_stream<float, 4>(cN, cf.c[3 + k] + off);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float nh, nl;
        split_f64(tn[v], nh, nl);
        S[v] = fmaf(cN[v], (nh - h[v]) + (nl - l[v]), S[v]);
      }
    }
    // the row sums: every cell's, or (ND: the rows of J sum to zero off the
    // x = 0 plane) the x = 0 cell's only
    float rh[4], rl[4];
    if constexpr (ND) {
      const float2 r0 = ix == 0 ? rsum[i] : make_float2(0.f, 0.f);
      rh[0] = r0.x;
      rl[0] = r0.y;
      rh[1] = rh[2] = rh[3] = rl[1] = rl[2] = rl[3] = 0.f;
    } else {
      const float4 r01 = *reinterpret_cast<const float4*>(rsum + i);
      const float4 r23 = *reinterpret_cast<const float4*>(rsum + i + 2);
      rh[0] = r01.x; rh[1] = r01.z; rh[2] = r23.x; rh[3] = r23.z;
      rl[0] = r01.y; rl[1] = r01.w; rl[2] = r23.y; rl[3] = r23.w;
    }
    double gv[4];
    float qv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float Sv = S[v] * jinv;
      // r_i T_i (+ b_i) as a float pair (p, e)
      float p = 0.f, e = 0.f;
      if (!ND || v == 0) {
        p = rh[v] * h[v];
        e = fmaf(rh[v], h[v], -p);
        e = fmaf(rh[v], l[v], e);
        e = fmaf(rl[v], h[v], e);
      }
      float ph = p;
      if (v == 0 && ix == 0) {  // the x = 0 cell: + b_i
        float bh, bl, s2;
        split_f64(b0[iy + g.ny * iz], bh, bl);
        two_sum(p, bh, ph, s2);
        e += s2 + bl;
      }
      // G = S + (ph + e): (gr, gl) with gr the rounded value
      float gh, g2;
      two_sum(ph, Sv, gh, g2);
      const float glo = g2 + e;
      const float gr = gh + glo;
      const float gl = glo - (gr - gh);
      qv[v] = gr;
      gv[v] = f2d_fast(gr) + f2d_fast(gl);
      bad |= !isfinite(gr);
    }
    stP<4>(G + i, gv);
    *reinterpret_cast<float4*>(q0 + i) = make_float4(qv[0], qv[1], qv[2], qv[3]);
  }
  if (bad) atomicOr(&ctrl->flags, FLAG_NONFINITE);
  const double bmax = block_reduce<2>(__longlong_as_double((long long)tmax), sh);
  double vals[1] = {bmax};
  if (publish_partials(part, cnt, vals, 1)) {
    const double a = gather_partials<2>(part, 0, sh);
    if (threadIdx.x == 0) {
      ctrl->yinf = a;
      *cnt = 0;
    }
  }
}

// q_0 = u (in the Leja precision); block 0 arms the control block.  The
// first Leja term starts the running sum from d_0 u.
template <typename Tq>
__global__ void k_leja_init(const double* __restrict__ u, Tq* __restrict__ q0, int Np,
                            StopParams sp, Ctrl* ctrl) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    arm_ctrl(ctrl, sp);
  }
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) q0[i] = (Tq)u[i];
}

// One Leja term, fused: q_m = (dt J / gamma - (c/gamma + xi_{m-1})) q_{m-1}
// (the stencil apply), the running sum P, and the partial sum of q_m^2 for
// the error estimate; the last block runs the stopping test.  Each thread
// owns VEC consecutive cells along x.
//
// The running sum is updated every other term, when both vectors it needs
// are in registers (q_{m-1} is the stencil's centre, q_m its result):
//   PM = 2 (m = 1):      P = d_0 p0 + d_1 q_1   (p0: the FP64 vector q_0 was made from)
//   PM = 1 (m odd > 1):  P += d_{m-1} q_{m-1} + d_m q_m
//   PM = 0 (m even):     P untouched (no P traffic: 16 fewer bytes per cell)
// The two products enter P one after the other, in the order of eq. newt,
// so P after term m (odd) has the bits of a sum updated at every term.  A
// substep stopped at an even degree M has P short of d_M q_M: its consumer
// adds it (k_finish, k_axpy, k_pfix).
//
// In FP32-bulk the squares of a thread's values are summed in FP32 with a
// compensated (two-sum) accumulator and enter the FP64 norm once per thread,
// so the FP64 pipe only carries the running sum.
template <typename Tq, int VEC, int DIM, int PM, bool ND>
__device__ __forceinline__ void leja_term_body(const Tq* __restrict__ qi, Tq* __restrict__ qo,
                                               double* __restrict__ P, const double* __restrict__ p0,
                                               const LejaCoef<Tq>& cf, const Geo& g,
                                               const double* __restrict__ xi,
                                               const double* __restrict__ dd, double cg, int m,
                                               double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  // Launched as a programmatic dependent of the previous term: wait until
  // that grid has completed and its writes are visible (a no-op when the
  // launch was an ordinary one), then let the next term be scheduled: its
  // blocks take the SM slots this grid's blocks free while its last block
  // reduces the norm, and wait here in turn.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  if (*(volatile int*)&ctrl->done) return;
  const Tq sh_m = (Tq)(cg + xi[m - 1]);
  const double dm = dd[m];
  const double dm1 = dd[m - 1];
  double acc = 0.0;
  float s_hi = 0.f, s_lo = 0.f;  // FP32-bulk: compensated sum of squares
  const int nvec = g.Np / VEC;
  const int vrow = g.px / VEC;
  for (int t = blockIdx.x * NT + threadIdx.x; t < nvec; t += gridDim.x * NT) {
    const int row = t / vrow;
    const int ix = (t - row * vrow) * VEC;
    const int iy = row % g.ny;
    const int iz = row / g.ny;
    const int i = row * g.px + ix;
    Tq qc[VEC], qs[VEC], qn[VEC], qb[VEC], qt[VEC];
    ldv<Tq, VEC>(qc, qi + i);
    ldv<Tq, VEC>(qs, qi + i - (iy > 0 ? g.px : 0));
    ldv<Tq, VEC>(qn, qi + i + (iy < g.ny - 1 ? g.px : 0));
    if (DIM == 3) {
      ldv<Tq, VEC>(qb, qi + i - (iz > 0 ? g.plane : 0));
      ldv<Tq, VEC>(qt, qi + i + (iz < g.nz - 1 ? g.plane : 0));
    }
    const Tq ql = ix > 0 ? qi[i - 1] : Tq(0);
    const Tq qr = ix + VEC < g.px ? qi[i + VEC] : Tq(0);
    Tq cD[VEC], cW[VEC], cE[VEC], cS[VEC], cN[VEC], cB[VEC], cT[VEC];
    Tq r0 = Tq(0);  // ND: the row sum of an x = 0 cell (every other row sums to zero)
    if constexpr (ND) {
      if (ix == 0) r0 = cf.r0[row];
    } else {
      ldv_stream<Tq, VEC>(cD, cf.c[0] + leja_off<32 * VEC>(i, cf.nc));
    }
    ldv_stream<Tq, VEC>(cW, cf.c[1] + leja_off<32 * VEC>(i, cf.nc));
    ldv_stream<Tq, VEC>(cE, cf.c[2] + leja_off<32 * VEC>(i, cf.nc));
    ldv_stream<Tq, VEC>(cS, cf.c[3] + leja_off<32 * VEC>(i, cf.nc));
    ldv_stream<Tq, VEC>(cN, cf.c[4] + leja_off<32 * VEC>(i, cf.nc));
    if (DIM == 3) {
      ldv_stream<Tq, VEC>(cB, cf.c[5] + leja_off<32 * VEC>(i, cf.nc));
      ldv_stream<Tq, VEC>(cT, cf.c[6] + leja_off<32 * VEC>(i, cf.nc));
    }
    double p[VEC];
    if constexpr (PM == 1) ldP<VEC>(p, P + i);
    if constexpr (PM == 2) ldP<VEC>(p, p0 + i);
    Tq out[VEC];
    Tq sq = Tq(0);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const Tq west = k == 0 ? ql : qc[k - 1];
      const Tq east = k == VEC - 1 ? qr : qc[k + 1];
      Tq a;
      if constexpr (ND) {
        // sum_j J_ij (q_j - q_i) + (r_i - shift) q_i
        a = ((k == 0 ? r0 : Tq(0)) - sh_m) * qc[k];
        a = fma(cW[k], west - qc[k], a);
        a = fma(cE[k], east - qc[k], a);
        a = fma(cS[k], qs[k] - qc[k], a);
        a = fma(cN[k], qn[k] - qc[k], a);
        if (DIM == 3) {
          a = fma(cB[k], qb[k] - qc[k], a);
          a = fma(cT[k], qt[k] - qc[k], a);
        }
      } else {
        a = (cD[k] - sh_m) * qc[k];
        a = fma(cW[k], west, a);
        a = fma(cE[k], east, a);
        a = fma(cS[k], qs[k], a);
        a = fma(cN[k], qn[k], a);
        if (DIM == 3) {
          a = fma(cB[k], qb[k], a);
          a = fma(cT[k], qt[k], a);
        }
      }
      out[k] = a;
      if constexpr (sizeof(Tq) == 4) {
        sq = fmaf(a, a, sq);
      } else {
        acc = fma(a, a, acc);
      }
    }
    // the running sum after the stencil (the coefficients are dead by now)
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      if constexpr (PM == 1) p[k] = fma(dm, to_f64_fast(out[k]), fma(dm1, to_f64_fast(qc[k]), p[k]));
      if constexpr (PM == 2) p[k] = fma(dm, to_f64_fast(out[k]), dm1 * p[k]);
    }
    if constexpr (sizeof(Tq) == 4) {
      // two-sum of the running FP32 sum and this vector's squares
      const float s = s_hi + sq;
      const float bp = s - s_hi;
      s_lo += (s_hi - (s - bp)) + (sq - bp);
      s_hi = s;
    }
    stv<Tq, VEC>(qo + i, out);
    if constexpr (PM != 0) stP<VEC>(P + i, p);
  }
  if constexpr (sizeof(Tq) == 4) acc = (double)s_hi + (double)s_lo;
  const double bs = block_reduce<0>(acc, sh);
  double vals[1] = {bs};
  if (publish_partials(part, cnt, vals, 1)) {
    const double S = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      stop_test(ctrl, m, dm, S);
    }
  }
}

// Terms m >= 2 (PM = 0 or 1), held to four resident blocks of 256 threads
// per SM, the grid the launcher sizes.
template <typename Tq, int VEC, int DIM, int PM, bool ND = false>
__global__ void __launch_bounds__(NT, 4)
k_leja_term(const Tq* __restrict__ qi, Tq* __restrict__ qo, double* __restrict__ P,
            LejaCoef<Tq> cf, Geo g, const double* __restrict__ xi, const double* __restrict__ dd,
            double cg, int m, double* part, unsigned* cnt, Ctrl* ctrl) {
  leja_term_body<Tq, VEC, DIM, PM, ND>(qi, qo, P, nullptr, cf, g, xi, dd, cg, m, part, cnt, ctrl);
}

// Term m = 1 (PM = 2), held to four resident blocks per SM like the others.
template <typename Tq, int VEC, int DIM, bool ND = false>
__global__ void __launch_bounds__(NT, 4)
k_leja_term1(const Tq* __restrict__ qi, Tq* __restrict__ qo, double* __restrict__ P,
             const double* __restrict__ p0, LejaCoef<Tq> cf, Geo g, const double* __restrict__ xi,
             const double* __restrict__ dd, double cg, double* part, unsigned* cnt, Ctrl* ctrl) {
  leja_term_body<Tq, VEC, DIM, 2, ND>(qi, qo, P, p0, cf, g, xi, dd, cg, 1, part, cnt, ctrl);
}

// Lagged Leja term m for small grids, where the last block's gather of the
// partial sums and the stopping test would be a large part of a term.  Block
// 0 does no sweep: it sums the partials of term m - 1 in block order and takes
// its stopping test, while blocks 1.. compute q_m = ((J - c) / gamma - xi_{m-1})
// q_{m-1}, add d_{m-1} q_{m-1} to P (m = 1: P = d_0 p0) and publish their
// partials of ||q_m||^2 (slot m & 1 of each block).  P thus receives the
// products one launch after the paired form and in the same order, so both
// leave the same P for the same degree; the launch after the stopping term
// completes P and its own q is not used.  A launch returns at once when the
// test stopped at least two terms before it (ctrl->stop_m, written by block 0
// of the launch after the stopping term, never acted on by that launch).
template <typename Tq, int VEC, int DIM, bool ND>
__global__ void __launch_bounds__(NT, 4)
k_leja_term_lag(const Tq* __restrict__ qi, Tq* __restrict__ qo, double* __restrict__ P,
                const double* __restrict__ p0, LejaCoef<Tq> cf, Geo g,
                const double* __restrict__ xi, const double* __restrict__ dd, double cg, int m,
                double* part, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  if (m >= *(volatile int*)&ctrl->stop_m + 2) return;
  if (blockIdx.x == 0) {
    if (m >= 2) {  // the stopping test of term m - 1
      double v = 0.0;
      for (int b = 1 + threadIdx.x; b < (int)gridDim.x; b += NT)
        v += __ldcg(part + (size_t)b * kRedSlots + ((m - 1) & 1));
      const double S = block_reduce<0>(v, sh);
      if (threadIdx.x == 0) {
        stop_test(ctrl, m - 1, dd[m - 1], S);
        if (ctrl->done) ctrl->stop_m = m - 1;
      }
    }
    return;
  }
  const Tq sh_m = (Tq)(cg + xi[m - 1]);
  const double dprev = m >= 2 ? dd[m - 1] : 0.0;
  const double d0 = dd[0];
  float s_hi = 0.f, s_lo = 0.f;  // FP32-bulk: compensated sum of squares
  double acc = 0.0;
  const int nvec = g.Np / VEC;
  const int vrow = g.px / VEC;
  const int G = (gridDim.x - 1) * NT;
  for (int t = (blockIdx.x - 1) * NT + threadIdx.x; t < nvec; t += G) {
    const int row = t / vrow;
    const int ix = (t - row * vrow) * VEC;
    const int iy = row % g.ny;
    const int iz = row / g.ny;
    const int i = row * g.px + ix;
    Tq qc[VEC], qs[VEC], qn[VEC], qb[VEC], qt[VEC];
    ldv<Tq, VEC>(qc, qi + i);
    ldv<Tq, VEC>(qs, qi + i - (iy > 0 ? g.px : 0));
    ldv<Tq, VEC>(qn, qi + i + (iy < g.ny - 1 ? g.px : 0));
    if (DIM == 3) {
      ldv<Tq, VEC>(qb, qi + i - (iz > 0 ? g.plane : 0));
      ldv<Tq, VEC>(qt, qi + i + (iz < g.nz - 1 ? g.plane : 0));
    }
    const Tq ql = ix > 0 ? qi[i - 1] : Tq(0);
    const Tq qr = ix + VEC < g.px ? qi[i + VEC] : Tq(0);
    Tq cD[VEC], cW[VEC], cE[VEC], cS[VEC], cN[VEC], cB[VEC], cT[VEC];
    Tq r0 = Tq(0);
    if constexpr (ND) {
      if (ix == 0) r0 = cf.r0[row];
    } else {
      ldv_stream<Tq, VEC>(cD, cf.c[0] + leja_off<32 * VEC>(i, cf.nc));
    }
    ldv_stream<Tq, VEC>(cW, cf.c[1] + leja_off<32 * VEC>(i, cf.nc));
    ldv_stream<Tq, VEC>(cE, cf.c[2] + leja_off<32 * VEC>(i, cf.nc));
    ldv_stream<Tq, VEC>(cS, cf.c[3] + leja_off<32 * VEC>(i, cf.nc));
    ldv_stream<Tq, VEC>(cN, cf.c[4] + leja_off<32 * VEC>(i, cf.nc));
    if (DIM == 3) {
      ldv_stream<Tq, VEC>(cB, cf.c[5] + leja_off<32 * VEC>(i, cf.nc));
      ldv_stream<Tq, VEC>(cT, cf.c[6] + leja_off<32 * VEC>(i, cf.nc));
    }
    double p[VEC];
    if (m == 1) ldP<VEC>(p, p0 + i);
    else ldP<VEC>(p, P + i);
    Tq out[VEC];
    Tq sq = Tq(0);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const Tq west = k == 0 ? ql : qc[k - 1];
      const Tq east = k == VEC - 1 ? qr : qc[k + 1];
      Tq a;
      if constexpr (ND) {
        a = ((k == 0 ? r0 : Tq(0)) - sh_m) * qc[k];
        a = fma(cW[k], west - qc[k], a);
        a = fma(cE[k], east - qc[k], a);
        a = fma(cS[k], qs[k] - qc[k], a);
        a = fma(cN[k], qn[k] - qc[k], a);
        if (DIM == 3) {
          a = fma(cB[k], qb[k] - qc[k], a);
          a = fma(cT[k], qt[k] - qc[k], a);
        }
      } else {
        a = (cD[k] - sh_m) * qc[k];
        a = fma(cW[k], west, a);
        a = fma(cE[k], east, a);
        a = fma(cS[k], qs[k], a);
        a = fma(cN[k], qn[k], a);
        if (DIM == 3) {
          a = fma(cB[k], qb[k], a);
          a = fma(cT[k], qt[k], a);
        }
      }
      out[k] = a;
      if constexpr (sizeof(Tq) == 4) sq = fmaf(a, a, sq);
      else acc = fma(a, a, acc);
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k)
      p[k] = m == 1 ? d0 * p[k] : fma(dprev, to_f64_fast(qc[k]), p[k]);
    if constexpr (sizeof(Tq) == 4) {
      const float s = s_hi + sq;
      const float bp = s - s_hi;
      s_lo += (s_hi - (s - bp)) + (sq - bp);
      s_hi = s;
    }
    stv<Tq, VEC>(qo + i, out);
    stP<VEC>(P + i, p);
  }
  if constexpr (sizeof(Tq) == 4) acc = (double)s_hi + (double)s_lo;
  const double bs = block_reduce<0>(acc, sh);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * kRedSlots + (m & 1)] = bs;
}

// P += d_M q_M: the last product of a substep stopped at an even degree M
// (the term kernel updates P at odd m only).
template <typename Tq>
__global__ void k_pfix(double* __restrict__ P, const Tq* __restrict__ q,
                       const double* __restrict__ dd, int M, int Np) {
  const double d = dd[M];
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT)
    P[i] = fma(d, to_f64_fast(q[i]), P[i]);
}

__global__ void k_unpack(const double* __restrict__ src, double* __restrict__ dst, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    dst[i] = src[ip];
  }
}

// ---------------------------------------------------------------------------
// Krylov phi_1 (§4.1, Algorithm alg:al2): Arnoldi with modified Gram-Schmidt
// in FP64 over the padded layout (pads hold 0 in every vector and 0
// coefficients, so sums over all Np cells equal sums over the real cells).
// The scalars h_ij, ||r|| and ||J v_{m+1}|| stay in the device block KrDev;
// each pass reads the scalar the previous pass wrote, so a whole basis is
// built without a host round trip.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kr_cell(int ip, const Geo& g, int& ix, int& iy, int& iz) {
  const int row = ip / g.px;
  ix = ip - row * g.px;
  iy = row % g.ny;
  iz = row / g.ny;
}

// Consecutive passes sweep the cells in opposite directions (rev = 1: from
// the last cell down), so that a pass starts on the cells whose vectors the
// previous pass left in L2.
__device__ __forceinline__ int kr_index(int idx, int Np, int rev) { return rev ? Np - 1 - idx : idx; }

// beta = ||r||_2, arms the breakdown flag
__global__ void k_kr_norm0(const double* __restrict__ r, Geo g, double btol, double* part,
                           unsigned* cnt, KrDev* K, int rev) {
  __shared__ double sh[NT / 32];
  double acc = 0.0;
  for (int idx = blockIdx.x * NT + threadIdx.x; idx < g.Np; idx += gridDim.x * NT) {
    const int ip = kr_index(idx, g.Np, rev);
    acc = fma(r[ip], r[ip], acc);
  }
  double vals[1] = {block_reduce<0>(acc, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      K->beta = sqrt(s);
      K->btol = btol;
      K->breakdown = K->beta <= 0.0 ? 0 : -1;
    }
  }
}

// v_j = w_in / h (h = beta for j = 0, else h_{j,j-1}); w_out = J v_j.
// mode 0: the partial dot w_out . v_0 -> H(0, j); mode 1: ||w_out||_2 -> avnorm.
__global__ void k_kr_matvec(JIn J, const double* __restrict__ w_in, double* __restrict__ v_out,
                            double* __restrict__ w_out, const double* __restrict__ v0, Geo g, int j,
                            int mode, double* part, unsigned* cnt, KrDev* K, int rev) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&K->breakdown >= 0) return;
  const double h = j == 0 ? K->beta : K->H[j * kKrMax + (j - 1)];
  const double s = 1.0 / h;
  double acc = 0.0;
  for (int idx = blockIdx.x * NT + threadIdx.x; idx < g.Np; idx += gridDim.x * NT) {
    const int ip = kr_index(idx, g.Np, rev);
    int ix, iy, iz;
    kr_cell(ip, g, ix, iy, iz);
    const double vc = s * w_in[ip];
    v_out[ip] = vc;
    // J v_j = s (J w_in): one scaling of the sum instead of one per operand
    // (ten FP64 operations per cell instead of fifteen)
    const double a = s * japply_cell(J, w_in, ip, ix, iy, iz, g);
    w_out[ip] = a;
    acc = fma(a, mode == 0 ? (j == 0 ? vc : v0[ip]) : a, acc);
  }
  double vals[1] = {block_reduce<0>(acc, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double d = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      if (mode == 0) K->H[j] = d;   // H(0, j)
      else K->avnorm = sqrt(d);
    }
  }
}

// w -= h_{i-1,j} v_{i-1}; then the partial dot w . v_i -> H(i, j), or for
// the last pass ||w||_2 -> h_{j+1,j} (and the breakdown test).
__global__ void k_kr_orth(double* __restrict__ w, const double* __restrict__ vprev,
                          const double* __restrict__ vi, Geo g, int i, int j, int last,
                          double* part, unsigned* cnt, KrDev* K, int rev) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&K->breakdown >= 0) return;
  const double h = K->H[(i - 1) * kKrMax + j];
  double acc = 0.0;
  for (int idx = blockIdx.x * NT + threadIdx.x; idx < g.Np; idx += gridDim.x * NT) {
    const int ip = kr_index(idx, g.Np, rev);
    const double x = w[ip] - h * vprev[ip];
    w[ip] = x;
    acc = fma(x, last ? x : vi[ip], acc);
  }
  double vals[1] = {block_reduce<0>(acc, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double d = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      if (!last) {
        K->H[i * kKrMax + j] = d;
      } else {
        const double hn = sqrt(d);
        K->H[(j + 1) * kKrMax + j] = hn;
        if (hn <= K->btol) K->breakdown = j;
      }
    }
  }
}

// y += sum_i coef_i v_i
__global__ void k_kr_combine(double* __restrict__ y, KrComb cb, int Np, int rev) {
  for (int idx = blockIdx.x * NT + threadIdx.x; idx < Np; idx += gridDim.x * NT) {
    const int ip = kr_index(idx, Np, rev);
    double a = y[ip];
    for (int k = 0; k < cb.n; ++k) a = fma(cb.coef[k], cb.v[k][ip], a);
    y[ip] = a;
  }
}

// ---------------------------------------------------------------------------
// Adjoint of frozen-schedule EREM steps (linear fluid model).  A step is the
// Newton polynomial of §4.2 in J with its schedule and interval held; its
// transpose is the same polynomial in J^T, evaluated here by the Horner
// recurrence s_j = d_j mu + B_j^T s_{j+1}, B_j = (delta J - c I)/gamma -
// xi_j I.  Every use of J on a vector x with adjoint y adds to the
// derivative with respect to the upwind face fluxes F = (rho c)_f v:
// (y_R / C_R - y_L / C_L) x_up on an interior face, -y x / C on the x = 1
// face (stored in the x-face slot of the last column), y x / C on an outflow
// x = 0 face (one value per row).
// ---------------------------------------------------------------------------
struct AdjFaces {
  const double *Fx, *Fy, *Fz, *F0, *icap;
  double *gx, *gy, *gz, *g0;
};

// Transposed Leja copy: row i of J^T holds D_i and the neighbours' couplings
// towards i (E of the cell to the west, W of the cell to the east, ...).
template <typename Tq, int T>
__global__ void k_adj_scale_jlT(JOut jc, Tq* __restrict__ out, double sc, Geo g, int nc) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.Np; i += gridDim.x * NT) {
    int ix, iy, iz;
    const int row = i / g.px;
    ix = i - row * g.px;
    iy = row % g.ny;
    iz = row / g.ny;
    double c[7] = {0, 0, 0, 0, 0, 0, 0};
    if (ix < g.nx) {
      c[0] = jc.c[0][i];
      if (ix > 0) c[1] = jc.c[2][i - 1];
      if (ix < g.nx - 1) c[2] = jc.c[1][i + 1];
      if (iy > 0) c[3] = jc.c[4][i - g.px];
      if (iy < g.ny - 1) c[4] = jc.c[3][i + g.px];
      if (nc == 7) {
        if (iz > 0) c[5] = jc.c[6][i - g.plane];
        if (iz < g.nz - 1) c[6] = jc.c[5][i + g.plane];
      }
    }
    const size_t base = (size_t)(i / T) * nc * T + (i % T);
    for (int k = 0; k < nc; ++k) out[base + (size_t)k * T] = (Tq)(sc * c[k]);
  }
}

// out = a + J^T x (FP64, over the real cells; pads keep 0)
__global__ void k_adj_jT_apply(JIn J, const double* __restrict__ x, const double* __restrict__ a,
                               double* __restrict__ out, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    double v = J.c[0][ip] * x[ip];
    if (ix > 0) v += J.c[2][ip - 1] * x[ip - 1];
    if (ix < g.nx - 1) v += J.c[1][ip + 1] * x[ip + 1];
    if (iy > 0) v += J.c[4][ip - g.px] * x[ip - g.px];
    if (iy < g.ny - 1) v += J.c[3][ip + g.px] * x[ip + g.px];
    if (g.dim == 3) {
      if (iz > 0) v += J.c[6][ip - g.plane] * x[ip - g.plane];
      if (iz < g.nz - 1) v += J.c[5][ip + g.plane] * x[ip + g.plane];
    }
    out[ip] = a[ip] + v;
  }
}

// Face-flux derivative of one use of J: y^T J x (y, x of any precision).
template <typename Ty, typename Tx>
__device__ __forceinline__ void adj_face_cell(const AdjFaces& f, const Ty* __restrict__ y,
                                              const Tx* __restrict__ x, int ip, int ix, int iy,
                                              int iz, const Geo& g, double scale) {
  const double yc = (double)y[ip] * f.icap[ip];
  const double xc = (double)x[ip];
  if (ix < g.nx - 1) {
    const double F = f.Fx[ip];
    const double xu = F >= 0.0 ? xc : (double)x[ip + 1];
    f.gx[ip] += scale * ((double)y[ip + 1] * f.icap[ip + 1] - yc) * xu;
  } else {
    f.gx[ip] += scale * (-yc * xc);
  }
  if (iy < g.ny - 1) {
    const double F = f.Fy[ip];
    const double xu = F >= 0.0 ? xc : (double)x[ip + g.px];
    f.gy[ip] += scale * ((double)y[ip + g.px] * f.icap[ip + g.px] - yc) * xu;
  }
  if (g.dim == 3 && iz < g.nz - 1) {
    const double F = f.Fz[ip];
    const double xu = F >= 0.0 ? xc : (double)x[ip + g.plane];
    f.gz[ip] += scale * ((double)y[ip + g.plane] * f.icap[ip + g.plane] - yc) * xu;
  }
  if (ix == 0) {
    const int r = iy + g.ny * iz;
    if (!(f.F0[r] > 0.0)) f.g0[r] += scale * yc * xc;
  }
}

template <typename Ty, typename Tx>
__global__ void k_adj_face_pair(AdjFaces f, const Ty* __restrict__ y, const Tx* __restrict__ x,
                                double scale, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    adj_face_cell<Ty, Tx>(f, y, x, ip, ix, iy, iz, g, scale);
  }
}

// One Horner step of the transposed polynomial (Leja precision):
// s_out = d_j mu + ((delta J^T - c I)/gamma - xi_j I) s_in, and the face
// derivative of the pair (s_in, q_j) with the factor delta^2 / gamma.
template <typename Tq>
__global__ void k_adj_horner(const Tq* __restrict__ s_in, Tq* __restrict__ s_out,
                             const double* __restrict__ mu, const Tq* __restrict__ q,
                             const Tq* __restrict__ jlT, int T_tile, int nc, double dj,
                             double shift, double scale, int faces, AdjFaces f, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const size_t base = (size_t)(ip / T_tile) * nc * T_tile + (ip % T_tile);
    auto cf = [&](int k) { return jlT[base + (size_t)k * T_tile]; };
    const Tq sc = s_in[ip];
    Tq a = (cf(0) - (Tq)shift) * sc;
    if (ix > 0) a = fma(cf(1), s_in[ip - 1], a);
    if (ix < g.nx - 1) a = fma(cf(2), s_in[ip + 1], a);
    if (iy > 0) a = fma(cf(3), s_in[ip - g.px], a);
    if (iy < g.ny - 1) a = fma(cf(4), s_in[ip + g.px], a);
    if (g.dim == 3) {
      if (iz > 0) a = fma(cf(5), s_in[ip - g.plane], a);
      if (iz < g.nz - 1) a = fma(cf(6), s_in[ip + g.plane], a);
    }
    s_out[ip] = (Tq)(dj * mu[ip] + (double)a);
    if (faces) adj_face_cell<Tq, Tq>(f, s_in, q, ip, ix, iy, iz, g, scale);
  }
}

// FP32-bulk form of the Horner pass.  The face derivative of a use of J
// needs, per face, only the upwind side (one bit per face, from the signs of
// the face fluxes), the capacities and the two vectors; it is accumulated in
// FP32 over one adjoint step and flushed into the FP64 sums at its end.  With
// mu, the capacities and the accumulators in FP32 the pass moves s in/out,
// the transposed coefficients, mu, q_j, one flag byte, the capacity and the
// three accumulators (73 B per cell in 3D) and does no FP64 arithmetic away
// from the x = 0 column.
struct AdjFaces32 {
  const unsigned char* up;   // bit 0/1/2: F_x/F_y/F_z >= 0; bit 3: x = 0 face not inflowing
  const float* icap;
  float *gx, *gy, *gz;
  double* g0;
};

__global__ void k_adj_aux32(const double* __restrict__ Fx, const double* __restrict__ Fy,
                            const double* __restrict__ Fz, const double* __restrict__ F0,
                            const double* __restrict__ icap, unsigned char* __restrict__ up,
                            float* __restrict__ icap32, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    unsigned fl = 0;
    if (ix < g.nx - 1 && Fx[ip] >= 0.0) fl |= 1u;
    if (iy < g.ny - 1 && Fy[ip] >= 0.0) fl |= 2u;
    if (g.dim == 3 && iz < g.nz - 1 && Fz[ip] >= 0.0) fl |= 4u;
    if (ix == 0 && !(F0[iy + g.ny * iz] > 0.0)) fl |= 8u;
    up[ip] = (unsigned char)fl;
    icap32[ip] = (float)icap[ip];
  }
}

// VEC consecutive cells of one padded row per thread (px is a multiple of
// 4, so every row starts on a 16-byte boundary): vector loads of the
// vectors, coefficients, capacities and face sums, scalar loads only for the
// x neighbours beyond the VEC.  Pad lanes (ix >= nx) compute nothing and
// store 0.  The neighbour loads are unconditional, at the cell's own address
// where the neighbour is missing (its coupling there is 0), so a thread has
// all of them in flight at once.  The transposed coefficients are
// interleaved per tile of 32 VEC cells (T_TILE), so a warp reads each as one
// contiguous run.
template <int VEC>
struct RowV {
  int ip0, ix0, iy, iz;
};
template <int VEC>
__device__ __forceinline__ RowV<VEC> rowv_of(int v, const Geo& g) {
  RowV<VEC> r;
  r.ip0 = VEC * v;
  const int row = r.ip0 / g.px;
  r.ix0 = r.ip0 - row * g.px;
  r.iy = row % g.ny;
  r.iz = row / g.ny;
  return r;
}

template <int VEC>
__device__ __forceinline__ void ld_flags(unsigned (&fl)[VEC], const unsigned char* p) {
  if constexpr (VEC == 4) {
    const uchar4 u = *reinterpret_cast<const uchar4*>(p);
    fl[0] = u.x; fl[1] = u.y; fl[2] = u.z; fl[3] = u.w;
  } else {
    const uchar2 u = *reinterpret_cast<const uchar2*>(p);
    fl[0] = u.x; fl[1] = u.y;
  }
}

template <int VEC>
__global__ void __launch_bounds__(NT, 4)
k_adj_horner32(const float* __restrict__ s_in, float* __restrict__ s_out,
               const float* __restrict__ mu, const float* __restrict__ q,
               const float* __restrict__ jlT, int nc, float dj, float shift, float scale,
               AdjFaces32 f, Geo g) {
  constexpr int T_TILE = 32 * VEC;
  const int nvec = g.Np / VEC;
  const float* __restrict__ icap = f.icap;
  const unsigned char* __restrict__ up = f.up;
  float* __restrict__ gxp = f.gx;
  float* __restrict__ gyp = f.gy;
  float* __restrict__ gzp = f.gz;
  for (int v = blockIdx.x * NT + threadIdx.x; v < nvec; v += gridDim.x * NT) {
    const RowV<VEC> R = rowv_of<VEC>(v, g);
    const int ip0 = R.ip0;
    const size_t base = (size_t)(ip0 / T_TILE) * nc * T_TILE + (ip0 % T_TILE);
    const bool has_w = R.ix0 > 0, has_e = R.ix0 + VEC < g.nx;
    const bool has_s = R.iy > 0, has_n = R.iy < g.ny - 1;
    const bool has_b = g.dim == 3 && R.iz > 0, has_t = g.dim == 3 && R.iz < g.nz - 1;
    const int oS = has_s ? -g.px : 0, oN = has_n ? g.px : 0;
    const int oB = has_b ? -g.plane : 0, oT = has_t ? g.plane : 0;
    const int oE = has_e ? VEC : 0;
    // every load of the vector first (the face-sum inputs do not depend on
    // the stencil), so that one round trip to memory covers them all
    float sc[VEC], sS[VEC], sN[VEC], sB[VEC], sT[VEC], cf[7][VEC], m4[VEC];
    ldv<float, VEC>(sc, s_in + ip0);
    ldv<float, VEC>(sS, s_in + ip0 + oS);
    ldv<float, VEC>(sN, s_in + ip0 + oN);
    if (g.dim == 3) {
      ldv<float, VEC>(sB, s_in + ip0 + oB);
      ldv<float, VEC>(sT, s_in + ip0 + oT);
    }
    const float sw = s_in[ip0 - (has_w ? 1 : 0)];
    const float se = s_in[ip0 + oE];
#pragma unroll
    for (int k = 0; k < 7; ++k)
      if (k < nc) ldv<float, VEC>(cf[k], jlT + base + k * T_TILE);
    ldv<float, VEC>(m4, mu + ip0);
    float ic[VEC], x4[VEC], gsx[VEC], icN[VEC], xN[VEC], gsy[VEC], icT[VEC], xT[VEC], gsz[VEC];
    unsigned fl[VEC];
    ldv<float, VEC>(ic, icap + ip0);
    ldv<float, VEC>(x4, q + ip0);
    ld_flags<VEC>(fl, up + ip0);
    const float ice = icap[ip0 + oE];
    const float qe = q[ip0 + oE];
    ldv<float, VEC>(gsx, gxp + ip0);
    ldv<float, VEC>(icN, icap + ip0 + oN);
    ldv<float, VEC>(xN, q + ip0 + oN);
    ldv<float, VEC>(gsy, gyp + ip0);
    if (g.dim == 3) {
      ldv<float, VEC>(icT, icap + ip0 + oT);
      ldv<float, VEC>(xT, q + ip0 + oT);
      ldv<float, VEC>(gsz, gzp + ip0);
    }

    float a[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      float x = (cf[0][j] - shift) * sc[j];
      x = fmaf(cf[1][j], j > 0 ? sc[j - 1] : (has_w ? sw : 0.0f), x);
      x = fmaf(cf[2][j], j < VEC - 1 ? sc[j + 1] : (has_e ? se : 0.0f), x);
      x = fmaf(cf[3][j], sS[j], x);
      x = fmaf(cf[4][j], sN[j], x);
      if (g.dim == 3) {
        x = fmaf(cf[5][j], sB[j], x);
        x = fmaf(cf[6][j], sT[j], x);
      }
      a[j] = R.ix0 + j < g.nx ? fmaf(dj, m4[j], x) : 0.0f;
    }
    stv<float, VEC>(s_out + ip0, a);

    // face derivative of the pair (s_in, q_j)
    float yc[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) yc[j] = sc[j] * ic[j];
    const float ye = has_e ? se * ice : 0.0f;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int ix = R.ix0 + j;
      if (ix < g.nx - 1) {
        const float yr = j < VEC - 1 ? yc[j + 1] : ye;
        const float xu = (fl[j] & 1u) ? x4[j] : (j < VEC - 1 ? x4[j + 1] : qe);
        gsx[j] += scale * ((yr - yc[j]) * xu);
      } else if (ix == g.nx - 1) {
        gsx[j] -= scale * (yc[j] * x4[j]);
      }
    }
    stv<float, VEC>(gxp + ip0, gsx);
    if (has_n) {
#pragma unroll
      for (int j = 0; j < VEC; ++j)
        if (R.ix0 + j < g.nx) {
          const float xu = (fl[j] & 2u) ? x4[j] : xN[j];
          gsy[j] += scale * (fmaf(sN[j], icN[j], -yc[j]) * xu);
        }
      stv<float, VEC>(gyp + ip0, gsy);
    }
    if (has_t) {
#pragma unroll
      for (int j = 0; j < VEC; ++j)
        if (R.ix0 + j < g.nx) {
          const float xu = (fl[j] & 4u) ? x4[j] : xT[j];
          gsz[j] += scale * (fmaf(sT[j], icT[j], -yc[j]) * xu);
        }
      stv<float, VEC>(gzp + ip0, gsz);
    }
    if (R.ix0 == 0 && (fl[0] & 8u)) f.g0[R.iy + g.ny * R.iz] += (double)(scale * (yc[0] * x4[0]));
  }
}

// the FP64 face sums += the FP32 ones of this adjoint step; FP32 sums = 0
__global__ void k_adj_flush32(float* __restrict__ gx32, float* __restrict__ gy32,
                              float* __restrict__ gz32, double* __restrict__ gx,
                              double* __restrict__ gy, double* __restrict__ gz, int Np) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) {
    gx[i] += (double)gx32[i];
    gx32[i] = 0.0f;
    gy[i] += (double)gy32[i];
    gy32[i] = 0.0f;
    if (gz32) {
      gz[i] += (double)gz32[i];
      gz32[i] = 0.0f;
    }
  }
}

// s = d mu in FP32 and the FP32 copy of mu
__global__ void k_adj_start32(const double* __restrict__ mu, double d, float* __restrict__ s,
                              float* __restrict__ mu32, int Np) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) {
    s[i] = (float)(d * mu[i]);
    mu32[i] = (float)mu[i];
  }
}

// z = delta s (FP64); zacc += z
template <typename Tq>
__global__ void k_adj_z(const Tq* __restrict__ s, double delta, double* __restrict__ z,
                        double* __restrict__ zacc, int Np) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) {
    const double v = delta * (double)s[i];
    z[i] = v;
    zacc[i] += v;
  }
}

// s = d mu in the Leja precision (the first Horner value)
template <typename Tq>
__global__ void k_adj_start(const double* __restrict__ mu, double d, Tq* __restrict__ s, int Np) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < Np; i += gridDim.x * NT) s[i] = (Tq)(d * mu[i]);
}

// the constant inflow term of G: y^T b through the x = 0 faces
__global__ void k_adj_b_use(AdjFaces f, const double* __restrict__ y, double T_in, Geo g) {
  const int nf = g.ny * g.nz;
  for (int r = blockIdx.x * NT + threadIdx.x; r < nf; r += gridDim.x * NT) {
    const int ip = g.px * r;
    if (f.F0[r] > 0.0) f.g0[r] += y[ip] * f.icap[ip] * T_in;
  }
}

// dL/dp from dL/dF (gathered per cell) into the right-hand side b of the
// pressure system; x = 0 as the initial guess.
__global__ void k_adj_dLdp(AdjFaces f, const double* __restrict__ lnk, double rc, Phys ph,
                           double* __restrict__ b, double* __restrict__ x,
                           const double* __restrict__ Ux, const double* __restrict__ Uy,
                           const double* __restrict__ Uz, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    double r = 0.0;
    if (ix < g.nx - 1) r += rc * f.gx[ip] * Ux[ip];
    if (ix > 0) r -= rc * f.gx[ip - 1] * Ux[ip - 1];
    if (iy < g.ny - 1) r += rc * f.gy[ip] * Uy[ip];
    if (iy > 0) r -= rc * f.gy[ip - g.px] * Uy[ip - g.px];
    if (g.dim == 3) {
      if (iz < g.nz - 1) r += rc * f.gz[ip] * Uz[ip];
      if (iz > 0) r -= rc * f.gz[ip - g.plane] * Uz[ip - g.plane];
    }
    const double uD = ph.ax * exp(lnk[ip]) / (0.5 * ph.hx);
    if (ix == 0) r -= rc * f.g0[iy + g.ny * iz] * uD;
    if (ix == g.nx - 1) r += rc * f.gx[ip] * uD;
    b[ip] = r;
    x[ip] = 0.0;
  }
}

// dL/dlnK per cell from dL/dF, the pressure p and the adjoint pressure mu
__global__ void k_adj_lnk(AdjFaces f, const double* __restrict__ lnk, const double* __restrict__ p,
                          const double* __restrict__ mu, double rc, Phys ph,
                          const double* __restrict__ Ux, const double* __restrict__ Uy,
                          const double* __restrict__ Uz, double* __restrict__ out, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double kc = exp(lnk[ip]);
    double acc = 0.0;
    auto face = [&](const double* gf, const double* U, int L, int R, int self_is_left) {
      const double kL = exp(lnk[L]), kR = exp(lnk[R]);
      const double phi_s = (p[L] - p[R]) * (rc * gf[L] - (mu[L] - mu[R]));
      acc += phi_s * U[L] * (self_is_left ? kR : kL) / (kL + kR);
    };
    if (ix < g.nx - 1) face(f.gx, Ux, ip, ip + 1, 1);
    if (ix > 0) face(f.gx, Ux, ip - 1, ip, 0);
    if (iy < g.ny - 1) face(f.gy, Uy, ip, ip + g.px, 1);
    if (iy > 0) face(f.gy, Uy, ip - g.px, ip, 0);
    if (g.dim == 3) {
      if (iz < g.nz - 1) face(f.gz, Uz, ip, ip + g.plane, 1);
      if (iz > 0) face(f.gz, Uz, ip - g.plane, ip, 0);
    }
    const double uD = ph.ax * kc / (0.5 * ph.hx);
    if (ix == 0) acc += uD * (ph.head_left - p[ip]) * (rc * f.g0[iy + g.ny * iz] + mu[ip]);
    if (ix == g.nx - 1) acc += uD * (p[ip] - ph.head_right) * (rc * f.gx[ip] - mu[ip]);
    out[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// pressure: TPFA mass-mobility transmissibilities and Jacobi-PCG
// ---------------------------------------------------------------------------
struct PresArr {
  double *x, *r, *z, *d0, *d1, *Ad, *Ux, *Uy, *Uz, *diag, *b;
};

// TPFA pressure matrix from the cell mobilities m: upper couplings, diagonal
// (with the Dirichlet faces at x = 0 and x = 1) and right-hand side
__global__ void k_pres_faces(const double* __restrict__ m, PresArr a, Geo g, Phys ph) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double mi = m[ip];
    double dg = 0.0, bb = 0.0;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    if (ix < g.nx - 1) ux = harm(ph.ax, 0.5 * ph.hx, mi, m[ip + 1]);
    if (iy < g.ny - 1) uy = harm(ph.ay, 0.5 * ph.hy, mi, m[ip + g.px]);
    if (g.dim == 3 && iz < g.nz - 1) uz = harm(ph.az, 0.5 * ph.hz, mi, m[ip + g.plane]);
    a.Ux[ip] = ux;
    a.Uy[ip] = uy;
    if (g.dim == 3) a.Uz[ip] = uz;
    dg += ux + uy + uz;
    if (ix > 0) dg += harm(ph.ax, 0.5 * ph.hx, m[ip - 1], mi);
    if (iy > 0) dg += harm(ph.ay, 0.5 * ph.hy, m[ip - g.px], mi);
    if (g.dim == 3 && iz > 0) dg += harm(ph.az, 0.5 * ph.hz, m[ip - g.plane], mi);
    const double uD = ph.ax * mi / (0.5 * ph.hx);
    if (ix == 0) { dg += uD; bb += uD * ph.head_left; }
    if (ix == g.nx - 1) { dg += uD; bb += uD * ph.head_right; }
    a.diag[ip] = dg;
    a.b[ip] = bb;
  }
}

__device__ __forceinline__ double pres_apply(const PresArr& a, const double* __restrict__ x, int ip,
                                             int ix, int iy, int iz, const Geo& g) {
  double v = a.diag[ip] * x[ip];
  if (ix < g.nx - 1) v -= a.Ux[ip] * x[ip + 1];
  if (ix > 0) v -= a.Ux[ip - 1] * x[ip - 1];
  if (iy < g.ny - 1) v -= a.Uy[ip] * x[ip + g.px];
  if (iy > 0) v -= a.Uy[ip - g.px] * x[ip - g.px];
  if (g.dim == 3) {
    if (iz < g.nz - 1) v -= a.Uz[ip] * x[ip + g.plane];
    if (iz > 0) v -= a.Uz[ip - g.plane] * x[ip - g.plane];
  }
  return v;
}

// r = b - A x, z = r / diag, d_old = 0; rz, rr, bb
__global__ void k_cg_init(PresArr a, Geo g, double tol, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double r = a.b[ip] - pres_apply(a, a.x, ip, ix, iy, iz, g);
    const double z = r / a.diag[ip];
    a.r[ip] = r;
    a.z[ip] = z;
    a.d0[ip] = 0.0;
    rz += r * z;
    rr += r * r;
    bb += a.b[ip] * a.b[ip];
  }
  double vals[3];
  vals[0] = block_reduce<0>(rz, sh);
  vals[1] = block_reduce<0>(rr, sh);
  vals[2] = block_reduce<0>(bb, sh);
  if (publish_partials(part, cnt, vals, 3)) {
    const double a0 = gather_partials<0>(part, 0, sh);
    const double a1 = gather_partials<0>(part, 1, sh);
    const double a2 = gather_partials<0>(part, 2, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin[K_RZ] = a0;
      ctrl->lin[K_RR] = a1;
      ctrl->lin[K_BB] = a2;
      ctrl->lin[K_BETA] = 0.0;
      ctrl->lin[K_TOL2] = tol * tol * a2;
      ctrl->lin_it = 0;
      ctrl->lin_break = 0;
      ctrl->lin_done = (a1 <= tol * tol * a2) ? 1 : 0;
    }
  }
}

// d_new = z + beta d_old; Ad = A d_new; (d, Ad) -> alpha.  z is the
// preconditioned residual: FP64 (Jacobi) or FP32 (polynomial preconditioner).
template <typename Tz>
__global__ void k_cg_dir(PresArr a, const Tz* __restrict__ z, const double* __restrict__ dold,
                         double* __restrict__ dnew, Geo g, double* part, unsigned* cnt,
                         Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  const double beta = ctrl->lin[K_BETA];
  double dad = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    auto dn = [&](int j) { return (double)z[j] + beta * dold[j]; };
    const double di = dn(ip);
    double v = a.diag[ip] * di;
    if (ix < g.nx - 1) v -= a.Ux[ip] * dn(ip + 1);
    if (ix > 0) v -= a.Ux[ip - 1] * dn(ip - 1);
    if (iy < g.ny - 1) v -= a.Uy[ip] * dn(ip + g.px);
    if (iy > 0) v -= a.Uy[ip - g.px] * dn(ip - g.px);
    if (g.dim == 3) {
      if (iz < g.nz - 1) v -= a.Uz[ip] * dn(ip + g.plane);
      if (iz > 0) v -= a.Uz[ip - g.plane] * dn(ip - g.plane);
    }
    dnew[ip] = di;
    a.Ad[ip] = v;
    dad += di * v;
  }
  double vals[1] = {block_reduce<0>(dad, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin[K_DAD] = s;
      if (!(s > 0.0) || !isfinite(s)) {
        ctrl->lin_break = 1;
        ctrl->lin_done = 1;
      } else {
        ctrl->lin[K_ALPHA] = ctrl->lin[K_RZ] / s;
      }
    }
  }
}

// x += alpha d, r -= alpha Ad, z = r / diag; rz_new, rr -> beta, convergence
__global__ void k_cg_upd(PresArr a, const double* __restrict__ d, Geo g, double* part,
                         unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  const double alpha = ctrl->lin[K_ALPHA];
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    a.x[ip] += alpha * d[ip];
    const double r = a.r[ip] - alpha * a.Ad[ip];
    const double z = r / a.diag[ip];
    a.r[ip] = r;
    a.z[ip] = z;
    rz += r * z;
    rr += r * r;
  }
  double vals[2] = {block_reduce<0>(rz, sh), 0.0};
  vals[1] = block_reduce<0>(rr, sh);
  if (publish_partials(part, cnt, vals, 2)) {
    const double s0 = gather_partials<0>(part, 0, sh);
    const double s1 = gather_partials<0>(part, 1, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin_it += 1;
      ctrl->lin[K_BETA] = s0 / ctrl->lin[K_RZ];
      ctrl->lin[K_RZ] = s0;
      ctrl->lin[K_RR] = s1;
      if (s1 <= ctrl->lin[K_TOL2]) ctrl->lin_done = 1;
      if (!isfinite(s1)) { ctrl->lin_break = 1; ctrl->lin_done = 1; }
    }
  }
}

// ---------------------------------------------------------------------------
// Polynomial preconditioner for the pressure CG.  z = p(D^-1 A) D^-1 r is
// `deg` steps of Chebyshev iteration for A z = r from z = 0 on the interval
// [2/ratio, 2] that contains the spectrum of D^-1 A above its low end (D the
// diagonal; the Gershgorin discs of D^-1 A lie in [0, 2]), so p(A) A has its
// spectrum compressed towards 1 and the outer CG needs about deg times fewer
// iterations.  The sweeps are stencil passes in FP32 (z, the residual copy and
// the matrix coefficients), bound by HBM; the outer CG stays FP64 and, since
// an FP32 polynomial is a fixed linear map only up to rounding, takes the
// Polak-Ribiere beta = z_new.(r_new - r_old) / (z_old.r_old), with
// r_new - r_old = -alpha A d, which is robust to it.
// ---------------------------------------------------------------------------
struct PcArr {
  float *dinv, *Ux, *Uy, *Uz, *r;
};

// FP32 coefficients: 1/diag and the face couplings
__global__ void k_pc_setup(PresArr a, PcArr p, float* __restrict__ diag32, Geo g) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    p.dinv[ip] = (float)(1.0 / a.diag[ip]);
    if (diag32) diag32[ip] = (float)a.diag[ip];
    p.Ux[ip] = (float)a.Ux[ip];
    p.Uy[ip] = (float)a.Uy[ip];
    if (g.dim == 3) p.Uz[ip] = (float)a.Uz[ip];
  }
}

// One Chebyshev step, four cells of a padded row per thread (RowV<4>).  FIRST:
// z_1 = D^-1 r / theta (c2 = 1/theta) and the FP32 copy of r.  Otherwise
// z_{j+1} = z_j + c1 (z_j - z_{j-1}) + c2 (D^-1 (r + N z_j) - z_j), A = D - N.
// LAST: also (z, r) and (z, A d) -> beta (zero on the first pass after the
// set-up) and (z, r) for alpha.  Pad lanes store 0 and enter no sum.
template <bool FIRST, bool LAST>
__global__ void k_pc_sweep(PresArr a, PcArr p, const float* __restrict__ zprev,
                           const float* __restrict__ zcur, float* __restrict__ znew, float c1,
                           float c2, Geo g, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  double rz = 0.0, zad = 0.0;
  const int nvec = g.Np / 4;
  for (int v = blockIdx.x * NT + threadIdx.x; v < nvec; v += gridDim.x * NT) {
    const RowV<4> R = rowv_of<4>(v, g);
    const int ip0 = R.ip0;
    float zn[4], di[4];
    ldv<float, 4>(di, p.dinv + ip0);
    if (FIRST) {
      const double2 ra = *reinterpret_cast<const double2*>(a.r + ip0);
      const double2 rb = *reinterpret_cast<const double2*>(a.r + ip0 + 2);
      float r32[4] = {(float)ra.x, (float)ra.y, (float)rb.x, (float)rb.y};
      if (!LAST) stv<float, 4>(p.r + ip0, r32);
#pragma unroll
      for (int j = 0; j < 4; ++j) zn[j] = c2 * (di[j] * r32[j]);
    } else {
      float zc[4], zp[4] = {0, 0, 0, 0}, s[4], u[4], nb[4];
      ldv<float, 4>(zc, zcur + ip0);
      if (zprev) ldv<float, 4>(zp, zprev + ip0);   // z_0 = 0
      ldv<float, 4>(s, p.r + ip0);
      ldv<float, 4>(u, p.Ux + ip0);                 // coupling to the east neighbour
      const bool has_w = R.ix0 > 0, has_e = R.ix0 + 4 < g.nx;
      const float uw = has_w ? p.Ux[ip0 - 1] : 0.0f;
      const float zw = has_w ? zcur[ip0 - 1] : 0.0f;
      const float ze = has_e ? zcur[ip0 + 4] : 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int ix = R.ix0 + j;
        if (ix < g.nx - 1) s[j] = fmaf(u[j], j < 3 ? zc[j + 1] : ze, s[j]);
        if (ix > 0) s[j] = fmaf(j > 0 ? u[j - 1] : uw, j > 0 ? zc[j - 1] : zw, s[j]);
      }
      if (R.iy < g.ny - 1) {
        ldv<float, 4>(u, p.Uy + ip0);
        ldv<float, 4>(nb, zcur + ip0 + g.px);
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] = fmaf(u[j], nb[j], s[j]);
      }
      if (R.iy > 0) {
        ldv<float, 4>(u, p.Uy + ip0 - g.px);
        ldv<float, 4>(nb, zcur + ip0 - g.px);
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] = fmaf(u[j], nb[j], s[j]);
      }
      if (g.dim == 3) {
        if (R.iz < g.nz - 1) {
          ldv<float, 4>(u, p.Uz + ip0);
          ldv<float, 4>(nb, zcur + ip0 + g.plane);
#pragma unroll
          for (int j = 0; j < 4; ++j) s[j] = fmaf(u[j], nb[j], s[j]);
        }
        if (R.iz > 0) {
          ldv<float, 4>(u, p.Uz + ip0 - g.plane);
          ldv<float, 4>(nb, zcur + ip0 - g.plane);
#pragma unroll
          for (int j = 0; j < 4; ++j) s[j] = fmaf(u[j], nb[j], s[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) zn[j] = zc[j] + c1 * (zc[j] - zp[j]) + c2 * fmaf(di[j], s[j], -zc[j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (R.ix0 + j >= g.nx) zn[j] = 0.0f;
    stv<float, 4>(znew + ip0, zn);
    if (LAST) {
      const double2 ra = *reinterpret_cast<const double2*>(a.r + ip0);
      const double2 rb = *reinterpret_cast<const double2*>(a.r + ip0 + 2);
      const double2 da = *reinterpret_cast<const double2*>(a.Ad + ip0);
      const double2 db = *reinterpret_cast<const double2*>(a.Ad + ip0 + 2);
      const double rr[4] = {ra.x, ra.y, rb.x, rb.y}, dd[4] = {da.x, da.y, db.x, db.y};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (R.ix0 + j < g.nx) {
          rz += (double)zn[j] * rr[j];
          zad += (double)zn[j] * dd[j];
        }
    }
  }
  if (!LAST) return;
  double vals[2] = {block_reduce<0>(rz, sh), 0.0};
  vals[1] = block_reduce<0>(zad, sh);
  if (publish_partials(part, cnt, vals, 2)) {
    const double s0 = gather_partials<0>(part, 0, sh);
    const double s1 = gather_partials<0>(part, 1, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      const double beta = ctrl->lin_it == 0 ? 0.0 : -ctrl->lin[K_ALPHA] * s1 / ctrl->lin[K_RZ];
      ctrl->lin[K_BETA] = beta;
      ctrl->lin[K_RZ] = s0;
      if (!(s0 > 0.0) || !isfinite(s0) || !isfinite(beta)) {
        ctrl->lin_break = 1;
        ctrl->lin_done = 1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Multigrid preconditioner for the pressure CG: aggregates of 2 x 2 (x 2)
// cells, piecewise-constant prolongation P and restriction P^T, Galerkin
// coarse operators P^T A P (again 5- or 7-point M-matrices: a coarse face
// coupling is the sum of the fine couplings across it, a coarse diagonal the
// sum of the children's diagonals minus twice their internal couplings),
// Chebyshev-Jacobi smoothing in FP32, the coarse correction over-weighted by
// omega (piecewise-constant prolongation under-corrects smooth errors), and
// a single-block CG on the coarsest level.  One V-cycle is the
// preconditioner of the flexible FP64 CG.
// ---------------------------------------------------------------------------
struct MgL {
  float *diag, *dinv, *Ux, *Uy, *Uz;
  Geo g;
};

// the children of coarse cell (X, Y, Z): [2X, min(2X+2, nx)) x ...
__global__ void k_mg_coarsen(MgL f, MgL c) {
  for (int I = blockIdx.x * NT + threadIdx.x; I < c.g.N; I += gridDim.x * NT) {
    int X, Y, Z, IP;
    cell_of(I, c.g, X, Y, Z, IP);
    const int xe = min(2 * X + 2, f.g.nx), ye = min(2 * Y + 2, f.g.ny);
    const int ze = f.g.dim == 3 ? min(2 * Z + 2, f.g.nz) : 1;
    double dg = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
    for (int iz = (f.g.dim == 3 ? 2 * Z : 0); iz < ze; ++iz)
      for (int iy = 2 * Y; iy < ye; ++iy)
        for (int ix = 2 * X; ix < xe; ++ix) {
          const int ip = ix + f.g.px * (iy + f.g.ny * iz);
          dg += f.diag[ip];
          if (ix + 1 < xe) dg -= 2.0 * f.Ux[ip];
          else if (ix + 1 < f.g.nx) ux += f.Ux[ip];
          if (iy + 1 < ye) dg -= 2.0 * f.Uy[ip];
          else if (iy + 1 < f.g.ny) uy += f.Uy[ip];
          if (f.g.dim == 3) {
            if (iz + 1 < ze) dg -= 2.0 * f.Uz[ip];
            else if (iz + 1 < f.g.nz) uz += f.Uz[ip];
          }
        }
    c.diag[IP] = (float)dg;
    c.dinv[IP] = (float)(1.0 / dg);
    c.Ux[IP] = (float)ux;
    c.Uy[IP] = (float)uy;
    if (c.g.dim == 3) c.Uz[IP] = (float)uz;
  }
}

// (N x)_i: the couplings of cell i to its neighbours applied to x
__device__ __forceinline__ float mg_offdiag(const MgL& L, const float* __restrict__ x, int ip, int ix,
                                            int iy, int iz) {
  float s = 0.0f;
  if (ix < L.g.nx - 1) s = fmaf(L.Ux[ip], x[ip + 1], s);
  if (ix > 0) s = fmaf(L.Ux[ip - 1], x[ip - 1], s);
  if (iy < L.g.ny - 1) s = fmaf(L.Uy[ip], x[ip + L.g.px], s);
  if (iy > 0) s = fmaf(L.Uy[ip - L.g.px], x[ip - L.g.px], s);
  if (L.g.dim == 3) {
    if (iz < L.g.nz - 1) s = fmaf(L.Uz[ip], x[ip + L.g.plane], s);
    if (iz > 0) s = fmaf(L.Uz[ip - L.g.plane], x[ip - L.g.plane], s);
  }
  return s;
}

// One Chebyshev-Jacobi step on a coarse level: xn = xc + c1 (xc - xp) +
// c2 (D^-1 (rhs + N xc) - xc); xc = NULL means x = 0 (xn = c2 D^-1 rhs),
// xp = NULL means 0.
__global__ void k_mg_sweep(MgL L, const float* __restrict__ rhs, const float* __restrict__ xp,
                           const float* __restrict__ xc, float* __restrict__ xn, float c1,
                           float c2) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < L.g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, L.g, ix, iy, iz, ip);
    if (!xc) {
      xn[ip] = c2 * (L.dinv[ip] * rhs[ip]);
      continue;
    }
    const float z = xc[ip];
    const float zp = xp ? xp[ip] : 0.0f;
    const float s = rhs[ip] + mg_offdiag(L, xc, ip, ix, iy, iz);
    xn[ip] = z + c1 * (z - zp) + c2 * fmaf(L.dinv[ip], s, -z);
  }
}

// rhs_c = P^T (rhs_f - A_f x_f)
__global__ void k_mg_restrict(MgL f, const float* __restrict__ rhs_f, const float* __restrict__ x_f,
                              MgL c, float* __restrict__ rhs_c) {
  for (int I = blockIdx.x * NT + threadIdx.x; I < c.g.N; I += gridDim.x * NT) {
    int X, Y, Z, IP;
    cell_of(I, c.g, X, Y, Z, IP);
    const int xe = min(2 * X + 2, f.g.nx), ye = min(2 * Y + 2, f.g.ny);
    const int ze = f.g.dim == 3 ? min(2 * Z + 2, f.g.nz) : 1;
    float acc = 0.0f;
    for (int iz = (f.g.dim == 3 ? 2 * Z : 0); iz < ze; ++iz)
      for (int iy = 2 * Y; iy < ye; ++iy)
        for (int ix = 2 * X; ix < xe; ++ix) {
          const int ip = ix + f.g.px * (iy + f.g.ny * iz);
          acc += rhs_f[ip] - fmaf(f.diag[ip], x_f[ip], -mg_offdiag(f, x_f, ip, ix, iy, iz));
        }
    rhs_c[IP] = acc;
  }
}

// x_f += omega P x_c
__global__ void k_mg_prolong(MgL f, float* __restrict__ x_f, MgL c, const float* __restrict__ x_c,
                             float omega) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < f.g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, f.g, ix, iy, iz, ip);
    const int I = (ix >> 1) + c.g.px * ((iy >> 1) + c.g.ny * (f.g.dim == 3 ? (iz >> 1) : 0));
    x_f[ip] = fmaf(omega, x_c[I], x_f[ip]);
  }
}

// Coarsest level: Jacobi-preconditioned CG in one block, from x = 0, to
// ||r|| <= rtol ||b|| or maxit iterations (N <= a few thousand cells).
constexpr int kMgCoarseThreads = 512;
constexpr float kMgCoarseRtol = 1e-3f;  // the coarsest solve only needs to remove smooth error
__device__ float mg_block_sum(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float t = threadIdx.x < (kMgCoarseThreads / 32) ? sh[threadIdx.x] : 0.0f;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) sh[32] = t;
  __syncthreads();
  return sh[32];
}

__global__ void __launch_bounds__(kMgCoarseThreads)
k_mg_coarse_cg(MgL L, const float* __restrict__ b, float* __restrict__ x, float* __restrict__ r,
               float* __restrict__ p, float* __restrict__ q, int maxit, float rtol) {
  __shared__ float sh[33];
  const int N = L.g.N;
  float rz = 0.0f, bb = 0.0f;
  for (int i = threadIdx.x; i < N; i += kMgCoarseThreads) {
    x[i] = 0.0f;
    r[i] = b[i];
    p[i] = L.dinv[i] * b[i];
    rz += r[i] * p[i];
    bb += b[i] * b[i];
  }
  rz = mg_block_sum(rz, sh);
  bb = mg_block_sum(bb, sh);
  const float stop = rtol * rtol * bb;
  for (int it = 0; it < maxit && bb > 0.0f; ++it) {
    float pq = 0.0f;
    for (int i = threadIdx.x; i < N; i += kMgCoarseThreads) {
      int ix, iy, iz, ip;
      cell_of(i, L.g, ix, iy, iz, ip);
      const float v = fmaf(L.diag[ip], p[ip], -mg_offdiag(L, p, ip, ix, iy, iz));
      q[ip] = v;
      pq += p[ip] * v;
    }
    pq = mg_block_sum(pq, sh);
    if (!(pq > 0.0f)) break;
    const float alpha = rz / pq;
    float rr = 0.0f, rzn = 0.0f;
    for (int i = threadIdx.x; i < N; i += kMgCoarseThreads) {
      x[i] = fmaf(alpha, p[i], x[i]);
      r[i] = fmaf(-alpha, q[i], r[i]);
      rr += r[i] * r[i];
      rzn += r[i] * (L.dinv[i] * r[i]);
    }
    rr = mg_block_sum(rr, sh);
    rzn = mg_block_sum(rzn, sh);
    if (rr <= stop) break;
    const float beta = rzn / rz;
    rz = rzn;
    for (int i = threadIdx.x; i < N; i += kMgCoarseThreads) p[i] = fmaf(beta, p[i], L.dinv[i] * r[i]);
    __syncthreads();
  }
}

// Sum over the block of two per-thread values, every thread getting both
// totals: warp sums in `slot` (one float2 per warp), one block sync, then each
// thread adds the warp sums itself in the same order (the same totals in every
// thread).  Two calls in a row take different slots.
__device__ __forceinline__ float2 mg_block_sum2(float a, float b, float2* slot) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = make_float2(a, b);
  __syncthreads();
  float2 t = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int w = 0; w < kMgCoarseThreads / 32; ++w) {
    const float2 v = slot[w];
    t.x += v.x;
    t.y += v.y;
  }
  return t;
}

// Coarsest level with at most kMgCoarseThreads cells: the Jacobi-PCG of
// k_mg_coarse_cg with one cell per thread, its coefficients, x and r in
// registers and only the direction p in shared memory (the stencil's
// neighbour reads); three block syncs per iteration.  rv is this thread's
// entry of the right-hand side (0 past N); returns its entry of x.
__device__ float mg_cg_block(const MgL& L, float rv, int maxit, float rtol, float* ps,
                             float2 (*slot)[kMgCoarseThreads / 32]) {
  const int N = L.g.N;
  const bool own = (int)threadIdx.x < N;
  int ix = 0, iy = 0, iz = 0, ip = 0;
  float dg = 0.0f, dinv = 0.0f, cw = 0.0f, ce = 0.0f, cs = 0.0f, cn = 0.0f, cb = 0.0f, ct = 0.0f;
  float xv = 0.0f;
  if (own) {
    cell_of((int)threadIdx.x, L.g, ix, iy, iz, ip);
    dg = L.diag[ip];
    dinv = L.dinv[ip];
    if (ix > 0) cw = L.Ux[ip - 1];
    if (ix < L.g.nx - 1) ce = L.Ux[ip];
    if (iy > 0) cs = L.Uy[ip - L.g.px];
    if (iy < L.g.ny - 1) cn = L.Uy[ip];
    if (L.g.dim == 3) {
      if (iz > 0) cb = L.Uz[ip - L.g.plane];
      if (iz < L.g.nz - 1) ct = L.Uz[ip];
    }
    ps[ip] = dinv * rv;
  }
  const float2 s0 = mg_block_sum2(rv * (dinv * rv), rv * rv, slot[0]);
  float rz = s0.x;
  const float stop = rtol * rtol * s0.y;
  for (int it = 0; it < maxit && s0.y > 0.0f; ++it) {
    __syncthreads();  // p complete
    float pv = 0.0f, v = 0.0f;
    if (own) {
      pv = ps[ip];
      float o = 0.0f;
      if (ix > 0) o = fmaf(cw, ps[ip - 1], o);
      if (ix < L.g.nx - 1) o = fmaf(ce, ps[ip + 1], o);
      if (iy > 0) o = fmaf(cs, ps[ip - L.g.px], o);
      if (iy < L.g.ny - 1) o = fmaf(cn, ps[ip + L.g.px], o);
      if (L.g.dim == 3) {
        if (iz > 0) o = fmaf(cb, ps[ip - L.g.plane], o);
        if (iz < L.g.nz - 1) o = fmaf(ct, ps[ip + L.g.plane], o);
      }
      v = fmaf(dg, pv, -o);
    }
    const float pq = mg_block_sum2(pv * v, 0.0f, slot[0]).x;
    if (!(pq > 0.0f)) break;
    const float alpha = rz / pq;
    xv = fmaf(alpha, pv, xv);
    rv = fmaf(-alpha, v, rv);
    const float zv = dinv * rv;
    const float2 s = mg_block_sum2(rv * rv, rv * zv, slot[1]);
    if (s.x <= stop) break;
    const float beta = s.y / rz;
    rz = s.y;
    if (own) ps[ip] = fmaf(beta, pv, zv);
  }
  return xv;
}

// The coarsest solve of one V-cycle by the block CG (when the level has no
// inverse); the result goes to x.
__global__ void __launch_bounds__(kMgCoarseThreads)
k_mg_coarse_cg1(MgL L, const float* __restrict__ b, float* __restrict__ x, int maxit, float rtol) {
  __shared__ float ps[kMgCoarseThreads];
  __shared__ float2 slot[2][kMgCoarseThreads / 32];
  const bool own = (int)threadIdx.x < L.g.N;
  const float xv = mg_cg_block(L, own ? b[threadIdx.x] : 0.0f, maxit, rtol, ps, slot);
  if (own) x[threadIdx.x] = xv;
}

// The inverse of the coarsest operator, once per set-up: block j solves
// A x = e_j by the block CG and writes column j (inv[j N + i] = x_i); the
// level is unpadded, so cell index and array index agree.
constexpr float kMgInvRtol = 1e-4f;
constexpr int kMgInvMaxit = 1000;
__global__ void __launch_bounds__(kMgCoarseThreads)
k_mg_coarse_inv(MgL L, float* __restrict__ inv) {
  __shared__ float ps[kMgCoarseThreads];
  __shared__ float2 slot[2][kMgCoarseThreads / 32];
  const int N = L.g.N;
  const int j = blockIdx.x;
  const float xv = mg_cg_block(L, (int)threadIdx.x == j ? 1.0f : 0.0f, kMgInvMaxit, kMgInvRtol, ps,
                               slot);
  if ((int)threadIdx.x < N) inv[(size_t)j * N + threadIdx.x] = xv;
}

// x = inv b on the coarsest level: thread i takes row i, the columns stream
// (inv[j N + i] for consecutive i is contiguous), b staged in shared memory.
constexpr int kMgApplyThreads = 128;
__global__ void __launch_bounds__(kMgApplyThreads)
k_mg_coarse_apply(const float* __restrict__ inv, const float* __restrict__ b, float* __restrict__ x,
                  int N) {
  __shared__ float bs[kMgCoarseThreads];
  for (int j = threadIdx.x; j < N; j += kMgApplyThreads) bs[j] = b[j];
  __syncthreads();
  const int i = blockIdx.x * kMgApplyThreads + threadIdx.x;
  if (i >= N) return;
  float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
  int j = 0;
  for (; j + 4 <= N; j += 4) {
    a0 = fmaf(inv[(size_t)j * N + i], bs[j], a0);
    a1 = fmaf(inv[(size_t)(j + 1) * N + i], bs[j + 1], a1);
    a2 = fmaf(inv[(size_t)(j + 2) * N + i], bs[j + 2], a2);
    a3 = fmaf(inv[(size_t)(j + 3) * N + i], bs[j + 3], a3);
  }
  for (; j < N; ++j) a0 = fmaf(inv[(size_t)j * N + i], bs[j], a0);
  x[i] = (a0 + a1) + (a2 + a3);
}

// x += alpha d, r -= alpha Ad; rr -> convergence (the preconditioner's
// sweeps follow and give z and beta)
__global__ void k_pcg_upd(PresArr a, const double* __restrict__ d, Geo g, double* part,
                          unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  const double alpha = ctrl->lin[K_ALPHA];
  double rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    a.x[ip] += alpha * d[ip];
    const double r = a.r[ip] - alpha * a.Ad[ip];
    a.r[ip] = r;
    rr += r * r;
  }
  double vals[1] = {block_reduce<0>(rr, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s1 = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin_it += 1;
      ctrl->lin[K_RR] = s1;
      if (s1 <= ctrl->lin[K_TOL2]) ctrl->lin_done = 1;
      if (!isfinite(s1)) { ctrl->lin_break = 1; ctrl->lin_done = 1; }
    }
  }
}

// sum over the cells of x^2 (the embedded Rosenbrock difference) -> K_EMB
__global__ void k_sumsq(const double* __restrict__ x, Geo g, double* part, unsigned* cnt,
                        Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  double s = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    s += x[ip] * x[ip];
  }
  double vals[1] = {block_reduce<0>(s, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double a = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin[K_EMB] = a;
    }
  }
}

// net Darcy inflow through x = 0 and the largest face speed |v| / |sigma|
__global__ void k_pres_post(const double* __restrict__ m, const double* __restrict__ x, Geo g,
                            Phys ph, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  double fin = 0.0, vmax = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double mi = m[ip];
    const double pi = x[ip];
    if (ix == 0) {
      const double v = (ph.ax * mi / (0.5 * ph.hx)) * (ph.head_left - pi);
      fin += v;
      vmax = fmax(vmax, fabs(v) / ph.ax);
    }
    if (ix < g.nx - 1) {
      const double v = harm(ph.ax, 0.5 * ph.hx, mi, m[ip + 1]) * (pi - x[ip + 1]);
      vmax = fmax(vmax, fabs(v) / ph.ax);
    } else {
      const double v = (ph.ax * mi / (0.5 * ph.hx)) * (pi - ph.head_right);
      vmax = fmax(vmax, fabs(v) / ph.ax);
    }
    if (iy < g.ny - 1) {
      const double v = harm(ph.ay, 0.5 * ph.hy, mi, m[ip + g.px]) * (pi - x[ip + g.px]);
      vmax = fmax(vmax, fabs(v) / ph.ay);
    }
    if (g.dim == 3 && iz < g.nz - 1) {
      const double v = harm(ph.az, 0.5 * ph.hz, mi, m[ip + g.plane]) * (pi - x[ip + g.plane]);
      vmax = fmax(vmax, fabs(v) / ph.az);
    }
  }
  double vals[2] = {block_reduce<0>(fin, sh), 0.0};
  vals[1] = block_reduce<2>(vmax, sh);
  if (publish_partials(part, cnt, vals, 2)) {
    const double s0 = gather_partials<0>(part, 0, sh);
    const double s1 = gather_partials<2>(part, 1, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->flux_in = s0;
      ctrl->vmax = s1;
    }
  }
}

// ---------------------------------------------------------------------------
// BiCGSTAB with Jacobi preconditioning for (sigma I - J) x = b, FP64
// ---------------------------------------------------------------------------
struct BiArr {
  double *x, *r, *rh, *p, *v, *y, *s, *z, *t, *dA;
};

__device__ __forceinline__ double stage_apply(const JIn& J, double sigma, const double* __restrict__ x,
                                              int ip, int ix, int iy, int iz, const Geo& g) {
  return sigma * x[ip] - japply_cell(J, x, ip, ix, iy, iz, g);
}

__global__ void k_bicg_init(JIn J, BiArr a, const double* __restrict__ b, double sigma, double tol,
                            Geo g, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  double bb = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double bi = b[ip];
    a.x[ip] = 0.0;
    a.r[ip] = bi;
    a.rh[ip] = bi;
    a.p[ip] = 0.0;
    a.v[ip] = 0.0;
    a.dA[ip] = sigma - J.c[0][ip];
    bb += bi * bi;
  }
  double vals[1] = {block_reduce<0>(bb, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin[K_BB] = s;
      ctrl->lin[K_RHO] = s;
      ctrl->lin[K_RHO_PREV] = 1.0;
      ctrl->lin[K_ALPHA] = 1.0;
      ctrl->lin[K_OMEGA] = 1.0;
      ctrl->lin[K_RR] = s;
      ctrl->lin[K_TOL2] = tol * tol * s;
      ctrl->lin_it = 0;
      ctrl->lin_break = 0;
      ctrl->lin_done = (s == 0.0) ? 1 : 0;
    }
  }
}

// p = r + beta (p - omega v); y = p / diag(A)
__global__ void k_bicg_p(BiArr a, Geo g, Ctrl* ctrl) {
  if (*(volatile int*)&ctrl->lin_done) return;
  const double* L = ctrl->lin;
  const double beta = (L[K_RHO] / L[K_RHO_PREV]) * (L[K_ALPHA] / L[K_OMEGA]);
  const double omega = L[K_OMEGA];
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double pn = a.r[ip] + beta * (a.p[ip] - omega * a.v[ip]);
    a.p[ip] = pn;
    a.y[ip] = pn / a.dA[ip];
  }
}

// v = A y; alpha = rho / (rh, v)
__global__ void k_bicg_v(JIn J, BiArr a, double sigma, Geo g, double* part, unsigned* cnt,
                         Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  double rv = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double v = stage_apply(J, sigma, a.y, ip, ix, iy, iz, g);
    a.v[ip] = v;
    rv += a.rh[ip] * v;
  }
  double vals[1] = {block_reduce<0>(rv, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      if (s == 0.0 || !isfinite(s)) {
        ctrl->lin_break = 1;
        ctrl->lin_done = 1;
      } else {
        ctrl->lin[K_ALPHA] = ctrl->lin[K_RHO] / s;
      }
    }
  }
}

// s = r - alpha v; x += alpha y; z = s / diag(A); ||s||^2 -> early exit
__global__ void k_bicg_s(BiArr a, Geo g, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  const double alpha = ctrl->lin[K_ALPHA];
  double ss = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double s = a.r[ip] - alpha * a.v[ip];
    a.s[ip] = s;
    a.x[ip] += alpha * a.y[ip];
    a.z[ip] = s / a.dA[ip];
    ss += s * s;
  }
  double vals[1] = {block_reduce<0>(ss, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin[K_SS] = s;
      if (s <= ctrl->lin[K_TOL2]) {
        ctrl->lin[K_RR] = s;
        ctrl->lin_it += 1;
        ctrl->lin_done = 1;
      }
    }
  }
}

// t = A z; omega = (t, s) / (t, t); x += omega z; r = s - omega t; new rho
__global__ void k_bicg_t(JIn J, BiArr a, double sigma, Geo g, double* part, unsigned* cnt,
                         Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  double ts = 0.0, tt = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double t = stage_apply(J, sigma, a.z, ip, ix, iy, iz, g);
    a.t[ip] = t;
    ts += t * a.s[ip];
    tt += t * t;
  }
  double vals[2] = {block_reduce<0>(ts, sh), 0.0};
  vals[1] = block_reduce<0>(tt, sh);
  if (publish_partials(part, cnt, vals, 2)) {
    const double s0 = gather_partials<0>(part, 0, sh);
    const double s1 = gather_partials<0>(part, 1, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      if (s1 == 0.0 || !isfinite(s1) || s0 == 0.0) {
        ctrl->lin_break = 1;
        ctrl->lin_done = 1;
      } else {
        ctrl->lin[K_OMEGA] = s0 / s1;
      }
    }
  }
}

__global__ void k_bicg_r(BiArr a, Geo g, double* part, unsigned* cnt, Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  const double omega = ctrl->lin[K_OMEGA];
  double rho = 0.0, rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    a.x[ip] += omega * a.z[ip];
    const double r = a.s[ip] - omega * a.t[ip];
    a.r[ip] = r;
    rho += a.rh[ip] * r;
    rr += r * r;
  }
  double vals[2] = {block_reduce<0>(rho, sh), 0.0};
  vals[1] = block_reduce<0>(rr, sh);
  if (publish_partials(part, cnt, vals, 2)) {
    const double s0 = gather_partials<0>(part, 0, sh);
    const double s1 = gather_partials<0>(part, 1, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin_it += 1;
      ctrl->lin[K_RHO_PREV] = ctrl->lin[K_RHO];
      ctrl->lin[K_RHO] = s0;
      ctrl->lin[K_RR] = s1;
      if (s1 <= ctrl->lin[K_TOL2]) ctrl->lin_done = 1;
      else if (s0 == 0.0 || !isfinite(s1)) {
        ctrl->lin_break = 1;
        ctrl->lin_done = 1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Multigrid preconditioner of the Rosenbrock stage systems (sigma I - J),
// non-symmetric (upwind): the same aggregates and piecewise-constant
// transfers as the pressure multigrid, a Galerkin coarse operator that keeps
// one coupling per direction (a coarse coupling sums the children's
// couplings that leave the aggregate that way, the coarse diagonal sums the
// children's diagonals minus their couplings inside the aggregate), damped
// Jacobi smoothing (weight 0.8, a fixed linear smoother: BiCGSTAB needs a
// fixed preconditioner) and a fixed number of damped Jacobi sweeps on the
// coarsest level.
// ---------------------------------------------------------------------------
struct MgN {
  float *D, *Dinv;
  float* c[6];  // west, east, south, north, bottom, top
  Geo g;
};

__device__ __forceinline__ float smg_offdiag(const MgN& L, const float* __restrict__ x, int ip, int ix,
                                             int iy, int iz) {
  float s = 0.0f;
  if (ix > 0) s = fmaf(L.c[0][ip], x[ip - 1], s);
  if (ix < L.g.nx - 1) s = fmaf(L.c[1][ip], x[ip + 1], s);
  if (iy > 0) s = fmaf(L.c[2][ip], x[ip - L.g.px], s);
  if (iy < L.g.ny - 1) s = fmaf(L.c[3][ip], x[ip + L.g.px], s);
  if (L.g.dim == 3) {
    if (iz > 0) s = fmaf(L.c[4][ip], x[ip - L.g.plane], s);
    if (iz < L.g.nz - 1) s = fmaf(L.c[5][ip], x[ip + L.g.plane], s);
  }
  return s;
}

// level 0: D = sigma - J_ii, c_k = J's coupling k (J >= 0 off the diagonal)
__global__ void k_smg_setup(JIn J, double sigma, MgN L) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < L.g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, L.g, ix, iy, iz, ip);
    const double d = sigma - J.c[0][ip];
    L.D[ip] = (float)d;
    L.Dinv[ip] = (float)(1.0 / d);
    const int nk = L.g.dim == 3 ? 6 : 4;
    for (int q = 0; q < nk; ++q) L.c[q][ip] = (float)J.c[q + 1][ip];
  }
}

__global__ void k_smg_coarsen(MgN f, MgN c) {
  for (int I = blockIdx.x * NT + threadIdx.x; I < c.g.N; I += gridDim.x * NT) {
    int X, Y, Z, IP;
    cell_of(I, c.g, X, Y, Z, IP);
    const int xs = 2 * X, ys = 2 * Y, zs = f.g.dim == 3 ? 2 * Z : 0;
    const int xe = min(xs + 2, f.g.nx), ye = min(ys + 2, f.g.ny);
    const int ze = f.g.dim == 3 ? min(zs + 2, f.g.nz) : 1;
    double d = 0.0, cc[6] = {0, 0, 0, 0, 0, 0};
    for (int iz = zs; iz < ze; ++iz)
      for (int iy = ys; iy < ye; ++iy)
        for (int ix = xs; ix < xe; ++ix) {
          const int ip = ix + f.g.px * (iy + f.g.ny * iz);
          d += f.D[ip];
          // a coupling inside the aggregate moves to the diagonal, one that
          // leaves it to the coarse coupling of that direction
          if (ix > 0) { if (ix - 1 >= xs) d -= f.c[0][ip]; else cc[0] += f.c[0][ip]; }
          if (ix < f.g.nx - 1) { if (ix + 1 < xe) d -= f.c[1][ip]; else cc[1] += f.c[1][ip]; }
          if (iy > 0) { if (iy - 1 >= ys) d -= f.c[2][ip]; else cc[2] += f.c[2][ip]; }
          if (iy < f.g.ny - 1) { if (iy + 1 < ye) d -= f.c[3][ip]; else cc[3] += f.c[3][ip]; }
          if (f.g.dim == 3) {
            if (iz > 0) { if (iz - 1 >= zs) d -= f.c[4][ip]; else cc[4] += f.c[4][ip]; }
            if (iz < f.g.nz - 1) { if (iz + 1 < ze) d -= f.c[5][ip]; else cc[5] += f.c[5][ip]; }
          }
        }
    c.D[IP] = (float)d;
    c.Dinv[IP] = (float)(1.0 / d);
    const int nk = c.g.dim == 3 ? 6 : 4;
    for (int q = 0; q < nk; ++q) c.c[q][IP] = (float)cc[q];
  }
}

// damped Jacobi: xo = xi + w D^-1 (rhs - A xi); xi = NULL means 0
__global__ void k_smg_jacobi(MgN L, const float* __restrict__ rhs, const float* __restrict__ xi,
                             float* __restrict__ xo, float w) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < L.g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, L.g, ix, iy, iz, ip);
    if (!xi) {
      xo[ip] = w * L.Dinv[ip] * rhs[ip];
      continue;
    }
    const float x = xi[ip];
    const float res = rhs[ip] - fmaf(L.D[ip], x, -smg_offdiag(L, xi, ip, ix, iy, iz));
    xo[ip] = fmaf(w * L.Dinv[ip], res, x);
  }
}

// rhs_c = P^T (rhs_f - A_f x_f)
__global__ void k_smg_restrict(MgN f, const float* __restrict__ rhs_f, const float* __restrict__ x_f,
                               MgN c, float* __restrict__ rhs_c) {
  for (int I = blockIdx.x * NT + threadIdx.x; I < c.g.N; I += gridDim.x * NT) {
    int X, Y, Z, IP;
    cell_of(I, c.g, X, Y, Z, IP);
    const int xe = min(2 * X + 2, f.g.nx), ye = min(2 * Y + 2, f.g.ny);
    const int ze = f.g.dim == 3 ? min(2 * Z + 2, f.g.nz) : 1;
    float acc = 0.0f;
    for (int iz = (f.g.dim == 3 ? 2 * Z : 0); iz < ze; ++iz)
      for (int iy = 2 * Y; iy < ye; ++iy)
        for (int ix = 2 * X; ix < xe; ++ix) {
          const int ip = ix + f.g.px * (iy + f.g.ny * iz);
          acc += rhs_f[ip] - fmaf(f.D[ip], x_f[ip], -smg_offdiag(f, x_f, ip, ix, iy, iz));
        }
    rhs_c[IP] = acc;
  }
}

// x_f += P x_c
__global__ void k_smg_prolong(Geo fg, float* __restrict__ x_f, Geo cg, const float* __restrict__ x_c) {
  for (int i = blockIdx.x * NT + threadIdx.x; i < fg.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, fg, ix, iy, iz, ip);
    x_f[ip] += x_c[(ix >> 1) + cg.px * ((iy >> 1) + cg.ny * (fg.dim == 3 ? (iz >> 1) : 0))];
  }
}

// coarsest level (N <= a few thousand): `sweeps` damped Jacobi sweeps from 0
// in one block, ping-ponging between x and tmp; the result ends in x
__global__ void __launch_bounds__(512) k_smg_coarse(MgN L, const float* __restrict__ rhs,
                                                    float* __restrict__ x, float* __restrict__ tmp,
                                                    int sweeps, float w) {
  const int N = L.g.N;
  for (int i = threadIdx.x; i < N; i += 512) x[i] = w * L.Dinv[i] * rhs[i];
  __syncthreads();
  float* a = x;
  float* b = tmp;
  for (int it = 1; it < sweeps; ++it) {
    for (int i = threadIdx.x; i < N; i += 512) {
      int ix, iy, iz, ip;
      cell_of(i, L.g, ix, iy, iz, ip);
      const float res = rhs[ip] - fmaf(L.D[ip], a[ip], -smg_offdiag(L, a, ip, ix, iy, iz));
      b[ip] = fmaf(w * L.Dinv[ip], res, a[ip]);
    }
    __syncthreads();
    float* t = a;
    a = b;
    b = t;
  }
  if (a != x) {
    for (int i = threadIdx.x; i < N; i += 512) x[i] = a[i];
  }
}

// Coarsest level with at most 512 cells: the damped Jacobi sweeps of
// k_smg_coarse with one cell per thread, its coefficients and rhs in registers
// and the iterate in shared memory (two buffers, one block sync per sweep).
__global__ void __launch_bounds__(512) k_smg_coarse1(MgN L, const float* __restrict__ rhs,
                                                     float* __restrict__ x, int sweeps, float w) {
  __shared__ float xs[2][512];
  const int N = L.g.N;
  const bool own = (int)threadIdx.x < N;
  int ix = 0, iy = 0, iz = 0, ip = 0;
  float d = 0.0f, wdi = 0.0f, r = 0.0f, cw = 0.0f, ce = 0.0f, cs = 0.0f, cn = 0.0f, cb = 0.0f,
        ct = 0.0f, xv = 0.0f;
  if (own) {
    cell_of((int)threadIdx.x, L.g, ix, iy, iz, ip);
    d = L.D[ip];
    wdi = w * L.Dinv[ip];
    r = rhs[ip];
    if (ix > 0) cw = L.c[0][ip];
    if (ix < L.g.nx - 1) ce = L.c[1][ip];
    if (iy > 0) cs = L.c[2][ip];
    if (iy < L.g.ny - 1) cn = L.c[3][ip];
    if (L.g.dim == 3) {
      if (iz > 0) cb = L.c[4][ip];
      if (iz < L.g.nz - 1) ct = L.c[5][ip];
    }
    xv = wdi * r;
    xs[0][ip] = xv;
  }
  int cur = 0;
  for (int it = 1; it < sweeps; ++it) {
    __syncthreads();  // xs[cur] complete
    if (own) {
      const float* a = xs[cur];
      float o = 0.0f;
      if (ix > 0) o = fmaf(cw, a[ip - 1], o);
      if (ix < L.g.nx - 1) o = fmaf(ce, a[ip + 1], o);
      if (iy > 0) o = fmaf(cs, a[ip - L.g.px], o);
      if (iy < L.g.ny - 1) o = fmaf(cn, a[ip + L.g.px], o);
      if (L.g.dim == 3) {
        if (iz > 0) o = fmaf(cb, a[ip - L.g.plane], o);
        if (iz < L.g.nz - 1) o = fmaf(ct, a[ip + L.g.plane], o);
      }
      const float res = r - fmaf(d, xv, -o);
      xv = fmaf(wdi, res, xv);
      xs[cur ^ 1][ip] = xv;
    }
    cur ^= 1;
  }
  if (own) x[ip] = xv;
}

// BiCGSTAB with the V-cycle as right preconditioner: the direction and the
// intermediate residual go to the V-cycle in FP32, its output comes back in
// FP64 (y, z of the Jacobi form)
__global__ void k_bicg_p_mg(BiArr a, float* __restrict__ p32, Geo g, Ctrl* ctrl) {
  if (*(volatile int*)&ctrl->lin_done) return;
  const double* L = ctrl->lin;
  const double beta = (L[K_RHO] / L[K_RHO_PREV]) * (L[K_ALPHA] / L[K_OMEGA]);
  const double omega = L[K_OMEGA];
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double pn = a.r[ip] + beta * (a.p[ip] - omega * a.v[ip]);
    a.p[ip] = pn;
    p32[ip] = (float)pn;
  }
}

__global__ void k_bicg_s_mg(BiArr a, float* __restrict__ s32, Geo g, double* part, unsigned* cnt,
                            Ctrl* ctrl) {
  __shared__ double sh[NT / 32];
  if (*(volatile int*)&ctrl->lin_done) return;
  const double alpha = ctrl->lin[K_ALPHA];
  double ss = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    const double s = a.r[ip] - alpha * a.v[ip];
    a.s[ip] = s;
    a.x[ip] += alpha * a.y[ip];
    s32[ip] = (float)s;
    ss += s * s;
  }
  double vals[1] = {block_reduce<0>(ss, sh)};
  if (publish_partials(part, cnt, vals, 1)) {
    const double s = gather_partials<0>(part, 0, sh);
    if (threadIdx.x == 0) {
      *cnt = 0;
      ctrl->lin[K_SS] = s;
      if (s <= ctrl->lin[K_TOL2]) {
        ctrl->lin[K_RR] = s;
        ctrl->lin_it += 1;
        ctrl->lin_done = 1;
      }
    }
  }
}

__global__ void k_f2d(const float* __restrict__ in, double* __restrict__ out, Geo g, Ctrl* ctrl) {
  if (*(volatile int*)&ctrl->lin_done) return;
  for (int i = blockIdx.x * NT + threadIdx.x; i < g.N; i += gridDim.x * NT) {
    int ix, iy, iz, ip;
    cell_of(i, g, ix, iy, iz, ip);
    out[ip] = (double)in[ip];
  }
}


// ---------------------------------------------------------------------------
// host-side argument packing
// ---------------------------------------------------------------------------
Geo geo_of(const erem_ctx* c) {
  Geo g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.nz = c->nz;
  g.px = c->px;
  g.dim = c->dim;
  g.N = (int)c->N;
  g.Np = (int)c->Np;
  g.plane = c->px * c->ny;
  return g;
}

Phys phys_of(const erem_ctx* c) {
  Phys p;
  p.rhoc_f = c->phys.rhoc_f;
  p.rhoc_s = c->phys.rhoc_s;
  p.head_left = c->phys.head_left;
  p.head_right = c->phys.head_right;
  p.T_in = c->phys.T_inflow;
  p.fm = c->phys.fluid_model;
  p.hx = c->hx;
  p.hy = c->hy;
  p.hz = c->hz;
  p.vol = c->vol;
  p.ax = c->ax;
  p.ay = c->ay;
  p.az = c->az;
  return p;
}

FaceIn face_in(const erem_ctx* c) {
  return FaceIn{c->Lx, c->Ly, c->Lz, c->Fx, c->Fy, c->Fz, c->icap, c->LD0, c->F0};
}
JIn jin(const erem_ctx* c) {
  JIn j;
  for (int k = 0; k < 7; ++k) j.c[k] = c->jc[k];
  return j;
}
PresArr pres_arr(const erem_ctx* c) {
  return PresArr{c->kv[0], c->kv[1], c->kv[2], c->kv[3], c->kv[4], c->kv[5],
                 c->kv[6], c->kv[7], c->kv[8], c->kv[9], c->kv[10]};
}
BiArr bi_arr(const erem_ctx* c) {
  return BiArr{c->kv[0], c->kv[1], c->kv[2], c->kv[3], c->kv[4],
               c->kv[5], c->kv[6], c->kv[7], c->kv[8], c->kv[9]};
}

int blocks_cells(const erem_ctx* c) { return grid_for(c, c->N); }
int blocks_padded(const erem_ctx* c) { return grid_for(c, c->Np); }

}  // namespace

int grid_for(const erem_ctx* c, long long items) {
  long long b = (items + NT - 1) / NT;
  if (b < 1) b = 1;
  if (b > c->red_blocks) b = c->red_blocks;
  return (int)b;
}

void launch_pack(const erem_ctx* c, const double* src, double* dst, cudaStream_t s) {
  ++c->launches;
  k_pack<<<blocks_cells(c), NT, 0, s>>>(src, dst, geo_of(c), &c->ctrl->flags);
}

PFix pfix_of(const erem_ctx* c, const PFixHost* f) {
  if (!f || !f->q) return PFix{nullptr, 0, nullptr, 0};
  return PFix{f->q, c->prec == EREM_FP32_BULK ? 1 : 0, c->dd_dev, f->M};
}

void launch_finish(const erem_ctx* c, double* out, const double* base, const double* w,
                   const double* P, double delta, cudaStream_t s, int in_place,
                   const PFixHost* fix) {
  ++c->launches;
  k_finish<<<blocks_cells(c), NT, 0, s>>>(out, base, w, P, pfix_of(c, fix), delta, in_place,
                                          geo_of(c));
}

// the cell mobilities K / mu(T) go to P (the Leja sum, which every step
// initialises after the assembly); T is T^n, or u when visc_u is set
void launch_faces(const erem_ctx* c, cudaStream_t s) {
  FieldIn in{c->lnk, c->phi, c->lam, c->p, c->Tn};
  FaceOut o{c->Lx, c->Ly, c->Lz, c->Fx, c->Fy, c->Fz, c->icap, c->LD0, c->F0};
  c->launches += 2;
  k_mobility<<<blocks_cells(c), NT, 0, s>>>(c->lnk, c->visc_u ? c->u : c->Tn, c->P, geo_of(c),
                                            phys_of(c), 1, 1, &c->ctrl->flags);
  k_faces<<<blocks_cells(c), NT, 0, s>>>(in, c->P, o, geo_of(c), phys_of(c), &c->ctrl->flags);
}

void launch_cellJ(const erem_ctx* c, cudaStream_t s) {
  JOut o;
  for (int k = 0; k < 7; ++k) o.c[k] = c->jc[k];
  o.b0 = c->b0;
  ++c->launches;
  k_cellJ<<<blocks_cells(c), NT, 0, s>>>(face_in(c), c->Tn, o, geo_of(c), phys_of(c), c->red_part,
                                         c->red_cnt, c->ctrl);
}

void launch_scale_jl(const erem_ctx* c, double sc, cudaStream_t s) {
  JOut jc;
  for (int k = 0; k < 7; ++k) jc.c[k] = c->jc[k];
  jc.b0 = nullptr;
  const int nc = c->dim == 3 ? 7 : 5;
  ++c->launches;
  if (c->prec == EREM_FP32_BULK)
    k_scale_jl<float, 128><<<blocks_padded(c), NT, 0, s>>>(jc, (float*)c->jl_all, sc, (int)c->Np, nc,
                                                           c->jrow, c->jl_nodiag ? 1 : 0, c->jl_r0,
                                                           c->px);
  else
    k_scale_jl<double, 64><<<blocks_padded(c), NT, 0, s>>>(jc, (double*)c->jl_all, sc, (int)c->Np, nc,
                                                           nullptr, 0, nullptr, c->px);
}

// Pointers of the interleaved Leja coefficients for kernels of vector width
// VEC (tile of 32 VEC cells).
template <typename Tq, int VEC>
LejaCoef<Tq> leja_coef(const erem_ctx* c) {
  LejaCoef<Tq> cf;
  const int nc = c->dim == 3 ? 7 : 5;
  const Tq* base = (const Tq*)c->jl_all;
  if (c->jl_nodiag) {  // couplings only: c[1..] from the start of the tile
    cf.nc = nc - 1;
    cf.c[0] = nullptr;
    for (int k = 1; k < 7; ++k) cf.c[k] = base + (k < nc ? (k - 1) * 32 * VEC : 0);
    cf.r0 = (const Tq*)c->jl_r0;
  } else {
    cf.nc = nc;
    for (int k = 0; k < 7; ++k) cf.c[k] = base + (k < nc ? k * 32 * VEC : 0);
    cf.r0 = nullptr;
  }
  return cf;
}

void launch_rhs(const erem_ctx* c, const double* T, double* G, int set_yinf, cudaStream_t s) {
  ++c->launches;
  k_rhs<<<blocks_cells(c), NT, 0, s>>>(face_in(c), T, G, geo_of(c), phys_of(c), set_yinf,
                                       c->red_part, c->red_cnt, c->ctrl);
}

void launch_sumsq(const erem_ctx* c, const double* x, cudaStream_t s) {
  ++c->launches;
  k_sumsq<<<blocks_cells(c), NT, 0, s>>>(x, geo_of(c), c->red_part, c->red_cnt, c->ctrl);
}

void launch_inflow_forced(const erem_ctx* c, double T_in, double rate, double* b, double* w,
                          cudaStream_t s) {
  ++c->launches;
  const int nf = c->ny * c->nz;
  k_inflow_forced<<<std::max(1, std::min(c->red_blocks, (nf + NT - 1) / NT)), NT, 0, s>>>(
      c->icap, c->LD0, c->F0, T_in, rate, b, w, geo_of(c));
}

void launch_japply_add(const erem_ctx* c, const double* x, const double* v, double* out,
                       cudaStream_t s) {
  ++c->launches;
  k_japply_add<<<blocks_cells(c), NT, 0, s>>>(jin(c), x, v, out, geo_of(c));
}

void launch_leja_init(const erem_ctx* c, const double* u, const StopParams& sp, cudaStream_t s) {
  ++c->launches;
  c->p0 = u;
  if (c->prec == EREM_FP32_BULK)
    k_leja_init<float><<<blocks_padded(c), NT, 0, s>>>(u, (float*)c->q[0], (int)c->Np, sp, c->ctrl);
  else
    k_leja_init<double><<<blocks_padded(c), NT, 0, s>>>(u, (double*)c->q[0], (int)c->Np, sp, c->ctrl);
}

void launch_step_init(const erem_ctx* c, const double* T, const StopParams& sp, cudaStream_t s,
                      double* Tcopy) {
  ++c->launches;
  c->p0 = c->vrhs;
  if (c->px == c->nx) {  // unpadded rows: four cells per thread
    const int nb = std::min(grid_for(c, c->Np / 4), c->term_grid);
    const Geo g = geo_of(c);
    if (c->prec == EREM_FP32_BULK) {  // G in the difference form on the FP32 pipe
      const LejaCoef<float> cf = leja_coef<float, 4>(c);
      const float jinv = (float)(1.0 / c->jl_sc);
      if (c->dim == 3 && c->jl_nodiag)
        k_step_init_df<3, true><<<nb, NT, 0, s>>>(cf, jinv, c->jrow, c->b0, T, Tcopy, c->vrhs,
                                                  (float*)c->q[0], g, sp, c->red_part, c->red_cnt,
                                                  c->ctrl);
      else if (c->dim == 3)
        k_step_init_df<3><<<nb, NT, 0, s>>>(cf, jinv, c->jrow, c->b0, T, Tcopy, c->vrhs,
                                            (float*)c->q[0], g, sp, c->red_part, c->red_cnt, c->ctrl);
      else if (c->jl_nodiag)
        k_step_init_df<2, true><<<nb, NT, 0, s>>>(cf, jinv, c->jrow, c->b0, T, Tcopy, c->vrhs,
                                                  (float*)c->q[0], g, sp, c->red_part, c->red_cnt,
                                                  c->ctrl);
      else
        k_step_init_df<2><<<nb, NT, 0, s>>>(cf, jinv, c->jrow, c->b0, T, Tcopy, c->vrhs,
                                            (float*)c->q[0], g, sp, c->red_part, c->red_cnt, c->ctrl);
    } else {
      if (c->dim == 3)
        k_step_init_vec<double, 3><<<nb, NT, 0, s>>>(jin(c), c->b0, T, Tcopy, c->vrhs, (double*)c->q[0],
                                                     g, sp, c->red_part, c->red_cnt, c->ctrl);
      else
        k_step_init_vec<double, 2><<<nb, NT, 0, s>>>(jin(c), c->b0, T, Tcopy, c->vrhs, (double*)c->q[0],
                                                     g, sp, c->red_part, c->red_cnt, c->ctrl);
    }
    return;
  }
  if (c->prec == EREM_FP32_BULK)
    k_step_init<float><<<blocks_cells(c), NT, 0, s>>>(jin(c), c->b0, T, Tcopy, c->vrhs,
                                                      (float*)c->q[0], geo_of(c), sp,
                                                      c->red_part, c->red_cnt, c->ctrl);
  else
    k_step_init<double><<<blocks_cells(c), NT, 0, s>>>(jin(c), c->b0, T, Tcopy, c->vrhs,
                                                       (double*)c->q[0], geo_of(c), sp,
                                                       c->red_part, c->red_cnt, c->ctrl);
}

// Resident blocks per SM of the one-term kernel of this context's precision
// and dimension (its grid-stride grid is one full wave of them; the three
// running-sum modes use the same registers or fewer than the first).
int leja_term_blocks_per_sm(const erem_ctx* c) {
  int n = 0;
  cudaError_t e;
  if (c->prec == EREM_FP32_BULK)
    e = c->dim == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_leja_term<float, 4, 3, 1>, NT, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_leja_term<float, 4, 2, 1>, NT, 0);
  else
    e = c->dim == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_leja_term<double, 2, 3, 1>, NT, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_leja_term<double, 2, 2, 1>, NT, 0);
  if (e != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 4;
  }
  return n;
}

template <typename Tq, int VEC, int DIM>
void term_launch(const erem_ctx* c, int m, const Tq* qi, Tq* qo, double cg, cudaStream_t s) {
  const LejaCoef<Tq> cf = leja_coef<Tq, VEC>(c);
  const Geo g = geo_of(c);
  const int nb = std::min(grid_for(c, c->Np / VEC), c->term_grid);
  ++c->launches;
  // every term after the first may start as a programmatic dependent of the
  // one before it (the grid is one resident wave, so all of the previous
  // grid's blocks have started when it is scheduled)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = (c->pdl && m > 1) ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (sizeof(Tq) == 4) {
    if (c->jl_nodiag) {  // the Leja copy holds the couplings only
      if (m == 1)
        cudaLaunchKernelEx(&cfg, k_leja_term1<Tq, VEC, DIM, true>, qi, qo, c->P, c->p0, cf, g,
                           (const double*)c->xi_dev, (const double*)c->dd_dev, cg, c->red_part,
                           c->red_cnt, c->ctrl);
      else if (m & 1)
        cudaLaunchKernelEx(&cfg, k_leja_term<Tq, VEC, DIM, 1, true>, qi, qo, c->P, cf, g,
                           (const double*)c->xi_dev, (const double*)c->dd_dev, cg, m, c->red_part,
                           c->red_cnt, c->ctrl);
      else
        cudaLaunchKernelEx(&cfg, k_leja_term<Tq, VEC, DIM, 0, true>, qi, qo, c->P, cf, g,
                           (const double*)c->xi_dev, (const double*)c->dd_dev, cg, m, c->red_part,
                           c->red_cnt, c->ctrl);
      return;
    }
  }
  if (m == 1)
    cudaLaunchKernelEx(&cfg, k_leja_term1<Tq, VEC, DIM>, qi, qo, c->P, c->p0, cf, g,
                       (const double*)c->xi_dev, (const double*)c->dd_dev, cg, c->red_part,
                       c->red_cnt, c->ctrl);
  else if (m & 1)
    cudaLaunchKernelEx(&cfg, k_leja_term<Tq, VEC, DIM, 1>, qi, qo, c->P, cf, g,
                       (const double*)c->xi_dev, (const double*)c->dd_dev, cg, m, c->red_part,
                       c->red_cnt, c->ctrl);
  else
    cudaLaunchKernelEx(&cfg, k_leja_term<Tq, VEC, DIM, 0>, qi, qo, c->P, cf, g,
                       (const double*)c->xi_dev, (const double*)c->dd_dev, cg, m, c->red_part,
                       c->red_cnt, c->ctrl);
}

template <typename Tq, int VEC, int DIM>
void term_launch_lag(const erem_ctx* c, int m, const Tq* qi, Tq* qo, double cg, cudaStream_t s) {
  const LejaCoef<Tq> cf = leja_coef<Tq, VEC>(c);
  const Geo g = geo_of(c);
  const int nb = std::min(grid_for(c, c->Np / VEC) + 1, c->term_grid);
  ++c->launches;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(nb, 2));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = (c->pdl && m > 1) ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (sizeof(Tq) == 4) {
    if (c->jl_nodiag) {
      cudaLaunchKernelEx(&cfg, k_leja_term_lag<Tq, VEC, DIM, true>, qi, qo, c->P, c->p0, cf, g,
                         (const double*)c->xi_dev, (const double*)c->dd_dev, cg, m, c->red_part,
                         c->ctrl);
      return;
    }
  }
  cudaLaunchKernelEx(&cfg, k_leja_term_lag<Tq, VEC, DIM, false>, qi, qo, c->P, c->p0, cf, g,
                     (const double*)c->xi_dev, (const double*)c->dd_dev, cg, m, c->red_part,
                     c->ctrl);
}

void launch_leja_term_lag(const erem_ctx* c, int m, int qin, double cg, cudaStream_t s) {
  const void* qi = c->q[qin];
  void* qo = c->q[qin ^ 1];
  if (c->prec == EREM_FP32_BULK) {
    if (c->dim == 3) term_launch_lag<float, 4, 3>(c, m, (const float*)qi, (float*)qo, cg, s);
    else term_launch_lag<float, 4, 2>(c, m, (const float*)qi, (float*)qo, cg, s);
  } else {
    if (c->dim == 3) term_launch_lag<double, 2, 3>(c, m, (const double*)qi, (double*)qo, cg, s);
    else term_launch_lag<double, 2, 2>(c, m, (const double*)qi, (double*)qo, cg, s);
  }
}

// One Leja term with explicit input/output vectors (the context's ping-pong
// pair, or the adjoint's store of Newton vectors).  The running sum is
// updated at odd m (see k_leja_term); m = 1 starts it from c->p0, the FP64
// vector the last Leja start kernel made q_0 from.
void launch_leja_term_ptr(const erem_ctx* c, int m, const void* qi, void* qo, double cg,
                          cudaStream_t s) {
  if (c->prec == EREM_FP32_BULK) {
    if (c->dim == 3) term_launch<float, 4, 3>(c, m, (const float*)qi, (float*)qo, cg, s);
    else term_launch<float, 4, 2>(c, m, (const float*)qi, (float*)qo, cg, s);
  } else {
    if (c->dim == 3) term_launch<double, 2, 3>(c, m, (const double*)qi, (double*)qo, cg, s);
    else term_launch<double, 2, 2>(c, m, (const double*)qi, (double*)qo, cg, s);
  }
}

void launch_leja_term(const erem_ctx* c, int m, int qin, double cg, cudaStream_t s) {
  launch_leja_term_ptr(c, m, c->q[qin], c->q[qin ^ 1], cg, s);
}

void launch_pfix(const erem_ctx* c, const void* q, int M, cudaStream_t s) {
  ++c->launches;
  if (c->prec == EREM_FP32_BULK)
    k_pfix<float><<<blocks_padded(c), NT, 0, s>>>(c->P, (const float*)q, c->dd_dev, M, (int)c->Np);
  else
    k_pfix<double><<<blocks_padded(c), NT, 0, s>>>(c->P, (const double*)q, c->dd_dev, M, (int)c->Np);
}

void launch_axpy(const erem_ctx* c, double* w, const double* P, double delta, int first,
                 cudaStream_t s, const PFixHost* fix) {
  ++c->launches;
  k_axpy<<<blocks_padded(c), NT, 0, s>>>(w, P, pfix_of(c, fix), delta, first, (int)c->Np);
}

void launch_lincomb(const erem_ctx* c, double* out, double a, const double* x, double b,
                    const double* y, cudaStream_t s) {
  ++c->launches;
  k_lincomb<<<blocks_padded(c), NT, 0, s>>>(out, a, x, b, y, (int)c->Np);
}

// the cell mobilities go to kv[1] (the CG residual, which k_cg_init writes
// afterwards; free again once the CG has converged)
void launch_pres_faces(const erem_ctx* c, const double* lnk, const double* T, cudaStream_t s) {
  const PresArr a = pres_arr(c);
  c->launches += 2;
  k_mobility<<<blocks_cells(c), NT, 0, s>>>(lnk, T, a.r, geo_of(c), phys_of(c), 0, 0,
                                            &c->ctrl->flags);
  k_pres_faces<<<blocks_cells(c), NT, 0, s>>>(a.r, a, geo_of(c), phys_of(c));
}

void launch_cg_init(const erem_ctx* c, double tol, cudaStream_t s) {
  ++c->launches;
  k_cg_init<<<blocks_cells(c), NT, 0, s>>>(pres_arr(c), geo_of(c), tol, c->red_part, c->red_cnt,
                                           c->ctrl);
}

void launch_cg_iter(const erem_ctx* c, int k, cudaStream_t s) {
  PresArr a = pres_arr(c);
  const double* dold = (k & 1) ? a.d1 : a.d0;
  double* dnew = (k & 1) ? a.d0 : a.d1;
  const int nb = blocks_cells(c);
  ++c->launches;
  k_cg_dir<double><<<nb, NT, 0, s>>>(a, a.z, dold, dnew, geo_of(c), c->red_part, c->red_cnt,
                                     c->ctrl);
  ++c->launches;
  k_cg_upd<<<nb, NT, 0, s>>>(a, dnew, geo_of(c), c->red_part, c->red_cnt, c->ctrl);
}

namespace {
PcArr pc_arr(const erem_ctx* c) {
  return PcArr{c->pc[0], c->pc[1], c->pc[2], c->pc[3], c->pc[4]};
}
}  // namespace

// FP32 coefficients, and A d = 0 so that the first (z, A d) is defined
void launch_pc_setup(const erem_ctx* c, cudaStream_t s) {
  ++c->launches;
  k_pc_setup<<<blocks_cells(c), NT, 0, s>>>(pres_arr(c), pc_arr(c), c->pc_diag, geo_of(c));
  cudaMemsetAsync(pres_arr(c).Ad, 0, sizeof(double) * c->Np, s);
}

namespace {
Geo geo_level(int dim, int nx, int ny, int nz) {
  Geo g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.px = nx;
  g.dim = dim;
  g.N = nx * ny * nz;
  g.Np = g.N;
  g.plane = nx * ny;
  return g;
}
MgL mg_fine(const erem_ctx* c) {
  return MgL{c->pc_diag, c->pc[0], c->pc[1], c->pc[2], c->pc[3], geo_of(c)};
}
MgL mg_level(const erem_ctx* c, int l) {
  const MgLevel& m = c->mg[l];
  return MgL{m.diag, m.dinv, m.Ux, m.Uy, m.Uz, geo_level(c->dim, m.nx, m.ny, m.nz)};
}
}  // namespace

// Galerkin operators of the coarse levels, after launch_pc_setup, and the
// inverse of the coarsest one.
void launch_mg_setup(const erem_ctx* c, cudaStream_t s) {
  for (size_t l = 0; l < c->mg.size(); ++l) {
    const MgL f = l == 0 ? mg_fine(c) : mg_level(c, (int)l - 1);
    const MgL cl = mg_level(c, (int)l);
    ++c->launches;
    k_mg_coarsen<<<grid_for(c, cl.g.N), NT, 0, s>>>(f, cl);
  }
  const MgLevel& last = c->mg.back();
  const MgL Lc = mg_level(c, (int)c->mg.size() - 1);
  if (last.inv && Lc.g.N <= kMgCoarseThreads && Lc.g.Np == Lc.g.N) {
    ++c->launches;
    k_mg_coarse_inv<<<Lc.g.N, kMgCoarseThreads, 0, s>>>(Lc, last.inv);
  }
}

namespace {
// smoothing on coarse level l: deg Chebyshev-Jacobi steps from x = 0 (pre) or
// from x[*cur] (post); returns the buffer index holding the result
int mg_smooth(const erem_ctx* c, int l, const PcPoly& poly, int cur, bool from_zero, cudaStream_t s) {
  const MgL L = mg_level(c, l);
  const MgLevel& m = c->mg[l];
  const int nb = grid_for(c, L.g.N);
  int prev = -1;
  for (int j = 0; j < poly.deg; ++j) {
    const int nxt = from_zero && j == 0 ? 0 : (cur + 1) % 3;
    const float* xc = (from_zero && j == 0) ? nullptr : m.x[cur];
    const float* xp = prev >= 0 ? m.x[prev] : nullptr;
    ++c->launches;
    k_mg_sweep<<<nb, NT, 0, s>>>(L, m.rhs, xp, xc, m.x[nxt], (float)poly.c1[j], (float)poly.c2[j]);
    prev = (from_zero && j == 0) ? -1 : cur;
    cur = nxt;
  }
  return cur;
}

// V-cycle below the fine level: the correction of coarse level l for its rhs
// (already restricted); returns the buffer index holding it
int mg_cycle(const erem_ctx* c, int l, const PcPoly& poly, float omega, cudaStream_t s) {
  const MgLevel& m = c->mg[l];
  const MgL L = mg_level(c, l);
  if (l + 1 == (int)c->mg.size()) {
    ++c->launches;
    if (m.inv && L.g.N <= kMgCoarseThreads && L.g.Np == L.g.N)
      k_mg_coarse_apply<<<(L.g.N + kMgApplyThreads - 1) / kMgApplyThreads, kMgApplyThreads, 0, s>>>(
          m.inv, m.rhs, m.x[0], L.g.N);
    else if (L.g.N <= kMgCoarseThreads && L.g.Np == L.g.N)
      k_mg_coarse_cg1<<<1, kMgCoarseThreads, 0, s>>>(L, m.rhs, m.x[0], 400, kMgCoarseRtol);
    else
      k_mg_coarse_cg<<<1, kMgCoarseThreads, 0, s>>>(L, m.rhs, m.x[0], m.x[1], m.x[2], m.x[3], 400,
                                                     kMgCoarseRtol);
    return 0;
  }
  int cur = mg_smooth(c, l, poly, 0, true, s);
  const MgL Lc = mg_level(c, l + 1);
  ++c->launches;
  k_mg_restrict<<<grid_for(c, Lc.g.N), NT, 0, s>>>(L, m.rhs, m.x[cur], Lc, c->mg[l + 1].rhs);
  const int ec = mg_cycle(c, l + 1, poly, omega, s);
  ++c->launches;
  k_mg_prolong<<<grid_for(c, L.g.N), NT, 0, s>>>(L, m.x[cur], Lc, c->mg[l + 1].x[ec], omega);
  return mg_smooth(c, l, poly, cur, false, s);
}
}  // namespace

// The preconditioner.  Chebyshev (pc_deg >= 2): deg sweeps, z ends in
// pc[5 + (deg - 1) % 3].  Multigrid (pc_deg = 0): pre-smoothing on the fine
// level from 0, restriction, the coarse V-cycle, prolongation of its
// correction and post-smoothing, the last sweep with the two dots.
const float* launch_pc_apply(const erem_ctx* c, const PcPoly& poly, cudaStream_t s) {
  const PresArr a = pres_arr(c);
  const PcArr p = pc_arr(c);
  const int nb = grid_for(c, c->Np / 4);
  float* const* zb = &c->pc[5];
  if (c->pc_deg == 0) {
    const int nu = poly.deg;
    // pre-smoothing: sweep 0 converts r to FP32 and starts from z = 0
    for (int j = 0; j < nu; ++j) {
      float* zn = zb[j % 3];
      const float* zc = j >= 1 ? zb[(j + 2) % 3] : nullptr;
      const float* zp = j >= 2 ? zb[(j + 1) % 3] : nullptr;
      ++c->launches;
      if (j == 0)
        k_pc_sweep<true, false><<<nb, NT, 0, s>>>(a, p, zp, zc, zn, (float)poly.c1[j],
                                                   (float)poly.c2[j], geo_of(c), c->red_part,
                                                   c->red_cnt, c->ctrl);
      else
        k_pc_sweep<false, false><<<nb, NT, 0, s>>>(a, p, zp, zc, zn, (float)poly.c1[j],
                                                    (float)poly.c2[j], geo_of(c), c->red_part,
                                                    c->red_cnt, c->ctrl);
    }
    const int x0 = (nu - 1) % 3;
    const MgL F = mg_fine(c);
    const MgL C1 = mg_level(c, 0);
    ++c->launches;
    k_mg_restrict<<<grid_for(c, C1.g.N), NT, 0, s>>>(F, p.r, zb[x0], C1, c->mg[0].rhs);
    const int ec = mg_cycle(c, 0, poly, c->mg_omega, s);
    ++c->launches;
    k_mg_prolong<<<blocks_cells(c), NT, 0, s>>>(F, zb[x0], C1, c->mg[0].x[ec], c->mg_omega);
    // post-smoothing from the corrected z
    for (int j = 0; j < nu; ++j) {
      const int cur = (x0 + j) % 3;
      float* zn = zb[(cur + 1) % 3];
      const float* zp = j >= 1 ? zb[(cur + 2) % 3] : nullptr;
      ++c->launches;
      if (j == nu - 1)
        k_pc_sweep<false, true><<<nb, NT, 0, s>>>(a, p, zp, zb[cur], zn, (float)poly.c1[j],
                                                   (float)poly.c2[j], geo_of(c), c->red_part,
                                                   c->red_cnt, c->ctrl);
      else
        k_pc_sweep<false, false><<<nb, NT, 0, s>>>(a, p, zp, zb[cur], zn, (float)poly.c1[j],
                                                    (float)poly.c2[j], geo_of(c), c->red_part,
                                                    c->red_cnt, c->ctrl);
    }
    return zb[(x0 + nu) % 3];
  }
  for (int j = 0; j < poly.deg; ++j) {
    const bool last = j == poly.deg - 1;
    float* zn = zb[j % 3];
    const float* zc = zb[(j + 2) % 3];
    const float* zp = j >= 2 ? zb[(j + 1) % 3] : nullptr;
    const float c1 = (float)poly.c1[j], c2 = (float)poly.c2[j];
    ++c->launches;
    if (j == 0 && last)
      k_pc_sweep<true, true><<<nb, NT, 0, s>>>(a, p, zp, zc, zn, c1, c2, geo_of(c), c->red_part,
                                                c->red_cnt, c->ctrl);
    else if (j == 0)
      k_pc_sweep<true, false><<<nb, NT, 0, s>>>(a, p, zp, zc, zn, c1, c2, geo_of(c), c->red_part,
                                                 c->red_cnt, c->ctrl);
    else if (last)
      k_pc_sweep<false, true><<<nb, NT, 0, s>>>(a, p, zp, zc, zn, c1, c2, geo_of(c), c->red_part,
                                                 c->red_cnt, c->ctrl);
    else
      k_pc_sweep<false, false><<<nb, NT, 0, s>>>(a, p, zp, zc, zn, c1, c2, geo_of(c), c->red_part,
                                                  c->red_cnt, c->ctrl);
  }
  return zb[(poly.deg - 1) % 3];
}

void launch_pcg_iter(const erem_ctx* c, const PcPoly& poly, const float* z, int k, cudaStream_t s) {
  PresArr a = pres_arr(c);
  const double* dold = (k & 1) ? a.d1 : a.d0;
  double* dnew = (k & 1) ? a.d0 : a.d1;
  const int nb = blocks_cells(c);
  ++c->launches;
  k_cg_dir<float><<<nb, NT, 0, s>>>(a, z, dold, dnew, geo_of(c), c->red_part, c->red_cnt, c->ctrl);
  ++c->launches;
  k_pcg_upd<<<nb, NT, 0, s>>>(a, dnew, geo_of(c), c->red_part, c->red_cnt, c->ctrl);
  // the next z lands in the same buffer (the preconditioner's sweep count is fixed)
  (void)launch_pc_apply(c, poly, s);
}

void launch_pres_post(const erem_ctx* c, const double* lnk, const double* T, cudaStream_t s) {
  const PresArr a = pres_arr(c);
  c->launches += 2;
  k_mobility<<<blocks_cells(c), NT, 0, s>>>(lnk, T, a.r, geo_of(c), phys_of(c), 1, 0, nullptr);
  k_pres_post<<<blocks_cells(c), NT, 0, s>>>(a.r, a.x, geo_of(c), phys_of(c), c->red_part,
                                             c->red_cnt, c->ctrl);
}

void launch_bicg_init(const erem_ctx* c, const double* b, double sigma, double tol,
                      cudaStream_t s) {
  ++c->launches;
  k_bicg_init<<<blocks_cells(c), NT, 0, s>>>(jin(c), bi_arr(c), b, sigma, tol, geo_of(c),
                                             c->red_part, c->red_cnt, c->ctrl);
}

namespace {
MgN smg_level(const erem_ctx* c, int l) {
  const SmgLevel& m = c->smg[l];
  MgN L;
  L.D = m.D;
  L.Dinv = m.Dinv;
  for (int q = 0; q < 6; ++q) L.c[q] = m.c[q];
  L.g = l == 0 ? geo_of(c) : geo_level(c->dim, m.nx, m.ny, m.nz);
  return L;
}

constexpr float kSmgW = 0.8f;       // damped Jacobi weight
constexpr int kSmgCoarseSweeps = 40;

// V-cycle on level l for smg[l].rhs: two damped Jacobi sweeps, restriction,
// the coarser correction, prolongation, two sweeps; returns the index of the
// buffer that holds the result
int smg_cycle(const erem_ctx* c, int l, cudaStream_t s) {
  const SmgLevel& m = c->smg[l];
  const MgN L = smg_level(c, l);
  if (l + 1 == (int)c->smg.size()) {
    ++c->launches;
    if (L.g.Np <= 512)
      k_smg_coarse1<<<1, 512, 0, s>>>(L, m.rhs, m.x[0], kSmgCoarseSweeps, kSmgW);
    else
      k_smg_coarse<<<1, 512, 0, s>>>(L, m.rhs, m.x[0], m.x[1], kSmgCoarseSweeps, kSmgW);
    return 0;
  }
  const int nb = grid_for(c, L.g.N);
  c->launches += 2;
  k_smg_jacobi<<<nb, NT, 0, s>>>(L, m.rhs, nullptr, m.x[0], kSmgW);
  k_smg_jacobi<<<nb, NT, 0, s>>>(L, m.rhs, m.x[0], m.x[1], kSmgW);
  const MgN Lc = smg_level(c, l + 1);
  ++c->launches;
  k_smg_restrict<<<grid_for(c, Lc.g.N), NT, 0, s>>>(L, m.rhs, m.x[1], Lc, c->smg[l + 1].rhs);
  const int ec = smg_cycle(c, l + 1, s);
  c->launches += 3;
  k_smg_prolong<<<nb, NT, 0, s>>>(L.g, m.x[1], Lc.g, c->smg[l + 1].x[ec]);
  k_smg_jacobi<<<nb, NT, 0, s>>>(L, m.rhs, m.x[1], m.x[2], kSmgW);
  k_smg_jacobi<<<nb, NT, 0, s>>>(L, m.rhs, m.x[2], m.x[0], kSmgW);
  return 0;
}
}  // namespace

void launch_smg_setup(const erem_ctx* c, double sigma, cudaStream_t s) {
  const MgN L0 = smg_level(c, 0);
  ++c->launches;
  k_smg_setup<<<blocks_cells(c), NT, 0, s>>>(jin(c), sigma, L0);
  for (size_t l = 1; l < c->smg.size(); ++l) {
    const MgN cl = smg_level(c, (int)l);
    ++c->launches;
    k_smg_coarsen<<<grid_for(c, cl.g.N), NT, 0, s>>>(smg_level(c, (int)l - 1), cl);
  }
}

void launch_bicg_iter_mg(const erem_ctx* c, double sigma, cudaStream_t s) {
  const int nb = blocks_cells(c);
  const Geo g = geo_of(c);
  BiArr a = bi_arr(c);
  float* rhs0 = c->smg[0].rhs;
  ++c->launches;
  k_bicg_p_mg<<<nb, NT, 0, s>>>(a, rhs0, g, c->ctrl);
  int e = smg_cycle(c, 0, s);
  ++c->launches;
  k_f2d<<<nb, NT, 0, s>>>(c->smg[0].x[e], a.y, g, c->ctrl);
  ++c->launches;
  k_bicg_v<<<nb, NT, 0, s>>>(jin(c), a, sigma, g, c->red_part, c->red_cnt, c->ctrl);
  ++c->launches;
  k_bicg_s_mg<<<nb, NT, 0, s>>>(a, rhs0, g, c->red_part, c->red_cnt, c->ctrl);
  e = smg_cycle(c, 0, s);
  ++c->launches;
  k_f2d<<<nb, NT, 0, s>>>(c->smg[0].x[e], a.z, g, c->ctrl);
  ++c->launches;
  k_bicg_t<<<nb, NT, 0, s>>>(jin(c), a, sigma, g, c->red_part, c->red_cnt, c->ctrl);
  ++c->launches;
  k_bicg_r<<<nb, NT, 0, s>>>(a, g, c->red_part, c->red_cnt, c->ctrl);
}

void launch_bicg_iter(const erem_ctx* c, double sigma, cudaStream_t s) {
  const int nb = blocks_cells(c);
  const Geo g = geo_of(c);
  BiArr a = bi_arr(c);
  ++c->launches;
  k_bicg_p<<<nb, NT, 0, s>>>(a, g, c->ctrl);
  ++c->launches;
  k_bicg_v<<<nb, NT, 0, s>>>(jin(c), a, sigma, g, c->red_part, c->red_cnt, c->ctrl);
  ++c->launches;
  k_bicg_s<<<nb, NT, 0, s>>>(a, g, c->red_part, c->red_cnt, c->ctrl);
  ++c->launches;
  k_bicg_t<<<nb, NT, 0, s>>>(jin(c), a, sigma, g, c->red_part, c->red_cnt, c->ctrl);
  ++c->launches;
  k_bicg_r<<<nb, NT, 0, s>>>(a, g, c->red_part, c->red_cnt, c->ctrl);
}



// ---------------------------------------------------------------------------
// batched ensemble
// ---------------------------------------------------------------------------
void launch_unpack(const erem_ctx* c, const double* src, double* dst, cudaStream_t s) {
  ++c->launches;
  k_unpack<<<blocks_cells(c), NT, 0, s>>>(src, dst, geo_of(c));
}


// ---------------------------------------------------------------------------
// Krylov
// ---------------------------------------------------------------------------
// the direction of the next Krylov pass: alternating
static int kr_dir(const erem_ctx* c) { return (int)(c->kr_pass++ & 1u); }

void launch_kr_norm0(const erem_ctx* c, const double* r, double btol, cudaStream_t s) {
  ++c->launches;
  k_kr_norm0<<<blocks_padded(c), NT, 0, s>>>(r, geo_of(c), btol, c->red_part, c->red_cnt, c->kr_dev,
                                             kr_dir(c));
}

void launch_kr_matvec(const erem_ctx* c, const double* w_in, double* v_out, double* w_out, int j,
                      int mode, cudaStream_t s) {
  ++c->launches;
  k_kr_matvec<<<blocks_padded(c), NT, 0, s>>>(jin(c), w_in, v_out, w_out, c->kr_V[0], geo_of(c), j,
                                              mode, c->red_part, c->red_cnt, c->kr_dev, kr_dir(c));
}

void launch_kr_orth(const erem_ctx* c, double* w, const double* vprev, const double* vi, int i,
                    int j, int last, cudaStream_t s) {
  ++c->launches;
  k_kr_orth<<<blocks_padded(c), NT, 0, s>>>(w, vprev, vi, geo_of(c), i, j, last, c->red_part,
                                            c->red_cnt, c->kr_dev, kr_dir(c));
}

void launch_kr_combine(const erem_ctx* c, double* y, const KrComb& cb, cudaStream_t s) {
  ++c->launches;
  k_kr_combine<<<blocks_padded(c), NT, 0, s>>>(y, cb, (int)c->Np, kr_dir(c));
}


// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
AdjFaces adj_faces(const erem_ctx* c) {
  return AdjFaces{c->Fx, c->Fy, c->Fz, c->F0, c->icap, c->adj_gx, c->adj_gy, c->adj_gz, c->adj_g0};
}

void launch_adj_scale_jlT(const erem_ctx* c, double sc, cudaStream_t s) {
  JOut jc;
  for (int k = 0; k < 7; ++k) jc.c[k] = c->jc[k];
  jc.b0 = nullptr;
  const int nc = c->dim == 3 ? 7 : 5;
  ++c->launches;
  if (c->prec == EREM_FP32_BULK && c->adj_vec == 2)
    k_adj_scale_jlT<float, 64><<<blocks_padded(c), NT, 0, s>>>(jc, (float*)c->jlT_all, sc, geo_of(c), nc);
  else if (c->prec == EREM_FP32_BULK)
    k_adj_scale_jlT<float, 128><<<blocks_padded(c), NT, 0, s>>>(jc, (float*)c->jlT_all, sc, geo_of(c), nc);
  else
    k_adj_scale_jlT<double, 64><<<blocks_padded(c), NT, 0, s>>>(jc, (double*)c->jlT_all, sc, geo_of(c), nc);
}

void launch_adj_jT_apply(const erem_ctx* c, const double* x, const double* a, double* out,
                         cudaStream_t s) {
  ++c->launches;
  k_adj_jT_apply<<<blocks_cells(c), NT, 0, s>>>(jin(c), x, a, out, geo_of(c));
}

void launch_adj_face_pair(const erem_ctx* c, const double* y, const double* x, double scale,
                          cudaStream_t s) {
  ++c->launches;
  k_adj_face_pair<double, double><<<blocks_cells(c), NT, 0, s>>>(adj_faces(c), y, x, scale, geo_of(c));
}

void launch_adj_start(const erem_ctx* c, const double* mu, double d, void* sbuf, cudaStream_t s) {
  ++c->launches;
  if (c->prec == EREM_FP32_BULK)
    k_adj_start32<<<blocks_padded(c), NT, 0, s>>>(mu, d, (float*)sbuf, c->adj_mu32, (int)c->Np);
  else
    k_adj_start<double><<<blocks_padded(c), NT, 0, s>>>(mu, d, (double*)sbuf, (int)c->Np);
}

void launch_adj_horner(const erem_ctx* c, const void* s_in, void* s_out, const double* mu,
                       const void* q, double dj, double shift, double scale, int faces,
                       cudaStream_t s) {
  const int nc = c->dim == 3 ? 7 : 5;
  ++c->launches;
  if (c->prec == EREM_FP32_BULK) {
    // mu is taken from its FP32 copy (written with the first Horner value)
    (void)mu;
    (void)faces;
    const AdjFaces32 f{c->adj_up, c->adj_icap32, c->adj_g32[0], c->adj_g32[1], c->adj_g32[2],
                       c->adj_g0};
    const int vec = c->adj_vec;
    const int nb = (int)std::min<long long>((c->Np / vec + NT - 1) / NT,
                                            (long long)c->adj_blocks_per_sm * c->sm_count);
    k_adj_horner32<2><<<nb, NT, 0, s>>>((const float*)s_in, (float*)s_out, c->adj_mu32,
                                        (const float*)q, (const float*)c->jlT_all, nc, (float)dj,
                                        (float)shift, (float)scale, f, geo_of(c));
  } else
    k_adj_horner<double><<<blocks_cells(c), NT, 0, s>>>((const double*)s_in, (double*)s_out, mu,
                                                        (const double*)q, (const double*)c->jlT_all,
                                                        64, nc, dj, shift, scale, faces, adj_faces(c),
                                                        geo_of(c));
}

// Cells per thread of the FP32 Horner pass (two: with every load of a
// vector issued before its arithmetic, four cells would not fit the register
// budget) and its resident blocks per SM.
void choose_adj_vec(erem_ctx* c) {
  int b2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_adj_horner32<2>, NT, 0) != cudaSuccess) {
    cudaGetLastError();
    b2 = 4;
  }
  c->adj_vec = 2;
  c->adj_blocks_per_sm = std::max(b2, 1);
}

void launch_adj_aux32(const erem_ctx* c, cudaStream_t s) {
  ++c->launches;
  k_adj_aux32<<<blocks_cells(c), NT, 0, s>>>(c->Fx, c->Fy, c->Fz, c->F0, c->icap, c->adj_up,
                                             c->adj_icap32, geo_of(c));
}

void launch_adj_flush32(const erem_ctx* c, cudaStream_t s) {
  ++c->launches;
  k_adj_flush32<<<blocks_padded(c), NT, 0, s>>>(c->adj_g32[0], c->adj_g32[1], c->adj_g32[2],
                                                c->adj_gx, c->adj_gy, c->adj_gz, (int)c->Np);
}

void launch_adj_z(const erem_ctx* c, const void* sbuf, double delta, double* z, double* zacc,
                  cudaStream_t s) {
  ++c->launches;
  if (c->prec == EREM_FP32_BULK)
    k_adj_z<float><<<blocks_padded(c), NT, 0, s>>>((const float*)sbuf, delta, z, zacc, (int)c->Np);
  else
    k_adj_z<double><<<blocks_padded(c), NT, 0, s>>>((const double*)sbuf, delta, z, zacc, (int)c->Np);
}

void launch_adj_b_use(const erem_ctx* c, const double* y, cudaStream_t s) {
  ++c->launches;
  const int nf = c->ny * c->nz;
  k_adj_b_use<<<std::max(1, std::min(c->red_blocks, (nf + NT - 1) / NT)), NT, 0, s>>>(
      adj_faces(c), y, c->phys.T_inflow, geo_of(c));
}

void launch_adj_dLdp(const erem_ctx* c, cudaStream_t s) {
  const PresArr a = pres_arr(c);
  ++c->launches;
  k_adj_dLdp<<<blocks_cells(c), NT, 0, s>>>(adj_faces(c), c->lnk, c->phys.rhoc_f, phys_of(c), a.b, a.x,
                                            a.Ux, a.Uy, a.Uz, geo_of(c));
}

void launch_adj_lnk(const erem_ctx* c, double* out, cudaStream_t s) {
  const PresArr a = pres_arr(c);
  ++c->launches;
  k_adj_lnk<<<blocks_cells(c), NT, 0, s>>>(adj_faces(c), c->lnk, c->p, a.x, c->phys.rhoc_f, phys_of(c),
                                           a.Ux, a.Uy, a.Uz, out, geo_of(c));
}

}  // namespace erem
