// Host FP64 scalar side of the real Leja method (arXiv 1209.5553, §4.2):
// the Leja point table (eq. lejaa) and the divided differences of phi_1
// (the matrix-function route of §4.2).  Both are small, sequential
// computations that run once per context (points) or once per spectral
// interval and substep count (divided differences).
#include <algorithm>
#include <cmath>
#include <limits>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "erem_internal.h"

namespace erem {
namespace {

// sum_k log|x - p_k| and its first two derivatives in x.
struct LogProd {
  const std::vector<double>& p;
  double value(double x) const {
    double s = 0.0;
    for (double pk : p) s += std::log(std::fabs(x - pk));
    return s;
  }
  void derivs(double x, double* d1, double* d2) const {
    double a = 0.0, b = 0.0;
    for (double pk : p) {
      const double r = 1.0 / (x - pk);
      a += r;
      b -= r * r;
    }
    *d1 = a;
    *d2 = b;
  }
};

// Maximiser of the log-product strictly inside (lo, hi), two consecutive
// points.  The log-product is concave there and its derivative runs from
// +inf to -inf, so Newton's method on the derivative, kept inside a
// bisection bracket, converges to its single root.
double gap_argmax(const LogProd& f, double lo, double hi) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double g, h;
    f.derivs(x, &g, &h);
    if (g > 0.0) lo = x; else hi = x;
    double xn = x - g / h;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 4.0 * std::numeric_limits<double>::epsilon() * std::fabs(x) ||
        xn == x || hi - lo <= std::numeric_limits<double>::denorm_min()) {
      x = xn;
      break;
    }
    x = xn;
  }
  return x;
}

std::mutex g_leja_mu;
std::vector<double> g_leja;  // process-wide table, extended on demand

void extend_leja(int M) {
  if ((int)g_leja.size() >= M + 1) return;
  if (g_leja.empty()) g_leja.push_back(2.0);        // xi_0 = beta -> 2
  if (M >= 1 && g_leja.size() < 2) g_leja.push_back(-2.0);  // farthest from 2
  std::vector<double> sorted(g_leja);
  std::sort(sorted.begin(), sorted.end());
  while ((int)g_leja.size() < M + 1) {
    LogProd f{g_leja};
    double best_x = 0.0, best_v = -INFINITY;
    std::vector<std::pair<double, double>> cand;
    cand.reserve(sorted.size());
    for (size_t k = 0; k + 1 < sorted.size(); ++k) {
      const double x = gap_argmax(f, sorted[k], sorted[k + 1]);
      const double v = f.value(x);
      cand.emplace_back(x, v);
      if (v > best_v) { best_v = v; best_x = x; }
    }
    // equal products (to 1e-12 relative) go to the smaller point
    const double tol = 1e-12 * std::max(1.0, std::fabs(best_v));
    for (auto& c : cand)
      if (c.second >= best_v - tol && c.first < best_x) best_x = c.first;
    g_leja.push_back(best_x);
    sorted.insert(std::upper_bound(sorted.begin(), sorted.end(), best_x), best_x);
  }
}

std::mutex g_fast_mu;
std::vector<double> g_fast;                 // fast points in the order chosen
std::vector<double> g_fast_sorted;          // the same, sorted
std::vector<std::pair<double, double>> g_fast_cand;  // (gap midpoint, log-product)

// The fast variant: each new point is the gap midpoint with the largest
// log-product over the points chosen so far (ties to the smaller point).
// Adding a point adds its log-distance to every candidate and replaces the
// candidate of the gap it splits by the midpoints of the two halves.
void extend_fast(int M) {
  if ((int)g_fast.size() >= M + 1) return;
  auto logprod = [](double x) {
    double s = 0.0;
    for (double pk : g_fast) s += std::log(std::fabs(x - pk));
    return s;
  };
  if (g_fast.empty()) {
    g_fast = {2.0};
    g_fast_sorted = {2.0};
  }
  if (M >= 1 && g_fast.size() < 2) {
    g_fast.push_back(-2.0);
    g_fast_sorted = {-2.0, 2.0};
    g_fast_cand = {{0.0, logprod(0.0)}};
  }
  while ((int)g_fast.size() < M + 1) {
    double best_v = -INFINITY;
    for (auto& c : g_fast_cand) best_v = std::max(best_v, c.second);
    const double tol = 1e-12 * std::max(1.0, std::fabs(best_v));
    size_t pick = 0;
    double best_x = INFINITY;
    for (size_t i = 0; i < g_fast_cand.size(); ++i)
      if (g_fast_cand[i].second >= best_v - tol && g_fast_cand[i].first < best_x) {
        best_x = g_fast_cand[i].first;
        pick = i;
      }
    // neighbours of the chosen midpoint in the sorted points
    const auto hi_it = std::upper_bound(g_fast_sorted.begin(), g_fast_sorted.end(), best_x);
    const double hi = *hi_it, lo = *(hi_it - 1);
    g_fast.push_back(best_x);
    g_fast_sorted.insert(hi_it, best_x);
    g_fast_cand.erase(g_fast_cand.begin() + pick);
    for (auto& c : g_fast_cand) c.second += std::log(std::fabs(c.first - best_x));
    for (double m : {0.5 * (lo + best_x), 0.5 * (best_x + hi)}) g_fast_cand.emplace_back(m, logprod(m));
  }
}

}  // namespace

void fast_leja_table(int M, std::vector<double>* out) {
  std::lock_guard<std::mutex> lk(g_fast_mu);
  extend_fast(M);
  out->assign(g_fast.begin(), g_fast.begin() + M + 1);
}

void leja_table(int M, std::vector<double>* out) {
  std::lock_guard<std::mutex> lk(g_leja_mu);
  extend_leja(M);
  out->assign(g_leja.begin(), g_leja.begin() + M + 1);
}

// Divided differences d_j = phi_1[xi_0..xi_j] of xi -> phi_1(c + gamma xi).
//
// phi_1(z) is the divided difference exp[0, z], so phi_1[z_0..z_j] =
// exp[0, z_0, .., z_j], an entry of the exponential of the lower bidiagonal
// matrix with diagonal (0, z_0, .., z_M) and ones below it (the Opitz form
// that §4.2 uses).  Scaling row/column k by gamma^(k-1) turns the divided
// differences in z into divided differences in xi: with subdiagonal
// (1, gamma, .., gamma) the entry (j+1, 0) of the exponential is d_j.
//
// exp(W) = exp(W / 2^s)^(2^s).  W / 2^s has norm <= 1/2 and at most
// 16 rows per squaring level (n / 2^s <= 16), and its exponential is taken
// from 64 Taylor terms built by repeated right-multiplication with the
// bidiagonal matrix (each power is banded).  Every entry of exp(W / 2^s) is
// non-negative (W has a non-negative off-diagonal), so the squarings and
// the products with a non-negative vector add terms of one sign and keep
// relative accuracy even for the tiny entries far below the diagonal.
// Only column 0 of exp(W) is needed: k squarings make F = exp(W / 2^s)^(2^k)
// and 2^(s-k) - 1 products F v, from v = F e_0, finish it, with k chosen
// to minimise the operations (k n^3 / 6 against n^2 / 2 per product).
//
// phi_2 (and phi_k) the same way: phi_k(z) = exp[0, .., 0, z] with k zeros,
// so the diagonal starts with k zeros, the subdiagonal with k ones, and the
// entry (j+k, 0) is the divided difference d_j of phi_k.
//
// threads > 1: the rows of the Taylor sum and of every squaring are shared
// out among that many host threads (row i to thread i mod threads), which
// meet at a barrier between squarings; the split between squarings and
// products follows the number of threads asked for, and every entry sums its
// terms in the same order, so a given thread count gives the same bits
// however many threads could be started.
namespace {

// Sense-counting barrier for a team of host threads.
class SpinBarrier {
 public:
  void set(int n) { n_ = n; }
  void wait() {
    const int g = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
      count_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_acq_rel);
    } else {
      while (gen_.load(std::memory_order_acquire) == g) std::this_thread::yield();
    }
  }

 private:
  int n_ = 1;
  std::atomic<int> count_{0}, gen_{0};
};

}  // namespace

int divided_differences_phi(int kphi, int M, const double* xi, double c, double gamma, double* d,
                            int threads) {
  if (kphi < 1 || kphi > 4 || M < 0 || !xi || !d || !std::isfinite(c) || !std::isfinite(gamma) ||
      gamma <= 0.0)
    return -1;
  const int n = M + 1 + kphi;
  std::vector<double> diag(n), sub(n, 0.0);  // sub[k] = W(k, k-1)
  for (int k = 0; k < n; ++k) {
    diag[k] = k < kphi ? 0.0 : c + gamma * xi[k - kphi];
    if (k > 0) sub[k] = (k <= kphi) ? 1.0 : gamma;
  }
  double norm = 0.0;  // ||W||_1: column k holds diag[k] and sub[k+1]
  for (int k = 0; k < n; ++k) norm = std::max(norm, std::fabs(diag[k]) + (k + 1 < n ? sub[k + 1] : 0.0));
  int s = 0;
  while (norm / std::ldexp(1.0, s) > 0.5) ++s;
  while ((double)n / std::ldexp(1.0, s) > 16.0) ++s;
  const double scale = std::ldexp(1.0, -s);
  for (int k = 0; k < n; ++k) { diag[k] *= scale; sub[k] *= scale; }
  const int T_want = std::max(1, std::min(threads, n / 24));
  std::vector<double> E((size_t)n * n, 0.0), Ta((size_t)n * n, 0.0), Tb((size_t)n * n, 0.0);
  std::vector<double> va(n, 0.0), vb(n, 0.0);
  for (int i = 0; i < n; ++i) { E[(size_t)i * n + i] = 1.0; Ta[(size_t)i * n + i] = 1.0; }
  SpinBarrier bar;
  // squarings k (shared by the team), then 2^(s-k) - 1 matrix-vector
  // products (one thread), k minimising the operations per thread of the
  // team asked for (not of the team started: the bits depend on k only)
  int ksq = s;
  {
    double best = 1e300;
    for (int k = std::max(0, s - 24); k <= s; ++k) {
      const double cost =
          k * (double)n * n * n / (6.0 * T_want) + (std::ldexp(1.0, s - k) - 1.0) * n * n / 2.0;
      if (cost < best) {
        best = cost;
        ksq = k;
      }
    }
  }
  auto team = [&](int t, int T) {
    // E = sum_{k=0}^{64} B^k / k!, lower triangular, row-major n x n; row i
    // of every power needs only row i of the one before, so each thread runs
    // all terms on its own rows
    const int K = 64;
    for (int i = t; i < n; i += T) {
      double* __restrict__ Tk = Ta.data() + (size_t)i * n;
      double* __restrict__ Tn = Tb.data() + (size_t)i * n;
      double* __restrict__ Ei = E.data() + (size_t)i * n;
      for (int k = 0; k < K; ++k) {
        const int band = std::min(k, n - 1);       // Tk is zero below band k
        const int nb = std::min(k + 1, n - 1);
        const double inv = 1.0 / (double)(k + 1);
        const int j0 = std::max(0, i - nb);
        for (int j = j0; j <= i; ++j) {
          // (Tk B)(i, j) = Tk(i, j) B(j, j) + Tk(i, j+1) B(j+1, j)
          double v = 0.0;
          if (i - j <= band) v += Tk[j] * diag[j];
          if (j + 1 <= i && i - (j + 1) <= band) v += Tk[j + 1] * sub[j + 1];
          Tn[j] = v * inv;
        }
        for (int j = j0; j <= i; ++j) Ei[j] += Tn[j];
        std::swap(Tk, Tn);
      }
    }
    bar.wait();
    // squarings of the lower triangle (row i of A A is sum_l A(i, l) (row
    // l of A); each entry sums in increasing l)
    double* A = E.data();
    double* F = Ta.data();
    for (int sq = 0; sq < ksq; ++sq) {
      for (int i = t; i < n; i += T) {
        double* __restrict__ Fi = F + (size_t)i * n;
        const double* __restrict__ Ai = A + (size_t)i * n;
        for (int j = 0; j <= i; ++j) Fi[j] = 0.0;
        for (int l = 0; l <= i; ++l) {
          const double a = Ai[l];
          const double* __restrict__ Al = A + (size_t)l * n;
#pragma GCC ivdep
          for (int j = 0; j <= l; ++j) Fi[j] += a * Al[j];
        }
      }
      std::swap(A, F);
      bar.wait();
    }
    if (t != 0) return;
    // v = A e_0, then v = A v
    double* v = va.data();
    double* w = vb.data();
    for (int i = 0; i < n; ++i) v[i] = A[(size_t)i * n];
    const long long nprod = (1LL << (s - ksq)) - 1;
    for (long long r = 0; r < nprod; ++r) {
      for (int i = 0; i < n; ++i) {
        const double* __restrict__ Ai = A + (size_t)i * n;
        double acc = 0.0;
        for (int l = 0; l <= i; ++l) acc += Ai[l] * v[l];
        w[i] = acc;
      }
      std::swap(v, w);
    }
    for (int j = 0; j <= M; ++j) d[j] = v[j + kphi];
  };
  // the helpers wait for the size of the team that could be started
  std::atomic<int> go{0};
  std::vector<std::thread> pool;
  for (int t = 1; t < T_want; ++t) {
    try {
      pool.emplace_back([&, t]() {
        int T;
        while ((T = go.load(std::memory_order_acquire)) == 0) std::this_thread::yield();
        team(t, T);
      });
    } catch (...) {  // fewer threads than asked for: the team is smaller
      break;
    }
  }
  const int T = (int)pool.size() + 1;
  bar.set(T);
  go.store(T, std::memory_order_release);
  team(0, T);
  for (auto& th : pool) th.join();
  return 0;
}

int divided_differences(int M, const double* xi, double c, double gamma, double* d) {
  return divided_differences_phi(1, M, xi, c, gamma, d);
}

// exp(A) of a small dense matrix (row-major n x n): a Taylor polynomial of
// degree 30 of A / 2^s with ||A / 2^s||_1 <= 1/2, then s squarings.
void expm_small(int n, const double* A, double* E) {
  double norm = 0.0;
  for (int j = 0; j < n; ++j) {
    double col = 0.0;
    for (int i = 0; i < n; ++i) col += std::fabs(A[(size_t)i * n + j]);
    norm = std::max(norm, col);
  }
  int s = 0;
  while (norm / std::ldexp(1.0, s) > 0.5) ++s;
  const double scale = std::ldexp(1.0, -s);
  std::vector<double> B((size_t)n * n), T((size_t)n * n, 0.0), U((size_t)n * n);
  for (size_t q = 0; q < B.size(); ++q) B[q] = A[q] * scale;
  for (int i = 0; i < n; ++i) T[(size_t)i * n + i] = 1.0;
  std::vector<double> S = T;
  for (int k = 1; k <= 30; ++k) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = 0.0;
        for (int l = 0; l < n; ++l) a += T[(size_t)i * n + l] * B[(size_t)l * n + j];
        U[(size_t)i * n + j] = a / k;
      }
    T.swap(U);
    for (size_t q = 0; q < S.size(); ++q) S[q] += T[q];
  }
  for (int r = 0; r < s; ++r) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = 0.0;
        for (int l = 0; l < n; ++l) a += S[(size_t)i * n + l] * S[(size_t)l * n + j];
        U[(size_t)i * n + j] = a;
      }
    S.swap(U);
  }
  std::copy(S.begin(), S.end(), E);
}

}  // namespace erem

extern "C" int erem_leja_points(int M, double* xi) {
  if (M < 0 || M > 4096 || !xi) return -1;
  std::vector<double> t;
  erem::leja_table(M, &t);
  std::copy(t.begin(), t.end(), xi);
  return 0;
}

extern "C" int erem_phi2_divided_differences(int M, const double* xi, double c, double gamma,
                                             double* d) {
  return erem::divided_differences_phi(2, M, xi, c, gamma, d);
}

extern "C" int erem_fast_leja_points(int M, double* xi) {
  if (M < 0 || M > 4096 || !xi) return -1;
  std::vector<double> t;
  erem::fast_leja_table(M, &t);
  std::copy(t.begin(), t.end(), xi);
  return 0;
}

extern "C" int erem_phi1_divided_differences(int M, const double* xi, double c, double gamma,
                                             double* d) {
  return erem::divided_differences(M, xi, c, gamma, d);
}
