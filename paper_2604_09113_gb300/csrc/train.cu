// Offline ROM training (Sec. 4.2, offline phase of Sec. 4.4), host C++.
//
// Snapshots I(mu) of Eq. (MDEIM I) are computed from the Legendre moments of the
// trimmed cell, M[a][b] = int_Omega P_a(2 xi1 - 1) P_b(2 xi2 - 1): every entry of
// I is a product f(xi1) g(xi2) of 1D polynomials of degree <= 2p+q, so
// I = F^T M G with F, G the Legendre coefficients of those 1D products.  The
// moments use the height-function form of the quadrature (Sec. 2.2.3): along
// xi2 the level set's roots are closed-form for the bilinear threshold and the
// Legendre antiderivatives integrate each solid interval exactly; along xi1 an
// adaptive Gauss rule is refined until the moment matrix converges.
//
// U_r: eigen-decomposition of the snapshot Gram matrix (cyclic Jacobi), the
// leading n_r left singular vectors re-orthonormalised (Sec. 4.2.2).
// Magic points: Algorithm 3 with the interpolatory projection of empirical
// interpolation.  I_r at the (r+1)^4 tensor GLL nodes of the box from the
// magic-point entries (Sec. 4.2.3).  Output: the ROM file of romb.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <thread>
#include <vector>

#include "romb_internal.cuh"
#include "tables.cuh"
#include "trim.cuh"

namespace {

struct Trainer {
  int family, kind, p, q, r, n_r;
  double lo, hi;
  int nB, nL, D, n_i, nF;
  std::vector<double> F;    // [nF][D+1] Legendre coefficients of the xi1 factors (= xi2 factors)
  std::vector<double> Fv;   // [(p+1)(q+1)][D+1] the same for the value products b_a l_c
  std::vector<double> gx, gw;   // outer Gauss rule on [0,1]

  void setup(const romb_train_spec& s) {
    family = s.family;
    kind = s.basis;
    p = s.p;
    q = s.q;
    r = s.r;
    n_r = s.n_r;
    lo = s.lo;
    hi = s.hi;
    init();
  }

  void init() {
    nB = (p + 1) * (p + 1);
    nL = (q + 1) * (q + 1);
    D = 2 * p + q;
    n_i = nB * nB * nL * 4;
    // 1D factor (a1, d1, a2, d2, c): b^(d1)_a1 b^(d2)_a2 l_c, index ((((a1*2+d1)*(p+1)+a2)*2+d2)*(q+1)+c)
    nF = (p + 1) * 2 * (p + 1) * 2 * (q + 1);
    F.assign((size_t)nF * (D + 1), 0.0);
    const int ng = D + 1;
    std::vector<double> x(ng), w(ng);
    gauss01(ng, x.data(), w.data());
    double gll[ROMB_MAX_P + 1], qn[8];
    gll_nodes01(p, gll);
    gll_nodes01(q, qn);
    for (int g = 0; g < ng; ++g) {
      double bv[ROMB_MAX_P + 1], bd[ROMB_MAX_P + 1], lv[8], P[64];
      if (kind == 0) lagrange1d_host(p, gll, x[g], bv, bd);
      else bernstein1d_host(p, x[g], bv, bd);
      lagrange1d_host(q, qn, x[g], lv, nullptr);
      legendre(D, 2.0 * x[g] - 1.0, P);
      for (int a1 = 0; a1 <= p; ++a1)
        for (int d1 = 0; d1 < 2; ++d1)
          for (int a2 = 0; a2 <= p; ++a2)
            for (int d2 = 0; d2 < 2; ++d2)
              for (int cc = 0; cc <= q; ++cc) {
                const int f = (((a1 * 2 + d1) * (p + 1) + a2) * 2 + d2) * (q + 1) + cc;
                const double v = (d1 ? bd[a1] : bv[a1]) * (d2 ? bd[a2] : bv[a2]) * lv[cc];
                for (int a = 0; a <= D; ++a) F[(size_t)f * (D + 1) + a] += (2 * a + 1) * w[g] * v * P[a];
              }
    }
    // 1D value products b_a l_c for the body-force volume integrals, index a (q+1) + c
    Fv.assign((size_t)(p + 1) * (q + 1) * (D + 1), 0.0);
    for (int g = 0; g < ng; ++g) {
      double bv[ROMB_MAX_P + 1], bd[ROMB_MAX_P + 1], lv[8], P[64];
      if (kind == 0) lagrange1d_host(p, gll, x[g], bv, bd);
      else bernstein1d_host(p, x[g], bv, bd);
      lagrange1d_host(q, qn, x[g], lv, nullptr);
      legendre(D, 2.0 * x[g] - 1.0, P);
      for (int a = 0; a <= p; ++a)
        for (int cc = 0; cc <= q; ++cc)
          for (int al = 0; al <= D; ++al)
            Fv[((size_t)a * (q + 1) + cc) * (D + 1) + al] += (2 * al + 1) * w[g] * bv[a] * lv[cc] * P[al];
    }
    gx.resize(20);
    gw.resize(20);
    gauss01(20, gx.data(), gw.data());
  }

  // V[k][k3] = int over the trimmed cell of B_k L_k3 from the moment matrix
  // (the volume part of the external-force integrals), k = ax + (p+1) ay,
  // k3 = cx + (q+1) cy
  void volume_from_moments(const double* M, double* V) const {
    const int n = D + 1, nv = (p + 1) * (q + 1);
    std::vector<double> H((size_t)n * nv);   // H[al][g] = sum_be M[al][be] Fv[g][be]
    for (int al = 0; al < n; ++al)
      for (int g = 0; g < nv; ++g) {
        double sum = 0.0;
        for (int be = 0; be < n; ++be) sum += M[al * n + be] * Fv[(size_t)g * n + be];
        H[(size_t)al * nv + g] = sum;
      }
    for (int ay = 0; ay <= p; ++ay)
      for (int ax = 0; ax <= p; ++ax)
        for (int cy = 0; cy <= q; ++cy)
          for (int cx = 0; cx <= q; ++cx) {
            const int f = ax * (q + 1) + cx, g = ay * (q + 1) + cy;
            double sum = 0.0;
            for (int al = 0; al < n; ++al) sum += Fv[(size_t)f * n + al] * H[(size_t)al * nv + g];
            V[(size_t)(ax + (p + 1) * ay) * nL + cx + (q + 1) * cy] = sum;
          }
  }

  static void lagrange1d_host(int n, const double* nodes, double t, double* v, double* d) {
    for (int i = 0; i <= n; ++i) {
      double den = 1.0, val = 1.0, der = 0.0;
      for (int j = 0; j <= n; ++j) {
        if (j == i) continue;
        den *= nodes[i] - nodes[j];
        der = der * (t - nodes[j]) + val;
        val *= t - nodes[j];
      }
      v[i] = val / den;
      if (d) d[i] = der / den;
    }
  }
  static void bernstein1d_host(int p, double t, double* v, double* d) {
    double binom = 1.0;
    for (int i = 0; i <= p; ++i) {
      if (i > 0) binom = binom * (p - i + 1) / i;
      v[i] = binom * pow(t, i) * pow(1.0 - t, p - i);
      double dv = 0.0;
      if (i > 0) dv += binom * i * pow(t, i - 1) * pow(1.0 - t, p - i);
      if (i < p) dv -= binom * (p - i) * pow(t, i) * pow(1.0 - t, p - i - 1);
      d[i] = dv;
    }
  }

  // moments of the solid part over xi1 in [a, b] with one 20-point Gauss panel
  void panel(const double* mu, double a, double b, double* M) const {
    const int n = D + 1;
    for (int i = 0; i < n * n; ++i) M[i] = 0.0;
    double lo[4], hi[4], P[64], Au[64], Av[64], inner[64];
    for (int g = 0; g < 20; ++g) {
      const double x = a + (b - a) * gx[g], w = (b - a) * gw[g];
      const int ni = solid_y(family, mu, x, lo, hi);
      for (int t = 0; t < n; ++t) inner[t] = 0.0;
      for (int k = 0; k < ni; ++k) {
        legendre_antideriv(D, lo[k], Au);
        legendre_antideriv(D, hi[k], Av);
        for (int t = 0; t < n; ++t) inner[t] += Av[t] - Au[t];
      }
      legendre(D, 2.0 * x - 1.0, P);
      for (int s = 0; s < n; ++s) {
        const double ws = w * P[s];
        for (int t = 0; t < n; ++t) M[s * n + t] += ws * inner[t];
      }
    }
  }

  void moments(const double* mu, double* M) const {
    const int n = D + 1, nn = n * n;
    for (int i = 0; i < nn; ++i) M[i] = 0.0;
    struct Item {
      double a, b;
      int depth;
      std::vector<double> Mp;
    };
    std::vector<Item> stack;
    for (int h = 0; h < 2; ++h) {
      Item it{0.5 * h, 0.5 * h + 0.5, 0, std::vector<double>(nn)};
      panel(mu, it.a, it.b, it.Mp.data());
      stack.push_back(std::move(it));
    }
    std::vector<double> L(nn), R(nn);
    while (!stack.empty()) {
      Item it = std::move(stack.back());
      stack.pop_back();
      const double m = 0.5 * (it.a + it.b);
      panel(mu, it.a, m, L.data());
      panel(mu, m, it.b, R.data());
      double err = 0.0;
      for (int i = 0; i < nn; ++i) err = fmax(err, fabs(it.Mp[i] - L[i] - R[i]));
      if (err <= 1e-15 || it.depth >= 50) {
        for (int i = 0; i < nn; ++i) M[i] += L[i] + R[i];
      } else {
        stack.push_back(Item{it.a, m, it.depth + 1, L});
        stack.push_back(Item{m, it.b, it.depth + 1, R});
      }
    }
  }

  // factor indices of entry e of I
  inline void factors(int e, int* f, int* g) const {
    const int j2 = e & 1, j1 = (e >> 1) & 1;
    int t = e >> 2;
    const int k3 = t % nL;
    t /= nL;
    const int k2 = t % nB, k1 = t / nB;
    const int a1 = k1 % (p + 1), b1 = k1 / (p + 1), a2 = k2 % (p + 1), b2 = k2 / (p + 1);
    const int c1 = k3 % (q + 1), c2 = k3 / (q + 1);
    // xi1 factor: derivative where j == 0; xi2 factor: derivative where j == 1
    *f = (((a1 * 2 + (j1 == 0)) * (p + 1) + a2) * 2 + (j2 == 0)) * (q + 1) + c1;
    *g = (((b1 * 2 + (j1 == 1)) * (p + 1) + b2) * 2 + (j2 == 1)) * (q + 1) + c2;
  }

  // I (all entries) from the moment matrix
  void snapshot_from_moments(const double* M, double* I) const {
    const int n = D + 1;
    std::vector<double> H((size_t)n * nF);   // H[a][g] = sum_b M[a][b] G[g][b]
    for (int a = 0; a < n; ++a)
      for (int g = 0; g < nF; ++g) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += M[a * n + b] * F[(size_t)g * n + b];
        H[(size_t)a * nF + g] = s;
      }
    for (int e = 0; e < n_i; ++e) {
      int f, g;
      factors(e, &f, &g);
      double s = 0.0;
      for (int a = 0; a < n; ++a) s += F[(size_t)f * n + a] * H[(size_t)a * nF + g];
      I[e] = s;
    }
  }

  double entry_from_moments(const double* M, int e) const {
    const int n = D + 1;
    int f, g;
    factors(e, &f, &g);
    double s = 0.0;
    for (int a = 0; a < n; ++a) {
      double h = 0.0;
      for (int b = 0; b < n; ++b) h += M[a * n + b] * F[(size_t)g * n + b];
      s += F[(size_t)f * n + a] * h;
    }
    return s;
  }
};

template <class Fn>
void parallel_for(int n, int nthreads, Fn fn) {
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&]() {
      for (int i = next++; i < n; i = next++) fn(i);
    });
  for (auto& x : th) x.join();
}

// symmetric eigen-decomposition by cyclic Jacobi: A (n x n, destroyed) -> eigenvalues w, vectors V (columns)
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int pp = 0; pp < n - 1; ++pp)
      for (int qq = pp + 1; qq < n; ++qq) {
        const double apq = A[(size_t)pp * n + qq];
        if (fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)pp * n + pp], aqq = A[(size_t)qq * n + qq];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + pp], akq = A[(size_t)k * n + qq];
          A[(size_t)k * n + pp] = c * akp - s * akq;
          A[(size_t)k * n + qq] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)pp * n + k], aqk = A[(size_t)qq * n + k];
          A[(size_t)pp * n + k] = c * apk - s * aqk;
          A[(size_t)qq * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + pp], vkq = V[(size_t)k * n + qq];
          V[(size_t)k * n + pp] = c * vkp - s * vkq;
          V[(size_t)k * n + qq] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// LU with partial pivoting (n small): solve A x = b for many b
struct LU {
  int n;
  std::vector<double> a;
  std::vector<int> piv;
  bool factor(int n_, const std::vector<double>& A) {
    n = n_;
    a = A;
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
      int m = k;
      for (int i = k + 1; i < n; ++i)
        if (fabs(a[(size_t)i * n + k]) > fabs(a[(size_t)m * n + k])) m = i;
      piv[k] = m;
      if (a[(size_t)m * n + k] == 0.0) return false;
      if (m != k)
        for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)m * n + j]);
      for (int i = k + 1; i < n; ++i) {
        a[(size_t)i * n + k] /= a[(size_t)k * n + k];
        for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
      }
    }
    return true;
  }
  void solve(double* b) const {
    for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < i; ++k) b[i] -= a[(size_t)i * n + k] * b[k];
    for (int i = n - 1; i >= 0; --i) {
      for (int k = i + 1; k < n; ++k) b[i] -= a[(size_t)i * n + k] * b[k];
      b[i] /= a[(size_t)i * n + i];
    }
  }
};

// ---- reduced model of the force integrals (Sec. 4.2 applied to Eq. SPEED L ext) ----
// J(mu)[e][s][k] = int over the solid part of cell edge e of b_s(t) l_k(t) dt,
// e = 0..3 (left, right, bottom, top), s along the edge, l_k the degree-q
// Lagrange polynomials on the edge's GLL nodes.  Solid intervals of a
// vertical edge are those of xi2 at xi1 = 0 / 1; a horizontal edge uses the
// same function with mu_2 and mu_3 exchanged (both families are symmetric
// under swapping xi1 and xi2 once the corners are swapped accordingly).
void edge_load_tensor(const romb_train_spec& sp, const double* mu, double* J) {
  const int p = sp.p, q = sp.q, nf = 4 * (p + 1) * (q + 1);
  for (int i = 0; i < nf; ++i) J[i] = 0.0;
  double gx[24], gw[24], gll[ROMB_MAX_P + 1], qn[8];
  gauss01(24, gx, gw);
  gll_nodes01(p, gll);
  gll_nodes01(q, qn);
  for (int e = 0; e < 4; ++e) {
    const double mt[4] = {mu[0], mu[2], mu[1], mu[3]};
    const double* me = e < 2 ? mu : mt;
    double lo[4], hi[4];
    const int ni = solid_y(sp.family, me, (e == 1 || e == 3) ? 1.0 : 0.0, lo, hi);
    for (int iv = 0; iv < ni; ++iv) {
      const double len = hi[iv] - lo[iv];
      for (int g = 0; g < 24; ++g) {
        const double t = lo[iv] + len * gx[g], w = len * gw[g];
        double bv[ROMB_MAX_P + 1], bd[ROMB_MAX_P + 1], lv[8];
        if (sp.basis == 0) Trainer::lagrange1d_host(p, gll, t, bv, bd);
        else Trainer::bernstein1d_host(p, t, bv, bd);
        Trainer::lagrange1d_host(q, qn, t, lv, nullptr);
        for (int si = 0; si <= p; ++si)
          for (int k = 0; k <= q; ++k) J[(e * (p + 1) + si) * (q + 1) + k] += w * bv[si] * lv[k];
      }
    }
  }
}

// J(mu) with the volume part when the spec asks for body forces: the edge
// integrals, then V[k][k3] = int over the trimmed cell of B_k L_k3 (from the
// Legendre moments of the trimmed cell, as the stiffness snapshots).
void external_tensor(const Trainer& T, const romb_train_spec& sp, const double* mu, double* J) {
  const int ne = 4 * (sp.p + 1) * (sp.q + 1);
  edge_load_tensor(sp, mu, J);
  if (!sp.body) return;
  std::vector<double> M((size_t)(T.D + 1) * (T.D + 1));
  T.moments(mu, M.data());
  T.volume_from_moments(M.data(), J + ne);
}

}  // namespace

// Tables shared with the GPU trainer: the Legendre coefficients F of the 1D
// factor products, the Gauss rule of one panel, and I_Pi (the untrimmed
// tensor, from the moments e_0 e_0^T).
// The tables depend on (family, basis, p, q) only; they are built once per
// process and key (the exact fallback of romb_factor asks for them on every
// factorisation that needs it).
namespace {
struct HostTables {
  std::vector<double> F, gx, gw, Ipi;
  int D = 0, nF = 0;
};
std::mutex g_tables_mu;
std::map<std::tuple<int, int, int, int>, HostTables> g_tables;
}  // namespace

romb_status train_host_tables(const romb_train_spec* sp, std::vector<double>& F, int* D, int* nF,
                              std::vector<double>& gx, std::vector<double>& gw, std::vector<double>& Ipi) {
  const auto key = std::make_tuple(sp->family, sp->basis, sp->p, sp->q);
  {
    std::lock_guard<std::mutex> lk(g_tables_mu);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
      F = it->second.F;
      *D = it->second.D;
      *nF = it->second.nF;
      gx = it->second.gx;
      gw = it->second.gw;
      Ipi = it->second.Ipi;
      return ROMB_OK;
    }
  }
  Trainer T;
  T.setup(*sp);
  HostTables H;
  H.F = T.F;
  H.D = T.D;
  H.nF = T.nF;
  H.gx = T.gx;
  H.gw = T.gw;
  H.Ipi.assign(T.n_i, 0.0);
  std::vector<double> M((size_t)(T.D + 1) * (T.D + 1), 0.0);
  M[0] = 1.0;
  T.snapshot_from_moments(M.data(), H.Ipi.data());
  F = H.F;
  *D = H.D;
  *nF = H.nF;
  gx = H.gx;
  gw = H.gw;
  Ipi = H.Ipi;
  std::lock_guard<std::mutex> lk(g_tables_mu);
  g_tables.emplace(key, std::move(H));
  return ROMB_OK;
}

void train_jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  jacobi_eig(n, A, w, V);
}

// The force model of a spec on the samples: U_f (eigenvectors of the
// n_f x n_f matrix S S^T of the J snapshots, those with singular values above
// 1e-7 of the largest), magic points (Algorithm 3), grid coefficients.
romb_status train_force_model(const romb_train_spec* sp, const double* samples, int n_s, RombForceModel* out) {
  const double lo4[4] = {sp->lo, sp->lo, sp->lo, sp->lo}, hi4[4] = {sp->hi, sp->hi, sp->hi, sp->hi};
  return train_force_model_box(sp, lo4, hi4, samples, n_s, out);
}

romb_status train_force_model_box(const romb_train_spec* sp, const double* lo4, const double* hi4,
                                  const double* samples, int n_s, RombForceModel* out) {
  const int nf = 4 * (sp->p + 1) * (sp->q + 1) + (sp->body ? (sp->p + 1) * (sp->p + 1) * (sp->q + 1) * (sp->q + 1) : 0);
  const int nth = sp->n_threads > 0 ? sp->n_threads : std::max(1u, std::thread::hardware_concurrency());
  Trainer T;
  T.setup(*sp);
  std::vector<double> S((size_t)n_s * nf);
  parallel_for(n_s, nth, [&](int si) { external_tensor(T, *sp, samples + 4 * si, &S[(size_t)si * nf]); });
  // U_f: the leading left singular vectors of the snapshots, from the smaller
  // of the two Gram matrices (n_f x n_f, or n_s x n_s by the method of
  // snapshots), those with singular values above 1e-7 of the largest
  const bool by_snap = n_s < nf;
  const int ng_ = by_snap ? n_s : nf;
  std::vector<double> C((size_t)ng_ * ng_, 0.0), w, V;
  for (int a = 0; a < ng_; ++a)
    for (int b = 0; b <= a; ++b) {
      double sum = 0.0;
      if (by_snap)
        for (int e = 0; e < nf; ++e) sum += S[(size_t)a * nf + e] * S[(size_t)b * nf + e];
      else
        for (int si = 0; si < n_s; ++si) sum += S[(size_t)si * nf + a] * S[(size_t)si * nf + b];
      C[(size_t)a * ng_ + b] = C[(size_t)b * ng_ + a] = sum;
    }
  jacobi_eig(ng_, C, w, V);
  std::vector<int> order(ng_);
  for (int i = 0; i < ng_; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  int rf = 0;
  const double wmax = w[order[0]];
  if (!(wmax > 0.0)) return ROMB_E_NAN;
  while (rf < nf && rf < n_s && w[order[rf]] > 1e-14 * wmax) ++rf;   // singular values above 1e-7 of the largest
  std::vector<double> U((size_t)rf * nf);
  if (!by_snap) {
    for (int k = 0; k < rf; ++k)
      for (int a = 0; a < nf; ++a) U[(size_t)k * nf + a] = V[(size_t)a * nf + order[k]];
  } else {
    // U_k = S^T v_k / sqrt(lambda_k), then two passes of modified Gram-Schmidt
    for (int k = 0; k < rf; ++k) {
      const double sc = 1.0 / sqrt(w[order[k]]);
      for (int e = 0; e < nf; ++e) {
        double sum = 0.0;
        for (int si = 0; si < n_s; ++si) sum += S[(size_t)si * nf + e] * V[(size_t)si * ng_ + order[k]];
        U[(size_t)k * nf + e] = sum * sc;
      }
    }
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < rf; ++k) {
        double* uk = &U[(size_t)k * nf];
        for (int j = 0; j < k; ++j) {
          const double* uj = &U[(size_t)j * nf];
          double d = 0.0;
          for (int e = 0; e < nf; ++e) d += uj[e] * uk[e];
          for (int e = 0; e < nf; ++e) uk[e] -= d * uj[e];
        }
        double nrm = 0.0;
        for (int e = 0; e < nf; ++e) nrm += uk[e] * uk[e];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) return ROMB_E_NAN;
        for (int e = 0; e < nf; ++e) uk[e] /= nrm;
      }
  }
  std::vector<long long> magic(rf);
  {
    std::vector<double> res(nf);
    for (int j = 0; j < rf; ++j) {
      std::vector<double> c(std::max(1, j));
      if (j > 0) {
        std::vector<double> A((size_t)j * j);
        for (int a = 0; a < j; ++a) {
          for (int b = 0; b < j; ++b) A[(size_t)a * j + b] = U[(size_t)b * nf + magic[a]];
          c[a] = U[(size_t)j * nf + magic[a]];
        }
        LU lu;
        if (!lu.factor(j, A)) return ROMB_E_NAN;
        lu.solve(c.data());
      }
      int m = 0;
      for (int e = 0; e < nf; ++e) {
        double v = U[(size_t)j * nf + e];
        for (int b = 0; b < j; ++b) v -= U[(size_t)b * nf + e] * c[b];
        res[e] = v;
        if (fabs(res[e]) > fabs(res[m])) m = e;
      }
      magic[j] = m;
    }
  }
  const int n1 = sp->r + 1, ng = n1 * n1 * n1 * n1;
  double g1d[12];
  gll_nodes01(sp->r, g1d);
  std::vector<double> Um((size_t)rf * rf);
  for (int a = 0; a < rf; ++a)
    for (int b = 0; b < rf; ++b) Um[(size_t)a * rf + b] = U[(size_t)b * nf + magic[a]];
  LU lu;
  if (!lu.factor(rf, Um)) return ROMB_E_NAN;
  std::vector<double> A((size_t)rf * ng);
  parallel_for(ng, nth, [&](int g) {
    const int ii[4] = {g % n1, (g / n1) % n1, (g / (n1 * n1)) % n1, g / (n1 * n1 * n1)};
    double mu[4];
    for (int d = 0; d < 4; ++d) mu[d] = lo4[d] + (hi4[d] - lo4[d]) * g1d[ii[d]];
    std::vector<double> J(nf), bb(rf);
    external_tensor(T, *sp, mu, J.data());
    for (int a = 0; a < rf; ++a) bb[a] = J[magic[a]];
    lu.solve(bb.data());
    for (int a = 0; a < rf; ++a) A[(size_t)a * ng + g] = bb[a];
  });
  out->n_f = nf;
  out->r_f = rf;
  out->U = std::move(U);
  out->A = std::move(A);
  out->magic = std::move(magic);
  return ROMB_OK;
}

bool write_force_section(FILE* f, const RombForceModel& m) {
  const int64_t hdr[2] = {m.n_f, m.r_f};
  bool ok = fwrite(hdr, 8, 2, f) == 2;
  ok = ok && fwrite(m.U.data(), 8, m.U.size(), f) == m.U.size();
  ok = ok && fwrite(m.A.data(), 8, m.A.size(), f) == m.A.size();
  ok = ok && fwrite(m.magic.data(), 8, m.magic.size(), f) == m.magic.size();
  return ok;
}

extern "C" romb_status romb_train_snapshot(const romb_train_spec* sp, const double* mu4, double* I_out) {
  if (!sp || !mu4 || !I_out || sp->p < 3 || sp->p > ROMB_MAX_P || sp->q != 2 || (sp->family < 0 || sp->family > 5))
    return ROMB_E_ARG;
  Trainer T;
  T.setup(*sp);
  std::vector<double> M((size_t)(T.D + 1) * (T.D + 1));
  T.moments(mu4, M.data());
  T.snapshot_from_moments(M.data(), I_out);
  return ROMB_OK;
}

extern "C" romb_status romb_train(const romb_train_spec* sp, const double* samples, int n_s, const char* path) {
  if (!sp || !samples || !path || n_s < 1 || sp->p < 3 || sp->p > ROMB_MAX_P || sp->q != 2 || sp->r < 1 ||
      sp->r > 10 || sp->n_r < 1 || sp->n_r > 127 || sp->n_r > n_s || !(sp->hi > sp->lo) ||
      (sp->family < 0 || sp->family > 5) || (sp->basis != 0 && sp->basis != 1))
    return ROMB_E_ARG;
  Trainer T;
  T.setup(*sp);
  const int nth = sp->n_threads > 0 ? sp->n_threads : std::max(1u, std::thread::hardware_concurrency());
  const int n_i = T.n_i, nm = (T.D + 1) * (T.D + 1);
  // snapshots (column s contiguous)
  std::vector<double> S((size_t)n_s * n_i);
  parallel_for(n_s, nth, [&](int s) {
    std::vector<double> M(nm);
    T.moments(samples + 4 * s, M.data());
    T.snapshot_from_moments(M.data(), &S[(size_t)s * n_i]);
  });
  // Gram matrix and its eigen-decomposition
  std::vector<double> G((size_t)n_s * n_s);
  parallel_for(n_s, nth, [&](int i) {
    for (int j = 0; j <= i; ++j) {
      const double* a = &S[(size_t)i * n_i];
      const double* b = &S[(size_t)j * n_i];
      double s = 0.0;
      for (int e = 0; e < n_i; ++e) s += a[e] * b[e];
      G[(size_t)i * n_s + j] = G[(size_t)j * n_s + i] = s;
    }
  });
  std::vector<double> w, V;
  jacobi_eig(n_s, G, w, V);
  std::vector<int> order(n_s);
  for (int i = 0; i < n_s; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  const int n_r = sp->n_r;
  // U_r columns = S v / sigma, then two passes of Gram-Schmidt
  std::vector<double> U((size_t)n_r * n_i, 0.0);
  parallel_for(n_r, nth, [&](int k) {
    const int j = order[k];
    double* u = &U[(size_t)k * n_i];
    for (int s = 0; s < n_s; ++s) {
      const double v = V[(size_t)s * n_s + j];
      const double* col = &S[(size_t)s * n_i];
      for (int e = 0; e < n_i; ++e) u[e] += v * col[e];
    }
  });
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < n_r; ++k) {
      double* u = &U[(size_t)k * n_i];
      for (int l = 0; l < k; ++l) {
        const double* v = &U[(size_t)l * n_i];
        double d = 0.0;
        for (int e = 0; e < n_i; ++e) d += u[e] * v[e];
        for (int e = 0; e < n_i; ++e) u[e] -= d * v[e];
      }
      double nrm = 0.0;
      for (int e = 0; e < n_i; ++e) nrm += u[e] * u[e];
      nrm = sqrt(nrm);
      if (!(nrm > 0.0)) return ROMB_E_NAN;
      for (int e = 0; e < n_i; ++e) u[e] /= nrm;
    }
  // magic points (Algorithm 3, interpolatory projection)
  std::vector<long long> magic(n_r);
  {
    auto argmax_abs = [&](const std::vector<double>& v) {
      int m = 0;
      for (int e = 1; e < n_i; ++e)
        if (fabs(v[e]) > fabs(v[m])) m = e;
      return m;
    };
    std::vector<double> res(U.begin(), U.begin() + n_i);
    magic[0] = argmax_abs(res);
    for (int j = 1; j < n_r; ++j) {
      std::vector<double> A((size_t)j * j), c(j);
      for (int a = 0; a < j; ++a) {
        for (int b = 0; b < j; ++b) A[(size_t)a * j + b] = U[(size_t)b * n_i + magic[a]];
        c[a] = U[(size_t)j * n_i + magic[a]];
      }
      LU lu;
      if (!lu.factor(j, A)) return ROMB_E_NAN;
      lu.solve(c.data());
      for (int e = 0; e < n_i; ++e) {
        double s = U[(size_t)j * n_i + e];
        for (int b = 0; b < j; ++b) s -= U[(size_t)b * n_i + e] * c[b];
        res[e] = s;
      }
      magic[j] = argmax_abs(res);
    }
  }
  // interpolation samples on the tensor GLL grid
  const int n1 = sp->r + 1;
  const int ng = n1 * n1 * n1 * n1;
  double g1d[12];
  gll_nodes01(sp->r, g1d);
  std::vector<double> Um((size_t)n_r * n_r);
  for (int a = 0; a < n_r; ++a)
    for (int b = 0; b < n_r; ++b) Um[(size_t)a * n_r + b] = U[(size_t)b * n_i + magic[a]];
  LU lu;
  if (!lu.factor(n_r, Um)) return ROMB_E_NAN;
  std::vector<double> A((size_t)n_r * ng);
  parallel_for(ng, nth, [&](int g) {
    const int i1 = g % n1, i2 = (g / n1) % n1, i3 = (g / (n1 * n1)) % n1, i4 = g / (n1 * n1 * n1);
    const double mu[4] = {sp->lo + (sp->hi - sp->lo) * g1d[i1], sp->lo + (sp->hi - sp->lo) * g1d[i2],
                          sp->lo + (sp->hi - sp->lo) * g1d[i3], sp->lo + (sp->hi - sp->lo) * g1d[i4]};
    std::vector<double> M(nm), b(n_r);
    T.moments(mu, M.data());
    for (int a = 0; a < n_r; ++a) b[a] = T.entry_from_moments(M.data(), (int)magic[a]);
    lu.solve(b.data());
    for (int a = 0; a < n_r; ++a) A[(size_t)a * ng + g] = b[a];
  });
  // I_Pi: untrimmed moments are e_0 e_0^T
  std::vector<double> Ipi(n_i);
  {
    std::vector<double> M(nm, 0.0);
    M[0] = 1.0;
    T.snapshot_from_moments(M.data(), Ipi.data());
  }
  RombForceModel force;
  if (romb_status fs = train_force_model(sp, samples, n_s, &force); fs != ROMB_OK) return fs;
  FILE* f = fopen(path, "wb");
  if (!f) return ROMB_E_ARG;
  unsigned char hdr[128];
  memset(hdr, 0, sizeof(hdr));
  memcpy(hdr, "ROMBDDC1", 8);
  const int32_t iv[8] = {2, sp->family, sp->basis, sp->p, sp->q, sp->r, n_r, 1};
  memcpy(hdr + 8, iv, 32);
  const double lohi[2] = {sp->lo, sp->hi};
  memcpy(hdr + 40, lohi, 16);
  const int64_t ni64 = n_i;
  memcpy(hdr + 56, &ni64, 8);
  bool ok = fwrite(hdr, 1, 128, f) == 128;
  ok = ok && fwrite(Ipi.data(), 8, n_i, f) == (size_t)n_i;
  ok = ok && fwrite(U.data(), 8, U.size(), f) == U.size();
  ok = ok && fwrite(A.data(), 8, A.size(), f) == A.size();
  ok = ok && fwrite(magic.data(), 8, n_r, f) == (size_t)n_r;
  ok = ok && write_force_section(f, force);
  fclose(f);
  return ok ? ROMB_OK : ROMB_E_ARG;
}
