// Host-side plan construction: quadrature, kernel prefactors, truncation radius, the
// FP64 gain/loss weight tables and the per-task phase tables (Secs. 3-4).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>

#include "dgfs_internal.h"

namespace dgfs {

static constexpr double kPi = 3.141592653589793238462643383279502884;

static bool supported_n(int N) {
  switch (N) {
    case 4: case 6: case 8: case 12: case 16: case 24: case 32: case 48: return true;
    default: return false;
  }
}

size_t real_size(const Plan& p) { return p.f32io() ? sizeof(float) : sizeof(double); }

// Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on the three-term
// recurrence of P_n, w = 2 / ((1 - x^2) P_n'(x)^2).  Writes n values into x and w (caller's
// arrays; no allocation, so the allocation-free entry point uses it too).
void gauss_legendre_rule(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  gauss_legendre_rule(n, x.data(), w.data());
}

// Gauss-Jacobi rule for the weight (1 + t)^beta on [-1, 1] (Golub-Welsch): the nodes are the
// eigenvalues of the symmetric tridiagonal Jacobi matrix of the weight, found by bisection on
// its Sturm sequence; the weights are mu_0 / sum_j p_j(x)^2 with p_j the orthonormal
// polynomials of the weight.
static void gauss_jacobi(int n, double beta, std::vector<double>& x, std::vector<double>& w) {
  const double a = 0.0, b = beta;
  std::vector<double> al(n), be(n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double s = 2.0 * i + a + b;
    al[i] = i == 0 ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (s * (s + 2.0));
    if (i >= 1) be[i] = 4.0 * i * (i + a) * (i + b) * (i + a + b) / (s * s * (s + 1.0) * (s - 1.0));
  }
  const double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) / std::tgamma(a + b + 2.0);
  auto below = [&](double xv) {  // number of eigenvalues below xv
    int c = 0;
    double d = al[0] - xv;
    if (d < 0) ++c;
    for (int i = 1; i < n; ++i) {
      if (d == 0.0) d = 1e-300;
      d = (al[i] - xv) - be[i] / d;
      if (d < 0) ++c;
    }
    return c;
  };
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (below(mid) > j) hi = mid; else lo = mid;
    }
    const double xv = 0.5 * (lo + hi);
    double p0 = 1.0, sum = 1.0;
    if (n > 1) {
      double p1 = (xv - al[0]) / std::sqrt(be[1]);
      sum += p1 * p1;
      for (int i = 1; i < n - 1; ++i) {
        const double p2 = ((xv - al[i]) * p1 - std::sqrt(be[i]) * p0) / std::sqrt(be[i + 1]);
        sum += p2 * p2;
        p0 = p1;
        p1 = p2;
      }
    }
    x[j] = xv;
    w[j] = mu0 / sum;
  }
}

// Built-in spherical designs with equal weights 4 pi / M: octahedron (M = 6),
// icosahedron (M = 12), icosahedron and dodecahedron together (M = 32).
static bool builtin_design(int M, std::vector<double>& s) {
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  s.clear();
  auto push = [&](double a, double b, double c) {
    const double n = std::sqrt(a * a + b * b + c * c);
    s.push_back(a / n);
    s.push_back(b / n);
    s.push_back(c / n);
  };
  auto icosa = [&]() {
    for (double a : {1.0, -1.0})
      for (double b : {g, -g}) {
        push(0.0, a, b);
        push(a, b, 0.0);
        push(b, 0.0, a);
      }
  };
  if (M == 6) {
    for (int d = 0; d < 3; ++d)
      for (double sg : {1.0, -1.0}) push(d == 0 ? sg : 0.0, d == 1 ? sg : 0.0, d == 2 ? sg : 0.0);
    return true;
  }
  if (M == 12) {
    icosa();
    return true;
  }
  if (M == 32) {
    icosa();
    for (double a : {1.0, -1.0})
      for (double b : {1.0, -1.0})
        for (double c : {1.0, -1.0}) push(a, b, c);
    const double ig = 1.0 / g;
    for (double a : {ig, -ig})
      for (double b : {g, -g}) {
        push(0.0, a, b);
        push(a, b, 0.0);
        push(b, 0.0, a);
      }
    return true;
  }
  return false;
}

// b_ij of Eq. NVSS
static double vss_prefactor(double mi, double mj, double omega, double alpha) {
  const double mu = mi * mj / (mi + mj);
  return alpha / (std::sqrt(1.0 + mi / mj) * std::pow(mu, omega - 0.5) * std::pow(2.0, 1.0 + alpha) *
                  std::tgamma(2.5 - omega) * kPi);
}

static int centred_mode(int n, int N) { return n < N / 2 ? n : n - N; }

// Gauss-Jordan inverse of a small symmetric positive definite matrix (FP64)
static bool invert(int n, const double* a, double* inv) {
  double m[6][12];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) m[r][c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[piv][c])) piv = r;
    if (!(std::fabs(m[piv][c]) > 0.0)) return false;
    for (int k = 0; k < 2 * n; ++k) std::swap(m[c][k], m[piv][k]);
    const double d = m[c][c];
    for (int k = 0; k < 2 * n; ++k) m[c][k] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const double f = m[r][c];
        for (int k = 0; k < 2 * n; ++k) m[r][k] -= f * m[c][k];
      }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) inv[r * n + c] = m[r][n + c];
  return true;
}

// Conservation blocks of Eq. consv on the cell-centred grid: for a self pair the rows
// (1, v_x, v_y, v_z, |v|^2) acting on Q_ii; for a cross pair the rows acting on [Q_ij; Q_ji]:
// mass of each half, (m_i w_ij v_d | m_j w_ji v_d), (m_i w_ij |v|^2 | m_j w_ji |v|^2), w = 1/b.
static int build_conservation(Plan& p) {
  const int N = p.N, s = p.s;
  const double dv = 2.0 * p.L / N;
  // grid moments sum_n v^a over one axis
  double m0 = N, m1 = 0, m2 = 0, m3 = 0, m4 = 0;
  for (int n = 0; n < N; ++n) {
    const double v = -p.L + (n + 0.5) * dv;
    m1 += v;
    m2 += v * v;
    m3 += v * v * v;
    m4 += v * v * v * v;
  }
  const double N2 = double(N) * N, N3 = N2 * N;
  // sums over the 3D grid of products of the basic rows 1, vx, vy, vz, |v|^2
  double G[5][5] = {};
  G[0][0] = N3;
  for (int d = 0; d < 3; ++d) {
    G[0][1 + d] = G[1 + d][0] = m1 * N2;
    for (int e = 0; e < 3; ++e) G[1 + d][1 + e] = d == e ? m2 * N2 : m1 * m1 * N;
    // sum vd |v|^2 = sum vd^3 N^2 + sum vd * (sum of the other two squares)
    G[1 + d][4] = G[4][1 + d] = m3 * N2 + 2.0 * m1 * m2 * N;
  }
  G[0][4] = G[4][0] = 3.0 * m2 * N2;
  G[4][4] = 3.0 * m4 * N2 + 6.0 * m2 * m2 * N;
  for (int i = 0; i < s; ++i)
    for (int j = i; j < s; ++j) {
      ConsBlock cb{};
      cb.i = i;
      cb.j = j;
      double A[36] = {};
      if (i == j) {
        cb.rows = 5;
        for (int r = 0; r < 5; ++r)
          for (int c = 0; c < 5; ++c) A[r * 5 + c] = G[r][c];
      } else {
        cb.rows = 6;
        cb.a = p.mass[i] / p.b[i * s + j];
        cb.b = p.mass[j] / p.b[j * s + i];
        // row k of the stacked block = (alpha_k e_k | beta_k e_k) over the basic rows:
        // k=0: (1 | 0), k=1: (0 | 1), k=2..4: (a v | b v), k=5: (a |v|^2 | b |v|^2)
        const int basic[6] = {0, 0, 1, 2, 3, 4};
        const double al[6] = {1.0, 0.0, cb.a, cb.a, cb.a, cb.a};
        const double be[6] = {0.0, 1.0, cb.b, cb.b, cb.b, cb.b};
        for (int r = 0; r < 6; ++r)
          for (int c = 0; c < 6; ++c)
            A[r * 6 + c] = (al[r] * al[c] + be[r] * be[c]) * G[basic[r]][basic[c]];
      }
      if (!invert(cb.rows, A, cb.minv)) return DGFS_ERR_INVALID_ARG;
      p.cons.push_back(cb);
    }
  return DGFS_OK;
}

int build_plan(const dgfs_plan_desc* d, Plan& p) {
  if (!d) return DGFS_ERR_INVALID_ARG;
  if (!supported_n(d->N)) return DGFS_ERR_UNSUPPORTED_N;
  if (!(d->L > 0.0) || d->s < 1 || d->s > 8 || !d->mass || !d->omega || !d->alpha) return DGFS_ERR_INVALID_ARG;
  if (d->N_rho < 1 || d->N_rho > 4096 || d->M < 1 || d->max_batch < 0) return DGFS_ERR_INVALID_ARG;
  if (d->precision != DGFS_FP64 && d->precision != DGFS_FP32 && d->precision != DGFS_BF16X3) return DGFS_ERR_INVALID_ARG;
  if ((d->flags & ~(DGFS_CONSERVE | DGFS_SUM_SPECIES | DGFS_LOSS_ACCURATE | DGFS_PER_PAIR_R)) != 0u)
    return DGFS_ERR_INVALID_ARG;
  if ((d->flags & DGFS_PER_PAIR_R) && d->R > 0.0) return DGFS_ERR_INVALID_ARG;
  const int s = d->s;
  p.N = d->N;
  p.L = d->L;
  p.s = s;
  p.N_rho = d->N_rho;
  p.precision = d->precision;
  p.flags = d->flags;
  p.max_batch = d->max_batch;
  p.mass.assign(d->mass, d->mass + s);
  p.omega.assign(d->omega, d->omega + s * s);
  p.alpha.assign(d->alpha, d->alpha + s * s);
  for (int i = 0; i < s; ++i)
    if (!(p.mass[i] > 0.0) || !std::isfinite(p.mass[i])) return DGFS_ERR_INVALID_ARG;
  for (int k = 0; k < s * s; ++k) {
    if (!(p.omega[k] >= 0.5 && p.omega[k] <= 1.0)) return DGFS_ERR_INVALID_ARG;
    if (!(p.alpha[k] >= 1.0 && p.alpha[k] <= 2.0)) return DGFS_ERR_INVALID_ARG;
    if (p.alpha[k] != 1.0) p.vss = true;
  }
  // the tensor-core path evaluates the sigma-independent (VHS) gain weight on N <= 24
  if (p.precision == DGFS_BF16X3) {
    if (!gemm_supported_n(p.N)) return DGFS_ERR_UNSUPPORTED_N;
    if (p.vss) return DGFS_ERR_UNSUPPORTED;
  }
  p.kappa.assign(s * s, 1.0);
  if (d->kappa)
    for (int k = 0; k < s * s; ++k) {
      if (!std::isfinite(d->kappa[k])) return DGFS_ERR_INVALID_ARG;
      p.kappa[k] = d->kappa[k];
    }
  p.b.assign(s * s, 0.0);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      p.b[i * s + j] = d->b_override ? d->b_override[i * s + j]
                                     : vss_prefactor(p.mass[i], p.mass[j], p.omega[i * s + j], p.alpha[i * s + j]);
      if (!std::isfinite(p.b[i * s + j])) return DGFS_ERR_INVALID_ARG;
    }
  if (!std::isfinite(d->R)) return DGFS_ERR_INVALID_ARG;
  // sphere rule
  p.M = d->M;
  if (d->sigma) {
    p.sigma.assign(d->sigma, d->sigma + 3 * d->M);
    for (int m = 0; m < d->M; ++m) {
      const double* v = &p.sigma[3 * m];
      const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (!(std::fabs(n - 1.0) < 1e-9)) return DGFS_ERR_INVALID_ARG;
    }
  } else if (!builtin_design(d->M, p.sigma)) {
    return DGFS_ERR_INVALID_ARG;
  }
  if (d->w_sigma) p.w_sigma.assign(d->w_sigma, d->w_sigma + d->M);
  else p.w_sigma.assign(d->M, 4.0 * kPi / d->M);
  for (int m = 0; m < d->M; ++m)
    if (!std::isfinite(p.w_sigma[m])) return DGFS_ERR_INVALID_ARG;
  // radial truncation: R = 2S, S the largest support allowed by Eq. domain for every pair
  // (S_ij for the pair alone, the minimum over the pairs for the common R)
  std::vector<double> S_pair(size_t(s) * s);
  double S = 1e300;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      const double cj = p.mass[j] / (p.mass[i] + p.mass[j]);
      const double den = std::max(4.0 * cj, 2.0) + std::sqrt(1.0 + p.mass[j] / p.mass[i]) + 1.0;
      S_pair[size_t(i) * s + j] = 2.0 * p.L / den;
      S = std::min(S, S_pair[size_t(i) * s + j]);
    }
  p.R = d->R > 0.0 ? d->R : 2.0 * S;
  std::vector<double> x, w;
  gauss_legendre(p.N_rho, x, w);
  p.rho.resize(p.N_rho);
  p.w_rho.resize(p.N_rho);
  for (int q = 0; q < p.N_rho; ++q) {
    p.rho[q] = 0.5 * p.R * (x[q] + 1.0);
    p.w_rho[q] = 0.5 * p.R * w[q];
  }
  const bool per_pair = (p.flags & DGFS_PER_PAIR_R) != 0u;
  p.pair_R.resize(size_t(s) * s);
  p.rho_p.resize(size_t(s) * s * p.N_rho);
  p.w_rho_p.resize(size_t(s) * s * p.N_rho);
  for (int o = 0; o < s * s; ++o) {
    p.pair_R[o] = per_pair ? 2.0 * S_pair[o] : p.R;
    for (int q = 0; q < p.N_rho; ++q) {
      p.rho_p[size_t(o) * p.N_rho + q] = 0.5 * p.pair_R[o] * (x[q] + 1.0);
      p.w_rho_p[size_t(o) * p.N_rho + q] = 0.5 * p.pair_R[o] * w[q];
    }
  }
  // Size of the Gauss-Jacobi rule in t of the VSS gain weight (F after Eq. GG, "precomputed
  // to high accuracy"): the integrand's bandwidth grows with the largest argument
  // a = pi rho c_j |k| / L over the table (largest rho node, |k| = sqrt(3) N / 2).  A
  // 64-point rule agrees with the converged integral to 1e-13 of its bound 2^alpha / alpha
  // up to a = 80; beyond, the size grows linearly with a (0.6 a + 14 points were measured
  // to converge; 0.75 a + 16 rounded up to a multiple of 32 keeps a margin).
  {
    double a_max = 0.0;
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) {
        const int o = i * s + j;
        const double cj = p.mass[j] / (p.mass[i] + p.mass[j]);
        for (int q = 0; q < p.N_rho; ++q)
          a_max = std::max(a_max, kPi * p.rho_p[size_t(o) * p.N_rho + q] * cj * std::sqrt(3.0) * 0.5 * p.N / p.L);
      }
    p.vss_a_max = a_max;
    p.n_t = a_max <= 80.0 ? 64 : 32 * int(std::ceil((0.75 * a_max + 16.0) / 32.0));
  }

  // antipodal partner of every direction (equal weights required for the pair reuse)
  const int M = p.M;
  std::vector<int> anti(M, -1);
  bool antipodal = true;
  for (int m = 0; m < M; ++m) {
    for (int k = 0; k < M; ++k) {
      const double* a = &p.sigma[3 * m];
      const double* c = &p.sigma[3 * k];
      if (std::fabs(a[0] + c[0]) < 1e-12 && std::fabs(a[1] + c[1]) < 1e-12 && std::fabs(a[2] + c[2]) < 1e-12 &&
          std::fabs(p.w_sigma[m] - p.w_sigma[k]) <= 1e-14 * std::fabs(p.w_sigma[m])) {
        anti[m] = k;
        break;
      }
    }
    if (anti[m] < 0) antipodal = false;
  }
  p.antipodal = antipodal;
  // slots of the VSS gain table: F(k, rho, -sigma) = conj F(k, rho, sigma) (the sphere
  // integral of Eq. GG with the plane wave's sign flipped), so a direction whose negation owns
  // a slot at a lower index reads that slot conjugated; every other direction owns a slot
  p.fslot.assign(M, -1);
  p.n_fslot = 0;
  for (int m = 0; m < M; ++m) {
    const double* a = &p.sigma[3 * m];
    for (int r = 0; r < m && p.fslot[m] < 0; ++r) {
      const double* c = &p.sigma[3 * r];
      if (!(p.fslot[r] & 1) && std::fabs(a[0] + c[0]) < 1e-12 && std::fabs(a[1] + c[1]) < 1e-12 &&
          std::fabs(a[2] + c[2]) < 1e-12)
        p.fslot[m] = p.fslot[r] | 1;
    }
    if (p.fslot[m] < 0) p.fslot[m] = 2 * p.n_fslot++;
  }
  auto positive = [&](int m) {
    const double* a = &p.sigma[3 * m];
    for (int dd = 0; dd < 3; ++dd) {
      if (a[dd] > 1e-12) return true;
      if (a[dd] < -1e-12) return false;
    }
    return true;
  };

  // tasks: unordered pairs with (i,j)/(j,i) reuse and halved self pairs when the rule is
  // antipodal; every ordered pair with the full rule otherwise
  p.tasks.clear();
  p.groups.clear();
  p.ent_w.clear();
  p.ent_sigma.clear();
  p.ent_m.clear();
  p.ent_ysh.clear();
  p.max_ent = 0;
  // the (i,j)/(j,i) product reuse needs one radial rule for both pairs
  const bool reuse = antipodal && !per_pair;
  for (int i = 0; i < s; ++i) {
    for (int j = reuse ? i : 0; j < s; ++j) {
      std::vector<std::pair<int, double>> ent;
      for (int m = 0; m < M; ++m) {
        if (antipodal && i == j) {
          // VHS: p(sigma) = p(-sigma) and F does not depend on sigma -> doubled weight;
          // VSS: the weight stays and the table adds F(sigma) + F(-sigma)
          if (positive(m)) ent.push_back({m, (p.vss ? 1.0 : 2.0) * p.w_sigma[m]});
        } else {
          ent.push_back({m, p.w_sigma[m]});
        }
      }
      // order by sigma_x (groups share the x pass), then by sigma_y (runs of equal sigma_y
      // inside a group share the y pass as well)
      std::stable_sort(ent.begin(), ent.end(), [&](const std::pair<int, double>& a, const std::pair<int, double>& c) {
        const double* u = &p.sigma[3 * a.first];
        const double* v = &p.sigma[3 * c.first];
        if (std::fabs(u[0] - v[0]) > 1e-12) return u[0] < v[0];
        return u[1] < v[1] - 1e-12;
      });
      TaskDesc tk;
      tk.i = i;
      tk.j = j;
      tk.out0 = i * s + j;
      tk.out1 = (reuse && i != j) ? j * s + i : -1;
      tk.ent_off = int(p.ent_w.size());
      tk.n_ent = int(ent.size());
      tk.grp_off = int(p.groups.size());
      // groups share sigma_x (VHS); with VSS every entry needs its own forward transform and
      // is its own group
      int first = 0;
      for (int e = 1; e <= int(ent.size()); ++e) {
        if (e == int(ent.size()) || p.vss ||
            std::fabs(p.sigma[3 * ent[e].first] - p.sigma[3 * ent[first].first]) > 1e-12) {
          p.groups.push_back({first, e - first});
          first = e;
        }
      }
      tk.n_grp = int(p.groups.size()) - tk.grp_off;
      for (size_t k = 0; k < ent.size(); ++k) {
        const auto& e = ent[k];
        p.ent_w.push_back(e.second);
        p.ent_sigma.push_back(e.first);
        // a halved self pair reads F(sigma) + F(-sigma) = 2 Re F(sigma): slot without the
        // conjugation bit, plus the antipode's code as the marker of the sum
        const bool halved = antipodal && i == j;
        p.ent_m.push_back(halved ? (p.fslot[e.first] & ~1) : p.fslot[e.first]);
        p.ent_m.push_back(antipodal ? p.fslot[anti[e.first]] : -1);
        bool ysh = false;
        if (k > 0 && !p.vss) {
          const double* u = &p.sigma[3 * ent[k - 1].first];
          const double* v = &p.sigma[3 * e.first];
          ysh = std::fabs(u[0] - v[0]) <= 1e-12 && std::fabs(u[1] - v[1]) <= 1e-12;
        }
        p.ent_ysh.push_back(ysh ? 1 : 0);
      }
      p.max_ent = std::max(p.max_ent, tk.n_ent);
      p.tasks.push_back(tk);
    }
  }
  if (p.flags & DGFS_CONSERVE) {
    for (int k = 0; k < s * s; ++k)
      if (!(std::fabs(p.b[k]) > 0.0)) return DGFS_ERR_INVALID_ARG;
    if (int rc = build_conservation(p)) return rc;
  }
  return DGFS_OK;
}

static int dalloc(Plan& p, void** dptr, size_t bytes) {
  if (cudaMallocAsync(dptr, bytes, p.home) != cudaSuccess) {
    cudaGetLastError();
    *dptr = nullptr;
    return DGFS_ERR_OOM;
  }
  return DGFS_OK;
}

template <typename V>
static int upload(Plan& p, const V* host, size_t count, void** dptr, size_t& total) {
  const size_t bytes = count * sizeof(V);
  if (int rc = dalloc(p, dptr, bytes)) return rc;
  if (cudaMemcpyAsync(*dptr, host, bytes, cudaMemcpyHostToDevice, p.home) != cudaSuccess) return DGFS_ERR_CUDA;
  total += bytes;
  return DGFS_OK;
}

// Device memory of the plan is stream-ordered on the plan's own stream (cudaMallocAsync /
// cudaFreeAsync), so creating and destroying plans never synchronises other streams; the
// function returns after the plan's stream has finished the uploads and table builds.
int upload_plan(Plan& p) {
  const int N = p.N, s = p.s, NR = p.N_rho;
  const size_t N3 = size_t(N) * N * N;
  const int P = s * s;
  if (!p.home && cudaStreamCreateWithFlags(&p.home, cudaStreamNonBlocking) != cudaSuccess) return DGFS_ERR_CUDA;
  if (!p.last_eval && cudaEventCreateWithFlags(&p.last_eval, cudaEventDisableTiming) != cudaSuccess)
    return DGFS_ERR_CUDA;
  // radial rule of the pair (i, j): node q of pair o
  auto rho_of = [&](int o, int q) { return p.rho_p[size_t(o) * NR + q]; };
  auto w_rho_of = [&](int o, int q) { return p.w_rho_p[size_t(o) * NR + q]; };
  // radial rule of the loss weight per pair: the gain's nodes, or (DGFS_LOSS_ACCURATE) 4 N_rho
  // Gauss-Legendre nodes of its own on [0, R_ij]
  const bool acc_loss = (p.flags & DGFS_LOSS_ACCURATE) != 0u;
  const int NL = acc_loss ? 4 * NR : NR;
  std::vector<double> lx, lwt;
  if (acc_loss) gauss_legendre(NL, lx, lwt);
  // per (pair, rho) constants of the weight tables: gain prefactor and sinc scale, loss
  // prefactor and sinc scale
  std::vector<double> fcoef(size_t(P) * NR * 2), gcoef(size_t(P) * NL), gscale(size_t(P) * NL);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      const int o = i * s + j;
      const double b = p.b[o], om = p.omega[o], al = p.alpha[o];
      const double cj = p.mass[j] / (p.mass[i] + p.mass[j]);
      for (int q = 0; q < NR; ++q) {
        const double rp = std::pow(rho_of(o, q), 4.0 - 2.0 * om);
        fcoef[2 * (size_t(o) * NR + q)] = w_rho_of(o, q) * 4.0 * kPi * b * rp / double(N3);
        fcoef[2 * (size_t(o) * NR + q) + 1] = kPi * rho_of(o, q) * cj / p.L;
      }
      for (int q = 0; q < NL; ++q) {
        const double lr = acc_loss ? 0.5 * p.pair_R[o] * (lx[q] + 1.0) : rho_of(o, q);
        const double lw = acc_loss ? 0.5 * p.pair_R[o] * lwt[q] : w_rho_of(o, q);
        gcoef[size_t(o) * NL + q] = 8.0 * kPi * kPi * std::pow(2.0, al) / al * b * lw * std::pow(lr, 4.0 - 2.0 * om);
        gscale[size_t(o) * NL + q] = kPi * lr / p.L;
      }
    }
  // phase factors exp(i pi shift_d k / L) per task, radial node, entry, role, axis
  const int NT = int(p.tasks.size());
  const size_t nph = size_t(NT) * NR * p.max_ent * 2 * 3 * N;
  std::vector<std::complex<double>> ph(nph, std::complex<double>(0.0, 0.0));
  for (int t = 0; t < NT; ++t) {
    const TaskDesc& tk = p.tasks[t];
    const double mi = p.mass[tk.i], mj = p.mass[tk.j];
    const double ci = mi / (mi + mj), cj = mj / (mi + mj);
    for (int q = 0; q < NR; ++q)
      for (int e = 0; e < tk.n_ent; ++e) {
        const double* sg = &p.sigma[3 * p.ent_sigma[tk.ent_off + e]];
        const double rq = rho_of(tk.out0, q);
        for (int role = 0; role < 2; ++role) {
          const double c = role == 0 ? rq * cj : -rq * ci;
          for (int ax = 0; ax < 3; ++ax) {
            const double sh = c * sg[ax];
            std::complex<double>* dst = &ph[((((size_t(t) * NR + q) * p.max_ent + e) * 2 + role) * 3 + ax) * N];
            for (int n = 0; n < N; ++n) {
              const double arg = kPi * sh * centred_mode(n, N) / p.L;
              dst[n] = std::complex<double>(std::cos(arg), std::sin(arg));
            }
          }
        }
      }
  }
  std::vector<float> phf;
  std::vector<double> phd;
  std::vector<uint16_t> mats;
  if (p.precision == DGFS_BF16X3) build_gemm_images(p, ph, mats);
  if (p.f32io()) {
    phf.resize(2 * nph);
    for (size_t n = 0; n < nph; ++n) {
      phf[2 * n] = float(ph[n].real());
      phf[2 * n + 1] = float(ph[n].imag());
    }
  } else {
    phd.resize(2 * nph);
    for (size_t n = 0; n < nph; ++n) {
      phd[2 * n] = ph[n].real();
      phd[2 * n + 1] = ph[n].imag();
    }
  }
  size_t total = 0;
  int rc;
  void *d_fcoef = nullptr, *d_gcoef = nullptr, *d_gscale = nullptr;
  size_t tmp = 0;
  // coefficient arrays the table kernels read: freed (stream-ordered) when this function
  // returns, on every path
  struct TempBuffers {
    cudaStream_t st;
    std::vector<void*> v;
    ~TempBuffers() {
      for (void* t : v)
        if (t) cudaFreeAsync(t, st);
    }
  } temps{p.home, {}};
  auto up_tmp = [&](const auto* host, size_t count, void** d) {
    const int r = upload(p, host, count, d, tmp);
    if (*d) temps.v.push_back(*d);
    return r;
  };
  if ((rc = dalloc(p, (void**)&p.d_Gm, size_t(P) * N3 * sizeof(double)))) return rc;
  total += size_t(P) * N3 * sizeof(double);
  if ((rc = up_tmp(gcoef.data(), gcoef.size(), &d_gcoef))) return rc;
  if ((rc = up_tmp(gscale.data(), gscale.size(), &d_gscale))) return rc;
  if (!p.vss) {
    if ((rc = dalloc(p, (void**)&p.d_Fw, size_t(P) * NR * N3 * sizeof(double)))) return rc;
    total += size_t(P) * NR * N3 * sizeof(double);
    if ((rc = up_tmp(fcoef.data(), fcoef.size(), &d_fcoef))) return rc;
    if ((rc = launch_vhs_tables(p, static_cast<double*>(d_fcoef), static_cast<double*>(d_gcoef),
                                static_cast<double*>(d_gscale), NL)))
      return rc;
  } else {
    // VSS gain weights: prefactor w_q 2 pi b rho^(4-2 omega) / N^3 and the scale of a per
    // (pair, rho); a Gauss-Jacobi rule of p.n_t points per pair; representatives of antipodal pairs
    const int n_t = p.n_t;
    std::vector<double> vcoef(size_t(P) * NR * 2), gj(size_t(P) * 3 * n_t);
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) {
        const int o = i * s + j;
        const double cj = p.mass[j] / (p.mass[i] + p.mass[j]);
        for (int q = 0; q < NR; ++q) {
          vcoef[2 * (size_t(o) * NR + q)] =
              w_rho_of(o, q) * 2.0 * kPi * p.b[o] * std::pow(rho_of(o, q), 4.0 - 2.0 * p.omega[o]) / double(N3);
          vcoef[2 * (size_t(o) * NR + q) + 1] = kPi * rho_of(o, q) * cj / p.L;
        }
        std::vector<double> tx, tw;
        gauss_jacobi(n_t, p.alpha[o] - 1.0, tx, tw);
        for (int k = 0; k < n_t; ++k) {
          gj[size_t(o) * 3 * n_t + k] = tx[k];
          gj[size_t(o) * 3 * n_t + n_t + k] = tw[k];
          gj[size_t(o) * 3 * n_t + 2 * n_t + k] = std::sqrt(std::max(0.0, 1.0 - tx[k] * tx[k]));
        }
      }
    // the direction that owns each slot
    std::vector<int> reps;
    for (int m = 0; m < p.M; ++m)
      if (!(p.fslot[m] & 1)) reps.push_back(m);
    void *d_vc = nullptr, *d_gj = nullptr, *d_sg = nullptr, *d_reps = nullptr;
    if ((rc = dalloc(p, (void**)&p.d_Fv, size_t(P) * NR * p.n_fslot * N3 * sizeof(double2)))) return rc;
    total += size_t(P) * NR * p.n_fslot * N3 * sizeof(double2);
    if ((rc = up_tmp(vcoef.data(), vcoef.size(), &d_vc))) return rc;
    if ((rc = up_tmp(gj.data(), gj.size(), &d_gj))) return rc;
    if ((rc = up_tmp(p.sigma.data(), p.sigma.size(), &d_sg))) return rc;
    if ((rc = up_tmp(reps.data(), reps.size(), &d_reps))) return rc;
    // FP32 plans build the table from a grid of the two-argument function Phi_alpha(p, q) (one
    // grid per distinct alpha, spacing 0.03: 4 x 4-point interpolation within 3e-9 of the
    // integral's bound at arguments up to 65); FP64 plans, and grids that would be too large,
    // sum the Gauss-Jacobi rule for every entry
    VssGrid gr;
    gr.h = 0.03;
    const double A = p.vss_a_max;
    std::vector<double> alphas;
    std::vector<int> grid_of_pair(P);
    for (int o = 0; o < P; ++o) {
      int g = -1;
      for (size_t a = 0; a < alphas.size(); ++a)
        if (alphas[a] == p.alpha[o]) g = int(a);
      if (g < 0) {
        g = int(alphas.size());
        alphas.push_back(p.alpha[o]);
      }
      grid_of_pair[o] = g;
    }
    gr.p0 = -A - 2.0 * gr.h;
    gr.q0 = -2.0 * gr.h;
    gr.np = int(std::ceil((2.0 * A + 4.0 * gr.h) / gr.h)) + 2;
    gr.nq = int(std::ceil((A + 4.0 * gr.h) / gr.h)) + 2;
    const size_t grid_bytes = alphas.size() * size_t(gr.np) * gr.nq * sizeof(double2);
    const size_t direct_terms = size_t(P) * NR * reps.size() * N3;
    p.vss_grid = p.f32io() && grid_bytes <= (size_t(1) << 30) && size_t(gr.np) * gr.nq < direct_terms;
    if (p.vss_grid) {
      std::vector<double> gja(alphas.size() * 3 * n_t);
      for (size_t a = 0; a < alphas.size(); ++a) {
        int o = 0;
        while (grid_of_pair[o] != int(a)) ++o;
        std::copy(gj.begin() + size_t(o) * 3 * n_t, gj.begin() + size_t(o + 1) * 3 * n_t, gja.begin() + a * 3 * n_t);
      }
      void *d_phi = nullptr, *d_gja = nullptr, *d_gop = nullptr;
      if ((rc = dalloc(p, &d_phi, grid_bytes))) return rc;
      temps.v.push_back(d_phi);
      if ((rc = up_tmp(gja.data(), gja.size(), &d_gja))) return rc;
      if ((rc = up_tmp(grid_of_pair.data(), grid_of_pair.size(), &d_gop))) return rc;
      if ((rc = launch_vss_tables_grid(p, static_cast<double*>(d_vc), static_cast<double2*>(d_phi),
                                       static_cast<double*>(d_gja), int(alphas.size()), n_t, gr,
                                       static_cast<int*>(d_gop), static_cast<double*>(d_sg),
                                       static_cast<int*>(d_reps), int(reps.size()))))
        return rc;
    } else if ((rc = launch_vss_tables(p, static_cast<double*>(d_vc), static_cast<double*>(d_gj), n_t,
                                       static_cast<double*>(d_sg), static_cast<int*>(d_reps), int(reps.size())))) {
      return rc;
    }
    if ((rc = launch_loss_table(p, static_cast<double*>(d_gcoef), static_cast<double*>(d_gscale), NL))) return rc;
    if ((rc = upload(p, p.ent_m.data(), p.ent_m.size(), (void**)&p.d_ent_m, total))) return rc;
  }
  if (p.f32io()) {
    // the FP32 kernel reads FP32 gain tables: each FP64 value rounded once here instead of
    // converted per element in the kernel (GB300's FP64 rate is a small fraction of its FP32
    // rate); with an antipodal design a self pair's slots take F(sigma) + F(-sigma) =
    // 2 Re F(sigma), the sum the FP64 kernel forms, so the FP32 results are unchanged bit for bit
    const size_t nF = size_t(P) * NR * (p.vss ? size_t(p.n_fslot) : 1) * N3;
    if (p.vss) {
      if ((rc = dalloc(p, (void**)&p.d_Fvf, nF * sizeof(float2)))) return rc;
    } else {
      if ((rc = dalloc(p, (void**)&p.d_Fwf, nF * sizeof(float)))) return rc;
    }
    if ((rc = launch_gain_tables_f32(p, p.antipodal ? 1 : 0))) return rc;
    const size_t nG = size_t(P) * N3;
    if ((rc = dalloc(p, (void**)&p.d_Gmf, nG * sizeof(float)))) return rc;
    if ((rc = launch_to_f32(p, p.d_Gm, p.d_Gmf, nG))) return rc;
    cudaFreeAsync(p.d_Gm, p.home);
    p.d_Gm = nullptr;
    total = total - nG * sizeof(double) + nG * sizeof(float);
    if (p.vss) {
      cudaFreeAsync(p.d_Fv, p.home);
      p.d_Fv = nullptr;
      total = total - nF * sizeof(double2) + nF * sizeof(float2);
    } else {
      cudaFreeAsync(p.d_Fw, p.home);
      p.d_Fw = nullptr;
      total = total - nF * sizeof(double) + nF * sizeof(float);
    }
  }
  if ((rc = upload(p, p.ent_w.data(), p.ent_w.size(), (void**)&p.d_ent_w, total))) return rc;
  if ((rc = upload(p, p.tasks.data(), p.tasks.size(), (void**)&p.d_tasks, total))) return rc;
  if ((rc = upload(p, p.groups.data(), p.groups.size(), (void**)&p.d_groups, total))) return rc;
  if ((rc = upload(p, p.ent_ysh.data(), p.ent_ysh.size(), (void**)&p.d_ent_ysh, total))) return rc;
  if (!mats.empty() && (rc = upload(p, mats.data(), mats.size(), (void**)&p.d_mats, total))) return rc;
  if (p.f32io()) {
    if ((rc = upload(p, phf.data(), phf.size(), &p.d_phase, total))) return rc;
  } else {
    if ((rc = upload(p, phd.data(), phd.size(), &p.d_phase, total))) return rc;
  }
  if ((rc = upload(p, p.kappa.data(), p.kappa.size(), (void**)&p.d_kappa, total))) return rc;
  if (!p.cons.empty() && (rc = upload(p, p.cons.data(), p.cons.size(), (void**)&p.d_cons, total))) return rc;
  p.table_bytes = total;
  if ((p.flags & DGFS_SUM_SPECIES) && p.max_batch > 0) {
    if ((rc = dalloc(p, &p.d_Qfull, size_t(p.max_batch) * s * s * N3 * real_size(p)))) return rc;
  }
  // the workspace between two guard blocks of a fixed byte pattern: dgfs_plan_check reads
  // them back to detect a kernel write outside the workspace
  if ((rc = dalloc(p, &p.d_scratch_raw, p.scratch_bytes + 2 * Plan::kGuardBytes))) return rc;
  p.d_scratch = static_cast<char*>(p.d_scratch_raw) + Plan::kGuardBytes;
  if (cudaMemsetAsync(p.d_scratch_raw, Plan::kGuardByte, Plan::kGuardBytes, p.home) != cudaSuccess ||
      cudaMemsetAsync(static_cast<char*>(p.d_scratch) + p.scratch_bytes, Plan::kGuardByte, Plan::kGuardBytes,
                      p.home) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  if ((rc = dalloc(p, (void**)&p.d_counter, 256))) return rc;
  // work counter and device status word start at zero
  if (cudaMemsetAsync(p.d_counter, 0, 256, p.home) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  // the host arrays above must outlive the copies
  if (cudaStreamSynchronize(p.home) != cudaSuccess) return DGFS_ERR_CUDA;
  return DGFS_OK;
}

void free_plan(Plan& p) {
  void* ptrs[] = {p.d_Fw,      p.d_Gm,      p.d_ent_w,   p.d_phase, p.d_tasks, p.d_groups, p.d_Fv,
                  p.d_scratch_raw, p.d_stage_f, p.d_stage_Q, p.d_cons, p.d_kappa, p.d_Qfull, p.d_ent_m,
                  p.d_counter, p.d_rk,      p.d_ent_ysh, p.d_Fwf,    p.d_Fvf,   p.d_Gmf,   p.d_mats,
                  p.d_scratch2_raw, p.d_counter2};
  if (p.home) {
    for (void* q : ptrs)
      if (q) cudaFreeAsync(q, p.home);
    cudaStreamSynchronize(p.home);
    cudaStreamDestroy(p.home);
    p.home = nullptr;
  }
  if (p.last_eval) {
    cudaEventDestroy(p.last_eval);
    p.last_eval = nullptr;
  }
  for (int k = 0; k < Plan::kMaxChunks; ++k) {
    if (p.ev_h2d[k]) cudaEventDestroy(p.ev_h2d[k]);
    if (p.ev_done[k]) cudaEventDestroy(p.ev_done[k]);
    p.ev_h2d[k] = p.ev_done[k] = nullptr;
  }
  if (p.ev_start) cudaEventDestroy(p.ev_start);
  if (p.h2d) cudaStreamDestroy(p.h2d);
  if (p.eval2) cudaStreamDestroy(p.eval2);
  p.eval2 = nullptr;
  p.d_scratch2_raw = p.d_scratch2 = nullptr;
  p.d_counter2 = nullptr;
  if (p.d2h) cudaStreamDestroy(p.d2h);
  p.ev_start = nullptr;
  p.h2d = p.d2h = nullptr;
  p.d_Fw = p.d_Gm = p.d_ent_w = nullptr;
  p.d_phase = p.d_scratch = p.d_scratch_raw = p.d_stage_f = p.d_stage_Q = nullptr;
  p.d_tasks = nullptr;
  p.d_groups = nullptr;
  p.d_cons = nullptr;
  p.d_kappa = nullptr;
  p.d_Qfull = nullptr;
  p.d_Fv = nullptr;
  p.d_Fwf = nullptr;
  p.d_Fvf = nullptr;
  p.d_Gmf = nullptr;
  p.d_ent_m = nullptr;
  p.d_ent_ysh = nullptr;
  p.d_counter = nullptr;
  p.d_rk = nullptr;
  p.d_mats = nullptr;
}

}  // namespace dgfs
