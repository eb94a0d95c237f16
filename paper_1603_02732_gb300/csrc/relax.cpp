// Local relaxation of one structure (Sec. II C), host side: the driver between the DE
// search and the batched energy/force evaluation.
//
// PCG: nonlinear preconditioned conjugate gradients whose preconditioner is the inverse
// Hessian of a classical force field fitted to the DFT forces.  The force field is a
// shifted-force Morse pair potential over periodic images, phi(r) = D [exp(-2a(r - r0)) -
// 2 exp(-a(r - r0))], parameters theta = (D, a, r0) fitted by Levenberg-Marquardt to the
// force sets of the last 64 evaluated configurations (with a weak pull towards the previous
// fit, which picks a solution when few forces leave theta undetermined), with the analytic
// Jacobian of the force residual.  Its Hessian is the
// second-order finite difference of the fitted energy; the three eigenpairs of the
// translations (smallest |tau|) are dropped and P = sum_j V_j V_j^T / |tau_j| over the
// others (|tau_j| floored at a fraction of the largest).  The fit and P are renewed every
// `refit` search directions.  CG: the same iteration with P = I / kappa0.  BFGS: inverse
// update from B0 = I / kappa0, steps capped per atom.
//
// The driver is a state machine: the caller evaluates the positions it asks for (first
// the initial ones) and hands back energy and forces.  sgo_relax_batch runs the drivers of
// a batch's members against sgo_energy_forces_batch, warm-starting every evaluation after
// the first from the member's previous density and wavefunctions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sgo.h"

namespace {

constexpr double kKappa0 = 0.5;   // Ha/bohr^2 behind unpreconditioned steps (CG, BFGS)
constexpr double kFloor = 0.02;   // kept force-field eigenvalues: |tau| >= kFloor max|tau|
constexpr double kHfd = 1e-3;     // bohr: central-difference step of the force-field Hessian
constexpr double kReg = 1e-6;     // weight of the pull towards the previous fit
constexpr int kHist = 64;         // the fit uses the last kHist evaluated configurations
constexpr double kSkin = 1.0;     // bohr: pair lists keep r < rc + kSkin (displacements of the
                                  // finite-difference Hessian stay far below it)

using Vec = std::vector<double>;

double dot(const Vec& a, const Vec& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// phi'(r) of the Morse pair
double morse_dphi(const double* th, double r) {
  const double e = std::exp(-th[1] * (r - th[2]));
  return 2.0 * th[0] * th[1] * (e - e * e);
}
// d phi'(r) / d(D, a, r0)
void morse_dphi_grad(const double* th, double r, double* g3) {
  const double D = th[0], a = th[1], e = std::exp(-a * (r - th[2]));
  const double g = e - e * e, h = 1.0 - 2.0 * e;
  g3[0] = 2.0 * a * g;
  g3[1] = 2.0 * D * g - 2.0 * D * a * h * (r - th[2]) * e;
  g3[2] = 2.0 * D * a * h * a * e;
}

// lattice translations n . A, |n_k| <= ceil(rc / width_k) + 1
Vec image_vectors(const double* cell, double rc) {
  // inverse of the cell (rows a_i); width_k = 1 / |column k of inv|
  const double* A = cell;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  int nmax[3];
  for (int k = 0; k < 3; ++k) {
    const double c = std::sqrt(inv[k] * inv[k] + inv[3 + k] * inv[3 + k] + inv[6 + k] * inv[6 + k]);
    nmax[k] = (int)std::ceil(rc * c) + 1;
  }
  Vec L;
  for (int i = -nmax[0]; i <= nmax[0]; ++i)
    for (int j = -nmax[1]; j <= nmax[1]; ++j)
      for (int k = -nmax[2]; k <= nmax[2]; ++k)
        for (int c = 0; c < 3; ++c) L.push_back(i * A[c] + j * A[3 + c] + k * A[6 + c]);
  return L;
}

// (i, j, image) triples with |R_j + L - R_i| < rmax, j != i: the candidates of the force
// sum for this configuration and for any configuration within (rmax - rc) / 2 of it
struct PairList {
  std::vector<int> i, j;
  Vec L;
};
PairList build_pairs(const Vec& Limg, double rmax, int n, const double* x) {
  PairList pl;
  const int nl = (int)Limg.size() / 3;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      for (int l = 0; l < nl; ++l) {
        double rv[3];
        for (int c = 0; c < 3; ++c) rv[c] = x[3 * j + c] + Limg[3 * l + c] - x[3 * i + c];
        if (rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2] < rmax * rmax) {
          pl.i.push_back(i);
          pl.j.push_back(j);
          for (int c = 0; c < 3; ++c) pl.L.push_back(Limg[3 * l + c]);
        }
      }
    }
  return pl;
}

// forces of the shifted-force Morse field: F_i = sum_{j != i, L} (phi'(r) - phi'(rc)) rv / r,
// rv = R_j + L - R_i, over r < rc (the pairs of a list built for nearby positions)
void ff_forces(const double* th, const PairList& pl, double rc, int n, const double* x, double* F) {
  const double dc = morse_dphi(th, rc);
  for (int k = 0; k < 3 * n; ++k) F[k] = 0.0;
  for (size_t p = 0; p < pl.i.size(); ++p) {
    const int i = pl.i[p], j = pl.j[p];
    double rv[3];
    for (int c = 0; c < 3; ++c) rv[c] = x[3 * j + c] + pl.L[3 * p + c] - x[3 * i + c];
    const double r = std::sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    if (!(r < rc) || !(r > 1e-12)) continue;
    const double f = (morse_dphi(th, r) - dc) / r;
    for (int c = 0; c < 3; ++c) F[3 * i + c] += f * rv[c];
  }
}

// dF/dtheta of ff_forces: J[(3 i + c) * 3 + k] = d F_{i,c} / d theta_k, each pair term
// (phi'(r) - phi'(rc)) rv / r differentiated analytically
void ff_forces_jac(const double* th, const PairList& pl, double rc, int n, const double* x, double* J) {
  double gc[3];
  morse_dphi_grad(th, rc, gc);
  for (int k = 0; k < 9 * n; ++k) J[k] = 0.0;
  for (size_t p = 0; p < pl.i.size(); ++p) {
    const int i = pl.i[p], j = pl.j[p];
    double rv[3];
    for (int c = 0; c < 3; ++c) rv[c] = x[3 * j + c] + pl.L[3 * p + c] - x[3 * i + c];
    const double r = std::sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    if (!(r < rc) || !(r > 1e-12)) continue;
    double g[3];
    morse_dphi_grad(th, r, g);
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 3; ++k) J[(3 * i + c) * 3 + k] += (g[k] - gc[k]) * (rv[c] / r);
  }
}

// 3x3 linear solve by Gaussian elimination with partial pivoting
bool solve3(double M[3][3], double b[3], double x[3]) {
  int p[3] = {0, 1, 2};
  for (int c = 0; c < 3; ++c) {
    int best = c;
    for (int r = c + 1; r < 3; ++r)
      if (std::fabs(M[p[r]][c]) > std::fabs(M[p[best]][c])) best = r;
    std::swap(p[c], p[best]);
    if (M[p[c]][c] == 0.0) return false;
    for (int r = c + 1; r < 3; ++r) {
      const double f = M[p[r]][c] / M[p[c]][c];
      for (int k = c; k < 3; ++k) M[p[r]][k] -= f * M[p[c]][k];
      b[p[r]] -= f * b[p[c]];
    }
  }
  for (int c = 2; c >= 0; --c) {
    double s = b[p[c]];
    for (int k = c + 1; k < 3; ++k) s -= M[p[c]][k] * x[k];
    x[c] = s / M[p[c]][c];
  }
  return true;
}

// cyclic Jacobi eigen-decomposition of a symmetric m x m matrix (row-major, destroyed);
// eigenvalues to tau, eigenvectors to the columns of V
void jacobi_eig(int m, Vec& A, Vec& tau, Vec& V) {
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double a = A[(size_t)i * m + j];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double tau_ = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (tau_ >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau_) + std::sqrt(1.0 + tau_ * tau_));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = c * akp - s * akq;
          A[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = c * apk - s * aqk;
          A[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - s * vkq;
          V[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  tau.resize(m);
  for (int i = 0; i < m; ++i) tau[i] = A[(size_t)i * m + i];
}

double fmax_of(int n, const double* F) {
  double m = 0.0;
  for (int i = 0; i < n; ++i)
    m = std::max(m, std::sqrt(F[3 * i] * F[3 * i] + F[3 * i + 1] * F[3 * i + 1] + F[3 * i + 2] * F[3 * i + 2]));
  return m;
}
double dmax_of(int n, const Vec& d) { return fmax_of(n, d.data()); }

}  // namespace

struct sgo_relax {
  int n = 0;
  double cell[9];
  sgo_relax_opts o;
  Vec L, Lnn;                    // images within rc (force field) and within 1 bohr (neighbours)
  // the last kHist evaluated configurations, their forces and pair lists (the fit's data)
  std::vector<Vec> hx, hf;
  std::vector<PairList> hp;
  int evals = 0, state = 0;      // state: 0 running, 1 converged, 2 stopped unconverged
  double best_e = 0.0;           // the lowest-energy configuration evaluated so far
  Vec best_x;
  Vec x, g;                      // current point and gradient (-F)
  Vec pending;                   // positions handed out for evaluation
  int phase = 0;                 // 0 initial point, 1 trial point, 2 line minimum, 3 BFGS step
  // (P)CG
  Vec d, s, d_prev, s_prev, g_prev, P, xt, gt;
  bool have_prev = false;
  double at = 0.0, p0 = 0.0, dmax = 0.0;
  double a_prev = 1.0;           // the previous line's minimising step: the next trial step
                                 // (1 again whenever the preconditioner is renewed)
  double theta[3] = {0, 0, 0};
  bool have_theta = false;
  int ndir = 0;
  // BFGS
  Vec B, dx;
};

namespace {

Vec ff_forces_v(const sgo_relax* r, const double* th, const PairList& pl, const Vec& x) {
  Vec F(x.size());
  ff_forces(th, pl, r->o.rc, r->n, x.data(), F.data());
  return F;
}

// Levenberg-Marquardt fit of theta to every evaluated force set (see the file comment)
void fit_force_field(sgo_relax* r) {
  const double t0[3] = {r->theta[0], r->theta[1], r->theta[2]};
  double th[3] = {t0[0], t0[1], t0[2]};
  double fsq = 0.0;
  size_t ncomp = 0;
  for (const Vec& f : r->hf) {
    for (double v : f) fsq += v * v;
    ncomp += f.size();
  }
  const double sw = std::sqrt(kReg * std::max(fsq / (double)ncomp, 1e-30) * (double)ncomp);
  auto resid = [&](const double* t) {
    Vec res;
    res.reserve(ncomp + 3);
    for (size_t k = 0; k < r->hx.size(); ++k) {
      const Vec F = ff_forces_v(r, t, r->hp[k], r->hx[k]);
      for (size_t i = 0; i < F.size(); ++i) res.push_back(F[i] - r->hf[k][i]);
    }
    for (int k = 0; k < 3; ++k) res.push_back(sw * (t[k] - t0[k]) / t0[k]);
    return res;
  };
  // Jacobian of the residual: the force field's analytic dF/dtheta, then the pull's rows
  auto jac = [&](const double* t) {
    std::vector<Vec> J(3, Vec());
    for (int k = 0; k < 3; ++k) J[k].reserve(ncomp + 3);
    Vec Jc(9 * (size_t)r->n);
    for (size_t h = 0; h < r->hx.size(); ++h) {
      ff_forces_jac(t, r->hp[h], r->o.rc, r->n, r->hx[h].data(), Jc.data());
      for (int row = 0; row < 3 * r->n; ++row)
        for (int k = 0; k < 3; ++k) J[k].push_back(Jc[(size_t)row * 3 + k]);
    }
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < 3; ++k) J[k].push_back(q == k ? sw / t0[k] : 0.0);
    return J;
  };
  Vec res = resid(th);
  double cost = dot(res, res);
  double lam = 1e-3;
  for (int it = 0; it < 60; ++it) {
    const std::vector<Vec> J = jac(th);
    double A[3][3], gr[3];
    for (int a = 0; a < 3; ++a) {
      gr[a] = dot(J[a], res);
      for (int b = 0; b < 3; ++b) A[a][b] = dot(J[a], J[b]);
    }
    bool improved = false;
    double step[3] = {0, 0, 0};
    while (lam < 1e12) {
      double M[3][3], rhs[3];
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) M[a][b] = A[a][b] + (a == b ? lam * (A[a][a] + 1e-30) : 0.0);
        rhs[a] = -gr[a];
      }
      if (solve3(M, rhs, step)) {
        const double t[3] = {th[0] + step[0], th[1] + step[1], th[2] + step[2]};
        if (t[0] > 0 && t[1] > 0 && t[2] > 0) {
          const Vec rn = resid(t);
          const double cn = dot(rn, rn);
          if (std::isfinite(cn) && cn < cost) {
            for (int k = 0; k < 3; ++k) th[k] = t[k];
            res = rn;
            cost = cn;
            lam = std::max(lam / 10.0, 1e-12);
            improved = true;
            break;
          }
        }
      }
      lam *= 10.0;
    }
    const double smax = std::max({std::fabs(step[0]), std::fabs(step[1]), std::fabs(step[2])});
    const double tmax = std::max({std::fabs(th[0]), std::fabs(th[1]), std::fabs(th[2])});
    if (!improved || smax <= 1e-10 * tmax) break;
  }
  if (std::isfinite(th[0]) && std::isfinite(th[1]) && std::isfinite(th[2]) && th[0] > 0 && th[1] > 0 && th[2] > 0)
    for (int k = 0; k < 3; ++k) r->theta[k] = th[k];
}

// P = truncated inverse of the force field's finite-difference Hessian at r->x
void build_preconditioner(sgo_relax* r) {
  const int m = 3 * r->n;
  Vec H((size_t)m * m);
  const PairList pl = build_pairs(r->L, r->o.rc + kSkin, r->n, r->x.data());
  for (int k = 0; k < m; ++k) {
    Vec xp = r->x, xm = r->x;
    xp[k] += kHfd;
    xm[k] -= kHfd;
    const Vec Fp = ff_forces_v(r, r->theta, pl, xp), Fm = ff_forces_v(r, r->theta, pl, xm);
    for (int i = 0; i < m; ++i) H[(size_t)i * m + k] = -(Fp[i] - Fm[i]) / (2.0 * kHfd);
  }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double v = 0.5 * (H[(size_t)i * m + j] + H[(size_t)j * m + i]);
      H[(size_t)i * m + j] = H[(size_t)j * m + i] = v;
    }
  Vec tau, V;
  jacobi_eig(m, H, tau, V);
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(tau[a]) < std::fabs(tau[b]); });
  double tmax = 0.0;
  for (int k = 3; k < m; ++k) tmax = std::max(tmax, std::fabs(tau[order[k]]));
  r->P.assign((size_t)m * m, 0.0);
  for (int k = 3; k < m; ++k) {
    const int j = order[k];
    const double t = std::max(std::fabs(tau[j]), kFloor * tmax);
    for (int a = 0; a < m; ++a) {
      const double va = V[(size_t)a * m + j] / t;
      for (int b = 0; b < m; ++b) r->P[(size_t)a * m + b] += va * V[(size_t)b * m + j];
    }
  }
}

double nearest_neighbour(const sgo_relax* r) {
  double best = 1e300;
  const int nl = (int)r->Lnn.size() / 3;
  for (int i = 0; i < r->n; ++i)
    for (int j = 0; j < r->n; ++j)
      for (int l = 0; l < nl; ++l) {
        double rv[3];
        for (int c = 0; c < 3; ++c) rv[c] = r->x[3 * j + c] + r->Lnn[3 * l + c] - r->x[3 * i + c];
        const double d = std::sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        if (d > 1e-9) best = std::min(best, d);
      }
  return best;
}

Vec matvec(const Vec& M, const Vec& v) {
  const size_t m = v.size();
  Vec out(m, 0.0);
  for (size_t a = 0; a < m; ++a) {
    double s = 0.0;
    for (size_t b = 0; b < m; ++b) s += M[a * m + b] * v[b];
    out[a] = s;
  }
  return out;
}

// new (P)CG search direction from r->x, r->g; hands out the trial point
void start_line(sgo_relax* r) {
  const int m = 3 * r->n;
  if (r->o.method == SGO_RELAX_PCG) {
    if (r->P.empty() || r->ndir % std::max(r->o.refit, 1) == 0) {
      if (!r->have_theta) {
        r->theta[0] = 0.1;
        r->theta[1] = 1.0;
        r->theta[2] = nearest_neighbour(r);
        r->have_theta = true;
      }
      fit_force_field(r);
      build_preconditioner(r);
      r->a_prev = 1.0;  // a step found under the previous preconditioner has its scale
    }
  } else if (r->P.empty()) {
    r->P.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) r->P[(size_t)i * m + i] = 1.0 / kKappa0;
  }
  r->s = matvec(r->P, r->g);
  r->d.resize(m);
  if (!r->have_prev) {
    for (int i = 0; i < m; ++i) r->d[i] = -r->s[i];
  } else {
    Vec ds(m);
    for (int i = 0; i < m; ++i) ds[i] = r->s[i] - r->s_prev[i];
    const double beta = std::max(0.0, dot(r->g, ds) / dot(r->g_prev, r->s_prev));
    for (int i = 0; i < m; ++i) r->d[i] = -r->s[i] + beta * r->d_prev[i];
    if (dot(r->d, r->g) >= 0.0)
      for (int i = 0; i < m; ++i) r->d[i] = -r->s[i];
  }
  r->ndir += 1;
  r->dmax = dmax_of(r->n, r->d);
  if (!(r->dmax > 0.0)) {
    r->state = 2;  // zero direction: the preconditioned gradient vanished without convergence
    r->pending = r->x;
    return;
  }
  r->at = std::min(r->a_prev, r->o.max_step / r->dmax);
  r->xt.resize(m);
  for (int i = 0; i < m; ++i) r->xt[i] = r->x[i] + r->at * r->d[i];
  r->pending = r->xt;
  r->phase = 1;
}

void bfgs_step(sgo_relax* r) {
  const int m = 3 * r->n;
  r->dx = matvec(r->B, r->g);
  for (double& v : r->dx) v = -v;
  const double mx = dmax_of(r->n, r->dx);
  if (mx > r->o.max_step)
    for (double& v : r->dx) v *= r->o.max_step / mx;
  r->pending.resize(m);
  for (int i = 0; i < m; ++i) r->pending[i] = r->x[i] + r->dx[i];
  r->phase = 3;
}

}  // namespace

extern "C" {

void sgo_relax_opts_default(sgo_relax_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = SGO_RELAX_PCG;
  o->fmax = 1e-3;
  o->max_step = 0.3;
  o->refit = 3;
  o->rc = 8.0;
  o->accept = 0.1;
  o->max_evals = 60;
}

sgo_status sgo_relax_create(int natoms, const double cell[9], const double* pos, const sgo_relax_opts* o,
                            sgo_relax** out) {
  if (!out) return SGO_ERR_ARG;
  *out = nullptr;
  if (natoms < 1 || !cell || !pos) return SGO_ERR_ARG;
  sgo_relax_opts oo;
  if (o) oo = *o;
  else sgo_relax_opts_default(&oo);
  if (oo.method < SGO_RELAX_PCG || oo.method > SGO_RELAX_BFGS || !(oo.fmax > 0) || !(oo.max_step > 0) ||
      !(oo.rc > 0) || oo.max_evals < 1 || !(oo.accept >= 0))
    return SGO_ERR_ARG;
  sgo_relax* r = new (std::nothrow) sgo_relax();
  if (!r) return SGO_ERR_OOM;
  r->n = natoms;
  std::memcpy(r->cell, cell, sizeof(r->cell));
  r->o = oo;
  r->L = image_vectors(cell, oo.rc);
  r->Lnn = image_vectors(cell, 1.0);
  r->x.assign(pos, pos + 3 * natoms);
  r->pending = r->x;
  r->phase = 0;
  if (oo.method == SGO_RELAX_BFGS) {
    const int m = 3 * natoms;
    r->B.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) r->B[(size_t)i * m + i] = 1.0 / kKappa0;
  }
  *out = r;
  return SGO_OK;
}

sgo_status sgo_relax_step(sgo_relax* r, double energy, const double* forces, double* next_pos, int* state) {
  if (!r || !forces || !next_pos) return SGO_ERR_ARG;
  (void)energy;  // the line minimisation uses directional derivatives only
  const int m = 3 * r->n;
  if (r->state != 0) {
    std::memcpy(next_pos, r->pending.data(), sizeof(double) * m);
    if (state) *state = r->state;
    return SGO_OK;
  }
  for (int i = 0; i < m; ++i)
    if (!std::isfinite(forces[i])) return SGO_ERR_NAN;
  const Vec F(forces, forces + m);
  const Vec xe = r->pending;  // the configuration these forces belong to
  if (r->evals == 0 || energy < r->best_e) {
    r->best_e = energy;
    r->best_x = xe;
  }
  r->evals += 1;
  r->hx.push_back(xe);
  r->hf.push_back(F);
  r->hp.push_back(build_pairs(r->L, r->o.rc + kSkin, r->n, xe.data()));
  if ((int)r->hx.size() > kHist) {
    r->hx.erase(r->hx.begin());
    r->hf.erase(r->hf.begin());
    r->hp.erase(r->hp.begin());
  }
  Vec ge(m);
  for (int i = 0; i < m; ++i) ge[i] = -F[i];
  if (fmax_of(r->n, forces) < r->o.fmax) {
    r->state = 1;
    r->x = xe;
    r->pending = xe;
  } else if (r->evals >= r->o.max_evals) {
    r->state = 2;
    r->x = xe;
    r->pending = xe;
  } else if (r->o.method == SGO_RELAX_BFGS) {
    if (r->phase == 3) {
      Vec y(m);
      for (int i = 0; i < m; ++i) y[i] = ge[i] - r->g[i];
      const double sy = dot(r->dx, y);
      if (sy > 1e-12) {
        // B <- (I - rho s y^T) B (I - rho y s^T) + rho s s^T
        const double rho = 1.0 / sy;
        const Vec By = matvec(r->B, y);   // B y (B symmetric)
        const double yBy = dot(y, By);
        for (int a = 0; a < m; ++a)
          for (int b = 0; b < m; ++b)
            r->B[(size_t)a * m + b] += -rho * (r->dx[a] * By[b] + By[a] * r->dx[b]) +
                                       (rho * rho * yBy + rho) * r->dx[a] * r->dx[b];
      }
    }
    r->x = xe;
    r->g = ge;
    bfgs_step(r);
  } else if (r->phase == 0) {
    r->x = xe;
    r->g = ge;
    start_line(r);
  } else if (r->phase == 1) {
    // trial point: secant of the directional derivative phi'(a) = g(a).d
    r->gt = ge;
    const double p0 = dot(r->g, r->d), pt = dot(ge, r->d);
    const double amax = r->o.max_step / r->dmax;
    double astar = pt - p0 > 0.0 ? r->at * p0 / (p0 - pt) : amax;
    astar = std::min(std::max(astar, 0.1 * r->at), amax);
    r->a_prev = astar;
    r->g_prev = r->g;
    r->s_prev = r->s;
    r->d_prev = r->d;
    r->have_prev = true;
    if (std::fabs(astar - r->at) <= r->o.accept * r->at || r->evals + 1 > r->o.max_evals) {
      r->x = xe;
      r->g = ge;
      start_line(r);
    } else {
      Vec xn(m);
      for (int i = 0; i < m; ++i) xn[i] = r->x[i] + astar * r->d[i];
      r->pending = xn;
      r->phase = 2;
    }
  } else {  // phase 2: the line minimum
    r->x = xe;
    r->g = ge;
    start_line(r);
  }
  std::memcpy(next_pos, r->pending.data(), sizeof(double) * m);
  if (state) *state = r->state;
  return SGO_OK;
}

sgo_status sgo_relax_positions(const sgo_relax* r, double* pos) {
  if (!r || !pos) return SGO_ERR_ARG;
  std::memcpy(pos, r->pending.data(), sizeof(double) * 3 * r->n);
  return SGO_OK;
}

sgo_status sgo_relax_best(const sgo_relax* r, double* energy, double* pos) {
  if (!r || r->evals == 0) return SGO_ERR_ARG;
  if (energy) *energy = r->best_e;
  if (pos) std::memcpy(pos, r->best_x.data(), sizeof(double) * 3 * r->n);
  return SGO_OK;
}

sgo_status sgo_relax_info(const sgo_relax* r, int* evals, int* state) {
  if (!r) return SGO_ERR_ARG;
  if (evals) *evals = r->evals;
  if (state) *state = r->state;
  return SGO_OK;
}

int sgo_relax_natoms(const sgo_relax* r) { return r ? r->n : 0; }

void sgo_relax_destroy(sgo_relax* r) { delete r; }

}  // extern "C"
