// Differential-evolution operators of the global search (Sec. II B), host side, and one
// generation over a batch: offspring, their local relaxation (sgo_relax_batch), greedy
// selection.
//
// An individual is a structure of natoms atoms (species fixed per atom slot) in a cell the
// population shares; its fitness is its relaxed free energy.  For every individual X_i:
// * triangle mutation (Eq. 2) from three distinct others r1, r2, r3 != i:
//   V = (X1 + X2 + X3)/3 + (p2 - p1)(X1 - X2) + (p3 - p2)(X2 - X3) + (p1 - p3)(X3 - X1),
//   p_k = |f_k| / sum |f|, in fractional coordinates with minimum-image differences
//   (X_k - X_1 wrapped into [-1/2, 1/2)), wrapped into the cell;
// * cut-and-splice crossover of V (kept side) with X_i (fill): a random plane through each
//   parent's centre, or a sphere of random radius around it; every species is filled up to
//   its count with X_i's atoms nearest the cut (plane: lowest projection; sphere: farthest
//   from the centre), so the child has the parents' composition in one pass;
// * distance repair: pairs closer than d_min (minimum image) are pushed apart, the later
//   atom moving along the separation, in passes (at most 100);
// * greedy selection: the relaxed child replaces X_i when its energy is lower;
// * migration between subpopulations (consecutive slices), in ring order: the best of one
//   replaces the worst of the next when better;
// * similarity (the initialisation's check between structures): sorted minimum-image pair
//   distances, similar when their root-mean-square difference is below a tolerance.
// The random numbers are inputs, SGO_DE_RANDOMS uniforms per offspring (3 partners, 2 for
// the plane normal, 1 for the scheme, 1 for the sphere radius).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sgo.h"

namespace {

using Vec = std::vector<double>;

struct Cell {
  double A[9], inv[9];
  explicit Cell(const double* a) {
    std::memcpy(A, a, sizeof(A));
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  }
  // row vector times matrix: s = x . inv, x = s . A
  void frac(const double* x, double* s) const {
    for (int c = 0; c < 3; ++c) s[c] = x[0] * inv[c] + x[1] * inv[3 + c] + x[2] * inv[6 + c];
  }
  void cart(const double* s, double* x) const {
    for (int c = 0; c < 3; ++c) x[c] = s[0] * A[c] + s[1] * A[3 + c] + s[2] * A[6 + c];
  }
};

double wrap(double s) { return s - std::floor(s); }
// minimum image of a fractional difference: d - round(d), halves to even
double mimg(double d) { return d - std::nearbyint(d); }

void partners(int i, int np, const double* u, int* r) {
  std::vector<int> pool;
  for (int k = 0; k < np; ++k)
    if (k != i) pool.push_back(k);
  for (int k = 0; k < 3; ++k) {
    const int j = std::min((int)(u[k] * (double)pool.size()), (int)pool.size() - 1);
    r[k] = pool[j];
    pool.erase(pool.begin() + j);
  }
}

void triangle_mutation(const Cell& cell, int n, const double* X1, const double* X2, const double* X3, double f1,
                       double f2, double f3, double* V) {
  const double tot = std::fabs(f1) + std::fabs(f2) + std::fabs(f3);
  double p1 = 1.0 / 3.0, p2 = 1.0 / 3.0, p3 = 1.0 / 3.0;
  if (tot > 0) {
    p1 = std::fabs(f1) / tot;
    p2 = std::fabs(f2) / tot;
    p3 = std::fabs(f3) / tot;
  }
  for (int a = 0; a < n; ++a) {
    double s1[3], t2[3], t3[3], s2[3], s3[3], v[3];
    cell.frac(X1 + 3 * a, s1);
    cell.frac(X2 + 3 * a, t2);
    cell.frac(X3 + 3 * a, t3);
    for (int c = 0; c < 3; ++c) {
      s2[c] = s1[c] + mimg(t2[c] - s1[c]);
      s3[c] = s1[c] + mimg(t3[c] - s1[c]);
      v[c] = wrap((s1[c] + s2[c] + s3[c]) / 3.0 + (p2 - p1) * (s1[c] - s2[c]) + (p3 - p2) * (s2[c] - s3[c]) +
                  (p1 - p3) * (s3[c] - s1[c]));
    }
    cell.cart(v, V + 3 * a);
  }
}

void cut_and_splice(int n, const int* species, const double* P1, const double* P2, const double* u, int scheme,
                    double* C) {
  double c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0};
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < 3; ++c) {
      c1[c] += P1[3 * a + c];
      c2[c] += P2[3 * a + c];
    }
  for (int c = 0; c < 3; ++c) {
    c1[c] /= n;
    c2[c] /= n;
  }
  const bool plane = scheme == SGO_DE_PLANE || (scheme == SGO_DE_RANDOM_SCHEME && u[5] < 0.5);
  std::vector<char> keep(n);
  Vec key2(n);
  if (plane) {
    const double z = 1.0 - 2.0 * u[3];
    const double r = std::sqrt(std::max(0.0, 1.0 - z * z));
    const double phi = 2.0 * M_PI * u[4];
    const double nv[3] = {r * std::cos(phi), r * std::sin(phi), z};
    for (int a = 0; a < n; ++a) {
      double k1 = 0.0, k2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        k1 += (P1[3 * a + c] - c1[c]) * nv[c];
        k2 += (P2[3 * a + c] - c2[c]) * nv[c];
      }
      keep[a] = k1 > 0.0;
      key2[a] = k2;
    }
  } else {
    Vec d1(n);
    double dmax = 0.0;
    for (int a = 0; a < n; ++a) {
      double s1 = 0.0, s2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        s1 += (P1[3 * a + c] - c1[c]) * (P1[3 * a + c] - c1[c]);
        s2 += (P2[3 * a + c] - c2[c]) * (P2[3 * a + c] - c2[c]);
      }
      d1[a] = std::sqrt(s1);
      key2[a] = -std::sqrt(s2);
      dmax = std::max(dmax, d1[a]);
    }
    const double R = u[6] * dmax;
    for (int a = 0; a < n; ++a) keep[a] = d1[a] < R;
  }
  std::vector<int> done(n, 0);
  for (int a = 0; a < n; ++a) {
    if (done[a]) continue;
    const int s = species[a];
    std::vector<int> slots, kept, order;
    for (int b = 0; b < n; ++b)
      if (species[b] == s) {
        slots.push_back(b);
        done[b] = 1;
        if (keep[b]) kept.push_back(b);
      }
    order = slots;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key2[x] < key2[y]; });
    const size_t need = slots.size() - kept.size();
    std::vector<int> fill(order.begin(), order.begin() + need);
    std::sort(fill.begin(), fill.end());
    for (size_t k = 0; k < kept.size(); ++k)
      for (int c = 0; c < 3; ++c) C[3 * slots[k] + c] = P1[3 * kept[k] + c];
    for (size_t k = 0; k < fill.size(); ++k)
      for (int c = 0; c < 3; ++c) C[3 * slots[kept.size() + k] + c] = P2[3 * fill[k] + c];
  }
}

void repair(const Cell& cell, int n, double d_min, double* X) {
  for (int pass = 0; pass < 100; ++pass) {
    bool moved = false;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        double dx[3], ds[3], dv[3];
        for (int c = 0; c < 3; ++c) dx[c] = X[3 * j + c] - X[3 * i + c];
        cell.frac(dx, ds);
        for (int c = 0; c < 3; ++c) ds[c] = mimg(ds[c]);
        cell.cart(ds, dv);
        const double d = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        if (d < d_min) {
          double e[3] = {1.0, 0.0, 0.0};
          if (d > 1e-12)
            for (int c = 0; c < 3; ++c) e[c] = dv[c] / d;
          for (int c = 0; c < 3; ++c) X[3 * j + c] += (d_min - d) * e[c];
          moved = true;
        }
      }
    if (!moved) break;
  }
  for (int a = 0; a < n; ++a) {
    double s[3];
    cell.frac(X + 3 * a, s);
    for (int c = 0; c < 3; ++c) s[c] = wrap(s[c]);
    cell.cart(s, X + 3 * a);
  }
}

// sorted minimum-image pair distances
Vec fingerprint(const Cell& cell, int n, const double* X) {
  Vec d;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double dx[3], ds[3], dv[3];
      for (int c = 0; c < 3; ++c) dx[c] = X[3 * j + c] - X[3 * i + c];
      cell.frac(dx, ds);
      for (int c = 0; c < 3; ++c) ds[c] = mimg(ds[c]);
      cell.cart(ds, dv);
      d.push_back(std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]));
    }
  std::sort(d.begin(), d.end());
  return d;
}

}  // namespace

extern "C" {

sgo_status sgo_de_similar(int natoms, const double cell[9], const double* a, const double* b, double tol,
                          int* similar) {
  if (natoms < 1 || !cell || !a || !b || !similar || !(tol >= 0)) return SGO_ERR_ARG;
  const Cell c(cell);
  const Vec fa = fingerprint(c, natoms, a), fb = fingerprint(c, natoms, b);
  if (fa.empty()) {
    *similar = 1;
    return SGO_OK;
  }
  double s = 0.0;
  for (size_t k = 0; k < fa.size(); ++k) s += (fa[k] - fb[k]) * (fa[k] - fb[k]);
  *similar = std::sqrt(s / (double)fa.size()) < tol ? 1 : 0;
  return SGO_OK;
}

sgo_status sgo_de_migrate(int np, int nsub, int natoms, double* pop, double* f) {
  if (np < 1 || nsub < 1 || np % nsub != 0 || natoms < 1 || !pop || !f) return SGO_ERR_ARG;
  if (nsub == 1) return SGO_OK;  // a single subpopulation has no neighbour
  const int size = np / nsub;
  const size_t sz = 3 * (size_t)natoms;
  // every subpopulation's best and its neighbour's worst are chosen on the population as
  // it was before this call, so that a migrant moves one step round the ring at most
  std::vector<int> best(nsub), worst(nsub);
  for (int s = 0; s < nsub; ++s) {
    int b = s * size, w = s * size;
    for (int k = s * size; k < (s + 1) * size; ++k) {
      if (f[k] < f[b]) b = k;
      if (f[k] > f[w]) w = k;
    }
    best[s] = b;
    worst[s] = w;
  }
  Vec xb(sz * nsub), fb(nsub), fw(nsub);
  for (int s = 0; s < nsub; ++s) {
    std::memcpy(xb.data() + sz * s, pop + sz * best[s], sizeof(double) * sz);
    fb[s] = f[best[s]];
    fw[s] = f[worst[s]];
  }
  for (int s = 0; s < nsub; ++s) {
    const int t = (s + 1) % nsub;
    if (fb[s] < fw[t]) {
      std::memcpy(pop + sz * worst[t], xb.data() + sz * s, sizeof(double) * sz);
      f[worst[t]] = fb[s];
    }
  }
  return SGO_OK;
}

sgo_status sgo_de_offspring(int np, int natoms, const double cell[9], const int* species, const double* pop,
                            const double* f, const double* u, int scheme, double d_min, double* children) {
  if (np < 4 || natoms < 1 || !cell || !species || !pop || !f || !u || !children || !(d_min >= 0) ||
      scheme < SGO_DE_RANDOM_SCHEME || scheme > SGO_DE_SPHERE)
    return SGO_ERR_ARG;
  const Cell c(cell);
  const size_t sz = 3 * (size_t)natoms;
  Vec V(sz);
  for (int i = 0; i < np; ++i) {
    const double* ui = u + (size_t)SGO_DE_RANDOMS * i;
    int r[3];
    partners(i, np, ui, r);
    triangle_mutation(c, natoms, pop + sz * r[0], pop + sz * r[1], pop + sz * r[2], f[r[0]], f[r[1]], f[r[2]],
                      V.data());
    double* C = children + sz * i;
    cut_and_splice(natoms, species, V.data(), pop + sz * i, ui, scheme, C);
    repair(c, natoms, d_min, C);
  }
  return SGO_OK;
}

}  // extern "C"
