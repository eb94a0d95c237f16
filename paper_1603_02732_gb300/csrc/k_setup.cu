// Per-cell and per-structure set-up kernels: the Gamma half-sphere basis within Ecut
// and its FFT column maps, FFT twiddles, per-atom phase tables, the local
// pseudopotential on the FFT box, and the Ewald ion-ion energy and forces.
#include "kernels.h"

namespace sgo {

namespace {
__device__ __forceinline__ void gcart(const Prob& P, int m1, int m2, int m3, double* G) {
  for (int d = 0; d < 3; ++d) G[d] = m1 * P.bvec[d] + m2 * P.bvec[3 + d] + m3 * P.bvec[6 + d];
}
__device__ __forceinline__ double g2_of(const Prob& P, int m1, int m2, int m3) {
  double G[3];
  gcart(P, m1, m2, m3, G);
  return G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
}
// canonical "positive" column of an inversion pair: m2 > 0, or m2 == 0 and m1 > 0
__device__ __forceinline__ bool positive_col(int m1, int m2) { return m2 > 0 || (m2 == 0 && m1 > 0); }
}  // namespace

// ---------------------------------------------------------------------------
// Basis.  Box column q = (m1 + box1)(2 box2 + 1) + (m2 + box2).  One thread per column.
// ---------------------------------------------------------------------------
__global__ void k_basis_count(KArgs ka) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  const Prob& P = ka.probs[p];
  const int w2 = 2 * P.box2 + 1;
  const int q = (blockIdx.x - ka.start[p]) * blockDim.x + threadIdx.x;
  if (q >= (2 * P.box1 + 1) * w2) return;
  const int m1 = q / w2 - P.box1, m2 = q % w2 - P.box2;
  const bool zero = (m1 == 0 && m2 == 0);
  int cnt = 0, mx = 0;
  if (zero || positive_col(m1, m2)) {
    for (int m3 = -P.box3; m3 <= P.box3; ++m3) {
      if (zero && m3 <= 0) continue;
      if (0.5 * g2_of(P, m1, m2, m3) <= P.ecut) {
        ++cnt;
        mx = max(mx, abs(m3));
      }
    }
  }
  P.bx_cnt[q] = cnt;
  P.bx_m3max[q] = mx;
}

// Sequential scan (one thread per problem): pair ids, entry offsets, sizes.
__global__ void k_basis_scan(KArgs ka) {
  const int p = blockIdx.x;
  const Prob& P = ka.probs[p];
  if (threadIdx.x != 0) return;
  const int w2 = 2 * P.box2 + 1, nq = (2 * P.box1 + 1) * w2;
  const int q0 = P.box1 * w2 + P.box2;  // the (0,0) column
  int off = 0, np = 0, m1max = 0, m2max = 0, m3max = 0;
  for (int q = 0; q < nq; ++q) P.bx_pair[q] = -1;
  // pair 0 = (0,0), always present
  P.bx_pair[q0] = np++;
  P.bx_off[q0] = off;
  off += P.bx_cnt[q0];
  m3max = P.bx_m3max[q0];
  for (int q = 0; q < nq; ++q) {
    if (q == q0 || P.bx_cnt[q] == 0) continue;
    const int m1 = q / w2 - P.box1, m2 = q % w2 - P.box2;
    P.bx_pair[q] = np++;
    P.bx_off[q] = off;
    off += P.bx_cnt[q];
    m1max = max(m1max, abs(m1));
    m2max = max(m2max, abs(m2));
    m3max = max(m3max, P.bx_m3max[q]);
  }
  P.setup_out[0] = off;
  P.setup_out[1] = np;
  P.setup_out[2] = m1max;
  P.setup_out[3] = m2max;
  P.setup_out[4] = m3max;
}

// Fill the tables (after the host allocated them with the sizes from the scan).
__global__ void k_basis_fill(KArgs ka) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  const Prob& P = ka.probs[p];
  const int w2 = 2 * P.box2 + 1;
  const int q = (blockIdx.x - ka.start[p]) * blockDim.x + threadIdx.x;
  if (q == 0) {
    P.cp_off[P.ncp] = P.nhalf;
    P.ekin[0] = 0.0;
    P.ekin32[0] = 0.f;
    for (int c = 0; c < 3; ++c) P.gvec[(size_t)c * P.ld] = 0.0;
  }
  if (q >= (2 * P.box1 + 1) * w2) return;
  const int pr = P.bx_pair[q];
  if (pr < 0) return;
  const int m1 = q / w2 - P.box1, m2 = q % w2 - P.box2;
  const bool zero = (m1 == 0 && m2 == 0);
  const int off = P.bx_off[q];
  P.cp_off[pr] = off;
  P.cp_m1[pr] = m1;
  P.cp_m2[pr] = m2;
  int e = off;
  for (int m3 = -P.box3; m3 <= P.box3; ++m3) {
    if (zero && m3 <= 0) continue;
    double G[3];
    gcart(P, m1, m2, m3, G);
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    if (0.5 * g2 > P.ecut) continue;
    P.ent_m[e] = m1;
    P.ent_m[P.nhalf + e] = m2;
    P.ent_m[2 * P.nhalf + e] = m3;
    P.ent_cp[e] = pr;
    P.ekin[1 + 2 * e] = 0.5 * g2;
    P.ekin[2 + 2 * e] = 0.5 * g2;
    P.ekin32[1 + 2 * e] = (float)(0.5 * g2);
    P.ekin32[2 + 2 * e] = (float)(0.5 * g2);
    for (int c = 0; c < 3; ++c) {
      P.gvec[(size_t)c * P.ld + 1 + 2 * e] = G[c];
      P.gvec[(size_t)c * P.ld + 2 + 2 * e] = G[c];
    }
    ++e;
  }
  // compact columns: pair 0 -> column 0; pair pr > 0 -> 2pr-1 (c+) and 2pr (c-)
  const int i1p = (m1 % P.n1 + P.n1) % P.n1, i2p = (m2 % P.n2 + P.n2) % P.n2;
  const int i1m = ((-m1) % P.n1 + P.n1) % P.n1, i2m = ((-m2) % P.n2 + P.n2) % P.n2;
  const int rows = 2 * P.m1max + 1, p2 = P.n2 | 1;
  auto sidx = [&](int i1, int i2) { return (i1 <= P.m1max ? i1 : i1 - P.n1 + rows) * p2 + i2; };
  if (pr == 0) {
    P.colmap[i1p * P.n2 + i2p] = 0;
    P.col_xy[0] = i1p * P.n2 + i2p;
    P.col_sidx[0] = sidx(i1p, i2p);
  } else {
    P.colmap[i1p * P.n2 + i2p] = 2 * pr - 1;
    P.col_xy[2 * pr - 1] = i1p * P.n2 + i2p;
    P.col_sidx[2 * pr - 1] = sidx(i1p, i2p);
    P.colmap[i1m * P.n2 + i2m] = 2 * pr;
    P.col_xy[2 * pr] = i1m * P.n2 + i2m;
    P.col_sidx[2 * pr] = sidx(i1m, i2m);
  }
}

// FFT twiddles exp(-2 pi i t / N_d), t < N_d, for the three axes, both precisions.
__global__ void k_roots(KArgs ka) {
  const int p = blockIdx.x;
  const Prob& P = ka.probs[p];
  const int tot = P.n1 + P.n2 + P.n3;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    int n, t;
    if (i < P.n1) { n = P.n1; t = i; }
    else if (i < P.n1 + P.n2) { n = P.n2; t = i - P.n1; }
    else { n = P.n3; t = i - P.n1 - P.n2; }
    double s, c;
    sincospi(-2.0 * t / n, &s, &c);
    P.roots64[i] = make_double2(c, s);
    P.roots32[i] = make_float2((float)c, (float)s);
  }
}

// Per-atom 1D phases exp(-i 2 pi m s_d) (s = fractional coordinates wrapped to [0,1)),
// indexed by grid index i_d with m = i_d or i_d - N_d.  CTA = (problem, atom).
__global__ void k_phases(KArgs ka) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int a = blockIdx.x - ka.start[p];
  double s[3];
  for (int d = 0; d < 3; ++d) {
    // s_d = R . b_d / (2 pi)
    double v = (P.pos[3 * a] * P.bvec[3 * d] + P.pos[3 * a + 1] * P.bvec[3 * d + 1] + P.pos[3 * a + 2] * P.bvec[3 * d + 2]) /
               (2.0 * PI);
    s[d] = v - floor(v);
  }
  const int tot = P.n1 + P.n2 + P.n3;
  double2* ph = P.phase + (size_t)a * tot;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    int n, t, d;
    if (i < P.n1) { n = P.n1; t = i; d = 0; }
    else if (i < P.n1 + P.n2) { n = P.n2; t = i - P.n1; d = 1; }
    else { n = P.n3; t = i - P.n1 - P.n2; d = 2; }
    int m = t < (n + 1) / 2 ? t : t - n;
    double x = -2.0 * m * s[d];
    x -= 2.0 * rint(0.5 * x);  // exact reduction of the argument (period 2 in units of pi)
    double sn, cs;
    sincospi(x, &sn, &cs);
    ph[i] = make_double2(cs, sn);
  }
}

// v_s(G) on the FFT box for every species (G = 0: the alpha term; Nyquist planes 0).
//   v_s(G) = (1/Omega) [-4 pi Z exp(-G^2 rc^2/4)/G^2 + A pi^{3/2} sigma^3 exp(-G^2 sigma^2/4)]
__global__ void k_vloc_table(KArgs ka) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  const Prob& P = ka.probs[p];
  const int base = (blockIdx.x - ka.start[p]) * 1024;
  const int end = min(P.ngrid, base + 1024);
  const double pi32 = PI * sqrt(PI);
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i2 = i % P.n2, t = i / P.n2, i1 = t % P.n1, i3 = t / P.n1;
    bool nyq = ((P.n1 & 1) == 0 && i1 == P.n1 / 2) || ((P.n2 & 1) == 0 && i2 == P.n2 / 2) ||
               ((P.n3 & 1) == 0 && i3 == P.n3 / 2);
    int m1 = i1 < (P.n1 + 1) / 2 ? i1 : i1 - P.n1;
    int m2 = i2 < (P.n2 + 1) / 2 ? i2 : i2 - P.n2;
    int m3 = i3 < (P.n3 + 1) / 2 ? i3 : i3 - P.n3;
    double g2 = g2_of(P, m1, m2, m3);
    P.g2box[i] = nyq ? -1.0 : g2;
    for (int s = 0; s < P.nspecies; ++s) {
      const double* sp = P.sp + s * 6;
      double Z = sp[0], rc = sp[1], A = sp[2], sg = sp[3];
      double v;
      if (nyq) v = 0.0;
      else if (g2 < 1e-14) v = (PI * Z * rc * rc + A * pi32 * sg * sg * sg) / P.omega;
      else
        v = (-4.0 * PI * Z * exp(-g2 * rc * rc * 0.25) / g2 + A * pi32 * sg * sg * sg * exp(-g2 * sg * sg * 0.25)) /
            P.omega;
      P.vloc_g[(size_t)s * P.ngrid + i] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Ewald (point charges Z_I in a neutralising background), FP64.
//   E = 1/2 sum' Z_I Z_J erfc(eta r)/r + (2 pi/Omega) sum_{G!=0} |S(G)|^2 exp(-G^2/4eta^2)/G^2
//     - eta/sqrt(pi) sum Z^2 - pi (sum Z)^2 / (2 Omega eta^2),  S(G) = sum_I Z_I exp(iG.R_I).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ew_ngbox(const Prob& P) {
  return (2 * P.ew_ng[0] + 1) * (2 * P.ew_ng[1] + 1) * (2 * P.ew_ng[2] + 1);
}
__device__ __forceinline__ void ew_gm(const Prob& P, int idx, int* m) {
  int w3 = 2 * P.ew_ng[2] + 1, w2 = 2 * P.ew_ng[1] + 1;
  m[2] = idx % w3 - P.ew_ng[2];
  idx /= w3;
  m[1] = idx % w2 - P.ew_ng[1];
  m[0] = idx / w2 - P.ew_ng[0];
}

// CTA = (problem, chunk of 256 G): S(G) table and the reciprocal energy partial.
__global__ void k_ewald_sg(KArgs ka) {
  __shared__ double red[33];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int chunk = blockIdx.x - ka.start[p];
  const int idx = chunk * 256 + threadIdx.x;
  double e = 0.0;
  if (idx < ew_ngbox(P)) {
    int m[3];
    ew_gm(P, idx, m);
    double G[3];
    gcart(P, m[0], m[1], m[2], G);
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    double sr = 0.0, si = 0.0;
    if (g2 > 1e-12 && g2 < P.ew_gmax * P.ew_gmax) {
      for (int a = 0; a < P.natom; ++a) {
        double z = P.sp[P.spec[a] * 6];
        double ph = G[0] * P.pos[3 * a] + G[1] * P.pos[3 * a + 1] + G[2] * P.pos[3 * a + 2];
        double s, c;
        sincos(ph, &s, &c);
        sr += z * c;
        si += z * s;
      }
      e = (sr * sr + si * si) * exp(-g2 / (4.0 * P.ew_eta * P.ew_eta)) / g2;
    }
    P.ew_sg[idx] = make_double2(sr, si);
  }
  e = block_sum(e, red);
  if (threadIdx.x == 0) P.ew_part[P.natom + chunk] = 2.0 * PI / P.omega * e;
}

// CTA = (problem, atom I): real-space energy share and the force on I.
__global__ void k_ewald_atom(KArgs ka) {
  __shared__ double red[33];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int I = blockIdx.x - ka.start[p];
  const double eta = P.ew_eta;
  const double zi = P.sp[P.spec[I] * 6];
  const int w0 = 2 * P.ew_nr[0] + 1, w1 = 2 * P.ew_nr[1] + 1, w2 = 2 * P.ew_nr[2] + 1;
  const int nimg = w0 * w1 * w2;
  double e = 0.0, f[3] = {0, 0, 0};
  for (int it = threadIdx.x; it < nimg * P.natom; it += blockDim.x) {
    int J = it / nimg, im = it % nimg;
    int l2 = im % w2 - P.ew_nr[2];
    int l1 = (im / w2) % w1 - P.ew_nr[1];
    int l0 = im / (w1 * w2) - P.ew_nr[0];
    double d[3];
    for (int c = 0; c < 3; ++c)
      d[c] = P.pos[3 * I + c] - P.pos[3 * J + c] + l0 * P.cell[c] + l1 * P.cell[3 + c] + l2 * P.cell[6 + c];
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r < 1e-12 || r >= P.ew_rmax) continue;
    double zz = zi * P.sp[P.spec[J] * 6];
    double ec = erfc(eta * r);
    e += 0.5 * zz * ec / r;
    double fac = zz * (ec / (r * r) + 2.0 * eta / sqrt(PI) * exp(-eta * eta * r * r) / r) / r;
    for (int c = 0; c < 3; ++c) f[c] += fac * d[c];
  }
  const int ng = ew_ngbox(P);
  for (int idx = threadIdx.x; idx < ng; idx += blockDim.x) {
    int m[3];
    ew_gm(P, idx, m);
    double G[3];
    gcart(P, m[0], m[1], m[2], G);
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    if (g2 <= 1e-12 || g2 >= P.ew_gmax * P.ew_gmax) continue;
    double w = exp(-g2 / (4.0 * eta * eta)) / g2;
    double ph = G[0] * P.pos[3 * I] + G[1] * P.pos[3 * I + 1] + G[2] * P.pos[3 * I + 2];
    double s, c;
    sincos(ph, &s, &c);
    double2 S = P.ew_sg[idx];
    // Im[exp(iG.R_I) S^*] = s Sr - c Si
    double im = s * S.x - c * S.y;
    double k = 4.0 * PI * zi / P.omega * w * im;
    for (int cc = 0; cc < 3; ++cc) f[cc] += k * G[cc];
  }
  e = block_sum(e, red);
  for (int c = 0; c < 3; ++c) {
    double t = block_sum(f[c], red);
    if (threadIdx.x == 0) P.ewald_f[3 * I + c] = t;
  }
  if (threadIdx.x == 0) P.ew_part[I] = e;
}

__global__ void k_ewald_reduce(KArgs ka) {
  const int p = blockIdx.x;
  if (!ka.active[p] || threadIdx.x != 0) return;
  const Prob& P = ka.probs[p];
  const int nch = (ew_ngbox(P) + 255) / 256;
  double e = 0.0, z2 = 0.0, zs = 0.0;
  for (int a = 0; a < P.natom; ++a) {
    e += P.ew_part[a];
    double z = P.sp[P.spec[a] * 6];
    z2 += z * z;
    zs += z;
  }
  for (int c = 0; c < nch; ++c) e += P.ew_part[P.natom + c];
  e -= P.ew_eta / sqrt(PI) * z2;
  e -= PI * zs * zs / (2.0 * P.omega * P.ew_eta * P.ew_eta);
  P.scal[SC_EEW] = e;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_basis_count(const Launch& L) {
  if (L.map.total) k_basis_count<<<L.map.total, 128, 0, L.stream>>>(L.ka);
}
void launch_basis_scan(const Launch& L) { k_basis_scan<<<L.ka.nprob, 32, 0, L.stream>>>(L.ka); }
void launch_basis_fill(const Launch& L) {
  if (L.map.total) k_basis_fill<<<L.map.total, 128, 0, L.stream>>>(L.ka);
}
void launch_roots(const Launch& L) { k_roots<<<L.ka.nprob, 128, 0, L.stream>>>(L.ka); }
void launch_phases(const Launch& Latoms) {
  if (Latoms.map.total) k_phases<<<Latoms.map.total, 128, 0, Latoms.stream>>>(Latoms.ka);
}
void launch_vloc_table(const Launch& Lew) {
  if (Lew.map.total) k_vloc_table<<<Lew.map.total, 256, 0, Lew.stream>>>(Lew.ka);
}
void launch_ewald(const Launch& Lsg, const Launch& Latoms, const Launch& Lprob) {
  if (Lsg.map.total) k_ewald_sg<<<Lsg.map.total, 256, 0, Lsg.stream>>>(Lsg.ka);
  if (Latoms.map.total) k_ewald_atom<<<Latoms.map.total, 256, 0, Latoms.stream>>>(Latoms.ka);
  k_ewald_reduce<<<Lprob.ka.nprob, 32, 0, Lprob.stream>>>(Lprob.ka);
}

}  // namespace sgo
