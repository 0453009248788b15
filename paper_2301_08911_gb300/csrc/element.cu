// Host-side constant tables: the hex8 element matrix, its macro-strain forces, the
// level-1 Galerkin tables and the filter weights.
//
// The element matrix is built from closed-form 1-D integrals of the trilinear shape
// functions (tensor-product structure) rather than by quadrature:
//   K0[(i,a),(j,b)] = lam * G^{ab}_{ij} + mu * G^{ba}_{ij} + mu * delta_ab * sum_c G^{cc}_{ij},
//   G^{ab}_{ij} = int over the unit cube of dN_i/dx_a * dN_j/dx_b,
// which is the bilinear form lam div u div v + 2 mu eps(u):eps(v) of isotropic
// elasticity (Sec. 3.2, E = 1) for a unit voxel.
#include <cmath>

#include "homo_internal.cuh"

namespace homo {

namespace {

// 1-D integrals on [0,1] of phi_0 = 1 - t, phi_1 = t and their derivatives.
double int_dd(int p, int q) { return p == q ? 1.0 : -1.0; }            // phi'_p phi'_q
double int_vv(int p, int q) { return p == q ? 1.0 / 3.0 : 1.0 / 6.0; }  // phi_p phi_q
double int_dv(int p, int /*q*/) { return p ? 0.5 : -0.5; }             // phi'_p phi_q

// G^{ab}_{ij} for unit cube, local vertices i, j (bit-coded offsets).
double grad_integral(int i, int a, int j, int b) {
  double v = 1.0;
  for (int d = 0; d < 3; ++d) {
    const int pi = (i >> d) & 1, pj = (j >> d) & 1;
    if (d == a && d == b) v *= int_dd(pi, pj);
    else if (d == a) v *= int_dv(pi, pj);
    else if (d == b) v *= int_dv(pj, pi);
    else v *= int_vv(pi, pj);
  }
  return v;
}

}  // namespace

void build_element_matrix(double nu, KeParam& ke, LoadParam& ld, ChiParam& chi) {
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  double K[24][24];
  for (int i = 0; i < 8; ++i)
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < 8; ++j)
        for (int b = 0; b < 3; ++b) {
          double v = lam * grad_integral(i, a, j, b) + mu * grad_integral(i, b, j, a);
          if (a == b)
            for (int c = 0; c < 3; ++c) v += mu * grad_integral(i, c, j, c);
          K[3 * i + a][3 * j + b] = v;
        }
  for (int r = 0; r < 24; ++r)
    for (int c = 0; c < 24; ++c) ke.k[r * 24 + c] = static_cast<float>(K[r][c]);

  // chi_i at local vertex j with coordinates (x0,x1,x2) in {0,1}^3 (Eq. 12).
  double X[6][24] = {};
  for (int j = 0; j < 8; ++j) {
    const double x0 = j & 1, x1 = (j >> 1) & 1, x2 = (j >> 2) & 1;
    double* c;
    c = &X[0][3 * j]; c[0] = x0;
    c = &X[1][3 * j]; c[1] = x1;
    c = &X[2][3 * j]; c[2] = x2;
    c = &X[3][3 * j]; c[0] = x1 / 2; c[1] = x0 / 2;
    c = &X[4][3 * j]; c[1] = x2 / 2; c[2] = x1 / 2;
    c = &X[5][3 * j]; c[0] = x2 / 2; c[2] = x0 / 2;
  }
  for (int i = 0; i < kCases; ++i)
    for (int r = 0; r < 24; ++r) {
      double s = 0;
      for (int c = 0; c < 24; ++c) s += K[r][c] * X[i][c];
      ld.fe[i][r] = static_cast<float>(s);
      ld.fe_lo[i][r] = static_cast<float>(s - static_cast<double>(ld.fe[i][r]));
      chi.chi[i][r] = static_cast<float>(X[i][r]);
    }
}

// B_f = P_f^T K0 P_f for the 8 fine elements f of a coarse element, where P_f maps the
// coarse element's 24 nodal values to fine element f's 24 nodal values by trilinear
// interpolation: weight of coarse local vertex J at fine local vertex j is
// prod over axes (1 - |f_d + j_d - 2 J_d| / 2). Summing E_f B_f over f gives the
// Galerkin coarse element matrix (Eq. 17-18 grouped by coarse element).
void build_level1_tables(const KeParam& ke, float* Bf) {
  for (int f = 0; f < 8; ++f) {
    double P[8][8];
    for (int j = 0; j < 8; ++j)
      for (int J = 0; J < 8; ++J) {
        double w = 1.0;
        for (int d = 0; d < 3; ++d) {
          const int pos = ((f >> d) & 1) + ((j >> d) & 1) - 2 * ((J >> d) & 1);
          w *= 1.0 - std::fabs(static_cast<double>(pos)) / 2.0;
        }
        P[j][J] = w < 0 ? 0.0 : w;
      }
    for (int J = 0; J < 8; ++J)
      for (int a = 0; a < 3; ++a)
        for (int L = 0; L < 8; ++L)
          for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int j = 0; j < 8; ++j) {
              if (P[j][J] == 0) continue;
              for (int l = 0; l < 8; ++l) {
                if (P[l][L] == 0) continue;
                s += P[j][J] * static_cast<double>(ke.k[(3 * j + a) * 24 + 3 * l + b]) * P[l][L];
              }
            }
            Bf[f * 576 + (3 * J + a) * 24 + 3 * L + b] = static_cast<float>(s);
          }
  }
}

// Eigen-decomposition of a symmetric n x n matrix (n <= 8) by cyclic Jacobi rotations in
// double: on return a is diagonal (the eigenvalues) and column k of v is eigenvector k.
void sym_eigen(int n, double* a, double* v) {
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) v[r * n + c] = r == c ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (std::fabs(a[p * n + q]) < 1e-300) continue;
        const double th = 0.5 * std::atan2(2 * a[p * n + q], a[q * n + q] - a[p * n + p]);
        const double cs = std::cos(th), sn = std::sin(th);
        for (int k = 0; k < n; ++k) {   // rotate columns p, q
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = cs * akp - sn * akq;
          a[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {   // rotate rows p, q
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = cs * apk - sn * aqk;
          a[q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = cs * vkp - sn * vkq;
          v[k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
}

// Largest eigenvalue of D_e^-1 K0, D_e the 3x3 block diagonal of K0. With
// x^T K x = sum_e E_e x_e^T K0 x_e <= lam sum_e E_e x_e^T D_e x_e = lam x^T D x it bounds
// the spectrum of D^-1 K on the finest level for any moduli E. Power iteration on the
// symmetric similar matrix D^-1/2 K0 D^-1/2, in double.
double element_jacobi_bound(const KeParam& ke) {
  double K[24][24], Dinvh[8][3][3];
  for (int r = 0; r < 24; ++r)
    for (int c = 0; c < 24; ++c) K[r][c] = 0.5 * (ke.k[r * 24 + c] + ke.k[c * 24 + r]);
  // D^-1/2 per 3x3 block by its eigen-decomposition (Jacobi rotations)
  for (int j = 0; j < 8; ++j) {
    double a[3][3], v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) a[r][c] = K[3 * j + r][3 * j + c];
    for (int sweep = 0; sweep < 50; ++sweep)
      for (int p = 0; p < 3; ++p)
        for (int q = p + 1; q < 3; ++q) {
          if (std::fabs(a[p][q]) < 1e-300) continue;
          const double th = 0.5 * std::atan2(2 * a[p][q], a[q][q] - a[p][p]);
          const double cs = std::cos(th), sn = std::sin(th);
          for (int k = 0; k < 3; ++k) {   // rotate columns p, q
            const double akp = a[k][p], akq = a[k][q];
            a[k][p] = cs * akp - sn * akq;
            a[k][q] = sn * akp + cs * akq;
          }
          for (int k = 0; k < 3; ++k) {   // rotate rows p, q
            const double apk = a[p][k], aqk = a[q][k];
            a[p][k] = cs * apk - sn * aqk;
            a[q][k] = sn * apk + cs * aqk;
          }
          for (int k = 0; k < 3; ++k) {
            const double vkp = v[k][p], vkq = v[k][q];
            v[k][p] = cs * vkp - sn * vkq;
            v[k][q] = sn * vkp + cs * vkq;
          }
        }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += v[r][k] * v[c][k] / std::sqrt(a[k][k]);
        Dinvh[j][r][c] = s;
      }
  }
  double M[24][24];
  for (int r = 0; r < 24; ++r)
    for (int c = 0; c < 24; ++c) {
      double s = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          s += Dinvh[r / 3][r % 3][a] * K[3 * (r / 3) + a][3 * (c / 3) + b] * Dinvh[c / 3][b][c % 3];
      M[r][c] = s;
    }
  double x[24], y[24], lam = 0;
  for (int i = 0; i < 24; ++i) x[i] = 1.0 + 0.01 * i;
  for (int it = 0; it < 2000; ++it) {
    double nrm = 0;
    for (int r = 0; r < 24; ++r) {
      double s = 0;
      for (int c = 0; c < 24; ++c) s += M[r][c] * x[c];
      y[r] = s;
      nrm += s * s;
    }
    nrm = std::sqrt(nrm);
    double rq = 0;
    for (int r = 0; r < 24; ++r) rq += x[r] * y[r];
    lam = rq;
    for (int r = 0; r < 24; ++r) x[r] = y[r] / nrm;
  }
  return lam;
}

int build_filter_param(double radius, FilterParam& fp) {
  if (!(radius > 0.0) || radius > 3.5) return HOMO_EINVAL;
  const int R = static_cast<int>(std::ceil(radius));
  int cnt = 0;
  double wsum = 0.0;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        const double w = radius - std::sqrt(static_cast<double>(dx * dx + dy * dy + dz * dz));
        if (w <= 0.0) continue;
        if (cnt >= 343) return HOMO_EINVAL;
        fp.off[cnt][0] = static_cast<signed char>(dx);
        fp.off[cnt][1] = static_cast<signed char>(dy);
        fp.off[cnt][2] = static_cast<signed char>(dz);
        fp.w[cnt] = static_cast<float>(w);
        wsum += w;
        ++cnt;
      }
  fp.count = cnt;
  fp.inv_wsum = static_cast<float>(1.0 / wsum);
  return HOMO_OK;
}

}  // namespace homo
