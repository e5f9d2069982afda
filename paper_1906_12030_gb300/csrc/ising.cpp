// Blocked critical-Ising Hamiltonian density (Eq. ham, Sec. II B), host code.
//
// Spins are blocked in pairs, so one lattice site carries local dimension 4
// (basis index 2*s0 + s1).  The 3-site density is
//   h3 = (h2 (x) 1 + 1 (x) h2) / 2,
// with h2 the coupling of two neighbouring blocked sites: the bond inside
// each block (shared by two pairs, weight 1/2), the bond between the blocks
// (weight 1), each bond being -X X - (hz/2)(Z 1 + 1 Z).  The largest
// eigenvalue of h3 (cyclic Jacobi rotations) is subtracted so that h1 is
// negative semidefinite.
#include <cmath>
#include <vector>

#include "../../include/mera.h"

namespace {

using Mat = std::vector<double>;  // row-major n x n

Mat kron(const Mat& a, int na, const Mat& b, int nb) {
  const int n = na * nb;
  Mat c(size_t(n) * n, 0.0);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < na; ++j)
      for (int k = 0; k < nb; ++k)
        for (int l = 0; l < nb; ++l) c[size_t(i * nb + k) * n + (j * nb + l)] = a[i * na + j] * b[k * nb + l];
  return c;
}

Mat eye(int n) {
  Mat e(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) e[size_t(i) * n + i] = 1.0;
  return e;
}

void axpy(Mat& y, double a, const Mat& x) {
  for (size_t i = 0; i < y.size(); ++i) y[i] += a * x[i];
}

// Largest eigenvalue of a symmetric matrix by cyclic Jacobi sweeps.
double max_eigenvalue(Mat a, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  double mx = a[0];
  for (int i = 1; i < n; ++i) mx = std::max(mx, a[i * n + i]);
  return mx;
}

}  // namespace

extern "C" mera_status mera_ising_h1(double hz, double* h1_host, double* shift_host) {
  if (!h1_host || !shift_host || !std::isfinite(hz)) return MERA_EINVAL;
  const Mat X = {0, 1, 1, 0}, Z = {1, 0, 0, -1}, I2 = eye(2);
  Mat bond = kron(X, 2, X, 2);
  for (double& v : bond) v = -v;
  axpy(bond, -0.5 * hz, kron(Z, 2, I2, 2));
  axpy(bond, -0.5 * hz, kron(I2, 2, Z, 2));
  // h2 on spins (0,1 | 2,3)
  Mat h2(256, 0.0);
  axpy(h2, 0.5, kron(bond, 4, eye(4), 4));
  axpy(h2, 1.0, kron(kron(I2, 2, bond, 4), 8, I2, 2));
  axpy(h2, 0.5, kron(eye(4), 4, bond, 4));
  Mat h3(64 * 64, 0.0);
  axpy(h3, 0.5, kron(h2, 16, eye(4), 4));
  axpy(h3, 0.5, kron(eye(4), 4, h2, 16));
  const double s = max_eigenvalue(h3, 64);
  for (int i = 0; i < 64 * 64; ++i) h1_host[i] = h3[i] - ((i / 64 == i % 64) ? s : 0.0);
  *shift_host = s;
  return MERA_OK;
}
