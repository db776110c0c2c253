// Host-side check of the compensated FP32 polar factors of the particle passes
// (polar_refine2 / polar_refine3 in mpm_common.cuh, compiled here as host code) against an
// extended-precision (long double) reference on random deformation gradients F = R S:
// random rotations (and small ones), symmetric stretches with strains from 1e-6 to 0.6.
// Prints one line per dimension: cases, failures, max |R - R_ref|, max |(F - R) - (F - R)_ref|
// relative to max |F - R|_ref (per case).
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1910_00935_gb300/csrc/mpm_common.cuh"

using mpm::polar_newton3;
using mpm::polar_refine2;
using mpm::polar_refine3;

// reference polar factor of F (3x3): Newton's iteration X <- (X + X^-T)/2 in long double
static void ref_polar3(const long double F[3][3], long double R[3][3]) {
  long double X[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = F[i][j];
  for (int it = 0; it < 60; ++it) {
    long double c[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        c[i][j] = X[i1][j1] * X[i2][j2] - X[i1][j2] * X[i2][j1];
      }
    const long double det = X[0][0] * c[0][0] + X[0][1] * c[0][1] + X[0][2] * c[0][2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) X[i][j] = 0.5L * X[i][j] + 0.5L * c[i][j] / det;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = X[i][j];
}

int main() {
  std::mt19937_64 g(1);
  std::normal_distribution<double> nd(0.0, 1.0);
  // 3D
  {
    const int n = 20000;
    int fails = 0;
    double wR = 0.0, wD = 0.0;
    for (int t = 0; t < n; ++t) {
      double q[4], qn = 0.0;
      for (double& v : q) {
        v = nd(g);
        qn += v * v;
      }
      qn = std::sqrt(qn);
      for (double& v : q) v /= qn;
      double Rq[3][3] = {{1 - 2 * (q[2] * q[2] + q[3] * q[3]), 2 * (q[1] * q[2] - q[0] * q[3]), 2 * (q[1] * q[3] + q[0] * q[2])},
                         {2 * (q[1] * q[2] + q[0] * q[3]), 1 - 2 * (q[1] * q[1] + q[3] * q[3]), 2 * (q[2] * q[3] - q[0] * q[1])},
                         {2 * (q[1] * q[3] - q[0] * q[2]), 2 * (q[2] * q[3] + q[0] * q[1]), 1 - 2 * (q[1] * q[1] + q[2] * q[2])}};
      if (t % 3 == 0) {  // small rotations about z
        const double a = 1e-3 * nd(g), c = std::cos(a), s = std::sin(a);
        const double Rs[3][3] = {{c, -s, 0}, {s, c, 0}, {0, 0, 1}};
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) Rq[i][j] = Rs[i][j];
      }
      const double mag = std::pow(10.0, -6.0 + 5.8 * (t % 97) / 96.0);
      double A[3][3], S[3][3], F[3][3];
      for (auto& r : A)
        for (double& v : r) v = nd(g) * mag / 3.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = (i == j ? 1.0 : 0.0) + 0.5 * (A[i][j] + A[j][i]);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          F[i][j] = 0.0;
          for (int k = 0; k < 3; ++k) F[i][j] += Rq[i][k] * S[k][j];
        }
      float E[3][3], Q[3][3];
      long double Fl[3][3], Rr[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          E[i][j] = (float)(F[i][j] - (i == j ? 1.0 : 0.0));
          Fl[i][j] = (long double)E[i][j] + (i == j ? 1.0L : 0.0L);
          Q[i][j] = E[i][j] + (i == j ? 1.0f : 0.0f);
        }
      ref_polar3(Fl, Rr);
      float Rh[3][3], Rl[3][3], Df[3][3];
      if (!polar_newton3<float>(Q, 1e-12f, 20) || !polar_refine3(E, Q, Rh, Rl, Df)) {
        ++fails;
        continue;
      }
      double eR = 0.0, nD = 0.0, eD = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          eR = std::fmax(eR, (double)fabsl((long double)Rh[i][j] + Rl[i][j] - Rr[i][j]));
          const long double d = Fl[i][j] - Rr[i][j];
          nD = std::fmax(nD, (double)fabsl(d));
          eD = std::fmax(eD, (double)fabsl((long double)Df[i][j] - d));
        }
      wR = std::fmax(wR, eR);
      if (nD > 0.0) wD = std::fmax(wD, eD / nD);
    }
    std::printf("3d %d %d %.6e %.6e\n", n, fails, wR, wD);
  }
  // 2D
  {
    const int n = 50000;
    int fails = 0;
    double wR = 0.0, wD = 0.0;
    for (int t = 0; t < n; ++t) {
      const double th = (t % 4 == 0) ? 1e-3 * nd(g) : 3.0 * nd(g);
      const double mag = std::pow(10.0, -6.0 + 5.8 * (t % 97) / 96.0);
      const double a = nd(g) * mag / 2, b = nd(g) * mag / 2, c2 = nd(g) * mag / 2;
      const double S[2][2] = {{1 + a, c2}, {c2, 1 + b}};
      const double Rq[2][2] = {{std::cos(th), -std::sin(th)}, {std::sin(th), std::cos(th)}};
      float E[2][2];
      long double Fl[2][2];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          const double f = Rq[i][0] * S[0][j] + Rq[i][1] * S[1][j];
          E[i][j] = (float)(f - (i == j ? 1.0 : 0.0));
          Fl[i][j] = (long double)E[i][j] + (i == j ? 1.0L : 0.0L);
        }
      const long double cc = Fl[0][0] + Fl[1][1], ss = Fl[1][0] - Fl[0][1], rr = sqrtl(cc * cc + ss * ss);
      const long double R[2][2] = {{cc / rr, -ss / rr}, {ss / rr, cc / rr}};
      const long double det = Fl[0][0] * Fl[1][1] - Fl[0][1] * Fl[1][0];
      float Rh[2][2], Rl[2][2], Df[2][2];
      const bool ok = polar_refine2(E, Rh, Rl, Df);
      if (!(det > 0.0L)) {  // inverted: refused, as intended
        if (ok) ++fails;
        continue;
      }
      if (!ok) {
        ++fails;
        continue;
      }
      double eR = 0.0, nD = 0.0, eD = 0.0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          eR = std::fmax(eR, (double)fabsl((long double)Rh[i][j] + Rl[i][j] - R[i][j]));
          const long double d = Fl[i][j] - R[i][j];
          nD = std::fmax(nD, (double)fabsl(d));
          eD = std::fmax(eD, (double)fabsl((long double)Df[i][j] - d));
        }
      wR = std::fmax(wR, eR);
      if (nD > 0.0) wD = std::fmax(wD, eD / nD);
    }
    std::printf("2d %d %d %.6e %.6e\n", n, fails, wR, wD);
  }
  return 0;
}
