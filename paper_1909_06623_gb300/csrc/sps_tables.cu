// Host-side spherical-harmonic tables for one order p.
//
//  * Grid (Sec. 5.4): p+1 Gauss-Legendre rings in cos(theta) (Newton iteration
//    on P_{p+1}) times 2p+2 uniform azimuths; (p+1)(2p+2) nodes, the count
//    behind the 486 unknowns per sphere quoted at p = 8 (Sec. 6.5).
//  * Y_n^m (Sec. 4.2): orthonormal, Condon-Shortley phase, built from the
//    standard three-term recurrences of the normalised associated Legendre
//    functions; dY/dtheta from the ladder relation
//      dPbar_n^m/dtheta = (sqrt((n-m)(n+m+1)) Pbar_n^{m+1}
//                          - sqrt((n+m)(n-m+1)) Pbar_n^{m-1}) / 2,
//    Pbar_n^{-1} = -Pbar_n^1.
//  * VSH (Sec. 4.2, eq. rhoshexp): V = G - (n+1) Y e_r, W = G + n Y e_r,
//    X = e_r x G, G = grad_Gamma Y; |V|^2 = (n+1)(2n+1), |W|^2 = n(2n+1),
//    |X|^2 = n(n+1).  Analysis rows give <sigma, conj(B)>/|B|^2 for m >= 0;
//    synthesis folds m < 0 by conjugate symmetry (factor 2 for m > 0).
//  * Self multipliers per degree (Sec. 4.2): on-surface single layer from
//    eq. ssgext at r = 1 (V: n/((2n+1)(2n+3)), W: (n+1)/((2n-1)(2n+1)),
//    X: 1/(2n+1)); principal-value traction = exterior traction at r -> 1+
//    plus half the density, the exterior traction of a degree-n mode being
//    V: -2n(n+2)/((2n+1)(2n+3)), W: -(2n^2+1)/((2n-1)(2n+1)), X: -(n+2)/(2n+1)
//    (from the single-layer jump conditions; the paper defers these maps to
//    its reference on VSH for spheres).
//  * kappa_nm: r^{-(n+1)} Y_n^m = kappa_nm H_n^m with H_n^m = (d_x + i d_y)^m
//    d_z^{n-m} (1/r), kappa_nm = (-1)^{n+m} sqrt((2n+1)/(4 pi)) /
//    sqrt((n-m)! (n+m)!).
#include <cmath>
#include <complex>
#include <cstring>

#include "sps_internal.cuh"

namespace sps {

static void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w) {
  t.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    // k-th root from the top, then stored ascending
    double x = std::cos(SPS_PI * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? x : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      double dp = n * (x * pn - pnm1) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) {
        if (it > 2) break;
      }
    }
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? x : p1, pnm1 = (n == 1) ? 1.0 : p0;
    double dp = n * (x * pn - pnm1) / (x * x - 1.0);
    t[n - 1 - k] = x;
    w[n - 1 - k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Normalised associated Legendre Pbar_n^m(cos theta), 0 <= m <= n <= L,
// stored at [n*(L+1) + m]; Condon-Shortley phase included.
static void legendre_table(int L, double ct, double st, std::vector<double>& P) {
  P.assign((L + 1) * (L + 1), 0.0);
  P[0] = 1.0 / std::sqrt(4.0 * SPS_PI);
  for (int m = 1; m <= L; ++m)
    P[m * (L + 1) + m] = -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * P[(m - 1) * (L + 1) + m - 1];
  for (int m = 0; m < L; ++m)
    P[(m + 1) * (L + 1) + m] = std::sqrt(2.0 * m + 3.0) * ct * P[m * (L + 1) + m];
  for (int m = 0; m <= L; ++m)
    for (int n = m + 2; n <= L; ++n) {
      double a = std::sqrt((4.0 * n * n - 1.0) / (double(n) * n - double(m) * m));
      double b = std::sqrt(((n - 1.0) * (n - 1.0) - double(m) * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
      P[n * (L + 1) + m] = a * (ct * P[(n - 1) * (L + 1) + m] - b * P[(n - 2) * (L + 1) + m]);
    }
}

void build_tables(int p, Tables& T) {
  T.p = p;
  const int nphi = 2 * p + 2;
  T.P = (p + 1) * nphi;
  T.NC = (p + 1) * (p + 2) / 2;
  T.NR = 6 * T.NC;
  T.L = p + 2;
  T.E = (T.L + 1) * (T.L + 2) / 2;
  const int P = T.P, NC = T.NC, NR = T.NR;
  gauss_legendre(p + 1, T.t, T.wgl);

  T.unit_nrm.assign(3 * P, 0.0);
  T.unit_w.assign(P, 0.0);
  T.anal.assign((size_t)NR * 3 * P, 0.0);
  T.synth.assign((size_t)3 * P * NR, 0.0);
  T.multS.assign(NR, 0.0);
  T.multK.assign(NR, 0.0);
  T.kappa.assign(NC, 0.0);
  // near-field potentials per degree n (eq. ssgext in Lamb form):
  //   0 a (on sW): n/(2(2n+1))       5 a (on sV): n/((2n+1)(2n+3))
  //   1 d (on sX): 1/(2n+1)          2 alpha (on sW): (2-n)/(2(2n-1))
  //   3 beta (on sW): (n+1)/(2n-1)   4 2 beta - P (on sW): 2(n+1)/(2n-1) - n
  T.potfac.assign((size_t)(p + 1) * 6, 0.0);
  for (int n = 0; n <= p; ++n) {
    const double d = n;
    double* f = &T.potfac[(size_t)n * 6];
    f[0] = d / (2 * (2 * d + 1));
    f[1] = 1.0 / (2 * d + 1);
    f[2] = (2 - d) / (2 * (2 * d - 1));
    f[3] = (d + 1) / (2 * d - 1);
    f[4] = 2 * (d + 1) / (2 * d - 1) - d;
    f[5] = d / ((2 * d + 1) * (2 * d + 3));
  }

  std::vector<double> Pl;
  const int Lq = p + 1;  // Pbar up to degree p+1 for the ladder relation
  for (int k = 0; k <= p; ++k) {
    const double ct = T.t[k], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    legendre_table(Lq, ct, st, Pl);
    auto Pb = [&](int n, int m) -> double {
      if (m < 0) return (m == -1) ? -Pl[n * (Lq + 1) + 1] : 0.0;
      if (m > n) return 0.0;
      return Pl[n * (Lq + 1) + m];
    };
    for (int l = 0; l < nphi; ++l) {
      const int node = k * nphi + l;
      const double ph = 2.0 * SPS_PI * l / nphi;
      const double cp = std::cos(ph), sp = std::sin(ph);
      const double er[3] = {st * cp, st * sp, ct};
      const double et[3] = {ct * cp, ct * sp, -st};
      const double ep[3] = {-sp, cp, 0.0};
      T.unit_nrm[0 * P + node] = er[0];
      T.unit_nrm[1 * P + node] = er[1];
      T.unit_nrm[2 * P + node] = er[2];
      const double w = T.wgl[k] * 2.0 * SPS_PI / nphi;
      T.unit_w[node] = w;
      for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
          const std::complex<double> E(std::cos(m * ph), std::sin(m * ph));
          const double pb = Pb(n, m);
          const double dpb = 0.5 * (std::sqrt(double(n - m) * (n + m + 1)) * Pb(n, m + 1) -
                                    std::sqrt(double(n + m) * (n - m + 1)) * Pb(n, m - 1));
          const std::complex<double> Y = pb * E, Yt = dpb * E;
          const std::complex<double> Yps = std::complex<double>(0.0, m) * (pb / st) * E;  // (1/s) dY/dphi
          std::complex<double> B[3][3];  // [type][cartesian]
          for (int c = 0; c < 3; ++c) {
            const std::complex<double> G = Yt * et[c] + Yps * ep[c];
            B[0][c] = G - double(n + 1) * Y * er[c];
            B[1][c] = G + double(n) * Y * er[c];
            B[2][c] = Yt * ep[c] - Yps * et[c];
          }
          const double nrm2[3] = {double(n + 1) * (2 * n + 1), double(n) * (2 * n + 1), double(n) * (n + 1)};
          const int ci = n * (n + 1) / 2 + m;
          const double eps = (m == 0) ? 1.0 : 2.0;
          for (int ty = 0; ty < 3; ++ty) {
            const int r0 = (ty * NC + ci) * 2;
            for (int c = 0; c < 3; ++c) {
              const int col = c * P + node;
              if (nrm2[ty] > 0) {
                T.anal[(size_t)r0 * 3 * P + col] = w * B[ty][c].real() / nrm2[ty];
                T.anal[(size_t)(r0 + 1) * 3 * P + col] = -w * B[ty][c].imag() / nrm2[ty];
              }
              T.synth[(size_t)col * NR + r0] = eps * B[ty][c].real();
              T.synth[(size_t)col * NR + r0 + 1] = -eps * B[ty][c].imag();
            }
          }
        }
    }
  }
  for (int n = 0; n <= p; ++n) {
    const double dn = n;
    const double sV = dn / ((2 * dn + 1) * (2 * dn + 3));
    const double sW = (dn + 1) / ((2 * dn - 1) * (2 * dn + 1));
    const double sX = 1.0 / (2 * dn + 1);
    const double kV = 0.5 - 2 * dn * (dn + 2) / ((2 * dn + 1) * (2 * dn + 3));
    const double kW = 0.5 - (2 * dn * dn + 1) / ((2 * dn - 1) * (2 * dn + 1));
    const double kX = 0.5 - (dn + 2) / (2 * dn + 1);
    for (int m = 0; m <= n; ++m) {
      const int ci = n * (n + 1) / 2 + m;
      const double ms[3] = {sV, n ? sW : 0.0, n ? sX : 0.0};
      const double mk[3] = {kV, n ? kW : 0.0, n ? kX : 0.0};
      for (int ty = 0; ty < 3; ++ty)
        for (int ri = 0; ri < 2; ++ri) {
          T.multS[(ty * NC + ci) * 2 + ri] = ms[ty];
          T.multK[(ty * NC + ci) * 2 + ri] = mk[ty];
        }
      double f = std::sqrt((2 * dn + 1) / (4 * SPS_PI)) /
                 std::sqrt(std::tgamma(n - m + 1.0) * std::tgamma(n + m + 1.0));
      T.kappa[ci] = ((n + m) % 2 ? -1.0 : 1.0) * f;
    }
  }
}

}  // namespace sps

extern "C" int sps_unit_tables(int p, double* nodes, double* weights, double* analysis,
                               double* synthesis) {
  if (p < 1 || p > sps::kMaxP) return SPS_ERR_INVALID_ARG;
  sps::Tables T;
  sps::build_tables(p, T);
  if (nodes) std::memcpy(nodes, T.unit_nrm.data(), T.unit_nrm.size() * sizeof(double));
  if (weights) std::memcpy(weights, T.unit_w.data(), T.unit_w.size() * sizeof(double));
  if (analysis) std::memcpy(analysis, T.anal.data(), T.anal.size() * sizeof(double));
  if (synthesis) std::memcpy(synthesis, T.synth.data(), T.synth.size() * sizeof(double));
  return SPS_OK;
}
