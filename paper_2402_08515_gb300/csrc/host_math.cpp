// Host-side arithmetic of the kes library: filter weights (eq. weightf,
// eq. disc_filtercoeff), the discrete filter response (eq. scalartimestep,
// eq. fullydiscfilter) and the dense symmetric eigensolver used for the
// projected problem (eq. projevp).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <limits>
#include <vector>

#include "kes_internal.h"

namespace kes {

// alpha_n = tau * alpha(n tau), n = 0..L, T = L tau. alpha(0) is the t -> 0 limit
// 2 (wmax - wmin) / pi of eq. (weightf); on (0, T] the weight is
// 4 / (pi t) sin(t (wmax - wmin) / 2) cos(t (wmax + wmin) / 2).
void alpha_table(double wmin, double wmax, double tau, int L, double* alpha) {
  const double pi = 3.14159265358979323846;
  alpha[0] = tau * 2.0 * (wmax - wmin) / pi;
  const double half_width = 0.5 * (wmax - wmin);
  const double half_centre = 0.5 * (wmax + wmin);
  for (int n = 1; n <= L; ++n) {
    const double t = n * tau;
    alpha[n] = tau * (4.0 / (pi * t)) * std::sin(t * half_width) * std::cos(t * half_centre);
  }
}

// Gaussian pass band (Sec. 4, "Weight function"): the inverse cosine transform
// alpha(t) = (2/pi) int_0^inf beta(s) cos(ts) ds of the even band
// beta(s) = exp(-(s-c)^2/(2 sigma^2)) + exp(-(s+c)^2/(2 sigma^2)) is
// 2 sigma sqrt(2/pi) exp(-sigma^2 t^2 / 2) cos(c t); alpha_n = tau alpha(n tau).
void alpha_gaussian(double center, double sigma, double tau, int L, double* alpha) {
  const double pi = 3.14159265358979323846;
  const double amp = 2.0 * sigma * std::sqrt(2.0 / pi);
  for (int n = 0; n <= L; ++n) {
    const double t = n * tau;
    alpha[n] = tau * amp * std::exp(-0.5 * sigma * sigma * t * t) * std::cos(center * t);
  }
}

// Triangular pass band: for the even band hat(s - c) + hat(s + c) with
// hat(u) = max(0, 1 - |u|/h), the same transform gives alpha(t) = (2h/pi) cos(c t)
// (sin(t h/2) / (t h/2))^2 (the hat's cosine integral is h times the squared sinc).
void alpha_triangle(double center, double half_width, double tau, int L, double* alpha) {
  const double pi = 3.14159265358979323846;
  for (int n = 0; n <= L; ++n) {
    const double t = n * tau;
    const double x = 0.5 * t * half_width;
    const double sinc = x == 0.0 ? 1.0 : std::sin(x) / x;
    alpha[n] = tau * 2.0 * half_width / pi * std::cos(center * t) * sinc * sinc;
  }
}

// beta~(omega) = sum_n alpha_n q_n(omega); q_{-1} = q_0 = 1,
// q_{n+1} = (2 - tau^2 omega^2) q_n - q_{n-1}.
void filter_response(double wmin, double wmax, double tau, int L, const double* omega, int64_t k,
                     double* beta) {
  std::vector<double> alpha(L + 1);
  alpha_table(wmin, wmax, tau, L, alpha.data());
  weights_response(alpha.data(), tau, L, omega, k, beta);
}

void weights_response(const double* alpha, double tau, int L, const double* omega, int64_t k, double* beta) {
  for (int64_t i = 0; i < k; ++i) {
    const double two_minus = 2.0 - tau * tau * omega[i] * omega[i];
    double q_prev = 1.0, q = 1.0, sum = alpha[0];
    for (int n = 1; n <= L; ++n) {
      const double q_next = two_minus * q - q_prev;
      q_prev = q;
      q = q_next;
      sum += alpha[n] * q;
    }
    beta[i] = sum;
  }
}

// ---------------------------------------------------------------------------
// Symmetric eigensolver (Golub & Van Loan, "Matrix Computations", Sec. 8.3:
// Householder tridiagonalisation, then implicit symmetric QR steps with the
// Wilkinson shift, eigenvectors accumulated).
// ---------------------------------------------------------------------------
// Blocks of at least this many rows or columns run their loops on OpenMP threads.
constexpr int kParallelEig = 256;

bool sym_eig(int k, const double* Ain, double* w, double* Vout) {
  if (k <= 0) return true;
  // full symmetric copy from the lower triangle
  std::vector<double> A(static_cast<size_t>(k) * k);
  auto a = [&](int i, int j) -> double& { return A[static_cast<size_t>(j) * k + i]; };
  for (int j = 0; j < k; ++j)
    for (int i = j; i < k; ++i) {
      a(i, j) = Ain[static_cast<size_t>(j) * k + i];
      a(j, i) = a(i, j);
    }
  std::vector<double> d(k), e(std::max(k - 1, 1), 0.0);
  std::vector<std::vector<double>> hv;  // Householder vectors (on rows j+1..k-1)
  std::vector<double> hbeta;
  std::vector<double> p(k), q(k);
  for (int j = 0; j + 2 < k; ++j) {
    const int m = k - j - 1;
    std::vector<double> v(m);
    double nrm2 = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = a(j + 1 + i, j);
      nrm2 += v[i] * v[i];
    }
    const double nrm = std::sqrt(nrm2);
    if (nrm == 0.0) {
      e[j] = 0.0;
      hv.emplace_back();
      hbeta.push_back(0.0);
      continue;
    }
    const double x0 = v[0];
    const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
    v[0] = x0 + sgn * nrm;
    const double vtv = nrm2 - x0 * x0 + v[0] * v[0];
    const double beta = 2.0 / vtv;
    e[j] = -sgn * nrm;
    // p = beta * A22 v ; q = p - (beta/2)(p.v) v ; A22 -= v q^T + q v^T
    // (the loops over independent rows or columns run on host threads for large blocks;
    // nothing is reduced across threads, so the result does not depend on their number)
#pragma omp parallel for schedule(static) if (m >= kParallelEig)
    for (int r = 0; r < m; ++r) {
      // row r of the trailing block read down its column (the block stays exactly
      // symmetric: both triangles get the same rank-2 update)
      double s = 0.0;
      for (int c = 0; c < m; ++c) s += a(j + 1 + c, j + 1 + r) * v[c];
      p[r] = beta * s;
    }
    double pv = 0.0;
    for (int r = 0; r < m; ++r) pv += p[r] * v[r];
    const double K = 0.5 * beta * pv;
    for (int r = 0; r < m; ++r) q[r] = p[r] - K * v[r];
#pragma omp parallel for schedule(static) if (m >= kParallelEig)
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < m; ++r) a(j + 1 + r, j + 1 + c) -= v[r] * q[c] + q[r] * v[c];
    hv.push_back(std::move(v));
    hbeta.push_back(beta);
  }
  for (int j = 0; j < k; ++j) d[j] = a(j, j);
  if (k >= 2) e[k - 2] = a(k - 1, k - 2);

  // Z = P_0 P_1 ... (backward accumulation)
  std::vector<double> Z(static_cast<size_t>(k) * k, 0.0);
  auto z = [&](int i, int j) -> double& { return Z[static_cast<size_t>(j) * k + i]; };
  for (int i = 0; i < k; ++i) z(i, i) = 1.0;
  for (int j = static_cast<int>(hv.size()) - 1; j >= 0; --j) {
    if (hbeta[j] == 0.0) continue;
    const std::vector<double>& v = hv[j];
    const int m = k - j - 1;
#pragma omp parallel for schedule(static) if (m >= kParallelEig)
    for (int c = j + 1; c < k; ++c) {
      double s = 0.0;
      for (int r = 0; r < m; ++r) s += v[r] * z(j + 1 + r, c);
      s *= hbeta[j];
      for (int r = 0; r < m; ++r) z(j + 1 + r, c) -= s * v[r];
    }
  }

  // implicit QR on the tridiagonal (d, e), e[i] couples i and i+1. The rotations of each
  // sweep are recorded and applied to the eigenvector matrix Z in batches of sweeps, its
  // rows in blocks of 32 over host threads for large k: every row sees the same rotations in
  // the same order as a row-by-row application, so the result does not depend on the split.
  struct Rot {
    int i;
    double c, s;
  };
  std::vector<Rot> rots;
  auto apply_rots = [&]() {
    if (rots.empty()) return;
#pragma omp parallel for schedule(static) if (k >= kParallelEig)
    for (int r0 = 0; r0 < k; r0 += 32) {
      const int r1 = std::min(k, r0 + 32);
      for (const Rot& q : rots)
        for (int row = r0; row < r1; ++row) {
          const double zi = z(row, q.i), zi1 = z(row, q.i + 1);
          z(row, q.i) = q.c * zi - q.s * zi1;
          z(row, q.i + 1) = q.s * zi + q.c * zi1;
        }
    }
    rots.clear();
  };
  const size_t batch = static_cast<size_t>(std::max(64, 8 * k));  // rotations per application
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = k - 1;
  int iters = 0;
  const int max_iters = 60 * k + 100;
  while (hi > 0) {
    // deflate negligible couplings at the bottom
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++iters > max_iters) return false;
    // Wilkinson shift from the trailing 2x2 block
    const double dd = 0.5 * (d[hi - 1] - d[hi]);
    const double eh = e[hi - 1];
    const double den = dd + std::copysign(std::hypot(dd, eh), dd == 0.0 ? 1.0 : dd);
    const double mu = d[hi] - eh * eh / den;
    double x = d[lo] - mu;
    double zz = e[lo];
    double bulge = 0.0;
    for (int i = lo; i < hi; ++i) {
      const double r = std::hypot(x, zz);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = -zz / r;
      }
      if (i > lo) e[i - 1] = r;
      const double di = d[i], ei = e[i], di1 = d[i + 1];
      d[i] = di * c * c - 2.0 * ei * c * s + di1 * s * s;
      d[i + 1] = di * s * s + 2.0 * ei * c * s + di1 * c * c;
      e[i] = (di - di1) * c * s + ei * (c * c - s * s);
      if (i + 1 < hi) {
        bulge = -s * e[i + 1];
        e[i + 1] = c * e[i + 1];
        x = e[i];
        zz = bulge;
      }
      rots.push_back({i, c, s});
    }
    if (rots.size() >= batch) apply_rots();
  }
  apply_rots();
  // sort ascending
  std::vector<int> order(k);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int i, int j) { return d[i] < d[j]; });
  for (int j = 0; j < k; ++j) {
    w[j] = d[order[j]];
    if (Vout)
      for (int i = 0; i < k; ++i) Vout[static_cast<size_t>(j) * k + i] = z(i, order[j]);
  }
  return true;
}

}  // namespace kes
