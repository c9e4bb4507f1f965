// Host-side FP64 setup of the 1D operators (runs once per handle).
//
// 1D B-spline matrices of section "Variational formulation" (definitions after
// eq. discrete4): M[l][i] = int B_i B_l, S[l][i] = int B_i' B_l',
// A[l][i] = int B_i' B_l, B[l][i] = int B_i B_l' (= A[i][l]); row l is the
// test function.  Open uniform knots on [0, 1], Gauss-Legendre with p + 1
// points per element (exact for the degree-2p integrands).  Banded storage:
// band[k*(2p+1) + d] = X[k][k + d - p].
//
// Banded LU without pivoting (the 1D systems of the alternating-direction
// solver): Doolittle on the band, stored as lower multipliers l[k][q]
// (column k - q), 1/U[k][k] and the normalised upper entries U[k][k+q]/U[k][k].
#include "adi_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace adi {

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_q.
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double z = std::cos(pi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      // p1 = P_q(z), p0 = P_{q-1}(z)
      double dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= q; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (q == 1) { p1 = z; p0 = 1.0; }
    double dp = q * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Values and derivatives of the p+1 B-splines that are nonzero on element e
// at point t (local functions e .. e+p), by the triangular Cox-de Boor table.
void local_basis(const std::vector<double>& U, int p, int e, double t, double* val, double* der) {
  const int span = e + p;
  // ndu[j][r]: degree-j values of functions span-j .. span
  std::vector<std::vector<double>> N(p + 1, std::vector<double>(p + 1, 0.0));
  N[0][0] = 1.0;
  std::vector<double> left(p + 1), right(p + 1);
  for (int j = 1; j <= p; ++j) {
    left[j] = t - U[span + 1 - j];
    right[j] = U[span + j] - t;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double den = right[r + 1] + left[j - r];
      double tmp = N[j - 1][r] / den;
      N[j][r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j][j] = saved;
  }
  for (int r = 0; r <= p; ++r) val[r] = N[p][r];
  // derivative of degree-p functions from degree p-1 values
  for (int r = 0; r <= p; ++r) der[r] = 0.0;
  if (p >= 1) {
    for (int r = 0; r <= p; ++r) {
      int i = span - p + r;  // global index
      // N'_{i,p} = p/(U[i+p]-U[i]) N_{i,p-1} - p/(U[i+p+1]-U[i+1]) N_{i+1,p-1}
      // degree p-1 functions on this span are span-p+1 .. span -> N[p-1][0..p-1]
      double a = 0.0, b = 0.0;
      int ia = i - (span - p + 1);      // index of N_{i,p-1} in N[p-1]
      int ib = i + 1 - (span - p + 1);  // index of N_{i+1,p-1}
      if (ia >= 0 && ia <= p - 1) {
        double d = U[i + p] - U[i];
        if (d > 0) a = p / d * N[p - 1][ia];
      }
      if (ib >= 0 && ib <= p - 1) {
        double d = U[i + p + 1] - U[i + 1];
        if (d > 0) b = p / d * N[p - 1][ib];
      }
      der[r] = a - b;
    }
  }
}

std::vector<double> knots(int n, int p, const std::vector<double>& breaks = {}) {
  std::vector<double> U;
  for (int i = 0; i < p; ++i) U.push_back(0.0);
  for (int i = 0; i <= n; ++i) U.push_back(breaks.empty() ? double(i) / n : breaks[i]);
  for (int i = 0; i < p; ++i) U.push_back(1.0);
  return U;
}

// Gauss point q (reference node gx, weight gw) of element e: position and weight
inline void elem_point(const Axis1D& ax, int e, double gx, double gw, double& t, double& w) {
  if (ax.breaks.empty()) {
    const double h = 1.0 / ax.n;
    t = (e + 0.5) * h + 0.5 * h * gx;
    w = 0.5 * h * gw;
  } else {
    const double a = ax.breaks[e], b = ax.breaks[e + 1];
    t = 0.5 * (a + b) + 0.5 * (b - a) * gx;
    w = 0.5 * (b - a) * gw;
  }
}

}  // namespace

void find_interior(Axis1D& ax);

void build_axis(int n, int p, Axis1D& ax, const double* breaks) {
  const int N = n + p, W = 2 * p + 1;
  ax.n = n;
  ax.p = p;
  ax.N = N;
  ax.breaks.clear();
  if (breaks) ax.breaks.assign(breaks, breaks + n + 1);
  ax.M.assign(size_t(N) * W, 0.0);
  ax.S.assign(size_t(N) * W, 0.0);
  ax.A.assign(size_t(N) * W, 0.0);
  ax.B.assign(size_t(N) * W, 0.0);
  ax.G.assign(size_t(N) * (p + 1), 0.0);
  std::vector<double> U = knots(n, p, ax.breaks), gx, gw;
  gauss_legendre(p + 1, gx, gw);
  std::vector<double> v(p + 1), d(p + 1);
  for (int e = 0; e < n; ++e) {
    for (int q = 0; q <= p; ++q) {
      double t, w;
      elem_point(ax, e, gx[q], gw[q], t, w);
      local_basis(U, p, e, t, v.data(), d.data());
      for (int a = 0; a <= p; ++a) {
        int l = e + a;  // test
        ax.G[size_t(l) * (p + 1) + (p - a)] += w * v[a];  // element e = l - (p - a)
        for (int b = 0; b <= p; ++b) {
          int i = e + b;  // trial
          int dd = i - l + p;
          ax.M[size_t(l) * W + dd] += w * v[b] * v[a];
          ax.S[size_t(l) * W + dd] += w * d[b] * d[a];
          ax.A[size_t(l) * W + dd] += w * d[b] * v[a];
          ax.B[size_t(l) * W + dd] += w * v[b] * d[a];
        }
      }
    }
  }
  find_interior(ax);
}

// Interior rows of an axis: the range around the middle row, inside
// 2p .. N-1-2p (where no band reaches a boundary row), whose band rows of M, S,
// A, B equal the middle row's to rounding; kernels use the constant stencil
// there and the tables elsewhere.  Uniform elements: all of 2p .. N-1-2p.
void find_interior(Axis1D& ax) {
  const int p = ax.p, N = ax.N, W = 2 * p + 1;
  ax.inner_lo = 1;
  ax.inner_hi = 0;
  const int lo = 2 * p, hi = N - 1 - 2 * p;
  if (lo > hi) return;
  const int mid = (lo + hi) / 2;
  const std::vector<double>* src[4] = {&ax.M, &ax.S, &ax.A, &ax.B};
  double scale = 0.0;
  for (int o = 0; o < 4; ++o)
    for (int q = 0; q < W; ++q) scale = std::fmax(scale, std::fabs((*src[o])[(size_t)mid * W + q]));
  auto same = [&](int r) {
    for (int o = 0; o < 4; ++o)
      for (int q = 0; q < W; ++q)
        if (std::fabs((*src[o])[(size_t)r * W + q] - (*src[o])[(size_t)mid * W + q]) > 1e-12 * scale) return false;
    return true;
  };
  int a = mid, b = mid;
  while (a - 1 >= lo && same(a - 1)) --a;
  while (b + 1 <= hi && same(b + 1)) ++b;
  ax.inner_lo = a;
  ax.inner_hi = b;
}

// The same integrals restricted to one element: loc[((e * 4 + op) * (p+1) + a) *
// (p+1) + b] = int over element e of the op's integrand for test function e + a
// and trial function e + b, op = M, S, A, B (as the bands; the bands are the
// sums of these blocks over the elements).  Used by the right-hand side with
// per-element material inside the integrals.
void element_matrices(const Axis1D& ax, std::vector<double>& loc) {
  const int n = ax.n, p = ax.p, Q = p + 1;
  loc.assign(size_t(n) * 4 * Q * Q, 0.0);
  std::vector<double> U = knots(n, p, ax.breaks), gx, gw;
  gauss_legendre(p + 1, gx, gw);
  std::vector<double> v(p + 1), d(p + 1);
  for (int e = 0; e < n; ++e) {
    double* blk = loc.data() + size_t(e) * 4 * Q * Q;
    for (int q = 0; q <= p; ++q) {
      double t, w;
      elem_point(ax, e, gx[q], gw[q], t, w);
      local_basis(U, p, e, t, v.data(), d.data());
      for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p; ++b) {
          blk[0 * Q * Q + a * Q + b] += w * v[b] * v[a];
          blk[1 * Q * Q + a * Q + b] += w * d[b] * d[a];
          blk[2 * Q * Q + a * Q + b] += w * d[b] * v[a];
          blk[3 * Q * Q + a * Q + b] += w * v[b] * d[a];
        }
    }
  }
}

// Doolittle LU without pivoting of the banded matrix base + diag(c) stiff on
// rows lo..hi (columns outside are dropped).  c may be null (c = 0).
void band_lu(const std::vector<double>& base, const std::vector<double>* stiff, int N, int p,
             int lo, int hi, BandLU& out) {
  const int W = 2 * p + 1;
  out.N = N;
  out.p = p;
  out.lo = lo;
  out.hi = hi;
  out.L.assign(size_t(N) * p, 0.0);
  out.inv_d.assign(N, 0.0);
  out.U.assign(size_t(N) * p, 0.0);
  // full upper rows U[k][k..k+p] for the recurrence
  std::vector<double> Ufull(size_t(N) * (p + 1), 0.0);
  auto A = [&](int k, int j) -> double {
    if (j < lo || j > hi) return 0.0;
    int dd = j - k + p;
    if (dd < 0 || dd >= W) return 0.0;
    double v = base[size_t(k) * W + dd];
    if (stiff) v += (*stiff)[size_t(k) * W + dd];
    return v;
  };
  auto Uat = [&](int m, int j) -> double {  // U[m][j], j in m..m+p
    if (m < lo) return 0.0;
    int q = j - m;
    if (q < 0 || q > p) return 0.0;
    return Ufull[size_t(m) * (p + 1) + q];
  };
  for (int k = lo; k <= hi; ++k) {
    std::vector<double> l(p + 1, 0.0);  // l[q] multiplies row k - q
    for (int j = std::max(lo, k - p); j < k; ++j) {
      double s = A(k, j);
      for (int m = std::max(lo, k - p); m < j; ++m) s -= l[k - m] * Uat(m, j);
      l[k - j] = s / Uat(j, j);
    }
    for (int j = k; j <= std::min(hi, k + p); ++j) {
      double s = A(k, j);
      for (int m = std::max(lo, std::max(k - p, j - p)); m < k; ++m) s -= l[k - m] * Uat(m, j);
      Ufull[size_t(k) * (p + 1) + (j - k)] = s;
    }
    double dkk = Ufull[size_t(k) * (p + 1)];
    out.inv_d[k] = 1.0 / dkk;
    for (int q = 1; q <= p; ++q) {
      out.L[size_t(k) * p + (q - 1)] = l[q];
      out.U[size_t(k) * p + (q - 1)] = Ufull[size_t(k) * (p + 1) + q] / dkk;
    }
  }
}

// Largest eigenvalue of M^{-1} S on the Dirichlet-reduced axis: Cholesky
// M = L L^T, C = L^{-1} S L^{-T} (dense, symmetric), cyclic Jacobi rotations.
double lambda_max(const Axis1D& ax) {
  const int p = ax.p, W = 2 * p + 1;
  const int n = ax.N - 2;
  if (n <= 0) return 0.0;
  std::vector<double> Md(size_t(n) * n, 0.0), Sd(size_t(n) * n, 0.0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      int k = r + 1, j = c + 1, dd = j - k + p;
      if (dd >= 0 && dd < W) {
        Md[size_t(r) * n + c] = ax.M[size_t(k) * W + dd];
        Sd[size_t(r) * n + c] = ax.S[size_t(k) * W + dd];
      }
    }
  // Cholesky of Md (lower)
  std::vector<double> L(size_t(n) * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = Md[size_t(j) * n + j];
    for (int k = 0; k < j; ++k) s -= L[size_t(j) * n + k] * L[size_t(j) * n + k];
    L[size_t(j) * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = Md[size_t(i) * n + j];
      for (int k = 0; k < j; ++k) t -= L[size_t(i) * n + k] * L[size_t(j) * n + k];
      L[size_t(i) * n + j] = t / L[size_t(j) * n + j];
    }
  }
  // X = L^{-1} S (forward substitution on columns), C = X L^{-T} = (L^{-1} X^T)^T
  std::vector<double> X(size_t(n) * n), C(size_t(n) * n);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = Sd[size_t(i) * n + c];
      for (int k = 0; k < i; ++k) s -= L[size_t(i) * n + k] * X[size_t(k) * n + c];
      X[size_t(i) * n + c] = s / L[size_t(i) * n + i];
    }
  for (int r = 0; r < n; ++r)  // row r of C = L^{-1} applied to row r of X (as a column)
    for (int i = 0; i < n; ++i) {
      double s = X[size_t(r) * n + i];
      for (int k = 0; k < i; ++k) s -= L[size_t(i) * n + k] * C[size_t(r) * n + k];
      C[size_t(r) * n + i] = s / L[size_t(i) * n + i];
    }
  for (int r = 0; r < n; ++r)  // symmetrise rounding
    for (int c = r + 1; c < n; ++c) {
      double m = 0.5 * (C[size_t(r) * n + c] + C[size_t(c) * n + r]);
      C[size_t(r) * n + c] = C[size_t(c) * n + r] = m;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double v = C[size_t(r) * n + c];
        if (r == c) diag += v * v; else off += v * v;
      }
    if (off <= 1e-28 * diag) break;
    for (int pi = 0; pi < n - 1; ++pi)
      for (int qi = pi + 1; qi < n; ++qi) {
        double apq = C[size_t(pi) * n + qi];
        if (std::fabs(apq) < 1e-300) continue;
        double app = C[size_t(pi) * n + pi], aqq = C[size_t(qi) * n + qi];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          double akp = C[size_t(k) * n + pi], akq = C[size_t(k) * n + qi];
          C[size_t(k) * n + pi] = cs * akp - sn * akq;
          C[size_t(k) * n + qi] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = C[size_t(pi) * n + k], aqk = C[size_t(qi) * n + k];
          C[size_t(pi) * n + k] = cs * apk - sn * aqk;
          C[size_t(qi) * n + k] = sn * apk + cs * aqk;
        }
      }
  }
  double mx = 0.0;
  for (int r = 0; r < n; ++r) mx = std::max(mx, C[size_t(r) * n + r]);
  return mx;
}

// Values of the p+1 B-splines nonzero at x0, and the index of the first one.
int point_basis(int n, int p, double x0, double* vals) {
  std::vector<double> U = knots(n, p), d(p + 1);
  int e = int(std::floor(x0 * n));
  if (e >= n) e = n - 1;
  if (e < 0) e = 0;
  local_basis(U, p, e, x0, vals, d.data());
  return e;
}

int point_basis(const Axis1D& ax, double x0, double* vals) {
  if (ax.breaks.empty()) return point_basis(ax.n, ax.p, x0, vals);
  std::vector<double> U = knots(ax.n, ax.p, ax.breaks), d(ax.p + 1);
  int e = int(std::upper_bound(ax.breaks.begin(), ax.breaks.end(), x0) - ax.breaks.begin()) - 1;
  if (e >= ax.n) e = ax.n - 1;
  if (e < 0) e = 0;
  local_basis(U, ax.p, e, x0, vals, d.data());
  return e;
}

}  // namespace adi
