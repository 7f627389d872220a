// Angle sets for the C ABI (sec. 3 of arXiv:1403.6126): level-symmetric
// LQ_N sets built from the Carlson (1963) construction, the 24-angle set the
// paper uses in sec. 5.2, and Gauss-Legendre slab sets.  Host code.
#include <cmath>
#include <cstring>
#include <vector>

#include "rt.h"

namespace {

struct Octant {
  std::vector<double> mu[3];  // direction cosines of the points
  std::vector<int> cls;       // weight class of each point
  int ncls = 0;
};

// Points (mu_i, mu_j, mu_k), i + j + k = N/2 + 2, with
// mu_i^2 = mu_1^2 + (i - 1) * 2 (1 - 3 mu_1^2) / (N - 2).  Points that are
// permutations of one another share a class.
Octant octant(int N, double mu1) {
  Octant o;
  int L = N / 2;
  std::vector<double> lev(L);
  if (N == 2) {
    lev[0] = 1.0 / std::sqrt(3.0);
  } else {
    double delta = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2);
    for (int i = 0; i < L; ++i) lev[i] = std::sqrt(mu1 * mu1 + delta * i);
  }
  std::vector<int> keys;
  for (int i = 1; i <= L; ++i)
    for (int j = 1; j <= L; ++j) {
      int k = L + 2 - i - j;
      if (k < 1 || k > L) continue;
      int a = i, b = j, c = k, t;
      if (a > b) { t = a; a = b; b = t; }
      if (b > c) { t = b; b = c; c = t; }
      if (a > b) { t = a; a = b; b = t; }
      int key = a * 10000 + b * 100 + c;
      int id = -1;
      for (size_t q = 0; q < keys.size(); ++q)
        if (keys[q] == key) id = (int)q;
      if (id < 0) { id = (int)keys.size(); keys.push_back(key); }
      o.mu[0].push_back(lev[i - 1]);
      o.mu[1].push_back(lev[j - 1]);
      o.mu[2].push_back(lev[k - 1]);
      o.cls.push_back(id);
    }
  o.ncls = (int)keys.size();
  return o;
}

// Solves A x = b (n <= 8) by elimination with partial pivoting.
bool solve_small(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
    b[k] = s / A[k * n + k];
  }
  return true;
}

// Class weights from sum = 1/8 per octant and <mu_x^2k> = 1/(2k+1) for
// k = 2..ncls; returns the residual of the k = ncls + 1 condition.
double class_weights(const Octant &o, double *w) {
  int n = o.ncls;
  double A[64], b[8];
  for (int r = 0; r <= n; ++r) {
    double row[8] = {0};
    for (size_t p = 0; p < o.cls.size(); ++p) row[o.cls[p]] += r == 0 ? 1.0 : std::pow(o.mu[0][p], 2.0 * (r + 1));
    double rhs = r == 0 ? 0.125 : 0.125 / (2.0 * (r + 1) + 1.0);
    if (r < n) {
      for (int c = 0; c < n; ++c) A[r * n + c] = row[c];
      b[r] = rhs;
    } else {
      if (!solve_small(n, A, b)) return NAN;
      double res = -rhs;
      for (int c = 0; c < n; ++c) {
        w[c] = b[c];
        res += row[c] * b[c];
      }
      return res;
    }
  }
  return NAN;
}

bool lq_mu1(int N, double *mu1) {
  const int G = 400;
  double lo = 0.02, hi = 1.0 / std::sqrt(3.0) - 1e-6;
  double w[8];
  int found = 0;
  double root = 0;
  double xa = lo, fa = class_weights(octant(N, xa), w);
  for (int i = 1; i <= G; ++i) {
    double xb = lo + (hi - lo) * i / G;
    double fb = class_weights(octant(N, xb), w);
    if (fa * fb < 0) {
      double a = xa, b = xb, f_a = fa;
      for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (a + b);
        double fm = class_weights(octant(N, m), w);
        if (fm == 0 || (b - a) < 1e-17) { a = b = m; break; }
        if ((fm < 0) == (f_a < 0)) { a = m; f_a = fm; } else { b = m; }
      }
      double x = 0.5 * (a + b);
      class_weights(octant(N, x), w);
      bool pos = true;
      Octant o = octant(N, x);
      for (int c = 0; c < o.ncls; ++c) pos = pos && w[c] > 0;
      if (pos) { ++found; root = x; }
    }
    xa = xb;
    fa = fb;
  }
  *mu1 = root;
  return found == 1;
}

int emit_sphere(const Octant &o, const double *wc, int cap, double *n, double *w) {
  int per = (int)o.cls.size(), M = 8 * per;
  if (cap < M) return -1;
  int idx = 0;
  for (int s = 0; s < 8; ++s) {
    double sx = (s & 4) ? -1.0 : 1.0, sy = (s & 2) ? -1.0 : 1.0, sz = (s & 1) ? -1.0 : 1.0;
    for (int p = 0; p < per; ++p, ++idx) {
      n[3 * idx] = sx * o.mu[0][p];
      n[3 * idx + 1] = sy * o.mu[1][p];
      n[3 * idx + 2] = sz * o.mu[2][p];
      w[idx] = wc[o.cls[p]];
    }
  }
  return M;
}

// Legendre P_M and its derivative at x by the three-term recurrence.
void legendre(int M, double x, double *p, double *dp) {
  double p0 = 1.0, p1 = x;
  if (M == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= M; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = M * (x * p1 - p0) / (x * x - 1.0);
}

}  // namespace

extern "C" rt_status rt_angle_set(int kind, int order, int cap, int *m_out, double *n_out, double *w_out) {
  if (!m_out || !n_out || !w_out) return RT_E_INVALID;
  if (kind == RT_ANGLES_GAUSS_LEGENDRE) {
    int M = order;
    if (M < 1 || M > 64 || cap < M) return RT_E_INVALID;
    for (int i = 0; i < M; ++i) {
      // Newton on P_M from the Tricomi estimate of the i-th root
      double x = std::cos(M_PI * (i + 0.75) / (M + 0.5));
      double p, dp;
      for (int it = 0; it < 100; ++it) {
        legendre(M, x, &p, &dp);
        double dx = p / dp;
        x -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
      legendre(M, x, &p, &dp);
      double wgl = 2.0 / ((1.0 - x * x) * dp * dp);
      int j = M - 1 - i;  // ascending mu
      n_out[3 * j] = x;
      n_out[3 * j + 1] = std::sqrt(1.0 - x * x);
      n_out[3 * j + 2] = 0.0;
      w_out[j] = 0.5 * wgl;
    }
    *m_out = M;
    return RT_OK;
  }
  if (kind == RT_ANGLES_LEVEL_SYMMETRIC || kind == RT_ANGLES_PAPER_S4) {
    int N = kind == RT_ANGLES_PAPER_S4 ? 4 : order;
    if (N != 2 && N != 4 && N != 6 && N != 8) return RT_E_INVALID;
    double mu1 = 0, wc[8];
    if (N == 2) {
      wc[0] = 0.125;
    } else if (kind == RT_ANGLES_PAPER_S4) {
      mu1 = 1.0 / 3.0;
      class_weights(octant(N, mu1), wc);
    } else {
      if (!lq_mu1(N, &mu1)) return RT_E_INVALID;
      class_weights(octant(N, mu1), wc);
    }
    int M = emit_sphere(octant(N, mu1), wc, cap, n_out, w_out);
    if (M < 0) return RT_E_INVALID;
    *m_out = M;
    return RT_OK;
  }
  return RT_E_INVALID;
}
