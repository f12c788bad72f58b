// Host-side setup of the Stokes multigrid library: basis, LDG assembly on the
// finest Cartesian mesh (Appendix A of arXiv:1911.05888), operator coarsening
// (Appendix B, Algorithms 2 and 3), the Stokes blocks of eq. (blockform) /
// (timedep2) in element-offset form, block inverses and the bottom-level
// pseudo-inverse.  Setup runs once per problem; the V-cycle itself runs in
// the CUDA kernels of kernels.cu.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>
#include <thread>

#include "stk_internal.h"
#include "../../include/stokes_mg.h"

namespace stk {

// ---------------------------------------------------------------------------
// Threads
// ---------------------------------------------------------------------------
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
  int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 32u);
  if (n < 64 || nt == 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t a = t * chunk, b = std::min<int64_t>(n, a + chunk);
    if (a >= b) break;
    th.emplace_back(fn, a, b);
  }
  for (auto& t : th) t.join();
}

// ---------------------------------------------------------------------------
// One-dimensional basis: psi_l = sqrt(2l+1) P_l on [-1, 1]
// ---------------------------------------------------------------------------
static void legendre(int p, double x, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (p >= 1) {
    P[1] = x;
    dP[1] = 1.0;
  }
  for (int l = 1; l < p; ++l) {
    P[l + 1] = ((2 * l + 1) * x * P[l] - l * P[l - 1]) / (l + 1);
    dP[l + 1] = dP[l - 1] + (2 * l + 1) * P[l];
  }
}

void psi_eval(int p, double x, double* v, double* dv) {
  double P[32], dP[32];
  legendre(p, x, P, dP);
  for (int l = 0; l <= p; ++l) {
    double c = std::sqrt(2.0 * l + 1.0);
    v[l] = c * P[l];
    if (dv) dv[l] = c * dP[l];
  }
}

void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P[40], dP[40];
      legendre(q, z, P, dP);
      double dz = P[q] / dP[q];
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P[40], dP[40];
    legendre(q, z, P, dP);
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dP[q] * dP[q]);
  }
}

struct Basis1 {
  int p;
  std::vector<double> K;            // K[m][l] = int psi_m psi_l'
  std::vector<double> tr[2];        // tr[0] = psi(-1), tr[1] = psi(+1)
  std::vector<double> child[2];     // child[c][m][l]
};

static Basis1 basis1(int p) {
  Basis1 B;
  B.p = p;
  int m = p + 1;
  std::vector<double> x, w;
  gauss_rule(p + 1, x, w);
  B.K.assign(m * m, 0.0);
  B.child[0].assign(m * m, 0.0);
  B.child[1].assign(m * m, 0.0);
  for (int qi = 0; qi < m; ++qi) {
    double v[32], dv[32];
    psi_eval(p, x[qi], v, dv);
    for (int a = 0; a < m; ++a)
      for (int l = 0; l < m; ++l) B.K[a * m + l] += w[qi] * v[a] * dv[l];
    for (int c = 0; c < 2; ++c) {
      double vc[32];
      psi_eval(p, 0.5 * (x[qi] + 2 * c - 1), vc, nullptr);
      for (int a = 0; a < m; ++a)
        for (int l = 0; l < m; ++l) B.child[c][a * m + l] += 0.5 * w[qi] * v[a] * vc[l];
    }
  }
  for (int sd = 0; sd < 2; ++sd) {
    B.tr[sd].resize(m);
    psi_eval(p, sd == 0 ? -1.0 : 1.0, B.tr[sd].data(), nullptr);
  }
  return B;
}

// Mode index a = sum_k a_k (p+1)^k (x fastest).
static inline int mode_digit(int a, int k, int m) {
  for (int j = 0; j < k; ++j) a /= m;
  return a % m;
}

// s x s matrix acting with T1 ((p+1) x (p+1)) on axis k, identity elsewhere.
static std::vector<double> kron_axis(int d, int p, int k, const double* T1) {
  int m = p + 1, s = 1;
  for (int j = 0; j < d; ++j) s *= m;
  std::vector<double> out(s * s, 0.0);
  for (int b = 0; b < s; ++b)
    for (int a = 0; a < s; ++a) {
      bool same = true;
      for (int j = 0; j < d; ++j)
        if (j != k && mode_digit(a, j, m) != mode_digit(b, j, m)) same = false;
      if (same) out[b * s + a] = T1[mode_digit(b, k, m) * m + mode_digit(a, k, m)];
    }
  return out;
}

// s x s tensor product prod_k T1[k][b_k][a_k].
static std::vector<double> kron_all(int d, int p, const double* const* T1) {
  int m = p + 1, s = 1;
  for (int j = 0; j < d; ++j) s *= m;
  std::vector<double> out(s * s, 1.0);
  for (int b = 0; b < s; ++b)
    for (int a = 0; a < s; ++a) {
      double v = 1.0;
      for (int k = 0; k < d; ++k) v *= T1[k][mode_digit(b, k, m) * m + mode_digit(a, k, m)];
      out[b * s + a] = v;
    }
  return out;
}

void child_matrices(int d, int p, std::vector<double>& out) {
  Basis1 B = basis1(p);
  int m = p + 1, s = 1;
  for (int j = 0; j < d; ++j) s *= m;
  out.assign((size_t)(1 << d) * s * s, 0.0);
  for (int c = 0; c < (1 << d); ++c) {
    const double* T[3];
    for (int k = 0; k < d; ++k) T[k] = B.child[(c >> k) & 1].data();
    auto P = kron_all(d, p, T);
    std::copy(P.begin(), P.end(), out.begin() + (size_t)c * s * s);
  }
}

// ---------------------------------------------------------------------------
// Small dense helpers (row-major)
// ---------------------------------------------------------------------------
// C += alpha * op(A) * B, A is (op: 'N' s x s, 'T' transposed), all s x s.
static void gemm_acc(int s, double alpha, const double* A, bool At, const double* B, double* C) {
  for (int i = 0; i < s; ++i)
    for (int k = 0; k < s; ++k) {
      double a = At ? A[k * s + i] : A[i * s + k];
      if (a == 0.0) continue;
      a *= alpha;
      const double* b = B + k * s;
      double* c = C + i * s;
      for (int j = 0; j < s; ++j) c[j] += a * b[j];
    }
}

// C += alpha * A^T * X * B  (the Galerkin triple product of coarsening).
static void triple_acc(int s, double alpha, const double* A, const double* X, const double* B,
                       double* C, std::vector<double>& tmp) {
  tmp.assign(s * s, 0.0);
  gemm_acc(s, 1.0, X, false, B, tmp.data());
  gemm_acc(s, alpha, A, true, tmp.data(), C);
}

static bool invert_dense(int n, const double* A, double* Ainv) {
  std::vector<double> a(A, A + (size_t)n * n);
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = std::fabs(a[(size_t)col * n + col]);
    for (int r = col + 1; r < n; ++r) {
      double v = std::fabs(a[(size_t)r * n + col]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (piv != col) {
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)piv * n + j], a[(size_t)col * n + j]);
        std::swap(inv[(size_t)piv * n + j], inv[(size_t)col * n + j]);
      }
    }
    double di = 1.0 / a[(size_t)col * n + col];
    for (int j = 0; j < n; ++j) {
      a[(size_t)col * n + j] *= di;
      inv[(size_t)col * n + j] *= di;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)r * n + j] -= f * a[(size_t)col * n + j];
        inv[(size_t)r * n + j] -= f * inv[(size_t)col * n + j];
      }
    }
  }
  std::copy(inv.begin(), inv.end(), Ainv);
  return true;
}

int invert_blocks(int n, int count, const double* A, double* Ainv, std::string& err) {
  std::atomic<int64_t> bad(-1);
  parallel_for(count, [&](int64_t a, int64_t b) {
    for (int64_t e = a; e < b; ++e)
      if (!invert_dense(n, A + (size_t)e * n * n, Ainv + (size_t)e * n * n)) bad = e;
  });
  if (bad >= 0) {
    err = "element block " + std::to_string((long long)bad.load()) + " is singular";
    return STK_ERR_SINGULAR_BLOCK;
  }
  return STK_OK;
}

// Cyclic Jacobi eigenvalue method for a symmetric matrix, then the
// least-squares inverse with |lambda| <= theta max|lambda| snapped to zero.
int pseudo_inverse_jacobi(int n, std::vector<double>& A, std::vector<double>& pinv, int& snapped,
                          double theta) {
  std::vector<double> V((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int pp = 0; pp < n - 1; ++pp)
      for (int qq = pp + 1; qq < n; ++qq) {
        double apq = A[(size_t)pp * n + qq];
        if (std::fabs(apq) < 1e-300) continue;
        double app = A[(size_t)pp * n + pp], aqq = A[(size_t)qq * n + qq];
        double th = (aqq - app) / (2.0 * apq);
        double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          double akp = A[(size_t)k * n + pp], akq = A[(size_t)k * n + qq];
          A[(size_t)k * n + pp] = cs * akp - sn * akq;
          A[(size_t)k * n + qq] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[(size_t)pp * n + k], aqk = A[(size_t)qq * n + k];
          A[(size_t)pp * n + k] = cs * apk - sn * aqk;
          A[(size_t)qq * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + pp], vkq = V[(size_t)k * n + qq];
          V[(size_t)k * n + pp] = cs * vkp - sn * vkq;
          V[(size_t)k * n + qq] = sn * vkp + cs * vkq;
        }
      }
  }
  double lmax = 0.0;
  for (int i = 0; i < n; ++i) lmax = std::max(lmax, std::fabs(A[(size_t)i * n + i]));
  std::vector<double> inv(n, 0.0);
  snapped = 0;
  for (int i = 0; i < n; ++i) {
    double l = A[(size_t)i * n + i];
    if (std::fabs(l) <= theta * lmax) {
      ++snapped;
    } else {
      inv[i] = 1.0 / l;
    }
  }
  pinv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double f = V[(size_t)i * n + k] * inv[k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) pinv[(size_t)i * n + j] += f * V[(size_t)j * n + k];
    }
  return STK_OK;
}

// Symmetric eigendecomposition by Householder reduction to tridiagonal form
// and the implicit symmetric QR iteration with Wilkinson shifts (the textbook
// method, e.g. Golub and Van Loan, Matrix Computations, Sections 8.3.1-8.3.3).
// A (row-major, symmetric, destroyed) = sum_k lam[k] q_k q_k^T with q_k the
// rows of Qt.  O(n^3) once, against cyclic Jacobi's O(n^3) per sweep.
// Returns false if the QR iteration does not converge in 30 n steps.
static bool symmetric_eigen(int n, std::vector<double>& A, std::vector<double>& lam, std::vector<double>& Qt) {
  std::vector<double> d(n, 0.0), e(std::max(n - 1, 1), 0.0), beta(std::max(n, 1), 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
    }
  // 1. Householder: H_k = I - beta_k v v^T maps A[k+1:, k] to e[k] e_1; the
  //    reflector v is kept in row k of A (right of the diagonal).
  std::vector<double> pv(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    double* v = &A[(size_t)k * n + k + 1];
    const int m = n - k - 1;
    double alpha = 0.0;
    for (int i = 0; i < m; ++i) alpha += v[i] * v[i];
    alpha = std::sqrt(alpha);
    d[k] = A[(size_t)k * n + k];
    if (alpha == 0.0) {
      e[k] = 0.0;
      beta[k] = 0.0;
      continue;
    }
    const double sg = v[0] >= 0 ? 1.0 : -1.0;
    e[k] = -sg * alpha;
    v[0] += sg * alpha;
    double vv = 0.0;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    const double b = 2.0 / vv;
    beta[k] = b;
    // trailing block B = A[k+1:, k+1:]: p = b B v, w = p - (b/2)(p.v) v,
    // B <- B - v w^T - w v^T
    double pvdot = 0.0;
    for (int i = 0; i < m; ++i) {
      const double* Bi = &A[(size_t)(k + 1 + i) * n + k + 1];
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc += Bi[j] * v[j];
      pv[i] = b * acc;
      pvdot += pv[i] * v[i];
    }
    const double K = 0.5 * b * pvdot;
    for (int i = 0; i < m; ++i) w[i] = pv[i] - K * v[i];
    for (int i = 0; i < m; ++i) {
      double* Bi = &A[(size_t)(k + 1 + i) * n + k + 1];
      const double vi = v[i], wi = w[i];
      for (int j = 0; j < m; ++j) Bi[j] -= vi * w[j] + wi * v[j];
    }
  }
  if (n >= 2) {
    d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
    e[n - 2] = A[(size_t)(n - 2) * n + n - 1];
  }
  d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
  // Qt = Q^T = H_{n-3} ... H_1 H_0 (rows k+1.. of Qt touched by H_k)
  Qt.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Qt[(size_t)i * n + i] = 1.0;
  std::vector<double> u(n);
  for (int k = 0; k + 2 < n; ++k) {
    if (beta[k] == 0.0) continue;
    const double* v = &A[(size_t)k * n + k + 1];
    const int m = n - k - 1;
    std::fill(u.begin(), u.end(), 0.0);
    for (int i = 0; i < m; ++i) {
      const double* row = &Qt[(size_t)(k + 1 + i) * n];
      for (int j = 0; j < n; ++j) u[j] += v[i] * row[j];
    }
    for (int i = 0; i < m; ++i) {
      double* row = &Qt[(size_t)(k + 1 + i) * n];
      const double f = beta[k] * v[i];
      for (int j = 0; j < n; ++j) row[j] -= f * u[j];
    }
  }
  // 2. Implicit symmetric QR on (d, e): each step chases the bulge of one
  //    Wilkinson-shifted rotation down the unreduced block [l, m]; the
  //    rotations R act as T <- R T R^T and Qt <- R Qt on rows k, k+1.
  //    An off-diagonal entry counts as zero below eps times its two diagonal
  //    neighbours or eps times the largest row sum of T (a backward error of
  //    the size every stable eigensolver makes).
  const double eps = 0.5 * std::numeric_limits<double>::epsilon();
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    tnorm = std::max(tnorm, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0));
  auto negligible = [&](int i) {
    const double a = std::fabs(e[i]);
    return a <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1])) || a <= eps * tnorm;
  };
  int m = n - 1, steps = 0;
  while (m > 0) {
    if (negligible(m - 1)) {
      e[m - 1] = 0.0;
      --m;
      continue;
    }
    int l = m - 1;
    while (l > 0 && !negligible(l - 1)) --l;
    if (++steps > 30 * n) return false;
    const double delta = 0.5 * (d[m - 1] - d[m]), bm = e[m - 1];
    const double mu = d[m] - bm * bm / (delta + std::copysign(std::hypot(delta, bm), delta));
    double x = d[l] - mu, z = e[l];
    for (int k = l; k < m; ++k) {
      const double r = std::hypot(x, z);
      const double c = r == 0.0 ? 1.0 : x / r, sn = r == 0.0 ? 0.0 : z / r;
      if (k > l) e[k - 1] = r;
      const double a = d[k], b = e[k], cc = d[k + 1];
      d[k] = c * c * a + 2.0 * c * sn * b + sn * sn * cc;
      d[k + 1] = sn * sn * a - 2.0 * c * sn * b + c * c * cc;
      e[k] = c * sn * (cc - a) + (c * c - sn * sn) * b;
      if (k + 1 < m) {
        z = sn * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      double* q0 = &Qt[(size_t)k * n];
      double* q1 = &Qt[(size_t)(k + 1) * n];
      for (int j = 0; j < n; ++j) {
        const double t0 = q0[j], t1 = q1[j];
        q0[j] = c * t0 + sn * t1;
        q1[j] = -sn * t0 + c * t1;
      }
    }
  }
  lam = d;
  return true;
}

// Least-squares (Moore-Penrose) inverse of a symmetric matrix, the bottom
// solver of Section 3's footnote.  The matrix is first equilibrated,
// A^ = S A S with S_i = (sum_j |A_ij|)^(-1/2): the eigenvalues of A^ with
// |lambda| <= theta max|lambda| are snapped to zero (a congruence keeps the
// number of zero eigenvalues, so an exact kernel is snapped alike), and
// G = S A^+ S solves A x = b for every b in the range of A.  With K the
// kernel of A (S times the snapped eigenvectors, orthonormalised) and
// P = I - K K^T, the least-squares inverse is P G P.  The equilibration keeps
// the blocks' graded scales (velocity against pressure rows, phases of
// different viscosity) out of the eigensolver's rounding error.
void equilibrate_sym(int n, const std::vector<double>& A, std::vector<double>& S, std::vector<double>& Ah) {
  S.assign(n, 1.0);
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    for (int j = 0; j < n; ++j) r += std::fabs(A[(size_t)i * n + j]);
    if (r > 0 && std::isfinite(r)) S[i] = 1.0 / std::sqrt(r);
  }
  Ah.resize((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ah[(size_t)i * n + j] = S[i] * A[(size_t)i * n + j] * S[j];
}

void project_off_kernel(int n, std::vector<double>& pinv, std::vector<double>& K, int nk) {
  if (nk == 0) return;
  // orthonormalise the rows of K by Gram-Schmidt done twice
  for (int a = 0; a < nk; ++a) {
    double* ka = &K[(size_t)a * n];
    for (int pass = 0; pass < 2; ++pass)
      for (int bb = 0; bb < a; ++bb) {
        const double* kb = &K[(size_t)bb * n];
        double dot = 0.0;
        for (int j = 0; j < n; ++j) dot += kb[j] * ka[j];
        for (int j = 0; j < n; ++j) ka[j] -= dot * kb[j];
      }
    double nrm = 0.0;
    for (int j = 0; j < n; ++j) nrm += ka[j] * ka[j];
    nrm = std::sqrt(nrm);
    for (int j = 0; j < n; ++j) ka[j] = nrm > 0 ? ka[j] / nrm : 0.0;
  }
  // pinv <- P G P with P = I - K^T K (K's rows orthonormal); G symmetric
  std::vector<double> GK((size_t)n * nk, 0.0), KGK((size_t)nk * nk, 0.0);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < nk; ++a) {
      double acc = 0.0;
      const double* ka = &K[(size_t)a * n];
      const double* gi = &pinv[(size_t)i * n];
      for (int j = 0; j < n; ++j) acc += gi[j] * ka[j];
      GK[(size_t)i * nk + a] = acc;
    }
  for (int a = 0; a < nk; ++a)
    for (int bb = 0; bb < nk; ++bb) {
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc += K[(size_t)a * n + i] * GK[(size_t)i * nk + bb];
      KGK[(size_t)a * nk + bb] = acc;
    }
  // P G P = G - GK K - K^T GK^T + K^T (K G K^T) K
  parallel_for(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      double* row = &pinv[(size_t)i * n];
      for (int a = 0; a < nk; ++a) {
        const double* ka = &K[(size_t)a * n];
        double ci = -GK[(size_t)i * nk + a];
        for (int bb = 0; bb < nk; ++bb) ci += K[(size_t)bb * n + i] * KGK[(size_t)bb * nk + a];
        const double kia = K[(size_t)a * n + i];
        for (int j = 0; j < n; ++j) row[j] += ci * ka[j] - kia * GK[(size_t)j * nk + a];
      }
    }
  });
}

int pseudo_inverse_sym(int n, std::vector<double>& A, std::vector<double>& pinv, int& snapped, double theta) {
  if (n < 1) return STK_ERR_INVALID_ARG;
  std::vector<double> S, Ah, lam, Qt;
  equilibrate_sym(n, A, S, Ah);
  if (!symmetric_eigen(n, Ah, lam, Qt)) return pseudo_inverse_jacobi(n, A, pinv, snapped, theta);
  double lmax = 0.0;
  for (int i = 0; i < n; ++i) lmax = std::max(lmax, std::fabs(lam[i]));
  std::vector<double> inv(n, 0.0);
  std::vector<int> kern;
  for (int i = 0; i < n; ++i) {
    if (std::fabs(lam[i]) <= theta * lmax) kern.push_back(i);
    else inv[i] = 1.0 / lam[i];
  }
  snapped = (int)kern.size();
  // G = S (sum_k q_k q_k^T / lam_k) S
  pinv.assign((size_t)n * n, 0.0);
  parallel_for(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      double* row = &pinv[(size_t)i * n];
      for (int k = 0; k < n; ++k) {
        const double f = Qt[(size_t)k * n + i] * inv[k];
        if (f == 0.0) continue;
        const double* q = &Qt[(size_t)k * n];
        for (int j = 0; j < n; ++j) row[j] += f * q[j];
      }
      for (int j = 0; j < n; ++j) row[j] *= S[i] * S[j];
    }
  });
  // K: S q_k for the snapped k (kernel vectors of A)
  std::vector<double> K((size_t)snapped * n);
  for (int a = 0; a < snapped; ++a)
    for (int j = 0; j < n; ++j) K[(size_t)a * n + j] = S[j] * Qt[(size_t)kern[a] * n + j];
  project_off_kernel(n, pinv, K, snapped);
  return STK_OK;
}

// ---------------------------------------------------------------------------
// Mesh helpers
// ---------------------------------------------------------------------------
void element_index(const int* n, int d, int64_t e, int* idx) {
  for (int k = 0; k < d; ++k) {
    idx[k] = (int)(e % n[k]);
    e /= n[k];
  }
}

static int64_t element_of(const int* n, int d, const int* idx) {
  int64_t e = 0, st = 1;
  for (int k = 0; k < d; ++k) {
    e += idx[k] * st;
    st *= n[k];
  }
  return e;
}

// Neighbour of element e at integer offset off (per-axis -1/0/1); -1 if it
// leaves a non-periodic box.
static int64_t neighbour(const Ctx& c, const int* n, int64_t e, const int* off) {
  int idx[3];
  element_index(n, c.d, e, idx);
  for (int k = 0; k < c.d; ++k) {
    int v = idx[k] + off[k];
    if (v < 0 || v >= n[k]) {
      if (c.bc[2 * k] != STK_BC_PERIODIC) return -1;
      v = (v + n[k]) % n[k];
    }
    idx[k] = v;
  }
  return element_of(n, c.d, idx);
}

static inline int slot_minus(int k) { return 1 + 2 * k; }
static inline int slot_plus(int k) { return 2 + 2 * k; }
// G_k slots: 0 the element, 1 its -e_k neighbour, 2 its +e_k neighbour.
constexpr int kGS = 3;

// ---------------------------------------------------------------------------
// Coupling pattern (derived from the one-sided fluxes u^ = u^-, sigma^ = sigma^+
// of eq. ustarflux / qstarflux and the lift into the + element, eq. gsum)
// ---------------------------------------------------------------------------
void build_pattern(int d, int p, int gamma, bool multiphase, Pattern& pat) {
  std::memset(&pat, 0, sizeof(pat));
  int s = 1;
  for (int k = 0; k < d; ++k) s *= (p + 1);
  pat.d = d;
  pat.s = s;
  pat.nb = (d + 1) * s;
  auto offset_slot = [&](int o0, int o1, int o2) {
    for (int i = 0; i < pat.NO; ++i)
      if (pat.off[i][0] == o0 && pat.off[i][1] == o1 && pat.off[i][2] == o2) return i;
    if (pat.NO >= kMaxOffsets) return 0;
    pat.off[pat.NO][0] = o0;
    pat.off[pat.NO][1] = o1;
    pat.off[pat.NO][2] = o2;
    return pat.NO++;
  };
  auto unit = [&](int k, int sgn, int* o) {
    o[0] = o[1] = o[2] = 0;
    o[k] = sgn;
  };
  auto add = [&](int rv, int cv, const int* o) {
    if (pat.T >= kMaxTasks) return;
    int t = pat.T++;
    pat.task_rv[t] = rv;
    pat.task_cv[t] = cv;
    pat.task_o[t] = offset_slot(o[0], o[1], o[2]);
  };
  // Fixed offset order: -e_k, +e_k for every axis first (the learned
  // smoother's features rely on it), then the others.
  for (int k = 0; k < d; ++k) {
    int o[3];
    unit(k, -1, o);
    offset_slot(o[0], o[1], o[2]);
    unit(k, 1, o);
    offset_slot(o[0], o[1], o[2]);
  }
  // Single phase: G_k(E, .) is nonzero at E and E - e_k (one-sided fluxes).
  // With interphase faces the lift can also land at E + e_k, so G_k has the
  // offsets {0, -e_k, +e_k} and products G^T M G reach +-2e_k and the
  // diagonal neighbours +-e_i +- e_j.
  for (int rv = 0; rv <= d; ++rv) {
    pat.rv_t0[rv] = pat.T;
    int o[3];
    if (rv < d) {
      int i = rv;
      for (int k = 0; k < d; ++k) {
        unit(k, -1, o);
        add(i, i, o);
        unit(k, 1, o);
        add(i, i, o);
        if (multiphase) {
          unit(k, -2, o);
          add(i, i, o);
          unit(k, 2, o);
          add(i, i, o);
        }
      }
      if (gamma) {
        for (int j = 0; j < d; ++j) {
          if (j == i) continue;
          if (!multiphase) {
            unit(i, -1, o);
            add(i, j, o);
            unit(j, 1, o);
            add(i, j, o);
            o[0] = o[1] = o[2] = 0;
            o[j] = 1;
            o[i] = -1;
            add(i, j, o);
          } else {
            for (int si = -1; si <= 1; ++si)
              for (int sj = -1; sj <= 1; ++sj) {
                if (si == 0 && sj == 0) continue;
                o[0] = o[1] = o[2] = 0;
                o[i] = si;
                o[j] = sj;
                add(i, j, o);
              }
          }
        }
      }
      unit(i, 1, o);
      add(i, d, o);
      if (multiphase) {
        unit(i, -1, o);
        add(i, d, o);
      }
    } else {
      for (int j = 0; j < d; ++j) {
        unit(j, -1, o);
        add(d, j, o);
        if (multiphase) {
          unit(j, 1, o);
          add(d, j, o);
        }
      }
      for (int k = 0; k < d; ++k) {
        unit(k, -1, o);
        add(d, d, o);
        unit(k, 1, o);
        add(d, d, o);
      }
    }
    pat.rv_t1[rv] = pat.T;
  }
  // Distinct gathers (offset, column variable).
  for (int t = 0; t < pat.T; ++t) {
    int g = -1;
    for (int i = 0; i < pat.NG; ++i)
      if (pat.g_o[i] == pat.task_o[t] && pat.g_cv[i] == pat.task_cv[t]) g = i;
    if (g < 0) {
      g = pat.NG++;
      pat.g_o[g] = pat.task_o[t];
      pat.g_cv[g] = pat.task_cv[t];
    }
    pat.task_g[t] = g;
  }
  pat.TR = pat.T * s;
  pat.TRP = (pat.TR + 7) / 8 * 8;
  pat.NBP = (pat.nb + 7) / 8 * 8;
}

// ---------------------------------------------------------------------------
// Sample points
// ---------------------------------------------------------------------------
static void centre_of(const Ctx& c, const int* n, const double* h, int64_t e, double* x) {
  int idx[3];
  element_index(n, c.d, e, idx);
  for (int k = 0; k < c.d; ++k) x[k] = c.lo[k] + (idx[k] + 0.5) * h[k];
}

// Enumerate faces of a kind: interior faces (kind 1) as (axis, right element);
// boundary faces (kind 2) as (axis, side, element).
struct Face {
  int k;
  int side;     // -1 / +1 side of element e
  int64_t e;    // right element (interior) or the boundary element
  int64_t L;    // left element (interior only)
};

static void enumerate_faces(const Ctx& c, int kind, std::vector<Face>& out) {
  out.clear();
  int64_t ne = 1;
  for (int k = 0; k < c.d; ++k) ne *= c.n[k];
  for (int k = 0; k < c.d; ++k) {
    bool per = c.bc[2 * k] == STK_BC_PERIODIC;
    if (kind == STK_PTS_INTERIOR_FACE) {
      for (int64_t e = 0; e < ne; ++e) {
        int idx[3];
        element_index(c.n, c.d, e, idx);
        if (idx[k] == 0 && !per) continue;
        if (c.n[k] == 1) continue;
        int off[3] = {0, 0, 0};
        off[k] = -1;
        out.push_back({k, -1, e, neighbour(c, c.n, e, off)});
      }
    } else {
      if (per) continue;
      for (int sd = -1; sd <= 1; sd += 2) {
        for (int64_t e = 0; e < ne; ++e) {
          int idx[3];
          element_index(c.n, c.d, e, idx);
          if (idx[k] != (sd < 0 ? 0 : c.n[k] - 1)) continue;
          out.push_back({k, sd, e, -1});
        }
      }
    }
  }
}

void face_points(const Ctx& c, int kind, std::vector<double>& xyz, std::vector<double>* nrm) {
  int d = c.d, q = c.q;
  std::vector<double> gx, gw;
  gauss_rule(q, gx, gw);
  double h[3];
  for (int k = 0; k < d; ++k) h[k] = (c.hi[k] - c.lo[k]) / c.n[k];
  xyz.clear();
  if (nrm) nrm->clear();
  if (kind == STK_PTS_VOLUME) {
    int64_t ne = 1;
    for (int k = 0; k < d; ++k) ne *= c.n[k];
    int Q = 1;
    for (int k = 0; k < d; ++k) Q *= q;
    xyz.resize((size_t)ne * Q * d);
    for (int64_t e = 0; e < ne; ++e) {
      double ctr[3];
      centre_of(c, c.n, h, e, ctr);
      for (int qi = 0; qi < Q; ++qi) {
        int r = qi;
        for (int k = 0; k < d; ++k) {
          xyz[((size_t)e * Q + qi) * d + k] = ctr[k] + 0.5 * h[k] * gx[r % q];
          r /= q;
        }
      }
    }
    return;
  }
  std::vector<Face> faces;
  enumerate_faces(c, kind, faces);
  int Qf = 1;
  for (int k = 0; k < d - 1; ++k) Qf *= q;
  xyz.resize(faces.size() * Qf * d);
  if (nrm) nrm->resize(faces.size() * Qf * d, 0.0);
  for (size_t f = 0; f < faces.size(); ++f) {
    double ctr[3];
    centre_of(c, c.n, h, faces[f].e, ctr);
    int k = faces[f].k;
    for (int qi = 0; qi < Qf; ++qi) {
      int r = qi;
      for (int j = 0; j < d; ++j) {
        double v;
        if (j == k) {
          v = ctr[j] + 0.5 * h[j] * faces[f].side;
        } else {
          v = ctr[j] + 0.5 * h[j] * gx[r % q];
          r /= q;
        }
        xyz[(f * Qf + qi) * d + j] = v;
        if (nrm) (*nrm)[(f * Qf + qi) * d + j] = (j == k) ? (double)faces[f].side : 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fine-level assembly (Appendix A)
// ---------------------------------------------------------------------------
struct Tensors {
  int d, p, s, m, q, Q, Qf;
  Basis1 B;
  std::vector<double> gw;                  // 1-D Gauss weights (q points)
  std::vector<double> Phi;                 // [Q][s] volume basis values
  std::vector<double> wQ;                  // [Q] tensor weights
  std::vector<double> PhiF[3][2];          // [axis][side][Qf][s] face basis values
  std::vector<double> wF;                  // [Qf]
  std::vector<double> Kax[3];              // kron_axis(K) per axis
  std::vector<double> F[3][2][2];          // F[k][sr][sc] = kron_axis(outer(tr_sr, tr_sc))
};

static Tensors make_tensors(int d, int p, int q) {
  Tensors T;
  T.d = d;
  T.p = p;
  T.m = p + 1;
  T.q = q;
  T.s = 1;
  for (int k = 0; k < d; ++k) T.s *= T.m;
  T.B = basis1(p);
  std::vector<double> gx;
  gauss_rule(q, gx, T.gw);
  T.Q = 1;
  for (int k = 0; k < d; ++k) T.Q *= q;
  T.Qf = T.Q / q;
  // psi table at the 1-D points
  std::vector<double> ps((size_t)q * T.m);
  for (int i = 0; i < q; ++i) psi_eval(p, gx[i], &ps[(size_t)i * T.m], nullptr);
  T.Phi.assign((size_t)T.Q * T.s, 1.0);
  T.wQ.assign(T.Q, 1.0);
  for (int qi = 0; qi < T.Q; ++qi) {
    int r = qi, qd[3];
    for (int k = 0; k < d; ++k) {
      qd[k] = r % q;
      r /= q;
      T.wQ[qi] *= T.gw[qd[k]];
    }
    for (int a = 0; a < T.s; ++a) {
      double v = 1.0;
      for (int k = 0; k < d; ++k) v *= ps[(size_t)qd[k] * T.m + mode_digit(a, k, T.m)];
      T.Phi[(size_t)qi * T.s + a] = v;
    }
  }
  T.wF.assign(T.Qf, 1.0);
  for (int qi = 0; qi < T.Qf; ++qi) {
    int r = qi;
    for (int k = 0; k < d - 1; ++k) {
      T.wF[qi] *= T.gw[r % q];
      r /= q;
    }
  }
  for (int k = 0; k < d; ++k) {
    for (int sd = 0; sd < 2; ++sd) {
      T.PhiF[k][sd].assign((size_t)T.Qf * T.s, 1.0);
      for (int qi = 0; qi < T.Qf; ++qi) {
        int r = qi, qd[3];
        for (int j = 0; j < d; ++j) {
          if (j == k) continue;
          qd[j] = r % q;
          r /= q;
        }
        for (int a = 0; a < T.s; ++a) {
          double v = 1.0;
          for (int j = 0; j < d; ++j) {
            int aj = mode_digit(a, j, T.m);
            v *= (j == k) ? T.B.tr[sd][aj] : ps[(size_t)qd[j] * T.m + aj];
          }
          T.PhiF[k][sd][(size_t)qi * T.s + a] = v;
        }
      }
    }
    T.Kax[k] = kron_axis(d, p, k, T.B.K.data());
    for (int sr = 0; sr < 2; ++sr)
      for (int sc = 0; sc < 2; ++sc) {
        std::vector<double> o((size_t)T.m * T.m);
        for (int a = 0; a < T.m; ++a)
          for (int b = 0; b < T.m; ++b) o[a * T.m + b] = T.B.tr[sr][a] * T.B.tr[sc][b];
        T.F[k][sr][sc] = kron_axis(d, p, k, o.data());
      }
  }
  return T;
}

static inline int sidx(int side) { return side < 0 ? 0 : 1; }

static void axpy_block(int s, double a, const std::vector<double>& X, double* Y) {
  for (int i = 0; i < s * s; ++i) Y[i] += a * X[i];
}

static void fine_assembly(Ctx& c, const Tensors& T, HostLevel& L) {
  int d = c.d, s = T.s, ss = s * s, nsl = 1 + 2 * d;
  int64_t ne = L.ne;
  bool unsteady = c.delta > 0;
  L.M.assign((size_t)ne * ss, 0.0);
  L.Mmu.assign((size_t)ne * ss, 0.0);
  if (unsteady) L.Mrho.assign((size_t)ne * ss, 0.0);
  L.G.assign((size_t)d * ne * kGS * ss, 0.0);
  L.Et.assign((size_t)ne * nsl * ss, 0.0);
  L.E.assign((size_t)ne * nsl * ss, 0.0);
  if (unsteady) {
    L.Emu.assign((size_t)ne * nsl * ss, 0.0);
    L.Erho.assign((size_t)ne * nsl * ss, 0.0);
  }
  double jac = L.vol / std::pow(2.0, d);
  parallel_for(ne, [&](int64_t a, int64_t b) {
    for (int64_t e = a; e < b; ++e) {
      for (int i = 0; i < s; ++i) L.M[(size_t)e * ss + i * s + i] = L.vol;
      // M_mu (and M_rho) = sum_q w_q mu_q phi(x_q) phi(x_q)^T, one rank-one
      // update per quadrature point, row by row (vectorisable inner loop)
      double* __restrict__ mm = &L.Mmu[(size_t)e * ss];
      for (int qi = 0; qi < T.Q; ++qi) {
        const double wm = jac * T.wQ[qi] * c.mu_vol[(size_t)e * T.Q + qi];
        const double* __restrict__ ph = &T.Phi[(size_t)qi * s];
        for (int i = 0; i < s; ++i) {
          const double a = wm * ph[i];
          double* __restrict__ row = mm + i * s;
          for (int j = 0; j < s; ++j) row[j] += a * ph[j];
        }
      }
      if (unsteady) {
        double* __restrict__ mr = &L.Mrho[(size_t)e * ss];
        for (int qi = 0; qi < T.Q; ++qi) {
          const double wr = jac * T.wQ[qi] * c.rho_vol[(size_t)e * T.Q + qi];
          const double* __restrict__ ph = &T.Phi[(size_t)qi * s];
          for (int i = 0; i < s; ++i) {
            const double a = wr * ph[i];
            double* __restrict__ row = mr + i * s;
            for (int j = 0; j < s; ++j) row[j] += a * ph[j];
          }
        }
      }
      for (int k = 0; k < d; ++k)
        axpy_block(s, 1.0 / L.h[k], T.Kax[k], &L.G[(((size_t)k * ne + e) * kGS + 0) * ss]);
    }
  });
  double wsum = 0.0;
  for (double w : T.wF) wsum += w;
  // Interior faces: lift into the right element, pressure (and intra-phase
  // velocity) penalties.
  std::vector<Face> faces;
  enumerate_faces(c, STK_PTS_INTERIOR_FACE, faces);
  for (size_t f = 0; f < faces.size(); ++f) {
    int k = faces[f].k;
    int64_t R = faces[f].e, Lf = faces[f].L;
    double hk = L.h[k], area = L.vol / hk;
    if (!L.chi.empty() && L.chi[Lf] != L.chi[R]) {
      // Interphase face (eq. gsum, eq. Epenalty): normal from the lower phase
      // (the - element) into the higher; lift (1-lambda)(u+ - u-) v- n +
      // lambda (u+ - u-) v+ n, lambda by viscosity upwinding
      // (eq. viscosityupwind); penalty tau_ij [u][v] with
      // tau_ij = 3 p min(mu-, mu+) / h; no pressure penalty.
      const bool lowL = L.chi[Lf] < L.chi[R];
      const int64_t mi = lowL ? Lf : R, pl = lowL ? R : Lf;
      const double sig = lowL ? 1.0 : -1.0;
      const int sm = lowL ? 1 : 0, sp = lowL ? 0 : 1;             // face-side index of - / + element
      const int slot_mp = lowL ? 2 : 1, slot_pm = lowL ? 1 : 2;   // G slot of the other element
      const double mum = c.mu_phase[L.chi[mi] - 1], mup = c.mu_phase[L.chi[pl] - 1];
      const double lam = mum < mup ? 0.0 : (mum == mup ? 0.5 : 1.0);
      const double am = (1.0 - lam) * sig * area / L.vol, ap = lam * sig * area / L.vol;
      axpy_block(s, am, T.F[k][sm][sp], &L.G[(((size_t)k * ne + mi) * kGS + slot_mp) * ss]);
      axpy_block(s, -am, T.F[k][sm][sm], &L.G[(((size_t)k * ne + mi) * kGS + 0) * ss]);
      axpy_block(s, ap, T.F[k][sp][sp], &L.G[(((size_t)k * ne + pl) * kGS + 0) * ss]);
      axpy_block(s, -ap, T.F[k][sp][sm], &L.G[(((size_t)k * ne + pl) * kGS + slot_pm) * ss]);
      const double t = 3.0 * c.p * std::min(mum, mup) / hk * area;
      const int psl_mp = lowL ? slot_plus(k) : slot_minus(k), psl_pm = lowL ? slot_minus(k) : slot_plus(k);
      axpy_block(s, t, T.F[k][sm][sm], &L.Et[((size_t)mi * nsl + 0) * ss]);
      axpy_block(s, -t, T.F[k][sm][sp], &L.Et[((size_t)mi * nsl + psl_mp) * ss]);
      axpy_block(s, -t, T.F[k][sp][sm], &L.Et[((size_t)pl * nsl + psl_pm) * ss]);
      axpy_block(s, t, T.F[k][sp][sp], &L.Et[((size_t)pl * nsl + 0) * ss]);
      continue;
    }
    double* GRR = &L.G[(((size_t)k * ne + R) * kGS + 0) * ss];
    double* GRL = &L.G[(((size_t)k * ne + R) * kGS + 1) * ss];
    axpy_block(s, area / L.vol, T.F[k][0][0], GRR);
    axpy_block(s, -area / L.vol, T.F[k][0][1], GRL);
    double muf = 0.0, rhof = 0.0;
    for (int qi = 0; qi < T.Qf; ++qi) {
      muf += T.wF[qi] * c.mu_if[f * T.Qf + qi];
      if (unsteady) rhof += T.wF[qi] * c.rho_if[f * T.Qf + qi];
    }
    muf /= wsum;
    rhof /= wsum;
    auto jump_pen = [&](std::vector<double>& Op, double tp) {
      double a = tp * area;
      axpy_block(s, a, T.F[k][1][1], &Op[((size_t)Lf * nsl + 0) * ss]);
      axpy_block(s, a, T.F[k][0][0], &Op[((size_t)R * nsl + 0) * ss]);
      axpy_block(s, -a, T.F[k][1][0], &Op[((size_t)Lf * nsl + slot_plus(k)) * ss]);
      axpy_block(s, -a, T.F[k][0][1], &Op[((size_t)R * nsl + slot_minus(k)) * ss]);
    };
    if (unsteady) {
      double tmu = c.tau * hk / muf;
      double trho = c.tau0 * c.delta / (hk * rhof);
      double tgen = 1.0 / (hk * rhof / (c.tau0 * c.delta) + muf / (c.tau * hk));
      jump_pen(L.E, tgen);
      jump_pen(L.Emu, tmu);
      jump_pen(L.Erho, trho);
    } else {
      jump_pen(L.E, c.tau * hk / muf);
    }
    if (c.c_intra > 0) jump_pen(L.Et, c.c_intra * c.p * muf / hk);
  }
  // Boundary faces: Dirichlet lift and velocity penalty.
  enumerate_faces(c, STK_PTS_BOUNDARY_FACE, faces);
  for (size_t f = 0; f < faces.size(); ++f) {
    int k = faces[f].k, sd = faces[f].side;
    int type = c.bc[2 * k + (sd < 0 ? 0 : 1)];
    if (type != STK_BC_DIRICHLET) continue;
    int64_t e = faces[f].e;
    double hk = L.h[k], area = L.vol / hk;
    axpy_block(s, -sd * area / L.vol, T.F[k][sidx(sd)][sidx(sd)],
               &L.G[(((size_t)k * ne + e) * kGS + 0) * ss]);
    double muf = 0.0;
    for (int qi = 0; qi < T.Qf; ++qi) muf += T.wF[qi] * c.mu_bf[f * T.Qf + qi];
    muf /= wsum;
    double tb = c.c_bdry * c.p * muf / hk;
    axpy_block(s, tb * area, T.F[k][sidx(sd)][sidx(sd)], &L.Et[((size_t)e * nsl + 0) * ss]);
  }
}

// ---------------------------------------------------------------------------
// Operator coarsening (Appendix B)
// ---------------------------------------------------------------------------
static void coarsen_level(const Ctx& c, const std::vector<double>& Pch, const HostLevel& F,
                          HostLevel& Cl) {
  int d = c.d, s = c.s, ss = s * s, nsl = 1 + 2 * d;
  bool unsteady = c.delta > 0;
  int64_t ne = Cl.ne, nef = F.ne;
  Cl.M.assign((size_t)ne * ss, 0.0);
  Cl.Mmu.assign((size_t)ne * ss, 0.0);
  if (unsteady) Cl.Mrho.assign((size_t)ne * ss, 0.0);
  Cl.G.assign((size_t)d * ne * kGS * ss, 0.0);
  Cl.Et.assign((size_t)ne * nsl * ss, 0.0);
  Cl.E.assign((size_t)ne * nsl * ss, 0.0);
  std::vector<double> Emu2, Erho2;
  if (unsteady) {
    Cl.Emu.assign((size_t)ne * nsl * ss, 0.0);
    Cl.Erho.assign((size_t)ne * nsl * ss, 0.0);
  }
  parallel_for(ne, [&](int64_t a, int64_t b) {
    std::vector<double> tmp, acc(ss), Minv(ss);
    for (int64_t C = a; C < b; ++C) {
      int I[3];
      element_index(Cl.n, d, C, I);
      // children
      for (int ch = 0; ch < (1 << d); ++ch) {
        int fi[3];
        for (int k = 0; k < d; ++k) fi[k] = 2 * I[k] + ((ch >> k) & 1);
        int64_t f = element_of(F.n, d, fi);
        const double* Pf = &Pch[(size_t)ch * ss];
        // Mass-type blocks: M_2h = I^T M I (Algorithms 2 and 3).
        triple_acc(s, 1.0, Pf, &F.M[(size_t)f * ss], Pf, &Cl.M[(size_t)C * ss], tmp);
        triple_acc(s, 1.0, Pf, &F.Mmu[(size_t)f * ss], Pf, &Cl.Mmu[(size_t)C * ss], tmp);
        if (unsteady)
          triple_acc(s, 1.0, Pf, &F.Mrho[(size_t)f * ss], Pf, &Cl.Mrho[(size_t)C * ss], tmp);
        // Face-coupled penalties: slot 0 and +-e_k.
        for (int sl = 0; sl < nsl; ++sl) {
          int k = (sl - 1) / 2;
          int sg = (sl == 0) ? 0 : ((sl % 2 == 1) ? -1 : 1);
          int fo[3] = {fi[0], fi[1], fi[2]};
          int co[3] = {0, 0, 0};
          if (sl > 0) {
            int v = fi[k] + sg;               // unwrapped fine neighbour index
            if ((v < 0 || v >= F.n[k]) && c.bc[2 * k] != STK_BC_PERIODIC) continue;
            int vc = (v >= 0) ? v / 2 : -1;   // floor(v / 2) for v >= -1
            co[k] = vc - I[k];
            fo[k] = ((v % F.n[k]) + F.n[k]) % F.n[k];
          }
          int64_t g = element_of(F.n, d, fo);
          int chg = 0;
          for (int kk = 0; kk < d; ++kk) chg |= (((fi[kk] + ((sl > 0 && kk == k) ? sg : 0)) & 1) << kk);
          const double* Pg = &Pch[(size_t)chg * ss];
          int csl = 0;
          for (int kk = 0; kk < d; ++kk)
            if (co[kk] != 0) csl = co[kk] < 0 ? slot_minus(kk) : slot_plus(kk);
          // Penalty coarsening: velocity penalty x1/2 and pressure penalty x2 (Algorithm 2);
          // E_mu x2 and E_rho x1/2 (Algorithm 3).
          triple_acc(s, 0.5, Pf, &F.Et[((size_t)f * nsl + sl) * ss], Pg,
                     &Cl.Et[((size_t)C * nsl + csl) * ss], tmp);
          if (unsteady) {
            triple_acc(s, 2.0, Pf, &F.Emu[((size_t)f * nsl + sl) * ss], Pg,
                       &Cl.Emu[((size_t)C * nsl + csl) * ss], tmp);
            triple_acc(s, 0.5, Pf, &F.Erho[((size_t)f * nsl + sl) * ss], Pg,
                       &Cl.Erho[((size_t)C * nsl + csl) * ss], tmp);
          } else {
            triple_acc(s, 2.0, Pf, &F.E[((size_t)f * nsl + sl) * ss], Pg,
                       &Cl.E[((size_t)C * nsl + csl) * ss], tmp);
          }
        }
      }
      // G_2h = M_2h^{-1} I^T M_h G_h I (Algorithm 2).
      std::string err;
      invert_dense(s, &Cl.M[(size_t)C * ss], Minv.data());
      for (int k = 0; k < d; ++k) {
        std::vector<double> sum[kGS];
        for (int t = 0; t < kGS; ++t) sum[t].assign(ss, 0.0);
        for (int ch = 0; ch < (1 << d); ++ch) {
          int fi[3];
          for (int kk = 0; kk < d; ++kk) fi[kk] = 2 * I[kk] + ((ch >> kk) & 1);
          int64_t f = element_of(F.n, d, fi);
          const double* Pf = &Pch[(size_t)ch * ss];
          for (int sl = 0; sl < kGS; ++sl) {
            int chg = ch, csl = 0;
            if (sl > 0) {
              const int sg = (sl == 1) ? -1 : 1;
              const int v = fi[k] + sg;                 // unwrapped fine neighbour index
              if ((v < 0 || v >= F.n[k]) && c.bc[2 * k] != STK_BC_PERIODIC) continue;
              const int vc = (v >= 0) ? v / 2 : -1;     // floor(v / 2) for v >= -1
              const int co = vc - I[k];
              csl = (co == 0) ? 0 : (co < 0 ? 1 : 2);
              chg = ch ^ (1 << k);
            }
            // P_f^T M_f G_f(slot) P_g  (Algorithm 2, before M_2h^{-1})
            std::vector<double> MG(ss, 0.0);
            gemm_acc(s, 1.0, &F.M[(size_t)f * ss], false, &F.G[(((size_t)k * nef + f) * kGS + sl) * ss], MG.data());
            triple_acc(s, 1.0, Pf, MG.data(), &Pch[(size_t)chg * ss], sum[csl].data(), tmp);
          }
        }
        for (int t = 0; t < kGS; ++t) {
          double* out = &Cl.G[(((size_t)k * ne + C) * kGS + t) * ss];
          std::fill(out, out + ss, 0.0);
          gemm_acc(s, 1.0, Minv.data(), false, sum[t].data(), out);
        }
      }
    }
  });
  if (unsteady) {
    // eq. (Etimedep): combine per element-pair block by Frobenius weights.
    for (size_t blk = 0; blk < (size_t)ne * nsl; ++blk) {
      const double* a = &Cl.Emu[blk * ss];
      const double* r = &Cl.Erho[blk * ss];
      double fa = 0, fr = 0;
      for (int i = 0; i < ss; ++i) {
        fa += a[i] * a[i];
        fr += r[i] * r[i];
      }
      fa = std::sqrt(fa);
      fr = std::sqrt(fr);
      double* out = &Cl.E[blk * ss];
      if (fa + fr > 0) {
        double wa = (fr / (fa + fr)) * (fr / (fa + fr));
        double wr = (fa / (fa + fr)) * (fa / (fa + fr));
        for (int i = 0; i < ss; ++i) out[i] = wa * a[i] + wr * r[i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Stokes blocks of a level (eq. blockform / timedep2 with eq. viscousop)
// ---------------------------------------------------------------------------
// Pointer to the G_k block (E, E + rel) with rel in {0, -e_k}; nullptr otherwise.
static const double* Gblk(const HostLevel& L, int d, int s, int k, int64_t E, const int* rel) {
  for (int j = 0; j < d; ++j)
    if (j != k && rel[j] != 0) return nullptr;
  int sl;
  if (rel[k] == 0) sl = 0;
  else if (rel[k] == -1) sl = 1;
  else if (rel[k] == 1) sl = 2;
  else return nullptr;
  return &L.G[(((size_t)k * L.ne + E) * kGS + sl) * s * s];
}

// Slot of a face-penalty operator for offset o (0, -e_k, +e_k), or -1.
static int pen_slot(int d, const int* o) {
  int nz = 0, k = -1;
  for (int j = 0; j < d; ++j)
    if (o[j] != 0) {
      ++nz;
      k = j;
    }
  if (nz == 0) return 0;
  if (nz > 1 || (o[k] != 1 && o[k] != -1)) return -1;
  return o[k] < 0 ? slot_minus(k) : slot_plus(k);
}

// Per-thread cache of the viscous term sum_k sum_E G_k(E, a)^T M_mu(E) G_k(E, a+o)
// of one element a, keyed by the offset o (each component in [-2, 2]): every
// diagonal velocity block (i, i) at offset o shares it.
struct LapCache {
  std::vector<double> val;
  std::vector<int64_t> owner;   // element whose term the slot holds, -1 if none
  void init(int ss) {
    val.assign((size_t)125 * ss, 0.0);
    owner.assign(125, -1);
  }
  static int key(const int* o) { return (o[0] + 2) * 25 + (o[1] + 2) * 5 + (o[2] + 2); }
};

// s x s block of the operator, row variable rv at element a, column variable
// cv at element a + o.
static void stokes_block(const Ctx& c, const HostLevel& L, int64_t a, int rv, int cv, const int* o,
                         double* out, std::vector<double>& tmp, LapCache* lap = nullptr) {
  int d = c.d, s = c.s, ss = s * s, nsl = 1 + 2 * d;
  std::fill(out, out + ss, 0.0);
  auto exists = [&](const int* off, int64_t& id) {
    id = neighbour(c, L.n, a, off);
    return id >= 0;
  };
  bool unsteady = c.delta > 0;
  if (rv < d && cv < d) {
    int i = rv, j = cv;
    // delta_ij sum_k G_k^T M_mu G_k  and  gamma G_j^T M_mu G_i
    auto add_term = [&](int kr, int kc, double alpha) {
      // sum over E = a + oE, oE in {0, +e_kr, -e_kr}: G_kr(E, a)^T M_mu(E) G_kc(E, a + o)
      for (int t = 0; t < 3; ++t) {
        int oE[3] = {0, 0, 0};
        if (t == 1) oE[kr] = 1;
        if (t == 2) oE[kr] = -1;
        int64_t E;
        if (!exists(oE, E)) continue;
        int relA[3] = {-oE[0], -oE[1], -oE[2]};
        int relB[3] = {o[0] - oE[0], o[1] - oE[1], o[2] - oE[2]};
        const double* Ga = Gblk(L, d, s, kr, E, relA);
        const double* Gb = Gblk(L, d, s, kc, E, relB);
        if (!Ga || !Gb) continue;
        triple_acc(s, alpha, Ga, &L.Mmu[(size_t)E * ss], Gb, out, tmp);
      }
    };
    if (i == j) {
      // the same for every i: computed once per (a, o) when a cache is given,
      // in the same order of accumulation, so the block is bit-identical
      double* cached = nullptr;
      if (lap) {
        const int key = LapCache::key(o);
        cached = &lap->val[(size_t)key * ss];
        if (lap->owner[key] != a) {
          std::fill(cached, cached + ss, 0.0);
          std::swap(cached, out);
          for (int k = 0; k < d; ++k) add_term(k, k, 1.0);
          std::swap(cached, out);
          lap->owner[key] = a;
        }
        std::copy(cached, cached + ss, out);
      } else {
        for (int k = 0; k < d; ++k) add_term(k, k, 1.0);
      }
    }
    if (c.gamma) add_term(j, i, 1.0);
    if (i == j) {
      int sl = pen_slot(d, o);
      if (sl >= 0) axpy_block(s, 1.0, std::vector<double>(&L.Et[((size_t)a * nsl + sl) * ss],
                                                          &L.Et[((size_t)a * nsl + sl) * ss] + ss),
                              out);
      if (unsteady && sl == 0)
        for (int t = 0; t < ss; ++t) out[t] += L.Mrho[(size_t)a * ss + t] / c.delta;
    }
  } else if (rv < d && cv == d) {
    // M Gcal_i = -G_i^T M : block (a, b) = -G_i(b, a)^T M(b)
    int64_t b;
    if (!exists(o, b)) return;
    int rel[3] = {-o[0], -o[1], -o[2]};
    const double* G = Gblk(L, d, s, rv, b, rel);
    if (!G) return;
    gemm_acc(s, -1.0, G, true, &L.M[(size_t)b * ss], out);
  } else if (rv == d && cv < d) {
    // Gcal_j^T M = -M G_j : block (a, b) = -M(a) G_j(a, b)
    int64_t b;
    if (!exists(o, b)) return;
    const double* G = Gblk(L, d, s, cv, a, o);
    if (!G) return;
    gemm_acc(s, -1.0, &L.M[(size_t)a * ss], false, G, out);
  } else {
    int sl = pen_slot(d, o);
    if (sl < 0) return;
    for (int t = 0; t < ss; ++t) out[t] = -L.E[((size_t)a * nsl + sl) * ss + t];
  }
}

static void stokes_level(const Ctx& c, HostLevel& L) {
  const Pattern& P = c.pat;
  int s = c.s, ss = s * s, nb = c.nb;
  int64_t ne = L.ne;
  L.D.assign((size_t)ne * nb * nb, 0.0);
  L.C.assign((size_t)ne * P.T * ss, 0.0);
  L.nbr.assign((size_t)ne * P.NO, -1);
  parallel_for(ne, [&](int64_t a0, int64_t a1) {
    std::vector<double> blk(ss), tmp;
    LapCache lap;
    lap.init(ss);
    int zero[3] = {0, 0, 0};
    for (int64_t a = a0; a < a1; ++a) {
      for (int rv = 0; rv <= c.d; ++rv)
        for (int cv = 0; cv <= c.d; ++cv) {
          stokes_block(c, L, a, rv, cv, zero, blk.data(), tmp, &lap);
          for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j)
              L.D[(size_t)a * nb * nb + (size_t)(rv * s + i) * nb + cv * s + j] = blk[i * s + j];
        }
      for (int t = 0; t < P.T; ++t) {
        const int* o = P.off[P.task_o[t]];
        stokes_block(c, L, a, P.task_rv[t], P.task_cv[t], o, &L.C[((size_t)a * P.T + t) * ss], tmp, &lap);
      }
      for (int oi = 0; oi < P.NO; ++oi) L.nbr[(size_t)a * P.NO + oi] = neighbour(c, L.n, a, P.off[oi]);
    }
  });
}

// ---------------------------------------------------------------------------
// Setup driver
// ---------------------------------------------------------------------------
// Greedy colouring of a level with phases (the coupling stencil reaches
// +-e_k, +-2e_k and +-e_i +- e_j): elements in order, each takes the smallest
// colour not taken by an already coloured element at any of those offsets.
void greedy_colours(const Ctx& c, const int* n, std::vector<int>& colour) {
  const int d = c.d;
  std::vector<std::array<int, 3>> offs;
  for (int k = 0; k < d; ++k)
    for (int m = 1; m <= 2; ++m)
      for (int sg = -1; sg <= 1; sg += 2) {
        std::array<int, 3> o = {0, 0, 0};
        o[k] = sg * m;
        offs.push_back(o);
      }
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j)
      for (int si = -1; si <= 1; si += 2)
        for (int sj = -1; sj <= 1; sj += 2) {
          std::array<int, 3> o = {0, 0, 0};
          o[i] = si;
          o[j] = sj;
          offs.push_back(o);
        }
  int64_t ne = 1;
  for (int k = 0; k < d; ++k) ne *= n[k];
  colour.assign(ne, -1);
  for (int64_t e = 0; e < ne; ++e) {
    uint64_t used = 0;
    for (const auto& o : offs) {
      int64_t j = neighbour(c, n, e, o.data());
      if (j >= 0 && colour[j] >= 0 && colour[j] < 64) used |= (1ULL << colour[j]);
    }
    int col = 0;
    while (used & (1ULL << col)) ++col;
    colour[e] = col;
  }
}

// sqrt(mu) scaling of Section 5.6 (multi-phase): per element mu_E^{-1/2} on
// velocity rows/columns, mu_E^{1/2} on pressure, mu_E the element mean of mu
// (M_mu(E)[0][0] / M(E)[0][0]); every level with its own mu_E.
static void scale_level(const Ctx& c, HostLevel& L) {
  const Pattern& P = c.pat;
  const int s = c.s, nb = c.nb, ss = s * s, d = c.d;
  const int64_t ne = L.ne;
  L.Dscale.assign((size_t)ne * nb, 1.0);
  for (int64_t e = 0; e < ne; ++e) {
    const double mu = L.Mmu[(size_t)e * ss] / L.M[(size_t)e * ss];
    for (int r = 0; r < nb; ++r) L.Dscale[(size_t)e * nb + r] = (r < d * s) ? 1.0 / std::sqrt(mu) : std::sqrt(mu);
  }
  for (int64_t a = 0; a < ne; ++a) {
    const double* da = &L.Dscale[(size_t)a * nb];
    double* D = &L.D[(size_t)a * nb * nb];
    for (int r = 0; r < nb; ++r)
      for (int q = 0; q < nb; ++q) D[(size_t)r * nb + q] *= da[r] * da[q];
    for (int t = 0; t < P.T; ++t) {
      const int64_t bb = L.nbr[(size_t)a * P.NO + P.task_o[t]];
      if (bb < 0) continue;
      const double fr = da[P.task_rv[t] * s], fc = L.Dscale[(size_t)bb * nb + P.task_cv[t] * s];
      double* C = &L.C[((size_t)a * P.T + t) * ss];
      for (int i = 0; i < ss; ++i) C[i] *= fr * fc;
    }
  }
}

int setup_host(Ctx& c) {
  int d = c.d;
  Tensors T = make_tensors(d, c.p, c.q);
  std::vector<double> Pch;
  child_matrices(d, c.p, Pch);
  c.host.clear();
  HostLevel L0;
  for (int k = 0; k < d; ++k) {
    L0.n[k] = c.n[k];
    L0.h[k] = (c.hi[k] - c.lo[k]) / c.n[k];
  }
  L0.ne = 1;
  L0.vol = 1.0;
  for (int k = 0; k < d; ++k) {
    L0.ne *= L0.n[k];
    L0.vol *= L0.h[k];
  }
  L0.chi = c.chi;
  fine_assembly(c, T, L0);
  c.host.push_back(std::move(L0));
  for (;;) {
    HostLevel& F = c.host.back();
    bool stop = false;
    for (int k = 0; k < d; ++k)
      if (F.n[k] % 2 == 1 || F.n[k] <= 2) stop = true;
    // an earlier bottom: this level is small enough for the dense eigen
    // pseudo-inverse (and is not the finest level)
    if (c.host.size() > 1 && c.bottom_max > 0 && (int64_t)F.ne * c.nb <= c.bottom_max) stop = true;
    if (stop) break;
    HostLevel Cl;
    Cl.ne = 1;
    Cl.vol = 1.0;
    for (int k = 0; k < d; ++k) {
      Cl.n[k] = F.n[k] / 2;
      Cl.h[k] = 2 * F.h[k];
      Cl.ne *= Cl.n[k];
      Cl.vol *= Cl.h[k];
    }
    if (!F.chi.empty()) {
      // Same-phase agglomeration (Section 3): every coarse cell must hold
      // children of a single phase, otherwise this is the bottom level.
      Cl.chi.assign(Cl.ne, 0);
      bool ok = true;
      for (int64_t f = 0; f < F.ne && ok; ++f) {
        int idx[3];
        element_index(F.n, d, f, idx);
        for (int k = 0; k < d; ++k) idx[k] /= 2;
        const int64_t C = element_of(Cl.n, d, idx);
        if (Cl.chi[C] == 0) Cl.chi[C] = F.chi[f];
        else if (Cl.chi[C] != F.chi[f]) ok = false;
      }
      if (!ok) break;
    }
    coarsen_level(c, Pch, F, Cl);
    c.host.push_back(std::move(Cl));
  }
  for (auto& L : c.host) {
    stokes_level(c, L);
    if (c.scale_mu) scale_level(c, L);
  }
  return STK_OK;
}

}  // namespace stk

namespace stk {

// Right-hand side (Appendix A, eq. appstokes1 / appstokes2, times M) from
// samples at the volume points (f_1..f_d, fdiv), boundary-face points
// (Dirichlet g or stress h) and, for interphase faces, interior-face points
// (g_ij then h_ij, normal from the lower phase into the higher).  b is
// [ne][nb], element-major, of the unscaled system.
int assemble_rhs_host2(const Ctx& c, const double* f_vol, const double* bdata, const double* idata, double* b) {
  int d = c.d, s = c.s, nb = c.nb, ss = s * s;
  Tensors T = make_tensors(d, c.p, c.q);
  const HostLevel& L = c.host[0];
  int64_t ne = L.ne;
  std::fill(b, b + (size_t)ne * nb, 0.0);
  double jac = L.vol / std::pow(2.0, d);
  for (int64_t e = 0; e < ne; ++e)
    for (int qi = 0; qi < T.Q; ++qi)
      for (int v = 0; v <= d; ++v) {
        double val = jac * T.wQ[qi] * f_vol[((size_t)e * T.Q + qi) * (d + 1) + v];
        for (int a = 0; a < s; ++a) b[(size_t)e * nb + v * s + a] += val * T.Phi[(size_t)qi * s + a];
      }
  std::vector<double> jg((size_t)d * d * ne * s, 0.0);   // [i][j][e][a]
  auto JG = [&](int i, int j, int64_t e, int a) -> double& { return jg[(((size_t)i * d + j) * ne + e) * s + a]; };
  std::vector<Face> faces;
  enumerate_faces(c, STK_PTS_BOUNDARY_FACE, faces);
  double wsum = 0.0;
  for (double w : T.wF) wsum += w;
  std::vector<double> integ(s), integ2(s);
  for (size_t f = 0; f < faces.size(); ++f) {
    int k = faces[f].k, sd = faces[f].side;
    int type = c.bc[2 * k + (sd < 0 ? 0 : 1)];
    int64_t e = faces[f].e;
    double hk = L.h[k], area = L.vol / hk, fj = area / std::pow(2.0, d - 1);
    const double* PhiF = T.PhiF[k][sidx(sd)].data();
    double muf = 0.0;
    for (int qi = 0; qi < T.Qf; ++qi) muf += T.wF[qi] * c.mu_bf[f * T.Qf + qi];
    muf /= wsum;
    for (int i = 0; i < d; ++i) {
      std::fill(integ.begin(), integ.end(), 0.0);
      for (int qi = 0; qi < T.Qf; ++qi) {
        double val = fj * T.wF[qi] * bdata[(f * T.Qf + qi) * d + i];
        for (int a = 0; a < s; ++a) integ[a] += val * PhiF[(size_t)qi * s + a];
      }
      if (type == STK_BC_DIRICHLET) {
        double tb = c.c_bdry * c.p * muf / hk;
        for (int a = 0; a < s; ++a) {
          b[(size_t)e * nb + i * s + a] += tb * integ[a];                     // -E_{u,g}(0)
          JG(i, k, e, a) += sd * integ[a];                                     // J_g,ik
        }
      } else if (type == STK_BC_STRESS) {
        for (int a = 0; a < s; ++a) b[(size_t)e * nb + i * s + a] += integ[a];  // J_h
      }
    }
  }
  // Interphase faces: J_g (eq. gsum), J_h (eq. wworkings), -E_{u,g}(0) (eq. Epenalty).
  if (!L.chi.empty() && idata) {
    enumerate_faces(c, STK_PTS_INTERIOR_FACE, faces);
    for (size_t f = 0; f < faces.size(); ++f) {
      const int64_t R = faces[f].e, Lf = faces[f].L;
      if (L.chi[Lf] == L.chi[R]) continue;
      const int k = faces[f].k;
      const bool lowL = L.chi[Lf] < L.chi[R];
      const int64_t mi = lowL ? Lf : R, pl = lowL ? R : Lf;
      const double sig = lowL ? 1.0 : -1.0;
      const int sm = lowL ? 1 : 0, sp = lowL ? 0 : 1;
      const double mum = c.mu_phase[L.chi[mi] - 1], mup = c.mu_phase[L.chi[pl] - 1];
      const double lam = mum < mup ? 0.0 : (mum == mup ? 0.5 : 1.0);
      const double hk = L.h[k], area = L.vol / hk, fj = area / std::pow(2.0, d - 1);
      const double tij = 3.0 * c.p * std::min(mum, mup) / hk;
      const double* Pm = T.PhiF[k][sm].data();
      const double* Pp = T.PhiF[k][sp].data();
      for (int i = 0; i < d; ++i) {
        // g part: components i of g at the face points; h part likewise
        for (int part = 0; part < 2; ++part) {
          std::fill(integ.begin(), integ.end(), 0.0);
          std::fill(integ2.begin(), integ2.end(), 0.0);
          for (int qi = 0; qi < T.Qf; ++qi) {
            const double val = fj * T.wF[qi] * idata[(f * T.Qf + qi) * 2 * d + part * d + i];
            for (int a = 0; a < s; ++a) {
              integ[a] += val * Pm[(size_t)qi * s + a];
              integ2[a] += val * Pp[(size_t)qi * s + a];
            }
          }
          for (int a = 0; a < s; ++a) {
            if (part == 0) {
              JG(i, k, mi, a) += (1.0 - lam) * sig * integ[a];
              JG(i, k, pl, a) += lam * sig * integ2[a];
              b[(size_t)mi * nb + i * s + a] += tij * integ[a];
              b[(size_t)pl * nb + i * s + a] -= tij * integ2[a];
            } else {
              b[(size_t)mi * nb + i * s + a] += lam * integ[a];
              b[(size_t)pl * nb + i * s + a] += (1.0 - lam) * integ2[a];
            }
          }
        }
      }
    }
  }
  // J_{g.n} = sum_i J_g,ii into the pressure rows (eq. ewv).
  for (int64_t e = 0; e < ne; ++e)
    for (int i = 0; i < d; ++i)
      for (int a = 0; a < s; ++a) b[(size_t)e * nb + d * s + a] += JG(i, i, e, a);
  // - sum_j G_j^T M_mu M^{-1} (J_g,ij + gamma J_g,ji)
  std::vector<double> w((size_t)ne * s);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      bool any = false;
      for (size_t t = 0; t < (size_t)ne * s && !any; ++t) {
        const int64_t e = (int64_t)(t / s);
        const int a = (int)(t % s);
        if (JG(i, j, e, a) != 0.0 || (c.gamma && JG(j, i, e, a) != 0.0)) any = true;
      }
      if (!any) continue;
      for (int64_t e = 0; e < ne; ++e) {
        double t[64];
        for (int a = 0; a < s; ++a)
          t[a] = (JG(i, j, e, a) + c.gamma * JG(j, i, e, a)) / L.M[(size_t)e * ss + a * s + a];
        for (int a = 0; a < s; ++a) {
          double acc = 0.0;
          for (int bb = 0; bb < s; ++bb) acc += L.Mmu[(size_t)e * ss + a * s + bb] * t[bb];
          w[(size_t)e * s + a] = acc;
        }
      }
      // (G_j^T w)(a) = sum over E with G_j(E, a) != 0: E = a (slot 0),
      // E = a + e_j (slot 1 of E), E = a - e_j (slot 2 of E).
      for (int64_t a = 0; a < ne; ++a) {
        for (int tt = 0; tt < kGS; ++tt) {
          int oE[3] = {0, 0, 0};
          if (tt == 1) oE[j] = 1;
          if (tt == 2) oE[j] = -1;
          int64_t E = neighbour(c, L.n, a, oE);
          if (E < 0) continue;
          const double* G = &L.G[(((size_t)j * ne + E) * kGS + tt) * ss];
          for (int m = 0; m < s; ++m) {
            double acc = 0.0;
            for (int r = 0; r < s; ++r) acc += G[r * s + m] * w[(size_t)E * s + r];
            b[(size_t)a * nb + i * s + m] -= acc;
          }
        }
      }
    }
  return STK_OK;
}

int assemble_rhs_host(const Ctx& c, const double* f_vol, const double* bdata, double* b) {
  return assemble_rhs_host2(c, f_vol, bdata, nullptr, b);
}

// Interior-face points: phase of the - and + element (0, 0 on intraphase
// faces) and the normal (+e_k, or the interphase normal from the lower phase).
void interface_info(const Ctx& c, std::vector<int>& chim, std::vector<int>& chip, std::vector<double>& nrm) {
  std::vector<Face> faces;
  enumerate_faces(c, STK_PTS_INTERIOR_FACE, faces);
  int Qf = 1;
  for (int k = 0; k < c.d - 1; ++k) Qf *= c.q;
  chim.assign(faces.size() * Qf, 0);
  chip.assign(faces.size() * Qf, 0);
  nrm.assign(faces.size() * Qf * c.d, 0.0);
  for (size_t f = 0; f < faces.size(); ++f) {
    const int64_t R = faces[f].e, Lf = faces[f].L;
    const int k = faces[f].k;
    double sig = 1.0;
    int cm = 0, cp = 0;
    if (!c.chi.empty() && c.chi[Lf] != c.chi[R]) {
      const bool lowL = c.chi[Lf] < c.chi[R];
      sig = lowL ? 1.0 : -1.0;
      cm = lowL ? c.chi[Lf] : c.chi[R];
      cp = lowL ? c.chi[R] : c.chi[Lf];
    }
    for (int qi = 0; qi < Qf; ++qi) {
      chim[f * Qf + qi] = cm;
      chip[f * Qf + qi] = cp;
      nrm[(f * Qf + qi) * c.d + k] = sig;
    }
  }
}

}  // namespace stk

extern "C" int stk_host_pseudo_inverse(int n, const double* A, double theta, double* pinv, int* snapped) {
  if (n < 1 || n > 20000 || !A || !pinv || !(theta >= 0 && theta < 1)) return STK_ERR_INVALID_ARG;
  try {
    std::vector<double> a(A, A + (size_t)n * n), p;
    int sn = 0;
    int rc = stk::pseudo_inverse_sym(n, a, p, sn, theta);
    if (rc != STK_OK) return rc;
    std::copy(p.begin(), p.end(), pinv);
    if (snapped) *snapped = sn;
    return STK_OK;
  } catch (const std::bad_alloc&) {
    return STK_ERR_OOM;
  }
}

namespace stk {

// Element clustering (Concluding Remarks: larger smoother blocks for p = 1):
// the level-H operator re-blocked into clusters of 2^d elements, the children
// of one cell of the halved mesh.  A cluster's unknowns are ordered
// [variable][child][mode] (child = sum_k (i_k mod 2) 2^k), so a cluster is an
// "element" of cp.s = 2^d ep.s modes per variable and the element kernels run
// it unchanged.  Couplings inside a cluster join its diagonal block; the
// others land in the task of cp whose (row variable, column variable, cluster
// offset) they have.  Fails (STK_ERR_INVALID_ARG) if some coupling has no task.
int build_cluster_level(const Ctx& c, const HostLevel& H, const Pattern& ep, const Pattern& cp, HostLevel& HC,
                        std::string& err) {
  const int d = c.d, s = ep.s, nb = ep.nb, nch = 1 << d;
  const int S2 = cp.s, NB2 = cp.nb;
  if (S2 != nch * s || NB2 != nch * nb) {
    err = "cluster pattern does not match the element pattern";
    return STK_ERR_INVALID_ARG;
  }
  HC = HostLevel();
  int64_t ne2 = 1;
  for (int k = 0; k < 3; ++k) {
    HC.n[k] = k < d ? H.n[k] / 2 : 1;
    HC.h[k] = k < d ? 2 * H.h[k] : 0;
    ne2 *= HC.n[k];
  }
  HC.ne = (int)ne2;
  HC.D.assign((size_t)ne2 * NB2 * NB2, 0.0);
  HC.C.assign((size_t)ne2 * cp.T * S2 * S2, 0.0);
  HC.nbr.assign((size_t)ne2 * cp.NO, -1);
  auto cluster_id = [&](const int* ci) -> int64_t {
    int64_t id = 0, stride = 1;
    for (int k = 0; k < d; ++k) {
      id += ci[k] * stride;
      stride *= HC.n[k];
    }
    return id;
  };
  for (int64_t C = 0; C < ne2; ++C) {
    int ci[3];
    element_index(HC.n, d, C, ci);
    for (int o = 0; o < cp.NO; ++o) {
      int cj[3];
      bool ok = true;
      for (int k = 0; k < d; ++k) {
        cj[k] = ci[k] + cp.off[o][k];
        if (cj[k] < 0 || cj[k] >= HC.n[k]) {
          if (c.bc[2 * k] == STK_BC_PERIODIC)
            cj[k] = (cj[k] + HC.n[k]) % HC.n[k];
          else
            ok = false;
        }
      }
      if (ok) HC.nbr[(size_t)C * cp.NO + o] = (int)cluster_id(cj);
    }
  }
  auto floordiv2 = [](int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); };
  for (int64_t e = 0; e < H.ne; ++e) {
    int ie[3];
    element_index(H.n, d, e, ie);
    int ci[3] = {0, 0, 0}, ch = 0;
    for (int k = 0; k < d; ++k) {
      ci[k] = ie[k] / 2;
      ch |= (ie[k] & 1) << k;
    }
    const int64_t C = cluster_id(ci);
    double* DC = &HC.D[(size_t)C * NB2 * NB2];
    const double* De = &H.D[(size_t)e * nb * nb];
    for (int rv = 0; rv <= d; ++rv)
      for (int cv = 0; cv <= d; ++cv)
        for (int a = 0; a < s; ++a)
          for (int b2 = 0; b2 < s; ++b2)
            DC[(size_t)(rv * S2 + ch * s + a) * NB2 + cv * S2 + ch * s + b2] += De[(size_t)(rv * s + a) * nb + cv * s + b2];
    for (int t = 0; t < ep.T; ++t) {
      const int slot = ep.task_o[t];
      const int64_t e2 = H.nbr[(size_t)e * ep.NO + slot];
      if (e2 < 0) continue;
      const int rv = ep.task_rv[t], cv = ep.task_cv[t];
      int ie2[3], co[3] = {0, 0, 0}, ch2 = 0;
      element_index(H.n, d, e2, ie2);
      bool same = true;
      for (int k = 0; k < d; ++k) {
        co[k] = floordiv2(ie[k] + ep.off[slot][k]) - ie[k] / 2;   // geometric cluster offset
        ch2 |= (ie2[k] & 1) << k;
        if (co[k] != 0) same = false;
      }
      const double* blk = &H.C[((size_t)e * ep.T + t) * s * s];
      if (same) {
        for (int a = 0; a < s; ++a)
          for (int b2 = 0; b2 < s; ++b2)
            DC[(size_t)(rv * S2 + ch * s + a) * NB2 + cv * S2 + ch2 * s + b2] += blk[a * s + b2];
        continue;
      }
      int o2 = -1;
      for (int o = 0; o < cp.NO; ++o)
        if (cp.off[o][0] == co[0] && cp.off[o][1] == co[1] && cp.off[o][2] == co[2]) o2 = o;
      int t2 = -1;
      for (int u = 0; u < cp.T && o2 >= 0; ++u)
        if (cp.task_rv[u] == rv && cp.task_cv[u] == cv && cp.task_o[u] == o2) t2 = u;
      if (t2 < 0) {
        err = "a coupling between clusters has no task in the cluster pattern";
        return STK_ERR_INVALID_ARG;
      }
      double* CC = &HC.C[((size_t)C * cp.T + t2) * S2 * S2];
      for (int a = 0; a < s; ++a)
        for (int b2 = 0; b2 < s; ++b2) CC[(size_t)(ch * s + a) * S2 + ch2 * s + b2] += blk[a * s + b2];
    }
  }
  return STK_OK;
}

}  // namespace stk
