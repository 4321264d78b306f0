// Host-side tableau and A0^{-1} transform (step a1 of the hot path).
//
// Families (Sec. 1.1, Eq. update/stages; Table 1 lists all three):
//   Gauss        abscissae = roots of P_s mapped to [0,1] (collocation, order 2s)
//   Radau IIA    roots of P_s - P_{s-1}, right end point c_s = 1 (collocation, order 2s-1)
//   Lobatto IIIC roots of P_s - P_{s-2}, both end points (order 2s-2, s >= 2)
// b follows from sum_j b_j c_j^q = 1/(q+1), q = 0..s-1.  Collocation rows
// satisfy sum_j a_ij c_j^q = c_i^{q+1}/(q+1), q = 0..s-1; Lobatto IIIC rows
// instead take a_i1 = b_1 and the same conditions for q = 0..s-2.
//
// Real Schur form (Sec. 3.1): A0^{-1} = Q0 R0 Q0^T, Q0 orthogonal, R0 block
// upper triangular with 1x1 blocks for real eigenvalues and standardized 2x2
// blocks [[eta, phi], [-beta^2/phi, eta]] for pairs eta +- i beta.  It is
// built by deflation: the eigenvalues are the roots of the characteristic
// polynomial; each real eigenvector (or the real span of a complex one) is
// completed to an orthonormal basis that splits off its block, and each 2x2
// block is finally rotated to equal diagonals by the smallest Givens angle.
// gamma* = eta + beta^2/eta (Eq. gamma*).
//
// Eigenvector basis (basis = 1): A0^{-1} = T R T^{-1} with T the real and
// imaginary parts of the eigenvectors and R block diagonal, [[eta, beta],
// [-beta, eta]] per pair (the phi = beta case of the standardized block).
// Algorithm 1 then needs T^{-1} in place of Q0^T and has no R0 coupling.
//
// SDIRK (the diagonally implicit methods of the comparisons in Sec. 7):
// lower triangular A with one diagonal value gamma, stiffly accurate (b =
// last row), L-stable: s = 1 backward Euler, s = 2 gamma = 1 - sqrt(1/2),
// s = 3 Alexander's method (c_2 = (1 + gamma)/2, b from B(3), gamma from the
// remaining order-3 condition), s = 5 the order-4 method of Hairer and
// Wanner (gamma = 1/4).  A0^{-1} is lower triangular with the one eigenvalue
// 1/gamma (not diagonalizable for s > 1), so its real Schur form is exact:
// Q0 = the reversal permutation J, R0 = J A0^{-1} J upper triangular, every
// block 1x1 with eta = 1/gamma, and every off-diagonal d-vector is zero.
// Everything runs in long double.
#include "irk_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

namespace irk {

typedef long double ld;
typedef std::complex<ld> cld;

static void legendre_roots(int s, ld* x) {
  for (int k = 0; k < s; ++k) {
    ld r = std::cos(3.14159265358979323846264338327950288L * (k + 0.75L) / (s + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1, p1 = r;
      for (int q = 1; q < s; ++q) {
        ld p2 = ((2 * q + 1) * r * p1 - q * p0) / (q + 1);
        p0 = p1;
        p1 = p2;
      }
      ld ps = p1, psm1 = p0;  // P_s(r), P_{s-1}(r)
      ld dp = s * (r * ps - psm1) / (r * r - 1);
      ld step = ps / dp;
      r -= step;
      if (std::fabs(step) < 1e-21L) break;
    }
    x[k] = r;
  }
}

// Solve M x = rhs (n x n, row-major) by Gaussian elimination with partial pivoting.
static bool solve_ld(int n, std::vector<ld> M, std::vector<ld>& rhs) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(M[r * n + col]) > std::fabs(M[piv * n + col])) piv = r;
    if (M[piv * n + col] == 0) return false;
    if (piv != col) {
      for (int k = 0; k < n; ++k) std::swap(M[piv * n + k], M[col * n + k]);
      std::swap(rhs[piv], rhs[col]);
    }
    for (int r = col + 1; r < n; ++r) {
      ld f = M[r * n + col] / M[col * n + col];
      for (int k = col; k < n; ++k) M[r * n + k] -= f * M[col * n + k];
      rhs[r] -= f * rhs[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    ld acc = rhs[r];
    for (int k = r + 1; k < n; ++k) acc -= M[r * n + k] * rhs[k];
    rhs[r] = acc / M[r * n + r];
  }
  return true;
}

static bool invert_ld(int n, const std::vector<ld>& A, std::vector<ld>& Ainv) {
  Ainv.assign(n * n, 0);
  for (int col = 0; col < n; ++col) {
    std::vector<ld> e(n, 0);
    e[col] = 1;
    if (!solve_ld(n, A, e)) return false;
    for (int r = 0; r < n; ++r) Ainv[r * n + col] = e[r];
  }
  return true;
}

// Characteristic polynomial coefficients p[0..n] (monic, p[n] = 1) by the
// Faddeev-LeVerrier recursion.
static void charpoly(int n, const std::vector<ld>& A, std::vector<ld>& p) {
  p.assign(n + 1, 0);
  p[n] = 1;
  std::vector<ld> Mk(n * n, 0), AM(n * n, 0);
  for (int k = 1; k <= n; ++k) {
    // Mk = A * M_{k-1} + p[n-k+1] I
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        ld acc = 0;
        for (int q = 0; q < n; ++q) acc += A[i * n + q] * Mk[q * n + j];
        AM[i * n + j] = acc;
      }
    for (int i = 0; i < n; ++i) AM[i * n + i] += p[n - k + 1];
    Mk = AM;
    ld tr = 0;
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < n; ++q) tr += A[i * n + q] * Mk[q * n + i];
    p[n - k] = -tr / k;
  }
}

static cld polyval(const std::vector<ld>& p, cld z) {
  cld acc = 0;
  for (int k = (int)p.size() - 1; k >= 0; --k) acc = acc * z + p[k];
  return acc;
}

static cld polyder(const std::vector<ld>& p, cld z) {
  cld acc = 0;
  for (int k = (int)p.size() - 1; k >= 1; --k) acc = acc * z + (ld)k * p[k];
  return acc;
}

// All roots of the monic polynomial p by Aberth-Ehrlich iteration.
static void poly_roots(const std::vector<ld>& p, std::vector<cld>& z) {
  int n = (int)p.size() - 1;
  ld rad = 0;
  for (int k = 0; k < n; ++k) rad = std::max(rad, std::pow(std::fabs(p[k]), 1.0L / (n - k)));
  rad = std::max(rad, (ld)1);
  z.resize(n);
  for (int k = 0; k < n; ++k)
    z[k] = std::polar(rad, (ld)(2 * 3.14159265358979323846264338327950288L * k / n + 0.4L));
  for (int it = 0; it < 500; ++it) {
    ld maxstep = 0;
    for (int k = 0; k < n; ++k) {
      cld ratio = polyval(p, z[k]) / polyder(p, z[k]);
      cld sum = 0;
      for (int j = 0; j < n; ++j)
        if (j != k) sum += (ld)1 / (z[k] - z[j]);
      cld w = ratio / ((ld)1 - ratio * sum);
      z[k] -= w;
      maxstep = std::max(maxstep, std::abs(w) / std::max((ld)1, std::abs(z[k])));
    }
    if (maxstep < 1e-20L) break;
  }
  for (int k = 0; k < n; ++k)  // Newton polish
    for (int it = 0; it < 3; ++it) {
      cld d = polyder(p, z[k]);
      if (std::abs(d) > 0) z[k] -= polyval(p, z[k]) / d;
    }
}

// Legendre polynomial P_n in the monomial basis (coefficients of x^0..x^n),
// from (q+1) P_{q+1} = (2q+1) x P_q - q P_{q-1}.
static std::vector<ld> legendre_poly(int n) {
  std::vector<ld> pm(1, 1), pc = {0, 1};
  if (n == 0) return pm;
  for (int q = 1; q < n; ++q) {
    std::vector<ld> pn(q + 2, 0);
    for (int i = 0; i <= q; ++i) pn[i + 1] += (ld)(2 * q + 1) * pc[i] / (q + 1);
    for (int i = 0; i < (int)pm.size(); ++i) pn[i] -= (ld)q * pm[i] / (q + 1);
    pm = pc;
    pc = pn;
  }
  return pc;
}

// Abscissae in [0,1], increasing.
static bool family_nodes(int family, int s, std::vector<ld>& c) {
  c.assign(s, 0);
  if (family == IRK_GAUSS) {
    std::vector<ld> x(s);
    legendre_roots(s, x.data());
    for (int k = 0; k < s; ++k) c[k] = (1 + x[k]) / 2;
    std::sort(c.begin(), c.end());
    return true;
  }
  std::vector<ld> p = legendre_poly(s);
  const std::vector<ld> q = legendre_poly(family == IRK_RADAU_IIA ? s - 1 : s - 2);
  for (size_t i = 0; i < q.size(); ++i) p[i] -= q[i];
  const ld lead = p[s];
  for (auto& v : p) v /= lead;
  std::vector<cld> z;
  poly_roots(p, z);
  for (int k = 0; k < s; ++k) {
    ld x = z[k].real();
    if (std::fabs(z[k].imag()) > 1e-12L) return false;
    for (int it = 0; it < 5; ++it) {  // real Newton polish
      const ld d = polyder(p, cld(x, 0)).real();
      if (d != 0) x -= polyval(p, cld(x, 0)).real() / d;
    }
    if (std::fabs(x - 1) < 1e-15L) x = 1;   // the end points are exact roots
    if (std::fabs(x + 1) < 1e-15L) x = -1;
    c[k] = (1 + x) / 2;
  }
  std::sort(c.begin(), c.end());
  return true;
}

// A null vector of the (nearly singular) m x m complex matrix B by Gaussian
// elimination with complete pivoting.
static void null_vector(int m, std::vector<cld> B, std::vector<cld>& x) {
  std::vector<int> colperm(m);
  for (int k = 0; k < m; ++k) colperm[k] = k;
  for (int k = 0; k < m - 1; ++k) {
    int pr = k, pc = k;
    ld best = -1;
    for (int r = k; r < m; ++r)
      for (int c = k; c < m; ++c)
        if (std::abs(B[r * m + c]) > best) { best = std::abs(B[r * m + c]); pr = r; pc = c; }
    for (int c = 0; c < m; ++c) std::swap(B[k * m + c], B[pr * m + c]);
    for (int r = 0; r < m; ++r) std::swap(B[r * m + k], B[r * m + pc]);
    std::swap(colperm[k], colperm[pc]);
    for (int r = k + 1; r < m; ++r) {
      cld f = B[r * m + k] / B[k * m + k];
      for (int c = k; c < m; ++c) B[r * m + c] -= f * B[k * m + c];
    }
  }
  std::vector<cld> y(m);
  y[m - 1] = 1;
  for (int r = m - 2; r >= 0; --r) {
    cld acc = 0;
    for (int c = r + 1; c < m; ++c) acc += B[r * m + c] * y[c];
    y[r] = -acc / B[r * m + r];
  }
  x.assign(m, 0);
  for (int k = 0; k < m; ++k) x[colperm[k]] = y[k];
}

// Orthonormal completion: H (m x m, row-major) whose first k columns span U.
static void complete_basis(int m, int k, const std::vector<ld>& U, std::vector<ld>& H) {
  std::vector<std::vector<ld>> cols;
  auto add = [&](std::vector<ld> v) {
    for (int pass = 0; pass < 2; ++pass)
      for (auto& q : cols) {
        ld d = 0;
        for (int i = 0; i < m; ++i) d += q[i] * v[i];
        for (int i = 0; i < m; ++i) v[i] -= d * q[i];
      }
    ld nr = 0;
    for (int i = 0; i < m; ++i) nr += v[i] * v[i];
    nr = std::sqrt(nr);
    if (nr < 1e-8L) return false;
    for (int i = 0; i < m; ++i) v[i] /= nr;
    cols.push_back(v);
    return true;
  };
  for (int j = 0; j < k; ++j) {
    std::vector<ld> v(m);
    for (int i = 0; i < m; ++i) v[i] = U[i * k + j];
    add(v);
  }
  for (int e = 0; e < m && (int)cols.size() < m; ++e) {
    // add the unit vector with the largest residual first for robustness
    int best = -1;
    ld bestnr = -1;
    for (int cand = 0; cand < m; ++cand) {
      std::vector<ld> v(m, 0);
      v[cand] = 1;
      for (auto& q : cols) {
        ld d = q[cand];
        for (int i = 0; i < m; ++i) v[i] -= d * q[i];
      }
      ld nr = 0;
      for (int i = 0; i < m; ++i) nr += v[i] * v[i];
      if (nr > bestnr) { bestnr = nr; best = cand; }
    }
    std::vector<ld> v(m, 0);
    v[best] = 1;
    add(v);
  }
  H.assign(m * m, 0);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) H[i * m + j] = cols[j][i];
}

// R <- G^T R G and Q <- Q G for G the identity except rows/cols [off, off+m)
// replaced by the m x m orthogonal H.
static void apply_similarity(int s, int off, int m, const std::vector<ld>& H,
                             std::vector<ld>& R, std::vector<ld>& Q) {
  std::vector<ld> T(s * s);
  // R G
  T = R;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < m; ++j) {
      ld acc = 0;
      for (int q = 0; q < m; ++q) acc += R[i * s + off + q] * H[q * m + j];
      T[i * s + off + j] = acc;
    }
  R = T;
  // G^T (R G)
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < s; ++j) {
      ld acc = 0;
      for (int q = 0; q < m; ++q) acc += H[q * m + i] * R[(off + q) * s + j];
      T[(off + i) * s + j] = acc;
    }
  R = T;
  std::vector<ld> QT = Q;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < m; ++j) {
      ld acc = 0;
      for (int q = 0; q < m; ++q) acc += Q[i * s + off + q] * H[q * m + j];
      QT[i * s + off + j] = acc;
    }
  Q = QT;
}

struct EigGroup {
  cld lam;   // eigenvalue of A0^{-1}; imag >= 0 represents a conjugate pair
  int size;  // 1 (real) or 2 (pair)
};

// Real eigenvector basis: column(s) of T per group in order, R block diagonal.
// A pair eta + i beta with eigenvector z = x + i y gives A0^{-1} [x y] =
// [x y] [[eta, beta], [-beta, eta]]; z is rotated so that x is orthogonal to
// y with |x| >= |y|, scaled to |z|^2 = 2 (unit norm for a real vector), and
// signed so that the largest entry of x is positive.
static bool eigen_basis(int s, const std::vector<ld>& Ainv, const std::vector<EigGroup>& groups,
                        HostTableau* t, std::vector<ld>& T, std::vector<ld>& R, char* err,
                        size_t errlen) {
  T.assign(s * s, 0);
  R.assign(s * s, 0);
  int off = 0, nb = 0;
  for (const EigGroup& g : groups) {
    std::vector<cld> B(s * s);
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) B[i * s + j] = Ainv[i * s + j];
    for (int i = 0; i < s; ++i) B[i * s + i] -= g.lam;
    std::vector<cld> z;
    null_vector(s, B, z);
    if (g.size == 1) {
      int big = 0;
      for (int i = 1; i < s; ++i)
        if (std::abs(z[i]) > std::abs(z[big])) big = i;
      const cld ph = std::conj(z[big]) / std::abs(z[big]);
      ld nr = 0;
      for (auto& v : z) { v *= ph; nr += v.real() * v.real(); }
      nr = std::sqrt(nr);
      for (int i = 0; i < s; ++i) T[i * s + off] = z[i].real() / nr;
      R[off * s + off] = g.lam.real();
    } else {
      ld xx = 0, yy = 0, xy = 0;
      for (auto& v : z) { xx += v.real() * v.real(); yy += v.imag() * v.imag(); xy += v.real() * v.imag(); }
      const ld th = 0.5L * std::atan2(-2 * xy, xx - yy);
      const cld rot = std::polar((ld)1, th);
      ld nr = 0;
      for (auto& v : z) { v *= rot; nr += std::norm(v); }
      const ld scale = std::sqrt(2 / nr);
      int big = 0;
      for (int i = 1; i < s; ++i)
        if (std::fabs(z[i].real()) > std::fabs(z[big].real())) big = i;
      const ld sg = (z[big].real() < 0) ? -scale : scale;
      for (int i = 0; i < s; ++i) {
        T[i * s + off] = z[i].real() * sg;
        T[i * s + off + 1] = z[i].imag() * sg;
      }
      const ld eta = g.lam.real(), beta = g.lam.imag();
      R[off * s + off] = R[(off + 1) * s + off + 1] = eta;
      R[off * s + off + 1] = beta;
      R[(off + 1) * s + off] = -beta;
    }
    t->bstart[nb] = off;
    t->bsize[nb] = g.size;
    t->eta[nb] = (double)g.lam.real();
    const ld beta2 = g.size == 2 ? g.lam.imag() * g.lam.imag() : 0;
    t->beta2[nb] = (double)beta2;
    t->gamma_star[nb] = (double)(g.lam.real() + beta2 / g.lam.real());
    ++nb;
    off += g.size;
  }
  t->nblk = nb;
  if (off != s) { snprintf(err, errlen, "eigenvalue groups do not cover the stages"); return false; }
  return true;
}

// A of the SDIRK method with s stages (row-major); false for other s.
static bool sdirk_matrix(int s, std::vector<ld>& A) {
  A.assign(s * s, 0);
  if (s == 1) {
    A[0] = 1;
    return true;
  }
  if (s == 2) {
    // stiffly accurate: b = (1 - g, g), c = (g, 1); order 2 needs b.c = 1/2,
    // i.e. g^2 - 2g + 1/2 = 0, and the root below 1 is L-stable
    const ld g = 1 - std::sqrt((ld)0.5);
    A[0] = g;
    A[2] = 1 - g;
    A[3] = g;
    return true;
  }
  if (s == 3) {
    // c = (g, (1 + g)/2, 1); b solves sum_j b_j c_j^q = 1/(q+1), q = 0..2;
    // g is the root in (0.3, 0.5) of b^T A c = 1/6 (bisection)
    auto fill = [&](ld g, std::vector<ld>& M) -> bool {
      const ld c2 = (1 + g) / 2;
      std::vector<ld> V = {1, 1, 1, g, c2, 1, g * g, c2 * c2, 1};
      std::vector<ld> b = {1, (ld)0.5, (ld)1 / 3};
      if (!solve_ld(3, V, b)) return false;
      M.assign(9, 0);
      M[0] = g;
      M[3] = c2 - g;
      M[4] = g;
      M[6] = b[0];
      M[7] = b[1];
      M[8] = g;
      return true;
    };
    auto cond = [&](ld g) -> ld {
      std::vector<ld> M;
      if (!fill(g, M)) return 0;
      const ld c[3] = {g, (1 + g) / 2, 1};
      ld acc = 0;
      for (int i = 0; i < 3; ++i) {
        ld ac = 0;
        for (int j = 0; j < 3; ++j) ac += M[i * 3 + j] * c[j];
        acc += M[6 + i] * ac;
      }
      return acc - (ld)1 / 6;
    };
    ld lo = (ld)0.3, hi = (ld)0.5;
    const bool neg_lo = cond(lo) < 0;
    for (int it = 0; it < 200; ++it) {
      const ld mid = (lo + hi) / 2;
      if ((cond(mid) < 0) == neg_lo) lo = mid; else hi = mid;
    }
    return fill((lo + hi) / 2, A);
  }
  if (s == 5) {
    static const ld tab[5][5] = {
        {(ld)1 / 4, 0, 0, 0, 0},
        {(ld)1 / 2, (ld)1 / 4, 0, 0, 0},
        {(ld)17 / 50, (ld)-1 / 25, (ld)1 / 4, 0, 0},
        {(ld)371 / 1360, (ld)-137 / 2720, (ld)15 / 544, (ld)1 / 4, 0},
        {(ld)25 / 24, (ld)-49 / 48, (ld)125 / 16, (ld)-85 / 12, (ld)1 / 4}};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) A[i * 5 + j] = tab[i][j];
    return true;
  }
  return false;
}

// Store A, b, c, A0^{-1}, T, T^{-1}, R and T R; false (with err) when the
// factorization does not reproduce A0^{-1}.
static bool store_tableau(int s, const std::vector<ld>& A, const std::vector<ld>& b,
                          const std::vector<ld>& c, const std::vector<ld>& Ainv,
                          const std::vector<ld>& Q, const std::vector<ld>& R,
                          const std::vector<ld>& Qinv, HostTableau* t, char* err, size_t errlen) {
  ld errmax = 0;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      ld acc = 0;
      for (int a = 0; a < s; ++a)
        for (int bb = 0; bb < s; ++bb) acc += Q[i * s + a] * R[a * s + bb] * Qinv[bb * s + j];
      errmax = std::max(errmax, std::fabs(acc - Ainv[i * s + j]));
    }
  if (errmax > 1e-12L) { snprintf(err, errlen, "A0^{-1} reconstruction error %.3Le", errmax); return false; }
  for (int i = 0; i < s; ++i) {
    t->b[i] = (double)b[i];
    t->c[i] = (double)c[i];
    for (int j = 0; j < s; ++j) {
      t->A[i * s + j] = (double)A[i * s + j];
      t->Ainv[i * s + j] = (double)Ainv[i * s + j];
      t->T[i * s + j] = (double)Q[i * s + j];
      t->Tinv[i * s + j] = (double)Qinv[i * s + j];
      t->R[i * s + j] = (double)R[i * s + j];
    }
  }
  // T R, the back-transform of Algorithm 1 (Q0 R0 in the Schur basis)
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      ld acc = 0;
      for (int a = 0; a < s; ++a) acc += Q[i * s + a] * R[a * s + j];
      t->TR[i * s + j] = (double)acc;
    }
  return true;
}

static int build_sdirk(int s, int basis, HostTableau* t, char* err, size_t errlen) {
  std::vector<ld> A;
  if (!sdirk_matrix(s, A)) { snprintf(err, errlen, "SDIRK stages must be 1, 2, 3 or 5"); return 1; }
  if (basis == 1 && s > 1) {
    snprintf(err, errlen, "SDIRK's A0^{-1} has one repeated eigenvalue and no eigenvector basis; use the Schur basis");
    return 1;
  }
  std::vector<ld> b(s), c(s, 0), Ainv;
  for (int i = 0; i < s; ++i) {
    b[i] = A[(s - 1) * s + i];
    for (int j = 0; j < s; ++j) c[i] += A[i * s + j];
  }
  if (!invert_ld(s, A, Ainv)) { snprintf(err, errlen, "A0 is singular"); return 1; }
  std::vector<ld> Q(s * s, 0), R(s * s, 0);
  for (int i = 0; i < s; ++i) Q[i * s + (s - 1 - i)] = 1;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) R[i * s + j] = (i <= j) ? Ainv[(s - 1 - i) * s + (s - 1 - j)] : 0;
  t->nblk = s;
  for (int k = 0; k < s; ++k) {
    t->bstart[k] = k;
    t->bsize[k] = 1;
    t->eta[k] = (double)R[k * s + k];
    t->beta2[k] = 0;
    t->gamma_star[k] = t->eta[k];
  }
  return store_tableau(s, A, b, c, Ainv, Q, R, Q, t, err, errlen) ? 0 : 1;
}

int build_tableau_single(double gamma, HostTableau* t) {
  if (!(gamma > 0)) return 1;
  memset(t, 0, sizeof(*t));
  t->s = 1;
  t->A[0] = gamma;
  t->b[0] = 1;
  t->c[0] = 0;
  t->Ainv[0] = 1 / (ld)gamma;
  t->T[0] = t->Tinv[0] = 1;
  t->R[0] = t->TR[0] = t->Ainv[0];
  t->nblk = 1;
  t->bstart[0] = 0;
  t->bsize[0] = 1;
  t->eta[0] = t->gamma_star[0] = t->R[0];
  t->beta2[0] = 0;
  return 0;
}

int build_tableau(int family, int s, int basis, HostTableau* t, char* err, size_t errlen) {
  if (family != IRK_GAUSS && family != IRK_RADAU_IIA && family != IRK_LOBATTO_IIIC &&
      family != IRK_SDIRK) {
    snprintf(err, errlen, "unknown family %d", family);
    return 1;
  }
  if (basis != 0 && basis != 1) { snprintf(err, errlen, "basis must be 0 (Schur) or 1 (eigenvectors)"); return 1; }
  if (s < 1 || s > IRK_MAXS) { snprintf(err, errlen, "stages must be 1..%d", IRK_MAXS); return 1; }
  if (family == IRK_LOBATTO_IIIC && s < 2) { snprintf(err, errlen, "Lobatto IIIC needs s >= 2"); return 1; }
  memset(t, 0, sizeof(*t));
  t->s = s;
  if (family == IRK_SDIRK) return build_sdirk(s, basis, t, err, errlen);
  std::vector<ld> c;
  if (!family_nodes(family, s, c)) { snprintf(err, errlen, "abscissae not real"); return 1; }
  std::vector<ld> V(s * s);
  for (int q = 0; q < s; ++q)
    for (int j = 0; j < s; ++j) V[q * s + j] = std::pow(c[j], (ld)q);
  std::vector<ld> b(s);
  for (int q = 0; q < s; ++q) b[q] = (ld)1 / (q + 1);
  if (!solve_ld(s, V, b)) { snprintf(err, errlen, "singular collocation system"); return 1; }
  std::vector<ld> A(s * s);
  for (int i = 0; i < s; ++i) {
    std::vector<ld> r(s), W = V;
    for (int q = 0; q < s; ++q) r[q] = std::pow(c[i], (ld)(q + 1)) / (q + 1);
    if (family == IRK_LOBATTO_IIIC) {
      // a_i1 = b_1 replaces the condition of the highest power: rows [e_1; c^0..c^{s-2}]
      for (int q = s - 1; q >= 1; --q) {
        for (int j = 0; j < s; ++j) W[q * s + j] = V[(q - 1) * s + j];
        r[q] = r[q - 1];
      }
      for (int j = 0; j < s; ++j) W[j] = (j == 0) ? 1 : 0;
      r[0] = b[0];
    }
    if (!solve_ld(s, W, r)) { snprintf(err, errlen, "singular collocation system"); return 1; }
    for (int j = 0; j < s; ++j) A[i * s + j] = r[j];
  }
  std::vector<ld> Ainv;
  if (!invert_ld(s, A, Ainv)) { snprintf(err, errlen, "A0 is singular"); return 1; }

  // eigenvalues of A0^{-1}
  std::vector<ld> p;
  charpoly(s, Ainv, p);
  std::vector<cld> ev;
  poly_roots(p, ev);
  // groups: real eigenvalues and one representative (imag > 0) per pair
  std::vector<EigGroup> groups;
  std::vector<bool> used(s, false);
  for (int k = 0; k < s; ++k) {
    if (used[k]) continue;
    ld scale = std::max((ld)1, std::abs(ev[k]));
    if (std::fabs(ev[k].imag()) < 1e-9L * scale) {
      groups.push_back({cld(ev[k].real(), 0), 1});
      used[k] = true;
    } else {
      int partner = -1;
      for (int j = 0; j < s; ++j)
        if (!used[j] && j != k && std::abs(ev[j] - std::conj(ev[k])) < 1e-8L * scale) partner = j;
      if (partner < 0) { snprintf(err, errlen, "unpaired complex eigenvalue"); return 1; }
      used[k] = used[partner] = true;
      groups.push_back({cld(ev[k].real(), std::fabs(ev[k].imag())), 2});
    }
  }
  // deterministic order: increasing real part, then increasing |imag|
  std::sort(groups.begin(), groups.end(), [](const EigGroup& a, const EigGroup& b) {
    if (a.lam.real() != b.lam.real()) return a.lam.real() < b.lam.real();
    return a.lam.imag() < b.lam.imag();
  });
  for (auto& g : groups)
    if (g.lam.real() <= 0) { snprintf(err, errlen, "Assumption 1 violated: eigenvalue of A0^{-1} with non-positive real part"); return 1; }

  std::vector<ld> R, Q, Qinv;
  if (basis == 1) {
    if (!eigen_basis(s, Ainv, groups, t, Q, R, err, errlen)) return 1;
    if (!invert_ld(s, Q, Qinv)) { snprintf(err, errlen, "eigenvector basis is singular"); return 1; }
  } else {
    R = Ainv;
    Q.assign(s * s, 0);
    for (int k = 0; k < s; ++k) Q[k * s + k] = 1;
    int off = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
      int m = s - off, k = groups[g].size;
      if (m == k) { off += k; break; }
      std::vector<cld> B(m * m);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) B[i * m + j] = R[(off + i) * s + off + j];
      for (int i = 0; i < m; ++i) B[i * m + i] -= groups[g].lam;
      std::vector<cld> xv;
      null_vector(m, B, xv);
      // fix the global phase: make the largest component real
      int big = 0;
      for (int i = 1; i < m; ++i)
        if (std::abs(xv[i]) > std::abs(xv[big])) big = i;
      cld ph = std::conj(xv[big]) / std::abs(xv[big]);
      for (auto& v : xv) v *= ph;
      std::vector<ld> U(m * k);
      for (int i = 0; i < m; ++i) {
        U[i * k + 0] = xv[i].real();
        if (k == 2) U[i * k + 1] = xv[i].imag();
      }
      std::vector<ld> H;
      complete_basis(m, k, U, H);
      apply_similarity(s, off, m, H, R, Q);
      for (int i = off + k; i < s; ++i)
        for (int j = off; j < off + k; ++j) R[i * s + j] = 0;
      off += k;
    }
    // block structure and standardization of the 2x2 blocks
    int nb = 0;
    for (int k = 0; k < s;) {
      bool two = (k + 1 < s) && std::fabs(R[(k + 1) * s + k]) > 1e-12L * (1 + std::fabs(R[k * s + k]));
      if (two) {
        ld pp = R[k * s + k], qq = R[k * s + k + 1], rr = R[(k + 1) * s + k], tt = R[(k + 1) * s + k + 1];
        ld theta;
        if (std::fabs(qq + rr) > 1e-30L) theta = 0.5L * std::atan((pp - tt) / (qq + rr));
        else theta = (std::fabs(pp - tt) > 0) ? 0.78539816339744830961566084581987572L : 0;
        std::vector<ld> G = {std::cos(theta), std::sin(theta), -std::sin(theta), std::cos(theta)};
        std::vector<ld> R2 = R, Q2 = Q;
        apply_similarity(s, k, 2, G, R2, Q2);
        if (std::fabs(R2[k * s + k] - R2[(k + 1) * s + k + 1]) > 1e-14L * (1 + std::fabs(pp))) {
          G = {std::cos(-theta), std::sin(-theta), -std::sin(-theta), std::cos(-theta)};
          R2 = R; Q2 = Q;
          apply_similarity(s, k, 2, G, R2, Q2);
        }
        R = R2; Q = Q2;
        ld d = 0.5L * (R[k * s + k] + R[(k + 1) * s + k + 1]);
        R[k * s + k] = R[(k + 1) * s + k + 1] = d;
        t->bstart[nb] = k; t->bsize[nb] = 2;
        t->eta[nb] = (double)d;
        ld beta2 = -R[k * s + k + 1] * R[(k + 1) * s + k];
        if (beta2 <= 0) { snprintf(err, errlen, "2x2 Schur block without a complex pair"); return 1; }
        t->beta2[nb] = (double)beta2;
        t->gamma_star[nb] = (double)(d + beta2 / d);
        ++nb;
        k += 2;
      } else {
        t->bstart[nb] = k; t->bsize[nb] = 1;
        t->eta[nb] = (double)R[k * s + k];
        t->beta2[nb] = 0;
        t->gamma_star[nb] = t->eta[nb];
        ++nb;
        k += 1;
      }
    }
    t->nblk = nb;
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j)
        if (i > j) {
          // strictly below the block diagonal must vanish
          int bi = -1, bj = -1;
          for (int q = 0; q < nb; ++q) {
            if (i >= t->bstart[q] && i < t->bstart[q] + t->bsize[q]) bi = q;
            if (j >= t->bstart[q] && j < t->bstart[q] + t->bsize[q]) bj = q;
          }
          if (bi != bj) R[i * s + j] = 0;
        }
    Qinv.assign(s * s, 0);
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) Qinv[i * s + j] = Q[j * s + i];
  }
  t->collocation = (family == IRK_GAUSS || family == IRK_RADAU_IIA);
  // residual check T R T^{-1} == A0^{-1}, then store
  return store_tableau(s, A, b, c, Ainv, Q, R, Qinv, t, err, errlen) ? 0 : 1;
}

}  // namespace irk
