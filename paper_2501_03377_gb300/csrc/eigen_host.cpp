// Host-side eigenpairs of the 1D FD minus-Laplacians (plan setup, Algorithm 5).
//
// The eigenpairs come from the closed forms of Lemmas spectrumP, spectrumD,
// spectrumN and spectrumM (Sec. 3.2), normalised to orthonormal columns so
// that L = V Lambda V^T (eq. eig-svd-decomp).  Every trigonometric argument is
// a rational multiple of pi whose numerator is reduced exactly in integer
// arithmetic before the (long double) sin/cos, and eigenvalues are evaluated
// as 4 sin^2(x/2) instead of 2 - 2 cos(x) to keep small eigenvalues accurate.
// The result is checked against the assembled L_l (footnote to eq.
// eig-svd-decomp: an eigenbasis is judged by ||L - V Lambda V^T||_F).
#include "tpcg_internal.h"

#include <cmath>
#include <vector>

namespace tpcg {

namespace {

// sin(pi * num / den) and cos(pi * num / den) with num reduced mod 2*den.
long double sinpi_frac(long long num, long long den) {
  long long m = num % (2 * den);
  if (m < 0) m += 2 * den;
  return sinl(3.141592653589793238462643383279502884L * (long double)m / (long double)den);
}
long double cospi_frac(long long num, long long den) {
  long long m = num % (2 * den);
  if (m < 0) m += 2 * den;
  return cosl(3.141592653589793238462643383279502884L * (long double)m / (long double)den);
}
// 4 sin^2(pi * num / (2 den)) = 2 - 2 cos(pi num / den)
double lam_from_frac(long long num, long long den) {
  long double s = sinpi_frac(num, 2 * den);
  return (double)(4.0L * s * s);
}

}  // namespace

// Dense L_n(alpha, beta, gamma) of eq. (lap1d), unit spacing, row-major.
std::vector<double> lap1d_dense(int n, int bc) {
  std::vector<double> L((size_t)n * n, 0.0);
  double alpha = 2, beta = 2, gamma = 0;
  switch (bc) {
    case kBcP: alpha = 2; beta = 2; gamma = -1; break;
    case kBcD: alpha = 2; beta = 2; gamma = 0; break;
    case kBcN: alpha = 1; beta = 1; gamma = 0; break;
    case kBcDN: alpha = 2; beta = 1; gamma = 0; break;
    case kBcND: alpha = 1; beta = 2; gamma = 0; break;
  }
  for (int i = 0; i < n; ++i) {
    L[(size_t)i * n + i] = 2.0;
    if (i > 0) L[(size_t)i * n + i - 1] = -1.0;
    if (i + 1 < n) L[(size_t)i * n + i + 1] = -1.0;
  }
  L[0] = alpha;
  L[(size_t)(n - 1) * n + (n - 1)] = beta;
  L[(size_t)(n - 1)] += gamma;
  L[(size_t)(n - 1) * n] += gamma;
  return L;
}

// Fills lam[k] and V[j*n + k] (row j, column k) with orthonormal eigenpairs of
// L_n for unit spacing.  Column 0 is the constant vector for P and N (the
// null space), so the null index of the Kronecker sum is (0, 0, 0).
void closed_form_eigenpairs(int n, int bc, std::vector<double>& lam, std::vector<double>& V) {
  lam.assign(n, 0.0);
  V.assign((size_t)n * n, 0.0);
  auto set = [&](int j, int k, long double v) { V[(size_t)j * n + k] = (double)v; };
  if (bc == kBcP) {
    // Lemma spectrumP: 1; cos(2 j k pi / n), sin(2 j k pi / n) for k = 1..l-1;
    // alternating vector when n is even.  Norms^2: n, n/2, n/2, n.
    const long double c0 = 1.0L / sqrtl((long double)n), c1 = sqrtl(2.0L / (long double)n);
    int col = 0;
    lam[col] = 0.0;
    for (int j = 0; j < n; ++j) set(j, col, c0);
    ++col;
    const int ell = (n % 2) ? (n + 1) / 2 : n / 2;
    for (int k = 1; k < ell; ++k) {
      const double lk = lam_from_frac(2LL * k, n);
      lam[col] = lk;
      lam[col + 1] = lk;
      for (int j = 0; j < n; ++j) {
        const long long num = 2LL * (j + 1) * k;  // rows j = 1..n of the lemma
        set(j, col, c1 * cospi_frac(num, n));
        set(j, col + 1, c1 * sinpi_frac(num, n));
      }
      col += 2;
    }
    if (n % 2 == 0) {
      lam[col] = 4.0;
      for (int j = 0; j < n; ++j) set(j, col, ((j % 2) ? -c0 : c0));
      ++col;
    }
  } else if (bc == kBcD) {
    // Lemma spectrumD: sin(j k pi / (n+1)), norm^2 (n+1)/2.
    const long double c = sqrtl(2.0L / (long double)(n + 1));
    for (int k = 1; k <= n; ++k) {
      lam[k - 1] = lam_from_frac(k, n + 1);
      for (int j = 1; j <= n; ++j) set(j - 1, k - 1, c * sinpi_frac((long long)j * k, n + 1));
    }
  } else if (bc == kBcN) {
    // Lemma spectrumN: cos((j - 1/2)(k - 1) pi / n) = cos((2j-1)(k-1) pi / (2n)),
    // norm^2 n for k = 1 and n/2 otherwise.
    for (int k = 1; k <= n; ++k) {
      lam[k - 1] = lam_from_frac(k - 1, n);
      const long double c = (k == 1) ? 1.0L / sqrtl((long double)n) : sqrtl(2.0L / (long double)n);
      for (int j = 1; j <= n; ++j) set(j - 1, k - 1, c * cospi_frac((long long)(2 * j - 1) * (k - 1), 2LL * n));
    }
  } else {
    // Lemma spectrumM: theta_k = (2k-1) pi / (2n+1).  DN: sin(j theta_k) (the
    // factor (-1)^k of the lemma is a sign); ND: cos((j - 1/2) theta_k).
    // Norm^2 (2n+1)/4 for both.
    const long double c = 2.0L / sqrtl((long double)(2 * n + 1));
    for (int k = 1; k <= n; ++k) {
      lam[k - 1] = lam_from_frac(2 * k - 1, 2 * n + 1);
      for (int j = 1; j <= n; ++j) {
        if (bc == kBcDN)
          set(j - 1, k - 1, c * sinpi_frac((long long)j * (2 * k - 1), 2LL * n + 1));
        else
          set(j - 1, k - 1, c * cospi_frac((long long)(2 * j - 1) * (2 * k - 1), 2LL * (2 * n + 1)));
      }
    }
  }
}

// max |V^T V - I| and ||L - V Lambda V^T||_F for unit spacing.
void eigen_check(int n, int bc, const std::vector<double>& lam, const std::vector<double>& V, double* orth_err,
                 double* recon_err) {
  const std::vector<double> L = lap1d_dense(n, bc);
  double oe = 0.0, re2 = 0.0;
  // FP64 accumulation (long double is software quad precision on some hosts);
  // the acceptance bounds below leave ample room for its rounding.
  std::vector<double> VT((size_t)n * n), VL((size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      VT[(size_t)k * n + j] = V[(size_t)j * n + k];
      VL[(size_t)j * n + k] = V[(size_t)j * n + k] * lam[k];
    }
  for (int a = 0; a < n; ++a) {
    const double* va = &VT[(size_t)a * n];
    const double* la = &VL[(size_t)a * n];
    for (int b = 0; b < n; ++b) {
      const double* vb = &VT[(size_t)b * n];
      const double* rb = &V[(size_t)b * n];
      double g = 0.0, r = 0.0;
      for (int j = 0; j < n; ++j) g += va[j] * vb[j];
      for (int k = 0; k < n; ++k) r += la[k] * rb[k];
      const double ge = fabs(g - (a == b ? 1.0 : 0.0));
      if (ge > oe) oe = ge;
      const double d = L[(size_t)a * n + b] - r;
      re2 += d * d;
    }
  }
  *orth_err = oe;
  *recon_err = sqrt(re2);
}

int build_axis(int len, int bc, double h, AxisBasis& ax) {
  ax.len = len;
  ax.bc = bc;
  ax.h = h;
  if (len == 1) {  // absent axis of a 2D problem: L = [0], V = [1]
    ax.lam.assign(1, 0.0);
    ax.V.assign(1, 1.0);
    ax.orth_err = ax.recon_err = 0.0;
    return 0;
  }
  std::vector<double> lam, V;
  closed_form_eigenpairs(len, bc, lam, V);
  eigen_check(len, bc, lam, V, &ax.orth_err, &ax.recon_err);
  // acceptance bounds: a few ulps per accumulated term
  if (!(ax.orth_err <= 1e-14 * len) || !(ax.recon_err <= 1e-13 * len)) return -1;
  const double ih2 = 1.0 / (h * h);
  ax.lam.resize(len);
  for (int k = 0; k < len; ++k) ax.lam[k] = lam[k] * ih2;
  ax.V = V;
  return 0;
}

}  // namespace tpcg
