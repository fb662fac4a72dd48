// Column interpolative decomposition (ID) by Householder QR with column pivoting.
//
// The butterfly's low-rank factorizations (Sec. 2) are column IDs
//     A ~= A(:, J) [I | T~] P^T,   T~ = R11^{-1} R12,
// where A P = Q R is the column-pivoted QR (Businger-Golub: at step k the remaining column
// of largest norm is pivoted in, ties to the lowest position) stopped at the first k with
// |R_kk| <= eps |R_11|.  The paper leaves the factorization type free; this is the reading
// used throughout the library.
#include <cmath>
#include <complex>
#include <numeric>

#include "internal.h"

namespace mht {
namespace {

// c_j -= beta (v^H c_j) v over rows [k, M), vectorized (the reduction order is free).
inline void reflect(const double* v, double* c, int64_t n, double beta) {
  double s = 0;
#pragma omp simd reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += v[i] * c[i];
  const double t = s * beta;
#pragma omp simd
  for (int64_t i = 0; i < n; ++i) c[i] -= t * v[i];
}
inline void reflect(const std::complex<double>* vz, std::complex<double>* cz, int64_t n, double beta) {
  const double* v = reinterpret_cast<const double*>(vz);
  double* c = reinterpret_cast<double*>(cz);
  double sr = 0, si = 0;  // conj(v) . c
#pragma omp simd reduction(+ : sr, si)
  for (int64_t i = 0; i < n; ++i) {
    sr += v[2 * i] * c[2 * i] + v[2 * i + 1] * c[2 * i + 1];
    si += v[2 * i] * c[2 * i + 1] - v[2 * i + 1] * c[2 * i];
  }
  const double tr = sr * beta, ti = si * beta;
#pragma omp simd
  for (int64_t i = 0; i < n; ++i) {
    const double vr = v[2 * i], vi = v[2 * i + 1];
    c[2 * i] -= tr * vr - ti * vi;
    c[2 * i + 1] -= tr * vi + ti * vr;
  }
}
inline double sumsq(const double* c, int64_t n) {
  double s = 0;
#pragma omp simd reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += c[i] * c[i];
  return s;
}
inline double sumsq(const std::complex<double>* c, int64_t n) {
  return sumsq(reinterpret_cast<const double*>(c), 2 * n);
}

inline double abs2(double x) { return x * x; }
inline double abs2(const std::complex<double>& x) { return std::norm(x); }

template <class S>
int qrcp_id(S* A, int64_t M, int64_t K, double eps, std::vector<int32_t>& perm,
            std::vector<double>& Tout) {
  constexpr int W = sizeof(S) / sizeof(double);
  perm.resize(K);
  std::iota(perm.begin(), perm.end(), 0);
  Tout.clear();
  if (M == 0 || K == 0) return 0;
  std::vector<double> nrm(K), nrm0(K);
  for (int64_t j = 0; j < K; ++j) {
    const double s = sumsq(A + j * M, M);
    if (!std::isfinite(s)) fail(MHT_ERR_NUMERIC, "non-finite entry in a block of Phi");
    nrm[j] = nrm0[j] = s;
  }
  const int64_t kmax = std::min(M, K);
  double r11 = 0;
  int64_t r = 0;
  for (int64_t k = 0; k < kmax; ++k) {
    int64_t p = k;
    for (int64_t j = k + 1; j < K; ++j)
      if (nrm[j] > nrm[p]) p = j;
    const double cn = std::sqrt(std::max(nrm[p], 0.0));
    if (k == 0) {
      r11 = cn;
      if (r11 == 0) break;
    }
    if (!(cn > eps * r11)) break;
    if (p != k) {
      std::swap_ranges(A + k * M, A + (k + 1) * M, A + p * M);
      std::swap(nrm[k], nrm[p]);
      std::swap(nrm0[k], nrm0[p]);
      std::swap(perm[k], perm[p]);
    }
    // Householder reflector H = I - beta v v^H zeroing A(k+1:M, k)
    S* col = A + k * M;
    const double sig = sumsq(col + k, M - k);
    const double alpha = std::sqrt(sig);
    S x0 = col[k];
    const double ax0 = std::sqrt(abs2(x0));
    S phase = (ax0 > 0) ? x0 / ax0 : S(1);
    S rkk = -phase * alpha;  // new diagonal entry R_kk
    S v0 = x0 - rkk;
    const double vnorm2 = sig - abs2(x0) + abs2(v0);
    if (vnorm2 > 0) {
      // v = [v0; col(k+1:M)], beta = 2 / (v^H v)
      const double beta = 2.0 / vnorm2;
      col[k] = v0;
      // one pass per trailing column: w = beta v^H c_j, c_j -= w v (column stays in cache)
      for (int64_t j = k + 1; j < K; ++j) reflect(col + k, A + j * M + k, M - k, beta);
    }
    col[k] = rkk;
    for (int64_t i = k + 1; i < M; ++i) col[i] = S(0);
    // downdate remaining column norms; recompute when cancellation is severe
    for (int64_t j = k + 1; j < K; ++j) {
      nrm[j] -= abs2(A[j * M + k]);
      if (nrm[j] < 1e-8 * nrm0[j]) nrm[j] = nrm0[j] = sumsq(A + j * M + k + 1, M - k - 1);
    }
    r = k + 1;
  }
  // T~ = R11^{-1} R12 by back substitution, stored row-major r x (K - r)
  const int64_t nc = K - r;
  Tout.assign(size_t(r * nc * W), 0.0);
  S* T = reinterpret_cast<S*>(Tout.data());
  for (int64_t j = 0; j < nc; ++j) {
    const S* c = A + (r + j) * M;
    for (int64_t i = r - 1; i >= 0; --i) {
      S s = c[i];
      for (int64_t q = i + 1; q < r; ++q) s -= A[q * M + i] * T[q * nc + j];
      T[i * nc + j] = s / A[i * M + i];
    }
  }
  for (double v : Tout)
    if (!std::isfinite(v)) fail(MHT_ERR_NUMERIC, "non-finite interpolation coefficient");
  return int(r);
}

}  // namespace

int interpolative_decomposition_real(double* A, int64_t M, int64_t K, double eps,
                                     std::vector<int32_t>& perm, std::vector<double>& T) {
  return qrcp_id<double>(A, M, K, eps, perm, T);
}

int interpolative_decomposition_complex(std::complex<double>* A, int64_t M, int64_t K,
                                        double eps, std::vector<int32_t>& perm,
                                        std::vector<double>& T) {
  return qrcp_id<std::complex<double>>(A, M, K, eps, perm, T);
}

}  // namespace mht
