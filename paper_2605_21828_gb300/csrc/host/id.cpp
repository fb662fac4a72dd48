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
#include <random>
#include <algorithm>

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

// ---------------------------------------------------------------------------------------
// Blocked column-pivoted QR with randomized block pivoting (HQRRP: Martinsson, Quintana-Orti,
// Heavner, van de Geijn, SIAM J. Sci. Comput. 2017; Duersch & Gu 2017), real FP64.
// A Gaussian sketch Y = G A (b + p rows) chooses b pivot columns at a time by an unblocked
// QRCP of the small sketch; the b columns are factored by Householder QR, the trailing
// matrix is updated with the compact WY form (GEMMs), and the sketch is downdated as
// Y2 <- Y2 - Y1 R11^{-1} R12.  Almost all flops are matrix-matrix products.  The rank is
// the first k with |R_kk| <= eps |R_11| (|R_11| = largest column norm, as in QRCP), or the
// point where every remaining column norm is below that threshold.
void gemm(bool transA, int m, int n, int k, double alpha, const double* A, int lda, const double* B, int ldb,
          double beta, double* C, int ldc);
void zgemm(bool conjTransA, int m, int n, int k, std::complex<double> alpha, const std::complex<double>* A, int lda,
           const std::complex<double>* B, int ldb, std::complex<double> beta, std::complex<double>* C, int ldc);

namespace {

// LAPACK-style elementary reflector: on exit x[0] = beta, x[1:] = v[1:], v[0] = 1.
double householder(double* x, int64_t n, double* beta) {
  if (n <= 0) { *beta = 0; return 0.0; }
  const double alpha = x[0];
  const double xn2 = n > 1 ? sumsq(x + 1, n - 1) : 0.0;
  if (xn2 == 0.0) { *beta = alpha; return 0.0; }
  const double nrm = std::sqrt(alpha * alpha + xn2);
  const double b = alpha >= 0 ? -nrm : nrm;
  const double tau = (b - alpha) / b;
  const double scale = 1.0 / (alpha - b);
  for (int64_t i = 1; i < n; ++i) x[i] *= scale;
  x[0] = b;
  *beta = b;
  return tau;
}

// Unblocked QRCP on the s x k sketch Y (column-major, ld s) for `steps` pivots; records the
// column swaps (position q <-> swaps[q]) so they can be replayed on A.
void sketch_pivots(std::vector<double>& Y, int s, int k, int steps, std::vector<int>& swaps) {
  std::vector<double> nr(k);
  for (int j = 0; j < k; ++j) nr[j] = sumsq(&Y[size_t(j) * s], s);
  swaps.assign(steps, 0);
  for (int q = 0; q < steps; ++q) {
    int p = q;
    for (int j = q + 1; j < k; ++j)
      if (nr[j] > nr[p]) p = j;
    swaps[q] = p;
    if (p != q) {
      std::swap_ranges(&Y[size_t(q) * s], &Y[size_t(q + 1) * s], &Y[size_t(p) * s]);
      std::swap(nr[q], nr[p]);
    }
    if (q >= s) continue;  // the sketch has no rows left to reflect
    double* col = &Y[size_t(q) * s];
    double beta;
    const double tau = householder(col + q, s - q, &beta);
    if (tau != 0.0) {
      const double v0 = col[q];
      col[q] = 1.0;
      for (int j = q + 1; j < k; ++j) reflect(col + q, &Y[size_t(j) * s + q], s - q, tau);
      col[q] = v0;
    }
    for (int j = q + 1; j < k; ++j) {
      const double a = Y[size_t(j) * s + q];
      nr[j] = std::max(0.0, nr[j] - a * a);
    }
  }
}

int qrcp_id_blocked(double* A, int64_t M, int64_t K, double eps, uint64_t seed, std::vector<int32_t>& perm,
                    std::vector<double>& Tout) {
  constexpr int b = 64, p = 8, s = b + p;
  perm.resize(K);
  std::iota(perm.begin(), perm.end(), 0);
  Tout.clear();
  double maxn = 0;
  for (int64_t j = 0; j < K; ++j) {
    const double v = sumsq(A + j * M, M);
    if (!std::isfinite(v)) fail(MHT_ERR_NUMERIC, "non-finite entry in a block of Phi");
    maxn = std::max(maxn, v);
  }
  if (maxn == 0.0) return 0;
  const double thr = eps * std::sqrt(maxn);  // eps |R_11|
  // sketch Y = G A with G Gaussian (s x M)
  std::vector<double> G(size_t(s) * M), Y(size_t(s) * K);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> N01;
  for (auto& g : G) g = N01(rng);
  gemm(false, s, int(K), int(M), 1.0, G.data(), s, A, int(M), 0.0, Y.data(), s);
  const int64_t kmax = std::min(M, K);
  int64_t r = kmax;
  std::vector<double> V, Tm, W, Ys, X;
  std::vector<int> swaps;
  for (int64_t j = 0; j < kmax; j += b) {
    const int bb = int(std::min<int64_t>(b, kmax - j));
    const int64_t M2 = M - j, K2 = K - j - bb;
    // a. pivots from the sketch of the remaining columns
    Ys.assign(Y.begin() + size_t(j) * s, Y.end());
    sketch_pivots(Ys, s, int(K - j), bb, swaps);
    for (int q = 0; q < bb; ++q) {
      const int64_t a = j + q, c = j + swaps[q];
      if (a == c) continue;
      std::swap_ranges(A + a * M, A + (a + 1) * M, A + c * M);
      std::swap_ranges(&Y[size_t(a) * s], &Y[size_t(a + 1) * s], &Y[size_t(c) * s]);
      std::swap(perm[a], perm[c]);
    }
    // b. Householder QR of the panel A(j:M, j:j+bb); V keeps the reflectors explicitly
    V.assign(size_t(M2) * bb, 0.0);
    std::vector<double> tau(bb, 0.0);
    int64_t rank_here = -1;
    for (int q = 0; q < bb; ++q) {
      double* col = A + (j + q) * M + j;  // rows j..M-1 of column j+q
      double beta;
      tau[q] = householder(col + q, M2 - q, &beta);
      if (rank_here < 0 && !(std::fabs(beta) > thr)) rank_here = j + q;
      double* v = &V[size_t(q) * M2];
      v[q] = 1.0;
      for (int64_t i = q + 1; i < M2; ++i) v[i] = col[i];
      for (int64_t i = q + 1; i < M2; ++i) col[i] = 0.0;
      if (tau[q] != 0.0)
        for (int c = q + 1; c < bb; ++c) reflect(v + q, A + (j + c) * M + j + q, M2 - q, tau[q]);
    }
    // c. compact WY: H_0 ... H_{bb-1} = I - V T V^T (T upper triangular)
    Tm.assign(size_t(bb) * bb, 0.0);
    for (int q = 0; q < bb; ++q) {
      Tm[size_t(q) * bb + q] = tau[q];
      if (q == 0 || tau[q] == 0.0) continue;
      std::vector<double> w(q, 0.0);  // w = -tau V(:, 0:q)^T v_q
      const double* vq = &V[size_t(q) * M2];
      for (int c = 0; c < q; ++c) {
        const double* vc = &V[size_t(c) * M2];
        double acc = 0;
#pragma omp simd reduction(+ : acc)
        for (int64_t i = q; i < M2; ++i) acc += vc[i] * vq[i];
        w[c] = -tau[q] * acc;
      }
      for (int a = 0; a < q; ++a) {  // T(0:q, q) = T(0:q, 0:q) w
        double acc = 0;
        for (int c = a; c < q; ++c) acc += Tm[size_t(c) * bb + a] * w[c];
        Tm[size_t(q) * bb + a] = acc;
      }
    }
    // d. trailing update A2 <- (I - V T V^T)^T A2 = A2 - V T^T (V^T A2)
    double* A2 = A + (j + bb) * M + j;
    if (K2 > 0) {
      W.assign(size_t(bb) * K2, 0.0);
      gemm(true, bb, int(K2), int(M2), 1.0, V.data(), int(M2), A2, int(M), 0.0, W.data(), bb);
      for (int64_t c = 0; c < K2; ++c) {  // W <- T^T W, in place from the bottom row up
        double* wc = &W[size_t(c) * bb];
        for (int a = bb - 1; a >= 0; --a) {
          double acc = 0;
          for (int q = 0; q <= a; ++q) acc += Tm[size_t(a) * bb + q] * wc[q];
          wc[a] = acc;
        }
      }
      gemm(false, int(M2), int(K2), bb, -1.0, V.data(), int(M2), W.data(), bb, 1.0, A2, int(M));
    }
    if (rank_here >= 0) { r = rank_here; break; }
    // e. stop when every remaining column is below the threshold
    double rem = 0;
    for (int64_t c = 0; c < K2; ++c) rem = std::max(rem, sumsq(A2 + c * M + bb, M2 - bb));
    if (K2 == 0 || std::sqrt(rem) <= thr || j + bb >= kmax) { r = std::min<int64_t>(j + bb, kmax); break; }
    // f. sketch downdate: Y2 <- Y2 - Y1 R11^{-1} R12
    X.assign(size_t(bb) * K2, 0.0);
    for (int64_t c = 0; c < K2; ++c) {
      double* xc = &X[size_t(c) * bb];
      for (int a = bb - 1; a >= 0; --a) {
        double acc = A2[c * M + a];
        for (int q = a + 1; q < bb; ++q) acc -= A[(j + q) * M + j + a] * xc[q];
        xc[a] = acc / A[(j + a) * M + j + a];
      }
    }
    gemm(false, s, int(K2), bb, -1.0, &Y[size_t(j) * s], s, X.data(), bb, 1.0, &Y[size_t(j + bb) * s], s);
  }
  // T~ = R11^{-1} R12 by blocked back substitution (column-major work array, row-major out)
  const int64_t nc = K - r;
  Tout.assign(size_t(r * nc), 0.0);
  if (r == 0 || nc == 0) return int(r);
  std::vector<double> Tc(size_t(r) * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t i = 0; i < r; ++i) Tc[size_t(c) * r + i] = A[(r + c) * M + i];
  constexpr int bs = 64;
  for (int64_t i1 = r; i1 > 0; i1 -= bs) {
    const int64_t i0 = std::max<int64_t>(0, i1 - bs), h = i1 - i0;
    if (i1 < r)  // Tc(i0:i1, :) -= R(i0:i1, i1:r) Tc(i1:r, :)
      gemm(false, int(h), int(nc), int(r - i1), -1.0, A + i1 * M + i0, int(M), &Tc[i1], int(r), 1.0, &Tc[i0], int(r));
    for (int64_t c = 0; c < nc; ++c) {
      double* tc = &Tc[size_t(c) * r];
      for (int64_t a = i1 - 1; a >= i0; --a) {
        double acc = tc[a];
        for (int64_t q = a + 1; q < i1; ++q) acc -= A[q * M + a] * tc[q];
        tc[a] = acc / A[a * M + a];
      }
    }
  }
  for (int64_t i = 0; i < r; ++i)
    for (int64_t c = 0; c < nc; ++c) Tout[size_t(i) * nc + c] = Tc[size_t(c) * r + i];
  for (double v : Tout)
    if (!std::isfinite(v)) fail(MHT_ERR_NUMERIC, "non-finite interpolation coefficient");
  return int(r);
}

}  // namespace

// Full-rank certificate for very tall blocks (M >= 16K): the Gram matrix A^T A by one GEMM and a
// diagonally pivoted Cholesky factorization.  Its pivots are the squared diagonal of the
// column-pivoted R, so if every pivot exceeds (10 eps)^2 times the largest column norm
// squared, QRCP would keep all K columns and the ID is the identity (rank K, empty T~).
// The factor 10 keeps the decision far above the rounding of the Gram matrix (~1e-16);
// blocks that do not pass go to the QR.
// Gram matrix A^T A (K x K, column-major) from its upper block triangle: one product per
// 64-column panel (half the flops of the full product, the same accumulation order per
// entry), the lower triangle copied from the upper.
static void gram_upper(const double* A, int64_t M, int64_t K, std::vector<double>& G) {
  G.assign(size_t(K) * K, 0.0);
  for (int64_t j0 = 0; j0 < K; j0 += 64) {
    const int64_t w = std::min<int64_t>(64, K - j0);
    gemm(true, int(j0 + w), int(w), int(M), 1.0, A, int(M), A + j0 * M, int(M), 0.0, &G[size_t(j0) * K], int(K));
  }
  for (int64_t j = 0; j < K; ++j)
    for (int64_t i = j + 1; i < K; ++i) G[size_t(j) * K + i] = G[size_t(i) * K + j];
}

static bool certify_full_rank(const double* A, int64_t M, int64_t K, double eps) {
  std::vector<double> G;
  gram_upper(A, M, K, G);
  double dmax = 0;
  for (int64_t j = 0; j < K; ++j) dmax = std::max(dmax, G[j * K + j]);
  if (!(dmax > 0) || !std::isfinite(dmax)) return false;
  const double floor = 100.0 * eps * eps * dmax;
  std::vector<int64_t> piv(K);
  std::iota(piv.begin(), piv.end(), int64_t(0));
  std::vector<double> d(K);
  for (int64_t j = 0; j < K; ++j) d[j] = G[j * K + j];
  // right-looking pivoted Cholesky on the permuted Gram matrix (lower triangle, in place)
  std::vector<double> Lc(size_t(K) * K, 0.0);
  for (int64_t k = 0; k < K; ++k) {
    int64_t p = k;
    for (int64_t j = k + 1; j < K; ++j)
      if (d[piv[j]] > d[piv[p]]) p = j;
    std::swap(piv[k], piv[p]);
    const double pk = d[piv[k]];
    if (!(pk > floor)) return false;
    const double lkk = std::sqrt(pk);
    for (int64_t j = k + 1; j < K; ++j) {
      double v = G[piv[j] * K + piv[k]];
      for (int64_t q = 0; q < k; ++q) v -= Lc[q * K + piv[j]] * Lc[q * K + piv[k]];
      v /= lkk;
      Lc[k * K + piv[j]] = v;
      d[piv[j]] -= v * v;
    }
  }
  return true;
}

int interpolative_decomposition_real(double* A, int64_t M, int64_t K, double eps,
                                     std::vector<int32_t>& perm, std::vector<double>& T, uint64_t seed,
                                     bool blocked) {
  if (blocked && K >= 32 && M >= 16 * K && certify_full_rank(A, M, K, eps)) {
    perm.resize(K);
    std::iota(perm.begin(), perm.end(), 0);
    T.clear();
    return int(K);
  }
  if (blocked && std::min(M, K) >= 128) return qrcp_id_blocked(A, M, K, eps, seed, perm, T);
  return qrcp_id<double>(A, M, K, eps, perm, T);
}

// ---------------------------------------------------------------------------------------
// Complex counterparts of the blocked ID and of the full-rank certificate, same algorithms.
// The reflectors are Hermitian, H = I - beta v v^H with beta = 2 / |v|^2 real and
// H x = R_kk e_1 (R_kk = -phase(x_0) |x|), as in the classical complex QRCP above; their
// product H_0 ... H_{b-1} = I - V T V^H has T upper triangular with T_qq = beta_q and
// T(0:q, q) = -beta_q T(0:q, 0:q) V(:, 0:q)^H v_q, so Q^H A2 = A2 - V T^H (V^H A2).
namespace {

using cd = std::complex<double>;

// Reflector of x (length n, n >= 1) in place: x becomes v (v_0 = x_0 - R_kk); returns beta.
double zhouse(cd* x, int64_t n, cd* rkk) {
  const double sig = sumsq(x, n);
  const double alpha = std::sqrt(sig);
  const double ax0 = std::abs(x[0]);
  const cd phase = ax0 > 0 ? x[0] / ax0 : cd(1.0);
  *rkk = -phase * alpha;
  x[0] -= *rkk;
  const double vn2 = 2.0 * alpha * (alpha + ax0);  // |x_0 + phase alpha|^2 + sig - |x_0|^2
  return vn2 > 0 ? 2.0 / vn2 : 0.0;
}

void zsketch_pivots(std::vector<cd>& Y, int s, int k, int steps, std::vector<int>& swaps) {
  std::vector<double> nr(k);
  for (int j = 0; j < k; ++j) nr[j] = sumsq(&Y[size_t(j) * s], s);
  swaps.assign(steps, 0);
  for (int q = 0; q < steps; ++q) {
    int p = q;
    for (int j = q + 1; j < k; ++j)
      if (nr[j] > nr[p]) p = j;
    swaps[q] = p;
    if (p != q) {
      std::swap_ranges(&Y[size_t(q) * s], &Y[size_t(q + 1) * s], &Y[size_t(p) * s]);
      std::swap(nr[q], nr[p]);
    }
    if (q >= s) continue;
    cd* col = &Y[size_t(q) * s];
    cd rkk;
    const double beta = zhouse(col + q, s - q, &rkk);
    if (beta != 0.0)
      for (int j = q + 1; j < k; ++j) reflect(col + q, &Y[size_t(j) * s + q], s - q, beta);
    col[q] = rkk;
    for (int j = q + 1; j < k; ++j) nr[j] = std::max(0.0, nr[j] - std::norm(Y[size_t(j) * s + q]));
  }
}

// X(:, c) = R^{-1} B(:, c) for the h x h upper-triangular R (ld ldr), column by column.
void ztrsm_upper(const cd* R, int64_t ldr, int64_t h, cd* X, int64_t ldx, int64_t ncols) {
  for (int64_t c = 0; c < ncols; ++c) {
    cd* xc = X + c * ldx;
    for (int64_t a = h - 1; a >= 0; --a) {
      cd acc = xc[a];
      for (int64_t q = a + 1; q < h; ++q) acc -= R[q * ldr + a] * xc[q];
      xc[a] = acc / R[a * ldr + a];
    }
  }
}

int zqrcp_id_blocked(cd* A, int64_t M, int64_t K, double eps, uint64_t seed, std::vector<int32_t>& perm,
                     std::vector<double>& Tout) {
  constexpr int b = 64, p = 8, s = b + p;
  perm.resize(K);
  std::iota(perm.begin(), perm.end(), 0);
  Tout.clear();
  double maxn = 0;
  for (int64_t j = 0; j < K; ++j) {
    const double v = sumsq(A + j * M, M);
    if (!std::isfinite(v)) fail(MHT_ERR_NUMERIC, "non-finite entry in a block of Phi");
    maxn = std::max(maxn, v);
  }
  if (maxn == 0.0) return 0;
  const double thr = eps * std::sqrt(maxn);
  // complex Gaussian sketch Y = G A (s x K)
  std::vector<cd> G(size_t(s) * M), Y(size_t(s) * K);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> N01;
  for (auto& g : G) g = cd(N01(rng), N01(rng));
  zgemm(false, s, int(K), int(M), 1.0, G.data(), s, A, int(M), 0.0, Y.data(), s);
  const int64_t kmax = std::min(M, K);
  int64_t r = kmax;
  std::vector<cd> V, Tm, W, Ys, X;
  std::vector<double> beta(b);
  std::vector<int> swaps;
  for (int64_t j = 0; j < kmax; j += b) {
    const int bb = int(std::min<int64_t>(b, kmax - j));
    const int64_t M2 = M - j, K2 = K - j - bb;
    // a. pivots from the sketch of the remaining columns, replayed on A, Y and perm
    Ys.assign(Y.begin() + size_t(j) * s, Y.end());
    zsketch_pivots(Ys, s, int(K - j), bb, swaps);
    for (int q = 0; q < bb; ++q) {
      const int64_t a = j + q, c = j + swaps[q];
      if (a == c) continue;
      std::swap_ranges(A + a * M, A + (a + 1) * M, A + c * M);
      std::swap_ranges(&Y[size_t(a) * s], &Y[size_t(a + 1) * s], &Y[size_t(c) * s]);
      std::swap(perm[a], perm[c]);
    }
    // b. Householder QR of the panel; V keeps the reflectors (zero above their diagonal)
    V.assign(size_t(M2) * bb, cd(0.0));
    int64_t rank_here = -1;
    for (int q = 0; q < bb; ++q) {
      cd* col = A + (j + q) * M + j;
      cd rkk;
      beta[q] = zhouse(col + q, M2 - q, &rkk);
      if (rank_here < 0 && !(std::abs(rkk) > thr)) rank_here = j + q;
      cd* v = &V[size_t(q) * M2];
      for (int64_t i = q; i < M2; ++i) v[i] = col[i];
      if (beta[q] != 0.0)
        for (int c = q + 1; c < bb; ++c) reflect(v + q, A + (j + c) * M + j + q, M2 - q, beta[q]);
      col[q] = rkk;
      for (int64_t i = q + 1; i < M2; ++i) col[i] = cd(0.0);
    }
    // c. T of the compact WY form
    Tm.assign(size_t(bb) * bb, cd(0.0));
    std::vector<cd> w(bb);
    for (int q = 0; q < bb; ++q) {
      Tm[size_t(q) * bb + q] = beta[q];
      if (q == 0 || beta[q] == 0.0) continue;
      const cd* vq = &V[size_t(q) * M2];
      for (int c = 0; c < q; ++c) {  // w = -beta_q V(:, 0:q)^H v_q (v_q is zero above row q)
        const cd* vc = &V[size_t(c) * M2];
        cd acc = 0;
        for (int64_t i = q; i < M2; ++i) acc += std::conj(vc[i]) * vq[i];
        w[c] = -beta[q] * acc;
      }
      for (int a = 0; a < q; ++a) {
        cd acc = 0;
        for (int c = a; c < q; ++c) acc += Tm[size_t(c) * bb + a] * w[c];
        Tm[size_t(q) * bb + a] = acc;
      }
    }
    // d. trailing update A2 <- A2 - V T^H (V^H A2)
    cd* A2 = A + (j + bb) * M + j;
    if (K2 > 0) {
      W.assign(size_t(bb) * K2, cd(0.0));
      zgemm(true, bb, int(K2), int(M2), 1.0, V.data(), int(M2), A2, int(M), 0.0, W.data(), bb);
      for (int64_t c = 0; c < K2; ++c) {  // W <- T^H W, bottom row first (T^H is lower triangular)
        cd* wc = &W[size_t(c) * bb];
        for (int a = bb - 1; a >= 0; --a) {
          cd acc = 0;
          for (int q = 0; q <= a; ++q) acc += std::conj(Tm[size_t(a) * bb + q]) * wc[q];
          wc[a] = acc;
        }
      }
      zgemm(false, int(M2), int(K2), bb, -1.0, V.data(), int(M2), W.data(), bb, 1.0, A2, int(M));
    }
    if (rank_here >= 0) { r = rank_here; break; }
    // e. stop when every remaining column is below the threshold
    double rem = 0;
    for (int64_t c = 0; c < K2; ++c) rem = std::max(rem, sumsq(A2 + c * M + bb, M2 - bb));
    if (K2 == 0 || std::sqrt(rem) <= thr || j + bb >= kmax) { r = std::min<int64_t>(j + bb, kmax); break; }
    // f. sketch downdate Y2 <- Y2 - Y1 R11^{-1} R12
    X.assign(size_t(bb) * K2, cd(0.0));
    for (int64_t c = 0; c < K2; ++c)
      for (int a = 0; a < bb; ++a) X[size_t(c) * bb + a] = A2[c * M + a];
    ztrsm_upper(A + j * M + j, M, bb, X.data(), bb, K2);
    zgemm(false, s, int(K2), bb, -1.0, &Y[size_t(j) * s], s, X.data(), bb, 1.0, &Y[size_t(j + bb) * s], s);
  }
  // T~ = R11^{-1} R12 by blocked back substitution, written row-major r x (K - r)
  const int64_t nc = K - r;
  Tout.assign(size_t(r * nc) * 2, 0.0);
  if (r == 0 || nc == 0) return int(r);
  std::vector<cd> Tc(size_t(r) * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t i = 0; i < r; ++i) Tc[size_t(c) * r + i] = A[(r + c) * M + i];
  constexpr int bs = 64;
  for (int64_t i1 = r; i1 > 0; i1 -= bs) {
    const int64_t i0 = std::max<int64_t>(0, i1 - bs), h = i1 - i0;
    if (i1 < r)
      zgemm(false, int(h), int(nc), int(r - i1), -1.0, A + i1 * M + i0, int(M), &Tc[i1], int(r), 1.0, &Tc[i0],
            int(r));
    ztrsm_upper(A + i0 * M + i0, M, h, &Tc[i0], r, nc);
  }
  cd* T = reinterpret_cast<cd*>(Tout.data());
  for (int64_t i = 0; i < r; ++i)
    for (int64_t c = 0; c < nc; ++c) T[size_t(i) * nc + c] = Tc[size_t(c) * r + i];
  for (double v : Tout)
    if (!std::isfinite(v)) fail(MHT_ERR_NUMERIC, "non-finite interpolation coefficient");
  return int(r);
}

// Complex full-rank certificate: Hermitian Gram matrix A^H A and diagonally pivoted Cholesky,
// same decision rule as the real one.
bool certify_full_rank_complex(const cd* A, int64_t M, int64_t K, double eps) {
  std::vector<cd> G(size_t(K) * K, cd(0.0));  // upper block triangle, lower = conjugate transpose
  for (int64_t j0 = 0; j0 < K; j0 += 64) {
    const int64_t w = std::min<int64_t>(64, K - j0);
    zgemm(true, int(j0 + w), int(w), int(M), 1.0, A, int(M), A + j0 * M, int(M), 0.0, &G[size_t(j0) * K], int(K));
  }
  for (int64_t j = 0; j < K; ++j)
    for (int64_t i = j + 1; i < K; ++i) G[size_t(j) * K + i] = std::conj(G[size_t(i) * K + j]);
  double dmax = 0;
  for (int64_t j = 0; j < K; ++j) dmax = std::max(dmax, G[j * K + j].real());
  if (!(dmax > 0) || !std::isfinite(dmax)) return false;
  const double floor = 100.0 * eps * eps * dmax;
  std::vector<int64_t> piv(K);
  std::iota(piv.begin(), piv.end(), int64_t(0));
  std::vector<double> d(K);
  for (int64_t j = 0; j < K; ++j) d[j] = G[j * K + j].real();
  std::vector<cd> Lc(size_t(K) * K, cd(0.0));  // Lc[q K + i] = L(i, q)
  for (int64_t k = 0; k < K; ++k) {
    int64_t p = k;
    for (int64_t j = k + 1; j < K; ++j)
      if (d[piv[j]] > d[piv[p]]) p = j;
    std::swap(piv[k], piv[p]);
    const double pk = d[piv[k]];
    if (!(pk > floor)) return false;
    const double lkk = std::sqrt(pk);
    for (int64_t j = k + 1; j < K; ++j) {
      cd v = G[piv[k] * K + piv[j]];  // G(piv_j, piv_k)
      for (int64_t q = 0; q < k; ++q) v -= Lc[q * K + piv[j]] * std::conj(Lc[q * K + piv[k]]);
      v /= lkk;
      Lc[k * K + piv[j]] = v;
      d[piv[j]] -= std::norm(v);
    }
  }
  return true;
}

}  // namespace

int interpolative_decomposition_complex(std::complex<double>* A, int64_t M, int64_t K,
                                        double eps, std::vector<int32_t>& perm,
                                        std::vector<double>& T, uint64_t seed, bool blocked) {
  if (blocked && K >= 32 && M >= 16 * K && certify_full_rank_complex(A, M, K, eps)) {
    perm.resize(K);
    std::iota(perm.begin(), perm.end(), 0);
    T.clear();
    return int(K);
  }
  if (blocked && std::min(M, K) >= 128) return zqrcp_id_blocked(A, M, K, eps, seed, perm, T);
  return qrcp_id<std::complex<double>>(A, M, K, eps, perm, T);
}

}  // namespace mht
