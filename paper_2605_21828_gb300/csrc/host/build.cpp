// Butterfly factorization build (Sec. 2, Algorithm 1; memory-bounded as in Sec. 4).
//
// Level 0: for each frequency leaf nu, the column ID Phi(:, nu) ~= Phi(:, J_nu) T_nu.
// Levels l = 1..L: for tau at depth l (parent p) and nu at height l (children c1, c2), the
// ID of [U_{p c1}(tau,:)  U_{p c2}(tau,:)] = Phi(tau, J_{p c1} u J_{p c2}) -- with nested IDs
// the column bases are submatrices of Phi, so each block only needs Phi at its rows and at
// its parent's skeleton columns.  Finally U_tau = Phi(tau, J_{tau, root}).
//
// Memory stays bounded by the result (the aim of Algorithm 3): no column block Phi(:, nu)
// is kept beyond its own ID; every block matrix is evaluated on demand, factored and freed.
// Blocks of one level are independent and run in parallel (OpenMP).
//
// Row sampling (the randomized IDs mentioned at the end of Sec. 2): when a block has many
// more rows than columns, the pivoted QR runs on a seeded uniform sample of
// min(|tau|, ceil(oversample K) + 16) rows; the column bases U are always exact.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <numeric>
#include <random>

#include "internal.h"

namespace mht {

int64_t Factorization::input_size(int l, int64_t b) const {
  const int64_t nb = int64_t(1) << (L - l);
  if (l == 0) return mode_off[b + 1] - mode_off[b];
  const int64_t q = pair_index(l, b);
  return int64_t(lv[l - 1][q].r) + int64_t(lv[l - 1][q + 1].r);
  (void)nb;
}

void Factorization::validate() const {
  const int64_t nb = nblk();
  auto is_perm = [](const std::vector<int64_t>& p, int64_t n) {
    if (int64_t(p.size()) != n) return false;
    std::vector<char> seen(n, 0);
    for (int64_t v : p) {
      if (v < 0 || v >= n || seen[v]) return false;
      seen[v] = 1;
    }
    return true;
  };
  auto offs_ok = [&](const std::vector<int64_t>& o, int64_t n) {
    if (int64_t(o.size()) != nb + 1 || o[0] != 0 || o[nb] != n) return false;
    for (int64_t i = 0; i < nb; ++i)
      if (o[i + 1] < o[i]) return false;
    return true;
  };
  if (L < 0 || L > 24) fail(MHT_ERR_FORMAT, "levels out of range");
  if (!is_perm(space_perm, n) || !offs_ok(space_off, n)) fail(MHT_ERR_FORMAT, "bad space permutation or offsets");
  if (!is_perm(mode_perm, m) || !offs_ok(mode_off, m)) fail(MHT_ERR_FORMAT, "bad mode permutation or offsets");
  if (int64_t(lv.size()) != L + 1) fail(MHT_ERR_FORMAT, "wrong number of levels");
  const int W = cplx ? 2 : 1;
  for (int l = 0; l <= L; ++l) {
    if (int64_t(lv[l].size()) != nb) fail(MHT_ERR_FORMAT, "wrong number of blocks");
    for (int64_t b = 0; b < nb; ++b) {
      const Block& B = lv[l][b];
      const int64_t K = input_size(l, b);
      if (B.K != K || B.r < 0 || B.r > K) fail(MHT_ERR_FORMAT, "inconsistent rank / input size at level " + std::to_string(l));
      if (int64_t(B.perm.size()) != K) fail(MHT_ERR_FORMAT, "bad local permutation size");
      std::vector<char> seen(K, 0);
      for (int32_t v : B.perm) {
        if (v < 0 || v >= K || seen[v]) fail(MHT_ERR_FORMAT, "local permutation is not a permutation");
        seen[v] = 1;
      }
      if (int64_t(B.T.size()) != int64_t(B.r) * (K - B.r) * W) fail(MHT_ERR_FORMAT, "bad transfer size");
    }
  }
  if (int64_t(U.size()) != nb) fail(MHT_ERR_FORMAT, "wrong number of column bases");
  for (int64_t t = 0; t < nb; ++t)
    if (int64_t(U[t].size()) != leaf_rows(t) * int64_t(lv[L][t].r) * W) fail(MHT_ERR_FORMAT, "bad column basis size");
  if (!weights.empty() && int64_t(weights.size()) != n) fail(MHT_ERR_FORMAT, "bad weights size");
}

namespace {

int tree_depth(int64_t n, int64_t leaf) {
  if (n <= leaf) return 0;
  int L = 0;
  while ((int64_t(leaf) << L) < n) ++L;
  return L;
}

// ID of the block Phi(rows, cols); returns the block and writes the skeleton columns.
Block factor_block(const Evaluator& ev, bool cplx, const std::vector<int64_t>& rows_all,
                   const std::vector<int64_t>& cols, double eps, double oversample,
                   uint64_t seed, std::vector<int64_t>& skel, bool blocked) {
  Block B;
  const int64_t K = int64_t(cols.size());
  B.K = int32_t(K);
  int64_t M = int64_t(rows_all.size());
  const std::vector<int64_t>* rows = &rows_all;
  std::vector<int64_t> sample;
  if (oversample > 0) {
    const int64_t s = std::min<int64_t>(M, int64_t(std::ceil(oversample * double(K))) + 16);
    if (s < M) {
      sample = rows_all;
      std::mt19937_64 rng(seed);
      for (int64_t i = 0; i < s; ++i) {  // partial Fisher-Yates
        std::uniform_int_distribution<int64_t> U(i, M - 1);
        std::swap(sample[i], sample[U(rng)]);
      }
      sample.resize(s);
      std::sort(sample.begin(), sample.end());
      rows = &sample;
      M = s;
    }
  }
  if (cplx) {
    std::vector<std::complex<double>> A(size_t(M * K));
    ev.eval(rows->data(), M, cols.data(), K, reinterpret_cast<double*>(A.data()));
    B.r = interpolative_decomposition_complex(A.data(), M, K, eps, B.perm, B.T, seed ^ 0x5bd1e995ull, blocked);
  } else {
    std::vector<double> A(size_t(M * K));
    ev.eval(rows->data(), M, cols.data(), K, A.data());
    B.r = interpolative_decomposition_real(A.data(), M, K, eps, B.perm, B.T, seed ^ 0x5bd1e995ull, blocked);
  }
  skel.resize(B.r);
  for (int32_t i = 0; i < B.r; ++i) skel[i] = cols[B.perm[i]];
  return B;
}

uint64_t mix(uint64_t a, uint64_t b) {
  uint64_t x = a ^ (b + 0x9e3779b97f4a7c15ull + (a << 6) + (a >> 2));
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33;
  return x;
}

}  // namespace

void build_factorization(const mht_problem& p, const mht_options& o, Factorization& F) {
  if (p.n <= 0 || p.m <= 0) fail(MHT_ERR_INVALID_ARG, "n and m must be positive");
  if (p.n > (int64_t(1) << 31) - 1 || p.m > (int64_t(1) << 31) - 1) fail(MHT_ERR_INVALID_ARG, "n, m must fit int32");
  if (!p.eigenvalues) fail(MHT_ERR_INVALID_ARG, "eigenvalues are required (frequency order)");
  if (!(o.eps > 0) || o.eps >= 1) fail(MHT_ERR_INVALID_ARG, "eps must be in (0, 1)");
  if (p.field != MHT_REAL && p.field != MHT_COMPLEX) fail(MHT_ERR_INVALID_ARG, "bad field");
  for (int64_t k = 0; k < p.m; ++k)
    if (!std::isfinite(p.eigenvalues[k])) fail(MHT_ERR_NUMERIC, "non-finite eigenvalue");
  int L;
  if (o.levels >= 0) L = o.levels;
  else {
    if (o.leaf_size <= 0) fail(MHT_ERR_INVALID_ARG, "leaf_size must be positive");
    L = tree_depth(p.n, o.leaf_size);
  }
  if (L > 20) fail(MHT_ERR_INVALID_ARG, "too many levels");
  F = Factorization();
  F.n = p.n; F.m = p.m; F.L = L; F.cplx = (p.field == MHT_COMPLEX);
  const bool verbose = std::getenv("MHT_VERBOSE") != nullptr;
  auto t_start = std::chrono::steady_clock::now();
  auto stamp = [&](const char* what, int l) {
    if (!verbose) return;
    const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    std::fprintf(stderr, "[mht build] %s %d at %.2f s\n", what, l, t);
  };
  frequency_tree(p.eigenvalues, p.m, L, F.mode_perm, F.mode_off);
  space_tree(p, o.tree, L, o.seed, F.space_perm, F.space_off);
  stamp("trees", L);
  if (p.weights) {
    F.weights.assign(p.weights, p.weights + p.n);
    for (double w : F.weights)
      if (!std::isfinite(w)) fail(MHT_ERR_NUMERIC, "non-finite weight");
  }
  std::unique_ptr<Evaluator> ev(make_evaluator(p));
  const bool blocked = o.id_method == MHT_ID_BLOCKED || (o.id_method == MHT_ID_AUTO && p.n * p.m >= (int64_t(1) << 28));
  const int64_t nb = F.nblk();
  F.lv.assign(L + 1, std::vector<Block>(nb));
  std::vector<std::vector<int64_t>> J(nb), Jn(nb);
  std::vector<int64_t> all(p.n);
  std::iota(all.begin(), all.end(), int64_t(0));
  // exceptions must not leave an OpenMP region: capture the first one
  Error first(MHT_OK, "");
  bool failed = false;
  auto guarded = [&](auto&& fn) {
    try {
      fn();
    } catch (const Error& e) {
#pragma omp critical(mht_build_err)
      if (!failed) { failed = true; first = e; }
    } catch (const std::bad_alloc&) {
#pragma omp critical(mht_build_err)
      if (!failed) { failed = true; first = Error(MHT_ERR_OOM, "host allocation failed during build"); }
    }
  };
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t nu = 0; nu < nb; ++nu)
    guarded([&] {
      std::vector<int64_t> cols(F.mode_perm.begin() + F.mode_off[nu], F.mode_perm.begin() + F.mode_off[nu + 1]);
      F.lv[0][nu] = factor_block(*ev, F.cplx, all, cols, o.eps, o.oversample, mix(o.seed, uint64_t(nu)), J[nu], blocked);
    });
  if (failed) throw first;
  stamp("level", 0);
  for (int l = 1; l <= L; ++l) {
    const int64_t nbl = int64_t(1) << (L - l);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nb; ++b)
      guarded([&] {
        const int64_t tau = b / nbl;
        const int64_t w = int64_t(1) << (L - l);
        std::vector<int64_t> rows(F.space_perm.begin() + F.space_off[tau * w],
                                  F.space_perm.begin() + F.space_off[(tau + 1) * w]);
        const int64_t q = F.pair_index(l, b);
        std::vector<int64_t> cand(J[q]);
        cand.insert(cand.end(), J[q + 1].begin(), J[q + 1].end());
        F.lv[l][b] = factor_block(*ev, F.cplx, rows, cand, o.eps, o.oversample,
                                  mix(mix(o.seed, uint64_t(l)), uint64_t(b)), Jn[b], blocked);
      });
    if (failed) throw first;
    J.swap(Jn);
    stamp("level", l);
  }
  // column bases U_tau = Phi(tau, J_{tau, root}), row-major |tau| x r_L (rows in tree order)
  F.U.assign(nb, {});
  const int W = F.cplx ? 2 : 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nb; ++t)
    guarded([&] {
      std::vector<int64_t> rows(F.space_perm.begin() + F.space_off[t], F.space_perm.begin() + F.space_off[t + 1]);
      const int64_t M = int64_t(rows.size()), R = int64_t(J[t].size());
      std::vector<double> cm(size_t(M * R * W));
      ev->eval(rows.data(), M, J[t].data(), R, cm.data());
      std::vector<double>& U = F.U[t];
      U.assign(size_t(M * R * W), 0.0);
      for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < R; ++j)
          for (int c = 0; c < W; ++c) {
            const double v = cm[(j * M + i) * W + c];
            if (!std::isfinite(v)) throw Error(MHT_ERR_NUMERIC, "non-finite column basis entry");
            U[(i * R + j) * W + c] = v;
          }
    });
  if (failed) throw first;
  stamp("column bases", L);
}

void import_factors(const mht_factors& in, Factorization& F) {
  if (in.n <= 0 || in.m <= 0 || in.levels < 0 || in.levels > 20) fail(MHT_ERR_INVALID_ARG, "bad n, m or levels");
  if (!in.space_perm || !in.space_offsets || !in.mode_perm || !in.mode_offsets || !in.ranks || !in.local_perm)
    fail(MHT_ERR_INVALID_ARG, "missing factor arrays");
  F = Factorization();
  F.n = in.n; F.m = in.m; F.L = in.levels; F.cplx = (in.field == MHT_COMPLEX);
  const int64_t nb = F.nblk();
  F.space_perm.assign(in.space_perm, in.space_perm + in.n);
  F.space_off.assign(in.space_offsets, in.space_offsets + nb + 1);
  F.mode_perm.assign(in.mode_perm, in.mode_perm + in.m);
  F.mode_off.assign(in.mode_offsets, in.mode_offsets + nb + 1);
  if (in.weights) F.weights.assign(in.weights, in.weights + in.n);
  const int W = F.cplx ? 2 : 1;
  // basic offset checks before sizes are derived from them
  for (int64_t i = 0; i < nb; ++i)
    if (F.mode_off[i + 1] < F.mode_off[i] || F.space_off[i + 1] < F.space_off[i]) fail(MHT_ERR_FORMAT, "offsets not monotone");
  if (F.mode_off[0] != 0 || F.mode_off[nb] != F.m || F.space_off[0] != 0 || F.space_off[nb] != F.n)
    fail(MHT_ERR_FORMAT, "offsets do not span the index ranges");
  F.lv.assign(F.L + 1, std::vector<Block>(nb));
  int64_t pp = 0, tp = 0;
  for (int l = 0; l <= F.L; ++l)
    for (int64_t b = 0; b < nb; ++b) {
      Block& B = F.lv[l][b];
      const int64_t K = F.input_size(l, b);
      const int64_t r = in.ranks[int64_t(l) * nb + b];
      if (r < 0 || r > K) fail(MHT_ERR_FORMAT, "rank out of range");
      B.K = int32_t(K);
      B.r = int32_t(r);
      B.perm.assign(in.local_perm + pp, in.local_perm + pp + K);
      pp += K;
      const int64_t te = r * (K - r) * W;
      if (te > 0 && !in.transfer) fail(MHT_ERR_INVALID_ARG, "missing transfer array");
      B.T.assign(in.transfer ? in.transfer + tp : nullptr, in.transfer ? in.transfer + tp + te : nullptr);
      tp += te;
    }
  F.U.assign(nb, {});
  int64_t up = 0;
  for (int64_t t = 0; t < nb; ++t) {
    const int64_t e = F.leaf_rows(t) * int64_t(F.lv[F.L][t].r) * W;
    if (e > 0 && !in.column_bases) fail(MHT_ERR_INVALID_ARG, "missing column_bases array");
    F.U[t].assign(in.column_bases ? in.column_bases + up : nullptr, in.column_bases ? in.column_bases + up + e : nullptr);
    up += e;
  }
  F.validate();
}

}  // namespace mht
