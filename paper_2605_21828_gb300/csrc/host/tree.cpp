// Row (space) and column (frequency) trees of the butterfly (Sec. 2 and Sec. 3).
//
// Both trees are complete binary trees of the same depth L.  Nodes are contiguous ranges
// of a permutation; only the leaf offsets are stored (a node at depth d, index i, covers
// leaves [i 2^(L-d), (i+1) 2^(L-d))).  Space nodes may be empty.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>

#include "internal.h"

namespace mht {

// Frequency tree: modes in stable eigenvalue order; each node's range is halved with
// floor(size / 2) to the left child, down to depth L.
void frequency_tree(const double* lam, int64_t m, int L, std::vector<int64_t>& perm,
                    std::vector<int64_t>& off) {
  perm.resize(m);
  std::iota(perm.begin(), perm.end(), int64_t(0));
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return lam[a] < lam[b]; });
  std::vector<int64_t> cur = {0, m};
  for (int d = 0; d < L; ++d) {
    std::vector<int64_t> nxt;
    nxt.push_back(0);
    for (size_t i = 0; i + 1 < cur.size(); ++i) {
      int64_t a = cur[i], b = cur[i + 1];
      nxt.push_back(a + (b - a) / 2);
      nxt.push_back(b);
    }
    cur.swap(nxt);
  }
  off = cur;
}

namespace {

struct Node {
  std::vector<int64_t> idx;
  double box[2][2];  // RECT: [axis][lo, hi]; unused otherwise
  bool periodic_root = false;
};

// Flat periodic square: phi_2 of the Neumann problem on a rectangle [a1,b1] x [a2,b2] is
// cos(pi (x - a) / w) along its longer side (ties: first axis); at the periodic root the
// second eigenspace is spanned by sin/cos of x1, x2 and sin(x1) is taken.  M_1 = {phi_2 <= 0}.
void split_rect(const double* X, Node& nd, Node& c1, Node& c2) {
  if (nd.periodic_root) {
    for (int64_t i : nd.idx) (std::sin(X[2 * i]) <= 0.0 ? c1 : c2).idx.push_back(i);
    c1.box[0][0] = -M_PI; c1.box[0][1] = 0.0; c1.box[1][0] = -M_PI; c1.box[1][1] = M_PI;
    c2.box[0][0] = 0.0; c2.box[0][1] = M_PI; c2.box[1][0] = -M_PI; c2.box[1][1] = M_PI;
    return;
  }
  const double w0 = nd.box[0][1] - nd.box[0][0], w1 = nd.box[1][1] - nd.box[1][0];
  const int ax = (w0 >= w1) ? 0 : 1;
  const double a = nd.box[ax][0], w = nd.box[ax][1] - a, mid = a + 0.5 * w;
  for (int64_t i : nd.idx)
    (std::cos(M_PI * (X[2 * i + ax] - a) / w) <= 0.0 ? c1 : c2).idx.push_back(i);
  for (int d = 0; d < 2; ++d)
    for (int e = 0; e < 2; ++e) c1.box[d][e] = c2.box[d][e] = nd.box[d][e];
  c1.box[ax][0] = mid;  // cos(...) <= 0 on the upper half
  c2.box[ax][1] = mid;
}

// Median split along the principal axis of the node's points (equal halves, floor to the
// left); ties broken by original index so the split is deterministic.
void split_pca(const double* X, int dim, Node& nd, Node& c1, Node& c2) {
  const int64_t k = int64_t(nd.idx.size());
  if (k == 0) return;
  std::vector<double> mean(dim, 0.0);
  for (int64_t i : nd.idx)
    for (int d = 0; d < dim; ++d) mean[d] += X[i * dim + d];
  for (int d = 0; d < dim; ++d) mean[d] /= double(k);
  std::vector<double> C(dim * dim, 0.0);
  for (int64_t i : nd.idx)
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b)
        C[a * dim + b] += (X[i * dim + a] - mean[a]) * (X[i * dim + b] - mean[b]);
  // dominant eigenvector by power iteration (dim <= 3)
  std::vector<double> v(dim, 1.0), w(dim);
  for (int d = 0; d < dim; ++d) v[d] = 1.0 + 0.1 * d;
  for (int it = 0; it < 200; ++it) {
    double nrm = 0;
    for (int a = 0; a < dim; ++a) {
      w[a] = 0;
      for (int b = 0; b < dim; ++b) w[a] += C[a * dim + b] * v[b];
      nrm += w[a] * w[a];
    }
    nrm = std::sqrt(nrm);
    if (nrm == 0) break;
    for (int a = 0; a < dim; ++a) v[a] = w[a] / nrm;
  }
  std::vector<std::pair<double, int64_t>> t(k);
  for (int64_t j = 0; j < k; ++j) {
    const int64_t i = nd.idx[j];
    double s = 0;
    for (int d = 0; d < dim; ++d) s += (X[i * dim + d] - mean[d]) * v[d];
    t[j] = {s, i};
  }
  std::sort(t.begin(), t.end());
  const int64_t h = k / 2;
  for (int64_t j = 0; j < k; ++j) (j < h ? c1 : c2).idx.push_back(t[j].second);
}

void fiedler_split(const double* X, int dim, const std::vector<int64_t>& idx, uint64_t seed,
                   std::vector<char>& in_m1);

}  // namespace

void space_tree(const mht_problem& p, mht_tree_kind kind, int L, uint64_t seed,
                std::vector<int64_t>& perm, std::vector<int64_t>& off) {
  const int64_t n = p.n;
  const int64_t nleaf = int64_t(1) << L;
  if (kind == MHT_TREE_GIVEN) {
    if (!p.space_perm || !p.space_offsets) fail(MHT_ERR_INVALID_ARG, "MHT_TREE_GIVEN needs space_perm and space_offsets");
    perm.assign(p.space_perm, p.space_perm + n);
    off.assign(p.space_offsets, p.space_offsets + nleaf + 1);
    return;
  }
  if (kind == MHT_TREE_AUTO)
    kind = (p.eval_kind == MHT_EVAL_TORUS) ? MHT_TREE_RECT : MHT_TREE_FIEDLER;
  if (!p.points) fail(MHT_ERR_INVALID_ARG, "space tree needs problem->points");
  if (kind == MHT_TREE_RECT && p.dim != 2) fail(MHT_ERR_INVALID_ARG, "MHT_TREE_RECT needs 2-D points");
  std::vector<Node> cur(1);
  cur[0].idx.resize(n);
  std::iota(cur[0].idx.begin(), cur[0].idx.end(), int64_t(0));
  cur[0].periodic_root = true;
  for (int d = 0; d < L; ++d) {
    std::vector<Node> nxt(cur.size() * 2);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < int64_t(cur.size()); ++i) {
      Node& nd = cur[i];
      Node& c1 = nxt[2 * i];
      Node& c2 = nxt[2 * i + 1];
      if (kind == MHT_TREE_RECT) {
        split_rect(p.points, nd, c1, c2);
      } else if (kind == MHT_TREE_PCA_MEDIAN) {
        split_pca(p.points, p.dim, nd, c1, c2);
      } else {
        std::vector<char> m1;
        fiedler_split(p.points, p.dim, nd.idx, seed + uint64_t(d) * 1000003ull + uint64_t(i), m1);
        for (size_t j = 0; j < nd.idx.size(); ++j) (m1[j] ? c1 : c2).idx.push_back(nd.idx[j]);
      }
      std::vector<int64_t>().swap(nd.idx);
    }
    cur.swap(nxt);
  }
  perm.clear();
  off.assign(1, 0);
  for (auto& nd : cur) {
    perm.insert(perm.end(), nd.idx.begin(), nd.idx.end());
    off.push_back(int64_t(perm.size()));
  }
}

namespace {

// ---- mesh-free Fiedler split (Sec. 3, Algorithm 2) --------------------------------------
// phi_2 of the kNN heat-kernel graph Laplacian on the node's points (the mesh-free
// construction of Sec. 7.3): weights exp(-d^2/t) on the symmetrized k-nearest-neighbour
// graph, t = mean squared neighbour distance; v_2 of (D - W) v = lambda D v, computed as the
// second eigenvector of S = D^{-1/2} W D^{-1/2} by Lanczos with full reorthogonalization
// against the known top eigenvector D^{1/2} 1.  M_1 = {phi_2 <= 0}.

struct Grid {  // uniform bucket grid for kNN queries
  int dim;
  double lo[3], h;
  int64_t nb[3];
  std::vector<int64_t> start, items;
};

void knn(const double* X, int dim, const std::vector<int64_t>& idx, int k,
         std::vector<int32_t>& nbr, std::vector<double>& d2) {
  const int64_t n = int64_t(idx.size());
  nbr.assign(n * k, -1);
  d2.assign(n * k, 0.0);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i : idx)
    for (int d = 0; d < dim; ++d) {
      lo[d] = std::min(lo[d], X[i * dim + d]);
      hi[d] = std::max(hi[d], X[i * dim + d]);
    }
  double vol = 1;
  int active = 0;
  for (int d = 0; d < dim; ++d)
    if (hi[d] - lo[d] > 0) { vol *= (hi[d] - lo[d]); ++active; }
  // about 2 points per cell
  double h = active ? std::pow(vol * 2.0 / double(std::max<int64_t>(n, 1)), 1.0 / active) : 1.0;
  if (!(h > 0)) h = 1.0;
  int64_t nb[3] = {1, 1, 1};
  for (int d = 0; d < dim; ++d) nb[d] = std::max<int64_t>(1, std::min<int64_t>(int64_t((hi[d] - lo[d]) / h) + 1, 1 << 10));
  auto cell = [&](int64_t i, int64_t* c) {
    for (int d = 0; d < 3; ++d) c[d] = 0;
    for (int d = 0; d < dim; ++d) c[d] = std::min<int64_t>(nb[d] - 1, std::max<int64_t>(0, int64_t((X[i * dim + d] - lo[d]) / h)));
  };
  const int64_t ncell = nb[0] * nb[1] * nb[2];
  std::vector<int64_t> cnt(ncell + 1, 0), items(n);
  std::vector<int64_t> cid(n);
  for (int64_t j = 0; j < n; ++j) {
    int64_t c[3];
    cell(idx[j], c);
    cid[j] = (c[0] * nb[1] + c[1]) * nb[2] + c[2];
    cnt[cid[j] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t j = 0; j < n; ++j) items[fill[cid[j]]++] = j;
#pragma omp parallel for schedule(static) if (n > 4096)
  for (int64_t j = 0; j < n; ++j) {
    int64_t c[3];
    cell(idx[j], c);
    std::vector<std::pair<double, int32_t>> best;
    for (int rad = 1;; ++rad) {
      best.clear();
      int64_t lo3[3], hi3[3];
      for (int d = 0; d < 3; ++d) {
        lo3[d] = std::max<int64_t>(0, c[d] - rad);
        hi3[d] = std::min<int64_t>(nb[d] - 1, c[d] + rad);
      }
      for (int64_t a = lo3[0]; a <= hi3[0]; ++a)
        for (int64_t b = lo3[1]; b <= hi3[1]; ++b)
          for (int64_t e = lo3[2]; e <= hi3[2]; ++e) {
            const int64_t cc = (a * nb[1] + b) * nb[2] + e;
            for (int64_t t = cnt[cc]; t < cnt[cc + 1]; ++t) {
              const int64_t q = items[t];
              if (q == j) continue;
              double s = 0;
              for (int d = 0; d < dim; ++d) {
                const double u = X[idx[q] * dim + d] - X[idx[j] * dim + d];
                s += u * u;
              }
              best.push_back({s, int32_t(q)});
            }
          }
      const bool covers_all = (lo3[0] == 0 && lo3[1] == 0 && lo3[2] == 0 && hi3[0] == nb[0] - 1 &&
                               hi3[1] == nb[1] - 1 && hi3[2] == nb[2] - 1);
      if (int64_t(best.size()) >= k || covers_all) {
        const int kk = int(std::min<int64_t>(k, int64_t(best.size())));
        std::partial_sort(best.begin(), best.begin() + kk, best.end());
        // neighbours inside radius rad*h are exact; accept if the k-th is within that
        if (covers_all || (kk > 0 && best[kk - 1].first <= double(rad) * double(rad) * h * h)) {
          for (int t = 0; t < kk; ++t) {
            nbr[j * k + t] = best[t].second;
            d2[j * k + t] = best[t].first;
          }
          break;
        }
      }
    }
  }
}

// symmetric tridiagonal eigenvector for the largest eigenvalue (bisection + inverse iteration)
std::vector<double> tridiag_top_vector(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = int(a.size());
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0) + (i + 1 < m ? std::fabs(b[i]) : 0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // Sturm count of eigenvalues < x
    int c = 0;
    double q = 1;
    for (int i = 0; i < m; ++i) {
      q = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
      if (q == 0) q = 1e-300;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m) hi = mid; else lo = mid;
    if (hi - lo < 1e-15 * std::max(1.0, std::fabs(hi))) break;
  }
  const double lam = hi + 1e-13 * std::max(1.0, std::fabs(hi));
  // inverse iteration on (T - lam I) via the Thomas algorithm
  std::vector<double> x(m, 1.0), y(m), c(m), d(m);
  for (int it = 0; it < 4; ++it) {
    // solve (T - lam) y = x
    std::vector<double> dd(m), cc(m), rr(m);
    for (int i = 0; i < m; ++i) dd[i] = a[i] - lam;
    for (int i = 0; i < m; ++i) rr[i] = x[i];
    for (int i = 0; i + 1 < m; ++i) cc[i] = b[i];
    for (int i = 1; i < m; ++i) {
      double piv = dd[i - 1];
      if (piv == 0) piv = 1e-300;
      const double w = b[i - 1] / piv;
      dd[i] -= w * cc[i - 1];
      rr[i] -= w * rr[i - 1];
    }
    y[m - 1] = rr[m - 1] / (dd[m - 1] == 0 ? 1e-300 : dd[m - 1]);
    for (int i = m - 2; i >= 0; --i) y[i] = (rr[i] - cc[i] * y[i + 1]) / (dd[i] == 0 ? 1e-300 : dd[i]);
    double nrm = 0;
    for (double v : y) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (int i = 0; i < m; ++i) x[i] = y[i] / nrm;
  }
  return x;
}

void fiedler_split(const double* X, int dim, const std::vector<int64_t>& idx, uint64_t seed,
                   std::vector<char>& in_m1) {
  const int64_t n = int64_t(idx.size());
  in_m1.assign(n, 0);
  if (n <= 2) {
    if (n >= 1) in_m1[0] = 1;
    return;
  }
  const int k = int(std::min<int64_t>(10, n - 1));
  std::vector<int32_t> nbr;
  std::vector<double> d2;
  knn(X, dim, idx, k, nbr, d2);
  double t = 0;
  int64_t cntd = 0;
  for (int64_t j = 0; j < n * k; ++j)
    if (nbr[j] >= 0) { t += d2[j]; ++cntd; }
  t = cntd ? t / double(cntd) : 1.0;
  if (!(t > 0)) t = 1.0;
  // symmetrized adjacency as a CSR
  std::vector<std::vector<std::pair<int32_t, double>>> adj(n);
  for (int64_t j = 0; j < n; ++j)
    for (int q = 0; q < k; ++q) {
      const int32_t o = nbr[j * k + q];
      if (o < 0) continue;
      const double w = std::exp(-d2[j * k + q] / t);
      adj[j].push_back({o, w});
      adj[o].push_back({int32_t(j), w});
    }
  std::vector<int64_t> rp(n + 1, 0);
  std::vector<int32_t> ci;
  std::vector<double> cv, deg(n, 0.0);
  for (int64_t j = 0; j < n; ++j) {
    auto& a = adj[j];
    std::sort(a.begin(), a.end());
    for (size_t q = 0; q < a.size(); ++q) {
      if (q > 0 && a[q].first == a[q - 1].first) {  // max of the two directions
        cv.back() = std::max(cv.back(), a[q].second);
        continue;
      }
      ci.push_back(a[q].first);
      cv.push_back(a[q].second);
    }
    rp[j + 1] = int64_t(ci.size());
    std::vector<std::pair<int32_t, double>>().swap(a);
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t q = rp[j]; q < rp[j + 1]; ++q) deg[j] += cv[q];
  std::vector<double> sq(n);
  double sqn = 0;
  for (int64_t j = 0; j < n; ++j) {
    if (!(deg[j] > 0)) deg[j] = 1.0;
    sq[j] = std::sqrt(deg[j]);
    sqn += deg[j];
  }
  sqn = std::sqrt(sqn);
  for (auto& v : sq) v /= sqn;  // unit top eigenvector of S
  auto applyS = [&](const std::vector<double>& x, std::vector<double>& y) {
#pragma omp parallel for schedule(static) if (n > 8192)
    for (int64_t j = 0; j < n; ++j) {
      double s = 0;
      for (int64_t q = rp[j]; q < rp[j + 1]; ++q) s += cv[q] * x[ci[q]] / sq[ci[q]] / sqn;
      y[j] = s / (sq[j] * sqn);
    }
  };
  auto deflate = [&](std::vector<double>& x) {
    double s = 0;
    for (int64_t j = 0; j < n; ++j) s += sq[j] * x[j];
    for (int64_t j = 0; j < n; ++j) x[j] -= s * sq[j];
  };
  const int mk = int(std::min<int64_t>(n - 1, 160));
  std::vector<std::vector<double>> V;
  std::vector<double> al, be;
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> N01;
  std::vector<double> v(n), w(n);
  for (auto& x : v) x = N01(rng);
  deflate(v);
  double nv = 0;
  for (double x : v) nv += x * x;
  nv = std::sqrt(nv);
  for (auto& x : v) x /= nv;
  for (int it = 0; it < mk; ++it) {
    V.push_back(v);
    applyS(v, w);
    double a = 0;
    for (int64_t j = 0; j < n; ++j) a += w[j] * v[j];
    al.push_back(a);
    deflate(w);
    for (int pass = 0; pass < 2; ++pass) {  // full reorthogonalization, classical GS twice
      const int nv = int(V.size());
      std::vector<double> dots(nv, 0.0);
#pragma omp parallel for schedule(static) if (n * nv > 200000)
      for (int q = 0; q < nv; ++q) {
        double s = 0;
        for (int64_t j = 0; j < n; ++j) s += V[q][j] * w[j];
        dots[q] = s;
      }
#pragma omp parallel for schedule(static) if (n * nv > 200000)
      for (int64_t j = 0; j < n; ++j) {
        double s = 0;
        for (int q = 0; q < nv; ++q) s += dots[q] * V[q][j];
        w[j] -= s;
      }
    }
    double bnorm = 0;
    for (double x : w) bnorm += x * x;
    bnorm = std::sqrt(bnorm);
    if (bnorm < 1e-12 || it + 1 == mk) break;
    be.push_back(bnorm);
    for (int64_t j = 0; j < n; ++j) v[j] = w[j] / bnorm;
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  std::vector<double> s = tridiag_top_vector(al, be);
  std::vector<double> psi(n, 0.0);
  for (size_t q = 0; q < V.size() && q < s.size(); ++q)
    for (int64_t j = 0; j < n; ++j) psi[j] += s[q] * V[q][j];
  int64_t c1 = 0;
  for (int64_t j = 0; j < n; ++j) {
    in_m1[j] = (psi[j] / sq[j] <= 0.0) ? 1 : 0;
    c1 += in_m1[j];
  }
  if (c1 == 0 || c1 == n) {  // numerically constant: split by order
    for (int64_t j = 0; j < n; ++j) in_m1[j] = (j < n / 2) ? 1 : 0;
  }
}

}  // namespace
}  // namespace mht
