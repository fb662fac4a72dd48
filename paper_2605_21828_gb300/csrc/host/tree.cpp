// Row (space) and column (frequency) trees of the butterfly (Sec. 2 and Sec. 3).
//
// Both trees are complete binary trees of the same depth L.  Nodes are contiguous ranges
// of a permutation; only the leaf offsets are stored (a node at depth d, index i, covers
// leaves [i 2^(L-d), (i+1) 2^(L-d))).  Space nodes may be empty.
#include <algorithm>
#include <cmath>
#include <functional>
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
  std::vector<int64_t> tris;  // FIEDLER_MESH: the node's triangles (patches)
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
void fiedler_split_mesh(const double* X, const int64_t* tris, const Node& nd, uint64_t seed, Node& c1,
                        Node& c2);

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
    kind = (p.eval_kind == MHT_EVAL_TORUS) ? MHT_TREE_RECT : (p.tris ? MHT_TREE_FIEDLER_MESH : MHT_TREE_FIEDLER);
  if (!p.points) fail(MHT_ERR_INVALID_ARG, "space tree needs problem->points");
  if (kind == MHT_TREE_RECT && p.dim != 2) fail(MHT_ERR_INVALID_ARG, "MHT_TREE_RECT needs 2-D points");
  if (kind == MHT_TREE_FIEDLER_MESH) {
    if (!p.tris || p.ntris <= 0) fail(MHT_ERR_INVALID_ARG, "MHT_TREE_FIEDLER_MESH needs problem->tris");
    if (p.dim != 3) fail(MHT_ERR_INVALID_ARG, "MHT_TREE_FIEDLER_MESH needs 3-D points (the mesh vertices)");
    for (int64_t j = 0; j < 3 * p.ntris; ++j)
      if (p.tris[j] < 0 || p.tris[j] >= n) fail(MHT_ERR_INVALID_ARG, "triangle vertex index out of range");
  }
  std::vector<Node> cur(1);
  cur[0].idx.resize(n);
  std::iota(cur[0].idx.begin(), cur[0].idx.end(), int64_t(0));
  cur[0].periodic_root = true;
  if (kind == MHT_TREE_FIEDLER_MESH) {
    cur[0].tris.resize(p.ntris);
    std::iota(cur[0].tris.begin(), cur[0].tris.end(), int64_t(0));
  }
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
      } else if (kind == MHT_TREE_FIEDLER_MESH) {
        fiedler_split_mesh(p.points, p.tris, nd, seed + uint64_t(d) * 1000003ull + uint64_t(i), c1, c2);
        std::vector<int64_t>().swap(nd.tris);
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

// Unit vector of the largest eigenvalue of the symmetric operator `op` on the orthogonal
// complement of the unit vector q (an eigenvector of op): Lanczos from a seeded Gaussian
// start, deflated against q and fully reorthogonalized (classical Gram-Schmidt twice) at every
// step, at most mk steps (stops early when the residual norm falls below `tiny`); returns the
// Ritz vector of the largest Ritz value.  When q's eigenvalue dominates the spectrum (the
// shifted FEM operator), the rounding-level q component that the Gram-Schmidt pass brings
// back grows by that ratio every step, so `redeflate` deflates once more after it.
std::vector<double> lanczos_top(int64_t n, const std::function<void(const std::vector<double>&, std::vector<double>&)>& op,
                                const std::vector<double>& q, uint64_t seed, int mk_max, double tiny,
                                bool redeflate = false) {
  auto deflate = [&](std::vector<double>& x) {
    double s = 0;
    for (int64_t j = 0; j < n; ++j) s += q[j] * x[j];
    for (int64_t j = 0; j < n; ++j) x[j] -= s * q[j];
  };
  const int mk = int(std::min<int64_t>(n - 1, mk_max));
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
    op(v, w);
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
    if (redeflate) deflate(w);
    double bnorm = 0;
    for (double x : w) bnorm += x * x;
    bnorm = std::sqrt(bnorm);
    if (bnorm < tiny || it + 1 == mk) break;
    be.push_back(bnorm);
    for (int64_t j = 0; j < n; ++j) v[j] = w[j] / bnorm;
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  std::vector<double> s = tridiag_top_vector(al, be);
  std::vector<double> psi(n, 0.0);
  for (size_t q = 0; q < V.size() && q < s.size(); ++q)
    for (int64_t j = 0; j < n; ++j) psi[j] += s[q] * V[q][j];
  return psi;
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
  const std::vector<double> psi = lanczos_top(n, applyS, sq, seed, 160, 1e-12);
  int64_t c1 = 0;
  for (int64_t j = 0; j < n; ++j) {
    in_m1[j] = (psi[j] / sq[j] <= 0.0) ? 1 : 0;
    c1 += in_m1[j];
  }
  if (c1 == 0 || c1 == n) {  // numerically constant: split by order
    for (int64_t j = 0; j < n; ++j) in_m1[j] = (j < n / 2) ? 1 : 0;
  }
}

// ---- patch rule of Algorithm 2 on a triangle mesh (Sec. 3) --------------------------------
// The node's sub-mesh is the union of its triangles; its vertices are the FEM nodes.  P1
// cotangent stiffness K (for the corner c of a triangle opposite edge (a, b): K_ab -= cot/2,
// K_aa, K_bb += cot/2) and barycentric lumped mass m (area / 3 per corner); no boundary term,
// which is the homogeneous Neumann condition of Eq. neumann-eigenproblem.  phi_2 solves
// K phi = lambda_2 M phi: psi = M^(1/2) phi is the top eigenvector of sigma I - M^(-1/2) K M^(-1/2)
// (sigma = its Gershgorin bound) on the complement of M^(1/2) 1 (the null vector).  Triangle P
// goes to M_1 when area(P) / 3 x (phi_2(a) + phi_2(b) + phi_2(c)) <= 0 (the exact integral of
// the P1 function); a point goes to M_1's side when it is a vertex of a triangle of M_1.
void fiedler_split_mesh(const double* X, const int64_t* tris, const Node& nd, uint64_t seed, Node& c1,
                        Node& c2) {
  const int64_t nt = int64_t(nd.tris.size());
  if (nt == 0 || nd.idx.empty()) {  // nothing to cut: points by order, triangles to the first child
    for (size_t j = 0; j < nd.idx.size(); ++j) (j < nd.idx.size() / 2 ? c1 : c2).idx.push_back(nd.idx[j]);
    c1.tris = nd.tris;
    return;
  }
  // local vertex numbering of the sub-mesh
  std::vector<int64_t> verts;
  verts.reserve(size_t(nt) * 3);
  for (int64_t t : nd.tris)
    for (int c = 0; c < 3; ++c) verts.push_back(tris[3 * t + c]);
  std::sort(verts.begin(), verts.end());
  verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
  const int64_t nv = int64_t(verts.size());
  auto local = [&](int64_t g) { return int64_t(std::lower_bound(verts.begin(), verts.end(), g) - verts.begin()); };
  std::vector<int64_t> lt(size_t(nt) * 3);
  std::vector<double> area(nt), mass(nv, 0.0);
  std::vector<std::vector<std::pair<int64_t, double>>> adj(nv);
  for (int64_t e = 0; e < nt; ++e) {
    const int64_t t = nd.tris[e];
    for (int c = 0; c < 3; ++c) lt[3 * e + c] = local(tris[3 * t + c]);
    const double* P[3] = {X + 3 * tris[3 * t], X + 3 * tris[3 * t + 1], X + 3 * tris[3 * t + 2]};
    double u[3], v[3], cr[3];
    for (int d = 0; d < 3; ++d) {
      u[d] = P[1][d] - P[0][d];
      v[d] = P[2][d] - P[0][d];
    }
    cr[0] = u[1] * v[2] - u[2] * v[1];
    cr[1] = u[2] * v[0] - u[0] * v[2];
    cr[2] = u[0] * v[1] - u[1] * v[0];
    area[e] = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int c = 0; c < 3; ++c) mass[lt[3 * e + c]] += area[e] / 3.0;
    for (int c = 0; c < 3; ++c) {  // corner c opposite edge (a, b)
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      double x[3], y[3], dot = 0;
      for (int d = 0; d < 3; ++d) {
        x[d] = P[a][d] - P[c][d];
        y[d] = P[b][d] - P[c][d];
        dot += x[d] * y[d];
      }
      const double twice_area = 2.0 * area[e];
      if (!(twice_area > 0)) continue;
      const double w = 0.5 * dot / twice_area;  // cot(angle at c) / 2
      const int64_t la = lt[3 * e + a], lb = lt[3 * e + b];
      adj[la].push_back({lb, -w});
      adj[lb].push_back({la, -w});
      adj[la].push_back({la, w});
      adj[lb].push_back({lb, w});
    }
  }
  // CSR of K with duplicates summed
  std::vector<int64_t> rp(nv + 1, 0), ci;
  std::vector<double> cv;
  for (int64_t i = 0; i < nv; ++i) {
    auto& a = adj[i];
    std::sort(a.begin(), a.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t q = 0; q < a.size(); ++q) {
      if (q > 0 && a[q].first == a[q - 1].first) {
        cv.back() += a[q].second;
        continue;
      }
      ci.push_back(a[q].first);
      cv.push_back(a[q].second);
    }
    rp[i + 1] = int64_t(ci.size());
    std::vector<std::pair<int64_t, double>>().swap(a);
  }
  std::vector<double> rs(nv), q(nv);  // M^(-1/2), unit M^(1/2) 1
  double qn = 0;
  for (int64_t i = 0; i < nv; ++i) {
    if (!(mass[i] > 0)) mass[i] = 1e-300;
    rs[i] = 1.0 / std::sqrt(mass[i]);
    q[i] = std::sqrt(mass[i]);
    qn += mass[i];
  }
  qn = std::sqrt(qn);
  for (auto& x : q) x /= qn;
  double sigma = 0;  // Gershgorin bound of S = M^(-1/2) K M^(-1/2)
  for (int64_t i = 0; i < nv; ++i) {
    double r = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) r += std::fabs(cv[k]) * rs[i] * rs[ci[k]];
    sigma = std::max(sigma, r);
  }
  if (!(sigma > 0)) sigma = 1.0;
  auto op = [&](const std::vector<double>& x, std::vector<double>& y) {  // y = sigma x - S x
#pragma omp parallel for schedule(static) if (nv > 8192)
    for (int64_t i = 0; i < nv; ++i) {
      double s = 0;
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += cv[k] * rs[ci[k]] * x[ci[k]];
      y[i] = sigma * x[i] - rs[i] * s;
    }
  };
  const std::vector<double> psi = lanczos_top(nv, op, q, seed, 240, 1e-12 * sigma, true);
  std::vector<char> vert_m1(nv, 0);
  for (int64_t e = 0; e < nt; ++e) {
    double s = 0;
    for (int c = 0; c < 3; ++c) s += psi[lt[3 * e + c]] * rs[lt[3 * e + c]];
    const bool m1 = area[e] / 3.0 * s <= 0.0;
    (m1 ? c1 : c2).tris.push_back(nd.tris[e]);
    if (m1)
      for (int c = 0; c < 3; ++c) vert_m1[lt[3 * e + c]] = 1;
  }
  for (int64_t g : nd.idx) {
    const int64_t i = local(g);
    const bool in = i < nv && verts[i] == g && vert_m1[i];
    (in ? c1 : c2).idx.push_back(g);
  }
  if (c1.idx.empty() || c2.idx.empty()) {  // numerically constant: points by order
    c1.idx.clear();
    c2.idx.clear();
    for (size_t j = 0; j < nd.idx.size(); ++j) (j < nd.idx.size() / 2 ? c1 : c2).idx.push_back(nd.idx[j]);
  }
}

}  // namespace
}  // namespace mht
