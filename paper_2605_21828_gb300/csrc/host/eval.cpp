// Entries of the transform matrix Phi_jk = phi_k(x_j) (Sec. 1, Eq. MHT-sum) for the build.
//
// Built-in closed forms: complex exponentials on the flat periodic square (Eq. 2D-DFT) and
// orthonormal real spherical harmonics on the unit sphere; plus a dense FP64 matrix and a
// user callback for numerically computed eigenfunctions.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>
#include <memory>

#include "internal.h"

namespace mht {
namespace {

struct CallbackEval : Evaluator {
  mht_eval_fn fn;
  void* ctx;
  CallbackEval(mht_eval_fn f, void* c) : fn(f), ctx(c) {}
  void eval(const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
            double* out) const override {
    if (nr == 0 || nc == 0) return;
    if (fn(ctx, rows, nr, cols, nc, out) != 0)
      fail(MHT_ERR_CALLBACK, "Phi evaluator callback returned an error");
  }
};

struct DenseEval : Evaluator {
  const double* A;
  int64_t ld;
  bool cplx;
  DenseEval(const double* a, int64_t l, bool c) : A(a), ld(l), cplx(c) {}
  void eval(const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
            double* out) const override {
    for (int64_t j = 0; j < nc; ++j) {
      if (cplx) {
        const double* col = A + 2 * cols[j] * ld;
        for (int64_t i = 0; i < nr; ++i) {
          out[2 * (j * nr + i)] = col[2 * rows[i]];
          out[2 * (j * nr + i) + 1] = col[2 * rows[i] + 1];
        }
      } else {
        const double* col = A + cols[j] * ld;
        for (int64_t i = 0; i < nr; ++i) out[j * nr + i] = col[rows[i]];
      }
    }
  }
};

// phi_k(x) = exp(i (k1 x1 + k2 x2)).
struct TorusEval : Evaluator {
  const double* X;
  const int64_t* K;
  TorusEval(const double* x, const int64_t* k) : X(x), K(k) {}
  void eval(const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
            double* out) const override {
    for (int64_t j = 0; j < nc; ++j) {
      const double k1 = double(K[2 * cols[j]]), k2 = double(K[2 * cols[j] + 1]);
      double* o = out + 2 * j * nr;
      for (int64_t i = 0; i < nr; ++i) {
        const double t = k1 * X[2 * rows[i]] + k2 * X[2 * rows[i] + 1];
        o[2 * i] = std::cos(t);
        o[2 * i + 1] = std::sin(t);
      }
    }
  }
};

// Orthonormal real spherical harmonics, column k = l^2 + l + mm.  The fully normalized
// associated Legendre functions Pbar_l^|mm| come from the standard recurrences
//   Pbar_0^0 = 1/sqrt(4 pi),  Pbar_mm^mm = sqrt((2mm+1)/(2mm)) sin(t) Pbar_{mm-1}^{mm-1},
//   Pbar_{mm+1}^mm = sqrt(2mm+3) z Pbar_mm^mm,
//   Pbar_l^mm = a (z Pbar_{l-1}^mm - b Pbar_{l-2}^mm),
//   a = sqrt((4l^2-1)/(l^2-mm^2)),  b = sqrt(((l-1)^2-mm^2)/(4(l-1)^2-1)),
// run vectorized over the rows for each order |mm| present among the requested columns.
struct SphereEval : Evaluator {
  int64_t n;
  std::vector<double> z, s, lon;
  SphereEval(const double* X, int64_t n_) : n(n_), z(n_), s(n_), lon(n_) {
    for (int64_t i = 0; i < n; ++i) {
      const double x = X[3 * i], y = X[3 * i + 1], w = X[3 * i + 2];
      const double r = std::sqrt(x * x + y * y + w * w);
      z[i] = w / r;
      s[i] = std::sqrt(std::fmax(0.0, 1.0 - z[i] * z[i]));
      lon[i] = std::atan2(y, x);
    }
  }
  // Rows are processed in chunks so the recurrence arrays stay in L1.
  void eval(const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
            double* out) const override {
    constexpr int64_t kChunk = 256;
    if (nr <= kChunk) {
      eval_chunk(rows, nr, cols, nc, out, nr);
      return;
    }
    for (int64_t r0 = 0; r0 < nr; r0 += kChunk)
      eval_chunk(rows + r0, std::min(kChunk, nr - r0), cols, nc, out + r0, nr);
  }
  // out(i, j) at out[j * ld + i]
  void eval_chunk(const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc, double* out,
                  int64_t ld) const {
    if (nr == 0 || nc == 0) return;
    // group requested columns by order |mm|: (l, signed mm, output column)
    std::map<int64_t, std::vector<std::array<int64_t, 3>>> groups;
    for (int64_t j = 0; j < nc; ++j) {
      const int64_t k = cols[j];
      int64_t l = int64_t(std::sqrt(double(k)));
      while (l * l > k) --l;
      while ((l + 1) * (l + 1) <= k) ++l;
      const int64_t mm = k - l * l - l;
      groups[mm < 0 ? -mm : mm].push_back({l, mm, j});
    }
    std::vector<double> zr(nr), sr(nr), pmm(nr), p1(nr), p2(nr), cosm(nr), sinm(nr);
    for (int64_t i = 0; i < nr; ++i) {
      zr[i] = z[rows[i]];
      sr[i] = s[rows[i]];
    }
    const double root2 = std::sqrt(2.0);
    // The orders are visited in increasing |mm| (std::map order), so Pbar_am^am continues from
    // the previous order's product, and cos / sin(am lon) advance by one rotation through lon
    // when am is the next order; they are recomputed directly every 16 orders and after a gap,
    // which bounds the rotations' rounding to a few ulps.
    std::vector<double> c1(nr), s1(nr);
    for (int64_t i = 0; i < nr; ++i) {
      pmm[i] = 1.0 / std::sqrt(4.0 * M_PI);
      c1[i] = std::cos(lon[rows[i]]);
      s1[i] = std::sin(lon[rows[i]]);
    }
    int64_t am_prev = -2;
    for (auto& kv : groups) {
      const int64_t am = kv.first;
      auto& list = kv.second;
      int64_t lmax = 0;
      for (auto& e : list) lmax = std::max(lmax, e[0]);
      for (int64_t k = std::max<int64_t>(am_prev, 0) + 1; k <= am; ++k) {
        const double f = std::sqrt((2.0 * k + 1.0) / (2.0 * k));
        for (int64_t i = 0; i < nr; ++i) pmm[i] *= f * sr[i];
      }
      if (am == am_prev + 1 && am % 16 != 0) {
        for (int64_t i = 0; i < nr; ++i) {
          const double cn = cosm[i] * c1[i] - sinm[i] * s1[i];
          sinm[i] = sinm[i] * c1[i] + cosm[i] * s1[i];
          cosm[i] = cn;
        }
      } else {
        for (int64_t i = 0; i < nr; ++i) {
          cosm[i] = std::cos(double(am) * lon[rows[i]]);
          sinm[i] = std::sin(double(am) * lon[rows[i]]);
        }
      }
      am_prev = am;
      // emit columns as the recurrence passes their degree
      std::sort(list.begin(), list.end());
      size_t next = 0;
      auto emit = [&](int64_t l, const double* P) {
        while (next < list.size() && list[next][0] == l) {
          const int64_t mm = list[next][1];
          double* o = out + list[next][2] * ld;
          if (mm == 0)
            for (int64_t i = 0; i < nr; ++i) o[i] = P[i];
          else if (mm > 0)
            for (int64_t i = 0; i < nr; ++i) o[i] = root2 * P[i] * cosm[i];
          else
            for (int64_t i = 0; i < nr; ++i) o[i] = root2 * P[i] * sinm[i];
          ++next;
        }
      };
      emit(am, pmm.data());
      if (lmax == am) continue;
      const double a1 = std::sqrt(2.0 * am + 3.0);
      for (int64_t i = 0; i < nr; ++i) {
        p2[i] = pmm[i];
        p1[i] = a1 * zr[i] * pmm[i];
      }
      emit(am + 1, p1.data());
      // Pbar_{l-1} in *cur, Pbar_{l-2} in *prev; each step overwrites the older one in place
      double* cur = p1.data();
      double* prev = p2.data();
      const double* z = zr.data();
      for (int64_t l = am + 2; l <= lmax; ++l) {
        const double dl = double(l), dm = double(am);
        const double a = std::sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
        const double b = std::sqrt(((dl - 1) * (dl - 1) - dm * dm) / (4.0 * (dl - 1) * (dl - 1) - 1.0));
#pragma omp simd
        for (int64_t i = 0; i < nr; ++i) prev[i] = a * (z[i] * cur[i] - b * prev[i]);
        std::swap(cur, prev);
        if (next < list.size() && list[next][0] == l) emit(l, cur);
      }
    }
  }
};

}  // namespace

Evaluator* make_evaluator(const mht_problem& p) {
  switch (p.eval_kind) {
    case MHT_EVAL_CALLBACK:
      if (!p.eval) fail(MHT_ERR_INVALID_ARG, "MHT_EVAL_CALLBACK needs problem->eval");
      return new CallbackEval(p.eval, p.eval_ctx);
    case MHT_EVAL_DENSE:
      if (!p.dense || p.ld_dense < p.n) fail(MHT_ERR_INVALID_ARG, "MHT_EVAL_DENSE needs dense and ld_dense >= n");
      return new DenseEval(p.dense, p.ld_dense, p.field == MHT_COMPLEX);
    case MHT_EVAL_TORUS:
      if (!p.points || p.dim != 2 || !p.torus_modes || p.field != MHT_COMPLEX)
        fail(MHT_ERR_INVALID_ARG, "MHT_EVAL_TORUS needs 2-D points, torus_modes and a complex field");
      return new TorusEval(p.points, p.torus_modes);
    case MHT_EVAL_SPHERE:
      if (!p.points || p.dim != 3 || p.field != MHT_REAL)
        fail(MHT_ERR_INVALID_ARG, "MHT_EVAL_SPHERE needs 3-D points and a real field");
      return new SphereEval(p.points, p.n);
  }
  fail(MHT_ERR_INVALID_ARG, "unknown eval_kind");
}

}  // namespace mht
