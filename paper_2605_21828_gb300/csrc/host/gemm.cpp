// Small FP64 dense kernels for the host build: a packed, register-blocked GEMM.
//
//   C (m x n, ldc) = beta C + alpha op(A) B,   op(A) = A (m x k, lda) or A^T (A is k x m)
//
// Column-major throughout.  op(A) is packed into panels of kMR rows and B into panels of
// kNR columns, both contiguous along k, so the micro-kernel streams two short vectors per k
// step and keeps a kMR x kNR accumulator tile in registers (the compiler vectorizes the
// fixed-size loops; no intrinsics, so the same code builds for x86-64 and aarch64).
// Single-threaded: the build parallelizes across butterfly blocks.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mht {
namespace {

constexpr int kMR = 8, kNR = 4;
constexpr int kMC = 128, kKC = 256, kNC = 1024;

inline void micro_kernel(int kc, const double* __restrict Ap, const double* __restrict Bp, double* __restrict C,
                         int ldc, int mr, int nr, double alpha) {
  double acc[kNR][kMR];
  for (int j = 0; j < kNR; ++j)
    for (int i = 0; i < kMR; ++i) acc[j][i] = 0.0;
  for (int p = 0; p < kc; ++p) {
    const double* a = Ap + p * kMR;
    const double* b = Bp + p * kNR;
    for (int j = 0; j < kNR; ++j) {
      const double bj = b[j];
#pragma omp simd
      for (int i = 0; i < kMR; ++i) acc[j][i] += a[i] * bj;
    }
  }
  if (mr == kMR && nr == kNR) {
    for (int j = 0; j < kNR; ++j)
#pragma omp simd
      for (int i = 0; i < kMR; ++i) C[j * ldc + i] += alpha * acc[j][i];
  } else {
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < mr; ++i) C[j * ldc + i] += alpha * acc[j][i];
  }
}

}  // namespace

void gemm(bool transA, int m, int n, int k, double alpha, const double* A, int lda, const double* B, int ldb,
          double beta, double* C, int ldc) {
  if (m <= 0 || n <= 0) return;
  if (beta != 1.0)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < m; ++i) C[j * ldc + i] = (beta == 0.0) ? 0.0 : beta * C[j * ldc + i];
  if (k <= 0 || alpha == 0.0) return;
  thread_local std::vector<double> Ab, Bb;
  Ab.resize(size_t(kMC + kMR) * kKC);
  Bb.resize(size_t(kNC + kNR) * kKC);
  for (int j0 = 0; j0 < n; j0 += kNC) {
    const int nc = std::min(kNC, n - j0);
    for (int p0 = 0; p0 < k; p0 += kKC) {
      const int kc = std::min(kKC, k - p0);
      // pack B(p0:p0+kc, j0:j0+nc) into kNR-column panels
      for (int jp = 0; jp < nc; jp += kNR) {
        double* dst = Bb.data() + size_t(jp) * kc;
        const int nr = std::min(kNR, nc - jp);
        for (int p = 0; p < kc; ++p)
          for (int j = 0; j < kNR; ++j)
            dst[p * kNR + j] = (j < nr) ? B[size_t(j0 + jp + j) * ldb + p0 + p] : 0.0;
      }
      for (int i0 = 0; i0 < m; i0 += kMC) {
        const int mc = std::min(kMC, m - i0);
        // pack op(A)(i0:i0+mc, p0:p0+kc) into kMR-row panels
        for (int ip = 0; ip < mc; ip += kMR) {
          double* dst = Ab.data() + size_t(ip) * kc;
          const int mr = std::min(kMR, mc - ip);
          if (!transA) {
            for (int p = 0; p < kc; ++p) {
              const double* src = A + size_t(p0 + p) * lda + i0 + ip;
              for (int i = 0; i < kMR; ++i) dst[p * kMR + i] = (i < mr) ? src[i] : 0.0;
            }
          } else {
            for (int i = 0; i < kMR; ++i) {
              if (i < mr) {
                const double* src = A + size_t(i0 + ip + i) * lda + p0;
                for (int p = 0; p < kc; ++p) dst[p * kMR + i] = src[p];
              } else {
                for (int p = 0; p < kc; ++p) dst[p * kMR + i] = 0.0;
              }
            }
          }
        }
        for (int jp = 0; jp < nc; jp += kNR)
          for (int ip = 0; ip < mc; ip += kMR)
            micro_kernel(kc, Ab.data() + size_t(ip) * kc, Bb.data() + size_t(jp) * kc,
                         C + size_t(j0 + jp) * ldc + i0 + ip, ldc, std::min(kMR, mc - ip), std::min(kNR, nc - jp),
                         alpha);
      }
    }
  }
}

}  // namespace mht
