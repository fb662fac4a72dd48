// Small FP64 dense kernels for the host build: a packed, register-blocked GEMM (real and
// complex).
//
//   C (m x n, ldc) = beta C + alpha op(A) B,   op(A) = A (m x k, lda) or A^T (A is k x m)
//
// Column-major throughout.  op(A) is packed into panels of kMR rows and B into panels of
// kNR columns, both contiguous along k, so the micro-kernel streams two short vectors per k
// step and keeps a kMR x kNR accumulator tile in registers (the compiler vectorizes the
// fixed-size loops; no intrinsics, so the same code builds for x86-64 and aarch64).
// Single-threaded: the build parallelizes across butterfly blocks.
#include <algorithm>
#include <complex>
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

// Complex variant, interleaved (re, im) storage:
//
//   C (m x n, ldc) = beta C + alpha op(A) B,   op(A) = A (m x k, lda) or A^H (A is k x m)
//
// Same blocking; the panels are split into real and imaginary planes when packed (A^H is
// conjugated there), and the micro-kernel keeps separate real and imaginary accumulators,
// four real FMAs per complex multiply-add.
namespace {

constexpr int kZMR = 8, kZNR = 2;
constexpr int kZMC = 128, kZKC = 128, kZNC = 512;
using cd = std::complex<double>;

inline void zmicro_kernel(int kc, const double* __restrict Ar, const double* __restrict Ai,
                          const double* __restrict Br, const double* __restrict Bi, cd* C, int ldc, int mr,
                          int nr, cd alpha) {
  double sr[kZNR][kZMR], si[kZNR][kZMR];
  for (int j = 0; j < kZNR; ++j)
    for (int i = 0; i < kZMR; ++i) sr[j][i] = si[j][i] = 0.0;
  for (int p = 0; p < kc; ++p) {
    const double* ar = Ar + p * kZMR;
    const double* ai = Ai + p * kZMR;
    for (int j = 0; j < kZNR; ++j) {
      const double br = Br[p * kZNR + j], bi = Bi[p * kZNR + j];
#pragma omp simd
      for (int i = 0; i < kZMR; ++i) {
        sr[j][i] += ar[i] * br - ai[i] * bi;
        si[j][i] += ar[i] * bi + ai[i] * br;
      }
    }
  }
  for (int j = 0; j < nr; ++j)
    for (int i = 0; i < mr; ++i) C[j * ldc + i] += alpha * cd(sr[j][i], si[j][i]);
}

}  // namespace

void zgemm(bool conjTransA, int m, int n, int k, cd alpha, const cd* A, int lda, const cd* B, int ldb, cd beta,
           cd* C, int ldc) {
  if (m <= 0 || n <= 0) return;
  if (beta != cd(1.0))
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < m; ++i) C[j * ldc + i] = (beta == cd(0.0)) ? cd(0.0) : beta * C[j * ldc + i];
  if (k <= 0 || alpha == cd(0.0)) return;
  thread_local std::vector<double> Ab, Bb;
  const size_t apl = size_t(kZMC + kZMR) * kZKC, bpl = size_t(kZNC + kZNR) * kZKC;
  Ab.resize(2 * apl);
  Bb.resize(2 * bpl);
  for (int j0 = 0; j0 < n; j0 += kZNC) {
    const int nc = std::min(kZNC, n - j0);
    for (int p0 = 0; p0 < k; p0 += kZKC) {
      const int kc = std::min(kZKC, k - p0);
      for (int jp = 0; jp < nc; jp += kZNR) {
        double* dr = Bb.data() + size_t(jp) * kc;
        double* di = dr + bpl;
        const int nr = std::min(kZNR, nc - jp);
        for (int p = 0; p < kc; ++p)
          for (int j = 0; j < kZNR; ++j) {
            const cd v = (j < nr) ? B[size_t(j0 + jp + j) * ldb + p0 + p] : cd(0.0);
            dr[p * kZNR + j] = v.real();
            di[p * kZNR + j] = v.imag();
          }
      }
      for (int i0 = 0; i0 < m; i0 += kZMC) {
        const int mc = std::min(kZMC, m - i0);
        for (int ip = 0; ip < mc; ip += kZMR) {
          double* dr = Ab.data() + size_t(ip) * kc;
          double* di = dr + apl;
          const int mr = std::min(kZMR, mc - ip);
          if (!conjTransA) {
            for (int p = 0; p < kc; ++p) {
              const cd* src = A + size_t(p0 + p) * lda + i0 + ip;
              for (int i = 0; i < kZMR; ++i) {
                const cd v = (i < mr) ? src[i] : cd(0.0);
                dr[p * kZMR + i] = v.real();
                di[p * kZMR + i] = v.imag();
              }
            }
          } else {
            for (int i = 0; i < kZMR; ++i) {
              const cd* src = (i < mr) ? A + size_t(i0 + ip + i) * lda + p0 : nullptr;
              for (int p = 0; p < kc; ++p) {
                const cd v = src ? std::conj(src[p]) : cd(0.0);
                dr[p * kZMR + i] = v.real();
                di[p * kZMR + i] = v.imag();
              }
            }
          }
        }
        for (int jp = 0; jp < nc; jp += kZNR)
          for (int ip = 0; ip < mc; ip += kZMR)
            zmicro_kernel(kc, Ab.data() + size_t(ip) * kc, Ab.data() + apl + size_t(ip) * kc,
                          Bb.data() + size_t(jp) * kc, Bb.data() + bpl + size_t(jp) * kc,
                          C + size_t(j0 + jp) * ldc + i0 + ip, ldc, std::min(kZMR, mc - ip),
                          std::min(kZNR, nc - jp), alpha);
      }
    }
  }
}

}  // namespace mht
