// Inverse transform: c = argmin ||Phi c - f||_2 by LSQR (Paige & Saunders 1982), the
// iterative least-squares solver the paper pairs with the fast transform (Sec. 7.1, Eq.
// inverse-MHT).  Every product with Phi and Phi^H is the butterfly apply; the LSQR vector
// updates are the small kernels below (per-column scalars, since each right-hand side runs its
// own recurrence).  The scalar recurrences (Givens rotations, stopping tests) run in FP64 on
// the host; column norms are reduced deterministically in FP64 on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../host/internal.h"

namespace mht {
namespace {

constexpr int kVecThreads = 256;
constexpr int kNormBlocks = 64;  // partial sums per column

// y[:, j] = a[j] x[:, j] + b[j] y[:, j] over `rows` scalars per column (complex: 2 per entry);
// b[j] == 0 does not read y, a[j] == 0 does not read x.
template <class R>
__global__ void k_axpby(const R* __restrict__ x, int64_t ldx, R* __restrict__ y, int64_t ldy, int64_t rows,
                        const double* __restrict__ a, const double* __restrict__ b) {
  const int j = blockIdx.y;
  const double aj = a[j], bj = b[j];
  const R* xc = x + j * ldx;
  R* yc = y + j * ldy;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows; i += int64_t(gridDim.x) * blockDim.x) {
    double v = 0.0;
    if (aj != 0.0) v = aj * double(xc[i]);
    if (bj != 0.0) v += bj * double(yc[i]);
    yc[i] = R(v);
  }
}

// partial[j * kNormBlocks + block] = sum of squares of a slice of column j
template <class R>
__global__ void k_sumsq_partial(const R* __restrict__ x, int64_t ldx, int64_t rows, double* __restrict__ partial) {
  __shared__ double red[kVecThreads / 32];
  const int j = blockIdx.y;
  const R* xc = x + j * ldx;
  double s = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = double(xc[i]);
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) t += red[w];
    partial[j * kNormBlocks + blockIdx.x] = t;
  }
}

__global__ void k_sumsq_final(const double* __restrict__ partial, double* __restrict__ out) {
  const int j = blockIdx.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < kNormBlocks; ++b) t += partial[j * kNormBlocks + b];
    out[j] = t;
  }
}

int ck(cudaError_t e, std::string& err, const char* what) {
  if (e == cudaSuccess) return 0;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return MHT_ERR_CUDA;
}

struct Scratch {
  uint8_t* u;        // n x k   left Lanczos vector
  uint8_t* an;       // n x k   A v
  uint8_t* v;        // m x k   right Lanczos vector
  uint8_t* w;        // m x k   search direction
  uint8_t* am;       // m x k   A^H u
  double* partial;   // k x kNormBlocks
  double* norms;     // k
  double* coef;      // 2 k: a then b of the next axpby
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

Scratch carve(uint8_t* base, int64_t n, int64_t m, int64_t k, int es) {
  Scratch s;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* p = base + off;
    off = al256(off + bytes);
    return p;
  };
  s.u = take(size_t(n) * k * es);
  s.an = take(size_t(n) * k * es);
  s.v = take(size_t(m) * k * es);
  s.w = take(size_t(m) * k * es);
  s.am = take(size_t(m) * k * es);
  s.partial = reinterpret_cast<double*>(take(size_t(k) * kNormBlocks * sizeof(double)));
  s.norms = reinterpret_cast<double*>(take(size_t(k) * sizeof(double)));
  s.coef = reinterpret_cast<double*>(take(size_t(2) * k * sizeof(double)));
  return s;
}

template <class R>
struct Ops {
  cudaStream_t st;
  int64_t k;
  int W;
  std::string& err;
  std::vector<double> host;  // staging of a / b for uploads
  double* coef;
  double* partial;
  double* norms;

  int axpby(const void* x, int64_t ldx, void* y, int64_t ldy, int64_t rows, const std::vector<double>& a,
            const std::vector<double>& b) {
    host.assign(a.begin(), a.end());
    host.insert(host.end(), b.begin(), b.end());
    if (int rc = ck(cudaMemcpyAsync(coef, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, st), err,
                    "lsqr scalars"))
      return rc;
    const int64_t r = rows * W;
    dim3 grid(unsigned(std::min<int64_t>((r + kVecThreads - 1) / kVecThreads, 1024)), unsigned(k));
    k_axpby<R><<<grid, kVecThreads, 0, st>>>(static_cast<const R*>(x), ldx * W, static_cast<R*>(y), ldy * W, r, coef,
                                             coef + k);
    return ck(cudaGetLastError(), err, "lsqr axpby");
  }
  // column norms (FP64), synchronizes the stream
  int norm(const void* x, int64_t ldx, int64_t rows, std::vector<double>& out) {
    dim3 grid(kNormBlocks, unsigned(k));
    k_sumsq_partial<R><<<grid, kVecThreads, 0, st>>>(static_cast<const R*>(x), ldx * W, rows * W, partial);
    k_sumsq_final<<<unsigned(k), 32, 0, st>>>(partial, norms);
    if (int rc = ck(cudaGetLastError(), err, "lsqr norm")) return rc;
    out.resize(k);
    if (int rc = ck(cudaMemcpyAsync(out.data(), norms, k * sizeof(double), cudaMemcpyDeviceToHost, st), err,
                    "lsqr norm read"))
      return rc;
    if (int rc = ck(cudaStreamSynchronize(st), err, "lsqr sync")) return rc;
    for (double& v : out) v = std::sqrt(v);
    return 0;
  }
};

template <class R>
int lsqr(const Factorization& F, const Packed& P, const DeviceView& d, const void* f, int64_t ldf, void* c, int64_t ldc,
         int64_t k, uint8_t* scratch, int max_iter, double tol, mht_apply_mode mode, cudaStream_t st, int* iters,
         double* relres, std::string& err) {
  const int64_t n = F.n, m = F.m;
  const Scratch s = carve(scratch, n, m, k, P.elem_bytes);
  Ops<R> op{st, k, P.cplx ? 2 : 1, err, {}, s.coef, s.partial, s.norms};
  const std::vector<double> one(k, 1.0), zero(k, 0.0);
  std::vector<double> alpha, beta, beta1, a(k), b(k);
  // beta u = f ; x = 0
  if (int rc = op.axpby(f, ldf, s.u, n, n, one, zero)) return rc;
  if (int rc = op.axpby(c, ldc, c, ldc, m, zero, zero)) return rc;
  if (int rc = op.norm(s.u, n, n, beta)) return rc;
  beta1 = beta;
  for (int64_t j = 0; j < k; ++j) a[j] = beta[j] > 0 ? 1.0 / beta[j] : 0.0;
  if (int rc = op.axpby(s.u, n, s.u, n, n, a, zero)) return rc;
  // alpha v = A^H u ; w = v
  if (int rc = apply_analyze(F, P, d, s.u, n, s.am, m, k, false, mode, st, err)) return rc;
  if (int rc = op.axpby(s.am, m, s.v, m, m, one, zero)) return rc;
  if (int rc = op.norm(s.v, m, m, alpha)) return rc;
  for (int64_t j = 0; j < k; ++j) a[j] = alpha[j] > 0 ? 1.0 / alpha[j] : 0.0;
  if (int rc = op.axpby(s.v, m, s.v, m, m, a, zero)) return rc;
  if (int rc = op.axpby(s.v, m, s.w, m, m, one, zero)) return rc;

  std::vector<double> phibar = beta, rhobar = alpha, anorm2(k, 0.0), rnorm = beta;
  std::vector<char> done(k, 0);
  for (int64_t j = 0; j < k; ++j) done[j] = (beta[j] == 0.0 || alpha[j] == 0.0);  // x = 0 is exact
  int it = 0;
  for (; it < max_iter; ++it) {
    if (std::all_of(done.begin(), done.end(), [](char v) { return v != 0; })) break;
    // beta u = A v - alpha u
    if (int rc = apply_synthesize(F, P, d, s.v, m, s.an, n, k, false, mode, st, err)) return rc;
    for (int64_t j = 0; j < k; ++j) b[j] = -alpha[j];
    if (int rc = op.axpby(s.an, n, s.u, n, n, one, b)) return rc;
    std::vector<double> bnew;
    if (int rc = op.norm(s.u, n, n, bnew)) return rc;
    for (int64_t j = 0; j < k; ++j) a[j] = bnew[j] > 0 ? 1.0 / bnew[j] : 0.0;
    if (int rc = op.axpby(s.u, n, s.u, n, n, a, zero)) return rc;
    // alpha v = A^H u - beta v
    if (int rc = apply_analyze(F, P, d, s.u, n, s.am, m, k, false, mode, st, err)) return rc;
    for (int64_t j = 0; j < k; ++j) b[j] = -bnew[j];
    if (int rc = op.axpby(s.am, m, s.v, m, m, one, b)) return rc;
    std::vector<double> anew;
    if (int rc = op.norm(s.v, m, m, anew)) return rc;
    for (int64_t j = 0; j < k; ++j) a[j] = anew[j] > 0 ? 1.0 / anew[j] : 0.0;
    if (int rc = op.axpby(s.v, m, s.v, m, m, a, zero)) return rc;
    // plane rotation; x += (phi / rho) w ; w = v - (theta / rho) w   (frozen columns: no change)
    std::vector<double> xa(k, 0.0), wb(k, 1.0), wa(k, 0.0);
    for (int64_t j = 0; j < k; ++j) {
      anorm2[j] += alpha[j] * alpha[j] + bnew[j] * bnew[j];
      if (done[j]) continue;
      const double rho = std::hypot(rhobar[j], bnew[j]);
      const double cs = rhobar[j] / rho, sn = bnew[j] / rho;
      const double theta = sn * anew[j];
      rhobar[j] = -cs * anew[j];
      const double phi = cs * phibar[j];
      phibar[j] = sn * phibar[j];
      xa[j] = phi / rho;
      wa[j] = 1.0;
      wb[j] = -theta / rho;
      rnorm[j] = phibar[j];
      // stopping tests: small residual, or small normal-equation residual |A^H r| / (|A| |r|)
      const double arnorm = phibar[j] * anew[j] * std::fabs(cs);
      const double an = std::sqrt(anorm2[j]);
      if (phibar[j] <= tol * beta1[j] || (an > 0 && phibar[j] > 0 && arnorm <= tol * an * phibar[j])) done[j] = 1;
    }
    if (int rc = op.axpby(s.w, m, c, ldc, m, xa, one)) return rc;
    if (int rc = op.axpby(s.v, m, s.w, m, m, wa, wb)) return rc;
    alpha = anew;
  }
  if (iters) *iters = it;
  if (relres) {
    double worst = 0.0;
    for (int64_t j = 0; j < k; ++j) worst = std::max(worst, beta1[j] > 0 ? rnorm[j] / beta1[j] : 0.0);
    *relres = worst;
  }
  return ck(cudaStreamSynchronize(st), err, "lsqr sync");
}

}  // namespace

size_t lsqr_scratch_bytes(const Packed& P, int64_t n, int64_t m, int64_t k) {
  const int es = P.elem_bytes;
  return 2 * al256(size_t(n) * k * es) + 3 * al256(size_t(m) * k * es) + al256(size_t(k) * kNormBlocks * 8) +
         al256(size_t(k) * 8) + al256(size_t(2) * k * 8);
}

int apply_lsqr(const Factorization& F, const Packed& P, const DeviceView& d, const void* f, int64_t ldf, void* c,
               int64_t ldc, int64_t k, void* scratch, int max_iter, double tol, mht_apply_mode mode, void* stream,
               int* iters, double* relres, std::string& err) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* s = static_cast<uint8_t*>(scratch);
  return P.fp64 ? lsqr<double>(F, P, d, f, ldf, c, ldc, k, s, max_iter, tol, mode, st, iters, relres, err)
                : lsqr<float>(F, P, d, f, ldf, c, ldc, k, s, max_iter, tol, mode, st, iters, relres, err);
}

}  // namespace mht
