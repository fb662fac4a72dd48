// Multi-RHS block products on the 5th-generation tensor cores (tcgen05), 3xTF32.
//
// With k right-hand sides every butterfly block product becomes a GEMM: M = rows of the
// stored matrix (T~ or U, or their transposes for the adjoint), N = k, K = its columns.  FP32
// accuracy on TF32 tensor cores comes from splitting both operands, x = hi + lo with
// hi = tf32(x) and lo = tf32(x - hi), and accumulating hi*hi + hi*lo + lo*hi in FP32
// (Markidis et al. 2018; Ootomo & Yokota 2022); the dropped lo*lo term is below FP32
// rounding.
//
// One CTA (16 warps) computes a 128-row tile of one block for N right-hand sides:
//   * K is streamed in chunks of 32.  The matrix rows (16-byte cp.async) and the gathered
//     input entries (4-byte cp.async) arrive two chunks ahead in a raw ring; both are split into
//     hi/lo and written to shared memory in the canonical no-swizzle K-major layout (core
//     matrices of 8 rows x 16 bytes; 128 bytes between core matrices along K, 1024 along M/N).
//   * One thread issues, per chunk, 4 x 3 tcgen05.mma.kind::tf32 (M = 128, K = 8 each): hi*hi
//     into one 128 x N FP32 tensor-memory buffer, hi*lo + lo*hi into a second, both starting
//     from zero, and commits them to the chunk's mbarrier.  A 2-stage shared-memory ring and
//     two pairs of TMEM buffers let the loads of chunk c+1 overlap the MMAs of chunk c.
//   * After a chunk's MMAs complete, every warp reads its rows of both buffers (tcgen05.ld;
//     warp w owns TMEM lanes 32 (w % 4) .. + 31 = tile rows, and quarter w / 4 of the columns)
//     and adds them to FP32 registers with round-to-nearest and Kahan compensation, so
//     tensor-core accumulation never spans more than one chunk of K.
//   * The epilogue adds the identity term of the interpolative decomposition and stores the row.
// Every mbarrier wait is bounded in time; on timeout the kernel sets a status bit, skips the
// remaining work, and still releases its tensor memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "../host/internal.h"

namespace mht {
namespace {

constexpr int kTcThreads = 512;  // 16 warps: TMEM lane quadrant = warp % 4, column quarter = warp / 4
constexpr int kTcDepth = 3;      // raw chunk slots: chunks c, c+1, c+2 in flight
constexpr int kTcM = 128;   // tile rows = tensor-memory lanes
constexpr int kTcK = 32;    // K per pipeline stage (TF32 elements)
constexpr unsigned long long kTcWaitNs = 2000000000ull;

enum TcMode { TC_SYN_ID = 0, TC_ADJ_ID = 1, TC_SYN_U = 2, TC_ADJ_U = 3 };

struct TcParams {
  const float* data;
  const int* idx;
  const MhtBlockDesc* desc;
  const MhtItem* items;
  const int* perm;
  const float* wts;
  const float* in0;
  const float* in1;
  long long is_e, is_k;
  float* out0;
  float* out1;
  long long os_e, os_k;
  int nrhs;
  unsigned* status;
};

__device__ __forceinline__ unsigned sa(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned ph) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok)
               : "r"(sa(b)), "r"(ph)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned ph) {
  if (mbar_try(b, ph)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(b, ph)) return true;
    if ((it & 255) == 0 && gtimer() - t0 > kTcWaitNs) return false;
  }
}
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - hi);
}
// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// 16-byte (A rows) and 4-byte (gathered B entries) asynchronous global -> shared copies; a
// source size of 0 zero-fills the destination without reading (the address stays valid).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// core-matrix byte offset of element group (row m, 4-column group c4) in a no-swizzle K-major
// tile with 32 columns: 8 x 16-byte core matrices, 128 bytes apart along K, 1024 along M/N
__device__ __forceinline__ int core_off(int m, int c4) { return (m >> 3) * 1024 + c4 * 128 + (m & 7) * 16; }
// A element group q (0..1023) of a 128 x 32 chunk: 8 consecutive q are the 8 rows of one core
// matrix (their 16-byte stores fill 128 contiguous bytes: no bank conflicts), and a warp's 32
// groups read 64 contiguous bytes from each of 8 rows
__device__ __forceinline__ int a_row(int q) { return (q >> 6) * 8 + (q & 7); }
__device__ __forceinline__ int a_col4(int q) { return (q >> 3) & 7; }

// C: complex factors and vectors.  The complex product y = A x is computed as one real
// product: A's interleaved storage is a real matrix of 2K columns, and column n of B holds
// (xr, -xi) for output n < N/2 (the real parts) and (xi, xr) for output N/2 + n (the imaginary
// parts), so a tile of N accumulator columns carries N/2 complex right-hand sides.
//
// Pipeline per chunk c (32 columns of K): the raw rows of A for chunk c + 2 and the gathered
// B entries are requested with cp.async into a 3-slot raw ring (each thread copies, and later
// converts, only its own elements, so no barrier separates the copy from the conversion);
// chunk c is split into TF32 hi / lo operand tiles (2 stages), one thread issues its 12 MMAs,
// and meanwhile every warp drains chunk c - 1 from tensor memory: warp w reads quarter w / 4 of
// the accumulator columns for TMEM lane quadrant w % 4.
template <int MODE, int N, bool C>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc3(TcParams p) {
  static_assert(N == 16 || N == 32 || N == 64, "RHS tile");
  constexpr int W = C ? 2 : 1;
  constexpr int NR = N / W;   // right-hand sides per tile
  constexpr int H = N / 4;    // accumulator columns drained per warp (one quarter)
  constexpr int A_BYTES = kTcM * kTcK * 4;
  constexpr int B_BYTES = N * kTcK * 4;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int NB = MODE == TC_ADJ_ID ? 2 : 1;  // raw B buffers (input and sibling)
  constexpr int RAW = A_BYTES + NB * B_BYTES;
  constexpr int NCOLS = 4 * N;  // two chunk buffers x (hi*hi sum, correction sum)
  constexpr int BG = N * (kTcK / 4);  // 4-entry groups of a B chunk
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm);       // [2]
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(sm + 64);
  volatile int* flag = reinterpret_cast<volatile int*>(sm + 68);
  int* ksrc = reinterpret_cast<int*>(sm + 128);            // [kTcDepth][kTcK]
  float* kw = reinterpret_cast<float*>(sm + 512);          // [kTcDepth][kTcK]
  unsigned char* stages = sm + 1024;                       // [2][STAGE]
  unsigned char* raw = stages + 2 * STAGE;                 // [kTcDepth][RAW]

  const MhtItem it = p.items[blockIdx.x];
  const MhtBlockDesc d = p.desc[it.blk];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r0 = blockIdx.y * NR;
  const int nk = min(NR, p.nrhs - r0);
  float* out = (MODE == TC_ADJ_ID && it.sib) ? p.out1 : p.out0;

  if (MODE == TC_ADJ_ID && it.start == 0) {  // identity part of [I | T~] P^T: out[skel_j] = z_j
    for (int e = tid; e < d.cols * nk; e += kTcThreads) {
      const int j = e / nk, t = e % nk;
      const long long a = (((long long)d.out_off + j) * p.is_e + (long long)(r0 + t) * p.is_k) * W;
      const long long o = ((long long)p.idx[d.idx_off + j] * p.os_e + (long long)(r0 + t) * p.os_k) * W;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        float v = p.in0[a + c];
        if (p.in1) v += p.in1[a + c];
        out[o + c] = v;
      }
    }
  }
  if (it.count == 0) return;

  const int K = d.cols * W;  // real columns
  const int nchunks = (K + kTcK - 1) / kTcK;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *flag = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)), "n"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  // instruction descriptor: D = F32, A = B = TF32, both K-major, N >> 3, M >> 4
  const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | (unsigned(N >> 3) << 17) | (unsigned(kTcM >> 4) << 24);
  const int ldr = d.ldt * W;  // real row stride of A

  // warp 0: sources (and weights) of chunk x's 32 real columns into ring slot x % kTcDepth
  auto sources = [&](int x) {
    const int kr = x * kTcK + (tid & 31);
    const int kk = kr / W;  // complex: real column kr is part kr & 1 of entry kr >> 1
    int src = -1;
    float w = 1.f;
    if (kr < K) {
      if (MODE == TC_SYN_ID) {
        src = p.idx[d.idx_off + d.rows + kk];
        if (p.wts) w = p.wts[src];  // leaf stage: diagonal scale of the coefficients
      }
      else if (MODE == TC_ADJ_ID) src = d.out_off + kk;
      else if (MODE == TC_SYN_U) src = d.in_off + kk;
      else {
        src = p.perm[d.out_off + kk];
        if (p.wts) w = p.wts[src];
      }
    }
    ksrc[(x % kTcDepth) * kTcK + (tid & 31)] = src;
    kw[(x % kTcDepth) * kTcK + (tid & 31)] = w;
  };
  // every thread: requests its elements of chunk x (A rows, gathered B entries) and commits
  auto request = [&](int x) {
    if (x < nchunks) {
      unsigned char* rs = raw + (x % kTcDepth) * RAW;
#pragma unroll
      for (int u = 0; u < A_BYTES / 16 / kTcThreads; ++u) {
        const int q = tid + kTcThreads * u;
        const int m = a_row(q), c4 = a_col4(q), kr = x * kTcK + c4 * 4;
        const bool ok = m < it.count && kr < ldr;
        const float* src = ok ? p.data + (d.t_off + (long long)(it.start + m) * d.ldt) * W + kr : p.data;
        cp_async16(rs + q * 16, src, ok ? 16u : 0u);
      }
      const int* ks = ksrc + (x % kTcDepth) * kTcK;
      for (int g = tid; g < BG; g += kTcThreads) {
        const int n = g % N, c4 = g / N;
        const int rn = C ? (n < NR ? n : n - NR) : n;  // right-hand side of column n
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int kl = c4 * 4 + j;
          const int src = ks[kl];
          const bool ok = src >= 0 && rn < nk;
          long long a = 0;
          if (ok) {
            a = ((long long)src * p.is_e + (long long)(r0 + rn) * p.is_k) * W;
            if (C) a += (n < NR) ? (kl & 1) : 1 - (kl & 1);  // (xr, -xi) / (xi, xr): component
          }
          // raw B layout [j][group]: a warp's copies of one j land in consecutive words
          cp_async4(rs + A_BYTES + (j * BG + g) * 4, ok ? p.in0 + a : p.in0, ok ? 4u : 0u);
          if (NB == 2)
            cp_async4(rs + A_BYTES + B_BYTES + (j * BG + g) * 4, (ok && p.in1) ? p.in1 + a : p.in0,
                      (ok && p.in1) ? 4u : 0u);
        }
      }
    }
    cp_async_commit();
  };

  // Kahan-compensated row sums of this thread's quarter of the accumulator columns
  float acc[H], cmp[H];
#pragma unroll
  for (int j = 0; j < H; ++j) acc[j] = cmp[j] = 0.f;
  const int quarter = warp >> 2;
  int issued = 0, drained = 0;
  // waits for chunk j's MMAs and adds its sums to acc; frees stage and TMEM buffer j & 1
  auto drain = [&](int j) {
    if (tid == 0 && *flag && !mbar_wait(&mbar[j & 1], unsigned((j >> 1) & 1))) {
      atomicOr(p.status, 32u);
      *flag = 0;
    }
    __syncthreads();
    if (*flag) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned base = tmem + (unsigned((warp & 3) * 32) << 16) + unsigned((j & 1) * 2 * N + quarter * H);
#pragma unroll
      for (int cb = 0; cb < H / 4; ++cb) {
        unsigned r[4], q[4];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                     : "r"(base + cb * 4)
                     : "memory");
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3])
                     : "r"(base + N + cb * 4)
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int n = cb * 4 + jj;
          const float y = (__uint_as_float(r[jj]) + __uint_as_float(q[jj])) - cmp[n];
          const float t = acc[n] + y;
          cmp[n] = (t - acc[n]) - y;
          acc[n] = t;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    drained = j + 1;
  };

  // prologue: sources of chunks 0..2, requests of chunks 0 and 1.  Afterwards the sources of
  // chunk c+3 are written during iteration c ahead of drain(c-1)'s barrier, which publishes
  // them before request(c+3) in the next iteration (two CTA barriers per chunk).
  if (warp == 0)
    for (int x = 0; x < kTcDepth && x < nchunks; ++x) sources(x);
  __syncthreads();
  for (int x = 0; x < kTcDepth - 1; ++x) request(x);
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;  // stage and TMEM buffer; chunk c-2 used them and was drained already
    unsigned char* st = stages + s * STAGE;
    unsigned char* Ahi = st;
    unsigned char* Alo = st + A_BYTES;
    unsigned char* Bhi = st + 2 * A_BYTES;
    unsigned char* Blo = st + 2 * A_BYTES + B_BYTES;
    request(c + kTcDepth - 1);
    cp_async_wait<kTcDepth - 1>();  // this thread's copies of chunk c have landed
    const unsigned char* rs = raw + (c % kTcDepth) * RAW;
#pragma unroll
    for (int u = 0; u < A_BYTES / 16 / kTcThreads; ++u) {
      const int q = tid + kTcThreads * u;
      const float4 v = *reinterpret_cast<const float4*>(rs + q * 16);
      float4 h, l;
      split(v.x, h.x, l.x);
      split(v.y, h.y, l.y);
      split(v.z, h.z, l.z);
      split(v.w, h.w, l.w);
      const int off = core_off(a_row(q), a_col4(q));
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = l;
    }
    const float* kwc = kw + (c % kTcDepth) * kTcK;
    for (int g = tid; g < BG; g += kTcThreads) {
      const int n = g % N, c4 = g / N;
      const float* rb = reinterpret_cast<const float*>(rs + A_BYTES);
      float x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] = rb[j * BG + g];
        if (NB == 2) x[j] += rb[BG * 4 + j * BG + g];  // sibling buffer (B_BYTES = 4 BG floats later)
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] *= kwc[c4 * 4 + j];
        if (C && n < NR && ((c4 * 4 + j) & 1)) x[j] = -x[j];  // (xr, -xi)
      }
      float4 h, l;
      split(x[0], h.x, l.x);
      split(x[1], h.y, l.y);
      split(x[2], h.z, l.z);
      split(x[3], h.w, l.w);
      const int off = core_off(n, c4);
      *reinterpret_cast<float4*>(Bhi + off) = h;
      *reinterpret_cast<float4*>(Blo + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned dmain = tmem + unsigned(s * 2 * N), dcorr = dmain + N;
#pragma unroll
      for (int k8 = 0; k8 < kTcK / 8; ++k8) {
        const uint64_t ah = smem_desc(sa(Ahi) + k8 * 256, 128, 1024);
        const uint64_t al = smem_desc(sa(Alo) + k8 * 256, 128, 1024);
        const uint64_t bh = smem_desc(sa(Bhi) + k8 * 256, 128, 1024);
        const uint64_t bl = smem_desc(sa(Blo) + k8 * 256, 128, 1024);
        mma_tf32(dmain, ah, bh, idesc, k8 > 0 ? 1u : 0u);
        mma_tf32(dcorr, ah, bl, idesc, k8 > 0 ? 1u : 0u);
        mma_tf32(dcorr, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       sa(&mbar[s]))
                   : "memory");
    }
    issued = c + 1;
    // sources of chunk c+3 into ring slot c % 3 (chunk c's weights were read before the last
    // barrier, its requests long before)
    if (warp == 0 && c + kTcDepth < nchunks) sources(c + kTcDepth);
    if (c >= 1) drain(c - 1);  // overlaps the MMAs of chunk c; its barrier publishes the sources
    else __syncthreads();
    if (!*flag) break;
  }
  cp_async_wait<0>();  // no copy may still target shared memory when the CTA exits
  if (issued > drained) drain(issued - 1);
  // error path: committed MMAs must finish before tensor memory is released
  if (tid == 0 && !*flag && issued > 0) mbar_wait(&mbar[(issued - 1) & 1], unsigned(((issued - 1) >> 1) & 1));

  const int m = (warp & 3) * 32 + (tid & 31);  // TMEM lane = tile row
  if (m < it.count) {
    const int i = it.start + m;
    long long dst;
    float wrow = 1.f;
    long long sidx = -1;
    if (MODE == TC_SYN_ID) {
      dst = (long long)d.out_off + i;
      sidx = p.idx[d.idx_off + i];
    } else if (MODE == TC_ADJ_ID) {
      dst = p.idx[d.idx_off + d.cols + i];
    } else if (MODE == TC_SYN_U) {
      dst = p.perm[d.out_off + i];
      if (p.wts) wrow = p.wts[dst];
    } else {
      dst = (long long)d.in_off + i;
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int col = quarter * H + j;
      const int c = C ? col / NR : 0;        // complex: real parts, then imaginary parts
      const int n = C ? col % NR : col;      // right-hand side within the tile
      if (n < nk) {
        float v = acc[j] - cmp[j];
        if (MODE == TC_SYN_ID)
          v += (p.wts ? p.wts[sidx] : 1.f) * p.in0[(sidx * p.is_e + (long long)(r0 + n) * p.is_k) * W + c];
        if (MODE == TC_SYN_U) v *= wrow;
        out[(dst * p.os_e + (long long)(r0 + n) * p.os_k) * W + c] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(NCOLS) : "memory");
}

template <int MODE, int N, bool C>
int launch_n(const TcLaunch& a, std::string& err) {
  constexpr int STAGE = 2 * kTcM * kTcK * 4 + 2 * N * kTcK * 4;
  constexpr int NR = C ? N / 2 : N;
  constexpr int RAW = kTcM * kTcK * 4 + (MODE == TC_ADJ_ID ? 2 : 1) * N * kTcK * 4;
  const size_t smem = 1024 + 2 * size_t(STAGE) + size_t(kTcDepth) * RAW;
  auto kern = k_tc3<MODE, N, C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) {
    err = std::string("tensor-core stage: ") + cudaGetErrorString(e);
    return MHT_ERR_CUDA;
  }
  TcParams p{a.data, a.idx, a.desc, a.items, a.perm, a.wts, a.in0, a.in1, a.is_e, a.is_k,
             a.out0, a.out1, a.os_e, a.os_k, int(a.nrhs), a.status};
  dim3 grid(unsigned(a.nitems), unsigned((a.nrhs + NR - 1) / NR));
  kern<<<grid, kTcThreads, smem, static_cast<cudaStream_t>(a.stream)>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("tensor-core stage launch: ") + cudaGetErrorString(e);
    return MHT_ERR_CUDA;
  }
  return 0;
}

// Accumulator tile: 16, 32 or 64 columns (complex: half as many right-hand sides); wider RHS
// counts take several tiles across grid.y.
template <int MODE, bool C>
int launch_mode(const TcLaunch& a, std::string& err) {
  const int64_t cols = a.nrhs * (C ? 2 : 1);
  if (cols <= 16) return launch_n<MODE, 16, C>(a, err);
  if (cols <= 32) return launch_n<MODE, 32, C>(a, err);
  return launch_n<MODE, 64, C>(a, err);
}

template <bool C>
int launch_field(const TcLaunch& a, std::string& err) {
  switch (a.mode) {
    case 0: return launch_mode<TC_SYN_ID, C>(a, err);
    case 1: return launch_mode<TC_ADJ_ID, C>(a, err);
    case 2: return launch_mode<TC_SYN_U, C>(a, err);
    default: return launch_mode<TC_ADJ_U, C>(a, err);
  }
}

}  // namespace

int tc_stage_launch(const TcLaunch& a, std::string& err) {
  if (a.nitems == 0) return 0;
  return a.cplx ? launch_field<true>(a, err) : launch_field<false>(a, err);
}

}  // namespace mht
