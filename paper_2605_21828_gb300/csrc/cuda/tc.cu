// Multi-RHS block products on the 5th-generation tensor cores (tcgen05), 3xTF32.
//
// With k right-hand sides every butterfly block product becomes a GEMM: M = rows of the
// stored matrix (T~ or U, or their transposes for the adjoint), N = k, K = its columns.  FP32
// accuracy on TF32 tensor cores comes from splitting both operands, x = hi + lo with
// hi = tf32(x) and lo = tf32(x - hi), and accumulating hi*hi + hi*lo + lo*hi in FP32
// (Markidis et al. 2018; Ootomo & Yokota 2022); the dropped lo*lo term is below FP32
// rounding.
//
// One CTA (4 warps) computes a 128-row tile of one block for N right-hand sides:
//   * K is streamed in chunks of 32.  The matrix rows are read with 128-bit loads (one chunk
//     ahead, in registers), the input rows are gathered per chunk; both are split into
//     hi/lo and written to shared memory in the canonical no-swizzle K-major layout (core
//     matrices of 8 rows x 16 bytes; 128 bytes between core matrices along K, 1024 along M/N).
//   * One thread issues, per chunk, 4 x 3 tcgen05.mma.kind::tf32 (M = 128, K = 8 each): hi*hi
//     into one 128 x N FP32 tensor-memory buffer, hi*lo + lo*hi into a second, both starting
//     from zero, and commits them to the chunk's mbarrier.  A 2-stage shared-memory ring and
//     two pairs of TMEM buffers let the loads of chunk c+1 overlap the MMAs of chunk c.
//   * After a chunk's MMAs complete, every thread reads its row of both buffers
//     (tcgen05.ld; thread i owns TMEM lane i = tile row i) and adds them to FP32 registers with
//     round-to-nearest and Kahan compensation, so tensor-core accumulation never spans more
//     than one chunk of K.
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

constexpr int kTcThreads = 128;
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
__device__ __forceinline__ float4 ldg_nc(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Splits this thread's 8 float4 of a chunk into the hi / lo core-matrix tiles.
__device__ __forceinline__ void store_a(const float4 (&r)[8], unsigned char* Ahi, unsigned char* Alo) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = threadIdx.x + kTcThreads * u;
    const int m = q >> 3, c4 = q & 7;
    const int off = (m >> 3) * 1024 + c4 * 128 + (m & 7) * 16;
    float4 h, l;
    split(r[u].x, h.x, l.x);
    split(r[u].y, h.y, l.y);
    split(r[u].z, h.z, l.z);
    split(r[u].w, h.w, l.w);
    *reinterpret_cast<float4*>(Ahi + off) = h;
    *reinterpret_cast<float4*>(Alo + off) = l;
  }
}

// Loads this thread's 8 float4 of a 128 x 32 chunk of the tile's rows (zero outside).
// Complex factors are read as real rows of 2 ldt floats (re, im interleaved).
template <int W>
__device__ __forceinline__ void load_a(const TcParams& p, const MhtBlockDesc& d, const MhtItem& it, int k0,
                                       float4 (&r)[8]) {
  const int ldr = d.ldt * W;  // real row stride
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = threadIdx.x + kTcThreads * u;
    const int m = q >> 3, c4 = q & 7, kk = k0 + c4 * 4;
    r[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < it.count && kk < ldr)
      r[u] = ldg_nc(p.data + (d.t_off + (long long)(it.start + m) * d.ldt) * W + kk);
  }
}

// C: complex factors and vectors.  The complex product y = A x is computed as one real
// product: A's interleaved storage is a real matrix of 2K columns, and column n of B holds
// (xr, -xi) for output n < N/2 (the real parts) and (xi, xr) for output N/2 + n (the imaginary
// parts), so a tile of N accumulator columns carries N/2 complex right-hand sides.
template <int MODE, int N, bool C>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc3(TcParams p) {
  static_assert(N == 16 || N == 32 || N == 64, "RHS tile");
  constexpr int W = C ? 2 : 1;
  constexpr int NR = N / W;  // right-hand sides per tile
  constexpr int A_BYTES = kTcM * kTcK * 4;
  constexpr int B_BYTES = N * kTcK * 4;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int NCOLS = 4 * N;  // two chunk buffers x (hi*hi sum, correction sum)
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm);       // [2]
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(sm + 64);
  volatile int* flag = reinterpret_cast<volatile int*>(sm + 68);
  int* ksrc = reinterpret_cast<int*>(sm + 128);            // [2][kTcK]
  float* kw = reinterpret_cast<float*>(sm + 384);          // [2][kTcK]
  unsigned char* stages = sm + 1024;

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

  // Row accumulators in registers (thread = tile row = TMEM lane).  Each chunk's MMAs start
  // from zero and its two partial sums are added here with FP32 round-to-nearest: the tensor
  // core's own accumulation is not round-to-nearest, and over a long K its error would exceed
  // the FP32 level that the split is meant to reach.
  float acc[N], cmp[N];  // running sums and their Kahan compensation
#pragma unroll
  for (int j = 0; j < N; ++j) acc[j] = cmp[j] = 0.f;
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
      const unsigned base = tmem + (unsigned(warp * 32) << 16) + unsigned((j & 1) * 2 * N);
#pragma unroll
      for (int cb = 0; cb < N / 16; ++cb) {
        unsigned r[16], q[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(base + cb * 16)
            : "memory");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
              "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
            : "r"(base + N + cb * 16)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int n = cb * 16 + jj;
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

  float4 ra[8];  // matrix rows of the next chunk, loaded one chunk ahead
  if (nchunks > 0) load_a<W>(p, d, it, 0, ra);
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;  // stage and TMEM buffer; chunk c-2 used them and was drained already
    unsigned char* st = stages + s * STAGE;
    float* Ahi = reinterpret_cast<float*>(st);
    float* Alo = reinterpret_cast<float*>(st + A_BYTES);
    float* Bhi = reinterpret_cast<float*>(st + 2 * A_BYTES);
    float* Blo = reinterpret_cast<float*>(st + 2 * A_BYTES + B_BYTES);
    const int k0 = c * kTcK;
    if (warp == 0) {
      // sources of this chunk's 32 real input columns (and their weights); complex: real
      // column k is part k & 1 of entry k >> 1
      const int kk = (k0 + (tid & 31)) / W;
      int src = -1;
      float w = 1.f;
      if (k0 + (tid & 31) < K) {
        if (MODE == TC_SYN_ID) src = p.idx[d.idx_off + d.rows + kk];
        else if (MODE == TC_ADJ_ID) src = d.out_off + kk;
        else if (MODE == TC_SYN_U) src = d.in_off + kk;
        else {
          src = p.perm[d.out_off + kk];
          if (p.wts) w = p.wts[src];
        }
      }
      ksrc[s * kTcK + (tid & 31)] = src;
      kw[s * kTcK + (tid & 31)] = w;
    }
    __syncthreads();
    if (!*flag) break;
    // A chunk (this thread's 8 float4, loaded one iteration earlier) -> hi / lo core matrices;
    // then load the matrix rows of chunk c+1 into the registers just freed
    store_a(ra, reinterpret_cast<unsigned char*>(Ahi), reinterpret_cast<unsigned char*>(Alo));
    if (c + 1 < nchunks) load_a<W>(p, d, it, k0 + kTcK, ra);
    // B chunk: N right-hand sides x 32 gathered input entries -> hi / lo core matrices
    for (int q = tid; q < N * (kTcK / 4); q += kTcThreads) {
      const int n = q % N, c4 = q / N;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kk = c4 * 4 + j;
        const int src = ksrc[s * kTcK + kk];
        float x = 0.f;
        const int rn = C ? (n < NR ? n : n - NR) : n;  // right-hand side of column n
        if (src >= 0 && rn < nk) {
          const long long a = ((long long)src * p.is_e + (long long)(r0 + rn) * p.is_k) * W;
          if (C) {
            // real part: (xr, -xi) against (Ar, Ai); imaginary part: (xi, xr)
            const int part = (k0 + kk) & 1;
            const int comp = (n < NR) ? part : 1 - part;
            x = __ldcg(p.in0 + a + comp);
            if (p.in1) x += __ldcg(p.in1 + a + comp);
            if (n < NR && part == 1) x = -x;
          } else {
            x = __ldcg(p.in0 + a);
            if (p.in1) x += __ldcg(p.in1 + a);
          }
          x *= kw[s * kTcK + kk];
        }
        v[j] = x;
      }
      float4 h, l;
      split(v[0], h.x, l.x);
      split(v[1], h.y, l.y);
      split(v[2], h.z, l.z);
      split(v[3], h.w, l.w);
      const int off = (n >> 3) * 1024 + c4 * 128 + (n & 7) * 16;
      *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Bhi) + off) = h;
      *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Blo) + off) = l;
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
    if (c >= 1) drain(c - 1);  // overlaps the MMAs of chunk c
  }
  if (issued > drained) drain(issued - 1);
  // error path: committed MMAs must finish before tensor memory is released
  if (tid == 0 && !*flag && issued > 0) mbar_wait(&mbar[(issued - 1) & 1], unsigned(((issued - 1) >> 1) & 1));

  const int m = tid;  // TMEM lane = tile row
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
    for (int n = 0; n < NR; ++n) {
      if (n < nk) {
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const int col = c * NR + n;
          float v = acc[col] - cmp[col];
          if (MODE == TC_SYN_ID) v += p.in0[(sidx * p.is_e + (long long)(r0 + n) * p.is_k) * W + c];
          if (MODE == TC_SYN_U) v *= wrow;
          out[(dst * p.os_e + (long long)(r0 + n) * p.os_k) * W + c] = v;
        }
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
  const size_t smem = 1024 + 2 * size_t(STAGE);
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
