// Multi-RHS block products on the 5th-generation tensor cores (tcgen05) with FP32-accurate
// split operands.
//
// With k right-hand sides every butterfly block product (Sec. 2: y = [I | T~] P^T x, and the
// column-basis products) becomes a GEMM: M = rows of the stored matrix (T~ or U, or their
// transposes for the adjoint), N = k, K = its columns.  The tensor cores multiply low-precision
// operands exactly and accumulate in FP32, so every FP32 operand is split into pieces and the
// significant piece products are summed:
//   * 6xBF16 (MHT_APPLY_6XBF16): x = x0 + x1 + x2 with x0 the leading 8 significant bits of x,
//     x1 those of x - x0 (Veltkamp-Dekker splitting) and x2 = x - x0 - x1 (exact: three 8-bit
//     significands cover FP32's 24 bits), and
//     a b ~ a0 b0 + (a0 b1 + a1 b0) + (a0 b2 + a1 b1 + a2 b0); the dropped terms are below
//     2^-23 |a b|.
//   * 3xTF32 (MHT_APPLY_3XTF32): x = hi + lo with hi = tf32(x), lo = tf32(x - hi) (22 of 24
//     bits), a b ~ hi hi + (hi lo + lo hi) (Markidis et al. 2018; Ootomo & Yokota 2022).
// The piece products a_i b_j (i + j < P) all accumulate into one TMEM accumulator, issued
// smallest order first (i + j = P - 1, ..., 0): the tensor core's rounding of the running sum is
// then relative to small partial sums until the two leading products a_0 b_0 land last.
//
// One persistent CTA per SM (608 threads) walks work units (128-row tile of one block x one
// tile of N accumulator columns), sorted by K on the host, in a fixed stride:
//   warp 0      TMA producer: 128 x 32 FP32 tiles of the stored matrix by 2-D tensor maps
//               (one per block, 128-byte swizzle, out-of-range rows / columns read as zero)
//               into a ring of raw slots;
//   warp 1      allocates tensor memory; one thread issues the MMAs of a chunk (K = 32) into
//               one of four TMEM accumulator buffers and commits them to mbarriers;
//   warp 2      gathers the chunk's input entries (the level vector rows named by the block's
//               index list, the index loaded a chunk ahead) with cp.async into raw B slots;
//   warps 3-18  split the raw A and B tiles into the pieces' canonical K-major core-matrix
//               layout (a ring of stages), then drain the accumulator of the chunk kDrainLag
//               back (tcgen05.ld; warp w owns TMEM lanes 32 (w % 4) .. and a quarter of the
//               columns) into FP32 registers with Kahan compensation, and write each unit's
//               rows in the epilogue (identity term of the ID, weights, scatter).
// Tensor-core accumulation never spans more than one chunk of 32 columns.  Every mbarrier wait
// is bounded in time; on timeout the kernel sets status bit 32 and an abort flag, every role
// leaves its loop, copies and MMAs still in flight are waited for, and the tensor memory is
// released.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../host/internal.h"

namespace mht {
namespace {

constexpr int kMathWarp0 = 3;      // warps 3 .. 18 split, drain and write
constexpr int kMathWarps = 16;     // four groups of four consecutive warps: lane quadrant x column group
constexpr int kTcThreads = 32 * (kMathWarp0 + kMathWarps);
constexpr int kTmemBufs = 4;       // accumulator buffers (N columns each) in flight
constexpr int kDrainLag = 2;       // chunks between a chunk's split and its drain (< kTmemBufs)
constexpr int kTcM = 128;          // tile rows = tensor-memory lanes
constexpr int kTcK = 32;           // FP32 columns of K per chunk
constexpr int kRawA = kTcM * kTcK * 4;  // one TMA box
constexpr unsigned long long kTcWaitNs = 2000000000ull;

enum TcMode { TC_SYN_ID = 0, TC_ADJ_ID = 1, TC_SYN_U = 2, TC_ADJ_U = 3 };

struct TcParams {
  const float* data;
  const int* idx;
  const MhtBlockDesc* desc;
  const MhtItem* items;
  const CUtensorMap* tmaps;  // one per block of the stage (this direction)
  const int* perm;
  const float* wts;
  const float* in0;
  const float* in1;
  long long is_e, is_k;
  float* out0;
  float* out1;
  long long os_e, os_k;
  int nitems, ntiles, nrhs;
  int vec;                    // input rows of the RHS tile are contiguous and 16-byte aligned
  int vec_out;                // output rows likewise (real plans)
  unsigned* status;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned sa(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
// The waiting thread may be suspended for a system-dependent time before the test returns
// false.  (A suspend-time hint, which lets it sleep longer, measured 1.5 % slower.)
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned ph) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(sa(b)), "r"(ph)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
// Bounded wait: false when it gave up (time limit: sets the status bit and the abort flag)
// or when another role already aborted.
__device__ __forceinline__ bool waitb(uint64_t* b, unsigned ph, volatile int* abort_flag, unsigned* status) {
  if (mbar_try(b, ph)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(b, ph)) return true;
    if ((it & 3) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > kTcWaitNs) {
        atomicOr(status, 32u);
        *abort_flag = 1;
        return false;
      }
    }
  }
}
// Bounded wait that ignores the abort flag (clean-up of copies and MMAs in flight).
__device__ __forceinline__ void wait_quiet(uint64_t* b, unsigned ph) {
  if (mbar_try(b, ph)) return;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(b, ph)) return;
    if ((it & 3) == 0 && gtimer() - t0 > kTcWaitNs) return;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          sa(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa(bar))
      : "memory");
}
// 16-byte / 4-byte asynchronous global -> shared copies; a source size of 0 zero-fills the
// destination without reading (the address stays valid).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(sa(b)) : "memory");
}
// shared-memory matrix descriptor: no swizzle, K-major (LBO: next core matrix along K, SBO:
// next 8-row group)
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
template <bool BF16>
__device__ __forceinline__ void mma(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  if constexpr (BF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Starts reading K consecutive 32-bit TMEM columns of this warp's 32 lanes (one row per
// thread) into v; the registers are written asynchronously and valid after tmem_wait(v).
template <int K>
__device__ __forceinline__ void tmem_ld(unsigned taddr, float (&v)[K]) {
  static_assert(K == 4 || K == 8 || K == 16 || K == 32, "columns per read");
  if constexpr (K == 32) {
    tmem_ld<16>(taddr, *reinterpret_cast<float(*)[16]>(&v[0]));
    tmem_ld<16>(taddr + 16, *reinterpret_cast<float(*)[16]>(&v[16]));
  } else if constexpr (K == 4)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(taddr)
                 : "memory");
  else if constexpr (K == 8)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr)
                 : "memory");
  else
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
          "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
        : "r"(taddr)
        : "memory");
}
// Waits for this thread's TMEM reads; the registers are operands, so no use of them can be
// scheduled before the wait.
template <int K>
__device__ __forceinline__ void tmem_wait(float (&v)[K]) {
  if constexpr (K == 32) {
    tmem_wait<16>(*reinterpret_cast<float(*)[16]>(&v[0]));
    tmem_wait<16>(*reinterpret_cast<float(*)[16]>(&v[16]));
  } else if constexpr (K == 4)
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3])::"memory");
  else if constexpr (K == 8)
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7])::"memory");
  else
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                   "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                   "+f"(v[15])::"memory");
}

// ---------------------------------------------------------------- operand splitting
// Veltkamp-Dekker splitting of two values at once (packed FP32): c = x (2^16 + 1),
// hi = c - (c - x) keeps the leading 8 significant bits of x (exactly representable in BF16),
// lo = x - hi is exact.  Full-rate FMA-pipe arithmetic instead of conversion instructions.
__device__ __forceinline__ void vsplit2(float2 x, float2& hi, float2& lo) {
  const float2 k = make_float2(65537.f, 65537.f), m1 = make_float2(-1.f, -1.f);
  const float2 c = __fmul2_rn(x, k);
  const float2 t = __ffma2_rn(x, m1, c);  // c - x
  hi = __ffma2_rn(t, m1, c);              // c - t
  lo = __ffma2_rn(hi, m1, x);             // x - hi, exact
}
// upper halves (the BF16 bits) of two FP32 values that are exactly BF16: element a in the low half
__device__ __forceinline__ unsigned pack_hi(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}
// x = x0 + x1 + x2 exactly for 2 values: three packed BF16 words
__device__ __forceinline__ void split3_pair(float a, float b, unsigned& w0, unsigned& w1, unsigned& w2) {
  float2 h0, r0, h1, r1;
  vsplit2(make_float2(a, b), h0, r0);
  vsplit2(r0, h1, r1);  // r1 has at most 8 significant bits: exactly BF16
  w0 = pack_hi(h0.x, h0.y);
  w1 = pack_hi(h1.x, h1.y);
  w2 = pack_hi(r1.x, r1.y);
}
// x = x0 + x1 + x2 exactly for 8 values; p[i] = piece i as four packed words
__device__ __forceinline__ void split_bf16(const float (&x)[8], uint4 (&p)[3]) {
  unsigned w[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) split3_pair(x[2 * j], x[2 * j + 1], w[0][j], w[1][j], w[2][j]);
#pragma unroll
  for (int i = 0; i < 3; ++i) p[i] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x = hi + lo (to 22 bits) for 8 values; p[i][h] = piece i, values 4h .. 4h+3
__device__ __forceinline__ void split_tf32(const float (&x)[8], uint4 (&p)[2][2]) {
  float h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h[j] = tf32_rna(x[j]);
    l[j] = tf32_rna(x[j] - h[j]);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    p[0][q] = make_uint4(__float_as_uint(h[4 * q]), __float_as_uint(h[4 * q + 1]), __float_as_uint(h[4 * q + 2]),
                         __float_as_uint(h[4 * q + 3]));
    p[1][q] = make_uint4(__float_as_uint(l[4 * q]), __float_as_uint(l[4 * q + 1]), __float_as_uint(l[4 * q + 2]),
                         __float_as_uint(l[4 * q + 3]));
  }
}
// Writes the pieces of 8 consecutive K values of operand row r (K offset 8 k8 within the chunk)
// into the canonical no-swizzle K-major layout: core matrices of 8 rows x 16 bytes, 128 bytes
// apart along K, SBO apart along rows; piece i of the operand starts at base + i * piece_bytes.
template <bool BF16>
__device__ __forceinline__ void put_pieces(unsigned char* base, int piece_bytes, int r, int k8, const float (&x)[8]) {
  if constexpr (BF16) {
    constexpr int SBO = kTcK * 2 / 16 * 128;  // 512
    uint4 p[3];
    split_bf16(x, p);
    const int off = (r >> 3) * SBO + k8 * 128 + (r & 7) * 16;
#pragma unroll
    for (int i = 0; i < 3; ++i) *reinterpret_cast<uint4*>(base + i * piece_bytes + off) = p[i];
  } else {
    constexpr int SBO = kTcK * 4 / 16 * 128;  // 1024
    uint4 p[2][2];
    split_tf32(x, p);
    const int off = (r >> 3) * SBO + (2 * k8) * 128 + (r & 7) * 16;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      *reinterpret_cast<uint4*>(base + i * piece_bytes + off) = p[i][0];
      *reinterpret_cast<uint4*>(base + i * piece_bytes + off + 128) = p[i][1];
    }
  }
}

// The same for 4 consecutive K values (K offset 4 k4 within the chunk).
template <bool BF16>
__device__ __forceinline__ void put_pieces4(unsigned char* base, int piece_bytes, int r, int k4, const float (&x)[4]) {
  if constexpr (BF16) {
    constexpr int SBO = kTcK * 2 / 16 * 128;  // 512
    unsigned w[3][2];
#pragma unroll
    for (int j = 0; j < 2; ++j) split3_pair(x[2 * j], x[2 * j + 1], w[0][j], w[1][j], w[2][j]);
    const int off = (r >> 3) * SBO + (k4 >> 1) * 128 + (r & 7) * 16 + (k4 & 1) * 8;
#pragma unroll
    for (int i = 0; i < 3; ++i) *reinterpret_cast<uint2*>(base + i * piece_bytes + off) = make_uint2(w[i][0], w[i][1]);
  } else {
    constexpr int SBO = kTcK * 4 / 16 * 128;  // 1024
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = tf32_rna(x[j]);
      l[j] = tf32_rna(x[j] - h[j]);
    }
    const int off = (r >> 3) * SBO + k4 * 128 + (r & 7) * 16;
    *reinterpret_cast<float4*>(base + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(base + piece_bytes + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

struct Unit {
  MhtItem it;
  MhtBlockDesc d;
  int r0;   // first right-hand side of the tile
  int nk;   // right-hand sides in the tile
  int nch;  // chunks of 32 FP32 columns (0: no stored columns)
};

template <int N, bool C>
__device__ __forceinline__ Unit get_unit(const TcParams& p, int u) {
  constexpr int NR = C ? N / 2 : N;
  Unit x;
  const int item = u / p.ntiles, rt = u % p.ntiles;
  x.it = p.items[item];
  x.d = p.desc[x.it.blk];
  x.r0 = rt * NR;
  x.nk = min(NR, p.nrhs - x.r0);
  x.nch = x.it.count > 0 ? (x.d.cols * (C ? 2 : 1) + kTcK - 1) / kTcK : 0;
  return x;
}

// Shared memory of one CTA: raw A slots, two split stages, raw B slots, weights, barriers.
template <int MODE, int N, bool C, bool BF16>
__host__ __device__ constexpr size_t tc_smem(int ra, int rb, int ns) {
  constexpr int W = C ? 2 : 1;
  constexpr int NP = BF16 ? 3 : 2;
  constexpr int PE = BF16 ? 2 : 4;
  constexpr int STAGE = NP * (kTcM * kTcK * PE + N * kTcK * PE);
  constexpr int RAWB = (MODE == TC_ADJ_ID ? 2 : 1) * kTcK * (N / W) * W * 4;
  return 1024 + size_t(ra) * kRawA + size_t(ns) * STAGE + size_t(rb) * RAWB + size_t(rb) * kTcK * 4 + 8 * 8 * 4 +
         8 * (8 + 2 * kTmemBufs) + 64 + 2 * 32 * kMathWarps * 16;
}
constexpr size_t kTcMaxSmem = 227 * 1024;
// Ring depths: three split stages (so that splitting runs ahead of the MMAs) when four raw A
// slots (TMA tiles in flight) and three raw B slots fit beside them, else two; then as many raw
// A slots (up to 8) as fit beside four raw B slots (fewer B slots, down to 2, before A drops
// below 3).
template <int MODE, int N, bool C, bool BF16>
__host__ __device__ constexpr int tc_ns() {
  return tc_smem<MODE, N, C, BF16>(4, 3, 3) <= kTcMaxSmem ? 3 : 2;
}
template <int MODE, int N, bool C, bool BF16>
__host__ __device__ constexpr int tc_ra() {
  int ra = 8;
  while (tc_smem<MODE, N, C, BF16>(ra, 4, tc_ns<MODE, N, C, BF16>()) > kTcMaxSmem && ra > 4) --ra;
  while (tc_smem<MODE, N, C, BF16>(ra, 2, tc_ns<MODE, N, C, BF16>()) > kTcMaxSmem && ra > 2) --ra;
  return ra;
}
template <int MODE, int N, bool C, bool BF16>
__host__ __device__ constexpr int tc_rb() {
  int rb = 4;
  while (tc_smem<MODE, N, C, BF16>(tc_ra<MODE, N, C, BF16>(), rb, tc_ns<MODE, N, C, BF16>()) > kTcMaxSmem && rb > 2)
    --rb;
  return rb;
}

// BF16: 6xBF16 split (3 pieces); else 3xTF32 (2 pieces).  N accumulator columns (complex:
// N / 2 right-hand sides, real parts then imaginary parts).
template <int MODE, int N, bool C, bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1) k_tcs(TcParams p) {
  static_assert(N == 16 || N == 32 || N == 64, "accumulator tile");
  constexpr int W = C ? 2 : 1;
  constexpr int NR = N / W;
  constexpr int NP = BF16 ? 3 : 2;          // pieces per operand
  constexpr int PE = BF16 ? 2 : 4;          // bytes per piece element
  constexpr int A_PIECE = kTcM * kTcK * PE;
  constexpr int B_PIECE = N * kTcK * PE;
  constexpr int STAGE = NP * (A_PIECE + B_PIECE);
  constexpr int NB = MODE == TC_ADJ_ID ? 2 : 1;  // raw B buffers (input and sibling)
  constexpr int RAWB = NB * kTcK * NR * W * 4;   // one chunk's gathered entries
  constexpr int KW = kTcK / W;                   // input entries per chunk
  constexpr int H = N / (kMathWarps / 4);        // accumulator columns per math thread
  constexpr int KSTEP = BF16 ? 16 : 8;           // K of one MMA
  constexpr int SBO = kTcK * PE / 16 * 128;
  constexpr int NCOLS = kTmemBufs * N <= 64 ? 64 : kTmemBufs * N <= 128 ? 128 : 256;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base (the 128-byte swizzle pattern repeats every 1024 bytes)
  unsigned char* sm = smem_raw + ((1024 - (sa(smem_raw) & 1023)) & 1023);
  constexpr int RA = tc_ra<MODE, N, C, BF16>(), RB = tc_rb<MODE, N, C, BF16>(), NS = tc_ns<MODE, N, C, BF16>();
  static_assert(tc_smem<MODE, N, C, BF16>(RA, RB, NS) <= kTcMaxSmem, "shared memory of the tensor-core kernel");
  unsigned char* rawA = sm;                                  // [RA][16 KB], 1024-aligned
  unsigned char* stages = rawA + size_t(RA) * kRawA;         // [NS][STAGE], 1024-aligned
  unsigned char* rawB = stages + NS * STAGE;                 // [RB][RAWB]
  float* kw = reinterpret_cast<float*>(rawB + size_t(RB) * RAWB);  // [RB][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(kw + RB * kTcK);
  uint64_t* a_full = bars;           // [RA]
  uint64_t* a_empty = a_full + 8;    // [RA]
  uint64_t* b_full = a_empty + 8;    // [RB]
  uint64_t* b_empty = b_full + 8;    // [RB]
  uint64_t* s_full = b_empty + 8;    // [NS] split stage written
  uint64_t* mma_done = s_full + 4;   // [NS] chunk's MMAs complete (split stage free)
  uint64_t* t_full = mma_done + 4;   // [kTmemBufs] chunk's sums ready in TMEM buffer
  uint64_t* t_empty = t_full + kTmemBufs;  // [kTmemBufs] TMEM buffer drained
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(t_empty + kTmemBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // per split/drain thread, two unit slots: output offset, identity-term offset, weight of its row
  int4* epi = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(bars) + 8 * (8 * 4 + 8 + 2 * kTmemBufs) + 64);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nunits = p.nitems * p.ntiles;
  if (tid == 0) {
    for (int i = 0; i < RA; ++i) {
      mbar_init(&a_full[i], 1);
      mbar_init(&a_empty[i], kMathWarps);
    }
    for (int i = 0; i < RB; ++i) {
      mbar_init(&b_full[i], 32);  // one gather warp's cp.async arrivals per chunk
      mbar_init(&b_empty[i], kMathWarps);
    }
    for (int i = 0; i < NS; ++i) {
      mbar_init(&s_full[i], kMathWarps);
      mbar_init(&mma_done[i], 1);
    }
    for (int i = 0; i < kTmemBufs; ++i) {
      mbar_init(&t_full[i], 1);
      mbar_init(&t_empty[i], kMathWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)), "n"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  long long a_issued = 0;  // producer: TMA loads issued
  int mma_issued = 0;      // MMA thread: chunks committed

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const Unit x = get_unit<N, C>(p, u);
        const CUtensorMap* map = p.tmaps + x.it.blk;
        for (int c = 0; c < x.nch; ++c) {
          const int s = int(a_issued % RA);
          const unsigned ph = unsigned((a_issued / RA) & 1);
          if (!waitb(&a_empty[s], ph ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&a_full[s], kRawA);
          tma_load_2d(rawA + size_t(s) * kRawA, map, c * kTcK, x.it.start, &a_full[s]);
          ++a_issued;
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // instruction descriptor: D = F32, A = B = BF16 (kind::f16) or TF32, both K-major,
      // M = 128, N columns
      const unsigned idesc = (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
                             (unsigned(N >> 3) << 17) | (unsigned(kTcM >> 4) << 24);
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const Unit x = get_unit<N, C>(p, u);
        for (int c = 0; c < x.nch; ++c, ++g) {
          const int s = g % NS, b = g % kTmemBufs;
          if (!waitb(&t_empty[b], unsigned((g / kTmemBufs) & 1) ^ 1u, abort_flag, p.status) ||
              !waitb(&s_full[s], unsigned((g / NS) & 1), abort_flag, p.status)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned char* st = stages + s * STAGE;
          const unsigned a0 = sa(st), b0 = sa(st + NP * A_PIECE);
          const unsigned d = tmem + unsigned(b * N);
          // piece products a_i b_j (i + j < NP) into one accumulator, smallest order first
          // (i + j = NP - 1, ..., 0), so that the tensor core's rounding of the running sum is
          // relative to small partial sums until the leading products a_0 b_0 land last
          bool first = true;
          // descriptor start addresses advance by (bytes >> 4) in their low field
          const uint64_t da = smem_desc(a0, 128, SBO), db = smem_desc(b0, 128, SBO);
#pragma unroll
          for (int ord = NP - 1; ord >= 0; --ord)
#pragma unroll
            for (int kk = 0; kk < kTcK / KSTEP; ++kk)
#pragma unroll
              for (int i = 0; i <= ord; ++i) {
                const int j = ord - i;
                mma<BF16>(d, da + uint64_t((i * A_PIECE + kk * 256) >> 4), db + uint64_t((j * B_PIECE + kk * 256) >> 4),
                          idesc, first ? 0u : 1u);
                first = false;
              }
          // stage s may be overwritten once these MMAs complete; the chunk's sums are ready
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           sa(&mma_done[s]))
                       : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           sa(&t_full[b]))
                       : "memory");
          mma_issued = g + 1;
        }
      }
    }
  } else if (warp < kMathWarp0) {
    // ------------------------------------------------------------ input gather (cp.async)
    // lane -> one input entry of the chunk (two lanes per entry for complex), whose index is
    // loaded one chunk ahead of its copies
    const bool vec = p.vec != 0;  // contiguous 16-byte aligned rows of the tile's RHS (host check)
    // per-input weights: the leaf stage's scale of the coefficients, the adjoint's W f
    const bool in_w = p.wts && (MODE == TC_SYN_ID || MODE == TC_ADJ_U);
    constexpr int P = 32 / KW;  // lanes per entry
    const int j = lane % KW, q = lane / KW;
    int u = blockIdx.x, c = 0;
    Unit x{};
    auto seek = [&]() -> bool {  // the next unit (from u on) with stored columns
      for (; u < nunits; u += gridDim.x) {
        x = get_unit<N, C>(p, u);
        if (x.nch > 0) return true;
      }
      return false;
    };
    auto advance = [&]() -> bool {
      if (++c < x.nch) return true;
      c = 0;
      u += gridDim.x;
      return seek();
    };
    // index of this lane's input entry in chunk (x, c); -1 outside the block
    auto src_of = [&]() -> int {
      const int kk = c * KW + j;
      if (kk >= x.d.cols) return -1;
      if (MODE == TC_SYN_ID) return p.idx[x.d.idx_off + x.d.rows + kk];
      if (MODE == TC_ADJ_ID) return x.d.out_off + kk;
      if (MODE == TC_SYN_U) return x.d.in_off + kk;
      return p.perm[x.d.out_off + kk];
    };
    bool have = seek();
    long long g = 0;
    int src_next = have ? src_of() : -1;
    bool ok = true;
    while (have && ok) {
      const int r0 = x.r0;
      const int src = src_next;
      have = advance();  // the next chunk; its index load is issued now
      if (have) src_next = src_of();
      const int s = int(g % RB);
      if (!waitb(&b_empty[s], unsigned((g / RB) & 1) ^ 1u, abort_flag, p.status)) {
        ok = false;
        break;
      }
      unsigned char* rb = rawB + size_t(s) * RAWB;
      if (in_w && q == 0) cp_async4(kw + s * kTcK + j, src >= 0 ? p.wts + src : p.wts, src >= 0 ? 4u : 0u);
      if (vec) {
        // the tile's right-hand sides r0 .. r0 + NR - 1 of entry src: N floats, 4 per copy (nrhs W
        // is a multiple of 4, so a copy is wholly inside or wholly outside the RHS range)
#pragma unroll
        for (int v = q; v < N / 4; v += P) {
          const bool okc = src >= 0 && (r0 + (v * 4) / W) < p.nrhs;
          const long long a = okc ? ((long long)src * p.is_e + r0) * W + v * 4 : 0;
          cp_async16(rb + (j * N + v * 4) * 4, p.in0 + a, okc ? 16u : 0u);
          if (NB == 2)
            cp_async16(rb + (KW * N + j * N + v * 4) * 4, (okc && p.in1) ? p.in1 + a : p.in0,
                       (okc && p.in1) ? 16u : 0u);
        }
      } else {
        for (int e = q; e < N; e += P) {
          const int n = e / W, cc = e % W;
          const bool okc = src >= 0 && r0 + n < p.nrhs;
          const long long a = okc ? ((long long)src * p.is_e + (long long)(r0 + n) * p.is_k) * W + cc : 0;
          cp_async4(rb + (j * N + e) * 4, p.in0 + a, okc ? 4u : 0u);
          if (NB == 2)
            cp_async4(rb + (KW * N + j * N + e) * 4, (okc && p.in1) ? p.in1 + a : p.in0, (okc && p.in1) ? 4u : 0u);
        }
      }
      cp_async_arrive(&b_full[s]);
      ++g;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    // ------------------------------------------------------------ split, drain, epilogue
    const int mw = warp - kMathWarp0;  // 0 .. kMathWarps - 1
    const int mt = tid - 32 * kMathWarp0;
    const int quad = warp & 3, quarter = mw >> 2;  // TMEM lane quadrant, column group
    static_assert(kMathWarps % 4 == 0, "whole groups of four warps cover the 128 TMEM lanes");
    const int row = quad * 32 + lane;  // TMEM lane = tile row of this thread
    const bool in_w = p.wts && (MODE == TC_SYN_ID || MODE == TC_ADJ_U);
    // Kahan sums of this thread's H columns, in pairs for the packed FP32 instructions: value =
    // acc + cmn (cmn holds the negated compensation)
    float2 acc[H / 2], cmn[H / 2];
#pragma unroll
    for (int j = 0; j < H / 2; ++j) acc[j] = cmn[j] = make_float2(0.f, 0.f);
    // chunks converted but not yet drained (at most kDrainLag), as packed epilogue entries
    int pq[kDrainLag], np = 0;  // oldest first
    auto pop = [&]() {
#pragma unroll
      for (int i = 0; i + 1 < kDrainLag; ++i) pq[i] = pq[i + 1];
      --np;
    };
    bool ok = true;
    int g = 0, gdr = 0;  // chunks converted, chunks drained

    // every lane polls the barrier itself; a lane that gave up sets the abort flag, which makes
    // the others give up as well, so the warp leaves together (the verdict is taken by vote)
    auto wwait = [&](uint64_t* b, unsigned ph) -> bool {
      const bool r = waitb(b, ph, abort_flag, p.status);
      return __all_sync(0xffffffffu, r);
    };
    // Per-unit epilogue data of this thread's row, prepared when the unit starts: the index loads
    // are issued before the unit's first split and their results stored afterwards, so that
    // their latency hides behind the split; the epilogue itself then only loads the identity
    // terms and stores.  A pending entry packs the unit's scalars: last chunk (bit 0), record
    // slot (1), sibling buffer (2), rows (3..10), right-hand sides in the tile (11..17).
    const int col0 = quarter * H;
    const int cc0 = C ? col0 / NR : 0;  // complex: real parts, then imaginary parts
    const int n0 = C ? col0 % NR : col0;
    int us = 0;  // units started by this CTA (record slot = us & 1)
    auto epi_issue = [&](const Unit& x, int& ld0) {  // index load of the row (-1 if none)
      ld0 = -1;
      if (row < x.it.count) {
        const int i = x.it.start + row;
        if (MODE == TC_SYN_ID) ld0 = p.idx[x.d.idx_off + i];
        else if (MODE == TC_ADJ_ID) ld0 = p.idx[x.d.idx_off + x.d.cols + i];
        else if (MODE == TC_SYN_U) ld0 = p.perm[x.d.out_off + i];
      }
    };
    auto epi_store = [&](const Unit& x, int ld0, int slot) -> int {
      int4 e = make_int4(0, 0, 0, __float_as_int(1.f));
      if (row < x.it.count) {
        const int i = x.it.start + row;
        long long dst = 0;
        float w = 1.f;
        if (MODE == TC_SYN_ID) {
          dst = (long long)x.d.out_off + i;
          if (p.wts) w = p.wts[ld0];  // the leaf stage's scale of the skeleton coefficient
          e.z = int(((long long)ld0 * p.is_e + (long long)(x.r0 + n0) * p.is_k) * W + cc0);
        } else if (MODE == TC_ADJ_ID) {
          dst = ld0;
        } else if (MODE == TC_SYN_U) {
          dst = ld0;
          if (p.wts) w = p.wts[ld0];
        } else {
          dst = (long long)x.d.in_off + i;
        }
        const long long o = (dst * p.os_e + (long long)(x.r0 + n0) * p.os_k) * W + cc0;
        e.x = int(o & 0xffffffff);
        e.y = int(o >> 32);
        e.w = __float_as_int(w);
      }
      epi[slot * 32 * kMathWarps + mt] = e;
      return (slot << 1) | ((MODE == TC_ADJ_ID && x.it.sib) ? 4 : 0) | (x.it.count << 3) | (x.nk << 11);
    };
    // rows of a unit: acc (Kahan-compensated sums) + identity term / weights, to the output
    auto epilogue = [&](int entry) {
      const int count = (entry >> 3) & 255, nk = (entry >> 11) & 127;
      if (row < count) {
        const int4 e = epi[((entry >> 1) & 1) * 32 * kMathWarps + mt];
        const long long ooff = (long long)(unsigned)e.x | ((long long)e.y << 32);
        float* o = ((entry & 4) ? p.out1 : p.out0) + ooff;
        const float* ip = p.in0 + e.z;  // identity term of the synthesis ID stage
        const float w = __int_as_float(e.w);
        const int nv = min(H, nk - n0);
        float v[H];
#pragma unroll
        for (int j = 0; j < H; ++j) v[j] = (j & 1) ? acc[j >> 1].y + cmn[j >> 1].y : acc[j >> 1].x + cmn[j >> 1].x;
        if (MODE == TC_SYN_ID) {
          if (!C && p.vec && nv == H) {  // contiguous real rows: 16-byte loads
#pragma unroll
            for (int j = 0; j < H; j += 4) {
              const float4 t = *reinterpret_cast<const float4*>(ip + j);
              v[j] += w * t.x;
              v[j + 1] += w * t.y;
              v[j + 2] += w * t.z;
              v[j + 3] += w * t.w;
            }
          } else {
            const long long istep = p.is_k * W;
#pragma unroll
            for (int j = 0; j < H; ++j)
              if (j < nv) v[j] += w * ip[j * istep];
          }
        }
        if (MODE == TC_SYN_U)
#pragma unroll
          for (int j = 0; j < H; ++j) v[j] *= w;
        if (p.vec_out && nv == H) {
#pragma unroll
          for (int j = 0; j < H; j += 4) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
          const long long ostep = p.os_k * W;
#pragma unroll
          for (int j = 0; j < H; ++j)
            if (j < nv) o[j * ostep] = v[j];
        }
      }
#pragma unroll
      for (int j = 0; j < H / 2; ++j) acc[j] = cmn[j] = make_float2(0.f, 0.f);
    };
    // drain of chunk gdr, first half: wait for its sums and start reading this thread's H
    // columns of its TMEM buffer (the read completes in drain_finish)
    auto drain_start = [&](float (&d)[H]) -> bool {
      const int b = gdr % kTmemBufs;
      if (!wwait(&t_full[b], unsigned((gdr / kTmemBufs) & 1))) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tmem_ld<H>(tmem + (unsigned(quad * 32) << 16) + unsigned(b * N + quarter * H), d);
      return true;
    };
    // second half: frees the buffer, adds the chunk into acc with Kahan compensation, and writes
    // the unit's rows after its last chunk
    auto drain_finish = [&](float (&d)[H], int entry) {
      tmem_wait<H>(d);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&t_empty[gdr % kTmemBufs]);
      ++gdr;
      const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
      for (int n = 0; n < H / 2; ++n) {  // Kahan: y = d - c, t = acc + y, c = (t - acc) - y
        const float2 y = __fadd2_rn(make_float2(d[2 * n], d[2 * n + 1]), cmn[n]);
        const float2 tt = __fadd2_rn(acc[n], y);
        cmn[n] = __fadd2_rn(__ffma2_rn(tt, m1, acc[n]), y);  // (acc - t) + y, exact a - t by the FMA
        acc[n] = tt;
      }
      if (entry & 1) epilogue(entry);
    };
    auto drain_one = [&](int entry) -> bool {
      float d[H];
      if (!drain_start(d)) return false;
      drain_finish(d, entry);
      return true;
    };
    // waits for chunk gg's raw tiles (and, with fewer stages than the drain lag, for the stage
    // to be free)
    auto convert_wait = [&](int gg) -> bool {
      // the stage's previous chunk (gg - NS) must have been consumed by its MMAs.  With at least
      // kDrainLag stages this is already known: every chunk up to gg - kDrainLag has been
      // drained (its sums, and so all earlier MMAs, complete) before chunk gg is split
      if (NS < kDrainLag && !wwait(&mma_done[gg % NS], unsigned((gg / NS) & 1) ^ 1u)) return false;
      return wwait(&a_full[gg % RA], unsigned((gg / RA) & 1)) && wwait(&b_full[gg % RB], unsigned((gg / RB) & 1));
    };
    // splits chunk gg (its raw tiles have arrived) into stage gg % NS
    auto convert = [&](int gg) {
      const int sa_ = gg % RA, sb_ = gg % RB;
      unsigned char* st = stages + (gg % NS) * STAGE;
      // A: raw 128 x 32 FP32 tile, 128-byte rows, 16-byte chunk j of row r at position j ^ (r & 7)
      const unsigned char* ra = rawA + size_t(sa_) * kRawA;
#pragma unroll
      // lane -> (row, 8-column group): the eight lanes of a quarter warp take the eight rows of
      // one core matrix, so that both the swizzled reads and the 16-byte piece stores of a
      // quarter warp fall on distinct banks
      for (int h2 = 0; h2 < 16 / kMathWarps; ++h2) {
        const int r = (mw + kMathWarps * h2) * 8 + (lane & 7), k8 = lane >> 3;
        const float4 v0 = *reinterpret_cast<const float4*>(ra + r * 128 + (((2 * k8) ^ (r & 7)) << 4));
        const float4 v1 = *reinterpret_cast<const float4*>(ra + r * 128 + (((2 * k8 + 1) ^ (r & 7)) << 4));
        const float xv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        put_pieces<BF16>(st, A_PIECE, r, k8, xv);
      }
      // B: row n (accumulator column) x 4 of the 32 real K columns per thread
      const float* rb = reinterpret_cast<const float*>(rawB + size_t(sb_) * RAWB);
      const float* kws = kw + sb_ * kTcK;
      for (int e = mt; e < 8 * N; e += 32 * kMathWarps) {
        const int n = e % N, k4 = e / N;
        float xv[4];
        if (!C) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int k = k4 * 4 + j;
            float v = rb[k * NR + n];
            if (NB == 2) v += rb[KW * NR + k * NR + n];
            if (in_w) v *= kws[k];
            xv[j] = v;
          }
        } else {
          const int rn = n < NR ? n : n - NR;  // right-hand side of this column
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int k = k4 * 2 + j;  // complex entry
            float2 v = *reinterpret_cast<const float2*>(rb + (k * NR + rn) * 2);
            if (NB == 2) {
              const float2 v1 = *reinterpret_cast<const float2*>(rb + (KW * NR + k * NR + rn) * 2);
              v.x += v1.x;
              v.y += v1.y;
            }
            if (in_w) {
              v.x *= kws[k];
              v.y *= kws[k];
            }
            // columns (2k, 2k+1) of A's real view meet (xr, -xi) for real parts, (xi, xr) for imaginary
            xv[2 * j] = n < NR ? v.x : v.y;
            xv[2 * j + 1] = n < NR ? -v.y : v.x;
          }
        }
        // piece j of B (N rows) sits at + j * B_PIECE
        put_pieces4<BF16>(st + NP * A_PIECE, B_PIECE, n, k4, xv);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&s_full[gg % NS]);
        mbar_arrive(&a_empty[sa_]);
        mbar_arrive(&b_empty[sb_]);
      }
    };

    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const Unit x = get_unit<N, C>(p, u);
      if (MODE == TC_ADJ_ID && x.it.start == 0) {
        // identity part of [I | T~] P^T for this tile's right-hand sides: out[skel_j] = z_j
        float* out = x.it.sib ? p.out1 : p.out0;
        for (int e = mt; e < x.d.cols * x.nk * W; e += 32 * kMathWarps) {
          const int j = e / (x.nk * W), q = e % (x.nk * W);
          const long long rhs = x.r0 + q / W;
          const int cc = q % W;
          const long long a = (((long long)x.d.out_off + j) * p.is_e + rhs * p.is_k) * W + cc;
          const long long o = ((long long)p.idx[x.d.idx_off + j] * p.os_e + rhs * p.os_k) * W + cc;
          float v = p.in0[a];
          if (p.in1) v += p.in1[a];
          out[o] = v;
        }
      }
      if (x.nch == 0) {  // no stored columns: drain what is pending, then the rows' identity terms
        while (ok && np > 0) {
          ok = drain_one(pq[0]);
          pop();
        }
        if (!ok) break;
        int ld0;
        epi_issue(x, ld0);
        epilogue(epi_store(x, ld0, us++ & 1) | 1);
        continue;
      }
      int ld0 = -1, ue = 0;  // the unit's epilogue record: index load, then packed entry
      epi_issue(x, ld0);
      for (int c = 0; c < x.nch; ++c, ++g) {
        // the chunk kDrainLag back drains before this chunk's split: its TMEM read is in flight
        // while this chunk's tiles are waited for; the later chunks' MMAs run meanwhile
        if (np == kDrainLag) {
          float d[H];
          if (!(ok = drain_start(d))) break;
          if (!(ok = convert_wait(g))) break;
          drain_finish(d, pq[0]);
          pop();
        } else if (!(ok = convert_wait(g))) {
          break;
        }
        convert(g);
        if (c == 0) ue = epi_store(x, ld0, us++ & 1);  // after the drains of the previous unit
        const int e = ue | (c == x.nch - 1 ? 1 : 0);
#pragma unroll
        for (int i = 0; i < kDrainLag; ++i)
          if (i == np) pq[i] = e;
        ++np;
      }
    }
    while (ok && np > 0) {
      ok = drain_one(pq[0]);
      pop();
    }
  }

  // ---------------------------------------------------------------- clean-up
  __syncthreads();
  if (*abort_flag) {
    // copies and MMAs still in flight must land before shared and tensor memory are released
    if (warp == 0 && lane == 0)
      for (long long j = (a_issued > RA ? a_issued - RA : 0ll); j < a_issued; ++j)
        wait_quiet(&a_full[j % RA], unsigned((j / RA) & 1));
    if (warp == 1 && lane == 0 && mma_issued > 0)
      wait_quiet(&mma_done[(mma_issued - 1) % NS], unsigned(((mma_issued - 1) / NS) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(NCOLS) : "memory");
  }
}


template <int MODE, int N, bool C, bool BF16>
int launch_n(const TcLaunch& a, std::string& err) {
  constexpr int NR = C ? N / 2 : N;
  size_t smem =
      tc_smem<MODE, N, C, BF16>(tc_ra<MODE, N, C, BF16>(), tc_rb<MODE, N, C, BF16>(), tc_ns<MODE, N, C, BF16>());
  // one CTA per SM: its tensor-memory allocation is sized for the whole SM's share
  smem = std::max<size_t>(smem, 120 * 1024);
  auto kern = k_tcs<MODE, N, C, BF16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) {
    err = std::string("tensor-core stage: ") + cudaGetErrorString(e);
    return MHT_ERR_CUDA;
  }
  TcParams p{};
  p.data = a.data;
  p.idx = a.idx;
  p.desc = a.desc;
  p.items = a.items;
  p.tmaps = static_cast<const CUtensorMap*>(a.tmaps);
  p.perm = a.perm;
  p.wts = a.wts;
  p.in0 = a.in0;
  p.in1 = a.in1;
  p.is_e = a.is_e;
  p.is_k = a.is_k;
  p.out0 = a.out0;
  p.out1 = a.out1;
  p.os_e = a.os_e;
  p.os_k = a.os_k;
  p.nitems = int(a.nitems);
  p.ntiles = int((a.nrhs + NR - 1) / NR);
  p.nrhs = int(a.nrhs);
  constexpr int W = C ? 2 : 1;
  const auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  p.vec = (a.is_k == 1 && (a.is_e * W) % 4 == 0 && (a.nrhs * W) % 4 == 0 && al16(a.in0) && (!a.in1 || al16(a.in1)))
              ? 1 : 0;
  p.vec_out = (!C && a.os_k == 1 && a.os_e % 4 == 0 && (a.nrhs % 4) == 0 && al16(a.out0) && (!a.out1 || al16(a.out1)))
                  ? 1 : 0;
  p.status = a.status;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long units = (long long)p.nitems * p.ntiles;
  const int grid = int(std::min<long long>(std::max(sms, 1), units));
  kern<<<grid, kTcThreads, smem, static_cast<cudaStream_t>(a.stream)>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("tensor-core stage launch: ") + cudaGetErrorString(e);
    return MHT_ERR_CUDA;
  }
  return 0;
}

// Accumulator tile: 16, 32 or 64 columns (complex: half as many right-hand sides); wider RHS
// counts take several tiles (work units).
template <int MODE, bool C, bool BF16>
int launch_mode(const TcLaunch& a, std::string& err) {
  const int64_t cols = a.nrhs * (C ? 2 : 1);
  if (cols <= 16) return launch_n<MODE, 16, C, BF16>(a, err);
  if (cols <= 32) return launch_n<MODE, 32, C, BF16>(a, err);
  return launch_n<MODE, 64, C, BF16>(a, err);
}

template <bool C, bool BF16>
int launch_field(const TcLaunch& a, std::string& err) {
  switch (a.mode) {
    case 0: return launch_mode<TC_SYN_ID, C, BF16>(a, err);
    case 1: return launch_mode<TC_ADJ_ID, C, BF16>(a, err);
    case 2: return launch_mode<TC_SYN_U, C, BF16>(a, err);
    default: return launch_mode<TC_ADJ_U, C, BF16>(a, err);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder(std::string& err) {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) {
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return nullptr;
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

}  // namespace

int tc_stage_launch(const TcLaunch& a, std::string& err) {
  if (a.nitems == 0) return 0;
  if (a.bf16) return a.cplx ? launch_field<true, true>(a, err) : launch_field<false, true>(a, err);
  return a.cplx ? launch_field<true, false>(a, err) : launch_field<false, false>(a, err);
}

// One 2-D tensor map per (direction, stage, block) of an FP32 image bound at `base_dev`: the
// stored matrix as rows x (cols * W) FP32 with its padded row stride, boxes of 128 rows x 32
// columns with the 128-byte swizzle; reads outside the matrix return zeros.
int tc_encode_tmaps(const Packed& P, const void* base_dev, std::vector<uint8_t>& out, std::string& err) {
  out.assign(P.tmap_bytes, 0);
  if (P.fp64 || P.tmap_bytes == 0) return 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder(err);
  if (!enc) return MHT_ERR_CUDA;
  const int W = P.cplx ? 2 : 1;
  const int nst = P.L + 2;
  for (int dir = 0; dir < 2; ++dir)
    for (int s = 0; s < nst; ++s) {
      const MhtBlockDesc* d = reinterpret_cast<const MhtBlockDesc*>(P.image.data() + P.st[s].dir[dir].desc_off);
      for (int64_t b = 0; b < P.nb; ++b) {
        CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out.data() + size_t((dir * nst + s) * P.nb + b) * 128);
        const uint8_t* addr = static_cast<const uint8_t*>(base_dev) + P.data_off + size_t(d[b].t_off) * W * 4;
        const cuuint64_t dims[2] = {cuuint64_t(std::max(1, d[b].cols * W)), cuuint64_t(std::max(1, d[b].rows))};
        const cuuint64_t strides[1] = {cuuint64_t(std::max(4, d[b].ldt * W)) * 4};
        const cuuint32_t box[2] = {cuuint32_t(kTcK), cuuint32_t(kTcM)};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<uint8_t*>(addr), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
          err = "cuTensorMapEncodeTiled failed (stage " + std::to_string(s) + ", block " + std::to_string(b) + ")";
          return MHT_ERR_CUDA;
        }
      }
    }
  return 0;
}

}  // namespace mht
