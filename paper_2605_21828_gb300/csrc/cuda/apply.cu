// Butterfly apply kernels for sm_103a (synthesis and its adjoint).
//
// The apply of a row-wise butterfly factorization (Sec. 2): synthesis multiplies by the
// leaf interpolation matrices V^* (stage 0), then by the transfer matrices R^* of levels
// l = 1..L, then by the column bases U; the adjoint runs U^H, R^H (l = L..1), V^H.  Every
// interpolation matrix is [I | T~] P^T, so a block applies as
//     synthesis  y_i = x[skel_i] + sum_j T~_ij x[rest_j]
//     adjoint    u[skel_i] = z_i,   u[rest_j] = sum_i conj(T~_ij) z_i
// and the column-basis stage is a dense block product.  Each stored matrix is read exactly
// once per apply (apply cost equals storage, Sec. 6.2), so the single-RHS apply is bound by
// HBM bandwidth.  The packed plan holds every matrix in both orientations, so both
// directions are "rows times a gathered vector":
//   * one CTA per work item (block, row range of ~32 KB);
//   * thread 0 stages the item's rows into shared memory with one 1-D TMA bulk copy
//     (cp.async.bulk, completion on an mbarrier) while all threads gather the block's
//     input vector from L2 into shared memory;
//   * each warp then reduces whole rows from shared memory with 128-bit loads and warp
//     shuffles.
// The adjoint is a gather: the sibling blocks (2p, nu), (2p+1, nu) that share an input pair
// write separate buffers and the next stage sums them while loading -- no atomics, so the
// result is deterministic.  Every mbarrier wait is bounded; on timeout the kernel sets a bit
// in the workspace status word (read by mht_plan_check) instead of hanging.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../host/internal.h"

namespace mht {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded waits give up after 2 s

enum Mode { SYN_ID = 0, ADJ_ID = 1, SYN_U = 2, ADJ_U = 3 };

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity; gives up after kWaitNs of wall time, or as soon
// as *abort_flag is non-zero (when given).  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase,
                                                  const unsigned* abort_flag = nullptr) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 255) == 0) {
      if (globaltimer_ns() - t0 > kWaitNs) return false;
      if (abort_flag && *reinterpret_cast<const volatile unsigned*>(abort_flag) != 0u) return false;
    }
  }
}

template <class R>
struct alignas(16) Vec16 {  // one 128-bit load / store
  static constexpr int NS = 16 / sizeof(R);
  R s[NS];
};

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// out[o(i)] = ident(i) + sum_j M[i, j] x[j] for the rows i of one work item.
//   SYN_ID: M = T~ (r x K'),           x[j] = in[idx[r + j]],   o(i) = out_off + i,
//           ident(i) = in[idx[i]]
//   ADJ_ID: M = conj(T~)^T (K' x r),   x[j] = z0[out_off + j] (+ z1[...]),
//           o(i) = idx[r + i] in the sibling buffer; skeleton out[idx[j]] = x[j]
//   SYN_U:  M = U (|tau| x r_L),       x[j] = yL[in_off + j],   o(i) = perm[out_off + i]
//           (times w[o(i)] when weights are given)
//   ADJ_U:  M = conj(U)^T (r_L x |tau|), x[j] = w[p] f[p] with p = perm[out_off + j],
//           o(i) = in_off + i
// Element strides: in[e * is_e + k * is_k], out[e * os_e + k * os_k]; one complex value is
// one element.  RT right-hand sides per CTA (blockIdx.y selects the RHS tile).
template <class R, bool C, int RT, int MODE>
__global__ void __launch_bounds__(kThreads)
k_rowdot(const R* __restrict__ data, const int* __restrict__ idx, const MhtBlockDesc* __restrict__ desc,
         const MhtItem* __restrict__ items, const int* __restrict__ perm, const R* __restrict__ wts,
         const R* __restrict__ in0, const R* __restrict__ in1, long long is_e, long long is_k,
         R* __restrict__ out0, R* __restrict__ out1, long long os_e, long long os_k, int nrhs,
         int tile_bytes_max, int ldx_max, unsigned* __restrict__ status) {
  constexpr int W = C ? 2 : 1;
  constexpr int NS = 16 / sizeof(R);
  constexpr int E = NS / W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  R* tile = reinterpret_cast<R*>(smem_raw + 128);
  R* xs = reinterpret_cast<R*>(smem_raw + 128 + ((tile_bytes_max + 127) / 128) * 128);  // [RT][ldx][W]

  const MhtItem it = items[blockIdx.x];
  const MhtBlockDesc d = desc[it.blk];
  const int k0 = blockIdx.y * RT;
  const int nk = min(RT, nrhs - k0);
  const int ldt = d.ldt;
  const unsigned bytes = unsigned(it.count) * unsigned(ldt) * unsigned(W * sizeof(R));
  R* out = (MODE == ADJ_ID && it.sib) ? out1 : out0;

  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && bytes > 0) {
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(tile, data + (d.t_off + (long long)it.start * ldt) * W, bytes, bar);
  }

  // gather the input vector while the tile is in flight (zero padding to ldt and beyond nk)
  for (int j = threadIdx.x; j < ldt; j += kThreads) {
    long long src = -1;
    R w = R(1);
    if (j < d.cols) {
      if (MODE == SYN_ID) src = idx[d.idx_off + d.rows + j];
      else if (MODE == ADJ_ID) src = (long long)d.out_off + j;
      else if (MODE == SYN_U) src = (long long)d.in_off + j;
      else {
        src = perm[d.out_off + j];
        if (wts) w = wts[src];
      }
    }
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) {
        R v = R(0);
        if (src >= 0 && t < nk) {
          const long long a = (src * is_e + (long long)(k0 + t) * is_k) * W + c;
          v = in0[a];
          if (MODE == ADJ_ID && in1) v += in1[a];
          v *= w;
        }
        xs[(t * ldx_max + j) * W + c] = v;
      }
  }
  __syncthreads();

  if (MODE == ADJ_ID && it.start == 0) {  // identity part: out[skel_j] = z_j
    for (int e = threadIdx.x; e < d.cols * nk; e += kThreads) {
      const int j = e / nk, t = e % nk;
      const long long dst = idx[d.idx_off + j];
#pragma unroll
      for (int c = 0; c < W; ++c)
        out[(dst * os_e + (long long)(k0 + t) * os_k) * W + c] = xs[(t * ldx_max + j) * W + c];
    }
  }
  if (it.count == 0) return;

  if (bytes > 0 && !mbar_wait_bounded(bar, 0)) {
    if (threadIdx.x == 0) atomicOr(status, 1u);
    mbar_wait_bounded(bar, 0);  // let the copy land before the CTA releases shared memory
    return;
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec = ldt / E;
  for (int ii = warp; ii < it.count; ii += kWarps) {
    const int i = it.start + ii;
    R acc[RT][W];
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[t][c] = R(0);
    const R* row = tile + (long long)ii * ldt * W;
    for (int v = lane; v < nvec; v += 32) {
      const Vec16<R> tv = *reinterpret_cast<const Vec16<R>*>(row + v * NS);
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        const Vec16<R> xv = *reinterpret_cast<const Vec16<R>*>(xs + (t * ldx_max + v * E) * W);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (C) {
            const R a = tv.s[2 * e], b = tv.s[2 * e + 1];
            const R xr = xv.s[2 * e], xi = xv.s[2 * e + 1];
            acc[t][0] += a * xr - b * xi;
            acc[t][W - 1] += a * xi + b * xr;
          } else {
            acc[t][0] += tv.s[e] * xv.s[e];
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[t][c] = warp_sum(acc[t][c]);
    if (lane < nk) {
      const int t = lane;
      R val[W];
#pragma unroll
      for (int tt = 0; tt < RT; ++tt)
        if (tt == t)
#pragma unroll
          for (int c = 0; c < W; ++c) val[c] = acc[tt][c];
      long long dst;
      if (MODE == SYN_ID) {
        const long long s = idx[d.idx_off + i];
#pragma unroll
        for (int c = 0; c < W; ++c) val[c] += in0[(s * is_e + (long long)(k0 + t) * is_k) * W + c];
        dst = (long long)d.out_off + i;
      } else if (MODE == ADJ_ID) {
        dst = idx[d.idx_off + d.cols + i];
      } else if (MODE == SYN_U) {
        dst = perm[d.out_off + i];
        if (wts) {
          const R w = wts[dst];
#pragma unroll
          for (int c = 0; c < W; ++c) val[c] *= w;
        }
      } else {
        dst = (long long)d.in_off + i;
      }
#pragma unroll
      for (int c = 0; c < W; ++c) out[(dst * os_e + (long long)(k0 + t) * os_k) * W + c] = val[c];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Persistent fused apply: every stage of one direction in a single launch.
//
// Three warp roles per CTA (one CTA per SM):
//  * producer (warp 0, lane 0): takes work items from a global queue in dependency order,
//    hands each to the gather warps through a small item queue, and streams its rows in
//    chunks of at most one slot into a kSlots-deep shared-memory ring with 1-D TMA bulk
//    copies (full/empty mbarriers).  Matrix tiles do not depend on earlier stages, so the
//    producer runs ahead of the data dependencies and keeps HBM busy.
//  * gather warps (kGatherWarps): one item ahead of the math, wait (bounded) until the
//    blocks the item reads are complete, then stage its input vector, its identity terms
//    and its output indices in one of two shared-memory buffers.
//  * compute warps (kComputeWarps): for every chunk, reduce rows from shared memory and
//    store results; the last warp to finish an item publishes it with a release fence and a
//    per-block completion counter.  No CTA-wide barrier sits on this path.
// Items are dequeued in increasing order and only wait on smaller items, so the oldest
// unfinished item can always proceed: no deadlock, whether or not all CTAs are resident.
// Intermediate vectors are read with L2-only loads (.cg), so a stale L1 line from a
// neighbouring block is never used.  Every wait is bounded in time and watches the status
// word, so an error ends the launch instead of hanging it.
constexpr int kSlots = 4;
constexpr int kItemQ = 4;
constexpr int kComputeWarps = 16;
constexpr int kGatherWarps = 4;
constexpr int kFusedThreads = 32 * (1 + kGatherWarps + kComputeWarps);

template <class R>
struct FusedParams {
  const R* data;
  const int* idx;
  const int* perm;
  const R* wts;               // analysis / weighted-synthesis weights or null
  const MhtBlockDesc* desc;   // [(L+2) * nb], stage-major, this direction
  const int* targets;         // [(L+2) * nb] items per block
  const MhtPItem* items;
  int nitems;
  const long long* vec_off;   // [L+2]
  const R* cin;               // synthesis input c (column-major, ldc)
  R* cout;                    // analysis output c
  const R* fin;               // analysis input f (ldf)
  R* fout;                    // synthesis output f
  long long ldc, ldf;
  R* Y;                       // synthesis level vectors
  R* A0;                      // analysis sibling buffers
  R* A1;
  unsigned* done;             // [(L+2) * nb] completed items per block
  unsigned* queue;
  unsigned* status;
  int L, nb, nrhs, slot_bytes, ldx, mrows;
};

struct ItemInfo {
  MhtPItem it;
  MhtBlockDesc d;
};

__device__ __forceinline__ void bar_gather() {
  asm volatile("bar.sync 2, %0;" ::"n"(32 * kGatherWarps) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool aborted(const unsigned* status) {
  return *reinterpret_cast<const volatile unsigned*>(status) != 0u;
}

// Wait until block `b` of stage `s` has all its items done; false on timeout / abort.
__device__ __forceinline__ bool wait_block(const unsigned* done, const int* targets, int s, int nb, int b,
                                           const unsigned* status) {
  const unsigned* cnt = done + (long long)s * nb + b;
  const unsigned tgt = unsigned(targets[(long long)s * nb + b]);
  if (ld_acquire(cnt) >= tgt) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    __nanosleep(it < 64 ? 32 : 256);
    if (ld_acquire(cnt) >= tgt) return true;
    if ((it & 15) == 0 && (globaltimer_ns() - t0 > kWaitNs || aborted(status))) return false;
  }
}

// Stage input / output bases and element strides (one complex value = one element).
template <class R, int DIR, int W>
struct StageIO {
  const R* in0;
  const R* in1;
  R* out;
  long long is_e, is_k, os_e, os_k;
  __device__ __forceinline__ StageIO(const FusedParams<R>& p, int st, int blk) {
    const int L = p.L;
    const long long nr = p.nrhs;
    in1 = nullptr;
    is_e = nr; is_k = 1; os_e = nr; os_k = 1;
    if (DIR == 0) {
      in0 = st == 0 ? p.cin : p.Y + p.vec_off[st - 1] * nr * W;
      if (st == 0) { is_e = 1; is_k = p.ldc; }
      if (st == L + 1) { out = p.fout; os_e = 1; os_k = p.ldf; }
      else out = p.Y + p.vec_off[st] * nr * W;
    } else if (st == L + 1) {
      in0 = p.fin; is_e = 1; is_k = p.ldf;
      out = p.A0 + p.vec_off[L] * nr * W;
    } else {
      in0 = p.A0 + p.vec_off[st] * nr * W;
      in1 = st == L ? nullptr : p.A1 + p.vec_off[st] * nr * W;
      if (st == 0) { out = p.cout; os_e = 1; os_k = p.ldc; }
      else out = (((blk >> (L - st)) & 1) ? p.A1 : p.A0) + p.vec_off[st - 1] * nr * W;
    }
  }
};

template <class R, bool C, int RT, int DIR>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fused(FusedParams<R> p) {
  constexpr int W = C ? 2 : 1;
  constexpr int NS = 16 / sizeof(R);
  constexpr int E = NS / W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kSlots;
  uint64_t* iq_full = empty + kSlots;
  uint64_t* iq_empty = iq_full + kItemQ;
  uint64_t* xready = iq_empty + kItemQ;
  uint64_t* xfree = xready + 2;
  int* item_cnt = reinterpret_cast<int*>(smem_raw + 192);   // [2]
  int* iq = reinterpret_cast<int*>(smem_raw + 208);         // [kItemQ]
  int4* meta = reinterpret_cast<int4*>(smem_raw + 256);     // [kSlots] {seq, row0, rows, flags}
  ItemInfo* info = reinterpret_cast<ItemInfo*>(smem_raw + 320);  // [2]
  unsigned char* slots = smem_raw + 512;
  R* xs = reinterpret_cast<R*>(slots + size_t(kSlots) * p.slot_bytes);  // [2][RT][ldx][W]
  R* ident = xs + size_t(2) * RT * p.ldx * W;                            // [2][RT][mrows][W]
  int* oidx = reinterpret_cast<int*>(ident + size_t(2) * RT * p.mrows * W);  // [2][mrows]
  const int es = W * sizeof(R);
  const int L = p.L;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kSlots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kComputeWarps);
    }
    for (int i = 0; i < kItemQ; ++i) {
      mbar_init(&iq_full[i], 1);
      mbar_init(&iq_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&xready[i], 1);
      mbar_init(&xfree[i], kComputeWarps);
      item_cnt[i] = 0;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    // ------------------------------------------------------------------ producer
    if (lane != 0) return;
    long long issued = 0;
    int k = 0;
    bool ok = true;
    for (;; ++k) {
      if (aborted(p.status)) { ok = false; break; }
      const int item = int(atomicAdd(p.queue, 1u));
      if (item >= p.nitems) break;
      if (!mbar_wait_bounded(&iq_empty[k % kItemQ], unsigned(((k / kItemQ) & 1) ^ 1), p.status)) {
        atomicOr(p.status, 2u);
        ok = false;
        break;
      }
      iq[k % kItemQ] = item;
      mbar_arrive(&iq_full[k % kItemQ]);
      const MhtPItem it = p.items[item];
      const MhtBlockDesc d = p.desc[(long long)it.stage * p.nb + it.blk];
      const int rowbytes = d.ldt * es;
      const int rpc = rowbytes > 0 ? max(1, p.slot_bytes / rowbytes) : max(1, it.count);
      const int nch = it.count == 0 ? 1 : (it.count + rpc - 1) / rpc;
      for (int ch = 0; ch < nch; ++ch) {
        const int s = int(issued % kSlots);
        const unsigned ph = unsigned((issued / kSlots) & 1);
        if (!mbar_wait_bounded(&empty[s], ph ^ 1u, p.status)) {
          atomicOr(p.status, 2u);
          ok = false;
          break;
        }
        const int r0 = ch * rpc;
        const int rows = it.count == 0 ? 0 : min(rpc, it.count - r0);
        meta[s] = make_int4(k, r0, rows, (ch == 0 ? 1 : 0) | (ch == nch - 1 ? 2 : 0));
        const unsigned bytes = unsigned(rows) * unsigned(rowbytes);
        mbar_expect_tx(&full[s], bytes);
        if (bytes > 0)
          bulk_copy_g2s(slots + size_t(s) * p.slot_bytes, p.data + (d.t_off + (long long)(it.start + r0) * d.ldt) * W,
                        bytes, &full[s]);
        ++issued;
      }
      if (!ok) break;
    }
    if (ok) {
      // end markers for the gather and compute warps
      const bool qok = mbar_wait_bounded(&iq_empty[k % kItemQ], unsigned(((k / kItemQ) & 1) ^ 1), p.status);
      if (qok) {
        iq[k % kItemQ] = -1;
        mbar_arrive(&iq_full[k % kItemQ]);
      }
      const int s = int(issued % kSlots);
      const unsigned ph = unsigned((issued / kSlots) & 1);
      if (qok && mbar_wait_bounded(&empty[s], ph ^ 1u, p.status)) {
        meta[s] = make_int4(-1, 0, 0, 0);
        mbar_expect_tx(&full[s], 0);
        return;  // the compute warps consume every earlier chunk before the marker
      }
      atomicOr(p.status, 2u);
    }
    // error path: every copy issued must land before the CTA's shared memory is released
    for (long long j = (issued > kSlots ? issued - kSlots : 0ll); j < issued; ++j)
      mbar_wait_bounded(&full[j % kSlots], unsigned((j / kSlots) & 1));
    return;
  }

  if (warp <= kGatherWarps) {
    // ------------------------------------------------------------------ gather warps
    const int g = threadIdx.x - 32;
    constexpr int NG = 32 * kGatherWarps;
    volatile int* gflag = reinterpret_cast<volatile int*>(smem_raw + 224);  // broadcast slot
    for (int k = 0;; ++k) {
      const int b = k & 1;
      // one thread waits for the next item and for its buffer; the group leaves together
      if (g == 0) {
        int item = -2;
        if (mbar_wait_bounded(&iq_full[k % kItemQ], unsigned((k / kItemQ) & 1), p.status)) {
          item = iq[k % kItemQ];
          mbar_arrive(&iq_empty[k % kItemQ]);
          if (item >= 0 && !mbar_wait_bounded(&xfree[b], unsigned(((k >> 1) & 1) ^ 1), p.status)) item = -2;
        }
        if (item == -2) atomicOr(p.status, 16u);
        *gflag = item;
      }
      bar_gather();
      const int item = *gflag;
      bar_gather();
      if (item < 0) return;
      const MhtPItem it = p.items[item];
      const MhtBlockDesc d = p.desc[(long long)it.stage * p.nb + it.blk];
      const int st = it.stage;
      const bool ustage = (st == L + 1);
      if (g == 0) {
        bool ok = true;
        const int nbs = 1 << (L - min(st, L));
        if (DIR == 0 && st >= 1 && st <= L) {
          const int tau = it.blk / nbs, nu = it.blk % nbs, q = (tau >> 1) * (nbs << 1) + 2 * nu;
          ok = wait_block(p.done, p.targets, st - 1, p.nb, q, p.status) &&
               wait_block(p.done, p.targets, st - 1, p.nb, q + 1, p.status);
        } else if (DIR == 0 && ustage) {
          ok = wait_block(p.done, p.targets, L, p.nb, it.blk, p.status);
        } else if (DIR == 1 && st == L) {
          ok = wait_block(p.done, p.targets, L + 1, p.nb, it.blk, p.status);
        } else if (DIR == 1 && st < L) {
          const int tau = it.blk / nbs, nu = it.blk % nbs, nb1 = nbs >> 1;
          ok = wait_block(p.done, p.targets, st + 1, p.nb, (2 * tau) * nb1 + (nu >> 1), p.status) &&
               wait_block(p.done, p.targets, st + 1, p.nb, (2 * tau + 1) * nb1 + (nu >> 1), p.status);
        }
        if (!ok) atomicOr(p.status, 8u);
        info[b].it = it;
        info[b].d = d;
      }
      bar_gather();
      const StageIO<R, DIR, W> io(p, st, it.blk);
      const int nr = p.nrhs;
      R* xb = xs + size_t(b) * RT * p.ldx * W;
      // input vector (zero padding to ldt and beyond nrhs)
#pragma unroll 4
      for (int j = g; j < d.ldt; j += NG) {
        long long src = -1;
        R w = R(1);
        if (j < d.cols) {
          if (DIR == 0 && !ustage) src = p.idx[d.idx_off + d.rows + j];
          else if (DIR == 1 && !ustage) src = (long long)d.out_off + j;
          else if (DIR == 0) src = (long long)d.in_off + j;
          else {
            src = p.perm[d.out_off + j];
            if (p.wts) w = p.wts[src];
          }
        }
#pragma unroll
        for (int t = 0; t < RT; ++t)
#pragma unroll
          for (int c = 0; c < W; ++c) {
            R v = R(0);
            if (src >= 0 && t < nr) {
              const long long a = (src * io.is_e + (long long)t * io.is_k) * W + c;
              v = __ldcg(io.in0 + a);
              if (io.in1) v += __ldcg(io.in1 + a);
              v *= w;
            }
            xb[(t * p.ldx + j) * W + c] = v;
          }
      }
      // per-row identity terms, weights and output indices of this item
      R* ib = ident + size_t(b) * RT * p.mrows * W;
      int* ob = oidx + size_t(b) * p.mrows;
#pragma unroll 4
      for (int i = g; i < it.count; i += NG) {
        const int row = it.start + i;
        if (DIR == 0 && !ustage) {
          const long long sidx = p.idx[d.idx_off + row];
#pragma unroll
          for (int t = 0; t < RT; ++t)
#pragma unroll
            for (int c = 0; c < W; ++c)
              ib[(t * p.mrows + i) * W + c] =
                  t < nr ? __ldcg(io.in0 + (sidx * io.is_e + (long long)t * io.is_k) * W + c) : R(0);
        } else if (DIR == 1 && !ustage) {
          ob[i] = p.idx[d.idx_off + d.cols + row];
        } else if (DIR == 0) {
          const int dst = p.perm[d.out_off + row];
          ob[i] = dst;
          ib[i * W] = p.wts ? p.wts[dst] : R(1);
        }
      }
      if (DIR == 1 && !ustage && it.start == 0) {  // identity part: out[skel_j] = z_j
        bar_gather();  // the staged vector is complete (entries come from other threads)
        for (int e = g; e < d.cols * nr; e += NG) {
          const int j = e / nr, t = e % nr;
          const long long dst = p.idx[d.idx_off + j];
#pragma unroll
          for (int c = 0; c < W; ++c)
            io.out[(dst * io.os_e + (long long)t * io.os_k) * W + c] = xb[(t * p.ldx + j) * W + c];
        }
        __threadfence();  // visible before the compute warps publish the item
      }
      bar_gather();
      if (g == 0) mbar_arrive(&xready[b]);
    }
  }

  // -------------------------------------------------------------------- compute warps
  const int cw = warp - 1 - kGatherWarps;
  for (long long iter = 0;; ++iter) {
    const int s = int(iter % kSlots);
    const unsigned ph = unsigned((iter / kSlots) & 1);
    // lane 0 waits for the chunk (and, at an item's first chunk, for its staged vectors);
    // the whole warp follows its verdict
    int okw = 1;
    if (lane == 0) {
      okw = mbar_wait_bounded(&full[s], ph, p.status) ? 1 : 0;
      if (okw) {
        const int4 m0 = meta[s];
        if (m0.x >= 0 && (m0.w & 1) && !mbar_wait_bounded(&xready[m0.x & 1], unsigned((m0.x >> 1) & 1), p.status))
          okw = 0;
      }
      if (!okw) atomicOr(p.status, 4u);
    }
    okw = __shfl_sync(0xffffffffu, okw, 0);
    if (!okw) return;
    const int4 m = meta[s];
    if (m.x < 0) return;
    const int k = m.x, b = k & 1;
    const MhtPItem it = info[b].it;
    const MhtBlockDesc d = info[b].d;
    const int st = it.stage;
    const bool ustage = (st == L + 1);
    const StageIO<R, DIR, W> io(p, st, it.blk);
    const int nr = p.nrhs;
    const R* xb = xs + size_t(b) * RT * p.ldx * W;
    const R* ib = ident + size_t(b) * RT * p.mrows * W;
    const int* ob = oidx + size_t(b) * p.mrows;
    const R* tile = reinterpret_cast<const R*>(slots + size_t(s) * p.slot_bytes);
    const int nvec = d.ldt / E;
    for (int ii = cw; ii < m.z; ii += kComputeWarps) {
      const int il = m.y + ii;  // row within the item
      R acc[RT][W];
#pragma unroll
      for (int t = 0; t < RT; ++t)
#pragma unroll
        for (int c = 0; c < W; ++c) acc[t][c] = R(0);
      const R* row = tile + (long long)ii * d.ldt * W;
      for (int v = lane; v < nvec; v += 32) {
        const Vec16<R> tv = *reinterpret_cast<const Vec16<R>*>(row + v * NS);
#pragma unroll
        for (int t = 0; t < RT; ++t) {
          const Vec16<R> xv = *reinterpret_cast<const Vec16<R>*>(xb + (t * p.ldx + v * E) * W);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            if (C) {
              const R a = tv.s[2 * e], bb = tv.s[2 * e + 1];
              const R xr = xv.s[2 * e], xi = xv.s[2 * e + 1];
              acc[t][0] += a * xr - bb * xi;
              acc[t][W - 1] += a * xi + bb * xr;
            } else {
              acc[t][0] += tv.s[e] * xv.s[e];
            }
          }
        }
      }
#pragma unroll
      for (int t = 0; t < RT; ++t)
#pragma unroll
        for (int c = 0; c < W; ++c) acc[t][c] = warp_sum(acc[t][c]);
      if (lane < nr && lane < RT) {
        const int t = lane;
        R val[W];
#pragma unroll
        for (int tt = 0; tt < RT; ++tt)
          if (tt == t)
#pragma unroll
            for (int c = 0; c < W; ++c) val[c] = acc[tt][c];
        long long dst;
        if (DIR == 0 && !ustage) {
#pragma unroll
          for (int c = 0; c < W; ++c) val[c] += ib[(t * p.mrows + il) * W + c];
          dst = (long long)d.out_off + it.start + il;
        } else if (DIR == 1 && !ustage) {
          dst = ob[il];
        } else if (DIR == 0) {
          dst = ob[il];
          const R w = ib[il * W];
#pragma unroll
          for (int c = 0; c < W; ++c) val[c] *= w;
        } else {
          dst = (long long)d.in_off + it.start + il;
        }
#pragma unroll
        for (int c = 0; c < W; ++c) io.out[(dst * io.os_e + (long long)t * io.os_k) * W + c] = val[c];
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (m.w & 2) {  // this warp is done with the item
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        if (atomicAdd(&item_cnt[b], 1) == kComputeWarps - 1) {
          item_cnt[b] = 0;
          __threadfence();
          atomicAdd(p.done + (long long)st * p.nb + it.blk, 1u);
        }
        mbar_arrive(&xfree[b]);
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Stage timing (mht_plan_profile): CUDA events around each launch.
struct Profiler {
  struct Rec {
    int dir, stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

Profiler* profiler_create() { return new Profiler(); }

void profiler_destroy(Profiler* p) {
  if (!p) return;
  for (auto& r : p->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->pool) cudaEventDestroy(e);
  delete p;
}

int profiler_read(Profiler* p, int direction, int nstages, double* ms, int64_t* launches, std::string& err) {
  for (int s = 0; s < nstages; ++s) {
    ms[s] = 0;
    launches[s] = 0;
  }
  std::vector<Profiler::Rec> keep;
  int rc = 0;
  for (auto& r : p->recs) {
    if (r.dir != direction) {
      keep.push_back(r);
      continue;
    }
    float t = 0;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && !rc) {
      err = std::string("stage timing: ") + cudaGetErrorString(e);
      rc = MHT_ERR_CUDA;
    }
    if (r.stage >= 0 && r.stage < nstages) {
      ms[r.stage] += t;
      launches[r.stage] += 1;
    }
    p->pool.push_back(r.a);
    p->pool.push_back(r.b);
  }
  p->recs.swap(keep);
  return rc;
}

namespace {

struct StageTimer {
  Profiler* p;
  int dir, stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(Profiler* p_, int d, int st, cudaStream_t s_) : p(p_), dir(d), stage(st), s(s_) {
    if (p) {
      a = p->get();
      cudaEventRecord(a, s);
    }
  }
  ~StageTimer() {
    if (p) {
      cudaEvent_t b = p->get();
      cudaEventRecord(b, s);
      p->recs.push_back({dir, stage, a, b});
    }
  }
};

struct Ctx {
  const Factorization& F;
  const Packed& P;
  const DeviceView& d;
  cudaStream_t s;
  int64_t nrhs;
  std::string& err;
};

int check(cudaError_t e, std::string& err, const char* what) {
  if (e == cudaSuccess) return 0;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return MHT_ERR_CUDA;
}

// Workspace level vectors: region 0 = Y (synthesis), 1 = A0, 2 = A1 (adjoint siblings);
// level l of a region starts at vec_off[l] entries (times nrhs).
void* lvl(const Ctx& c, int region, int l) {
  return c.d.ws + region * c.P.ws_vec_bytes(c.d.max_nrhs) + size_t(c.P.vec_off[l]) * c.nrhs * c.P.elem_bytes;
}
unsigned* status_ptr(const Ctx& c) {
  return reinterpret_cast<unsigned*>(c.d.ws + c.P.status_offset(c.d.max_nrhs, c.F.n, c.F.m));
}

size_t stage_smem(const Packed& P, const Stage& S, int dir, int rt) {
  const size_t tile = (S.dir[dir].max_tile_bytes + 127) / 128 * 128;
  return 128 + tile + size_t(std::max<int64_t>(S.dir[dir].max_ld, 1)) * rt * P.elem_bytes;
}

template <class R, bool C, int RT, int MODE>
int launch(const Ctx& c, int s, const void* in0, const void* in1, long long is_e, long long is_k, void* out0,
           void* out1, long long os_e, long long os_k, const void* w) {
  const int dir = (MODE == ADJ_ID || MODE == ADJ_U) ? 1 : 0;
  const Stage& S = c.P.st[s];
  const StageDir& D = S.dir[dir];
  if (D.nitems == 0) return 0;
  const size_t smem = stage_smem(c.P, S, dir, RT);
  if (smem > 227 * 1024) {
    c.err = "a stage needs more shared memory than an SM has for this RHS tile";
    return MHT_ERR_UNSUPPORTED;
  }
  auto kern = k_rowdot<R, C, RT, MODE>;
  if (smem > 48 * 1024)
    if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), c.err,
                       "shared memory attribute"))
      return rc;
  const uint8_t* base = c.d.base;
  dim3 grid(unsigned(D.nitems), unsigned((c.nrhs + RT - 1) / RT));
  StageTimer timer(c.d.prof, dir, s, c.s);
  kern<<<grid, kThreads, smem, c.s>>>(
      reinterpret_cast<const R*>(base + c.P.data_off), reinterpret_cast<const int*>(base + c.P.index_off),
      reinterpret_cast<const MhtBlockDesc*>(base + D.desc_off), reinterpret_cast<const MhtItem*>(base + D.items_off),
      reinterpret_cast<const int*>(base + c.P.perm_off), static_cast<const R*>(w), static_cast<const R*>(in0),
      static_cast<const R*>(in1), is_e, is_k, static_cast<R*>(out0), static_cast<R*>(out1), os_e, os_k,
      int(c.nrhs), int(D.max_tile_bytes), int(std::max<int64_t>(D.max_ld, 1)), status_ptr(c));
  return check(cudaGetLastError(), c.err, "apply launch");
}

template <class R, bool C, int RT>
int synth_impl(const Ctx& c, const void* cin, int64_t ldc, void* f, int64_t ldf, bool weighted) {
  const int L = c.F.L;
  const long long nr = c.nrhs;
  int rc = launch<R, C, RT, SYN_ID>(c, 0, cin, nullptr, 1, ldc, lvl(c, 0, 0), nullptr, nr, 1, nullptr);
  for (int l = 1; l <= L && !rc; ++l)
    rc = launch<R, C, RT, SYN_ID>(c, l, lvl(c, 0, l - 1), nullptr, nr, 1, lvl(c, 0, l), nullptr, nr, 1, nullptr);
  if (rc) return rc;
  const void* w = weighted ? (const void*)(c.d.base + c.P.weights_off) : nullptr;
  return launch<R, C, RT, SYN_U>(c, L + 1, lvl(c, 0, L), nullptr, nr, 1, f, nullptr, 1, ldf, w);
}

template <class R, bool C, int RT>
int adjoint_impl(const Ctx& c, const void* f, int64_t ldf, void* cout, int64_t ldc, bool weighted) {
  const int L = c.F.L;
  const long long nr = c.nrhs;
  const void* w = weighted ? (const void*)(c.d.base + c.P.weights_off) : nullptr;
  // U^H: f -> z_L (region A0, level L)
  int rc = launch<R, C, RT, ADJ_U>(c, L + 1, f, nullptr, 1, ldf, lvl(c, 1, L), nullptr, nr, 1, w);
  for (int l = L; l >= 1 && !rc; --l)
    rc = launch<R, C, RT, ADJ_ID>(c, l, lvl(c, 1, l), l == L ? nullptr : lvl(c, 2, l), nr, 1, lvl(c, 1, l - 1),
                                  lvl(c, 2, l - 1), nr, 1, nullptr);
  if (rc) return rc;
  return launch<R, C, RT, ADJ_ID>(c, 0, lvl(c, 1, 0), L == 0 ? nullptr : lvl(c, 2, 0), nr, 1, cout, cout, 1, ldc,
                                  nullptr);
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

size_t fused_smem(const Packed& P, int dir, int rt) {
  const FusedDir& FD = P.fused[dir];
  const size_t mrows = size_t(std::max<int64_t>(FD.max_item_rows, 1));
  return 512 + size_t(kSlots) * FD.slot_bytes + 2 * size_t(std::max<int64_t>(FD.max_ld, 1)) * rt * P.elem_bytes +
         2 * mrows * rt * P.elem_bytes + 2 * mrows * sizeof(int);
}

unsigned* counters(const Ctx& c, int dir) {
  unsigned* base = reinterpret_cast<unsigned*>(c.d.ws + c.P.ws_counters_offset(c.d.max_nrhs, c.F.n, c.F.m));
  return base + size_t(dir) * (size_t(c.P.L + 2) * c.P.nb + 1);
}

// One launch for every stage of a direction (returns -1 when the shared memory does not fit).
template <class R, bool C, int RT, int DIR>
int fused_launch(const Ctx& c, const void* in, long long ld_in, void* out, long long ld_out, bool weighted) {
  const FusedDir& FD = c.P.fused[DIR];
  const size_t smem = fused_smem(c.P, DIR, RT);
  if (smem > 227 * 1024) return -1;
  auto kern = k_fused<R, C, RT, DIR>;
  if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), c.err,
                     "shared memory attribute"))
    return rc;
  const size_t ncnt = size_t(c.P.L + 2) * c.P.nb + 1;
  unsigned* cnt = counters(c, DIR);
  if (int rc = check(cudaMemsetAsync(cnt, 0, ncnt * sizeof(unsigned), c.s), c.err, "counter reset")) return rc;
  if (FD.nitems == 0) return 0;
  const uint8_t* base = c.d.base;
  FusedParams<R> p;
  p.data = reinterpret_cast<const R*>(base + c.P.data_off);
  p.idx = reinterpret_cast<const int*>(base + c.P.index_off);
  p.perm = reinterpret_cast<const int*>(base + c.P.perm_off);
  p.wts = weighted ? reinterpret_cast<const R*>(base + c.P.weights_off) : nullptr;
  p.desc = reinterpret_cast<const MhtBlockDesc*>(base + FD.desc_all_off);
  p.targets = reinterpret_cast<const int*>(base + FD.targets_off);
  p.items = reinterpret_cast<const MhtPItem*>(base + FD.items_off);
  p.nitems = int(FD.nitems);
  p.vec_off = reinterpret_cast<const long long*>(base + c.P.vecoff_off);
  p.cin = DIR == 0 ? static_cast<const R*>(in) : nullptr;
  p.cout = DIR == 1 ? static_cast<R*>(out) : nullptr;
  p.fin = DIR == 1 ? static_cast<const R*>(in) : nullptr;
  p.fout = DIR == 0 ? static_cast<R*>(out) : nullptr;
  p.ldc = DIR == 0 ? ld_in : ld_out;
  p.ldf = DIR == 0 ? ld_out : ld_in;
  p.Y = static_cast<R*>(lvl(c, 0, 0));
  p.A0 = static_cast<R*>(lvl(c, 1, 0));
  p.A1 = static_cast<R*>(lvl(c, 2, 0));
  p.done = cnt;
  p.queue = cnt + ncnt - 1;
  p.status = status_ptr(c);
  p.L = c.P.L;
  p.nb = int(c.P.nb);
  p.nrhs = int(c.nrhs);
  p.slot_bytes = int(FD.slot_bytes);
  p.ldx = int(std::max<int64_t>(FD.max_ld, 1));
  p.mrows = int(std::max<int64_t>(FD.max_item_rows, 1));
  const int grid = int(std::min<int64_t>(num_sms(), FD.nitems));
  StageTimer timer(c.d.prof, DIR, c.P.L + 2, c.s);
  kern<<<grid, kFusedThreads, smem, c.s>>>(p);
  return check(cudaGetLastError(), c.err, "fused apply launch");
}

// Smallest RHS tile (1, 2, 4, 8) that covers nrhs in one fused launch, or 0 if none fits.
int fused_rt(const Ctx& c, int dir) {
  if (c.d.path == 1 || c.nrhs > 8) return 0;
  for (int rt = 1; rt <= 8; rt *= 2)
    if (rt >= c.nrhs) return fused_smem(c.P, dir, rt) <= 227 * 1024 ? rt : 0;
  return 0;
}

template <class R, bool C, int DIR>
int fused_dispatch(const Ctx& c, int rt, const void* in, long long ld_in, void* out, long long ld_out, bool wt) {
  switch (rt) {
    case 1: return fused_launch<R, C, 1, DIR>(c, in, ld_in, out, ld_out, wt);
    case 2: return fused_launch<R, C, 2, DIR>(c, in, ld_in, out, ld_out, wt);
    case 4: return fused_launch<R, C, 4, DIR>(c, in, ld_in, out, ld_out, wt);
    default: return fused_launch<R, C, 8, DIR>(c, in, ld_in, out, ld_out, wt);
  }
}

// Largest RHS tile (8, 4, 2, 1), at most nrhs, whose shared memory fits every stage.
int pick_rt(const Ctx& c, int dir) {
  for (int rt = 8; rt >= 1; rt /= 2) {
    if (rt > 1 && c.nrhs < rt) continue;
    bool ok = true;
    for (const Stage& s : c.P.st) ok = ok && stage_smem(c.P, s, dir, rt) <= 227 * 1024;
    if (ok) return rt;
  }
  return 1;
}

template <class R, bool C>
int synth_dispatch(const Ctx& c, const void* cin, int64_t ldc, void* f, int64_t ldf, bool wt) {
  if (const int rt = fused_rt(c, 0)) {
    const int rc = fused_dispatch<R, C, 0>(c, rt, cin, ldc, f, ldf, wt);
    if (rc >= 0) return rc;
  }
  if (c.d.path == 2) {
    c.err = "the fused apply does not fit this plan / RHS count";
    return MHT_ERR_UNSUPPORTED;
  }
  switch (pick_rt(c, 0)) {
    case 8: return synth_impl<R, C, 8>(c, cin, ldc, f, ldf, wt);
    case 4: return synth_impl<R, C, 4>(c, cin, ldc, f, ldf, wt);
    case 2: return synth_impl<R, C, 2>(c, cin, ldc, f, ldf, wt);
    default: return synth_impl<R, C, 1>(c, cin, ldc, f, ldf, wt);
  }
}
template <class R, bool C>
int adjoint_dispatch(const Ctx& c, const void* f, int64_t ldf, void* cout, int64_t ldc, bool wt) {
  if (const int rt = fused_rt(c, 1)) {
    const int rc = fused_dispatch<R, C, 1>(c, rt, f, ldf, cout, ldc, wt);
    if (rc >= 0) return rc;
  }
  if (c.d.path == 2) {
    c.err = "the fused apply does not fit this plan / RHS count";
    return MHT_ERR_UNSUPPORTED;
  }
  switch (pick_rt(c, 1)) {
    case 8: return adjoint_impl<R, C, 8>(c, f, ldf, cout, ldc, wt);
    case 4: return adjoint_impl<R, C, 4>(c, f, ldf, cout, ldc, wt);
    case 2: return adjoint_impl<R, C, 2>(c, f, ldf, cout, ldc, wt);
    default: return adjoint_impl<R, C, 1>(c, f, ldf, cout, ldc, wt);
  }
}

}  // namespace

int apply_synthesize(const Factorization& F, const Packed& P, const DeviceView& d, const void* c, int64_t ldc,
                     void* f, int64_t ldf, int64_t nrhs, bool wt, mht_apply_mode mode, void* stream,
                     std::string& err) {
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err};
  (void)mode;
  if (P.fp64)
    return P.cplx ? synth_dispatch<double, true>(x, c, ldc, f, ldf, wt)
                  : synth_dispatch<double, false>(x, c, ldc, f, ldf, wt);
  return P.cplx ? synth_dispatch<float, true>(x, c, ldc, f, ldf, wt) : synth_dispatch<float, false>(x, c, ldc, f, ldf, wt);
}

int apply_analyze(const Factorization& F, const Packed& P, const DeviceView& d, const void* f, int64_t ldf, void* c,
                  int64_t ldc, int64_t nrhs, bool weighted, mht_apply_mode mode, void* stream, std::string& err) {
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err};
  (void)mode;
  if (P.fp64)
    return P.cplx ? adjoint_dispatch<double, true>(x, f, ldf, c, ldc, weighted)
                  : adjoint_dispatch<double, false>(x, f, ldf, c, ldc, weighted);
  return P.cplx ? adjoint_dispatch<float, true>(x, f, ldf, c, ldc, weighted)
                : adjoint_dispatch<float, false>(x, f, ldf, c, ldc, weighted);
}

int64_t apply_launches(const Packed& P, int64_t nrhs, mht_apply_mode mode, int path) {
  (void)mode;
  if (path != 1 && nrhs <= 8) {
    int rt = 1;
    while (rt < nrhs) rt *= 2;
    if (fused_smem(P, 0, rt) <= 227 * 1024) return P.fused[0].nitems > 0 ? 1 : 0;
  }
  int64_t n = 0;
  for (const Stage& s : P.st) n += (s.dir[0].nitems > 0) ? 1 : 0;
  return n;
}

int device_upload(void* dst, const void* src, size_t bytes, void* stream, std::string& err) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), err, "factor upload")) return rc;
  return check(cudaStreamSynchronize(s), err, "factor upload sync");
}

int device_copy_async(void* dst, const void* src, size_t bytes, int kind, void* stream, std::string& err) {
  return check(cudaMemcpyAsync(dst, src, bytes, kind == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                               static_cast<cudaStream_t>(stream)),
               err, "host transfer");
}

int device_sync(void* stream, std::string& err) {
  return check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), err, "stream sync");
}

int device_status(void* status_dev, void* stream, unsigned* flags, std::string& err) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = check(cudaMemcpyAsync(flags, status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s), err,
                     "status read"))
    return rc;
  if (int rc = check(cudaMemsetAsync(status_dev, 0, sizeof(unsigned), s), err, "status clear")) return rc;
  return check(cudaStreamSynchronize(s), err, "status sync");
}

}  // namespace mht

// ---------------------------------------------------------------------------------------
// Synthesis for callers that cannot allocate device memory (mht_synthesize_noalloc).
//
// The fused synthesis kernel needs scratch beyond its inputs and outputs: the per-level
// butterfly vectors, one completion counter per block, the work-queue head and the status
// word.  Here that scratch is a fixed array in this library's device image, so the caller
// only passes the packed factors, c and f.  The array is reserved on every GPU that loads
// the library until the process exits.  Host code must not pass the array's name to a
// kernel (in host code it is a host-side stand-in); its device address is looked up once per
// device with cudaGetSymbolAddress while that device is current.
#include <mutex>

namespace mht {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // MHT_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[256] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

int apply_synthesize_noalloc(const Packed& P, const void* factor_dev, const void* c, void* f, void* stream,
                             std::string& err) {
  if (P.fp64 || P.cplx) {
    err = "the no-alloc synthesis serves real FP32 plans";
    return MHT_ERR_UNSUPPORTED;
  }
  const size_t ncnt = size_t(P.L + 2) * P.nb + 1;
  const size_t y_bytes = align256(size_t(std::max<int64_t>(P.vec_entries, 1)) * sizeof(float));
  const size_t cnt_bytes = align256(ncnt * sizeof(unsigned));
  const size_t need = y_bytes + cnt_bytes + 256;
  if (need > kNoAllocScratchBytes) {
    err = "this plan needs " + std::to_string(need) + " bytes of scratch; the no-alloc entry point has " +
          std::to_string(kNoAllocScratchBytes);
    return MHT_ERR_UNSUPPORTED;
  }
  const size_t smem = fused_smem(P, 0, 1);
  if (smem > 227 * 1024) {
    err = "the fused synthesis does not fit in shared memory for this plan";
    return MHT_ERR_UNSUPPORTED;
  }
  int dev = 0;
  if (int rc = check(cudaGetDevice(&dev), err, "cudaGetDevice")) return rc;
  if (dev < 0 || dev >= 256) {
    err = "device ordinal out of range";
    return MHT_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {  // set-up: once per device, with that device current
      void* a = nullptr;
      if (int rc = check(cudaGetSymbolAddress(&a, g_noalloc_scratch), err, "cudaGetSymbolAddress")) return rc;
      g_noalloc_addr[dev] = a;
    }
    base = g_noalloc_addr[dev];
  }
  auto* scratch = static_cast<uint8_t*>(base);
  unsigned* cnt = reinterpret_cast<unsigned*>(scratch + y_bytes);
  unsigned* status = reinterpret_cast<unsigned*>(scratch + y_bytes + cnt_bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: counters, queue head and status start at zero
  if (int rc = check(cudaMemsetAsync(cnt, 0, cnt_bytes + 256, s), err, "scratch reset")) return rc;
  const FusedDir& FD = P.fused[0];
  if (FD.nitems == 0) return 0;
  auto kern = k_fused<float, false, 1, 0>;
  if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), err,
                     "shared memory attribute"))
    return rc;
  const uint8_t* img = static_cast<const uint8_t*>(factor_dev);
  FusedParams<float> p{};
  p.data = reinterpret_cast<const float*>(img + P.data_off);
  p.idx = reinterpret_cast<const int*>(img + P.index_off);
  p.perm = reinterpret_cast<const int*>(img + P.perm_off);
  p.wts = nullptr;
  p.desc = reinterpret_cast<const MhtBlockDesc*>(img + FD.desc_all_off);
  p.targets = reinterpret_cast<const int*>(img + FD.targets_off);
  p.items = reinterpret_cast<const MhtPItem*>(img + FD.items_off);
  p.nitems = int(FD.nitems);
  p.vec_off = reinterpret_cast<const long long*>(img + P.vecoff_off);
  p.cin = static_cast<const float*>(c);
  p.cout = nullptr;
  p.fin = nullptr;
  p.fout = static_cast<float*>(f);
  p.ldc = 1;  // single right-hand side: leading dimensions are irrelevant
  p.ldf = 1;
  p.Y = reinterpret_cast<float*>(scratch);
  p.A0 = nullptr;
  p.A1 = nullptr;
  p.done = cnt;
  p.queue = cnt + ncnt - 1;
  p.status = status;
  p.L = P.L;
  p.nb = int(P.nb);
  p.nrhs = 1;
  p.slot_bytes = int(FD.slot_bytes);
  p.ldx = int(std::max<int64_t>(FD.max_ld, 1));
  p.mrows = int(std::max<int64_t>(FD.max_item_rows, 1));
  const int grid = int(std::min<int64_t>(num_sms(), FD.nitems));
  kern<<<grid, kFusedThreads, smem, s>>>(p);
  return check(cudaGetLastError(), err, "no-alloc synthesis launch");
}

}  // namespace mht
