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
//   * k_rowdot: one persistent launch per stage; each CTA takes work items (block, row range
//     of up to 512 KB, less in small stages) in a fixed stride, and thread 0 keeps a ring of
//     shared-memory slots (size and depth autotuned) filled by 1-D TMA bulk copies
//     (cp.async.bulk, completion on mbarriers) across item boundaries, while all threads
//     gather the block's input vector from L2;
//   * each warp then reduces whole rows from shared memory with 128-bit loads, compensated
//     FP32 sums and warp shuffles (building blocks in rowdot.cuh);
//   * k_fused: one persistent launch for all stages with per-block completion counters
//     (selected explicitly; also the engine of the allocation-free synthesis);
//   * this file also holds the per-stage dispatch, the autotuner and the spectral filter graph.
// The adjoint is a gather: the sibling blocks (2p, nu), (2p+1, nu) that share an input pair
// write separate buffers and the next stage sums them while loading -- no atomics, so the
// result is deterministic.  Every mbarrier wait is bounded; on timeout the kernel sets a bit
// in the workspace status word (read by mht_plan_check) instead of hanging.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../host/internal.h"
#include "rowdot.cuh"

namespace mht {
namespace {

// One launch per stage and direction, persistent: CTA b computes items b, b + gridDim.x, ...
template <class R, bool C, int RT, int MODE>
__global__ void __launch_bounds__(kThreads)
k_rowdot(RowArgs<R> a, const MhtItem* __restrict__ items, int nitems, int slot_bytes, int nslot, int ldx_max,
         int rows_max, unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RowSmem sm = row_smem<R, C>(smem_raw, slot_bytes, nslot, ldx_max, rows_max);
  RowProducer<R, C> prod{items, a.desc, a.data, nitems, int(gridDim.x), (a.nrhs + RT - 1) / RT, int(blockIdx.x)};
  if (threadIdx.x == 0) {
    for (int i = 0; i < nslot; ++i) mbar_init(&sm.bar[i], 1);
    *sm.flag = 1;
    prod.load(slot_bytes);
    while (prod.issued < unsigned(nslot) && prod.issue(sm)) {
    }
  }
  __syncthreads();
  unsigned cons = 0;
  bool ok = true;
  for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
    const MhtItem it = items[item];
    const MhtBlockDesc d = a.desc[it.blk];
    ok = row_item<R, C, RT, MODE>(a, it, d, sm, cons, status, [&] { prod.issue(sm); });
  }
  if (threadIdx.x == 0 && !ok) row_drain(sm, cons, prod.issued);
}

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
  int first_stage;            // the launch's first stage: its inputs are complete, no waits
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
        if (st == p.first_stage) {
          // a launch over a range of stages: the earlier stages completed in earlier launches
        } else if (DIR == 0 && st >= 1 && st <= L) {
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
      row_dot<R, C, RT>(tile + (long long)ii * d.ldt * W, xb, p.ldx, nvec, lane, acc);
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

// Around every kernel launch of an apply: an NVTX range named for the direction and stage (so
// that a profiler's timeline shows which stage a launch belongs to; without an attached tool
// the range costs a few nanoseconds), and, while stage timing is enabled, CUDA events.
struct StageTimer {
  Profiler* p;
  int dir, stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(Profiler* p_, int d, int st, cudaStream_t s_) : p(p_), dir(d), stage(st), s(s_) {
    char name[64];
    std::snprintf(name, sizeof(name), "mht %s stage %d", d == 0 ? "synthesis" : "analysis", st);
    nvtxRangePushA(name);
    if (p) {
      a = p->get();
      cudaEventRecord(a, s);
    }
  }
  ~StageTimer() {
    nvtxRangePop();
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
  mht_apply_mode mode = MHT_APPLY_FP32;
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

int num_sms();

// Ring slot of the per-stage kernel: slot_kb KB (default 32), or one padded row if wider.
size_t stage_slot_bytes(const Packed& P, const Stage& S, int dir, int slot_kb = 0) {
  const size_t row = size_t(std::max<int64_t>(S.dir[dir].max_ld, 1)) * P.elem_bytes;
  return std::max<size_t>(size_t(slot_kb > 0 ? slot_kb : 32) * 1024, (row + 127) / 128 * 128);
}

size_t stage_smem(const Packed& P, const Stage& S, int dir, int rt, int nslot, int slot_kb = 0) {
  const size_t rows = size_t(std::max<int64_t>(S.dir[dir].max_item_rows, 1));
  return 128 + nslot * stage_slot_bytes(P, S, dir, slot_kb) +
         size_t(std::max<int64_t>(S.dir[dir].max_ld, 1)) * rt * P.elem_bytes + rows * rt * P.elem_bytes +
         rows * sizeof(int);
}

// Default ring: kRowSlots slots (fewer if shared memory is short); 0 if none fits.
int stage_nslot(const Packed& P, const Stage& S, int dir, int rt, int slot_kb = 0, int max_slots = kRowSlots) {
  for (int ns = max_slots; ns >= 1; --ns)
    if (stage_smem(P, S, dir, rt, ns, slot_kb) <= 227 * 1024) return ns;
  return 0;
}

template <class R, bool C, int RT, int MODE>
int launch(const Ctx& c, int s, const void* in0, const void* in1, long long is_e, long long is_k, void* out0,
           void* out1, long long os_e, long long os_k, const void* w, const StageCfg& cfg) {
  const int dir = (MODE == ADJ_ID || MODE == ADJ_U) ? 1 : 0;
  const Stage& S = c.P.st[s];
  const StageDir& D = S.dir[dir];
  if (D.nitems == 0) return 0;
  const int nslot = stage_nslot(c.P, S, dir, RT, cfg.slot_kb, cfg.nslot > 0 ? cfg.nslot : kRowSlots);
  if (nslot == 0) {
    c.err = "a stage needs more shared memory than an SM has for this RHS tile";
    return MHT_ERR_UNSUPPORTED;
  }
  const size_t smem = stage_smem(c.P, S, dir, RT, nslot, cfg.slot_kb);
  auto kern = k_rowdot<R, C, RT, MODE>;
  if (smem > 48 * 1024)
    if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), c.err,
                       "shared memory attribute"))
      return rc;
  const uint8_t* base = c.d.base;
  RowArgs<R> a{reinterpret_cast<const R*>(base + c.P.data_off), reinterpret_cast<const int*>(base + c.P.index_off),
               reinterpret_cast<const MhtBlockDesc*>(base + D.desc_off), reinterpret_cast<const int*>(base + c.P.perm_off),
               static_cast<const R*>(w), static_cast<const R*>(in0), static_cast<const R*>(in1), is_e, is_k,
               static_cast<R*>(out0), static_cast<R*>(out1), os_e, os_k, int(c.nrhs)};
  int per_sm = 0;
  if (int rc = check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem), c.err, "occupancy"))
    return rc;
  per_sm = std::max(per_sm, 1);
  if (cfg.per_sm > 0) per_sm = std::min(per_sm, cfg.per_sm);
  const int64_t grid = std::min<int64_t>(D.nitems, int64_t(per_sm) * num_sms());
  StageTimer timer(c.d.prof, dir, s, c.s);
  kern<<<unsigned(grid), kThreads, smem, c.s>>>(a, reinterpret_cast<const MhtItem*>(base + D.items_off), int(D.nitems),
                                               int(stage_slot_bytes(c.P, S, dir, cfg.slot_kb)), nslot,
                                               int(std::max<int64_t>(D.max_ld, 1)),
                                               int(std::max<int64_t>(D.max_item_rows, 1)), status_ptr(c));
  return check(cudaGetLastError(), c.err, "apply launch");
}

template <class R, bool C, int RT>
int launch_mode(const Ctx& c, int s, int mode, const void* in0, const void* in1, long long is_e, long long is_k,
                void* out0, void* out1, long long os_e, long long os_k, const void* w, const StageCfg& cfg) {
  switch (mode) {
    case SYN_ID: return launch<R, C, RT, SYN_ID>(c, s, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
    case ADJ_ID: return launch<R, C, RT, ADJ_ID>(c, s, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
    case SYN_U: return launch<R, C, RT, SYN_U>(c, s, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
    default: return launch<R, C, RT, ADJ_U>(c, s, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
  }
}

int tc_launch(const Ctx& c, int s, int dir, int mode, const void* in0, const void* in1, long long is_e,
              long long is_k, void* out0, void* out1, long long os_e, long long os_k, const void* w);

// One stage with the given configuration: the SIMT kernel with RHS tile cfg.rt, or (FP32
// plans) the tensor-core kernel.
template <class R, bool C>
int run_stage(const Ctx& c, int s, int mode, const void* in0, const void* in1, long long is_e, long long is_k,
              void* out0, void* out1, long long os_e, long long os_k, const void* w, const StageCfg& cfg) {
  if constexpr (sizeof(R) == 4) {
    if (cfg.tensor) {
      const int dir = (mode == ADJ_ID || mode == ADJ_U) ? 1 : 0;
      return tc_launch(c, s, dir, mode, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w);
    }
  }
  switch (cfg.rt) {
    case 8: return launch_mode<R, C, 8>(c, s, mode, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
    case 4: return launch_mode<R, C, 4>(c, s, mode, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
    case 2: return launch_mode<R, C, 2>(c, s, mode, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
    default: return launch_mode<R, C, 1>(c, s, mode, in0, in1, is_e, is_k, out0, out1, os_e, os_k, w, cfg);
  }
}

// The stages of one direction in apply order: synthesis V, R (l = 1..L), U; the adjoint U^H,
// R^H (l = L..1), V^H.  cfg(dir, s) gives each stage's configuration.
template <class R, bool C, class Cfg>
int synth_stages(const Ctx& c, const void* cin, int64_t ldc, void* f, int64_t ldf, bool weighted, Cfg&& cfg,
                 const void* scale = nullptr, int s_lo = 0, int s_hi = -1) {
  const int L = c.F.L;
  if (s_hi < 0) s_hi = L + 2;
  const long long nr = c.nrhs;
  int rc = 0;
  if (s_lo == 0 && s_hi > 0)
    rc = run_stage<R, C>(c, 0, SYN_ID, cin, nullptr, 1, ldc, lvl(c, 0, 0), nullptr, nr, 1, scale, cfg(0, 0));
  for (int l = std::max(1, s_lo); l <= L && l < s_hi && !rc; ++l)
    rc = run_stage<R, C>(c, l, SYN_ID, lvl(c, 0, l - 1), nullptr, nr, 1, lvl(c, 0, l), nullptr, nr, 1, nullptr,
                         cfg(0, l));
  if (rc || s_hi <= L + 1) return rc;
  const void* w = weighted ? (const void*)(c.d.base + c.P.weights_off) : nullptr;
  return run_stage<R, C>(c, L + 1, SYN_U, lvl(c, 0, L), nullptr, nr, 1, f, nullptr, 1, ldf, w, cfg(0, L + 1));
}

// The adjoint's stages k_lo .. k_hi - 1 in dependency order (stage L + 1 - k).
template <class R, bool C, class Cfg>
int adjoint_stages(const Ctx& c, const void* f, int64_t ldf, void* cout, int64_t ldc, bool weighted, Cfg&& cfg,
                   int k_lo = 0, int k_hi = -1) {
  const int L = c.F.L;
  if (k_hi < 0) k_hi = L + 2;
  const long long nr = c.nrhs;
  const void* w = weighted ? (const void*)(c.d.base + c.P.weights_off) : nullptr;
  int rc = 0;
  // U^H: f -> z_L (region A0, level L)
  if (k_lo == 0 && k_hi > 0)
    rc = run_stage<R, C>(c, L + 1, ADJ_U, f, nullptr, 1, ldf, lvl(c, 1, L), nullptr, nr, 1, w, cfg(1, L + 1));
  for (int l = L; l >= 1 && !rc; --l) {
    const int k = L + 1 - l;
    if (k < k_lo || k >= k_hi) continue;
    rc = run_stage<R, C>(c, l, ADJ_ID, lvl(c, 1, l), l == L ? nullptr : lvl(c, 2, l), nr, 1, lvl(c, 1, l - 1),
                         lvl(c, 2, l - 1), nr, 1, nullptr, cfg(1, l));
  }
  if (rc || k_hi <= L + 1) return rc;
  return run_stage<R, C>(c, 0, ADJ_ID, lvl(c, 1, 0), L == 0 ? nullptr : lvl(c, 2, 0), nr, 1, cout, cout, 1, ldc,
                         nullptr, cfg(1, 0));
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
int fused_launch(const Ctx& c, const void* in, long long ld_in, void* out, long long ld_out, bool weighted,
                 int k_lo = 0, int k_hi = -1) {
  const FusedDir& FD = c.P.fused[DIR];
  const int nst = c.P.L + 2;
  if (k_hi < 0) k_hi = nst;
  const int64_t it0 = FD.stage_first[k_lo], nit = FD.stage_first[k_hi] - it0;
  const size_t smem = fused_smem(c.P, DIR, RT);
  if (smem > 227 * 1024) return -1;
  auto kern = k_fused<R, C, RT, DIR>;
  if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), c.err,
                     "shared memory attribute"))
    return rc;
  const size_t ncnt = size_t(c.P.L + 2) * c.P.nb + 1;
  unsigned* cnt = counters(c, DIR);
  if (int rc = check(cudaMemsetAsync(cnt, 0, ncnt * sizeof(unsigned), c.s), c.err, "counter reset")) return rc;
  if (nit == 0) return 0;
  const uint8_t* base = c.d.base;
  FusedParams<R> p;
  p.data = reinterpret_cast<const R*>(base + c.P.data_off);
  p.idx = reinterpret_cast<const int*>(base + c.P.index_off);
  p.perm = reinterpret_cast<const int*>(base + c.P.perm_off);
  p.wts = weighted ? reinterpret_cast<const R*>(base + c.P.weights_off) : nullptr;
  p.desc = reinterpret_cast<const MhtBlockDesc*>(base + FD.desc_all_off);
  p.targets = reinterpret_cast<const int*>(base + FD.targets_off);
  p.items = reinterpret_cast<const MhtPItem*>(base + FD.items_off) + it0;
  p.nitems = int(nit);
  p.first_stage = DIR == 0 ? k_lo : nst - 1 - k_lo;
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
  const int grid = int(std::min<int64_t>(num_sms(), nit));
  StageTimer timer(c.d.prof, DIR, c.P.L + 2, c.s);
  kern<<<grid, kFusedThreads, smem, c.s>>>(p);
  return check(cudaGetLastError(), c.err, "fused apply launch");
}

// Smallest RHS tile (1, 2, 4, 8) that covers nrhs in one fused launch, or 0 if none fits.
int fused_rt_fit(const Ctx& c, int dir) {
  if (c.nrhs > 8) return 0;
  for (int rt = 1; rt <= 8; rt *= 2)
    if (rt >= c.nrhs) return fused_smem(c.P, dir, rt) <= 227 * 1024 ? rt : 0;
  return 0;
}
int fused_rt(const Ctx& c, int dir) { return c.d.path == 2 ? fused_rt_fit(c, dir) : 0; }

// One persistent launch for the stages k_lo .. k_hi - 1 (dependency order) of a direction.
template <class R, bool C, int DIR>
int fused_dispatch(const Ctx& c, int rt, const void* in, long long ld_in, void* out, long long ld_out, bool wt,
                   int k_lo = 0, int k_hi = -1) {
  switch (rt) {
    case 1: return fused_launch<R, C, 1, DIR>(c, in, ld_in, out, ld_out, wt, k_lo, k_hi);
    case 2: return fused_launch<R, C, 2, DIR>(c, in, ld_in, out, ld_out, wt, k_lo, k_hi);
    case 4: return fused_launch<R, C, 4, DIR>(c, in, ld_in, out, ld_out, wt, k_lo, k_hi);
    default: return fused_launch<R, C, 8, DIR>(c, in, ld_in, out, ld_out, wt, k_lo, k_hi);
  }
}

// ---- tensor-core stages (3xTF32, FP32 plans, at least 16 real or 8 complex RHS) ----------
bool use_tc(const Ctx& c) { return tensor_mode(c.mode) && !c.P.fp64 && c.nrhs >= (c.P.cplx ? 8 : 16); }

int tc_launch(const Ctx& c, int s, int dir, int mode, const void* in0, const void* in1, long long is_e,
              long long is_k, void* out0, void* out1, long long os_e, long long os_k, const void* w) {
  const StageDir& D = c.P.st[s].dir[dir];
  TcLaunch a;
  a.data = reinterpret_cast<const float*>(c.d.base + c.P.data_off);
  a.idx = reinterpret_cast<const int*>(c.d.base + c.P.index_off);
  a.desc = reinterpret_cast<const MhtBlockDesc*>(c.d.base + D.desc_off);
  a.items = reinterpret_cast<const MhtItem*>(c.d.base + D.tc_items_off);
  a.nitems = D.tc_nitems;
  a.perm = reinterpret_cast<const int*>(c.d.base + c.P.perm_off);
  a.wts = static_cast<const float*>(w);
  a.in0 = static_cast<const float*>(in0);
  a.in1 = static_cast<const float*>(in1);
  a.is_e = is_e;
  a.is_k = is_k;
  a.out0 = static_cast<float*>(out0);
  a.out1 = static_cast<float*>(out1);
  a.os_e = os_e;
  a.os_k = os_k;
  a.nrhs = c.nrhs;
  a.mode = mode;
  a.cplx = c.P.cplx ? 1 : 0;
  a.bf16 = c.mode == MHT_APPLY_6XBF16 ? 1 : 0;
  a.tmaps = c.d.base + c.P.tmap_off + size_t(dir * (c.P.L + 2) + s) * c.P.nb * 128;
  a.status = status_ptr(c);
  a.stream = c.s;
  StageTimer timer(c.d.prof, dir, s, c.s);
  return tc_stage_launch(a, c.err);
}

// Largest RHS tile (8, 4, 2, 1), at most nrhs, whose shared memory fits every stage.
int pick_rt(const Ctx& c, int dir) {
  for (int rt = 8; rt >= 1; rt /= 2) {
    if (rt > 1 && c.nrhs < rt) continue;
    bool ok = true;
    for (const Stage& s : c.P.st) ok = ok && stage_nslot(c.P, s, dir, rt) > 0;
    if (ok) return rt;
  }
  return 1;
}

// Configuration of stage s in direction dir for this apply: the autotuned one when the plan
// was tuned for this RHS count, else the defaults (tensor cores in 3xTF32 mode from 16 real /
// 8 complex RHS, else the widest RHS tile that fits, all ring slots, all resident CTAs).
StageCfg stage_cfg(const Ctx& c, int dir, int s, int default_rt) {
  if (c.d.tune_nrhs == c.nrhs && size_t(s) < c.d.tune[dir].size() &&
      (c.d.tune_mode == c.mode || !c.d.tune[dir][s].tensor))
    return c.d.tune[dir][s];
  StageCfg g;
  g.tensor = use_tc(c) ? 1 : 0;
  g.rt = default_rt;
  return g;
}

// A direction with its first h and last t stages (dependency order) each in one persistent launch
// with per-block dependency counters, the stages between them one launch each (h = t = 0: every
// stage its own launch).  The small stages at both ends then overlap instead of each paying a
// launch, a ramp and a tail.  Returns -1 when the persistent kernel does not fit.
template <class R, bool C, int DIR>
int run_direction(const Ctx& c, const void* in, int64_t ld_in, void* out, int64_t ld_out, bool wt, int h, int t) {
  const int nst = c.P.L + 2;
  const int rt = pick_rt(c, DIR);
  auto cfg = [&](int dir, int s) { return stage_cfg(c, dir, s, rt); };
  const int frt = (h > 0 || t > 0) ? fused_rt_fit(c, DIR) : 0;
  if ((h > 0 || t > 0) && !frt) return -1;
  int rc = h > 0 ? fused_dispatch<R, C, DIR>(c, frt, in, ld_in, out, ld_out, wt, 0, h) : 0;
  if (rc) return rc;
  if (h + t < nst)
    rc = DIR == 0 ? synth_stages<R, C>(c, in, ld_in, out, ld_out, wt, cfg, nullptr, h, nst - t)
                  : adjoint_stages<R, C>(c, in, ld_in, out, ld_out, wt, cfg, h, nst - t);
  if (rc) return rc;
  return t > 0 ? fused_dispatch<R, C, DIR>(c, frt, in, ld_in, out, ld_out, wt, std::max(h, nst - t), nst) : 0;
}

// The stage grouping tuned for this RHS count (both ends, per direction), if any.
bool tuned_grouping(const Ctx& c, int dir, int& h, int& t) {
  h = t = 0;
  if (c.d.tune_nrhs != c.nrhs || c.d.tune_mode != c.mode || use_tc(c) || c.d.path != 0) return false;
  h = c.d.fuse_head[dir];
  t = c.d.fuse_tail[dir];
  return h > 0 || t > 0;
}

template <class R, bool C>
int synth_dispatch(const Ctx& c, const void* cin, int64_t ldc, void* f, int64_t ldf, bool wt,
                   const void* scale = nullptr) {
  if (scale) {  // the fused kernel has no input scale: per-stage launches
    const int rt = pick_rt(c, 0);
    return synth_stages<R, C>(c, cin, ldc, f, ldf, wt, [&](int dir, int s) { return stage_cfg(c, dir, s, rt); },
                              scale);
  }
  if (!use_tc(c))
    if (const int rt = fused_rt(c, 0)) {  // only when the persistent path is selected
      const int rc = fused_dispatch<R, C, 0>(c, rt, cin, ldc, f, ldf, wt);
      if (rc >= 0) return rc;
    }
  if (c.d.path == 2) {
    c.err = "the fused apply does not fit this plan / RHS count";
    return MHT_ERR_UNSUPPORTED;
  }
  int h, t;
  if (tuned_grouping(c, 0, h, t)) {
    const int rc = run_direction<R, C, 0>(c, cin, ldc, f, ldf, wt, h, t);
    if (rc >= 0) return rc;
  }
  const int rt = pick_rt(c, 0);
  return synth_stages<R, C>(c, cin, ldc, f, ldf, wt, [&](int dir, int s) { return stage_cfg(c, dir, s, rt); });
}
template <class R, bool C>
int adjoint_dispatch(const Ctx& c, const void* f, int64_t ldf, void* cout, int64_t ldc, bool wt) {
  if (!use_tc(c))
    if (const int rt = fused_rt(c, 1)) {  // only when the persistent path is selected
      const int rc = fused_dispatch<R, C, 1>(c, rt, f, ldf, cout, ldc, wt);
      if (rc >= 0) return rc;
    }
  if (c.d.path == 2) {
    c.err = "the fused apply does not fit this plan / RHS count";
    return MHT_ERR_UNSUPPORTED;
  }
  int h, t;
  if (tuned_grouping(c, 1, h, t)) {
    const int rc = run_direction<R, C, 1>(c, f, ldf, cout, ldc, wt, h, t);
    if (rc >= 0) return rc;
  }
  const int rt = pick_rt(c, 1);
  return adjoint_stages<R, C>(c, f, ldf, cout, ldc, wt, [&](int dir, int s) { return stage_cfg(c, dir, s, rt); });
}

// ---- autotuner ---------------------------------------------------------------------------
// Times every candidate configuration of every stage (RHS tile, ring slots, resident CTAs per
// SM, tensor cores or not) on the bound workspace and keeps the fastest.  Each stage runs on
// its own (zeroed) buffers: stage 0 reads the host-staging area for c, the last stage writes
// the one for f, so nothing of the caller's is touched.
template <class R, bool C>
int autotune(Ctx& c, DeviceView& dv, std::vector<TuneRecord>* report) {
  const Packed& P = c.P;
  const int L = c.F.L;
  const int64_t nr = c.nrhs;
  // host-staging areas of the workspace: c (m x max_nrhs) then f (n x max_nrhs)
  uint8_t* cbuf = dv.ws + 3 * P.ws_vec_bytes(dv.max_nrhs);
  uint8_t* fbuf = dv.ws + P.ws_counters_offset(dv.max_nrhs, c.F.n, c.F.m) -
                  (size_t(c.F.n) * dv.max_nrhs * P.elem_bytes + 255) / 256 * 256;
  if (int rc = check(cudaMemsetAsync(dv.ws, 0, P.ws_counters_offset(dv.max_nrhs, c.F.n, c.F.m), c.s), c.err, "tune zero"))
    return rc;
  std::vector<StageCfg> cands;
  const bool tc_ok = sizeof(R) == 4 && tensor_mode(c.mode);
  // single RHS (bandwidth-bound): the ring's slot size and depth and the resident CTAs;
  // several RHS (issue-bound): the RHS tile, a few ring depths and CTA counts
  auto add = [&](int rt, int kb, int ns, int ps) {
    StageCfg g;
    g.rt = rt;
    g.slot_kb = kb;
    g.nslot = ns;
    g.per_sm = ps;
    cands.push_back(g);
  };
  if (nr == 1) {
    for (int kb : {16, 32, 64})
      for (int ns = 1; ns <= kMaxRowSlots && ns * kb <= 192; ++ns)
        for (int ps = 1; ps <= 4; ++ps) add(1, kb, ns, ps);
  } else {
    for (int rt : {2, 4, 8})
      if (rt <= nr && (rt == 8 || 2 * rt > nr))  // the widest tile that fits, and 8
        for (int ns = 1; ns <= kRowSlots; ++ns)
          for (int ps = 1; ps <= 2; ++ps) add(rt, 32, ns, ps);
  }
  if (tc_ok) {
    StageCfg g;
    g.tensor = 1;
    cands.push_back(g);
  }
  cudaEvent_t e0, e1;
  if (int rc = check(cudaEventCreate(&e0), c.err, "event")) return rc;
  if (int rc = check(cudaEventCreate(&e1), c.err, "event")) return rc;
  int rc = 0;
  for (int dir = 0; dir < 2 && !rc; ++dir) {
    dv.tune[dir].assign(L + 2, StageCfg());
    for (int s = 0; s < L + 2 && !rc; ++s) {
      if (P.st[s].dir[dir].nitems == 0) continue;
      float best = 1e30f;
      StageCfg best_cfg;
      for (const StageCfg& g : cands) {
        // skip slot / CTA counts that do not fit: they would repeat a smaller configuration
        if (!g.tensor) {
          const int fit = stage_nslot(P, P.st[s], dir, g.rt, g.slot_kb, kMaxRowSlots);
          if (g.nslot > fit) continue;
          if (stage_slot_bytes(P, P.st[s], dir, g.slot_kb) > size_t(g.slot_kb) * 1024 && g.slot_kb != 64) continue;
          const size_t smem = stage_smem(P, P.st[s], dir, g.rt, g.nslot, g.slot_kb);
          if (g.per_sm > 1 && size_t(g.per_sm) * (smem + 1024) > 228 * 1024) continue;  // cannot be resident
        }
        // the stage's own input and output levels, each in its own region (exact sizes)
        auto one = [&]() -> int {
          if (dir == 0) {
            const void* in0 = s == 0 ? (const void*)cbuf : lvl(c, 0, s - 1);
            void* out0 = s == L + 1 ? (void*)fbuf : lvl(c, 1, s);
            return run_stage<R, C>(c, s, s == L + 1 ? SYN_U : SYN_ID, in0, nullptr, s == 0 ? 1 : nr,
                                   s == 0 ? c.F.m : 1, out0, nullptr, s == L + 1 ? 1 : nr, s == L + 1 ? c.F.n : 1,
                                   nullptr, g);
          }
          if (s == L + 1)
            return run_stage<R, C>(c, s, ADJ_U, fbuf, nullptr, 1, c.F.n, lvl(c, 2, L), nullptr, nr, 1, nullptr, g);
          void* out0 = s == 0 ? (void*)cbuf : lvl(c, 2, s - 1);
          return run_stage<R, C>(c, s, ADJ_ID, lvl(c, 1, s), nullptr, nr, 1, out0, out0, s == 0 ? 1 : nr,
                                 s == 0 ? c.F.m : 1, nullptr, g);
        };
        if ((rc = one())) {  // a configuration that cannot launch is skipped
          rc = 0;
          cudaGetLastError();
          continue;
        }
        float ms = 0.f;
        constexpr int kReps = 3;
        if ((rc = check(cudaEventRecord(e0, c.s), c.err, "event"))) break;
        for (int r = 0; r < kReps && !rc; ++r) rc = one();
        if (rc) break;
        if ((rc = check(cudaEventRecord(e1, c.s), c.err, "event"))) break;
        if ((rc = check(cudaEventSynchronize(e1), c.err, "event sync"))) break;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= kReps;
        if (ms < best) {
          best = ms;
          best_cfg = g;
        }
      }
      dv.tune[dir][s] = best_cfg;
      if (report) report->push_back({dir, s, best_cfg, double(best)});
    }
  }
  if (rc) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dv.tune[0].clear();
    dv.tune[1].clear();
    dv.tune_nrhs = 0;
    return rc;
  }
  dv.tune_nrhs = nr;
  dv.tune_mode = c.mode;
  // stage grouping at both ends of each direction (one persistent launch for the first h and
  // one for the last t stages), timed on whole directions with the tuned per-stage shapes
  dv.fuse_head[0] = dv.fuse_head[1] = dv.fuse_tail[0] = dv.fuse_tail[1] = 0;
  if (!use_tc(c) && c.d.path == 0 && fused_rt_fit(c, 0) && fused_rt_fit(c, 1)) {
    const int nst = L + 2;
    for (int dir = 0; dir < 2 && !rc; ++dir) {
      float best = 1e30f;
      int bh = 0, bt = 0;
      for (int h : {0, 2, 3, 4, 5})
        for (int t : {0, 2, 3, 4}) {
          if (h + t > nst || (h > 0 && h >= nst) || (t > 0 && t >= nst)) continue;
          auto one = [&]() -> int {
            return dir == 0 ? run_direction<R, C, 0>(c, cbuf, c.F.m, fbuf, c.F.n, false, h, t)
                            : run_direction<R, C, 1>(c, fbuf, c.F.n, cbuf, c.F.m, false, h, t);
          };
          if (one() != 0) {  // does not fit or cannot launch: skipped
            cudaGetLastError();
            continue;
          }
          if ((rc = check(cudaEventRecord(e0, c.s), c.err, "event"))) break;
          for (int r = 0; r < 3 && !rc; ++r) rc = one();
          if (!rc) rc = check(cudaEventRecord(e1, c.s), c.err, "event");
          if (!rc) rc = check(cudaEventSynchronize(e1), c.err, "event sync");
          if (rc) break;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if ((h == 0 && t == 0) || ms < best * 0.98f) {  // a grouping must win by 2%
            best = ms;
            bh = h;
            bt = t;
          }
        }
      dv.fuse_head[dir] = bh;
      dv.fuse_tail[dir] = bt;
      if (report) report->push_back({dir, -1, StageCfg{0, bh, bt, 0, 0}, double(best)});
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    dv.tune[0].clear();
    dv.tune[1].clear();
    dv.tune_nrhs = 0;
    dv.fuse_head[0] = dv.fuse_head[1] = dv.fuse_tail[0] = dv.fuse_tail[1] = 0;
    return rc;
  }
  return check(cudaStreamSynchronize(c.s), c.err, "tune sync");
}

}  // namespace

int apply_synthesize(const Factorization& F, const Packed& P, const DeviceView& d, const void* c, int64_t ldc,
                     void* f, int64_t ldf, int64_t nrhs, bool wt, mht_apply_mode mode, void* stream,
                     std::string& err, const void* scale) {
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err, mode};
  if (P.fp64)
    return P.cplx ? synth_dispatch<double, true>(x, c, ldc, f, ldf, wt, scale)
                  : synth_dispatch<double, false>(x, c, ldc, f, ldf, wt, scale);
  return P.cplx ? synth_dispatch<float, true>(x, c, ldc, f, ldf, wt, scale)
                : synth_dispatch<float, false>(x, c, ldc, f, ldf, wt, scale);
}

struct FilterGraph {
  const void *f_in = nullptr, *filter = nullptr;
  void* f_out = nullptr;
  int64_t ldi = 0, ldo = 0, nrhs = 0, tune_nrhs = 0;
  bool weighted = false;
  mht_apply_mode mode = MHT_APPLY_FP32;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec = nullptr;
};

void filter_graph_destroy(FilterGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->capture) cudaStreamDestroy(g->capture);
  delete g;
}

int apply_filter(const Factorization& F, const Packed& P, DeviceView& d, const void* f_in, int64_t ldi, void* f_out,
                 int64_t ldo, int64_t nrhs, const void* filter, bool weighted, mht_apply_mode mode, void* stream,
                 std::string& err) {
  FilterGraph* g = d.filter;
  const bool same = g && g->exec && g->f_in == f_in && g->filter == filter && g->f_out == f_out && g->ldi == ldi &&
                    g->ldo == ldo && g->nrhs == nrhs && g->weighted == weighted && g->mode == mode &&
                    g->tune_nrhs == d.tune_nrhs;
  if (!same) {
    if (!g) g = d.filter = new FilterGraph();
    if (g->exec) {
      cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
    }
    if (!g->capture)
      if (int rc = check(cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking), err, "filter stream")) return rc;
    // coefficients in the host-staging area for c (m x max_nrhs, leading dimension m)
    void* coef = d.ws + 3 * P.ws_vec_bytes(d.max_nrhs);
    if (int rc = check(cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal), err, "filter capture"))
      return rc;
    int rc = apply_analyze(F, P, d, f_in, ldi, coef, F.m, nrhs, weighted, mode, g->capture, err);
    if (!rc) rc = apply_synthesize(F, P, d, coef, F.m, f_out, ldo, nrhs, false, mode, g->capture, err, filter);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->capture, &graph);
    if (!rc && e != cudaSuccess) rc = check(e, err, "filter capture end");
    if (!rc) rc = check(cudaGraphInstantiate(&g->exec, graph, 0), err, "filter graph");
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    g->f_in = f_in;
    g->filter = filter;
    g->f_out = f_out;
    g->ldi = ldi;
    g->ldo = ldo;
    g->nrhs = nrhs;
    g->weighted = weighted;
    g->mode = mode;
    g->tune_nrhs = d.tune_nrhs;
  }
  return check(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), err, "filter launch");
}

int apply_autotune(const Factorization& F, const Packed& P, DeviceView& d, int64_t nrhs, mht_apply_mode mode,
                   void* stream, std::vector<TuneRecord>* report, std::string& err) {
  d.tune_nrhs = 0;  // tune with the default configurations out of the way
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err, mode};
  if (P.fp64) return P.cplx ? autotune<double, true>(x, d, report) : autotune<double, false>(x, d, report);
  return P.cplx ? autotune<float, true>(x, d, report) : autotune<float, false>(x, d, report);
}

int apply_analyze(const Factorization& F, const Packed& P, const DeviceView& d, const void* f, int64_t ldf, void* c,
                  int64_t ldc, int64_t nrhs, bool weighted, mht_apply_mode mode, void* stream, std::string& err) {
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err, mode};
  if (P.fp64)
    return P.cplx ? adjoint_dispatch<double, true>(x, f, ldf, c, ldc, weighted)
                  : adjoint_dispatch<double, false>(x, f, ldf, c, ldc, weighted);
  return P.cplx ? adjoint_dispatch<float, true>(x, f, ldf, c, ldc, weighted)
                : adjoint_dispatch<float, false>(x, f, ldf, c, ldc, weighted);
}

int64_t apply_launches(const Packed& P, int64_t nrhs, mht_apply_mode mode, int path) {
  (void)mode;
  if (path == 2 && nrhs <= 8) {
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

bool tensor_mode(mht_apply_mode m) { return m == MHT_APPLY_3XTF32 || m == MHT_APPLY_6XBF16; }

int device_upload_image(const Packed& P, void* base_dev, void* stream, std::string& err) {
  if (int rc = device_upload(base_dev, P.image.data(), P.image.size(), stream, err)) return rc;
  if (P.fp64 || P.tmap_bytes == 0) return 0;
  std::vector<uint8_t> maps;
  if (int rc = tc_encode_tmaps(P, base_dev, maps, err)) return rc;
  return device_upload(static_cast<uint8_t*>(base_dev) + P.tmap_off, maps.data(), maps.size(), stream, err);
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
//
// Layout of the array: [0, 256) the status word (sticky: set by a bounded wait that gave up,
// cleared only by mht_noalloc_check), then the level vectors, then the completion counters
// and the queue head (cleared by every call).
#include <mutex>

namespace mht {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(MHT_NOALLOC_SCRATCH_BYTES);
static_assert(kNoAllocScratchBytes == (size_t(16) << 20), "scratch size of the allocation-free synthesis");
constexpr size_t kNoAllocStatusBytes = 256;  // the status word's slot at the start of the array
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[256] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_base(uint8_t** base, std::string& err) {
  int dev = 0;
  if (int rc = check(cudaGetDevice(&dev), err, "cudaGetDevice")) return rc;
  if (dev < 0 || dev >= 256) {
    err = "device ordinal out of range";
    return MHT_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {  // set-up: once per device, with that device current
    void* a = nullptr;
    if (int rc = check(cudaGetSymbolAddress(&a, g_noalloc_scratch), err, "cudaGetSymbolAddress")) return rc;
    g_noalloc_addr[dev] = a;
  }
  *base = static_cast<uint8_t*>(g_noalloc_addr[dev]);
  return 0;
}

}  // namespace

size_t noalloc_scratch_need(const Packed& P) {
  const size_t ncnt = size_t(P.L + 2) * P.nb + 1;
  return kNoAllocStatusBytes + align256(size_t(std::max<int64_t>(P.vec_entries, 1)) * sizeof(float)) +
         align256(ncnt * sizeof(unsigned));
}

int apply_synthesize_noalloc(const Packed& P, const void* factor_dev, const void* c, void* f, void* stream,
                             std::string& err) {
  if (P.fp64 || P.cplx) {
    err = "the no-alloc synthesis serves real FP32 plans";
    return MHT_ERR_UNSUPPORTED;
  }
  const size_t ncnt = size_t(P.L + 2) * P.nb + 1;
  const size_t y_bytes = align256(size_t(std::max<int64_t>(P.vec_entries, 1)) * sizeof(float));
  const size_t cnt_bytes = align256(ncnt * sizeof(unsigned));
  const size_t need = noalloc_scratch_need(P);
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
  uint8_t* scratch = nullptr;
  if (int rc = noalloc_base(&scratch, err)) return rc;
  unsigned* status = reinterpret_cast<unsigned*>(scratch);
  float* y = reinterpret_cast<float*>(scratch + kNoAllocStatusBytes);
  unsigned* cnt = reinterpret_cast<unsigned*>(scratch + kNoAllocStatusBytes + y_bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: counters and queue head start at zero (the
  // status word is left for mht_noalloc_check)
  if (int rc = check(cudaMemsetAsync(cnt, 0, cnt_bytes, s), err, "scratch reset")) return rc;
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
  p.Y = y;
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

int noalloc_status(void* stream, unsigned* flags, std::string& err) {
  uint8_t* scratch = nullptr;
  if (int rc = noalloc_base(&scratch, err)) return rc;
  return device_status(scratch, stream, flags, err);
}

int noalloc_debug_hold(const Packed& P, void* factor_dev, bool hold, void* stream, std::string& err) {
  // completion target of block 0 of stage 0 in the synthesis work list (later stages wait for it)
  int32_t v = 0;
  const size_t off = P.fused[0].targets_off;
  std::memcpy(&v, P.image.data() + off, sizeof(v));
  if (hold) v = 0x7fffffff;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = check(cudaMemcpyAsync(static_cast<uint8_t*>(factor_dev) + off, &v, sizeof(v), cudaMemcpyHostToDevice, s),
                     err, "debug hold"))
    return rc;
  return check(cudaStreamSynchronize(s), err, "debug hold sync");
}

}  // namespace mht
