// Batched ragged apply: every stage of many plans (instances of different n, m, depth L,
// field and RHS count) in one persistent launch.
//
// The work items of all instances form one queue in dependency order: phase k of an
// instance (synthesis: stage k; adjoint: stage L+1-k) may start once all items of its phase
// k-1 are done.  CTAs claim items from the queue with an atomic ticket; a claimed item's
// dependencies all hold smaller tickets, which are claimed by running CTAs, so the waits
// always end (no co-residency requirement, no grid barrier).  Thread 0 of each CTA keeps a
// ring of shared-memory slots filled with 1-D bulk copies of the matrix rows of its claimed
// items, up to kBatchQ items ahead: matrix data does not depend on earlier phases, so its
// copies overlap the dependency wait and the previous item's compute.  An item's input vector
// is gathered only after the wait.  Completion is published per (instance, phase) counter with
// a release increment; waits are acquire loads, bounded in time, and an abort word stops all
// CTAs once one wait gives up (status value 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "../host/internal.h"
#include "rowdot.cuh"

namespace mht {
namespace {

constexpr int kBatchQ = 4;  // items a CTA may hold claimed ahead of the one it computes

struct BatchParams {
  const MhtBatchRec* recs;
  const MhtBItem* items;
  int nitems;
  unsigned* ticket;  // queue head
  unsigned* done;    // per (instance, direction, phase) completed items
  unsigned* abort;   // non-zero once any wait gave up
  unsigned* status;
  int use_wts;
  int slot_bytes, nslot, ldx_max, rows_max;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until *ctr >= need; false when it gave up (kWaitNs, or another CTA aborted).
__device__ bool wait_count(const unsigned* ctr, unsigned need, const unsigned* abort) {
  if (ld_acquire_u32(ctr) >= need) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    __nanosleep(100);
    if (ld_acquire_u32(ctr) >= need) return true;
    if ((it & 31) == 0) {
      if (*reinterpret_cast<const volatile unsigned*>(abort) != 0u) return false;
      if (globaltimer_ns() - t0 > kWaitNs) return false;
    }
  }
}

__device__ __forceinline__ int rec_rt(const MhtBatchRec& r) { return r.nrhs > 1 ? 8 : 1; }

// Thread-0 state: the claimed-item queue and the bulk-copy producer that runs ahead of the
// consumer through the claimed items.
struct BatchProducer {
  const BatchParams* p;
  int* q;               // shared: claimed tickets, ring of kBatchQ
  unsigned qh = 0;      // next ticket to compute (index into q)
  unsigned qt = 0;      // tickets claimed
  bool exhausted = false;
  unsigned pq = 0;      // claimed item whose chunks are being issued
  bool loaded = false;
  int j = 0, total = 0, rpc = 1, nch = 1, rowbytes = 0, start = 0, count = 0, ldt = 0;
  const float* data = nullptr;
  long long t_off = 0;
  unsigned issued = 0;

  __device__ void claim() {
    const unsigned t = atomicAdd(p->ticket, 1u);
    if (t >= unsigned(p->nitems)) {
      exhausted = true;
      return;
    }
    q[qt % kBatchQ] = int(t);
    ++qt;
  }
  __device__ void load(int slot_bytes) {
    const MhtBItem bi = p->items[q[pq % kBatchQ]];
    const MhtBatchRec& r = p->recs[bi.rec];
    const MhtBlockDesc d = reinterpret_cast<const MhtBlockDesc*>(r.desc)[bi.blk];
    count = bi.count_sib & 0x7fffffff;
    start = bi.start;
    ldt = d.ldt;
    t_off = d.t_off;
    data = reinterpret_cast<const float*>(r.data);
    const int W = r.cplx ? 2 : 1;
    rowbytes = d.ldt * W * 4;
    total = 0;
    j = 0;
    if (rowbytes > 0 && count > 0) {
      rpc = max(1, slot_bytes / rowbytes);
      nch = (count + rpc - 1) / rpc;
      const int rt = rec_rt(r);
      total = nch * ((r.nrhs + rt - 1) / rt);
    }
    loaded = true;
  }
  // keeps up to nslot copies in flight (cons = chunks consumed so far)
  __device__ void pump(const RowSmem& sm, unsigned cons) {
    while (issued - cons < unsigned(sm.nslot)) {
      if (pq == qt) {
        if (exhausted || qt - qh >= unsigned(kBatchQ)) return;
        claim();
        if (exhausted) return;
      }
      if (!loaded) load(sm.slot_bytes);
      if (j >= total) {  // no copies (left) for this item
        ++pq;
        loaded = false;
        continue;
      }
      const int ch = j % nch;
      const int W = rowbytes / (ldt * 4);
      const unsigned slot = issued % unsigned(sm.nslot);
      const unsigned bytes = unsigned(min(rpc, count - ch * rpc)) * unsigned(rowbytes);
      mbar_expect_tx(&sm.bar[slot], bytes);
      bulk_copy_g2s(sm.slots + size_t(slot) * sm.slot_bytes, data + (t_off + (long long)(start + ch * rpc) * ldt) * W,
                    bytes, &sm.bar[slot]);
      ++issued;
      ++j;
    }
  }
};

template <bool C, int RT>
__device__ bool batch_item(const MhtBatchRec& r, const MhtItem& it, const MhtBlockDesc& d, const RowSmem& sm,
                           unsigned& cons, unsigned* status, int use_wts, BatchProducer& prod) {
  RowArgs<float> a{reinterpret_cast<const float*>(r.data), reinterpret_cast<const int*>(r.idx),
                   reinterpret_cast<const MhtBlockDesc*>(r.desc), reinterpret_cast<const int*>(r.perm),
                   use_wts ? reinterpret_cast<const float*>(r.wts) : nullptr, reinterpret_cast<const float*>(r.in0),
                   reinterpret_cast<const float*>(r.in1), r.is_e, r.is_k, reinterpret_cast<float*>(r.out0),
                   reinterpret_cast<float*>(r.out1), r.os_e, r.os_k, r.nrhs};
  auto refill = [&] { prod.pump(sm, cons); };
  switch (r.mode) {
    case SYN_ID: return row_item<float, C, RT, SYN_ID>(a, it, d, sm, cons, status, refill);
    case ADJ_ID: return row_item<float, C, RT, ADJ_ID>(a, it, d, sm, cons, status, refill);
    case SYN_U: return row_item<float, C, RT, SYN_U>(a, it, d, sm, cons, status, refill);
    default: return row_item<float, C, RT, ADJ_U>(a, it, d, sm, cons, status, refill);
  }
}

__global__ void __launch_bounds__(kThreads) k_batch(BatchParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RowSmem sm = row_smem<float, true>(smem_raw, p.slot_bytes, p.nslot, p.ldx_max, p.rows_max);
  int* q = reinterpret_cast<int*>(smem_raw + 80);                          // [kBatchQ]
  volatile int* s_ticket = reinterpret_cast<volatile int*>(smem_raw + 112);  // item to compute
  BatchProducer prod;
  prod.p = &p;
  prod.q = q;
  if (threadIdx.x == 0) {
    for (int i = 0; i < p.nslot; ++i) mbar_init(&sm.bar[i], 1);
    *sm.flag = 1;
  }
  unsigned cons = 0;
  bool ok = true;
  for (;;) {
    if (threadIdx.x == 0) {
      if (prod.qh == prod.qt && !prod.exhausted) prod.claim();
      *s_ticket = prod.qh < prod.qt ? q[prod.qh % kBatchQ] : -1;
      prod.pump(sm, cons);
    }
    __syncthreads();
    const int t = *s_ticket;
    if (t < 0) break;
    const MhtBItem bi = p.items[t];
    const MhtBatchRec& r = p.recs[bi.rec];
    const int cplx = r.cplx, rt = rec_rt(r), wait_ctr = r.wait_ctr, done_ctr = r.done_ctr;
    const MhtItem it{bi.blk, bi.start, bi.count_sib & 0x7fffffff, int(unsigned(bi.count_sib) >> 31)};
    const MhtBlockDesc d = reinterpret_cast<const MhtBlockDesc*>(r.desc)[bi.blk];
    if (threadIdx.x == 0 && wait_ctr >= 0 && !wait_count(p.done + wait_ctr, r.wait_count, p.abort)) {
      atomicOr(p.status, 2u);
      atomicExch(p.abort, 1u);
      *sm.flag = 0;
    }
    __syncthreads();
    if (!*sm.flag) {
      ok = false;
      break;
    }
    if (cplx)
      ok = rt == 1 ? batch_item<true, 1>(r, it, d, sm, cons, p.status, p.use_wts, prod)
                   : batch_item<true, 8>(r, it, d, sm, cons, p.status, p.use_wts, prod);
    else
      ok = rt == 1 ? batch_item<false, 1>(r, it, d, sm, cons, p.status, p.use_wts, prod)
                   : batch_item<false, 8>(r, it, d, sm, cons, p.status, p.use_wts, prod);
    if (!ok) {
      atomicExch(p.abort, 1u);
      break;
    }
    if (threadIdx.x == 0) {  // every thread's outputs precede this (row_item ends with a barrier)
      ++prod.qh;
      __threadfence();
      atomicAdd(p.done + done_ctr, 1u);
    }
  }
  if (threadIdx.x == 0 && !ok) row_drain(sm, cons, prod.issued);
}

}  // namespace

// Shared memory of the batch kernel for the given maxima (RT 8, complex layout).
size_t batch_smem(int slot_bytes, int nslot, int ldx_max, int rows_max) {
  return 128 + size_t(nslot) * slot_bytes + size_t(ldx_max) * 8 * 8 + size_t(rows_max) * 8 * 8 +
         size_t(rows_max) * sizeof(int);
}

namespace {

BatchParams make_params(const BatchLaunch& b) {
  BatchParams p{};
  p.recs = reinterpret_cast<const MhtBatchRec*>(b.recs);
  p.items = reinterpret_cast<const MhtBItem*>(b.items);
  p.nitems = b.nitems;
  p.ticket = b.ticket;
  p.done = b.done;
  p.abort = b.abort;
  p.status = b.status;
  p.use_wts = b.use_wts;
  p.slot_bytes = b.slot_bytes;
  p.nslot = b.nslot;
  p.ldx_max = b.ldx_max;
  p.rows_max = b.rows_max;
  return p;
}

int cuda_check(cudaError_t e, std::string& err, const char* what) {
  if (e == cudaSuccess) return 0;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return MHT_ERR_CUDA;
}

// Grid of the persistent launch: as many CTAs as fit on the GPU at once, at most one per item.
int batch_config(const BatchLaunch& b, int* grid, size_t* smem, std::string& err) {
  *smem = batch_smem(b.slot_bytes, b.nslot, b.ldx_max, b.rows_max);
  int per_sm = 0, dev = 0, sms = 0;
  if (int rc = cuda_check(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem)), err,
                          "batch kernel shared memory"))
    return rc;
  if (int rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, *smem), err,
                          "batch kernel occupancy"))
    return rc;
  if (int rc = cuda_check(cudaGetDevice(&dev), err, "device")) return rc;
  if (int rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), err, "SM count")) return rc;
  if (per_sm < 1) {
    err = "the batch kernel does not fit an SM";
    return MHT_ERR_UNSUPPORTED;
  }
  if (b.per_sm > 0) per_sm = std::min(per_sm, b.per_sm);
  *grid = int(std::min<int64_t>(int64_t(per_sm) * sms, std::max(b.nitems, 1)));
  return 0;
}

}  // namespace

struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int batch_launch(const BatchLaunch& b, void* stream, std::string& err) {
  int grid = 0;
  size_t smem = 0;
  if (int rc = batch_config(b, &grid, &smem, err)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = cuda_check(cudaMemsetAsync(b.counters, 0, b.counter_bytes, s), err, "batch counters")) return rc;
  k_batch<<<grid, kThreads, smem, s>>>(make_params(b));
  return cuda_check(cudaGetLastError(), err, "batch launch");
}

// The same two operations (zero the counters, run the persistent kernel) as a CUDA graph
// built node by node, so that a launch costs one cudaGraphLaunch.
int batch_graph_create(const BatchLaunch& b, BatchGraph** out, std::string& err) {
  *out = nullptr;
  int grid = 0;
  size_t smem = 0;
  if (int rc = batch_config(b, &grid, &smem, err)) return rc;
  BatchGraph* g = new BatchGraph();
  auto fail = [&](int rc) {
    batch_graph_destroy(g);
    return rc;
  };
  if (int rc = cuda_check(cudaGraphCreate(&g->graph, 0), err, "graph create")) return fail(rc);
  cudaMemsetParams mp{};
  mp.dst = b.counters;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = b.counter_bytes / 4;
  mp.height = 1;
  mp.pitch = 0;
  cudaGraphNode_t zero = nullptr, kern = nullptr;
  if (int rc = cuda_check(cudaGraphAddMemsetNode(&zero, g->graph, nullptr, 0, &mp), err, "graph memset node"))
    return fail(rc);
  BatchParams p = make_params(b);
  void* args[] = {&p};
  cudaKernelNodeParams kp{};
  kp.func = reinterpret_cast<void*>(&k_batch);
  kp.gridDim = dim3(unsigned(grid));
  kp.blockDim = dim3(kThreads);
  kp.sharedMemBytes = unsigned(smem);
  kp.kernelParams = args;
  kp.extra = nullptr;
  if (int rc = cuda_check(cudaGraphAddKernelNode(&kern, g->graph, &zero, 1, &kp), err, "graph kernel node"))
    return fail(rc);
  if (int rc = cuda_check(cudaGraphInstantiate(&g->exec, g->graph, 0), err, "graph instantiate")) return fail(rc);
  *out = g;
  return 0;
}

int batch_graph_launch(BatchGraph* g, void* stream, std::string& err) {
  return cuda_check(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), err, "graph launch");
}

void batch_graph_destroy(BatchGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

// Times one synthesis and one analysis launch for every (ring slots, CTAs per SM) pair and
// returns the fastest pair; the launches use the batch's own vectors.
int batch_autotune(const BatchLaunch& syn, const BatchLaunch& ana, int max_nslot, void* stream, int* nslot,
                   int* per_sm, double* best_ms, std::string& err) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (int rc = cuda_check(cudaEventCreate(&e0), err, "event")) return rc;
  if (int rc = cuda_check(cudaEventCreate(&e1), err, "event")) return rc;
  float best = 1e30f;
  int rc = 0;
  for (int ns = 1; ns <= max_nslot && !rc; ++ns)
    for (int ps = 1; ps <= 4 && !rc; ++ps) {
      BatchLaunch a = syn, b = ana;
      a.nslot = b.nslot = ns;
      a.per_sm = b.per_sm = ps;
      int g = 0;
      size_t smem = 0;
      if (batch_config(a, &g, &smem, err) != 0) {  // does not fit: skip
        cudaGetLastError();
        continue;
      }
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kThreads, smem);
      if (ps > per) continue;  // same launch as a smaller count
      if ((rc = batch_launch(a, stream, err)) || (rc = batch_launch(b, stream, err))) break;  // warm-up
      if ((rc = cuda_check(cudaEventRecord(e0, s), err, "event"))) break;
      for (int r = 0; r < 3 && !rc; ++r)
        if (!(rc = batch_launch(a, stream, err))) rc = batch_launch(b, stream, err);
      if (rc) break;
      if ((rc = cuda_check(cudaEventRecord(e1, s), err, "event"))) break;
      if ((rc = cuda_check(cudaEventSynchronize(e1), err, "event sync"))) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 3 < best) {
        best = ms / 3;
        *nslot = ns;
        *per_sm = ps;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = best;
  return rc;
}

struct TcGroup {
  static constexpr int kStreams = 8;
  cudaStream_t s0 = nullptr;
  cudaStream_t side[kStreams] = {};
  cudaEvent_t ev[kStreams + 1] = {};
  cudaGraphExec_t exec = nullptr;
};

void tc_group_destroy(TcGroup* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : g->side)
    if (s) cudaStreamDestroy(s);
  if (g->s0) cudaStreamDestroy(g->s0);
  delete g;
}

int batch_tc_run(mht_batch& B, int dir, bool weighted, void* stream, std::string& err) {
  TcGroup*& g = B.tc[dir == 0 ? 0 : (weighted ? 2 : 1)];
  if (!g) {
    g = new TcGroup();
    int rc = cuda_check(cudaStreamCreateWithFlags(&g->s0, cudaStreamNonBlocking), err, "stream");
    for (int k = 0; k < TcGroup::kStreams && !rc; ++k)
      rc = cuda_check(cudaStreamCreateWithFlags(&g->side[k], cudaStreamNonBlocking), err, "stream");
    for (int k = 0; k <= TcGroup::kStreams && !rc; ++k)
      rc = cuda_check(cudaEventCreateWithFlags(&g->ev[k], cudaEventDisableTiming), err, "event");
    if (!rc) rc = cuda_check(cudaStreamBeginCapture(g->s0, cudaStreamCaptureModeThreadLocal), err, "capture");
    if (rc) {
      tc_group_destroy(g);
      g = nullptr;
      return rc;
    }
    // fork: every side stream starts after the capture origin
    rc = cuda_check(cudaEventRecord(g->ev[TcGroup::kStreams], g->s0), err, "fork");
    for (int k = 0; k < TcGroup::kStreams && !rc; ++k)
      rc = cuda_check(cudaStreamWaitEvent(g->side[k], g->ev[TcGroup::kStreams], 0), err, "fork");
    for (int i = 0; i < B.n && !rc; ++i) {
      const BatchInst& I = B.inst[i];
      DeviceView dv;
      dv.base = B.image_dev + I.image_off;
      dv.ws = B.ws_dev + I.ws_off;
      dv.ws_bytes = I.ws_bytes;
      dv.max_nrhs = I.nrhs;
      dv.path = 1;
      cudaStream_t st = g->side[i % TcGroup::kStreams];
      void* c = reinterpret_cast<void*>(I.c);
      void* f = reinterpret_cast<void*>(I.f);
      rc = dir == 0 ? apply_synthesize(I.shape, I.meta, dv, c, I.ldc, f, I.ldf, I.nrhs, false, B.mode, st, err)
                    : apply_analyze(I.shape, I.meta, dv, f, I.ldf, c, I.ldc, I.nrhs, weighted, B.mode, st, err);
    }
    // join: the origin waits for every side stream
    for (int k = 0; k < TcGroup::kStreams && !rc; ++k) {
      rc = cuda_check(cudaEventRecord(g->ev[k], g->side[k]), err, "join");
      if (!rc) rc = cuda_check(cudaStreamWaitEvent(g->s0, g->ev[k], 0), err, "join");
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->s0, &graph);
    if (!rc && e != cudaSuccess) rc = cuda_check(e, err, "capture end");
    if (!rc) rc = cuda_check(cudaGraphInstantiate(&g->exec, graph, 0), err, "graph instantiate");
    if (graph) cudaGraphDestroy(graph);
    if (rc) {
      tc_group_destroy(g);
      g = nullptr;
      return rc;
    }
  }
  return cuda_check(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), err, "graph launch");
}

int batch_grid_size(const BatchLaunch& b, std::string& err) {
  int grid = 0;
  size_t smem = 0;
  if (int rc = batch_config(b, &grid, &smem, err)) return -rc;
  return grid;
}

}  // namespace mht
