// Device building blocks shared by the butterfly apply kernels: bounded mbarrier waits and
// 1-D bulk copies, compensated row dot products, and the streamed computation of one work
// item (a row range of one stored block) for all right-hand sides.  Included by the CUDA
// translation units only; everything has internal linkage.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../layout.h"

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

// One row of a block product, reduced by a warp: acc[t] = sum_j row[j] * x_t[j] for the RT
// staged right-hand sides x_t (xs + t * ldx elements).  Lane l takes the 16-byte vectors
// l, l + 32, ...; the lanes are then combined by a butterfly of shuffles, so every lane ends
// with the full sums.
//
// In FP32 the sums are compensated (Kahan 1965): the products of one 16-byte vector are
// summed by a chain of fused multiply-adds, and that short partial enters the lane's running
// sum with Kahan's correction; for a single RHS each lane keeps two such sums (even and odd
// vectors) for instruction-level parallelism, and the partials are combined with error-free two-sums
// (Knuth's TwoSum).  Plain FP32 accumulation loses about u * sum_j |row[j] x[j]|, which after
// the cancellation in these products and L + 2 chained stages amounts to ~1e-6 relative error
// at 65536 points; with compensation the error is dominated by rounding the factors and the
// stored vectors to FP32.  FP64 accumulates plainly.
template <class R>
__device__ __forceinline__ R fmad(R a, R b, R c) { return fma(a, b, c); }

template <class R>
__device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
  s = a + b;
  const R bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// s - c holds the running sum; adds y with Kahan's correction
template <class R>
__device__ __forceinline__ void kahan_add(R& s, R& c, R y) {
  const R yc = y - c;
  const R t = s + yc;
  c = (t - s) - yc;
  s = t;
}

// Products of one 16-byte vector of the row with the same entries of x_t: one partial per
// component (real; or real and imaginary part of sum (p + iq)(xr + i xi)).
template <class R, bool C>
__device__ __forceinline__ void vec_partial(const Vec16<R>& tv, const Vec16<R>& xv, R (&part)[C ? 2 : 1]) {
  constexpr int NS = 16 / sizeof(R);
  if (C) {
    R re = tv.s[0] * xv.s[0], im = tv.s[0] * xv.s[1];
    re = fmad(-tv.s[1], xv.s[1], re);
    im = fmad(tv.s[1], xv.s[0], im);
#pragma unroll
    for (int e = 1; e < NS / 2; ++e) {
      re = fmad(tv.s[2 * e], xv.s[2 * e], re);
      re = fmad(-tv.s[2 * e + 1], xv.s[2 * e + 1], re);
      im = fmad(tv.s[2 * e], xv.s[2 * e + 1], im);
      im = fmad(tv.s[2 * e + 1], xv.s[2 * e], im);
    }
    part[0] = re;
    part[C ? 1 : 0] = im;
  } else {
    R p = tv.s[0] * xv.s[0];
#pragma unroll
    for (int e = 1; e < NS; ++e) p = fmad(tv.s[e], xv.s[e], p);
    part[0] = p;
  }
}

template <class R, bool C, int RT>
__device__ __forceinline__ void row_dot(const R* __restrict__ row, const R* __restrict__ xs, int ldx, int nvec, int lane,
                                        R (&acc)[RT][C ? 2 : 1]) {
  constexpr int W = C ? 2 : 1;
  constexpr int NS = 16 / sizeof(R);
  constexpr int E = NS / W;
  constexpr bool COMP = sizeof(R) == 4;
  if (!COMP) {
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[t][c] = R(0);
    for (int v = lane; v < nvec; v += 32) {
      const Vec16<R> tv = *reinterpret_cast<const Vec16<R>*>(row + v * NS);
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        const Vec16<R> xv = *reinterpret_cast<const Vec16<R>*>(xs + (t * ldx + v * E) * W);
        R part[W];
        vec_partial<R, C>(tv, xv, part);
#pragma unroll
        for (int c = 0; c < W; ++c) acc[t][c] += part[c];
      }
    }
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[t][c] = warp_sum(acc[t][c]);
    return;
  }
  // a second chain only for a single RHS, where the tile alone gives too little parallelism
  // (every tile of two or more RHS then rounds identically, whatever its width)
  constexpr int NC = RT == 1 ? 2 : 1;
  R s0[RT][W], c0[RT][W], s1[RT][W], c1[RT][W];
#pragma unroll
  for (int t = 0; t < RT; ++t)
#pragma unroll
    for (int c = 0; c < W; ++c) s0[t][c] = c0[t][c] = s1[t][c] = c1[t][c] = R(0);
  for (int v = lane; v < nvec; v += 32 * NC) {
    const bool two = NC == 2 && v + 32 < nvec;
    const Vec16<R> ta = *reinterpret_cast<const Vec16<R>*>(row + v * NS);
    Vec16<R> tb;
    if (two) tb = *reinterpret_cast<const Vec16<R>*>(row + (v + 32) * NS);
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const Vec16<R> xa = *reinterpret_cast<const Vec16<R>*>(xs + (t * ldx + v * E) * W);
      R pa[W];
      vec_partial<R, C>(ta, xa, pa);
#pragma unroll
      for (int c = 0; c < W; ++c) kahan_add(s0[t][c], c0[t][c], pa[c]);
      if (two) {
        const Vec16<R> xb = *reinterpret_cast<const Vec16<R>*>(xs + (t * ldx + (v + 32) * E) * W);
        R pb[W];
        vec_partial<R, C>(tb, xb, pb);
#pragma unroll
        for (int c = 0; c < W; ++c) kahan_add(s1[t][c], c1[t][c], pb[c]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < RT; ++t)
#pragma unroll
    for (int c = 0; c < W; ++c) {
      R sum, err;
      two_sum(s0[t][c], s1[t][c], sum, err);
      err = err - c0[t][c] - c1[t][c];  // the Kahan corrections enter with their sign flipped
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const R so = __shfl_xor_sync(0xffffffffu, sum, o);
        const R eo = __shfl_xor_sync(0xffffffffu, err, o);
        R s2, e2;
        two_sum(sum, so, s2, e2);
        sum = s2;
        err = err + eo + e2;
      }
      acc[t][c] = sum + err;
    }
}

// Two rows of a real block at once for RT >= 2 RHS (one Kahan chain per RHS, as in row_dot):
// the staged inputs are loaded once for both rows, halving the shared-memory traffic per
// multiply-add; each row's arithmetic is exactly row_dot's, so results are identical.
template <class R, int RT>
__device__ __forceinline__ void row_dot2(const R* __restrict__ rowa, const R* __restrict__ rowb,
                                         const R* __restrict__ xs, int ldx, int nvec, int lane, R (&acca)[RT][1],
                                         R (&accb)[RT][1]) {
  static_assert(RT >= 2, "pairs of rows are for RHS tiles");
  constexpr int NS = 16 / sizeof(R);
  R sa[RT], ca[RT], sb[RT], cb[RT];
#pragma unroll
  for (int t = 0; t < RT; ++t) sa[t] = ca[t] = sb[t] = cb[t] = R(0);
  for (int v = lane; v < nvec; v += 32) {
    const Vec16<R> ta = *reinterpret_cast<const Vec16<R>*>(rowa + v * NS);
    const Vec16<R> tb = *reinterpret_cast<const Vec16<R>*>(rowb + v * NS);
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const Vec16<R> xv = *reinterpret_cast<const Vec16<R>*>(xs + t * ldx + v * NS);
      R pa[1], pb[1];
      vec_partial<R, false>(ta, xv, pa);
      vec_partial<R, false>(tb, xv, pb);
      if (sizeof(R) == 4) {
        kahan_add(sa[t], ca[t], pa[0]);
        kahan_add(sb[t], cb[t], pb[0]);
      } else {
        sa[t] += pa[0];
        sb[t] += pb[0];
      }
    }
  }
#pragma unroll
  for (int t = 0; t < RT; ++t) {
    if (sizeof(R) == 4) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        R sum = h ? sb[t] : sa[t], err = h ? -cb[t] : -ca[t];
        // same combination as row_dot with a single chain: TwoSum against a zero second chain
        R s2, e2;
        two_sum(sum, R(0), s2, e2);
        sum = s2;
        err = e2 + err;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const R so = __shfl_xor_sync(0xffffffffu, sum, o);
          const R eo = __shfl_xor_sync(0xffffffffu, err, o);
          two_sum(sum, so, s2, e2);
          sum = s2;
          err = err + eo + e2;
        }
        (h ? accb : acca)[t][0] = sum + err;
      }
    } else {
      acca[t][0] = warp_sum(sa[t]);
      accb[t][0] = warp_sum(sb[t]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// out[o(i)] = ident(i) + sum_j M[i, j] x[j] for the rows i of one work item.
//   SYN_ID: M = T~ (r x K'),           x[j] = in[idx[r + j]],   o(i) = out_off + i,
//           ident(i) = in[idx[i]]  (times w[idx[.]] when a scale is given: leaf stage only)
//   ADJ_ID: M = conj(T~)^T (K' x r),   x[j] = z0[out_off + j] (+ z1[...]),
//           o(i) = idx[r + i] in the sibling buffer; skeleton out[idx[j]] = x[j]
//   SYN_U:  M = U (|tau| x r_L),       x[j] = yL[in_off + j],   o(i) = perm[out_off + i]
//           (times w[o(i)] when weights are given)
//   ADJ_U:  M = conj(U)^T (r_L x |tau|), x[j] = w[p] f[p] with p = perm[out_off + j],
//           o(i) = in_off + i
// Element strides: in[e * is_e + k * is_k], out[e * os_e + k * os_k]; one complex value is
// one element.  The item's RHS are processed in tiles of RT: the rows are streamed through
// a ring of shared-memory slots by 1-D bulk copies (the first tile reads them from HBM, later
// tiles re-read the same ~128 KB from L2), and each tile's input vector, identity terms and
// output indices are staged once per tile.
constexpr int kRowSlots = 3;     // default bulk copies in flight per CTA
constexpr int kMaxRowSlots = 8;  // barrier area holds up to 8 slot barriers

template <class R>
struct RowArgs {
  const R* data;
  const int* idx;
  const MhtBlockDesc* desc;
  const int* perm;
  const R* wts;
  const R* in0;
  const R* in1;
  long long is_e, is_k;
  R* out0;
  R* out1;
  long long os_e, os_k;
  int nrhs;
};

// Shared memory of one CTA: [barriers 64 B][flag][slots nslot x slot_bytes at 128][xs][ident][oidx]
struct RowSmem {
  uint64_t* bar;
  volatile int* flag;
  unsigned char* slots;
  int slot_bytes, nslot, ldx_max, rows_max;
};

template <class R, bool C>
__device__ __forceinline__ RowSmem row_smem(unsigned char* raw, int slot_bytes, int nslot, int ldx_max, int rows_max) {
  RowSmem m;
  m.bar = reinterpret_cast<uint64_t*>(raw);
  m.flag = reinterpret_cast<volatile int*>(raw + 64);
  m.slots = raw + 128;
  m.slot_bytes = slot_bytes;
  m.nslot = nslot;
  m.ldx_max = ldx_max;
  m.rows_max = rows_max;
  return m;
}

// Producer of the bulk-copy ring (thread 0 of a CTA).  It walks the CTA's items in the order
// the CTA consumes them (items first, start, first + stride, ...; per item tile-major: every
// chunk of RHS tile 0, then of tile 1, ...) and keeps up to nslot chunks in flight, so copies
// for the next item are already landing while the current one is computed.  Chunk g of the
// sequence goes to slot g % nslot; its barrier phase is (g / nslot) & 1.
template <class R, bool C>
struct RowProducer {
  static constexpr int W = C ? 2 : 1;
  const MhtItem* items;
  const MhtBlockDesc* desc;
  const R* data;
  int nitems, stride, ntile;
  int item;          // item being issued (>= nitems: done)
  int j = 0, total = 0, rpc = 1, nch = 0, rowbytes = 0;
  MhtItem it{};
  MhtBlockDesc d{};
  unsigned issued = 0;

  __device__ void load(int slot_bytes) {  // advance to the first item (from `item` on) that has copies
    for (; item < nitems; item += stride) {
      it = items[item];
      d = desc[it.blk];
      rowbytes = d.ldt * int(W * sizeof(R));
      if (rowbytes > 0 && it.count > 0) break;
    }
    if (item < nitems) {
      rpc = max(1, slot_bytes / rowbytes);
      nch = (it.count + rpc - 1) / rpc;
      total = nch * ntile;
      j = 0;
    }
  }
  // issues the next chunk into its slot; false when the CTA has no more copies
  __device__ bool issue(const RowSmem& sm) {
    if (item >= nitems) return false;
    const int ch = j % nch;
    const unsigned slot = issued % unsigned(sm.nslot);
    const unsigned bytes = unsigned(min(rpc, it.count - ch * rpc)) * unsigned(rowbytes);
    mbar_expect_tx(&sm.bar[slot], bytes);
    bulk_copy_g2s(sm.slots + size_t(slot) * sm.slot_bytes, data + (d.t_off + (long long)(it.start + ch * rpc) * d.ldt) * W,
                  bytes, &sm.bar[slot]);
    ++issued;
    if (++j == total) {
      item += stride;
      load(sm.slot_bytes);
    }
    return true;
  }
};

// Computes one work item for all RHS from the chunks the producer streams in.  `cons` is the
// CTA's count of consumed chunks (uniform across threads); after each chunk thread 0 calls
// refill() to issue the next copy into the slot just freed.  Returns false when a bounded wait
// gave up (status bit set).  Called by all threads of the CTA; ends with a barrier, so the
// shared buffers may be reused right after.
template <class R, bool C, int RT, int MODE, class Refill>
__device__ bool row_item(const RowArgs<R>& a, const MhtItem& it, const MhtBlockDesc& d, const RowSmem& sm,
                         unsigned& cons, unsigned* status, Refill&& refill) {
  constexpr int W = C ? 2 : 1;
  constexpr int NS = 16 / sizeof(R);
  constexpr int E = NS / W;
  const int nslot = sm.nslot, ldx_max = sm.ldx_max, rows_max = sm.rows_max;
  R* xs = reinterpret_cast<R*>(sm.slots + size_t(nslot) * sm.slot_bytes);  // [RT][ldx][W]
  R* ident = xs + size_t(RT) * ldx_max * W;                                 // [RT][rows][W]
  int* oidx = reinterpret_cast<int*>(ident + size_t(RT) * rows_max * W);    // [rows]
  volatile int* flag = sm.flag;

  const int ldt = d.ldt;
  const int rowbytes = ldt * int(W * sizeof(R));
  const bool copies = rowbytes > 0 && it.count > 0;
  const int rpc = rowbytes > 0 ? max(1, sm.slot_bytes / rowbytes) : max(1, it.count);  // rows per chunk
  const int nch = it.count == 0 ? 0 : (it.count + rpc - 1) / rpc;
  const int ntile = (a.nrhs + RT - 1) / RT;
  R* out = (MODE == ADJ_ID && it.sib) ? a.out1 : a.out0;
  // every warp: lane 0 waits (bounded) for chunk g of the CTA's sequence and the warp follows
  // its verdict; a warp that gave up clears the CTA's flag, and the next barrier makes every
  // warp stop (the rows it computed meanwhile are unspecified, as the status bit reports)
  auto wait_chunk = [&](unsigned g) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
      ok = mbar_wait_bounded(&sm.bar[g % unsigned(nslot)], (g / unsigned(nslot)) & 1u) ? 1 : 0;
      if (!ok) {
        atomicOr(status, 1u);
        *flag = 0;
      }
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
  };

  if (MODE == ADJ_ID || MODE == SYN_U)
    for (int ii = threadIdx.x; ii < it.count; ii += kThreads) {
      const int i = it.start + ii;
      if (MODE == ADJ_ID) {
        oidx[ii] = a.idx[d.idx_off + d.cols + i];
      } else {
        const int dst = a.perm[d.out_off + i];
        oidx[ii] = dst;
        ident[ii * W] = a.wts ? a.wts[dst] : R(1);
      }
    }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec = ldt / E;
  for (int tile = 0; tile < ntile; ++tile) {
    const int k0 = tile * RT;
    const int nk = min(RT, a.nrhs - k0);
    // stage this tile's input vector (zero padding to ldt and beyond nk) and identity terms
    for (int jj = threadIdx.x; jj < ldt; jj += kThreads) {
      long long src = -1;
      R w = R(1);
      if (jj < d.cols) {
        if (MODE == SYN_ID) {
          src = a.idx[d.idx_off + d.rows + jj];
          if (a.wts) w = a.wts[src];  // leaf stage: diagonal scale of the coefficients
        }
        else if (MODE == ADJ_ID) src = (long long)d.out_off + jj;
        else if (MODE == SYN_U) src = (long long)d.in_off + jj;
        else {
          src = a.perm[d.out_off + jj];
          if (a.wts) w = a.wts[src];
        }
      }
#pragma unroll
      for (int t = 0; t < RT; ++t)
#pragma unroll
        for (int c = 0; c < W; ++c) {
          R v = R(0);
          if (src >= 0 && t < nk) {
            const long long e = (src * a.is_e + (long long)(k0 + t) * a.is_k) * W + c;
            v = __ldcg(a.in0 + e);
            if (MODE == ADJ_ID && a.in1) v += __ldcg(a.in1 + e);
            v *= w;
          }
          xs[(t * ldx_max + jj) * W + c] = v;
        }
    }
    if (MODE == SYN_ID)
      for (int ii = threadIdx.x; ii < it.count; ii += kThreads) {
        const long long sidx = a.idx[d.idx_off + it.start + ii];
        const R sw = a.wts ? a.wts[sidx] : R(1);
#pragma unroll
        for (int t = 0; t < RT; ++t)
#pragma unroll
          for (int c = 0; c < W; ++c)
            ident[(t * rows_max + ii) * W + c] =
                t < nk ? sw * __ldcg(a.in0 + (sidx * a.is_e + (long long)(k0 + t) * a.is_k) * W + c) : R(0);
      }
    __syncthreads();  // the tile's inputs are staged
    if (MODE == ADJ_ID && it.start == 0) {  // identity part: out[skel_j] = z_j
      for (int e = threadIdx.x; e < d.cols * nk; e += kThreads) {
        const int jj = e / nk, t = e % nk;
        const long long dst = a.idx[d.idx_off + jj];
#pragma unroll
        for (int c = 0; c < W; ++c)
          out[(dst * a.os_e + (long long)(k0 + t) * a.os_k) * W + c] = xs[(t * ldx_max + jj) * W + c];
      }
    }
    for (int ch = 0; ch < nch; ++ch) {
      const int slot = int(cons % unsigned(nslot));
      const bool ready = !copies || wait_chunk(cons);  // each warp waits for the chunk itself
      const R* rows = reinterpret_cast<const R*>(sm.slots + size_t(slot) * sm.slot_bytes);
      const int cnt = min(rpc, it.count - ch * rpc);
      // writes row ii of the item for this tile's RHS (lane t holds RHS t)
      auto store_row = [&](int ii, const R (&acc)[RT][W]) {
        const int i = it.start + ii;
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
#pragma unroll
            for (int c = 0; c < W; ++c) val[c] += ident[(t * rows_max + ii) * W + c];
            dst = (long long)d.out_off + i;
          } else if (MODE == ADJ_ID) {
            dst = oidx[ii];
          } else if (MODE == SYN_U) {
            dst = oidx[ii];
            const R w = ident[ii * W];
#pragma unroll
            for (int c = 0; c < W; ++c) val[c] *= w;
          } else {
            dst = (long long)d.in_off + i;
          }
#pragma unroll
          for (int c = 0; c < W; ++c) out[(dst * a.os_e + (long long)(k0 + t) * a.os_k) * W + c] = val[c];
        }
      };
      if constexpr (!C && RT >= 4) {
        // pairs of rows (rr, rr + kWarps) share their staged-input loads
        for (int rr = ready ? warp : cnt; rr < cnt; rr += 2 * kWarps) {
          const int rr2 = rr + kWarps;
          if (rr2 < cnt) {
            R acca[RT][W], accb[RT][W];
            row_dot2<R, RT>(rows + (long long)rr * ldt * W, rows + (long long)rr2 * ldt * W, xs, ldx_max, nvec, lane,
                            acca, accb);
            store_row(ch * rpc + rr, acca);
            store_row(ch * rpc + rr2, accb);
          } else {
            R acc[RT][W];
            row_dot<R, C, RT>(rows + (long long)rr * ldt * W, xs, ldx_max, nvec, lane, acc);
            store_row(ch * rpc + rr, acc);
          }
        }
      } else {
        for (int rr = ready ? warp : cnt; rr < cnt; rr += kWarps) {
          R acc[RT][W];
          row_dot<R, C, RT>(rows + (long long)rr * ldt * W, xs, ldx_max, nvec, lane, acc);
          store_row(ch * rpc + rr, acc);
        }
      }
      // one barrier per chunk: the slot (and after the tile's last chunk, xs / ident) is free
      // and thread 0 refills it at once
      __syncthreads();
      if (!*flag) return false;
      if (copies) {
        ++cons;
        if (threadIdx.x == 0) refill();
      }
    }
    if (nch == 0) __syncthreads();  // xs was read by the identity part only
  }
  return true;
}

// Waits (bounded) for every copy issued but not consumed, so that no bulk copy is still
// writing shared memory when the CTA exits.
__device__ __forceinline__ void row_drain(const RowSmem& sm, unsigned cons, unsigned issued) {
  for (unsigned g = cons; g < issued; ++g) mbar_wait_bounded(&sm.bar[g % unsigned(sm.nslot)], (g / unsigned(sm.nslot)) & 1u);
}

}  // namespace
}  // namespace mht
