// Butterfly apply kernels for sm_103a (synthesis and its adjoint).
//
// The apply of a row-wise butterfly factorization (Sec. 2): synthesis multiplies by the
// leaf interpolation matrices V^* (stage 0), then by the transfer matrices R^* of levels
// l = 1..L, then by the column bases U; the adjoint runs U^H, R^H (l = L..1), V^H.  Every
// interpolation matrix is [I | T~] P^T, so a block applies as
//     synthesis  y_i = x[skel_i] + sum_j T~_ij x[rest_j]
//     adjoint    u[skel_i] = z_i,   u[rest_j] = sum_i conj(T~_ij) z_i
// and the column-basis stage is a dense block product.  Each stored matrix is read exactly
// once per apply (the paper's observation that apply cost equals storage, Sec. 6.2), so
// the single-RHS apply is bound by HBM bandwidth: the kernels stream each matrix with
// 128-bit non-allocating loads, gather the short input vector into shared memory, and
// reduce with warp shuffles.  The adjoint is a gather: the two sibling blocks (2p, nu),
// (2p+1, nu) that share an input pair write two separate buffers, and the next stage sums
// them while loading -- no atomics, deterministic results.
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

__device__ __forceinline__ uint4 ldg_stream(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

template <class R>
struct Vec16 {
  static constexpr int NS = 16 / sizeof(R);
  R s[NS];
};

template <class R>
__device__ __forceinline__ Vec16<R> load16(const R* p) {
  uint4 u = ldg_stream(p);
  Vec16<R> v;
  memcpy(&v, &u, 16);
  return v;
}

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// Synthesis, one work item = (block, rows [start, start+count)), RT right-hand sides.
//   ID stage (U_STAGE = false):  y[out_off + i] = x[idx[i]] + T~[i,:] . x[idx[r + :]]
//   U stage  (U_STAGE = true):   f[perm[out_off + i]] = U[i,:] . y_L[in_off + :]
// Element strides: input x[e * xs_e + k * xs_k], output y[e * ys_e + k * ys_k] (in elements;
// one complex value is one element).
template <class R, bool C, int RT, bool U_STAGE>
__global__ void __launch_bounds__(kThreads)
k_synth(const R* __restrict__ data, const int* __restrict__ idx, const MhtBlockDesc* __restrict__ desc,
        const MhtItem* __restrict__ items, const int* __restrict__ perm, const R* __restrict__ wts,
        const R* __restrict__ x, long long xs_e, long long xs_k,
        R* __restrict__ y, long long ys_e, long long ys_k, int nrhs) {
  constexpr int W = C ? 2 : 1;
  constexpr int NS = 16 / sizeof(R);
  constexpr int E = NS / W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* xs = reinterpret_cast<R*>(smem_raw);  // [RT][ldt][W], each RHS row 16-byte aligned

  const MhtItem it = items[blockIdx.x];
  const MhtBlockDesc d = desc[it.blk];
  const int k0 = blockIdx.y * RT;
  const int nk = min(RT, nrhs - k0);
  const int ldt = d.ldt;

  // gather the input columns of the matrix (zero padding up to ldt, and beyond nk)
  for (int j = threadIdx.x; j < ldt; j += kThreads) {
    long long src = -1;
    if (j < d.cols) src = U_STAGE ? (long long)(d.in_off + j) : (long long)idx[d.idx_off + d.rows + j];
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) {
        R v = R(0);
        if (src >= 0 && t < nk) v = x[(src * xs_e + (long long)(k0 + t) * xs_k) * W + c];
        xs[(t * ldt + j) * W + c] = v;
      }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec = ldt / E;
  for (int i = it.start + warp; i < it.start + it.count; i += kWarps) {
    R acc[RT][W];
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) acc[t][c] = R(0);
    const R* row = data + (d.t_off + (long long)i * ldt) * W;
#pragma unroll 4
    for (int v = lane; v < nvec; v += 32) {
      const Vec16<R> tv = load16(row + v * NS);
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        const Vec16<R> xv = *reinterpret_cast<const Vec16<R>*>(xs + (t * ldt + v * E) * W);
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
      if (U_STAGE) {
        dst = (long long)perm[d.out_off + i];
        if (wts) {
          const R w = wts[dst];
#pragma unroll
          for (int c = 0; c < W; ++c) val[c] *= w;
        }
      } else {
        const long long s = idx[d.idx_off + i];
#pragma unroll
        for (int c = 0; c < W; ++c) val[c] += x[(s * xs_e + (long long)(k0 + t) * xs_k) * W + c];
        dst = (long long)(d.out_off + i);
      }
#pragma unroll
      for (int c = 0; c < W; ++c) y[(dst * ys_e + (long long)(k0 + t) * ys_k) * W + c] = val[c];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Adjoint, one work item = (block, matrix columns [start, start+count)), RT RHS.
//   ID stage:  z_i = z0[out_off + i] (+ z1[out_off + i]);  out[idx[i]] = z_i (first item);
//              out[idx[r + j]] = sum_i conj(T~_ij) z_i;  out = sibling buffer `sib`
//   U stage:   g_i = w[perm[out_off + i]] f[perm[out_off + i]];
//              zL[in_off + j] = sum_i conj(U_ij) g_i
template <class R, bool C, int RT, bool U_STAGE>
__global__ void __launch_bounds__(kThreads)
k_adjoint(const R* __restrict__ data, const int* __restrict__ idx, const MhtBlockDesc* __restrict__ desc,
          const MhtItem* __restrict__ items, const int* __restrict__ perm, const R* __restrict__ wts,
          const R* __restrict__ z0, const R* __restrict__ z1, long long zs_e, long long zs_k,
          R* __restrict__ out0, R* __restrict__ out1, long long os_e, long long os_k, int nrhs) {
  constexpr int W = C ? 2 : 1;
  constexpr int NS = 16 / sizeof(R);
  constexpr int E = NS / W;
  constexpr int VPL = 2;                  // 16-byte vectors per lane per row
  constexpr int NCOL = 32 * E * VPL;      // columns per item
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* red = reinterpret_cast<R*>(smem_raw);                 // [kWarps][NCOL][RT][W]
  R* zs = red + kWarps * NCOL * RT * W;                    // [rows][RT][W]

  const MhtItem it = items[blockIdx.x];
  const MhtBlockDesc d = desc[it.blk];
  const int k0 = blockIdx.y * RT;
  const int nk = min(RT, nrhs - k0);
  R* out = it.sib ? out1 : out0;

  for (int i = threadIdx.x; i < d.rows; i += kThreads) {
    long long src;
    R w = R(1);
    if (U_STAGE) {
      src = perm[d.out_off + i];
      if (wts) w = wts[src];
    } else {
      src = d.out_off + i;
    }
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int c = 0; c < W; ++c) {
        R v = R(0);
        if (t < nk) {
          const long long a = (src * zs_e + (long long)(k0 + t) * zs_k) * W + c;
          v = z0[a];
          if (!U_STAGE && z1) v += z1[a];
          v *= w;
        }
        zs[(i * RT + t) * W + c] = v;
      }
  }
  __syncthreads();

  if (!U_STAGE && it.start == 0) {  // identity part of [I | T~] P^T
    for (int e = threadIdx.x; e < d.rows * nk; e += kThreads) {
      const int i = e / nk, t = e % nk;
      const long long dst = idx[d.idx_off + i];
#pragma unroll
      for (int c = 0; c < W; ++c) out[(dst * os_e + (long long)(k0 + t) * os_k) * W + c] = zs[(i * RT + t) * W + c];
    }
  }
  if (it.count == 0) return;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec = d.ldt / E;
  const int v0 = it.start / E;
  R acc[VPL][E][RT][W];
#pragma unroll
  for (int u = 0; u < VPL; ++u)
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int t = 0; t < RT; ++t)
#pragma unroll
        for (int c = 0; c < W; ++c) acc[u][e][t][c] = R(0);
#pragma unroll 2
  for (int i = warp; i < d.rows; i += kWarps) {
    const R* row = data + (d.t_off + (long long)i * d.ldt) * W;
    Vec16<R> tv[VPL];
#pragma unroll
    for (int u = 0; u < VPL; ++u) {
      const int v = v0 + lane + 32 * u;
      if (v < nvec) tv[u] = load16(row + v * NS);
      else
#pragma unroll
        for (int q = 0; q < NS; ++q) tv[u].s[q] = R(0);
    }
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      R zr = zs[(i * RT + t) * W], zi = C ? zs[(i * RT + t) * W + W - 1] : R(0);
#pragma unroll
      for (int u = 0; u < VPL; ++u)
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (C) {  // conj(a + ib) (zr + i zi)
            const R a = tv[u].s[2 * e], b = tv[u].s[2 * e + 1];
            acc[u][e][t][0] += a * zr + b * zi;
            acc[u][e][t][W - 1] += a * zi - b * zr;
          } else {
            acc[u][e][t][0] += tv[u].s[e] * zr;
          }
        }
    }
  }
#pragma unroll
  for (int u = 0; u < VPL; ++u)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int col = (lane + 32 * u) * E + e;
#pragma unroll
      for (int t = 0; t < RT; ++t)
#pragma unroll
        for (int c = 0; c < W; ++c) red[((warp * NCOL + col) * RT + t) * W + c] = acc[u][e][t][c];
    }
  __syncthreads();
  for (int e = threadIdx.x; e < it.count * nk; e += kThreads) {
    const int col = e / nk, t = e % nk;
    const int j = it.start + col;
    R s[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      s[c] = R(0);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s[c] += red[((w * NCOL + col) * RT + t) * W + c];
    }
    const long long dst = U_STAGE ? (long long)(d.in_off + j) : (long long)idx[d.idx_off + d.rows + j];
#pragma unroll
    for (int c = 0; c < W; ++c) out[(dst * os_e + (long long)(k0 + t) * os_k) * W + c] = s[c];
  }
}

// ---------------------------------------------------------------------------------------
}  // namespace

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

struct StageTimer {  // records events around one launch when profiling is enabled
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

template <class R>
const R* data_ptr(const Ctx& c) { return reinterpret_cast<const R*>(c.d.base + c.P.data_off); }
const int* idx_ptr(const Ctx& c) { return reinterpret_cast<const int*>(c.d.base + c.P.index_off); }
const int* perm_ptr(const Ctx& c) { return reinterpret_cast<const int*>(c.d.base + c.P.perm_off); }
const MhtBlockDesc* desc_ptr(const Ctx& c, int s) {
  return reinterpret_cast<const MhtBlockDesc*>(c.d.base + c.P.st[s].desc_off);
}
const MhtItem* items_ptr(const Ctx& c, int s, bool syn) {
  return reinterpret_cast<const MhtItem*>(c.d.base + (syn ? c.P.st[s].items_syn_off : c.P.st[s].items_adj_off));
}

int check(cudaError_t e, std::string& err, const char* what) {
  if (e == cudaSuccess) return 0;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return MHT_ERR_CUDA;
}


template <class R, bool C, int RT, bool U>
int launch_synth(const Ctx& c, int s, const void* x, long long xs_e, long long xs_k, void* y,
                 long long ys_e, long long ys_k, const void* w = nullptr) {
  const Stage& S = c.P.st[s];
  if (S.nitems_syn == 0) return 0;
  constexpr int W = C ? 2 : 1;
  int64_t maxldt = 0;
  {
    constexpr int E = 16 / sizeof(R) / W;
    maxldt = (S.max_cols + E - 1) / E * E;
  }
  const size_t smem = size_t(std::max<int64_t>(maxldt, 1)) * RT * W * sizeof(R);
  auto kern = k_synth<R, C, RT, U>;
  if (smem > 227 * 1024) {
    c.err = "synthesis stage needs too much shared memory for this RHS tile";
    return MHT_ERR_UNSUPPORTED;
  }
  if (smem > 48 * 1024) {
    if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), c.err, "smem attr")) return rc;
  }
  dim3 grid(unsigned(S.nitems_syn), unsigned((c.nrhs + RT - 1) / RT));
  StageTimer timer(c.d.prof, 0, s, c.s);
  kern<<<grid, kThreads, smem, c.s>>>(data_ptr<R>(c), idx_ptr(c), desc_ptr(c, s), items_ptr(c, s, true), perm_ptr(c),
                                      static_cast<const R*>(w), static_cast<const R*>(x), xs_e, xs_k,
                                      static_cast<R*>(y), ys_e, ys_k,
                                      int(c.nrhs));
  return check(cudaGetLastError(), c.err, "synthesis launch");
}

template <class R, bool C, int RT, bool U>
int launch_adjoint(const Ctx& c, int s, const void* z0, const void* z1, long long zs_e, long long zs_k,
                   void* o0, void* o1, long long os_e, long long os_k, const void* w) {
  const Stage& S = c.P.st[s];
  if (S.nitems_adj == 0) return 0;
  constexpr int W = C ? 2 : 1;
  constexpr int E = 16 / sizeof(R) / W;
  constexpr int NCOL = 32 * E * 2;
  const size_t smem = (size_t(kWarps) * NCOL * RT * W + size_t(std::max<int64_t>(S.max_rows, 1)) * RT * W) * sizeof(R);
  auto kern = k_adjoint<R, C, RT, U>;
  if (smem > 227 * 1024) {
    c.err = "adjoint stage needs too much shared memory for this RHS tile";
    return MHT_ERR_UNSUPPORTED;
  }
  if (smem > 48 * 1024) {
    if (int rc = check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), c.err, "smem attr")) return rc;
  }
  dim3 grid(unsigned(S.nitems_adj), unsigned((c.nrhs + RT - 1) / RT));
  StageTimer timer(c.d.prof, 1, s, c.s);
  kern<<<grid, kThreads, smem, c.s>>>(data_ptr<R>(c), idx_ptr(c), desc_ptr(c, s), items_ptr(c, s, false), perm_ptr(c),
                                      static_cast<const R*>(w), static_cast<const R*>(z0), static_cast<const R*>(z1),
                                      zs_e, zs_k, static_cast<R*>(o0), static_cast<R*>(o1), os_e, os_k, int(c.nrhs));
  return check(cudaGetLastError(), c.err, "adjoint launch");
}

size_t vec_bytes(const Ctx& c) {
  return (size_t(std::max<int64_t>(c.P.vec_entries, 1)) * c.d.max_nrhs * c.P.elem_bytes + 255) / 256 * 256;
}
void* wsbuf(const Ctx& c, int i) { return c.d.ws + i * vec_bytes(c); }

template <class R, bool C, int RT>
int synth_impl(const Ctx& c, const void* cin, int64_t ldc, void* f, int64_t ldf, bool weighted) {
  const int L = c.F.L;
  const long long nr = c.nrhs;
  int cur = 0;
  int rc = launch_synth<R, C, RT, false>(c, 0, cin, 1, ldc, wsbuf(c, cur), nr, 1);
  if (rc) return rc;
  for (int l = 1; l <= L; ++l) {
    rc = launch_synth<R, C, RT, false>(c, l, wsbuf(c, cur), nr, 1, wsbuf(c, 1 - cur), nr, 1);
    if (rc) return rc;
    cur = 1 - cur;
  }
  const void* w = weighted ? (const void*)(c.d.base + c.P.weights_off) : nullptr;
  return launch_synth<R, C, RT, true>(c, L + 1, wsbuf(c, cur), nr, 1, f, 1, ldf, w);
}

template <class R, bool C, int RT>
int adjoint_impl(const Ctx& c, const void* f, int64_t ldf, void* cout, int64_t ldc, bool weighted) {
  const int L = c.F.L;
  const long long nr = c.nrhs;
  const void* w = weighted ? (const void*)(c.d.base + c.P.weights_off) : nullptr;
  // U^H: f -> z_L (buffer 0)
  int rc = launch_adjoint<R, C, RT, true>(c, L + 1, f, nullptr, 1, ldf, wsbuf(c, 0), wsbuf(c, 0), nr, 1, w);
  if (rc) return rc;
  const void* z0 = wsbuf(c, 0);
  const void* z1 = nullptr;
  int pair = 0;  // output pairs alternate (1,2) and (3,0)
  for (int l = L; l >= 1; --l) {
    void* o0 = wsbuf(c, pair == 0 ? 1 : 3);
    void* o1 = wsbuf(c, pair == 0 ? 2 : 0);
    rc = launch_adjoint<R, C, RT, false>(c, l, z0, z1, nr, 1, o0, o1, nr, 1, nullptr);
    if (rc) return rc;
    z0 = o0;
    z1 = o1;
    pair = 1 - pair;
  }
  return launch_adjoint<R, C, RT, false>(c, 0, z0, z1, nr, 1, cout, cout, 1, ldc, nullptr);
}

// Largest RHS tile (8, 4, 2, 1) whose shared memory fits every stage.
template <class R, bool C>
int pick_rt(const Ctx& c, bool synth) {
  constexpr int W = C ? 2 : 1;
  constexpr int E = 16 / sizeof(R) / W;
  constexpr int NCOL = 32 * E * 2;
  int64_t maxcols = 1, maxrows = 1;
  for (const Stage& s : c.P.st) {
    maxcols = std::max<int64_t>(maxcols, (s.max_cols + E - 1) / E * E);
    maxrows = std::max<int64_t>(maxrows, s.max_rows);
  }
  for (int rt = 8; rt >= 1; rt /= 2) {
    if (rt > 1 && c.nrhs < rt) continue;
    const size_t need = synth ? size_t(maxcols) * rt * W * sizeof(R)
                              : (size_t(kWarps) * NCOL + size_t(maxrows)) * rt * W * sizeof(R);
    if (need <= 227 * 1024) return rt;
  }
  return 1;
}

template <class R, bool C>
int synth_dispatch(const Ctx& c, const void* cin, int64_t ldc, void* f, int64_t ldf, bool wt) {
  switch (pick_rt<R, C>(c, true)) {
    case 8: return synth_impl<R, C, 8>(c, cin, ldc, f, ldf, wt);
    case 4: return synth_impl<R, C, 4>(c, cin, ldc, f, ldf, wt);
    case 2: return synth_impl<R, C, 2>(c, cin, ldc, f, ldf, wt);
    default: return synth_impl<R, C, 1>(c, cin, ldc, f, ldf, wt);
  }
}
template <class R, bool C>
int adjoint_dispatch(const Ctx& c, const void* f, int64_t ldf, void* cout, int64_t ldc, bool wt) {
  switch (pick_rt<R, C>(c, false)) {
    case 8: return adjoint_impl<R, C, 8>(c, f, ldf, cout, ldc, wt);
    case 4: return adjoint_impl<R, C, 4>(c, f, ldf, cout, ldc, wt);
    case 2: return adjoint_impl<R, C, 2>(c, f, ldf, cout, ldc, wt);
    default: return adjoint_impl<R, C, 1>(c, f, ldf, cout, ldc, wt);
  }
}


}  // namespace

int apply_synthesize(const Factorization& F, const Packed& P, const DeviceView& d, const void* c,
                     int64_t ldc, void* f, int64_t ldf, int64_t nrhs, bool wt, mht_apply_mode mode,
                     void* stream, std::string& err) {
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err};
  (void)mode;
  if (P.fp64) return P.cplx ? synth_dispatch<double, true>(x, c, ldc, f, ldf, wt) : synth_dispatch<double, false>(x, c, ldc, f, ldf, wt);
  return P.cplx ? synth_dispatch<float, true>(x, c, ldc, f, ldf, wt) : synth_dispatch<float, false>(x, c, ldc, f, ldf, wt);
}

int apply_analyze(const Factorization& F, const Packed& P, const DeviceView& d, const void* f,
                  int64_t ldf, void* c, int64_t ldc, int64_t nrhs, bool weighted,
                  mht_apply_mode mode, void* stream, std::string& err) {
  Ctx x{F, P, d, static_cast<cudaStream_t>(stream), nrhs, err};
  (void)mode;
  if (P.fp64) return P.cplx ? adjoint_dispatch<double, true>(x, f, ldf, c, ldc, weighted) : adjoint_dispatch<double, false>(x, f, ldf, c, ldc, weighted);
  return P.cplx ? adjoint_dispatch<float, true>(x, f, ldf, c, ldc, weighted) : adjoint_dispatch<float, false>(x, f, ldf, c, ldc, weighted);
}

int64_t apply_launches(const Packed& P, int64_t nrhs, mht_apply_mode mode) {
  (void)mode;
  (void)nrhs;
  int64_t n = 0;
  for (const Stage& s : P.st) n += (s.nitems_syn > 0) ? 1 : 0;
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

}  // namespace mht
