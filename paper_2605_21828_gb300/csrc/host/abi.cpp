// extern "C" entry points of libmht (declared in include/mht.h).
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>

#include "internal.h"

namespace mht {
namespace {
std::atomic<size_t> g_alloc_limit{0};
}
size_t host_alloc_limit() { return g_alloc_limit.load(); }
void set_host_alloc_limit(size_t bytes) { g_alloc_limit.store(bytes); }
}  // namespace mht

namespace {

thread_local std::string g_last_error;

mht_status set_error(mht_status s, const std::string& m) {
  g_last_error = m;
  return s;
}

template <class Fn>
mht_status guarded(Fn&& fn) {
  try {
    g_last_error.clear();
    return fn();
  } catch (const mht::Error& e) {
    return set_error(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return set_error(MHT_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(MHT_ERR_INVALID_ARG, e.what());
  }
}

bool fp64_mode(mht_apply_mode m) { return m == MHT_APPLY_FP64; }

void check_mode(mht_apply_mode m) {
  if (m != MHT_APPLY_FP64 && m != MHT_APPLY_FP32 && m != MHT_APPLY_3XTF32 && m != MHT_APPLY_6XBF16)
    mht::fail(MHT_ERR_INVALID_ARG, "bad apply mode");
}

// ---- plan file: magic, version, header, arrays, FNV-1a 64 checksum ---------------------
constexpr uint64_t kMagic = 0x3130544854464d42ull;  // "BMFTHT01"
constexpr uint32_t kVersion = 1;

struct Writer {
  std::vector<uint8_t> buf;
  template <class T> void pod(const T& v) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
    buf.insert(buf.end(), p, p + sizeof(T));
  }
  template <class T> void vec(const std::vector<T>& v) {
    pod<uint64_t>(v.size());
    const uint8_t* p = reinterpret_cast<const uint8_t*>(v.data());
    buf.insert(buf.end(), p, p + v.size() * sizeof(T));
  }
};

struct Reader {
  const uint8_t* p;
  size_t n, at = 0;
  template <class T> T pod() {
    if (at + sizeof(T) > n) mht::fail(MHT_ERR_FORMAT, "truncated plan file");
    T v;
    std::memcpy(&v, p + at, sizeof(T));
    at += sizeof(T);
    return v;
  }
  template <class T> void vec(std::vector<T>& v, uint64_t maxn) {
    const uint64_t k = pod<uint64_t>();
    if (k > maxn || at + k * sizeof(T) > n) mht::fail(MHT_ERR_FORMAT, "corrupt array length in plan file");
    v.resize(k);
    std::memcpy(v.data(), p + at, k * sizeof(T));
    at += k * sizeof(T);
  }
};

uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

extern "C" {

const char* mht_last_error(void) { return g_last_error.c_str(); }
const char* mht_version(void) { return "mht 0.1 (sm_103a)"; }

mht_status mht_build_plan(const mht_problem* problem, const mht_options* options, mht_plan** out) {
  return guarded([&]() -> mht_status {
    if (!problem || !options || !out) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    check_mode(options->mode);
    if (options->num_threads > 0) omp_set_num_threads(options->num_threads);
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<mht_plan> plan(new mht_plan());
    mht::build_factorization(*problem, *options, plan->F);
    plan->mode = options->mode;
    plan->eps = options->eps;
    mht::pack(plan->F, fp64_mode(options->mode), plan->P);
    plan->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = plan.release();
    return MHT_OK;
  });
}

mht_status mht_problem_eval(const mht_problem* problem, const int64_t* rows, int64_t nrows, const int64_t* cols,
                            int64_t ncols, double* out) {
  return guarded([&]() -> mht_status {
    if (!problem || nrows < 0 || ncols < 0) mht::fail(MHT_ERR_INVALID_ARG, "bad argument");
    if (nrows == 0 || ncols == 0) return MHT_OK;
    if (!rows || !cols || !out) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    for (int64_t i = 0; i < nrows; ++i)
      if (rows[i] < 0 || rows[i] >= problem->n) mht::fail(MHT_ERR_INVALID_ARG, "row index out of range");
    for (int64_t j = 0; j < ncols; ++j)
      if (cols[j] < 0 || cols[j] >= problem->m) mht::fail(MHT_ERR_INVALID_ARG, "column index out of range");
    std::unique_ptr<mht::Evaluator> ev(mht::make_evaluator(*problem));
    ev->eval(rows, nrows, cols, ncols, out);
    return MHT_OK;
  });
}

mht_status mht_plan_import(const mht_factors* factors, const mht_options* options, mht_plan** out) {
  return guarded([&]() -> mht_status {
    if (!factors || !options || !out) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    check_mode(options->mode);
    std::unique_ptr<mht_plan> plan(new mht_plan());
    mht::import_factors(*factors, plan->F);
    plan->mode = options->mode;
    plan->eps = options->eps;
    mht::pack(plan->F, fp64_mode(options->mode), plan->P);
    *out = plan.release();
    return MHT_OK;
  });
}

mht_status mht_plan_clone(const mht_plan* src, const mht_options* options, mht_plan** out) {
  return guarded([&]() -> mht_status {
    if (!src || !options || !out) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    check_mode(options->mode);
    std::unique_ptr<mht_plan> plan(new mht_plan());
    plan->F = src->F;
    plan->mode = options->mode;
    plan->eps = src->eps;
    plan->build_seconds = src->build_seconds;
    mht::pack(plan->F, fp64_mode(options->mode), plan->P);
    *out = plan.release();
    return MHT_OK;
  });
}

mht_status mht_plan_export(const mht_plan* plan, mht_factors* fa) {
  return guarded([&]() -> mht_status {
    if (!plan || !fa) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    const mht::Factorization& F = plan->F;
    fa->n = F.n; fa->m = F.m; fa->levels = F.L; fa->field = F.cplx ? MHT_COMPLEX : MHT_REAL;
    const int64_t nb = F.nblk();
    if (fa->space_perm) std::copy(F.space_perm.begin(), F.space_perm.end(), fa->space_perm);
    if (fa->space_offsets) std::copy(F.space_off.begin(), F.space_off.end(), fa->space_offsets);
    if (fa->mode_perm) std::copy(F.mode_perm.begin(), F.mode_perm.end(), fa->mode_perm);
    if (fa->mode_offsets) std::copy(F.mode_off.begin(), F.mode_off.end(), fa->mode_offsets);
    int64_t pp = 0, tp = 0;
    for (int l = 0; l <= F.L; ++l)
      for (int64_t b = 0; b < nb; ++b) {
        const mht::Block& B = F.lv[l][b];
        if (fa->ranks) fa->ranks[l * nb + b] = B.r;
        if (fa->local_perm) std::copy(B.perm.begin(), B.perm.end(), fa->local_perm + pp);
        if (fa->transfer) std::copy(B.T.begin(), B.T.end(), fa->transfer + tp);
        pp += B.K;
        tp += int64_t(B.T.size());
      }
    int64_t up = 0;
    for (int64_t t = 0; t < nb; ++t) {
      if (fa->column_bases) std::copy(F.U[t].begin(), F.U[t].end(), fa->column_bases + up);
      up += int64_t(F.U[t].size());
    }
    if (fa->weights && !F.weights.empty()) std::copy(F.weights.begin(), F.weights.end(), fa->weights);
    return MHT_OK;
  });
}

mht_status mht_plan_info(const mht_plan* plan, mht_plan_info_t* info) {
  return guarded([&]() -> mht_status {
    if (!plan || !info) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    const mht::Factorization& F = plan->F;
    const mht::Packed& P = plan->P;
    std::memset(info, 0, sizeof(*info));
    info->n = F.n; info->m = F.m; info->levels = F.L;
    info->field = F.cplx ? MHT_COMPLEX : MHT_REAL;
    info->mode = plan->mode;
    info->eps = plan->eps;
    info->blocks_per_level = F.nblk();
    int64_t maxr = 0;
    for (auto& lvl : F.lv)
      for (auto& B : lvl) {
        info->local_perm_entries += B.K;
        info->transfer_entries += int64_t(B.r) * (B.K - B.r);
        maxr = std::max<int64_t>(maxr, B.r);
      }
    for (int64_t t = 0; t < F.nblk(); ++t) info->column_basis_entries += F.leaf_rows(t) * F.lv[F.L][t].r;
    info->stored_entries = info->transfer_entries + info->column_basis_entries;
    info->max_rank = maxr;
    info->workspace_entries_per_rhs = P.vec_entries;
    info->factor_bytes = P.image.size();
    const size_t es = size_t(P.elem_bytes);
    size_t descs = 0;
    for (const auto& s : P.st) descs += size_t(s.nblocks) * sizeof(MhtBlockDesc);
    info->algorithmic_bytes = size_t(info->stored_entries) * es + size_t(P.index_entries) * 4 + descs +
                              size_t(F.n) * 4 + size_t(F.n + F.m) * es;
    info->build_seconds = plan->build_seconds;
    return MHT_OK;
  });
}

mht_status mht_plan_level_info(const mht_plan* plan, int32_t level, mht_level_info_t* info) {
  return guarded([&]() -> mht_status {
    if (!plan || !info) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    const mht::Factorization& F = plan->F;
    if (level < 0 || level > F.L + 1) mht::fail(MHT_ERR_INVALID_ARG, "level out of range");
    std::memset(info, 0, sizeof(*info));
    std::vector<int64_t> r;
    const int L = F.L;
    for (int64_t b = 0; b < F.nblk(); ++b) r.push_back(level <= L ? F.lv[level][b].r : F.lv[L][b].r);
    std::sort(r.begin(), r.end());
    info->rank_min = r.front();
    info->rank_max = r.back();
    info->rank_median = r[r.size() / 2];
    for (int64_t v : r) info->rank_sum += v;
    info->transfer_entries = plan->P.st[level].t_entries;
    info->bytes = plan->P.st[level].dir[0].data_bytes + plan->P.st[level].dir[1].data_bytes;
    info->algorithmic_bytes = plan->P.st[level].alg_bytes;
    return MHT_OK;
  });
}

mht_status mht_plan_device_bytes(const mht_plan* plan, int64_t max_nrhs, size_t* factor_bytes,
                                 size_t* workspace_bytes) {
  return guarded([&]() -> mht_status {
    if (!plan || !factor_bytes || !workspace_bytes || max_nrhs < 1) mht::fail(MHT_ERR_INVALID_ARG, "bad argument");
    *factor_bytes = plan->P.image.size();
    *workspace_bytes = plan->P.workspace_bytes(max_nrhs, plan->F.n, plan->F.m);
    return MHT_OK;
  });
}

mht_status mht_plan_bind_device(mht_plan* plan, void* factor_dev, size_t factor_bytes, void* workspace_dev,
                                size_t workspace_bytes, int64_t max_nrhs, void* stream) {
  return guarded([&]() -> mht_status {
    if (!plan || !factor_dev || !workspace_dev || max_nrhs < 1) mht::fail(MHT_ERR_INVALID_ARG, "NULL buffer or bad max_nrhs");
    if ((reinterpret_cast<uintptr_t>(factor_dev) | reinterpret_cast<uintptr_t>(workspace_dev)) & 255)
      mht::fail(MHT_ERR_INVALID_ARG, "device buffers must be 256-byte aligned");
    if (factor_bytes < plan->P.image.size()) mht::fail(MHT_ERR_OOM, "factor buffer too small");
    if (workspace_bytes < plan->P.workspace_bytes(max_nrhs, plan->F.n, plan->F.m))
      mht::fail(MHT_ERR_OOM, "workspace buffer too small for max_nrhs");
    std::string err;
    plan->bound = false;
    if (int rc = mht::device_upload_image(plan->P, factor_dev, stream, err)) return set_error(mht_status(rc), err);
    plan->dev.base = static_cast<const uint8_t*>(factor_dev);
    plan->dev.ws = static_cast<uint8_t*>(workspace_dev);
    plan->dev.ws_bytes = workspace_bytes;
    plan->dev.max_nrhs = max_nrhs;
    unsigned flags = 0;
    if (int rc = mht::device_status(plan->dev.ws + plan->P.status_offset(max_nrhs, plan->F.n, plan->F.m), stream,
                                    &flags, err))
      return set_error(mht_status(rc), err);
    plan->bound = true;
    return MHT_OK;
  });
}

static void check_apply(const mht_plan* plan, const void* a, int64_t lda, int64_t rows_a, const void* b, int64_t ldb,
                        int64_t rows_b, int64_t nrhs) {
  if (!plan) mht::fail(MHT_ERR_INVALID_ARG, "NULL plan");
  if (!plan->bound) mht::fail(MHT_ERR_NOT_BOUND, "plan has no bound device buffers");
  if (!a || !b) mht::fail(MHT_ERR_INVALID_ARG, "NULL vector");
  if (nrhs < 1 || nrhs > plan->dev.max_nrhs) mht::fail(MHT_ERR_INVALID_ARG, "nrhs outside [1, bound max_nrhs]");
  if (lda < rows_a || ldb < rows_b) mht::fail(MHT_ERR_INVALID_ARG, "leading dimension too small");
}

mht_status mht_synthesize(mht_plan* plan, const void* c_dev, int64_t ldc, void* f_dev, int64_t ldf, int64_t nrhs,
                          void* stream) {
  return guarded([&]() -> mht_status {
    check_apply(plan, c_dev, ldc, plan ? plan->F.m : 0, f_dev, ldf, plan ? plan->F.n : 0, nrhs);
    std::string err;
    int rc = mht::apply_synthesize(plan->F, plan->P, plan->dev, c_dev, ldc, f_dev, ldf, nrhs, false, plan->mode,
                                   stream, err);
    return rc ? set_error(mht_status(rc), err) : MHT_OK;
  });
}

mht_status mht_synthesize_scaled(mht_plan* plan, const void* c_dev, int64_t ldc, const void* scale_dev, void* f_dev,
                                 int64_t ldf, int64_t nrhs, void* stream) {
  return guarded([&]() -> mht_status {
    check_apply(plan, c_dev, ldc, plan ? plan->F.m : 0, f_dev, ldf, plan ? plan->F.n : 0, nrhs);
    if (!scale_dev) mht::fail(MHT_ERR_INVALID_ARG, "NULL scale");
    std::string err;
    int rc = mht::apply_synthesize(plan->F, plan->P, plan->dev, c_dev, ldc, f_dev, ldf, nrhs, false, plan->mode, stream,
                                   err, scale_dev);
    if (rc) mht::fail(mht_status(rc), err);
    return MHT_OK;
  });
}

mht_status mht_filter(mht_plan* plan, const void* f_in_dev, int64_t ldi, void* f_out_dev, int64_t ldo, int64_t nrhs,
                      const void* filter_dev, int32_t weighted, void* stream) {
  return guarded([&]() -> mht_status {
    check_apply(plan, f_in_dev, ldi, plan ? plan->F.n : 0, f_out_dev, ldo, plan ? plan->F.n : 0, nrhs);
    if (!filter_dev) mht::fail(MHT_ERR_INVALID_ARG, "NULL filter");
    if (f_in_dev == f_out_dev) mht::fail(MHT_ERR_INVALID_ARG, "f_in and f_out must not alias");
    std::string err;
    int rc = mht::apply_filter(plan->F, plan->P, plan->dev, f_in_dev, ldi, f_out_dev, ldo, nrhs, filter_dev,
                               weighted != 0, plan->mode, stream, err);
    if (rc) mht::fail(mht_status(rc), err);
    return MHT_OK;
  });
}

mht_status mht_lsqr_scratch_bytes(const mht_plan* plan, int64_t nrhs, size_t* bytes) {
  return guarded([&]() -> mht_status {
    if (!plan || !bytes || nrhs < 1) mht::fail(MHT_ERR_INVALID_ARG, "bad argument");
    *bytes = mht::lsqr_scratch_bytes(plan->P, plan->F.n, plan->F.m, nrhs);
    return MHT_OK;
  });
}

mht_status mht_inverse_lsqr(mht_plan* plan, const void* f_dev, int64_t ldf, void* c_dev, int64_t ldc, int64_t nrhs,
                            void* scratch_dev, size_t scratch_bytes, int32_t max_iter, double tol, void* stream,
                            int32_t* iters, double* relres) {
  return guarded([&]() -> mht_status {
    check_apply(plan, f_dev, ldf, plan ? plan->F.n : 0, c_dev, ldc, plan ? plan->F.m : 0, nrhs);
    if (!scratch_dev || scratch_bytes < mht::lsqr_scratch_bytes(plan->P, plan->F.n, plan->F.m, nrhs))
      mht::fail(MHT_ERR_INVALID_ARG, "scratch smaller than mht_lsqr_scratch_bytes");
    if (reinterpret_cast<uintptr_t>(scratch_dev) & 255) mht::fail(MHT_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    if (max_iter < 0 || !(tol >= 0)) mht::fail(MHT_ERR_INVALID_ARG, "bad iteration limit or tolerance");
    std::string err;
    int it = 0;
    double rr = 0;
    int rc = mht::apply_lsqr(plan->F, plan->P, plan->dev, f_dev, ldf, c_dev, ldc, nrhs, scratch_dev, max_iter, tol,
                             plan->mode, stream, &it, &rr, err);
    if (rc) mht::fail(mht_status(rc), err);
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return MHT_OK;
  });
}

mht_status mht_synthesize_weighted(mht_plan* plan, const void* c_dev, int64_t ldc, void* f_dev, int64_t ldf,
                                   int64_t nrhs, void* stream) {
  return guarded([&]() -> mht_status {
    check_apply(plan, c_dev, ldc, plan ? plan->F.m : 0, f_dev, ldf, plan ? plan->F.n : 0, nrhs);
    std::string err;
    int rc = mht::apply_synthesize(plan->F, plan->P, plan->dev, c_dev, ldc, f_dev, ldf, nrhs, true, plan->mode,
                                   stream, err);
    return rc ? set_error(mht_status(rc), err) : MHT_OK;
  });
}

mht_status mht_analyze(mht_plan* plan, const void* f_dev, int64_t ldf, void* c_dev, int64_t ldc, int64_t nrhs,
                       int32_t weighted, void* stream) {
  return guarded([&]() -> mht_status {
    check_apply(plan, f_dev, ldf, plan ? plan->F.n : 0, c_dev, ldc, plan ? plan->F.m : 0, nrhs);
    std::string err;
    int rc = mht::apply_analyze(plan->F, plan->P, plan->dev, f_dev, ldf, c_dev, ldc, nrhs, weighted != 0, plan->mode,
                                stream, err);
    return rc ? set_error(mht_status(rc), err) : MHT_OK;
  });
}

static void* staging(mht_plan* plan, int which) {
  const mht::Packed& P = plan->P;
  const size_t sc = (size_t(plan->F.m) * plan->dev.max_nrhs * P.elem_bytes + 255) / 256 * 256;
  return plan->dev.ws + 3 * P.ws_vec_bytes(plan->dev.max_nrhs) + (which == 0 ? 0 : sc);
}

static mht_status host_transform(mht_plan* plan, bool synth, const void* in, int64_t ldi, void* out, int64_t ldo,
                                 int64_t nrhs, bool weighted, void* stream) {
  const int64_t nin = synth ? plan->F.m : plan->F.n, nout = synth ? plan->F.n : plan->F.m;
  check_apply(plan, in, ldi, nin, out, ldo, nout, nrhs);
  const size_t es = size_t(plan->P.elem_bytes);
  uint8_t* din = static_cast<uint8_t*>(staging(plan, synth ? 0 : 1));
  uint8_t* dout = static_cast<uint8_t*>(staging(plan, synth ? 1 : 0));
  std::string err;
  int rc = 0;
  for (int64_t k = 0; k < nrhs && !rc; ++k)
    rc = mht::device_copy_async(din + size_t(k * nin) * es, static_cast<const uint8_t*>(in) + size_t(k * ldi) * es,
                                size_t(nin) * es, 0, stream, err);
  if (!rc)
    rc = synth ? mht::apply_synthesize(plan->F, plan->P, plan->dev, din, nin, dout, nout, nrhs, false, plan->mode,
                                       stream, err)
               : mht::apply_analyze(plan->F, plan->P, plan->dev, din, nin, dout, nout, nrhs, weighted, plan->mode,
                                    stream, err);
  for (int64_t k = 0; k < nrhs && !rc; ++k)
    rc = mht::device_copy_async(static_cast<uint8_t*>(out) + size_t(k * ldo) * es, dout + size_t(k * nout) * es,
                                size_t(nout) * es, 1, stream, err);
  if (!rc) rc = mht::device_sync(stream, err);
  return rc ? set_error(mht_status(rc), err) : MHT_OK;
}

mht_status mht_synthesize_host(mht_plan* plan, const void* c_host, int64_t ldc, void* f_host, int64_t ldf,
                               int64_t nrhs, void* stream) {
  return guarded([&]() { return host_transform(plan, true, c_host, ldc, f_host, ldf, nrhs, false, stream); });
}

mht_status mht_analyze_host(mht_plan* plan, const void* f_host, int64_t ldf, void* c_host, int64_t ldc, int64_t nrhs,
                            int32_t weighted, void* stream) {
  return guarded([&]() { return host_transform(plan, false, f_host, ldf, c_host, ldc, nrhs, weighted != 0, stream); });
}

mht_status mht_apply_launch_count(const mht_plan* plan, int64_t nrhs, int64_t* launches) {
  return guarded([&]() -> mht_status {
    if (!plan || !launches || nrhs < 1) mht::fail(MHT_ERR_INVALID_ARG, "bad argument");
    *launches = mht::apply_launches(plan->P, nrhs, plan->mode, plan->dev.path);
    return MHT_OK;
  });
}

mht_status mht_synthesize_noalloc(const mht_plan* plan, const void* factor_dev, const void* c_dev, void* f_dev,
                                  void* stream) {
  return guarded([&]() -> mht_status {
    if (!plan || !factor_dev || !c_dev || !f_dev) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(factor_dev) & 255) mht::fail(MHT_ERR_INVALID_ARG, "factor_dev must be 256-byte aligned");
    std::string err;
    int rc = mht::apply_synthesize_noalloc(plan->P, factor_dev, c_dev, f_dev, stream, err);
    return rc ? set_error(mht_status(rc), err) : MHT_OK;
  });
}

mht_status mht_debug_host_alloc_limit(size_t bytes) {
  mht::set_host_alloc_limit(bytes);
  return MHT_OK;
}

mht_status mht_noalloc_check(void* stream, int32_t* flags) {
  return guarded([&]() -> mht_status {
    if (!flags) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    std::string err;
    unsigned f = 0;
    if (int rc = mht::noalloc_status(stream, &f, err)) return set_error(mht_status(rc), err);
    *flags = int32_t(f);
    if (f) return set_error(MHT_ERR_TIMEOUT, "a bounded device wait of the no-alloc synthesis gave up (status flags " +
                                                 std::to_string(f) + ")");
    return MHT_OK;
  });
}

mht_status mht_noalloc_debug_hold(const mht_plan* plan, void* factor_dev, int32_t hold, void* stream) {
  return guarded([&]() -> mht_status {
    if (!plan || !factor_dev) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    if (plan->P.fp64 || plan->P.cplx) mht::fail(MHT_ERR_UNSUPPORTED, "the no-alloc synthesis serves real FP32 plans");
    if (plan->P.fused[0].nitems == 0) mht::fail(MHT_ERR_INVALID_ARG, "the plan has no synthesis work items");
    std::string err;
    if (int rc = mht::noalloc_debug_hold(plan->P, factor_dev, hold != 0, stream, err))
      return set_error(mht_status(rc), err);
    return MHT_OK;
  });
}

mht_status mht_plan_check(mht_plan* plan, void* stream, int32_t* flags) {
  return guarded([&]() -> mht_status {
    if (!plan || !flags) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    if (!plan->bound) mht::fail(MHT_ERR_NOT_BOUND, "plan has no bound device buffers");
    std::string err;
    unsigned f = 0;
    int rc = mht::device_status(plan->dev.ws + plan->P.status_offset(plan->dev.max_nrhs, plan->F.n, plan->F.m), stream,
                                &f, err);
    if (rc) return set_error(mht_status(rc), err);
    *flags = int32_t(f);
    if (f) return set_error(MHT_ERR_TIMEOUT, "a bounded device wait gave up (status flags " + std::to_string(f) + ")");
    return MHT_OK;
  });
}

mht_status mht_plan_set_path(mht_plan* plan, int32_t path) {
  return guarded([&]() -> mht_status {
    if (!plan || path < 0 || path > 2) mht::fail(MHT_ERR_INVALID_ARG, "bad plan or path");
    plan->dev.path = path;
    return MHT_OK;
  });
}

mht_status mht_plan_set_mode(mht_plan* plan, mht_apply_mode mode) {
  return guarded([&]() -> mht_status {
    if (!plan) mht::fail(MHT_ERR_INVALID_ARG, "NULL plan");
    if (plan->P.fp64 || (mode != MHT_APPLY_FP32 && !mht::tensor_mode(mode)))
      mht::fail(MHT_ERR_INVALID_ARG, "set_mode switches only between FP32, 3XTF32 and 6XBF16 on a float plan");
    plan->mode = mode;
    return MHT_OK;
  });
}

mht_status mht_plan_autotune(mht_plan* plan, int64_t nrhs, void* stream) {
  return guarded([&]() -> mht_status {
    if (!plan) mht::fail(MHT_ERR_INVALID_ARG, "NULL plan");
    if (!plan->bound) mht::fail(MHT_ERR_NOT_BOUND, "plan is not bound to device memory");
    if (nrhs < 1 || nrhs > plan->dev.max_nrhs) mht::fail(MHT_ERR_INVALID_ARG, "nrhs outside 1..max_nrhs");
    std::string err;
    plan->tune_report.clear();
    if (int rc = mht::apply_autotune(plan->F, plan->P, plan->dev, nrhs, plan->mode, stream, &plan->tune_report, err))
      mht::fail(mht_status(rc), err);
    return MHT_OK;
  });
}

mht_status mht_plan_tune_info(const mht_plan* plan, int32_t direction, int32_t stage, int32_t* cfg, double* ms) {
  return guarded([&]() -> mht_status {
    if (!plan || !cfg) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    for (const mht::TuneRecord& r : plan->tune_report)
      if (r.dir == direction && r.stage == stage) {
        cfg[0] = r.cfg.tensor;
        cfg[1] = r.cfg.rt;
        cfg[2] = r.cfg.nslot;
        cfg[3] = r.cfg.per_sm;
        cfg[4] = r.cfg.slot_kb;
        if (ms) *ms = r.ms;
        return MHT_OK;
      }
    mht::fail(MHT_ERR_INVALID_ARG, "no tuned configuration for this stage");
    return MHT_OK;
  });
}

mht_status mht_plan_profile(mht_plan* plan, int32_t enable) {
  return guarded([&]() -> mht_status {
    if (!plan) mht::fail(MHT_ERR_INVALID_ARG, "NULL plan");
    if (enable && !plan->dev.prof) plan->dev.prof = mht::profiler_create();
    if (!enable && plan->dev.prof) {
      mht::profiler_destroy(plan->dev.prof);
      plan->dev.prof = nullptr;
    }
    return MHT_OK;
  });
}

mht_status mht_plan_stage_times(mht_plan* plan, int32_t direction, double* ms, int64_t* launches) {
  return guarded([&]() -> mht_status {
    if (!plan || !ms || !launches || (direction != 0 && direction != 1)) mht::fail(MHT_ERR_INVALID_ARG, "bad argument");
    if (!plan->dev.prof) mht::fail(MHT_ERR_INVALID_ARG, "stage timing is not enabled");
    std::string err;
    int rc = mht::profiler_read(plan->dev.prof, direction, plan->F.L + 3, ms, launches, err);
    return rc ? set_error(mht_status(rc), err) : MHT_OK;
  });
}

mht_status mht_plan_save(const mht_plan* plan, const char* path) {
  return guarded([&]() -> mht_status {
    if (!plan || !path) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    const mht::Factorization& F = plan->F;
    Writer w;
    w.pod<int64_t>(F.n); w.pod<int64_t>(F.m); w.pod<int32_t>(F.L); w.pod<int32_t>(F.cplx ? 1 : 0);
    w.pod<double>(plan->eps);
    w.vec(F.space_perm); w.vec(F.space_off); w.vec(F.mode_perm); w.vec(F.mode_off); w.vec(F.weights);
    for (auto& lvl : F.lv)
      for (auto& B : lvl) {
        w.pod<int32_t>(B.r); w.pod<int32_t>(B.K);
        w.vec(B.perm); w.vec(B.T);
      }
    for (auto& u : F.U) w.vec(u);
    FILE* fp = std::fopen(path, "wb");
    if (!fp) mht::fail(MHT_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
    const uint64_t h = fnv1a(w.buf.data(), w.buf.size());
    const uint64_t sz = w.buf.size();
    bool ok = std::fwrite(&kMagic, 8, 1, fp) == 1 && std::fwrite(&kVersion, 4, 1, fp) == 1 &&
              std::fwrite(&sz, 8, 1, fp) == 1 && std::fwrite(&h, 8, 1, fp) == 1 &&
              (sz == 0 || std::fwrite(w.buf.data(), 1, sz, fp) == sz);
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) mht::fail(MHT_ERR_INVALID_ARG, std::string("write failed: ") + path);
    return MHT_OK;
  });
}

mht_status mht_plan_load(const char* path, const mht_options* options, mht_plan** out) {
  return guarded([&]() -> mht_status {
    if (!path || !options || !out) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    check_mode(options->mode);
    FILE* fp = std::fopen(path, "rb");
    if (!fp) mht::fail(MHT_ERR_INVALID_ARG, std::string("cannot open: ") + path);
    uint64_t magic = 0, sz = 0, h = 0;
    uint32_t ver = 0;
    bool ok = std::fread(&magic, 8, 1, fp) == 1 && std::fread(&ver, 4, 1, fp) == 1 && std::fread(&sz, 8, 1, fp) == 1 &&
              std::fread(&h, 8, 1, fp) == 1;
    if (!ok || magic != kMagic) { std::fclose(fp); mht::fail(MHT_ERR_FORMAT, "not a plan file"); }
    if (ver != kVersion) { std::fclose(fp); mht::fail(MHT_ERR_FORMAT, "unsupported plan file version"); }
    std::fseek(fp, 0, SEEK_END);
    const long total = std::ftell(fp);
    if (total < 0 || uint64_t(total) != 28 + sz) { std::fclose(fp); mht::fail(MHT_ERR_FORMAT, "plan file size mismatch"); }
    std::fseek(fp, 28, SEEK_SET);
    std::vector<uint8_t> buf(sz);
    ok = sz == 0 || std::fread(buf.data(), 1, sz, fp) == sz;
    std::fclose(fp);
    if (!ok) mht::fail(MHT_ERR_FORMAT, "truncated plan file");
    if (fnv1a(buf.data(), buf.size()) != h) mht::fail(MHT_ERR_FORMAT, "plan file checksum mismatch");
    Reader r{buf.data(), buf.size()};
    std::unique_ptr<mht_plan> plan(new mht_plan());
    mht::Factorization& F = plan->F;
    F.n = r.pod<int64_t>(); F.m = r.pod<int64_t>(); F.L = r.pod<int32_t>(); F.cplx = r.pod<int32_t>() != 0;
    plan->eps = r.pod<double>();
    if (F.n <= 0 || F.m <= 0 || F.L < 0 || F.L > 24) mht::fail(MHT_ERR_FORMAT, "bad plan header");
    const uint64_t big = uint64_t(sz);
    r.vec(F.space_perm, big); r.vec(F.space_off, big); r.vec(F.mode_perm, big); r.vec(F.mode_off, big);
    r.vec(F.weights, big);
    const int64_t nb = F.nblk();
    F.lv.assign(F.L + 1, std::vector<mht::Block>(nb));
    for (auto& lvl : F.lv)
      for (auto& B : lvl) {
        B.r = r.pod<int32_t>(); B.K = r.pod<int32_t>();
        r.vec(B.perm, big); r.vec(B.T, big);
      }
    F.U.assign(nb, {});
    for (auto& u : F.U) r.vec(u, big);
    if (int64_t(F.space_off.size()) != nb + 1 || int64_t(F.mode_off.size()) != nb + 1)
      mht::fail(MHT_ERR_FORMAT, "bad offsets in plan file");
    F.validate();
    plan->mode = options->mode;
    mht::pack(F, fp64_mode(options->mode), plan->P);
    *out = plan.release();
    return MHT_OK;
  });
}

mht_status mht_destroy(mht_plan* plan) {
  delete plan;
  return MHT_OK;
}

// ---- batched apply ---------------------------------------------------------------------

mht_status mht_batch_create(mht_plan* const* plans, int32_t count, const int64_t* nrhs, mht_batch** out) {
  return guarded([&]() -> mht_status {
    if (!out) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::unique_ptr<mht_batch> b(new mht_batch());
    mht::batch_init(*b, plans, count, nrhs);
    *out = b.release();
    return MHT_OK;
  });
}

mht_status mht_batch_device_bytes(const mht_batch* batch, size_t* image_bytes, size_t* workspace_bytes) {
  return guarded([&]() -> mht_status {
    if (!batch || !image_bytes || !workspace_bytes) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    *image_bytes = batch->image_bytes;
    *workspace_bytes = batch->ws_bytes;
    return MHT_OK;
  });
}

mht_status mht_batch_bind_device(mht_batch* batch, void* image_dev, size_t image_bytes, void* workspace_dev,
                                 size_t workspace_bytes, void* stream) {
  return guarded([&]() -> mht_status {
    if (!batch || !image_dev || !workspace_dev) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    if (image_bytes < batch->image_bytes || workspace_bytes < batch->ws_bytes)
      mht::fail(MHT_ERR_INVALID_ARG, "device buffers smaller than mht_batch_device_bytes");
    if ((reinterpret_cast<uintptr_t>(image_dev) | reinterpret_cast<uintptr_t>(workspace_dev)) & 255)
      mht::fail(MHT_ERR_INVALID_ARG, "device buffers must be 256-byte aligned");
    for (auto*& g : batch->graphs) {
      mht::batch_graph_destroy(g);
      g = nullptr;
    }
    batch->image_dev = static_cast<uint8_t*>(image_dev);
    batch->ws_dev = static_cast<uint8_t*>(workspace_dev);
    std::string err;
    for (const mht::BatchInst& I : batch->inst)
      if (int rc = mht::device_upload_image(I.plan->P, batch->image_dev + I.image_off, stream, err))
        mht::fail(mht_status(rc), err);
    for (int dir = 0; dir < 2; ++dir)
      if (int rc = mht::device_upload(batch->image_dev + batch->items_off[dir], batch->items[dir].data(),
                                      batch->items[dir].size() * sizeof(MhtBItem), stream, err))
        mht::fail(mht_status(rc), err);
    std::vector<uint8_t> zero(256, 0);
    if (int rc = mht::device_upload(batch->ws_dev + batch->status_off, zero.data(), 256, stream, err))
      mht::fail(mht_status(rc), err);
    for (const mht::BatchInst& I : batch->inst) {  // status words of the per-instance workspaces
      const size_t so = I.meta.status_offset(I.nrhs, I.n, I.m);
      if (int rc = mht::device_upload(batch->ws_dev + I.ws_off + so, zero.data(), sizeof(unsigned), stream, err))
        mht::fail(mht_status(rc), err);
    }
    for (auto*& g : batch->tc) {
      mht::tc_group_destroy(g);
      g = nullptr;
    }
    for (mht::BatchInst& I : batch->inst) I.plan = nullptr;
    batch->bound = true;
    batch->io_set = false;
    return MHT_OK;
  });
}

mht_status mht_batch_set_io(mht_batch* batch, void* const* c_dev, const int64_t* ldc, void* const* f_dev,
                            const int64_t* ldf, void* stream) {
  return guarded([&]() -> mht_status {
    if (!batch || !c_dev || !ldc || !f_dev || !ldf) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    if (!batch->bound) mht::fail(MHT_ERR_NOT_BOUND, "batch is not bound to device memory");
    for (int i = 0; i < batch->n; ++i) {
      mht::BatchInst& I = batch->inst[i];
      if (!c_dev[i] || !f_dev[i]) mht::fail(MHT_ERR_INVALID_ARG, "NULL vector in batch");
      if ((I.nrhs > 1 && (ldc[i] < I.m || ldf[i] < I.n)) || ldc[i] < 1 || ldf[i] < 1)
        mht::fail(MHT_ERR_INVALID_ARG, "leading dimension smaller than the vector length");
      I.c = reinterpret_cast<uint64_t>(c_dev[i]);
      I.f = reinterpret_cast<uint64_t>(f_dev[i]);
      I.ldc = ldc[i];
      I.ldf = ldf[i];
    }
    mht::batch_fill_records(*batch);
    std::string err;
    for (int dir = 0; dir < 2; ++dir)
      if (int rc = mht::device_upload(batch->image_dev + batch->recs_off[dir], batch->recs[dir].data(),
                                      batch->recs[dir].size() * sizeof(MhtBatchRec), stream, err))
        mht::fail(mht_status(rc), err);
    for (auto*& g : batch->tc) {  // captured with the previous vectors
      mht::tc_group_destroy(g);
      g = nullptr;
    }
    batch->io_set = true;
    return MHT_OK;
  });
}

namespace {
static mht_status batch_run(mht_batch* batch, int dir, bool weighted, void* stream) {
  if (!batch) mht::fail(MHT_ERR_INVALID_ARG, "NULL batch");
  if (!batch->bound || !batch->io_set) mht::fail(MHT_ERR_NOT_BOUND, "batch is not bound or has no vectors");
  std::string err;
  if (mht::tensor_mode(batch->mode)) {
    if (int rc = mht::batch_tc_run(*batch, dir, weighted, stream, err)) mht::fail(mht_status(rc), err);
    return MHT_OK;
  }
  const mht::BatchLaunch b = mht::batch_launch_desc(*batch, dir, weighted);
  if (!batch->use_graph) {
    if (int rc = mht::batch_launch(b, stream, err)) mht::fail(mht_status(rc), err);
    return MHT_OK;
  }
  mht::BatchGraph*& g = batch->graphs[dir == 0 ? 0 : (weighted ? 2 : 1)];
  if (!g)
    if (int rc = mht::batch_graph_create(b, &g, err)) mht::fail(mht_status(rc), err);
  if (int rc = mht::batch_graph_launch(g, stream, err)) mht::fail(mht_status(rc), err);
  return MHT_OK;
}
}  // namespace

mht_status mht_batch_synthesize(mht_batch* batch, void* stream) {
  return guarded([&]() -> mht_status { return batch_run(batch, 0, false, stream); });
}

mht_status mht_batch_analyze(mht_batch* batch, int32_t weighted, void* stream) {
  return guarded([&]() -> mht_status { return batch_run(batch, 1, weighted != 0, stream); });
}

mht_status mht_batch_set_mode(mht_batch* batch, mht_apply_mode mode) {
  return guarded([&]() -> mht_status {
    if (!batch) mht::fail(MHT_ERR_INVALID_ARG, "NULL batch");
    if (mode != MHT_APPLY_FP32 && !mht::tensor_mode(mode))
      mht::fail(MHT_ERR_INVALID_ARG, "FP32, 3XTF32 or 6XBF16 only");
    if (mode != batch->mode)
      for (auto*& g : batch->tc) {  // the captured per-instance applies hold the arithmetic
        mht::tc_group_destroy(g);
        g = nullptr;
      }
    batch->mode = mode;
    return MHT_OK;
  });
}

mht_status mht_batch_set_graph(mht_batch* batch, int32_t use_graph) {
  return guarded([&]() -> mht_status {
    if (!batch) mht::fail(MHT_ERR_INVALID_ARG, "NULL batch");
    batch->use_graph = use_graph ? 1 : 0;
    return MHT_OK;
  });
}

mht_status mht_batch_info(const mht_batch* batch, int64_t* items_synthesis, int64_t* items_analysis, int32_t* grid) {
  return guarded([&]() -> mht_status {
    if (!batch) mht::fail(MHT_ERR_INVALID_ARG, "NULL batch");
    if (items_synthesis) *items_synthesis = int64_t(batch->items[0].size());
    if (items_analysis) *items_analysis = int64_t(batch->items[1].size());
    if (grid) {
      std::string err;
      const int g = mht::batch_grid_size(mht::batch_launch_desc(*batch, 0, false), err);
      if (g < 0) mht::fail(mht_status(-g), err);
      *grid = g;
    }
    return MHT_OK;
  });
}

mht_status mht_batch_check(mht_batch* batch, void* stream, int32_t* flags) {
  return guarded([&]() -> mht_status {
    if (!batch || !flags) mht::fail(MHT_ERR_INVALID_ARG, "NULL argument");
    if (!batch->bound) mht::fail(MHT_ERR_NOT_BOUND, "batch is not bound to device memory");
    unsigned v = 0;
    std::string err;
    if (int rc = mht::device_status(batch->ws_dev + batch->status_off, stream, &v, err)) mht::fail(mht_status(rc), err);
    for (const mht::BatchInst& I : batch->inst) {  // the tensor-core form reports per instance
      unsigned u = 0;
      const size_t so = I.meta.status_offset(I.nrhs, I.n, I.m);
      if (int rc = mht::device_status(batch->ws_dev + I.ws_off + so, stream, &u, err)) mht::fail(mht_status(rc), err);
      v |= u;
    }
    *flags = int32_t(v);
    if (v) return set_error(MHT_ERR_TIMEOUT, "a bounded wait in the batched apply gave up");
    return MHT_OK;
  });
}

mht_status mht_batch_autotune(mht_batch* batch, void* stream, double* best_ms) {
  return guarded([&]() -> mht_status {
    if (!batch) mht::fail(MHT_ERR_INVALID_ARG, "NULL batch");
    if (!batch->bound || !batch->io_set) mht::fail(MHT_ERR_NOT_BOUND, "batch is not bound or has no vectors");
    batch->tuned_nslot = batch->tuned_per_sm = 0;
    const mht::BatchLaunch syn = mht::batch_launch_desc(*batch, 0, false);
    const mht::BatchLaunch ana = mht::batch_launch_desc(*batch, 1, true);
    int ns = 0, ps = 0;
    double ms = 0;
    std::string err;
    if (int rc = mht::batch_autotune(syn, ana, batch->nslot, stream, &ns, &ps, &ms, err)) mht::fail(mht_status(rc), err);
    batch->tuned_nslot = ns;
    batch->tuned_per_sm = ps;
    for (auto*& g : batch->graphs) {  // rebuilt with the tuned shape at the next launch
      mht::batch_graph_destroy(g);
      g = nullptr;
    }
    if (best_ms) *best_ms = ms;
    return MHT_OK;
  });
}

mht_status mht_batch_debug_hold(mht_batch* batch, int32_t direction, int32_t instance, int32_t phase, void* stream) {
  return guarded([&]() -> mht_status {
    if (!batch) mht::fail(MHT_ERR_INVALID_ARG, "NULL batch");
    if (!batch->bound || !batch->io_set) mht::fail(MHT_ERR_NOT_BOUND, "batch is not bound or has no vectors");
    if (direction < 0 || direction > 1 || instance < 0 || instance >= batch->n)
      mht::fail(MHT_ERR_INVALID_ARG, "bad direction or instance");
    const mht::BatchInst& I = batch->inst[instance];
    if (phase < 1 || phase >= I.L + 2) mht::fail(MHT_ERR_INVALID_ARG, "phase must have a predecessor");
    const int rec = I.rec_base[direction] + phase;
    MhtBatchRec r = batch->recs[direction][rec];
    r.wait_count = 0xffffffffu;  // more completions than the previous phase has items
    std::string err;
    if (int rc = mht::device_upload(batch->image_dev + batch->recs_off[direction] + size_t(rec) * sizeof(MhtBatchRec), &r,
                                    sizeof r, stream, err))
      mht::fail(mht_status(rc), err);
    return MHT_OK;
  });
}

mht_status mht_batch_destroy(mht_batch* batch) {
  delete batch;
  return MHT_OK;
}

}  // extern "C"
