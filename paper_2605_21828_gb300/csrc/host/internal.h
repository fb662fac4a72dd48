// Host-side internals of the BF-MHT library: factorization storage, evaluators, trees,
// interpolative decompositions, packing and the device-apply interface.
#pragma once
#include <complex>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../../include/mht.h"
#include "../layout.h"

namespace mht {

struct Error : std::runtime_error {
  mht_status code;
  Error(mht_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};
[[noreturn]] inline void fail(mht_status c, const std::string& m) { throw Error(c, m); }

// One interpolative decomposition block of Sec. 2: input of size K, rank r, local input
// indices `perm` (skeleton first) and T~ (r x (K - r), row-major; complex interleaved).
struct Block {
  int32_t r = 0, K = 0;
  std::vector<int32_t> perm;
  std::vector<double> T;
};

// The butterfly factorization in FP64 (the content of mht_factors).
struct Factorization {
  int64_t n = 0, m = 0;
  int L = 0;
  bool cplx = false;
  std::vector<int64_t> space_perm, space_off, mode_perm, mode_off;
  std::vector<std::vector<Block>> lv;  // [L+1][2^L], block b = tau * 2^(L-l) + nu
  std::vector<std::vector<double>> U;  // [2^L], |tau| x r_L row-major
  std::vector<double> weights;         // [n] or empty (= ones)

  int64_t nblk() const { return int64_t(1) << L; }
  int64_t leaf_rows(int64_t tau) const { return space_off[tau + 1] - space_off[tau]; }
  // Input size K of block b at level l (level 0: |nu|; else r(p,2nu) + r(p,2nu+1)).
  int64_t input_size(int l, int64_t b) const;
  // Offset of the pair (p, 2nu), (p, 2nu+1) at level l-1 read by block b of level l.
  int64_t pair_index(int l, int64_t b) const {
    int64_t nb = int64_t(1) << (L - l);
    int64_t tau = b / nb, nu = b % nb, p = tau >> 1;
    return p * (nb << 1) + 2 * nu;
  }
  void validate() const;  // throws MHT_ERR_FORMAT on inconsistency
};

// --- Phi evaluators ------------------------------------------------------------------
// Fill out (column-major nr x nc; complex: interleaved pairs) with Phi(rows, cols).
struct Evaluator {
  virtual ~Evaluator() = default;
  virtual void eval(const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
                    double* out) const = 0;
};
Evaluator* make_evaluator(const mht_problem& p);  // caller owns

// --- trees -------------------------------------------------------------------------------
void frequency_tree(const double* eigenvalues, int64_t m, int L, std::vector<int64_t>& perm,
                    std::vector<int64_t>& off);
void space_tree(const mht_problem& p, mht_tree_kind kind, int L, uint64_t seed,
                std::vector<int64_t>& perm, std::vector<int64_t>& off);

// --- interpolative decomposition ----------------------------------------------------------
// Column ID of the column-major M x K matrix A (overwritten) by Householder QR with column
// pivoting; rank = #{k : |R_kk| > eps |R_11|}.  Writes perm (skeleton first) and
// T~ = R11^{-1} R12 (row-major r x (K-r)).  Returns r.
// blocked = true selects the randomized block-pivoted variant (HQRRP) for large blocks and a
// Gram-matrix full-rank certificate for very tall ones (real and complex).
int interpolative_decomposition_real(double* A, int64_t M, int64_t K, double eps,
                                     std::vector<int32_t>& perm, std::vector<double>& T, uint64_t seed = 0,
                                     bool blocked = false);
int interpolative_decomposition_complex(std::complex<double>* A, int64_t M, int64_t K,
                                        double eps, std::vector<int32_t>& perm,
                                        std::vector<double>& T, uint64_t seed = 0, bool blocked = false);

// --- build ---------------------------------------------------------------------------------
void build_factorization(const mht_problem& p, const mht_options& o, Factorization& F);
void import_factors(const mht_factors& in, Factorization& F);

// --- packing -------------------------------------------------------------------------------
// Each stage is stored twice: as applied by synthesis (T~ r x K', U |tau| x r_L) and as
// applied by the adjoint (conj(T~)^T K' x r, conj(U)^T r_L x |tau|), so both directions
// stream contiguous rows.  dir[0] = synthesis, dir[1] = analysis.
struct StageDir {
  size_t desc_off = 0, items_off = 0;  // byte offsets in the image
  int64_t nitems = 0;
  int64_t max_ld = 0;                  // widest padded row (elements)
  int64_t max_item_rows = 0;           // most rows in one work item
  size_t data_bytes = 0;               // padded device bytes of this direction's matrices
  size_t tc_items_off = 0;             // 128-row tiles for the tensor-core stages
  int64_t tc_nitems = 0;
};

struct Stage {
  int64_t nblocks = 0;
  int64_t out_entries = 0;      // entries of the synthesis output vector (per RHS)
  int64_t in_entries = 0;       // entries of the synthesis input vector (per RHS)
  int64_t max_rank = 0;
  int64_t t_entries = 0;        // stored matrix entries (one orientation)
  size_t alg_bytes = 0;         // algorithmic bytes of one single-RHS launch
  StageDir dir[2];
};

// Persistent (fused) apply of one direction: all stages in one launch, dependency order.
struct FusedDir {
  size_t desc_all_off = 0;      // [(L+2) * nb] descriptors, stage-major (= dir desc arrays)
  size_t targets_off = 0;       // [(L+2) * nb] int32 persistent items per block
  size_t items_off = 0;         // persistent work list
  int64_t nitems = 0;
  size_t slot_bytes = 0;        // bytes of one ring slot (>= the widest row)
  int64_t max_ld = 0;
  int64_t max_item_rows = 0;    // largest persistent item (rows)
  std::vector<int64_t> stage_first;  // [L+3] first item of the k-th stage in dependency order
};

struct Packed {
  bool fp64 = false, cplx = false;
  int elem_bytes = 4;           // bytes of one (possibly complex) element
  int L = 0;
  int64_t nb = 0;
  std::vector<uint8_t> image;
  size_t data_off = 0, index_off = 0, perm_off = 0, weights_off = 0, vecoff_off = 0;
  // tensor maps of the tensor-core stages: one 128-byte CUtensorMap per (direction, stage,
  // block), encoded when the image is bound (they hold device addresses); FP32 images only
  size_t tmap_off = 0, tmap_bytes = 0;
  std::vector<Stage> st;        // L+2 stages: ID levels 0..L, then U
  FusedDir fused[2];
  std::vector<int64_t> vec_off; // [L+2] offsets of the level vectors (per RHS), vec_off[L+1] = total
  int64_t vec_entries = 0;      // total butterfly-vector entries over all levels (per RHS)
  int64_t index_entries = 0;
  // workspace: Y, A0, A1 level vectors, host staging for c and f, counters, status word
  size_t ws_vec_bytes(int64_t nrhs) const;
  size_t ws_counters_offset(int64_t nrhs, int64_t n, int64_t m) const;
  size_t status_offset(int64_t nrhs, int64_t n, int64_t m) const;
  size_t workspace_bytes(int64_t nrhs, int64_t n, int64_t m) const;
};
void pack(const Factorization& F, bool fp64, Packed& P);
// Testing aid: packed images larger than this many bytes fail as a host allocation failure
// would (0: no limit).
size_t host_alloc_limit();
void set_host_alloc_limit(size_t bytes);
// Checks every descriptor, index, permutation entry and work item of a packed image against
// the buffers the kernels address with them (throws MHT_ERR_FORMAT).
void validate_packed(const Packed& P, int64_t n, int64_t m);

}  // namespace mht

// Device binding and apply (implemented in the CUDA translation unit).
namespace mht {
struct Profiler;  // per-stage CUDA event records (apply.cu)
// Launch configuration of one stage (0 = default / all that fit).
struct StageCfg {
  int tensor = 0;  // 3xTF32 tensor-core kernel instead of the SIMT one
  int rt = 1;      // SIMT RHS tile
  int nslot = 0;   // bulk-copy ring slots
  int slot_kb = 0; // ring slot size in KB (0: 32)
  int per_sm = 0;  // resident CTAs per SM
};
struct TuneRecord {
  int dir, stage;
  StageCfg cfg;
  double ms;
};
struct DeviceView {
  const uint8_t* base = nullptr;  // bound factor image
  uint8_t* ws = nullptr;          // workspace
  size_t ws_bytes = 0;
  int64_t max_nrhs = 0;
  Profiler* prof = nullptr;       // non-null while stage timing is enabled
  int path = 0;                   // 0 auto, 1 per-stage launches, 2 fused persistent launch
  int64_t tune_nrhs = 0;          // RHS count the stage configurations were tuned for (0: none)
  mht_apply_mode tune_mode = MHT_APPLY_FP32;
  std::vector<StageCfg> tune[2];  // per direction and stage
  // stages at the start / end of each direction that run as one persistent launch with
  // per-block dependency counters (0: none), chosen by the autotuner for tune_nrhs
  int fuse_head[2] = {0, 0}, fuse_tail[2] = {0, 0};
  struct FilterGraph* filter = nullptr;  // cached CUDA graph of the last spectral filter call
};
void filter_graph_destroy(FilterGraph* g);
// f_out = Phi diag(filter) Phi^H [W] f_in in one CUDA graph (captured on the first call with
// these arguments, replayed afterwards); the coefficients pass through the workspace's
// host-staging area for c.
int apply_filter(const Factorization& F, const Packed& P, DeviceView& d, const void* f_in, int64_t ldi, void* f_out,
                 int64_t ldo, int64_t nrhs, const void* filter, bool weighted, mht_apply_mode mode, void* stream,
                 std::string& err);
Profiler* profiler_create();
void profiler_destroy(Profiler* p);
int profiler_read(Profiler* p, int direction, int nstages, double* ms, int64_t* launches, std::string& err);
// scale (optional, device, m real entries in the plan's precision, caller's mode order):
// f = Phi diag(scale) c, the scale fused into the leaf stage's gather.
int apply_synthesize(const Factorization& F, const Packed& P, const DeviceView& d,
                     const void* c, int64_t ldc, void* f, int64_t ldf, int64_t nrhs,
                     bool weighted, mht_apply_mode mode, void* stream, std::string& err,
                     const void* scale = nullptr);
int apply_analyze(const Factorization& F, const Packed& P, const DeviceView& d, const void* f,
                  int64_t ldf, void* c, int64_t ldc, int64_t nrhs, bool weighted,
                  mht_apply_mode mode, void* stream, std::string& err);
int64_t apply_launches(const Packed& P, int64_t nrhs, mht_apply_mode mode, int path);
// Times the candidate configurations of every stage for `nrhs` RHS and stores the fastest in
// d.tune (used by later applies with that RHS count); synchronizes `stream`.
int apply_autotune(const Factorization& F, const Packed& P, DeviceView& d, int64_t nrhs, mht_apply_mode mode,
                   void* stream, std::vector<TuneRecord>* report, std::string& err);
int device_upload(void* dst, const void* src, size_t bytes, void* stream, std::string& err);
int device_copy_async(void* dst, const void* src, size_t bytes, int kind, void* stream,
                      std::string& err);
int device_sync(void* stream, std::string& err);
// One stage of a multi-RHS apply on the tensor cores (3xTF32, FP32 plans, real or complex).
struct TcLaunch {
  const float* data;
  const int* idx;
  const MhtBlockDesc* desc;
  const MhtItem* items;
  int64_t nitems;
  const int* perm;
  const float* wts;
  const float* in0;
  const float* in1;
  long long is_e, is_k;
  float* out0;
  float* out1;
  long long os_e, os_k;
  int64_t nrhs;
  int mode;  // 0 synthesis ID stage, 1 adjoint ID stage, 2 synthesis column bases, 3 adjoint
  int cplx;  // complex factors and vectors (interleaved float pairs)
  int bf16;  // 1: 6xBF16 split products, 0: 3xTF32
  const void* tmaps;  // the stage's tensor maps (one per block, this direction) in the image
  unsigned* status;
  void* stream;
};
int tc_stage_launch(const TcLaunch& a, std::string& err);
// Tensor maps of an FP32 image bound at base_dev (P.tmap_bytes bytes, for [P.tmap_off]).
int tc_encode_tmaps(const Packed& P, const void* base_dev, std::vector<uint8_t>& out, std::string& err);
// Uploads the image to base_dev and, for FP32 plans, its tensor maps (synchronous).
int device_upload_image(const Packed& P, void* base_dev, void* stream, std::string& err);
bool tensor_mode(mht_apply_mode m);
// Fused FP32 synthesis of one vector with scratch from a fixed library array (no allocation).
int apply_synthesize_noalloc(const Packed& P, const void* factor_dev, const void* c, void* f, void* stream,
                             std::string& err);
// Bytes of the fixed scratch array a plan's no-alloc synthesis needs (status word included).
size_t noalloc_scratch_need(const Packed& P);
// Reads and clears the no-alloc status word on the current device; synchronizes the stream.
int noalloc_status(void* stream, unsigned* flags, std::string& err);
// Makes (hold) or undoes an unreachable completion target in the caller's factor image.
int noalloc_debug_hold(const Packed& P, void* factor_dev, bool hold, void* stream, std::string& err);
// Copies the device status word to *flags, clears it, and synchronizes the stream.
int device_status(void* status_dev, void* stream, unsigned* flags, std::string& err);

// Inverse transform by LSQR (lsqr.cu): c = argmin ||Phi c - f||_2 per column; scratch of
// lsqr_scratch_bytes in caller device memory; synchronous on `stream`.
size_t lsqr_scratch_bytes(const Packed& P, int64_t n, int64_t m, int64_t k);
int apply_lsqr(const Factorization& F, const Packed& P, const DeviceView& d, const void* f, int64_t ldf, void* c,
               int64_t ldc, int64_t k, void* scratch, int max_iter, double tol, mht_apply_mode mode, void* stream,
               int* iters, double* relres, std::string& err);

// Batched apply of many FP32 plans in one persistent launch (batch.cu).
struct BatchLaunch {
  const void* recs;         // MhtBatchRec[] of the direction (device)
  const void* items;        // MhtBItem[] of the direction, dependency order (device)
  int nitems;
  unsigned* ticket;         // queue head, abort word and completion counters: all inside
  unsigned* abort;          // [counters, counters + counter_bytes), zeroed before every launch
  unsigned* done;
  void* counters;
  size_t counter_bytes;
  unsigned* status;         // status word (bit 0 copy wait, bit 1 dependency wait gave up)
  int use_wts;
  int slot_bytes, nslot, ldx_max, rows_max;  // shared-memory layout maxima over all items
  int per_sm;               // resident CTAs per SM (0: as many as fit)
};
struct BatchGraph;
size_t batch_smem(int slot_bytes, int nslot, int ldx_max, int rows_max);
int batch_launch(const BatchLaunch& b, void* stream, std::string& err);
int batch_graph_create(const BatchLaunch& b, BatchGraph** g, std::string& err);
int batch_graph_launch(BatchGraph* g, void* stream, std::string& err);
void batch_graph_destroy(BatchGraph* g);
int batch_grid_size(const BatchLaunch& b, std::string& err);  // CTAs of one launch (< 0: error)
int batch_autotune(const BatchLaunch& syn, const BatchLaunch& ana, int max_nslot, void* stream, int* nslot,
                   int* per_sm, double* best_ms, std::string& err);
}  // namespace mht

struct mht_plan {
  mht::Factorization F;
  mht::Packed P;
  mht_apply_mode mode = MHT_APPLY_FP32;
  double eps = 0;
  double build_seconds = 0;
  mht::DeviceView dev;
  std::vector<mht::TuneRecord> tune_report;
  bool bound = false;
  ~mht_plan() {
    mht::profiler_destroy(dev.prof);
    mht::filter_graph_destroy(dev.filter);
  }
};

// A batch of FP32 plans applied together (batch.cpp, batch.cu).
namespace mht {
struct BatchInst {
  const mht_plan* plan = nullptr;  // needed until the batch is bound
  int64_t n = 0, m = 0, nrhs = 1;
  int L = 0, es = 4;
  bool cplx = false;
  std::vector<int64_t> vec_off;
  size_t image_off = 0, image_bytes = 0, data_off = 0, index_off = 0, perm_off = 0, weights_off = 0;
  std::vector<size_t> desc_off[2];  // per stage, relative to the instance image
  int rec_base[2] = {0, 0}, ctr_base[2] = {0, 0};
  size_t ws_off = 0, region_bytes = 0, ws_bytes = 0;  // a full per-plan workspace each
  uint64_t c = 0, f = 0;            // caller vectors (set_io)
  int64_t ldc = 0, ldf = 0;
  Packed meta;                      // the plan's packing without its image (per-plan applies)
  Factorization shape;              // n, m, L only
};
struct TcGroup;                      // CUDA graph of per-instance applies (tensor-core form)
void tc_group_destroy(TcGroup* g);
}  // namespace mht

struct mht_batch {
  int n = 0;
  std::vector<mht::BatchInst> inst;
  std::vector<MhtBatchRec> recs[2];
  std::vector<MhtBItem> items[2];
  size_t recs_off[2] = {0, 0}, items_off[2] = {0, 0}, image_bytes = 0;
  size_t counters_off = 0, counter_bytes = 0, status_off = 0, ws_bytes = 0;
  int nctr = 0;
  int slot_bytes = 0, nslot = 0, ldx_max = 0, rows_max = 0;
  int tuned_nslot = 0, tuned_per_sm = 0;  // autotuned launch shape (0: defaults)
  uint8_t* image_dev = nullptr;
  uint8_t* ws_dev = nullptr;
  bool bound = false, io_set = false;
  int use_graph = 1;
  mht_apply_mode mode = MHT_APPLY_FP32;  // 3XTF32: graph of per-instance tensor-core applies
  mht::BatchGraph* graphs[3] = {nullptr, nullptr, nullptr};  // synthesis, analysis, weighted
  mht::TcGroup* tc[3] = {nullptr, nullptr, nullptr};
  ~mht_batch();
};

namespace mht {
void batch_init(mht_batch& B, mht_plan* const* plans, int count, const int64_t* nrhs);
void batch_fill_records(mht_batch& B);
// Checks the dependency order of the batch work list (throws MHT_ERR_FORMAT).
void batch_validate(const mht_batch& B);
BatchLaunch batch_launch_desc(const mht_batch& B, int dir, bool weighted);
// Tensor-core form of a batch: every instance's own per-stage apply (3xTF32 products from 16
// real / 8 complex RHS) on 8 forked streams, captured once into a CUDA graph and replayed.
int batch_tc_run(mht_batch& B, int dir, bool weighted, void* stream, std::string& err);
}  // namespace mht
