// Batched ragged apply: host-side layout of a batch of FP32 plans (device image, workspace,
// dependency-ordered work list, per-stage records) for the persistent kernel in batch.cu.
//
// Device image:  [instance images, 256-aligned][records dir 0][records dir 1][items dir 0]
//                [items dir 1]
// Workspace:     [per instance: Y, A0, A1 level vectors for its RHS count][counters][status]
// The counters (queue head, abort word, one completion counter per instance, direction and
// phase) are zeroed before every launch.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace mht {
namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

void batch_init(mht_batch& B, mht_plan* const* plans, int count, const int64_t* nrhs) {
  if (count <= 0 || !plans || !nrhs) fail(MHT_ERR_INVALID_ARG, "batch needs plans and RHS counts");
  B.n = count;
  B.inst.resize(count);
  size_t img = 0;
  int64_t max_ld = 1, max_rows = 1, max_row_bytes = 1;
  for (int i = 0; i < count; ++i) {
    const mht_plan* p = plans[i];
    if (!p) fail(MHT_ERR_INVALID_ARG, "NULL plan in batch");
    if (p->P.fp64) fail(MHT_ERR_INVALID_ARG, "batched apply takes FP32 plans only");
    if (nrhs[i] < 1 || nrhs[i] > (int64_t(1) << 20)) fail(MHT_ERR_INVALID_ARG, "bad RHS count in batch");
    BatchInst& I = B.inst[i];
    I.plan = p;
    I.n = p->F.n;
    I.m = p->F.m;
    I.L = p->F.L;
    I.cplx = p->P.cplx;
    I.es = p->P.elem_bytes;
    I.nrhs = nrhs[i];
    I.vec_off = p->P.vec_off;
    I.image_off = img;
    I.image_bytes = p->P.image.size();
    I.data_off = p->P.data_off;
    I.index_off = p->P.index_off;
    I.perm_off = p->P.perm_off;
    I.weights_off = p->P.weights_off;
    {  // the packing's layout without its (large) image
      const Packed& Q = p->P;
      Packed& M = I.meta;
      M.fp64 = Q.fp64;
      M.cplx = Q.cplx;
      M.elem_bytes = Q.elem_bytes;
      M.L = Q.L;
      M.nb = Q.nb;
      M.data_off = Q.data_off;
      M.index_off = Q.index_off;
      M.perm_off = Q.perm_off;
      M.weights_off = Q.weights_off;
      M.vecoff_off = Q.vecoff_off;
      M.tmap_off = Q.tmap_off;
      M.tmap_bytes = Q.tmap_bytes;
      M.st = Q.st;
      M.fused[0] = Q.fused[0];
      M.fused[1] = Q.fused[1];
      M.vec_off = Q.vec_off;
      M.vec_entries = Q.vec_entries;
      M.index_entries = Q.index_entries;
    }
    I.shape.n = p->F.n;
    I.shape.m = p->F.m;
    I.shape.L = p->F.L;
    I.shape.cplx = p->F.cplx;
    for (int dir = 0; dir < 2; ++dir) {
      I.desc_off[dir].resize(I.L + 2);
      for (int s = 0; s < I.L + 2; ++s) I.desc_off[dir][s] = p->P.st[s].dir[dir].desc_off;
    }
    img = align256(img + I.image_bytes);
    for (const Stage& S : p->P.st)
      for (int dir = 0; dir < 2; ++dir) {
        max_ld = std::max(max_ld, S.dir[dir].max_ld);
        max_rows = std::max(max_rows, S.dir[dir].max_item_rows);
        max_row_bytes = std::max<int64_t>(max_row_bytes, S.dir[dir].max_ld * I.es);
      }
  }
  // shared-memory layout for every item: 32 KB slots (or the widest row), RT 8, complex
  B.slot_bytes = int(std::max<int64_t>(32 * 1024, (max_row_bytes + 127) / 128 * 128));
  B.ldx_max = int((max_ld + 3) / 4 * 4);  // 16-byte rows of staged inputs for real and complex items
  B.rows_max = int(max_rows);
  B.nslot = 0;
  for (int ns = 3; ns >= 1 && !B.nslot; --ns)
    if (batch_smem(B.slot_bytes, ns, B.ldx_max, B.rows_max) <= 227 * 1024) B.nslot = ns;
  if (!B.nslot) fail(MHT_ERR_UNSUPPORTED, "a batch block needs more shared memory than an SM has");

  // records and the work list, phase-major so that each instance's phase k precedes k+1
  int maxph = 0;
  for (const BatchInst& I : B.inst) maxph = std::max(maxph, I.L + 2);
  int nctr = 0;
  for (int dir = 0; dir < 2; ++dir) {
    B.recs[dir].clear();
    B.items[dir].clear();
    for (BatchInst& I : B.inst) {
      I.rec_base[dir] = int(B.recs[dir].size());
      I.ctr_base[dir] = nctr;
      nctr += I.L + 2;
      B.recs[dir].resize(B.recs[dir].size() + I.L + 2);
    }
    std::vector<int> count_of(B.recs[dir].size(), 0);
    for (int ph = 0; ph < maxph; ++ph)
      for (int i = 0; i < count; ++i) {
        BatchInst& I = B.inst[i];
        if (ph >= I.L + 2) continue;
        const int s = dir == 0 ? ph : I.L + 1 - ph;  // stage of this phase
        const StageDir& D = I.plan->P.st[s].dir[dir];
        const MhtItem* src = reinterpret_cast<const MhtItem*>(I.plan->P.image.data() + D.items_off);
        const int rec = I.rec_base[dir] + ph;
        for (int64_t k = 0; k < D.nitems; ++k) {
          const MhtItem& it = src[k];
          B.items[dir].push_back({rec, it.blk, it.start, it.count | (it.sib ? int(0x80000000u) : 0)});
        }
        count_of[rec] = int(D.nitems);
      }
    for (BatchInst& I : B.inst)
      for (int ph = 0; ph < I.L + 2; ++ph) {
        MhtBatchRec& r = B.recs[dir][I.rec_base[dir] + ph];
        std::memset(&r, 0, sizeof r);
        const int s = dir == 0 ? ph : I.L + 1 - ph;
        r.nrhs = int(I.nrhs);
        r.cplx = I.cplx ? 1 : 0;
        r.mode = dir == 0 ? (s == I.L + 1 ? 2 : 0) : (s == I.L + 1 ? 3 : 1);
        r.done_ctr = I.ctr_base[dir] + ph;
        r.wait_ctr = ph == 0 ? -1 : I.ctr_base[dir] + ph - 1;
        r.wait_count = ph == 0 ? 0u : unsigned(count_of[I.rec_base[dir] + ph - 1]);
      }
  }
  if (B.items[0].size() > size_t(1) << 30 || B.items[1].size() > size_t(1) << 30)
    fail(MHT_ERR_UNSUPPORTED, "too many work items in one batch");
  B.recs_off[0] = img;
  B.recs_off[1] = align256(B.recs_off[0] + B.recs[0].size() * sizeof(MhtBatchRec));
  B.items_off[0] = align256(B.recs_off[1] + B.recs[1].size() * sizeof(MhtBatchRec));
  B.items_off[1] = align256(B.items_off[0] + B.items[0].size() * sizeof(MhtBItem));
  B.image_bytes = align256(B.items_off[1] + B.items[1].size() * sizeof(MhtBItem));

  size_t ws = 0;
  for (BatchInst& I : B.inst) {
    I.ws_off = ws;
    I.region_bytes = align256(size_t(std::max<int64_t>(I.vec_off.back(), 1)) * I.nrhs * I.es);
    // a full per-plan workspace (its first three regions are the level vectors the persistent
    // kernel uses), so that the tensor-core form can run each instance's own apply in place
    I.ws_bytes = align256(I.meta.workspace_bytes(I.nrhs, I.n, I.m));
    ws += I.ws_bytes;
  }
  B.counters_off = ws;
  B.nctr = nctr;
  B.counter_bytes = align256((size_t(2) + nctr) * sizeof(unsigned));
  B.status_off = B.counters_off + B.counter_bytes;
  B.ws_bytes = B.status_off + 256;
  batch_validate(B);
}

// The persistent batch kernel claims items in ticket (list) order and lets an item wait until
// the completion counter of its dependency reaches the dependency's item count.  That ends
// without co-residency only if every dependency's items come earlier in the list; this checks
// it, with the counters' uniqueness and the wait counts, before anything reaches the GPU.
void batch_validate(const mht_batch& B) {
  auto bad = [](const char* what) { fail(MHT_ERR_FORMAT, std::string("batch layout: ") + what); };
  for (int dir = 0; dir < 2; ++dir) {
    const std::vector<MhtBatchRec>& R = B.recs[dir];
    const std::vector<MhtBItem>& I = B.items[dir];
    const size_t nr = R.size();
    std::vector<int64_t> first(nr, INT64_MAX), last(nr, -1), count(nr, 0);
    for (size_t k = 0; k < I.size(); ++k) {
      const int r = I[k].rec;
      if (r < 0 || size_t(r) >= nr) bad("item record out of range");
      if ((I[k].count_sib & 0x7fffffff) > B.rows_max || I[k].start < 0 || I[k].blk < 0) bad("item rows");
      first[size_t(r)] = std::min<int64_t>(first[size_t(r)], int64_t(k));
      last[size_t(r)] = int64_t(k);
      ++count[size_t(r)];
    }
    std::vector<int> rec_of(size_t(B.nctr), -1);
    for (size_t r = 0; r < nr; ++r) {
      const int c = R[r].done_ctr;
      if (c < 0 || c >= B.nctr || rec_of[size_t(c)] != -1) bad("completion counters");
      rec_of[size_t(c)] = int(r);
    }
    for (size_t r = 0; r < nr; ++r) {
      if (R[r].wait_ctr < 0) {
        if (R[r].wait_count != 0) bad("wait count without a dependency");
        continue;
      }
      if (R[r].wait_ctr >= B.nctr || rec_of[size_t(R[r].wait_ctr)] < 0) bad("dependency counter");
      const size_t d = size_t(rec_of[size_t(R[r].wait_ctr)]);
      if (d == r || int64_t(R[r].wait_count) != count[d]) bad("wait count differs from the dependency's items");
      if (count[r] > 0 && count[d] > 0 && last[d] >= first[r]) bad("a dependency's items follow its dependent's");
    }
  }
}

// Fills the device addresses of every record (after binding; c / f after set_io).
void batch_fill_records(mht_batch& B) {
  const uint64_t img = reinterpret_cast<uint64_t>(B.image_dev);
  const uint64_t ws = reinterpret_cast<uint64_t>(B.ws_dev);
  for (int i = 0; i < B.n; ++i) {
    const BatchInst& I = B.inst[i];
    const uint64_t base = img + I.image_off;
    const long long nr = I.nrhs;
    auto lvl = [&](int region, int l) -> uint64_t {
      return ws + I.ws_off + size_t(region) * I.region_bytes + uint64_t(I.vec_off[l]) * nr * I.es;
    };
    for (int dir = 0; dir < 2; ++dir)
      for (int ph = 0; ph < I.L + 2; ++ph) {
        MhtBatchRec& r = B.recs[dir][I.rec_base[dir] + ph];
        const int s = dir == 0 ? ph : I.L + 1 - ph;
        r.data = base + I.data_off;
        r.idx = base + I.index_off;
        r.desc = base + I.desc_off[dir][s];
        r.perm = base + I.perm_off;
        r.wts = base + I.weights_off;
        r.in1 = r.out1 = 0;
        if (dir == 0) {
          r.in0 = s == 0 ? I.c : lvl(0, s - 1);
          r.is_e = s == 0 ? 1 : nr;
          r.is_k = s == 0 ? I.ldc : 1;
          r.out0 = s == I.L + 1 ? I.f : lvl(0, s);
          r.os_e = s == I.L + 1 ? 1 : nr;
          r.os_k = s == I.L + 1 ? I.ldf : 1;
        } else if (s == I.L + 1) {
          r.in0 = I.f;
          r.is_e = 1;
          r.is_k = I.ldf;
          r.out0 = lvl(1, I.L);
          r.os_e = nr;
          r.os_k = 1;
        } else {
          r.in0 = lvl(1, s);
          r.in1 = s == I.L ? 0 : lvl(2, s);
          r.is_e = nr;
          r.is_k = 1;
          r.out0 = s == 0 ? I.c : lvl(1, s - 1);
          r.out1 = s == 0 ? I.c : lvl(2, s - 1);
          r.os_e = s == 0 ? 1 : nr;
          r.os_k = s == 0 ? I.ldc : 1;
        }
      }
  }
}

BatchLaunch batch_launch_desc(const mht_batch& B, int dir, bool weighted) {
  BatchLaunch b{};
  b.recs = B.image_dev + B.recs_off[dir];
  b.items = B.image_dev + B.items_off[dir];
  b.nitems = int(B.items[dir].size());
  unsigned* ctr = reinterpret_cast<unsigned*>(B.ws_dev + B.counters_off);
  b.ticket = ctr;
  b.abort = ctr + 1;
  b.done = ctr + 2;
  b.counters = ctr;
  b.counter_bytes = B.counter_bytes;
  b.status = reinterpret_cast<unsigned*>(B.ws_dev + B.status_off);
  b.use_wts = weighted ? 1 : 0;
  b.slot_bytes = B.slot_bytes;
  b.nslot = B.tuned_nslot > 0 ? B.tuned_nslot : B.nslot;
  b.per_sm = B.tuned_per_sm;
  b.ldx_max = B.ldx_max;
  b.rows_max = B.rows_max;
  return b;
}

}  // namespace mht

mht_batch::~mht_batch() {
  for (auto*& g : graphs) {
    mht::batch_graph_destroy(g);
    g = nullptr;
  }
  for (auto*& g : tc) {
    mht::tc_group_destroy(g);
    g = nullptr;
  }
}
