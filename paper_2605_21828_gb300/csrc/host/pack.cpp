// Packing of a factorization into the device image (layout in ../layout.h).
//
// Every stored matrix is laid out row-major with rows padded to 16 bytes, in two
// orientations: as synthesis applies it (T~ is r x K', U_tau is |tau| x r_L) and as the
// adjoint applies it (conj(T~)^T is K' x r, conj(U_tau)^T is r_L x |tau|).  With both
// orientations each direction is a set of independent row-times-vector products over
// contiguous rows, split into work items (block, row range) of about kTileBytes so a CTA
// stages one item's rows into shared memory with a single bulk copy.  Index lists are
// absolute (level 0 composes the frequency-tree permutation, levels >= 1 add the offset of
// the input pair), so kernels gather without further indirection.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>

#include "internal.h"

namespace mht {
namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr size_t kTileBytes = 512 * 1024;   // target matrix bytes per per-stage work item
constexpr size_t kMinTileBytes = 32 * 1024; // smallest target (stages with little data)
constexpr size_t kResidentCtas = 608;       // 4 CTAs on each of 152 SMs
constexpr size_t kItemsPerCta = 4;
constexpr int kItemRows = 512;               // and at most this many rows
constexpr size_t kPItemBytes = 256 * 1024;  // largest persistent work item
constexpr int kPItemRows = 1024;             // and at most this many rows (staged per item)
constexpr size_t kSlotBytes = 32 * 1024;    // ring slot of the persistent kernel

}  // namespace

size_t Packed::ws_vec_bytes(int64_t nrhs) const {
  return align_up(size_t(std::max<int64_t>(vec_entries, 1)) * nrhs * elem_bytes, 256);
}

size_t Packed::ws_counters_offset(int64_t nrhs, int64_t n, int64_t m) const {
  const size_t sc = align_up(size_t(m) * nrhs * elem_bytes, 256);
  const size_t sf = align_up(size_t(n) * nrhs * elem_bytes, 256);
  return 3 * ws_vec_bytes(nrhs) + sc + sf;
}

size_t Packed::status_offset(int64_t nrhs, int64_t n, int64_t m) const {
  // counters: per direction (L+2) * nb completion counts, then two queue heads
  const size_t cnt = align_up((size_t(2) * (L + 2) * nb + 2) * sizeof(unsigned), 256);
  return ws_counters_offset(nrhs, n, m) + cnt;
}

size_t Packed::workspace_bytes(int64_t nrhs, int64_t n, int64_t m) const {
  return status_offset(nrhs, n, m) + 256;
}

void pack(const Factorization& F, bool fp64, Packed& P) {
  P = Packed();
  P.fp64 = fp64;
  P.cplx = F.cplx;
  const int W = F.cplx ? 2 : 1;
  const int sb = fp64 ? 8 : 4;             // bytes of one real scalar
  const int es = sb * W;
  P.elem_bytes = es;
  const int E = 16 / es;                    // elements per 16-byte vector
  const int L = F.L;
  const int64_t nb = F.nblk();
  P.L = L;
  P.nb = nb;
  const int nst = L + 2;
  P.st.assign(nst, Stage());
  auto pad = [&](int64_t c) { return (c + E - 1) / E * E; };

  // butterfly-vector offsets per level
  std::vector<std::vector<int64_t>> off(L + 1, std::vector<int64_t>(nb + 1, 0));
  for (int l = 0; l <= L; ++l)
    for (int64_t b = 0; b < nb; ++b) off[l][b + 1] = off[l][b] + F.lv[l][b].r;
  P.vec_off.assign(L + 2, 0);
  for (int l = 0; l <= L; ++l) {
    if (off[l][nb] > INT32_MAX) fail(MHT_ERR_UNSUPPORTED, "a butterfly level has more than 2^31 - 1 entries");
    P.vec_off[l + 1] = P.vec_off[l] + off[l][nb];
  }
  P.vec_entries = P.vec_off[L + 1];

  // descriptors for both directions; matrix element offsets run synthesis data first
  // (stages 0..L+1), then adjoint data (stages L+1..0)
  std::vector<std::vector<MhtBlockDesc>> desc[2];
  desc[0].assign(nst, std::vector<MhtBlockDesc>(nb));
  desc[1].assign(nst, std::vector<MhtBlockDesc>(nb));
  int64_t elem = 0, ient = 0;
  for (int s = 0; s < nst; ++s) {
    Stage& S = P.st[s];
    S.nblocks = nb;
    const int64_t start = elem;
    for (int64_t b = 0; b < nb; ++b) {
      MhtBlockDesc& d = desc[0][s][b];
      if (s <= L) {
        const Block& B = F.lv[s][b];
        d.rows = B.r;
        d.cols = B.K - B.r;
        if (ient + B.K > INT32_MAX) fail(MHT_ERR_UNSUPPORTED, "more than 2^31 - 1 interpolation indices");
        d.idx_off = int(ient);
        d.out_off = int(off[s][b]);
        d.in_off = (s == 0) ? int(F.mode_off[b]) : int(off[s - 1][F.pair_index(s, b)]);
        ient += B.K;
        S.max_rank = std::max<int64_t>(S.max_rank, B.r);
      } else {
        d.rows = int(F.leaf_rows(b));
        d.cols = F.lv[L][b].r;
        d.idx_off = -1;
        d.out_off = int(F.space_off[b]);
        d.in_off = int(off[L][b]);
        S.max_rank = std::max<int64_t>(S.max_rank, d.cols);
      }
      d.ldt = int(pad(d.cols));
      d.t_off = elem;
      elem += int64_t(d.rows) * d.ldt;
      S.t_entries += int64_t(d.rows) * d.cols;
      S.dir[0].max_ld = std::max<int64_t>(S.dir[0].max_ld, d.ldt);
    }
    S.dir[0].data_bytes = size_t(elem - start) * es;
    S.in_entries = (s == 0) ? F.m : off[s - 1][nb];
    S.out_entries = (s <= L) ? off[s][nb] : F.n;
  }
  for (int s = nst - 1; s >= 0; --s) {
    Stage& S = P.st[s];
    const int64_t start = elem;
    for (int64_t b = 0; b < nb; ++b) {
      const MhtBlockDesc& d0 = desc[0][s][b];
      MhtBlockDesc& d = desc[1][s][b];
      d = d0;
      d.rows = d0.cols;  // transposed
      d.cols = d0.rows;
      d.ldt = int(pad(d.cols));
      d.t_off = elem;
      elem += int64_t(d.rows) * d.ldt;
      S.dir[1].max_ld = std::max<int64_t>(S.dir[1].max_ld, d.ldt);
    }
    S.dir[1].data_bytes = size_t(elem - start) * es;
  }
  P.index_entries = ient;

  // algorithmic bytes per single-RHS launch: matrices (unpadded), indices, descriptors,
  // gathered inputs and written outputs (the same for both directions)
  for (int s = 0; s < nst; ++s) {
    Stage& S = P.st[s];
    if (s <= L) {
      int64_t sumk = 0, sumr = 0;
      for (int64_t b = 0; b < nb; ++b) { sumk += F.lv[s][b].K; sumr += F.lv[s][b].r; }
      S.alg_bytes = size_t(S.t_entries) * es + size_t(sumk) * 4 + size_t(nb) * sizeof(MhtBlockDesc) +
                    size_t(sumk + sumr) * es;
    } else {
      int64_t sumr = 0;
      for (int64_t t = 0; t < nb; ++t) sumr += F.lv[L][t].r;
      S.alg_bytes = size_t(S.t_entries) * es + size_t(nb) * sizeof(MhtBlockDesc) + size_t(sumr) * es +
                    size_t(F.n) * (4 + es);
    }
  }

  // work items: row ranges of about kTileBytes, smaller in stages too small to give every
  // resident CTA of a persistent launch (about kResidentCtas) several items to stream
  std::vector<std::vector<MhtItem>> items[2];
  items[0].assign(nst, {});
  items[1].assign(nst, {});
  for (int dir = 0; dir < 2; ++dir)
    for (int s = 0; s < nst; ++s) {
      StageDir& D = P.st[s].dir[dir];
      const size_t stage_bytes = size_t(P.st[s].t_entries) * es;
      const size_t tile = std::max(kMinTileBytes, std::min(kTileBytes, stage_bytes / (kItemsPerCta * kResidentCtas)));
      for (int64_t b = 0; b < nb; ++b) {
        const MhtBlockDesc& d = desc[dir][s][b];
        const int sib = (dir == 1 && s >= 1 && s <= L) ? int((b >> (L - s)) & 1) : 0;
        const size_t rowbytes = size_t(d.ldt) * es;
        const int rpi = int(std::min<size_t>(kItemRows, std::max<size_t>(1, rowbytes ? tile / rowbytes
                                                                                       : size_t(kItemRows))));
        if (d.rows == 0) {
          // adjoint of an ID block without T~ (full rank): still copies the skeleton out
          if (dir == 1 && s <= L && d.cols > 0) items[dir][s].push_back({int(b), 0, 0, sib});
          continue;
        }
        for (int r0 = 0; r0 < d.rows; r0 += rpi) {
          const int cnt = std::min(rpi, d.rows - r0);
          items[dir][s].push_back({int(b), r0, cnt, sib});
          D.max_item_rows = std::max<int64_t>(D.max_item_rows, cnt);
        }
      }
      D.nitems = int64_t(items[dir][s].size());
    }

  // tensor-core work items: 128-row tiles (skeleton-only items as for the SIMT lists)
  std::vector<std::vector<MhtItem>> tcitems[2];
  for (int dir = 0; dir < 2; ++dir) {
    tcitems[dir].assign(nst, {});
    for (int s = 0; s < nst; ++s) {
      for (int64_t b = 0; b < nb; ++b) {
        const MhtBlockDesc& d = desc[dir][s][b];
        const int sib = (dir == 1 && s >= 1 && s <= L) ? int((b >> (L - s)) & 1) : 0;
        if (d.rows == 0) {
          if (dir == 1 && s <= L && d.cols > 0) tcitems[dir][s].push_back({int(b), 0, 0, sib});
          continue;
        }
        for (int r0 = 0; r0 < d.rows; r0 += 128)
          tcitems[dir][s].push_back({int(b), r0, std::min(128, d.rows - r0), sib});
      }
      // longest first (K columns stream per tile): the persistent kernel deals tiles out in a
      // fixed stride, so this order balances the CTAs
      const std::vector<MhtBlockDesc>& dd = desc[dir][s];
      std::stable_sort(tcitems[dir][s].begin(), tcitems[dir][s].end(), [&](const MhtItem& a, const MhtItem& b) {
        return (a.count > 0 ? dd[a.blk].cols : -1) > (b.count > 0 ? dd[b.blk].cols : -1);
      });
      P.st[s].dir[dir].tc_nitems = int64_t(tcitems[dir][s].size());
    }
  }

  // persistent work lists: dependency order (synthesis 0..L+1, analysis L+1..0), items of
  // at most kPItemBytes, and the number of items per (stage, block) as completion targets
  std::vector<MhtPItem> pitems[2];
  std::vector<int32_t> targets[2];
  for (int dir = 0; dir < 2; ++dir) {
    targets[dir].assign(size_t(nst) * nb, 0);
    FusedDir& FD = P.fused[dir];
    FD.slot_bytes = kSlotBytes;
    FD.stage_first.assign(nst + 1, 0);
    for (int k = 0; k < nst; ++k) {
      FD.stage_first[k] = int64_t(pitems[dir].size());
      const int s = dir == 0 ? k : nst - 1 - k;
      for (int64_t b = 0; b < nb; ++b) {
        const MhtBlockDesc& d = desc[dir][s][b];
        const size_t rowbytes = size_t(d.ldt) * es;
        FD.slot_bytes = std::max(FD.slot_bytes, (rowbytes + 127) / 128 * 128);
        FD.max_ld = std::max<int64_t>(FD.max_ld, d.ldt);
        int n_it = 0;
        if (d.rows == 0) {
          if (dir == 1 && s <= L && d.cols > 0) {
            pitems[dir].push_back({s, int(b), 0, 0});
            n_it = 1;
          }
        } else {
          const int rpi = int(std::min<size_t>(kPItemRows, std::max<size_t>(1, rowbytes ? kPItemBytes / rowbytes
                                                                                         : size_t(kPItemRows))));
          for (int r0 = 0; r0 < d.rows; r0 += rpi, ++n_it) pitems[dir].push_back({s, int(b), r0, std::min(rpi, d.rows - r0)});
        }
        targets[dir][size_t(s) * nb + b] = n_it;
      }
    }
    FD.nitems = int64_t(pitems[dir].size());
    FD.stage_first[nst] = FD.nitems;
    for (const MhtPItem& it : pitems[dir]) FD.max_item_rows = std::max<int64_t>(FD.max_item_rows, it.count);
  }

  // assemble the image
  size_t pos = align_up(size_t(elem) * es, 256);
  P.data_off = 0;
  P.index_off = pos;
  pos = align_up(pos + size_t(ient) * 4, 256);
  for (int dir = 0; dir < 2; ++dir) {
    P.fused[dir].desc_all_off = pos;  // stage-major, contiguous over the stages
    for (int s = 0; s < nst; ++s) P.st[s].dir[dir].desc_off = pos + size_t(s) * nb * sizeof(MhtBlockDesc);
    pos = align_up(pos + size_t(nst) * nb * sizeof(MhtBlockDesc), 256);
    for (int s = 0; s < nst; ++s) {
      P.st[s].dir[dir].items_off = pos;
      pos = align_up(pos + items[dir][s].size() * sizeof(MhtItem), 256);
    }
    for (int s = 0; s < nst; ++s) {
      P.st[s].dir[dir].tc_items_off = pos;
      pos = align_up(pos + tcitems[dir][s].size() * sizeof(MhtItem), 256);
    }
    P.fused[dir].targets_off = pos;
    pos = align_up(pos + targets[dir].size() * 4, 256);
    P.fused[dir].items_off = pos;
    pos = align_up(pos + pitems[dir].size() * sizeof(MhtPItem), 256);
  }
  P.vecoff_off = pos;
  pos = align_up(pos + P.vec_off.size() * 8, 256);
  P.perm_off = pos;
  pos = align_up(pos + size_t(F.n) * 4, 256);
  P.weights_off = pos;
  pos = align_up(pos + size_t(F.n) * sb, 256);
  P.tmap_off = pos;
  P.tmap_bytes = fp64 ? 0 : size_t(2) * nst * nb * 128;
  pos = align_up(pos + P.tmap_bytes, 256);
  if (const size_t cap = host_alloc_limit(); cap && pos > cap) throw std::bad_alloc();  // testing aid
  P.image.assign(pos, 0);
  uint8_t* img = P.image.data();

  // element (i, j) of a row-major matrix with W scalars per element; conj negates imag
  auto store = [&](int64_t eoff, int64_t i, int64_t j, int ldt, const double* v, bool conj) {
    for (int c = 0; c < W; ++c) {
      const double x = (conj && c == 1) ? -v[c] : v[c];
      const size_t at = size_t((eoff + i * ldt + j) * W + c);
      if (fp64) reinterpret_cast<double*>(img)[at] = x;
      else reinterpret_cast<float*>(img)[at] = float(x);
    }
  };
  int32_t* idx = reinterpret_cast<int32_t*>(img + P.index_off);
  // every (stage, block) writes its own matrices and index list: blocks in parallel, each
  // matrix and its transpose in 32 x 32 tiles
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t sb = 0; sb < int64_t(nst) * nb; ++sb) {
    const int s = int(sb / nb);
    const int64_t b = sb % nb;
    const MhtBlockDesc& d = desc[0][s][b];
    const MhtBlockDesc& dt = desc[1][s][b];
    const double* src = (s <= L) ? F.lv[s][b].T.data() : F.U[b].data();
    for (int64_t i0 = 0; i0 < d.rows; i0 += 32)
      for (int64_t j0 = 0; j0 < d.cols; j0 += 32)
        for (int64_t i = i0; i < std::min<int64_t>(i0 + 32, d.rows); ++i)
          for (int64_t j = j0; j < std::min<int64_t>(j0 + 32, d.cols); ++j) {
            const double* v = src + (i * d.cols + j) * W;
            store(d.t_off, i, j, d.ldt, v, false);
            store(dt.t_off, j, i, dt.ldt, v, true);
          }
    if (s <= L) {
      const Block& B = F.lv[s][b];
      for (int j = 0; j < B.K; ++j) {
        const int64_t loc = B.perm[j];
        idx[d.idx_off + j] = int32_t(s == 0 ? F.mode_perm[F.mode_off[b] + loc] : int64_t(d.in_off) + loc);
      }
    }
  }
  for (int dir = 0; dir < 2; ++dir) {
    for (int s = 0; s < nst; ++s) {
      std::memcpy(img + P.st[s].dir[dir].desc_off, desc[dir][s].data(), size_t(nb) * sizeof(MhtBlockDesc));
      if (!items[dir][s].empty())
        std::memcpy(img + P.st[s].dir[dir].items_off, items[dir][s].data(), items[dir][s].size() * sizeof(MhtItem));
    }
    for (int s = 0; s < nst; ++s)
      if (!tcitems[dir][s].empty())
        std::memcpy(img + P.st[s].dir[dir].tc_items_off, tcitems[dir][s].data(),
                    tcitems[dir][s].size() * sizeof(MhtItem));
    std::memcpy(img + P.fused[dir].targets_off, targets[dir].data(), targets[dir].size() * 4);
    if (!pitems[dir].empty())
      std::memcpy(img + P.fused[dir].items_off, pitems[dir].data(), pitems[dir].size() * sizeof(MhtPItem));
  }
  std::memcpy(img + P.vecoff_off, P.vec_off.data(), P.vec_off.size() * 8);
  int32_t* perm = reinterpret_cast<int32_t*>(img + P.perm_off);
  for (int64_t i = 0; i < F.n; ++i) perm[i] = int32_t(F.space_perm[i]);
  for (int64_t i = 0; i < F.n; ++i) {
    const double w = F.weights.empty() ? 1.0 : F.weights[i];
    if (fp64) reinterpret_cast<double*>(img + P.weights_off)[i] = w;
    else reinterpret_cast<float*>(img + P.weights_off)[i] = float(w);
  }
  validate_packed(P, F.n, F.m);
}

// Every address the apply kernels form from the image must stay inside its buffer; this
// replays their accesses (the table above the row kernel: matrix rows, gathered indices,
// output positions, permutation entries, work-item row ranges) on the host.
void validate_packed(const Packed& P, int64_t n, int64_t m) {
  auto bad = [](const char* what) { fail(MHT_ERR_FORMAT, std::string("packed plan: ") + what); };
  const size_t isz = P.image.size();
  const int L = P.L;
  const int64_t nb = P.nb, es = P.elem_bytes;
  if (int(P.st.size()) != L + 2 || int(P.vec_off.size()) != L + 2) bad("stage count");
  for (int l = 0; l <= L; ++l)
    if (P.vec_off[l + 1] < P.vec_off[l]) bad("level vector offsets");
  auto len = [&](int l) { return P.vec_off[l + 1] - P.vec_off[l]; };
  if (P.index_off < P.data_off || P.index_off + size_t(P.index_entries) * 4 > isz) bad("index region");
  if (P.perm_off + size_t(n) * 4 > isz) bad("permutation region");
  const int32_t* idx = reinterpret_cast<const int32_t*>(P.image.data() + P.index_off);
  const int32_t* perm = reinterpret_cast<const int32_t*>(P.image.data() + P.perm_off);
  {
    std::vector<uint8_t> seen(size_t(n), 0);
    for (int64_t i = 0; i < n; ++i) {
      if (perm[i] < 0 || perm[i] >= n || seen[size_t(perm[i])]) bad("space permutation");
      seen[size_t(perm[i])] = 1;
    }
  }
  auto desc_at = [&](int dir, int s) {
    const size_t off = P.st[s].dir[dir].desc_off;
    if (off + size_t(nb) * sizeof(MhtBlockDesc) > isz) bad("descriptor region");
    return reinterpret_cast<const MhtBlockDesc*>(P.image.data() + off);
  };
  for (int dir = 0; dir < 2; ++dir)
    for (int s = 0; s <= L + 1; ++s) {
      const MhtBlockDesc* D = desc_at(dir, s);
      for (int64_t b = 0; b < nb; ++b) {
        const MhtBlockDesc& d = D[b];
        if (d.rows < 0 || d.cols < 0 || d.ldt < d.cols || (int64_t(d.ldt) * es) % 16 != 0 || d.t_off < 0 ||
            (d.t_off * es) % 16 != 0 || size_t(d.t_off + int64_t(d.rows) * d.ldt) * es > P.index_off)
          bad("matrix extent or alignment");
        if (s <= L) {
          const int64_t K = int64_t(d.rows) + d.cols;            // r + (K - r) in either direction
          const int64_t r = dir == 0 ? d.rows : d.cols;
          const int64_t in_len = s == 0 ? m : len(s - 1);
          if (d.idx_off < 0 || d.idx_off + K > P.index_entries) bad("index list extent");
          for (int64_t j = 0; j < K; ++j)
            if (idx[d.idx_off + j] < 0 || idx[d.idx_off + j] >= in_len) bad("gathered index out of range");
          if (d.out_off < 0 || d.out_off + r > len(s)) bad("output position out of range");
          if (d.in_off < 0 || d.in_off + K > in_len) bad("input range");
        } else {
          const int64_t pts = dir == 0 ? d.rows : d.cols, rl = dir == 0 ? d.cols : d.rows;
          if (d.out_off < 0 || d.out_off + pts > n) bad("space leaf range");
          if (d.in_off < 0 || d.in_off + rl > len(L)) bad("level-L vector range");
        }
      }
      auto check_items = [&](size_t off, int64_t count) {
        if (off + size_t(count) * sizeof(MhtItem) > isz) bad("work-item region");
        const MhtItem* it = reinterpret_cast<const MhtItem*>(P.image.data() + off);
        for (int64_t k = 0; k < count; ++k) {
          if (it[k].blk < 0 || it[k].blk >= nb || it[k].start < 0 || it[k].count < 0 || it[k].sib < 0 || it[k].sib > 1)
            bad("work item");
          const MhtBlockDesc& d = D[it[k].blk];
          if (it[k].start + int64_t(it[k].count) > d.rows || (it[k].count == 0 && d.rows != 0))
            bad("work-item rows");
        }
      };
      check_items(P.st[s].dir[dir].items_off, P.st[s].dir[dir].nitems);
      check_items(P.st[s].dir[dir].tc_items_off, P.st[s].dir[dir].tc_nitems);
    }
  for (int dir = 0; dir < 2; ++dir) {
    const FusedDir& FD = P.fused[dir];
    if (FD.items_off + size_t(FD.nitems) * sizeof(MhtPItem) > isz ||
        FD.targets_off + size_t(L + 2) * nb * 4 > isz)
      bad("persistent work-list region");
    const MhtPItem* it = reinterpret_cast<const MhtPItem*>(P.image.data() + FD.items_off);
    const int32_t* tgt = reinterpret_cast<const int32_t*>(P.image.data() + FD.targets_off);
    std::vector<int32_t> per(size_t(L + 2) * nb, 0);
    for (int64_t k = 0; k < FD.nitems; ++k) {
      if (it[k].stage < 0 || it[k].stage > L + 1 || it[k].blk < 0 || it[k].blk >= nb || it[k].start < 0 ||
          it[k].count < 0)
        bad("persistent work item");
      const MhtBlockDesc& d = desc_at(dir, it[k].stage)[it[k].blk];
      if (it[k].start + int64_t(it[k].count) > d.rows) bad("persistent work-item rows");
      ++per[size_t(it[k].stage) * nb + it[k].blk];
    }
    for (size_t k = 0; k < per.size(); ++k)
      if (per[k] != tgt[k]) bad("completion targets");
  }
}

}  // namespace mht
