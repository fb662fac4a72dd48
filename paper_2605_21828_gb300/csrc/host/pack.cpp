// Packing of a factorization into the device image (layout in ../layout.h).
//
// Every stored matrix is laid out row-major with rows padded to 16 bytes so that kernels
// stream it with aligned 128-bit loads; matrices follow each other in apply order, so one
// stage's data is one contiguous span.  Index lists are made absolute (level 0 composes the
// frequency-tree permutation, levels >= 1 add the offset of the input pair), so kernels
// gather without further indirection.  Work items split large blocks into row tiles
// (synthesis) and column tiles (analysis) of roughly equal byte counts.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace mht {
namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr size_t kItemBytes = 48 * 1024;   // target matrix bytes per synthesis work item
constexpr int kWarps = 8;                  // warps per CTA of the SIMT apply kernels

}  // namespace

size_t Packed::workspace_bytes(int64_t nrhs, int64_t n, int64_t m) const {
  const size_t vec = align_up(size_t(std::max<int64_t>(vec_entries, 1)) * nrhs * elem_bytes, 256);
  const size_t sc = align_up(size_t(m) * nrhs * elem_bytes, 256);
  const size_t sf = align_up(size_t(n) * nrhs * elem_bytes, 256);
  return 4 * vec + sc + sf + 256;
}

void pack(const Factorization& F, bool fp64, Packed& P) {
  P = Packed();
  P.fp64 = fp64;
  P.cplx = F.cplx;
  const int W = F.cplx ? 2 : 1;
  const int sb = fp64 ? 8 : 4;             // bytes of one real scalar
  P.elem_bytes = sb * W;
  const int E = 16 / P.elem_bytes;          // elements per 16-byte vector
  const int L = F.L;
  const int64_t nb = F.nblk();
  const int nst = L + 2;
  P.st.assign(nst, Stage());

  // vector offsets per level
  std::vector<std::vector<int64_t>> off(L + 1, std::vector<int64_t>(nb + 1, 0));
  for (int l = 0; l <= L; ++l)
    for (int64_t b = 0; b < nb; ++b) off[l][b + 1] = off[l][b] + F.lv[l][b].r;
  P.vec_entries = 0;
  for (int l = 0; l <= L; ++l) P.vec_entries = std::max(P.vec_entries, off[l][nb]);

  // data section sizes
  std::vector<std::vector<MhtBlockDesc>> desc(nst, std::vector<MhtBlockDesc>(nb));
  int64_t elem = 0;    // running element offset in [data]
  int64_t ient = 0;    // running offset in [index]
  for (int l = 0; l <= L; ++l) {
    Stage& S = P.st[l];
    S.nblocks = nb;
    S.in_entries = (l == 0) ? F.m : off[l - 1][nb];
    S.out_entries = off[l][nb];
    for (int64_t b = 0; b < nb; ++b) {
      const Block& B = F.lv[l][b];
      const int cols = B.K - B.r;
      const int ldt = int((cols + E - 1) / E * E);
      MhtBlockDesc& d = desc[l][b];
      d.t_off = elem;
      d.ldt = ldt;
      d.rows = B.r;
      d.cols = cols;
      d.idx_off = int(ient);
      d.out_off = int(off[l][b]);
      d.in_off = (l == 0) ? int(F.mode_off[b]) : int(off[l - 1][F.pair_index(l, b)]);
      elem += int64_t(B.r) * ldt;
      ient += B.K;
      S.t_entries += int64_t(B.r) * cols;
      S.max_k = std::max<int64_t>(S.max_k, B.K);
      S.max_rows = std::max<int64_t>(S.max_rows, B.r);
      S.max_cols = std::max<int64_t>(S.max_cols, cols);
    }
    S.data_bytes = size_t(elem - desc[l][0].t_off) * P.elem_bytes;
  }
  {
    Stage& S = P.st[L + 1];
    S.nblocks = nb;
    S.in_entries = off[L][nb];
    S.out_entries = F.n;
    const int64_t start = elem;
    for (int64_t t = 0; t < nb; ++t) {
      const int rows = int(F.leaf_rows(t));
      const int cols = F.lv[L][t].r;
      const int ldt = int((cols + E - 1) / E * E);
      MhtBlockDesc& d = desc[L + 1][t];
      d.t_off = elem;
      d.ldt = ldt;
      d.rows = rows;
      d.cols = cols;
      d.idx_off = -1;
      d.out_off = int(F.space_off[t]);
      d.in_off = int(off[L][t]);
      elem += int64_t(rows) * ldt;
      S.t_entries += int64_t(rows) * cols;
      S.max_k = std::max<int64_t>(S.max_k, rows);
      S.max_rows = std::max<int64_t>(S.max_rows, rows);
      S.max_cols = std::max<int64_t>(S.max_cols, cols);
    }
    S.data_bytes = size_t(elem - start) * P.elem_bytes;
  }
  P.index_entries = ient;
  // algorithmic bytes per single-RHS launch: matrices (unpadded), indices, descriptors,
  // gathered inputs and written outputs
  for (int l = 0; l <= L; ++l) {
    Stage& S = P.st[l];
    int64_t sumk = 0, sumr = 0;
    for (int64_t b = 0; b < nb; ++b) { sumk += F.lv[l][b].K; sumr += F.lv[l][b].r; }
    S.alg_bytes = size_t(S.t_entries) * P.elem_bytes + size_t(sumk) * 4 + size_t(nb) * sizeof(MhtBlockDesc) +
                  size_t(sumk + sumr) * P.elem_bytes;
  }
  {
    Stage& S = P.st[L + 1];
    int64_t sumr = 0;
    for (int64_t t = 0; t < nb; ++t) sumr += F.lv[L][t].r;
    S.alg_bytes = size_t(S.t_entries) * P.elem_bytes + size_t(nb) * sizeof(MhtBlockDesc) +
                  size_t(sumr) * P.elem_bytes + size_t(F.n) * (4 + P.elem_bytes);
  }

  // work items
  std::vector<std::vector<MhtItem>> isyn(nst), iadj(nst);
  const int cols_per_item = 32 * E * 2;  // two 16-byte vectors per lane
  for (int s = 0; s < nst; ++s) {
    Stage& S = P.st[s];
    S.cols_per_item = cols_per_item;
    int64_t maxldt = 0;
    for (int64_t b = 0; b < nb; ++b) maxldt = std::max<int64_t>(maxldt, desc[s][b].ldt);
    for (int64_t b = 0; b < nb; ++b) {
      const MhtBlockDesc& d = desc[s][b];
      const int64_t rowbytes = int64_t(std::max(d.ldt, E)) * P.elem_bytes;
      int rpi = int(std::max<int64_t>(kWarps, int64_t(kItemBytes) / rowbytes));
      rpi = (rpi + kWarps - 1) / kWarps * kWarps;
      for (int r0 = 0; r0 < d.rows; r0 += rpi)
        isyn[s].push_back({int(b), r0, std::min(rpi, d.rows - r0), 0});
      const bool id_stage = (s <= L);
      const int sib = (id_stage && s >= 1) ? int((b >> (L - s)) & 1) : 0;
      const int ncol_total = d.cols;
      const bool has_out = id_stage ? (d.rows + d.cols > 0) : (d.cols > 0);
      if (!has_out) continue;
      if (ncol_total == 0) {
        iadj[s].push_back({int(b), 0, 0, sib});
      } else {
        for (int c0 = 0; c0 < ncol_total; c0 += cols_per_item)
          iadj[s].push_back({int(b), c0, std::min(cols_per_item, ncol_total - c0), sib});
      }
    }
    S.rows_per_item = 0;
    S.nitems_syn = int64_t(isyn[s].size());
    S.nitems_adj = int64_t(iadj[s].size());
    (void)maxldt;
  }

  // assemble the image
  size_t pos = 0;
  P.data_off = 0;
  pos = align_up(size_t(elem) * P.elem_bytes, 256);
  P.index_off = pos;
  pos = align_up(pos + size_t(ient) * 4, 256);
  for (int s = 0; s < nst; ++s) {
    P.st[s].desc_off = pos;
    pos = align_up(pos + size_t(nb) * sizeof(MhtBlockDesc), 256);
    P.st[s].items_syn_off = pos;
    pos = align_up(pos + isyn[s].size() * sizeof(MhtItem), 256);
    P.st[s].items_adj_off = pos;
    pos = align_up(pos + iadj[s].size() * sizeof(MhtItem), 256);
  }
  P.perm_off = pos;
  pos = align_up(pos + size_t(F.n) * 4, 256);
  P.weights_off = pos;
  pos = align_up(pos + size_t(F.n) * sb, 256);
  P.image.assign(pos, 0);
  uint8_t* img = P.image.data();

  auto put = [&](int64_t eoff, const double* src, int64_t rows, int64_t cols, int ldt) {
    for (int64_t i = 0; i < rows; ++i)
      for (int64_t j = 0; j < cols; ++j)
        for (int c = 0; c < W; ++c) {
          const double v = src[(i * cols + j) * W + c];
          const size_t at = size_t((eoff + i * ldt + j) * W + c);
          if (fp64) reinterpret_cast<double*>(img)[at] = v;
          else reinterpret_cast<float*>(img)[at] = float(v);
        }
  };
  int32_t* idx = reinterpret_cast<int32_t*>(img + P.index_off);
  for (int l = 0; l <= L; ++l)
    for (int64_t b = 0; b < nb; ++b) {
      const Block& B = F.lv[l][b];
      const MhtBlockDesc& d = desc[l][b];
      put(d.t_off, B.T.data(), B.r, B.K - B.r, d.ldt);
      for (int j = 0; j < B.K; ++j) {
        const int64_t loc = B.perm[j];
        idx[d.idx_off + j] = int32_t(l == 0 ? F.mode_perm[F.mode_off[b] + loc] : int64_t(d.in_off) + loc);
      }
    }
  for (int64_t t = 0; t < nb; ++t) {
    const MhtBlockDesc& d = desc[L + 1][t];
    put(d.t_off, F.U[t].data(), d.rows, d.cols, d.ldt);
  }
  for (int s = 0; s < nst; ++s) {
    std::memcpy(img + P.st[s].desc_off, desc[s].data(), size_t(nb) * sizeof(MhtBlockDesc));
    if (!isyn[s].empty()) std::memcpy(img + P.st[s].items_syn_off, isyn[s].data(), isyn[s].size() * sizeof(MhtItem));
    if (!iadj[s].empty()) std::memcpy(img + P.st[s].items_adj_off, iadj[s].data(), iadj[s].size() * sizeof(MhtItem));
  }
  int32_t* perm = reinterpret_cast<int32_t*>(img + P.perm_off);
  for (int64_t i = 0; i < F.n; ++i) perm[i] = int32_t(F.space_perm[i]);
  for (int64_t i = 0; i < F.n; ++i) {
    const double w = F.weights.empty() ? 1.0 : F.weights[i];
    if (fp64) reinterpret_cast<double*>(img + P.weights_off)[i] = w;
    else reinterpret_cast<float*>(img + P.weights_off)[i] = float(w);
  }
}

}  // namespace mht
