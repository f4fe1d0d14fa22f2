// CSR -> SELL-C-sigma packing (C = 32 rows per slice, one warp lane per row).
//
// Within a slice the entries are stored column-major (entry k of the slice's
// lane l at slice_ptr[s] + 32 k + l), so that a warp reading entry k of its 32
// rows touches one contiguous 256-byte (FP64) or 128-byte (FP32/int32) span.
// Rows of a slice are padded to the slice's longest row.
#include <algorithm>
#include <numeric>

#include "kes_internal.h"

namespace kes {

SellHost build_sell(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, int sigma) {
  SellHost s;
  s.n = n;
  s.nnz = row_ptr[n];
  s.n_slices = (n + kSliceC - 1) / kSliceC;
  std::vector<int32_t> perm;
  std::vector<int32_t> iperm;
  if (sigma > 1) {
    perm.resize(n);
    std::iota(perm.begin(), perm.end(), 0);
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
      const int64_t w1 = std::min<int64_t>(n, w0 + sigma);
      std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int32_t a, int32_t b) {
        return (row_ptr[a + 1] - row_ptr[a]) > (row_ptr[b + 1] - row_ptr[b]);
      });
    }
    bool identity = true;
    for (int64_t i = 0; i < n && identity; ++i) identity = perm[i] == i;
    if (identity) perm.clear();
  }
  if (!perm.empty()) {
    iperm.resize(n);
    for (int64_t i = 0; i < n; ++i) iperm[perm[i]] = static_cast<int32_t>(i);
  }
  auto old_row = [&](int64_t i) -> int64_t { return perm.empty() ? i : perm[i]; };

  s.slice_ptr.resize(s.n_slices + 1);
  s.slice_ptr[0] = 0;
  for (int64_t sl = 0; sl < s.n_slices; ++sl) {
    int64_t width = 0;
    for (int64_t l = 0; l < kSliceC; ++l) {
      const int64_t i = sl * kSliceC + l;
      if (i < n) width = std::max<int64_t>(width, row_ptr[old_row(i) + 1] - row_ptr[old_row(i)]);
    }
    s.slice_ptr[sl + 1] = s.slice_ptr[sl] + width * kSliceC;
  }
  s.nnz_pad = s.slice_ptr[s.n_slices];
  s.col.assign(s.nnz_pad, 0);
  s.val.assign(s.nnz_pad, 0.0);
  std::vector<std::pair<int32_t, double>> rowbuf;
  for (int64_t sl = 0; sl < s.n_slices; ++sl) {
    const int64_t base = s.slice_ptr[sl];
    const int64_t width = (s.slice_ptr[sl + 1] - base) / kSliceC;
    for (int64_t l = 0; l < kSliceC; ++l) {
      const int64_t i = sl * kSliceC + l;
      if (i >= n) {
        for (int64_t k = 0; k < width; ++k) s.col[base + k * kSliceC + l] = static_cast<int32_t>(n - 1);
        continue;
      }
      const int64_t r = old_row(i);
      rowbuf.clear();
      for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
        rowbuf.emplace_back(iperm.empty() ? col[p] : iperm[col[p]], val[p]);
      if (!iperm.empty()) std::sort(rowbuf.begin(), rowbuf.end(),
                                    [](const auto& a, const auto& b) { return a.first < b.first; });
      const int64_t len = static_cast<int64_t>(rowbuf.size());
      for (int64_t k = 0; k < width; ++k) {
        const int64_t at = base + k * kSliceC + l;
        if (k < len) {
          s.col[at] = rowbuf[k].first;
          s.val[at] = rowbuf[k].second;
        } else {
          s.col[at] = static_cast<int32_t>(i);
          s.val[at] = 0.0;
        }
      }
    }
  }
  s.perm = std::move(perm);
  return s;
}

}  // namespace kes
