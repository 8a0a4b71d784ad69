// Cell-list geometry of the pair search (Sec. 5) and the scratch layout of the
// standalone search, shared by a run, ibm_lbm_pair_search (caller scratch) and
// ibm_lbm_pair_search_static (the library's fixed array), so all three bucket the
// centres alike.
//
// Cells: floor(L / reach) per axis, at least one, so a cell side is >= reach = D_p +
// zeta and a pair lies in neighbouring cells (3^D of them).  A periodic axis with fewer
// than three cells keeps one (its neighbour scan would visit a cell twice).  The total
// is kept at most kMaxSearchCells by merging cells on the axis with the most (a larger
// side keeps the search complete), so every cell index fits in an int and no byte
// count below can overflow.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace ibmlbm {

constexpr long long kMaxSearchCells = 1LL << 30;
constexpr size_t kPairScratchAlign = 256;

inline void cell_grid(int D, const double* L, const int* per, double reach, int* nc, double* H) {
  for (int k = 0; k < 3; ++k) {
    nc[k] = 1;
    H[k] = k < D ? L[k] : 1.0;
    if (k >= D) continue;
    const double c = std::floor(L[k] / reach);  // L <= 2^31 nodes: exact in a double
    nc[k] = c < 1.0 ? 1 : (c > 2147483647.0 ? 2147483647 : (int)c);
  }
  for (;;) {
    for (int k = 0; k < D; ++k)
      if (per[k] && nc[k] < 3) nc[k] = 1;
    const double cells = (double)nc[0] * nc[1] * nc[2];
    if (cells <= (double)kMaxSearchCells) break;
    int big = 0;
    for (int k = 1; k < D; ++k)
      if (nc[k] > nc[big]) big = k;
    nc[big] = nc[big] / 2 + (nc[big] & 1);  // ceil(nc / 2) without overflow
  }
  for (int k = 0; k < D; ++k) H[k] = L[k] / nc[k];
}

// Byte offsets of the search's lists in one scratch block (kPairScratchAlign-aligned
// pieces); ok = false if a size would not fit in size_t.
struct PairScratch {
  size_t cell_count, cell_ids, nbr, nbr_count, gt, status, total;
  int cell_cap;
  bool ok;
};

inline bool pair_scratch_take(size_t& off, size_t count, size_t elem, size_t& at) {
  size_t bytes;
  if (__builtin_mul_overflow(count, elem, &bytes)) return false;
  if (bytes == 0) bytes = 1;
  size_t end;
  if (__builtin_add_overflow(off, bytes, &end) ||
      __builtin_add_overflow(end, kPairScratchAlign - 1, &end))
    return false;
  at = off;
  off = end / kPairScratchAlign * kPairScratchAlign;
  return true;
}

inline PairScratch pair_scratch(int n, int kmax, const int* nc) {
  PairScratch p{};
  const long long ncells = (long long)nc[0] * nc[1] * nc[2];  // <= kMaxSearchCells
  p.cell_cap = cell_capacity(n, ncells);
  size_t off = 0, ids = 0;
  p.ok = !__builtin_mul_overflow((size_t)ncells, (size_t)p.cell_cap, &ids) &&
         pair_scratch_take(off, (size_t)ncells, sizeof(int), p.cell_count) &&
         pair_scratch_take(off, ids, sizeof(int), p.cell_ids) &&
         pair_scratch_take(off, (size_t)n * (size_t)kmax, sizeof(int), p.nbr) &&
         pair_scratch_take(off, (size_t)n, sizeof(int), p.nbr_count) &&
         pair_scratch_take(off, 2 * ((size_t)n + 1), sizeof(int), p.gt) &&
         pair_scratch_take(off, 1, sizeof(uint32_t), p.status);
  p.total = off;
  return p;
}

}  // namespace ibmlbm
