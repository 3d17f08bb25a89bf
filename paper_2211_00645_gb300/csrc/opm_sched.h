// Work units of the fast projection and their static schedule onto the
// persistent CTAs.
#pragma once

#include <algorithm>
#include <cstdint>

#ifndef __CUDACC__
#define __align__(n) alignas(n)  // host-only builds of this header
#endif

namespace opm {

// Rows [ks, ke) of j-tile jt at x-tile xt of item `item` (0 for a single
// stack).  `list` and `seq` are scheduling scratch.
struct __align__(16) WorkUnit {
  int item, xt, jt, ks, ke;
  int list, seq, pad;
};
static_assert(sizeof(WorkUnit) == 32, "WorkUnit is 32 bytes");

// Largest and smallest rows per work unit of the single-stack fast
// projection, the average units per CTA list the plan's choice between them
// aims for, and columns x per unit (one TMA box row of the fast kernels).
constexpr int kChunkRows = 256;
constexpr int kMinChunkRows = 16;
constexpr double kUnitsPerList = 1.1;
constexpr int kUnitX = 128;

// Upper bound on the number of CTA lists (4 CTAs per SM on up to 256 SMs).
constexpr int kMaxLists = 1024;

// Cost of a unit in ring stages (two camera rows each), plus a fixed
// per-unit term for the job's set-up and its z-MIP fold.
inline int unit_cost(const WorkUnit& u) { return (u.ke - u.ks + 1) / 2 + 3; }

// Longest-processing-time-first schedule: units are taken by decreasing
// cost (ties in the given order) and each goes to the list with the least
// load so far (ties to the lowest list).  On return `units` is ordered list
// by list, each list in the order its units were assigned, and
// offsets[l] .. offsets[l + 1] delimit list l (offsets has nlists + 1
// entries).  In place and without allocation; nlists <= kMaxLists.
inline void schedule_lpt(WorkUnit* units, int n, int nlists, int* offsets) {
  for (int i = 0; i < n; ++i) units[i].seq = i;
  std::sort(units, units + n, [](const WorkUnit& a, const WorkUnit& b) {
    const int ca = unit_cost(a), cb = unit_cost(b);
    return ca != cb ? ca > cb : a.seq < b.seq;
  });
  // binary min-heap of (load, list)
  int64_t hload[kMaxLists];
  int hlist[kMaxLists];
  for (int l = 0; l < nlists; ++l) {
    hload[l] = 0;
    hlist[l] = l;
  }
  auto less = [&](int a, int b) { return hload[a] != hload[b] ? hload[a] < hload[b] : hlist[a] < hlist[b]; };
  for (int i = 0; i < n; ++i) {
    units[i].list = hlist[0];
    units[i].seq = i;
    hload[0] += unit_cost(units[i]);
    // sift the root down
    int r = 0;
    for (;;) {
      const int a = 2 * r + 1, b = a + 1;
      int m = r;
      if (a < nlists && less(a, m)) m = a;
      if (b < nlists && less(b, m)) m = b;
      if (m == r) break;
      std::swap(hload[r], hload[m]);
      std::swap(hlist[r], hlist[m]);
      r = m;
    }
  }
  std::sort(units, units + n, [](const WorkUnit& a, const WorkUnit& b) {
    return a.list != b.list ? a.list < b.list : a.seq < b.seq;
  });
  for (int l = 0; l <= nlists; ++l) offsets[l] = 0;
  for (int i = 0; i < n; ++i) offsets[units[i].list + 1] += 1;
  for (int l = 0; l < nlists; ++l) offsets[l + 1] += offsets[l];
}

}  // namespace opm
