// schedule.h - member ranges of the step schedule (host code only).
//
// The members of a group (one grid) are independent problems, so a step can
// run over any partition of a batch into units, each a range [m0, m1) of one
// group's members.  These are the two rules that cut groups into units; they
// hold no device code and are compiled on their own by the CPU tests.
#pragma once

#include <algorithm>
#include <cstddef>
#include <vector>

namespace sbi {

struct Unit {
  int group, m0, m1;
  bool operator==(const Unit& o) const { return group == o.group && m0 == o.m0 && m1 == o.m1; }
};

// Units of at most cap points each (cap 0: one unit per group): group g, of
// pts[g] points over n[g] members, is cut into min(n[g], ceil(pts[g] / cap))
// nearly equal member ranges when sliceable[g], else kept whole.
inline std::vector<Unit> units_for_cap(const std::vector<size_t>& pts, const std::vector<int>& n, size_t cap,
                                       const std::vector<bool>& sliceable) {
  std::vector<Unit> u;
  for (size_t gi = 0; gi < pts.size(); ++gi) {
    int k = 1;
    if (sliceable[gi] && cap > 0) k = (int)std::min<size_t>((size_t)n[gi], (pts[gi] + cap - 1) / cap);
    for (int q = 0; q < k; ++q)
      u.push_back(Unit{(int)gi, (int)((long long)q * n[gi] / k), (int)((long long)(q + 1) * n[gi] / k)});
  }
  return u;
}

// Each unit cut into k nearly equal member ranges (at most one member each).
inline std::vector<Unit> split_units(const std::vector<Unit>& units, int k) {
  std::vector<Unit> out;
  for (const Unit& u : units) {
    const int n = u.m1 - u.m0, kk = std::max(1, std::min(k, n));
    for (int q = 0; q < kk; ++q)
      out.push_back(Unit{u.group, u.m0 + (int)((long long)q * n / kk), u.m0 + (int)((long long)(q + 1) * n / kk)});
  }
  return out;
}

}  // namespace sbi
