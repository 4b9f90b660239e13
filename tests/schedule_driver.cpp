// Reads batches from stdin and prints the units the step-schedule rules of
// schedule.h give, for the CPU test of those rules.
//   input per case:  G cap k, then G lines "points members sliceable"
//   output per case: "cap" units, then "split" units (cut k ways), one
//                    "group m0 m1" triple each, each list ended by "end"
#include <cstdio>
#include <vector>

#include "schedule.h"

int main() {
  int G, k;
  unsigned long long cap;
  while (std::scanf("%d %llu %d", &G, &cap, &k) == 3) {
    std::vector<size_t> pts(G);
    std::vector<int> n(G);
    std::vector<bool> sl(G);
    for (int g = 0; g < G; ++g) {
      unsigned long long p;
      int m, s;
      if (std::scanf("%llu %d %d", &p, &m, &s) != 3) return 1;
      pts[g] = p;
      n[g] = m;
      sl[g] = s != 0;
    }
    const std::vector<sbi::Unit> u = sbi::units_for_cap(pts, n, (size_t)cap, sl);
    for (const auto& x : u) std::printf("%d %d %d\n", x.group, x.m0, x.m1);
    std::printf("end\n");
    for (const auto& x : sbi::split_units(u, k)) std::printf("%d %d %d\n", x.group, x.m0, x.m1);
    std::printf("end\n");
  }
  return 0;
}
