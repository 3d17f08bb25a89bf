// Checks opm::schedule_lpt on seeded random unit sets: the output is a
// permutation of the input, list offsets partition it, every list keeps its
// units in assignment order (non-increasing cost), and the makespan is
// within the longest-processing-time bound of 4/3 of a lower bound on the
// optimum (max of the average load and the largest unit).
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "opm_sched.h"

int main() {
  std::mt19937 rng(12345);
  int failures = 0;
  for (int trial = 0; trial < 200; ++trial) {
    const int n = (int)(rng() % 5000);
    const int L = 1 + (int)(rng() % 700);
    std::vector<opm::WorkUnit> u(n);
    long long total = 0, biggest = 0, key_in = 0;
    for (int i = 0; i < n; ++i) {
      const int ks = (int)(rng() % 400), len = 1 + (int)(rng() % (trial % 2 ? 128 : 300));
      u[i] = opm::WorkUnit{(int)(rng() % 7), (int)(rng() % 16), (int)(rng() % 40), ks, ks + len, 0, 0, 0};
      total += opm::unit_cost(u[i]);
      biggest = std::max<long long>(biggest, opm::unit_cost(u[i]));
      key_in += (long long)u[i].item * 1000003LL + u[i].xt * 10007LL + u[i].jt * 101LL + u[i].ks * 7LL + u[i].ke;
    }
    std::vector<int> off(L + 1);
    opm::schedule_lpt(u.data(), n, L, off.data());
    long long key_out = 0, makespan = 0;
    bool ok = off[0] == 0 && off[L] == n;
    for (int l = 0; l < L && ok; ++l) {
      if (off[l + 1] < off[l]) ok = false;
      long long load = 0;
      for (int i = off[l]; i < off[l + 1]; ++i) {
        if (u[i].list != l) ok = false;
        if (i > off[l] && opm::unit_cost(u[i]) > opm::unit_cost(u[i - 1])) ok = false;
        load += opm::unit_cost(u[i]);
      }
      makespan = std::max(makespan, load);
    }
    for (int i = 0; i < n; ++i)
      key_out += (long long)u[i].item * 1000003LL + u[i].xt * 10007LL + u[i].jt * 101LL + u[i].ks * 7LL + u[i].ke;
    const long long lower = std::max((total + L - 1) / L, biggest);
    if (key_in != key_out) ok = false;
    if (n > 0 && 3 * makespan > 4 * lower + 3) ok = false;
    if (!ok) {
      std::printf("trial %d failed: n=%d L=%d makespan=%lld lower=%lld\n", trial, n, L, makespan, lower);
      ++failures;
    }
  }
  std::printf("%s\n", failures ? "FAIL" : "OK");
  return failures ? 1 : 0;
}
