// Test probe of the library's launch-decomposition rules (csrc/tc_setup.cpp): reads lines
//   split <items> <partners> <sms>         -> prints pick_split
//   near <n> <t1> ... <tn>                  -> prints smallest_near_best
// from standard input and prints one integer per line.
#include <cstdio>
#include <cstring>
#include <vector>

#include "tc_setup.hpp"

int main() {
  char cmd[16];
  while (std::scanf("%15s", cmd) == 1) {
    if (!std::strcmp(cmd, "split")) {
      int items = 0, partners = 0, sms = 0;
      if (std::scanf("%d %d %d", &items, &partners, &sms) != 3) return 2;
      std::printf("%d\n", tc::pick_split(items, partners, sms));
    } else if (!std::strcmp(cmd, "near")) {
      int n = 0;
      if (std::scanf("%d", &n) != 1 || n < 1) return 2;
      std::vector<double> t(n + 1, 0.0);
      for (int s = 1; s <= n; ++s)
        if (std::scanf("%lf", &t[s]) != 1) return 2;
      std::printf("%d\n", tc::smallest_near_best(t.data(), n));
    } else {
      return 2;
    }
  }
  return 0;
}
