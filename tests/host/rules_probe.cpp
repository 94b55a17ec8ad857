// Test probe of the library's launch-decomposition rules (csrc/tc_setup.cpp): reads lines
//   split <items> <partners> <sms>         -> prints pick_split
//   near <n> <t1> ... <tn>                  -> prints smallest_near_best
//   span <count> <m1 m2 m3> x count         -> prints miller_span of one sphere of count vectors
//   grid <n> <span>                          -> prints left_from_right_exact and pair_support_len
//   mirror <fp64> <nkb> <L> <support> <Nk> <no> <free> -> prints mirror_buffer_bytes
// from standard input and prints one integer per line.
#include <cstdio>
#include <array>
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
    } else if (!std::strcmp(cmd, "span")) {
      int count = 0;
      if (std::scanf("%d", &count) != 1 || count < 0) return 2;
      std::vector<std::vector<std::array<int, 3>>> miller(1);
      for (int i = 0; i < count; ++i) {
        std::array<int, 3> m{};
        if (std::scanf("%d %d %d", &m[0], &m[1], &m[2]) != 3) return 2;
        miller[0].push_back(m);
      }
      std::printf("%d\n", tc::miller_span(miller));
    } else if (!std::strcmp(cmd, "grid")) {
      int n = 0, span = 0;
      if (std::scanf("%d %d", &n, &span) != 2) return 2;
      std::printf("%d %d\n", tc::left_from_right_exact(n, span) ? 1 : 0, tc::pair_support_len(n, span));
    } else if (!std::strcmp(cmd, "mirror")) {
      int fp64 = 0, nkb = 0, L = 0, sup = 0, nk = 0, no = 0;
      unsigned long long fr = 0;
      if (std::scanf("%d %d %d %d %d %d %llu", &fp64, &nkb, &L, &sup, &nk, &no, &fr) != 7) return 2;
      std::printf("%llu\n", (unsigned long long)tc::mirror_buffer_bytes(fp64 != 0, nkb, L, sup, nk, no, (size_t)fr));
    } else {
      return 2;
    }
  }
  return 0;
}
