/* Exhaustive check of the oracle's bounded draw: calls ora_bounded on every
 * 32-bit word for the bound s given on the command line and prints
 * "min_count max_count rejected". */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int ora_bounded(uint32_t w, uint32_t s, uint32_t* out);

int main(int argc, char** argv) {
  uint32_t s = (uint32_t)strtoul(argv[1], NULL, 10);
  uint64_t* cnt = calloc(s, sizeof(uint64_t));
  uint64_t rejected = 0;
  uint32_t w = 0;
  do {
    uint32_t v;
    if (ora_bounded(w, s, &v)) {
      if (v >= s) { printf("out-of-range\n"); return 1; }
      ++cnt[v];
    } else {
      ++rejected;
    }
  } while (++w != 0);
  uint64_t mn = cnt[0], mx = cnt[0];
  for (uint32_t i = 1; i < s; ++i) { if (cnt[i] < mn) mn = cnt[i]; if (cnt[i] > mx) mx = cnt[i]; }
  printf("%llu %llu %llu\n", (unsigned long long)mn, (unsigned long long)mx, (unsigned long long)rejected);
  return 0;
}
