// Prints Philox4x32-10 words from PyTorch's header-only at::philox_engine for
// (key, counter) quadruples read from stdin, one "k0 k1 c0 c1 c2 c3" per line.
// torch's engine takes key = seed, counter words 0-1 = offset, 2-3 = subsequence.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
  unsigned k0, k1, c0, c1, c2, c3;
  while (std::scanf("%u %u %u %u %u %u", &k0, &k1, &c0, &c1, &c2, &c3) == 6) {
    uint64_t seed = (uint64_t(k1) << 32) | k0;
    uint64_t subseq = (uint64_t(c3) << 32) | c2;
    uint64_t offset = (uint64_t(c1) << 32) | c0;
    at::philox_engine e(seed, subseq, offset);
    unsigned w0 = e(), w1 = e(), w2 = e(), w3 = e();
    std::printf("%u %u %u %u\n", w0, w1, w2, w3);
  }
  return 0;
}
