// philox_ref_aten.cpp -- an independent Philox4x32-10 for pinning the oracle's
// stream: PyTorch's ATen engine (ATen/core/PhiloxRNGEngine.h), driven through its
// public interface only.  Reads lines "c0 c1 c2 c3 k0 k1" (decimal 32-bit words)
// on stdin and prints the four output words of Philox4x32-10 for counter
// (c0, c1, c2, c3) and key (k0, k1), one line per input line.
//
// The engine's constructor takes (seed, subsequence, offset) and sets
// key = (seed_lo, seed_hi), counter = (offset_lo, offset_hi, subsequence_lo,
// subsequence_hi); each call returns the next of the four words of one block.
#include <ATen/core/PhiloxRNGEngine.h>

#include <cinttypes>
#include <cstdio>

int main()
{
    unsigned long long c0, c1, c2, c3, k0, k1;
    while (std::scanf("%llu %llu %llu %llu %llu %llu", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        const uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
        const uint64_t sub = (uint64_t)c2 | ((uint64_t)c3 << 32);
        const uint64_t off = (uint64_t)c0 | ((uint64_t)c1 << 32);
        at::philox_engine e(seed, sub, off);
        const uint32_t w0 = e(), w1 = e(), w2 = e(), w3 = e();
        std::printf("%u %u %u %u\n", w0, w1, w2, w3);
    }
    return 0;
}
