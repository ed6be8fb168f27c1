// Reference Philox4x32-10 for the oracle's pin: drives PyTorch's header-only engine
// (ATen/core/PhiloxRNGEngine.h, an implementation independent of the oracle) with an
// arbitrary counter and key.  Reads lines "c0 c1 c2 c3 k0 k1" (hex) from stdin and
// prints the four output words.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>

int main() {
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%x %x %x %x %x %x", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
        uint64_t subsequence = (uint64_t)c2 | ((uint64_t)c3 << 32);
        uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
        at::Philox4_32 engine(seed, subsequence, offset);
        unsigned w0 = engine(), w1 = engine(), w2 = engine(), w3 = engine();
        std::printf("%08x %08x %08x %08x\n", w0, w1, w2, w3);
    }
    return 0;
}
