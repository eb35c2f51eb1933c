// Reference Philox4x32-10 outputs from PyTorch's header-only engine
// (ATen/core/PhiloxRNGEngine.h), an implementation independent of the oracle.
// Reads lines "c0 c1 c2 c3 k0 k1" (decimal) from stdin, prints the 4 outputs.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>

int main() {
    unsigned long long c0, c1, c2, c3, k0, k1;
    while (std::scanf("%llu %llu %llu %llu %llu %llu", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
        uint64_t subsequence = (uint64_t)c2 | ((uint64_t)c3 << 32);
        // The engine's counter is (offset lo, offset hi, subsequence lo, subsequence hi).
        at::Philox4_32 eng(seed, subsequence, 0);
        eng.set_offset((uint64_t)c0 | ((uint64_t)c1 << 32));
        uint32_t a = eng(), b = eng(), c = eng(), d = eng();
        std::printf("%u %u %u %u\n", a, b, c, d);
    }
    return 0;
}
