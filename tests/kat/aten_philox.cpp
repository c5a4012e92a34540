// Known-answer source for the oracle's Philox4x32-10 on the host: PyTorch's
// header-only Philox engine (ATen/core/PhiloxRNGEngine.h), an implementation
// of the same published generator (Salmon et al., SC'11) that shares nothing
// with this repository.  Its key is the 64-bit seed, counter words 2..3 the
// 64-bit subsequence and counter words 0..1 the 64-bit offset, so any
// (counter, key) pair is reachable; four draws return the four output words.
#include <ATen/core/PhiloxRNGEngine.h>

#include <cstdint>

extern "C" void aten_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                                   int n) {
    for (int i = 0; i < n; ++i) {
        const uint64_t seed = (uint64_t)key[2 * i] | ((uint64_t)key[2 * i + 1] << 32);
        const uint64_t sub = (uint64_t)ctr[4 * i + 2] | ((uint64_t)ctr[4 * i + 3] << 32);
        const uint64_t off = (uint64_t)ctr[4 * i] | ((uint64_t)ctr[4 * i + 1] << 32);
        at::Philox4_32 eng(seed, sub, 0);
        eng.set_offset(off);
        for (int w = 0; w < 4; ++w) out[4 * i + w] = eng();
    }
}
