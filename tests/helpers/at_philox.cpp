// Test-only helper: PyTorch's open-source Philox4x32-10 engine
// (ATen/core/PhiloxRNGEngine.h, at::Philox4_32) behind a C entry point, so
// the tests can hold the oracle's generator against an implementation
// written by someone else.  Built by tests/test_philox_pin.py into a
// temporary directory; never linked into the oracle or the library.
//
// at::Philox4_32(seed, subsequence, offset) starts at the counter
// (offset_lo, offset_hi, subsequence_lo, subsequence_hi) under the key
// (seed_lo, seed_hi); its first draw is word 0 of that block.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>

extern "C" void at_philox_w0(const uint32_t* ctr, const uint64_t* seed, int64_t count,
                             uint32_t* out)
{
    for (int64_t i = 0; i < count; ++i) {
        const uint32_t* c = ctr + 4 * i;
        uint64_t offset = (uint64_t)c[0] | ((uint64_t)c[1] << 32);
        uint64_t subseq = (uint64_t)c[2] | ((uint64_t)c[3] << 32);
        at::Philox4_32 eng(seed[i], subseq, offset);
        out[i] = eng();
    }
}

// All four words of the block, read as four consecutive draws.
extern "C" void at_philox_block(const uint32_t* ctr, uint64_t seed, uint32_t* out)
{
    uint64_t offset = (uint64_t)ctr[0] | ((uint64_t)ctr[1] << 32);
    uint64_t subseq = (uint64_t)ctr[2] | ((uint64_t)ctr[3] << 32);
    at::Philox4_32 eng(seed, subseq, offset);
    for (int k = 0; k < 4; ++k) out[k] = eng();
}
