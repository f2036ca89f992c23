// The engine's Philox4x32-10 (csrc/device_f64.cuh, built for the host) against
// the oracle's, written separately from the same published round function:
// 2.5e8 blocks, 10^9 words, over counters laid out as the engine lays them
// out (simulation, attempt, purpose << 24 | j, block) and over arbitrary ones,
// under many keys.  Prints the number of words compared and of mismatches.
// Built and run by tests/test_devmath_host.py, linked with the oracle library.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "../paper_1309_7695_b300/csrc/device_f64.cuh"

extern "C" void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

int main(int argc, char **argv)
{
    const uint64_t blocks = argc > 1 ? strtoull(argv[1], nullptr, 10) : 250000000ull;
    uint64_t words = 0, mismatches = 0;
    uint64_t lcg = 0x243F6A8885A308D3ull;
    for (uint64_t b = 0; b < blocks; ++b) {
        lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
        uint32_t ctr[4] = {(uint32_t)(b & 0xffffffu), (uint32_t)(b >> 12), (uint32_t)(((1u + (b & 3)) << 24) | ((b >> 2) & 0x3ff)),
                           (uint32_t)(lcg >> 60)};
        if (b & 1) {   // arbitrary first two words
            ctr[0] = (uint32_t)(lcg >> 32);
            ctr[1] = (uint32_t)lcg;
        }
        const uint32_t key[2] = {(uint32_t)(0x9E3779B9u * (uint32_t)(b >> 12)), (uint32_t)((b >> 12) * 2654435761u + 7u)};
        uint32_t o[4];
        oracle_philox4x32_10(ctr, key, o);
        const uint4 d = tl::f64::philox4x32_10(make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]), key[0], key[1]);
        mismatches += (d.x != o[0]) + (d.y != o[1]) + (d.z != o[2]) + (d.w != o[3]);
        words += 4;
    }
    printf("%llu %llu\n", (unsigned long long)words, (unsigned long long)mismatches);
    return 0;
}
