// Host check of the random-number path of the SSA kernels against the
// oracle's independent implementation: philox10 of
// paper_0912_2551_gb300/csrc/smc_device.cuh (compiled for the host through
// host_cuda_shims.h), with round keys from the published Philox4x32 key
// schedule (key plus r times the Weyl increments 0x9E3779B9, 0xBB67AE85),
// must equal orc_philox4x32_10 of oracle/smc_oracle.c word for word on the
// counters (event, trajectory, instance, 0) the kernels use; the FP64
// uniform map must equal the oracle's, and the FP32 one its definition
// ((w >> 9) + 1/2) 2^-23.  Usage: philox_check <blocks>; prints
// "blocks=<n> mismatches=<m> u52=<m> u23=<m>" and exits 0 when all are 0.
#include <stdio.h>
#include <stdlib.h>

#include "host_cuda_shims.h"
#include "smc_device.cuh"

extern "C" void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
extern "C" double orc_u01(uint32_t hi, uint32_t lo);

int main(int argc, char **argv)
{
    const uint64_t blocks = argc > 1 ? strtoull(argv[1], nullptr, 10) : 100000000ull;
    const uint64_t seeds[] = {0ull, 0x5EED5EED5EEDull, 0xFFFFFFFFFFFFFFFFull, 1234567ull};
    uint64_t mism = 0, m52 = 0, m23 = 0, done = 0;
    for (uint64_t seed : seeds) {
        const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t rk0[10], rk1[10];
        for (int r = 0; r < 10; ++r) {
            rk0[r] = key[0] + (uint32_t)r * 0x9E3779B9u;
            rk1[r] = key[1] + (uint32_t)r * 0xBB67AE85u;
        }
        const uint64_t n = blocks / 4;
        for (uint64_t i = 0; i < n; ++i) {
            // event, trajectory, instance: a dense low range and scattered
            // 32-bit values (splitmix-style), as the kernels' counters run
            uint64_t z = i * 0x9E3779B97F4A7C15ull + seed;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            const uint32_t e = (i & 1) ? (uint32_t)(i >> 1) : (uint32_t)z;
            const uint32_t traj = (i & 2) ? (uint32_t)(i >> 12) : (uint32_t)(z >> 32);
            const uint32_t inst = (uint32_t)(i % 4099);
            uint32_t w0, w1, w2, w3, o[4];
            philox10(e, traj, inst, 0u, rk0, rk1, w0, w1, w2, w3);
            const uint32_t ctr[4] = {e, traj, inst, 0u};
            orc_philox4x32_10(ctr, key, o);
            mism += (w0 != o[0]) | (w1 != o[1]) | (w2 != o[2]) | (w3 != o[3]);
            if ((i & 15) == 0) {
                m52 += u01_52(w0, w1) != orc_u01(w0, w1);
                m52 += u01_52(w2, w3) != orc_u01(w2, w3);
                m23 += (double)u01_23(w0) != ((double)(w0 >> 9) + 0.5) * 0x1p-23;
                m23 += (double)u01_23(w2) != ((double)(w2 >> 9) + 0.5) * 0x1p-23;
            }
            ++done;
        }
    }
    // the ends of the maps: all-zero and all-one words
    m52 += u01_52(0u, 0u) != 0x1p-53 || u01_52(~0u, ~0u) != 1.0 - 0x1p-53;
    m23 += u01_23(0u) != 0x1p-24f || u01_23(~0u) != 1.0f - 0x1p-24f;
    printf("blocks=%llu mismatches=%llu u52=%llu u23=%llu\n", (unsigned long long)done, (unsigned long long)mism,
           (unsigned long long)m52, (unsigned long long)m23);
    return (mism || m52 || m23) ? 1 : 0;
}
