// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), for the shots of a
// measurement and the SPSA perturbations.  Usable on the host and the device.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define QAOA_HD __host__ __device__ __forceinline__
#else
#define QAOA_HD inline
#endif

namespace qaoa {

struct Philox4 {
    uint32_t w[4];
};

QAOA_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// Ten rounds; each multiplies words 0 and 2 by the round multipliers and mixes
// the high halves with words 1, 3 and the key, which is bumped by the Weyl
// constants between rounds.
QAOA_HD Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t h0, l0, h1, l1;
        mulhilo32(0xD2511F53u, c0, h0, l0);
        mulhilo32(0xCD9E8D57u, c2, h1, l1);
        const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    return Philox4{{c0, c1, c2, c3}};
}

// 64-bit random integer of shot s in stream t under seed k: counter
// (s lo, s hi, t lo, t hi), key (k lo, k hi), value out0 + 2^32 out1.
QAOA_HD uint64_t shot_random(uint64_t seed, uint64_t stream, uint64_t s) {
    const Philox4 o = philox4x32_10((uint32_t)s, (uint32_t)(s >> 32), (uint32_t)stream, (uint32_t)(stream >> 32),
                                    (uint32_t)seed, (uint32_t)(seed >> 32));
    return (uint64_t)o.w[0] | ((uint64_t)o.w[1] << 32);
}

// SPSA perturbation sign of parameter i of start b at iteration k: +1 when bit
// 0 of out0 of counter (i, b, k, 0x53505341) is clear, else -1.
QAOA_HD double spsa_sign(uint64_t seed, uint32_t k, uint32_t b, uint32_t i) {
    const Philox4 o = philox4x32_10(i, b, k, 0x53505341u, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (o.w[0] & 1u) ? -1.0 : 1.0;
}

}  // namespace qaoa
