// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based generator of the
// sampling step and of the IK starting points, and the Box-Muller transform of its words: ten rounds, each multiplying words 0 and 2
// by the round constants, xor-ing the high halves with the other words and the round key,
// the key bumped by the Weyl constants between rounds.
#pragma once

#include <cstdint>

namespace cp {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;

static __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    return c;
}

// The ten round keys of one key (k0, k1): round r uses (k0 + r W0, k1 + r W1) mod 2^32.
// Formed once on the host and passed by value to a kernel, they sit in its constant bank,
// so the rounds read them as operands instead of adding the Weyl constants per call.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1)
{
    PhiloxKeys k;
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = k0 + (uint32_t)r * kWeyl0;
        k.k1[r] = k1 + (uint32_t)r * kWeyl1;
    }
    return k;
}

// philox4x32_10 with the round keys given (the same words).
static __device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &key)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ key.k0[r], lo1, hi0 ^ c.w ^ key.k1[r], lo0);
    }
    return c;
}

// Box-Muller on the top 24 bits of two words: u1 in (0, 1], u2 in [0, 1), both exact.
static __device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1)
{
    const float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(b >> 8) * 0x1p-24f;
    const float r = sqrtf(-2.f * logf(u1));
    float s, c;
    sincospif(2.f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

}  // namespace cp
