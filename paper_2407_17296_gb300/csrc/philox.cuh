// philox.cuh -- counter-based common random numbers for the CRN particle filter.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit multiplies and XORs with a
// Weyl-sequence key schedule.  Written from the published description.
//
// Layout of the common random numbers (Sec. I: one seed per SMC^2 sample and
// iteration; Sec. II-A: fixed numbers make sampling and resampling
// deterministic functions of theta):
//   key = (seed_lo ^ iteration, seed_hi ^ sample_row)
//   ctr = (t, call, stream, 0)
//   stream 0 propagation at step t (normal n = j*d_x + k, call n/4, lane n%4)
//   stream 1 resampling uniforms before step t (systematic: call 0 word 0;
//            multinomial: particle i -> call i/4 word i%4)
//   stream 2 initial particles (t = 0, same normal indexing as stream 0)
//   stream 3 outer-sampler normals (t = 0, normal index d)
//   stream 4 outer-sampler resampling uniform (t = 0, call 0 word 0, row 0)
//   stream 5 NUTS move (t = doubling j, call = point n of the doubling: word 0 of call 0 gives
//            the direction, word 2 of call 0 the merge uniform, word 1 the selection uniform)
// Uniforms: (0,1] = ((u >> 8) + 1) * 2^-24 (exact in FP32); [0,1) = (u >> 8) * 2^-24.
// Box-Muller on (u0, u1): r = sqrt(-2 ln U(0,1](u0)), phi = 2 pi U[0,1)(u1),
// z0 = r cos phi, z1 = r sin phi; (u2, u3) give z2, z3 the same way.
#pragma once
#include <cstdint>

namespace smc2 {

enum : uint32_t { kStreamProp = 0, kStreamResample = 1, kStreamInit = 2,
                  kStreamOuterXi = 3, kStreamOuterNu = 4, kStreamNuts = 5 };

// The key with its ten round keys (the Weyl schedule k + r * W), expanded once per filter:
// a filter draws thousands of blocks with the same key.
struct PhiloxKey {
    uint32_t k0[10], k1[10];
};

__host__ __device__ __forceinline__ PhiloxKey philox_key(uint32_t seed_lo, uint32_t seed_hi,
                                                         uint32_t iter, uint32_t row) {
    PhiloxKey k;
    k.k0[0] = seed_lo ^ iter;
    k.k1[0] = seed_hi ^ row;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        k.k0[r] = k.k0[r - 1] + 0x9E3779B9u;
        k.k1[r] = k.k1[r - 1] + 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey& key) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c.x;
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ key.k0[r], lo1, hi0 ^ c.w ^ key.k1[r], lo0);
    }
    return c;
}

// k * 2^-24 for an integer k in [0, 2^24], exactly: k converts to FP32 without rounding (24
// significant bits at most) and the power-of-two scale is exact.  (The conversion measured
// cheaper here than building the float from bits: 2-3% on the filter forward passes.)
__device__ __forceinline__ float exact_u24_scaled(uint32_t k) {
    return __uint2float_rn(k) * 5.9604644775390625e-08f;
}

__device__ __forceinline__ float u01_open(uint32_t u) {   // (0, 1]
    return exact_u24_scaled((u >> 8) + 1u);
}

// One Box-Muller pair from two words.  The angle is evaluated as
// phi' = 2 pi (U[0,1) - 1/2) in [-pi, pi), where the hardware sine/cosine are accurate
// (absolute error ~2^-21), and cos(phi') = -cos(2 pi U), sin(phi') = -sin(2 pi U) restore
// the definition.  The radius keeps the accurate logf (a hardware base-2 logarithm, ~2^-22
// absolute, moved cumulative weights of 128-particle filters by more than 1e-6 through the
// normals it perturbs); sqrt(s) = s * rsqrt(s), with rsqrt's argument raised to the smallest
// normal float so that s = 0 (the uniform equal to 1) gives 0 (every other s is at least
// 2^-23).  The angle folds U[0,1)'s scale 2^-24 into the constant: (k 2^-24) (2 pi) and
// k (2 pi 2^-24) are the same exact product, so the fused multiply-add rounds the same value.
__device__ __forceinline__ void box_muller(uint32_t ua, uint32_t ub, float& z0, float& z1) {
    constexpr float kTwoPi = 6.2831853071795864769f;
    const float s = -2.0f * logf(u01_open(ua));
    const float r = s * rsqrtf(fmaxf(s, 1.17549435e-38f));
    const float ph = fmaf(__uint2float_rn(ub >> 8), kTwoPi * 5.9604644775390625e-08f, -3.1415926535897932385f);
    float sn, cs;
    __sincosf(ph, &sn, &cs);
    z0 = -r * cs;
    z1 = -r * sn;
}

// Normals n0 .. n0+COUNT-1 of (key, t, stream) into out[].  n0 % 4 == 0 when
// COUNT % 4 == 0; otherwise any n0 (the covering calls are evaluated).
template <int COUNT>
__device__ __forceinline__ void normals(const PhiloxKey& key, uint32_t t, uint32_t stream, uint32_t n0,
                                        float (&out)[COUNT]) {
    if constexpr (COUNT % 4 == 0) {
#pragma unroll
        for (int c = 0; c < COUNT / 4; ++c) {
            const uint4 w = philox4x32_10(make_uint4(t, n0 / 4 + c, stream, 0u), key);
            box_muller(w.x, w.y, out[4 * c + 0], out[4 * c + 1]);
            box_muller(w.z, w.w, out[4 * c + 2], out[4 * c + 3]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < COUNT; ++q) {
            const uint32_t n = n0 + q;
            const uint4 w = philox4x32_10(make_uint4(t, n / 4, stream, 0u), key);
            const uint32_t lane = n & 3u;
            const uint32_t ua = (lane < 2) ? w.x : w.z;
            const uint32_t ub = (lane < 2) ? w.y : w.w;
            float z0, z1;
            box_muller(ua, ub, z0, z1);
            out[q] = (lane & 1u) ? z1 : z0;
        }
    }
}

}  // namespace smc2
