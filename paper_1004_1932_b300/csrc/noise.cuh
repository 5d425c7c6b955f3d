// Additive Brownian noise with a constant mobility factor, the dilute-limit
// approximation the paper proposes in place of a Cholesky factor of the full
// hydrodynamic tensor (closing remarks of Sec. IV): every sphere receives the
// displacement sigma z per Heun step, sigma = sqrt(2 kT dt / (6 pi mu a)),
// z ~ N(0, I_3), the same z in the predictor and the corrector of a step
// (the Heun scheme for additive noise).
//
// z comes from a counter-based generator, so that any thread can draw the
// numbers of any (step, sphere) without state: Philox4x32-10 (Salmon, Moraes,
// Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) on the
// counter (n mod 2^32, n / 2^32, sphere index, 0) with the 64-bit seed as key,
// and the Box-Muller transform on the four uniforms u = (r + 1/2) 2^-32:
//   z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1),
//   z2 = sqrt(-2 ln u2) cos(2 pi u3).
#pragma once
#include <cstdint>

namespace dbs {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;  // round multipliers
    constexpr unsigned W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;  // key increments (Weyl sequence)
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        const unsigned lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const unsigned lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 sphere_bits(unsigned long long seed, int64_t n, int64_t i)
{
    const unsigned long long un = (unsigned long long)n;
    return philox4x32_10(make_uint4((unsigned)un, (unsigned)(un >> 32), (unsigned)i, 0u),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// -2 ln u for u = (r + 1/2) 2^-32 in FP32, accurate over the whole range: for
// u > 1/2 through log1p of the complement, which FP32 holds exactly.
__device__ __forceinline__ float neg2_log_u(unsigned r)
{
    constexpr float s = 2.3283064365386963e-10f;  // 2^-32
    if (r < 0x80000000u) return -2.f * logf(((float)r + 0.5f) * s);
    return -2.f * log1pf(-((float)(0xffffffffu - r) + 0.5f) * s);
}

// Standard normals of sphere i at step n; FP64 or FP32 arithmetic.
__device__ __forceinline__ void sphere_normals(unsigned long long seed, int64_t n, int64_t i, double z[3])
{
    const uint4 r = sphere_bits(seed, n, i);
    constexpr double s = 2.3283064365386962890625e-10;  // 2^-32
    const double ra = sqrt(-2.0 * log(((double)r.x + 0.5) * s));
    const double rb = sqrt(-2.0 * log(((double)r.z + 0.5) * s));
    double sa, ca, sb, cb;
    sincospi(2.0 * (((double)r.y + 0.5) * s), &sa, &ca);
    sincospi(2.0 * (((double)r.w + 0.5) * s), &sb, &cb);
    z[0] = ra * ca;
    z[1] = ra * sa;
    z[2] = rb * cb;
}

__device__ __forceinline__ void sphere_normals(unsigned long long seed, int64_t n, int64_t i, float z[3])
{
    const uint4 r = sphere_bits(seed, n, i);
    constexpr float s = 2.3283064365386963e-10f;
    const float ra = sqrtf(neg2_log_u(r.x)), rb = sqrtf(neg2_log_u(r.z));
    float sa, ca, sb, cb;
    sincospif(2.f * (((float)r.y + 0.5f) * s), &sa, &ca);
    sincospif(2.f * (((float)r.w + 0.5f) * s), &sb, &cb);
    z[0] = ra * ca;
    z[1] = ra * sa;
    z[2] = rb * cb;
}

}  // namespace dbs
