// Philox4x32-10 counter-based generator for the device (Salmon, Moraes, Dror
// & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), and the
// mapping of its words to the uniforms and normals the sampler consumes.
//
// Counter layout of one draw: (t, voxel, chain << 8 | call, 0); key = (seed
// lo, seed hi).  Iteration t = 0xFFFFFFFF is reserved for the initial state.
// Proposal normals come from Box-Muller pairs on words (2j, 2j+1); the word
// after the last pair is the acceptance uniform.
#pragma once
#include <cstdint>

namespace gac {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kInitIteration = 0xFFFFFFFFu;

struct Words4 {
    uint32_t w[4];
};

// One round with round key (k0, k1): two 32x32->64 multiplies (one IMAD.WIDE
// each) and two three-input XORs.
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                             uint32_t k0, uint32_t k1) {
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
    c1 = static_cast<uint32_t>(p1);
    c3 = static_cast<uint32_t>(p0);
    c0 = n0;
    c2 = n2;
}

// Ten rounds, round r keyed (k0 + r W0, k1 + r W1).  The key schedule depends
// only on the seed, so it stays in uniform registers when the seed is a
// kernel argument.
__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    Words4 out;
    out.w[0] = c0;
    out.w[1] = c1;
    out.w[2] = c2;
    out.w[3] = c3;
    return out;
}

// Number of words per MH iteration for P parameters: 2*ceil(P/2) normals
// words + 1 acceptance word.
__host__ __device__ constexpr int n_words(int P) { return 2 * ((P + 1) / 2) + 1; }
__host__ __device__ constexpr int n_calls(int P) { return (n_words(P) + 3) / 4; }

// Fills w[0 .. 4*n_calls(P)) for draw (t, v, c).
template <int NW>
__device__ __forceinline__ void draw_words(uint32_t (&w)[NW], uint32_t t, uint32_t v, uint32_t c,
                                           uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int k = 0; 4 * k < NW; ++k) {
        Words4 o = philox4x32_10(t, v, (c << 8) | static_cast<uint32_t>(k), 0u, k0, k1);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * k + j < NW) w[4 * k + j] = o.w[j];
    }
}

// (w + 1/2) 2^-32 in float: exact for w < 2^24, relative error <= 2^-24 above.
__device__ __forceinline__ float u01_f(uint32_t w) {
    return fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
}
__device__ __forceinline__ double u01_d(uint32_t w) {
    return (static_cast<double>(w) + 0.5) * 0x1p-32;
}

// Box-Muller in FP32 on the special-function unit.  Radius
// sqrt(-2 ln u1) from the hardware log2 (absolute error ~2e-7 near u1 = 1,
// 3 ulp elsewhere) and reciprocal square root, guarded so that a log that
// rounds to >= 0 gives radius ~0 rather than NaN; angle 2 pi u2 taken
// through the signed word, 2 pi ((int32) w + 1/2) 2^-32 in [-pi, pi) -- the
// same sine and cosine -- where the hardware sin/cos is accurate to ~4e-7.
// The pair stays rotationally symmetric, so the proposal stays symmetric
// and the Metropolis rule exact; the deviation from exact Box-Muller normals
// is ~1e-6 (up to ~1e-3 only when u1 is within 1e-6 of 1).
// The radius is taken as sqrt(k log2 u1) with k = -2 ln 2 s^2, which scales
// both normals by s > 0 (the MH step multiplier) at no extra cost; the
// default k gives the standard pair (s = 1).
// The pair is built in two parts: bm_prefix (log2 u1 and the angle's sine and
// cosine: what depends only on the words) and bm_finish (the radius, which
// takes the step multiplier); the lane-split sampler draws the prefixes ahead.
constexpr float kNeg2Ln2 = -1.38629436111989061883f;  // -2 ln 2
__device__ __forceinline__ void bm_prefix(uint32_t w1, uint32_t w2, float &lg, float &s, float &c) {
    lg = __log2f(u01_f(w1));
    const float ang = fmaf(static_cast<float>(static_cast<int32_t>(w2)), 1.46291807926715968e-9f,
                           7.31459039633579840e-10f);  // 2 pi 2^-32, pi 2^-32
    __sincosf(ang, &s, &c);
}
__device__ __forceinline__ void bm_finish(float lg, float s, float c, float k, float &z0, float &z1) {
    const float x = fmaxf(k * lg, 1e-30f);
    const float r = x * rsqrtf(x);
    z0 = r * c;
    z1 = r * s;
}
__device__ __forceinline__ void box_muller_f(uint32_t w1, uint32_t w2, float &z0, float &z1,
                                             float k = kNeg2Ln2) {
    float lg, s, c;
    bm_prefix(w1, w2, lg, s, c);
    bm_finish(lg, s, c, k, z0, z1);
}

// k = -2 s^2 scales both normals by s > 0; -2 gives the standard pair.
__device__ __forceinline__ void box_muller_d(uint32_t w1, uint32_t w2, double &z0, double &z1,
                                             double k = -2.0) {
    const double u1 = u01_d(w1);
    const double u2 = u01_d(w2);
    const double r = sqrt(k * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

}  // namespace gac
