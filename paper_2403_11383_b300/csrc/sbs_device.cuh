// Device building blocks of the SBS controller: counter-based random numbers,
// the single-rigid-body model step, the stage cost and block reductions.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "sbs_internal.h"

namespace sbs {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Lane values.  The rollout's arithmetic is written once over a lane type V:
// float carries one sample per thread; float2 carries two samples per thread,
// and its additions, multiplications and fused multiply-adds issue as single
// packed FP32x2 instructions (sm_100 and later), so two samples' arithmetic
// takes one issue slot.  Every operation is explicit and rounded once
// (round-to-nearest, no contraction left to the compiler), so a sample's result
// has the same bits whichever lane type carries it.
// ---------------------------------------------------------------------------
template <class V>
struct Lane;

template <>
struct Lane<float> {
    static constexpr int N = 1;
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
    static __device__ __forceinline__ float bc(float s) { return s; }
    static __device__ __forceinline__ float get(float v, int) { return v; }
    static __device__ __forceinline__ void set(float& v, int, float s) { v = s; }
};

// The packed forms are written as PTX with an explicit round-to-nearest
// modifier.  A packed difference whose operand is a packed product was still
// measured to round as if fused (a - b c in one rounding) on sm_103a, so the
// model never subtracts a product: a b - c d is written fma(a, b, (-c) d), with
// the negation exact, in both lane widths.
__device__ __forceinline__ unsigned long long f2_bits(float2 v)
{
    unsigned long long r;
    memcpy(&r, &v, 8);
    return r;
}

__device__ __forceinline__ float2 f2_from(unsigned long long r)
{
    float2 v;
    memcpy(&v, &r, 8);
    return v;
}

template <>
struct Lane<float2> {
    static constexpr int N = 2;
    static __device__ __forceinline__ float2 add(float2 a, float2 b)
    {
        unsigned long long d;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
        return f2_from(d);
    }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b)
    {
        unsigned long long d;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
        return f2_from(d);
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b)
    {
        unsigned long long d;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
        return f2_from(d);
    }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c)
    {
        unsigned long long d;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
        return f2_from(d);
    }
    static __device__ __forceinline__ float2 neg(float2 a) { return mul(a, make_float2(-1.0f, -1.0f)); }
    static __device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
    static __device__ __forceinline__ float get(float2 v, int i) { return i ? v.y : v.x; }
    static __device__ __forceinline__ void set(float2& v, int i, float s)
    {
        if (i) v.y = s;
        else v.x = s;
    }
};

// Model and cost constants duplicated into lane pairs (staged once per block in
// shared memory for the two-sample rollout).
struct __align__(16) PairConsts {
    float2 Q[12];
    float2 R[3], w_fc;
    float2 foot[12], nfoot[12];  // lever arms and their negatives
    float2 gyro[3], inv_mass;
    float2 inv_inertia[3], dt;
    float2 gravity[3], nmu;      // -mu
    float2 fe[3], zero;          // f_ext
};

// The constants a lane type reads: the parameter block itself for one sample
// per thread, the duplicated pairs for two.
template <class V>
struct Consts;

template <>
struct Consts<float> {
    const InstParams& P;
    __device__ __forceinline__ float Q(int c) const { return P.Q[c]; }
    __device__ __forceinline__ float R(int a) const { return P.R[a]; }
    __device__ __forceinline__ float w_fc() const { return P.w_fc; }
    __device__ __forceinline__ float nmu() const { return -P.mu; }
    __device__ __forceinline__ float foot(int i) const { return P.foot[i]; }
    __device__ __forceinline__ float nfoot(int i) const { return -P.foot[i]; }
    __device__ __forceinline__ float gyro(int a) const { return P.gyro[a]; }
    __device__ __forceinline__ float inv_inertia(int a) const { return P.inv_inertia[a]; }
    __device__ __forceinline__ float inv_mass() const { return P.inv_mass; }
    __device__ __forceinline__ float dt() const { return P.dt; }
    __device__ __forceinline__ float gravity(int a) const { return P.gravity[a]; }
};

template <>
struct Consts<float2> {
    const PairConsts& C;
    __device__ __forceinline__ float2 Q(int c) const { return C.Q[c]; }
    __device__ __forceinline__ float2 R(int a) const { return C.R[a]; }
    __device__ __forceinline__ float2 w_fc() const { return C.w_fc; }
    __device__ __forceinline__ float2 nmu() const { return C.nmu; }
    __device__ __forceinline__ float2 foot(int i) const { return C.foot[i]; }
    __device__ __forceinline__ float2 nfoot(int i) const { return C.nfoot[i]; }
    __device__ __forceinline__ float2 gyro(int a) const { return C.gyro[a]; }
    __device__ __forceinline__ float2 inv_inertia(int a) const { return C.inv_inertia[a]; }
    __device__ __forceinline__ float2 inv_mass() const { return C.inv_mass; }
    __device__ __forceinline__ float2 dt() const { return C.dt; }
    __device__ __forceinline__ float2 gravity(int a) const { return C.gravity[a]; }
};

// Fill the pair constants (threads 0..63 of a block; f_ext given).
__device__ __forceinline__ void fill_pair_consts(PairConsts& C, const InstParams& P, const float fe[3])
{
    const int t = threadIdx.x;
    auto dup = [](float v) { return make_float2(v, v); };
    if (t < 12) {
        C.Q[t] = dup(P.Q[t]);
        C.foot[t] = dup(P.foot[t]);
        C.nfoot[t] = dup(-P.foot[t]);
    } else if (t < 15) {
        const int a = t - 12;
        C.R[a] = dup(P.R[a]);
        C.gyro[a] = dup(P.gyro[a]);
        C.inv_inertia[a] = dup(P.inv_inertia[a]);
        C.gravity[a] = dup(P.gravity[a]);
        C.fe[a] = dup(fe[a]);
    } else if (t == 15) {
        C.w_fc = dup(P.w_fc);
        C.inv_mass = dup(P.inv_mass);
        C.dt = dup(P.dt);
        C.nmu = dup(-P.mu);
        C.zero = dup(0.0f);
    }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies; the high halves are XORed with the other counter words and the
// round key, which advances by the Weyl constants each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// Philox4x32-10 for one sample k and one tick: counters (k, d, iter lo, iter hi)
// with only the draw index d varying along the rollout.  The first round's
// products involve only k and iter, the second round's second product only
// round-one words that do not depend on d, and the third round's first product
// only such words again; those products (and the round keys folded into the
// XORs) are formed once per sample, leaving one product in round two, one in
// round three and two in each of rounds four to ten per draw.  Bit-identical to
// philox4x32_10.
struct PhiloxPre {
    uint32_t B;    // round 1 word x XOR d (hi(M1 iter_lo) ^ k0)
    uint32_t W1K;  // round 1 word w ^ round-2 key k1
    uint32_t Y2K;  // round 2 word y ^ round-3 key k0
    uint32_t FHK;  // hi(M0 x2) ^ round-3 key k1
    uint32_t FLO;  // lo(M0 x2): round 3 word w
    uint32_t k0, k1;
};

__device__ __forceinline__ PhiloxPre philox_pre(uint32_t k, uint64_t iter, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    const uint32_t lo = (uint32_t)iter, hi = (uint32_t)(iter >> 32);
    const uint64_t a = (uint64_t)M0 * k, b = (uint64_t)M1 * lo;
    PhiloxPre p;
    p.B = (uint32_t)(b >> 32) ^ k0;
    const uint32_t y1 = (uint32_t)b, z1 = (uint32_t)(a >> 32) ^ hi ^ k1, w1 = (uint32_t)a;
    const uint64_t e = (uint64_t)M1 * z1;
    const uint32_t x2 = (uint32_t)(e >> 32) ^ y1 ^ (k0 + W0), y2 = (uint32_t)e;
    const uint64_t f = (uint64_t)M0 * x2;
    p.W1K = w1 ^ (k1 + W1);
    p.Y2K = y2 ^ (k0 + 2u * W0);
    p.FHK = (uint32_t)(f >> 32) ^ (k1 + 2u * W1);
    p.FLO = (uint32_t)f;
    p.k0 = k0;
    p.k1 = k1;
    return p;
}

__device__ __forceinline__ uint4 philox_draw(const PhiloxPre& p, uint32_t d)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    const uint64_t c = (uint64_t)M0 * (p.B ^ d);  // round 2, first product
    const uint32_t z2 = (uint32_t)(c >> 32) ^ p.W1K;
    const uint64_t g = (uint64_t)M1 * z2;  // round 3, second product
    uint4 s = make_uint4((uint32_t)(g >> 32) ^ p.Y2K, (uint32_t)g, p.FHK ^ (uint32_t)c, p.FLO);
    uint32_t k0 = p.k0 + 3u * W0, k1 = p.k1 + 3u * W1;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)M0 * s.x, p1 = (uint64_t)M1 * s.z;
        s = make_uint4((uint32_t)(p1 >> 32) ^ s.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ s.w ^ k1, (uint32_t)p0);
        k0 += W0;
        k1 += W1;
    }
    return s;
}

// Square root by the hardware approximation: relative error below 1.1e-7 (under
// one ulp; measured against double precision over every single-precision
// mantissa of both exponent parities), sqrt(0) = 0.
__device__ __forceinline__ float sqrt_hw(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box-Muller on two words (the step-frequency draw): the top 24 bits give exact
// uniforms u1 in (0, 1] and u2 in [0, 1).  The radius uses the accurate
// logarithm, since the frequency's rounding to integer mHz must match the exact
// transform (its argument is often within a few ulp of 1), and x * rsqrt(x) for
// the square root; the angle uses the hardware sine/cosine, whose absolute error
// (about 4e-7 on [0, 2 pi)) moves a normal by at most 3e-6.
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b)
{
    const float two_m24 = 5.9604644775390625e-8f;
    const float u1 = __uint2float_rn((a >> 8) + 1u) * two_m24;
    const float u2 = __uint2float_rn(b >> 8) * two_m24;
    const float r2 = -2.0f * logf(u1);
    const float r = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
    float s, c;
    __sincosf(6.28318530717958648f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

// Box-Muller on two 21-bit integers (the force normals): u1 = (a + 1) 2^-21 in
// (0, 1] and u2 = b 2^-21 in [0, 1) (exact).  The radius uses the hardware
// base-2 logarithm (absolute error at most 2^-22 on [0.5, 2], 2 ulp below), so
// ln u1 is off by at most e = 2^-22 ln 2 = 1.65e-7 there: with r = sqrt(-2 ln u1)
// the radius moves by at most min(2 e / r, sqrt(2 e)), about 1e-6 at typical radii
// and at most sqrt(2 e) = 5.7e-4 at the smallest (u1 within a few 2^-21 of 1).
// These are the sampler's draws, not model arithmetic: the accurate routine cost
// 12 % of the rollout.  The square root is sqrt_hw (a logarithm slightly above 0
// gives r = 0); the angle is as above.  The integers (at most 2^21) are turned
// into floats without a conversion instruction: 0x4B000000 | n is the float
// 2^23 + n, and fma(2^23 + n, c, -2^23 c) is n c rounded once, the same bits as
// float(n) * c.
template <class V>
__device__ __forceinline__ void box_muller21_v(const uint32_t* a, const uint32_t* b, V& z0, V& z1)
{
    using L = Lane<V>;
    const float two_m21 = 4.76837158203125e-7f;
    const float c_ang = 6.28318530717958648f * two_m21;
    V ia, ib;
#pragma unroll
    for (int i = 0; i < L::N; ++i) {
        L::set(ia, i, __int_as_float(0x4b000000 | (int)(a[i] + 1u)));
        L::set(ib, i, __int_as_float(0x4b000000 | (int)b[i]));
    }
    const V u1 = L::fma(ia, L::bc(two_m21), L::bc(-4.0f));
    const V ang = L::fma(ib, L::bc(c_ang), L::bc(-8388608.0f * c_ang));
    V lg, r, sn, cs;
#pragma unroll
    for (int i = 0; i < L::N; ++i) L::set(lg, i, __log2f(L::get(u1, i)));
    const V r2 = L::mul(L::bc(-1.38629436111989061f), lg);  // -2 ln 2 log2(u1)
#pragma unroll
    for (int i = 0; i < L::N; ++i) {
        L::set(r, i, sqrt_hw(fmaxf(L::get(r2, i), 0.0f)));
        float si, ci;
        __sincosf(L::get(ang, i), &si, &ci);
        L::set(sn, i, si);
        L::set(cs, i, ci);
    }
    z0 = L::mul(r, cs);
    z1 = L::mul(r, sn);
}

__device__ __forceinline__ float2 box_muller21(uint32_t a, uint32_t b)
{
    float z0, z1;
    box_muller21_v<float>(&a, &b, z0, z1);
    return make_float2(z0, z1);
}

// The six force normals of one 128-bit draw: six 21-bit integers (the top 21
// bits of each word, then the low 11 bits of words 0 and 2 joined to the low 10
// bits of words 1 and 3), Box-Muller on the pairs (u0, u1), (u2, u3), (u4, u5).
template <class V>
__device__ __forceinline__ void normals6_v(const uint4* w, V* e)
{
    constexpr int N = Lane<V>::N;
    uint32_t a[3][N], b[3][N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        a[0][i] = w[i].x >> 11;
        b[0][i] = w[i].y >> 11;
        a[1][i] = w[i].z >> 11;
        b[1][i] = w[i].w >> 11;
        a[2][i] = ((w[i].x & 0x7ffu) << 10) | (w[i].y & 0x3ffu);
        b[2][i] = ((w[i].z & 0x7ffu) << 10) | (w[i].w & 0x3ffu);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) box_muller21_v<V>(a[p], b[p], e[2 * p], e[2 * p + 1]);
}

__device__ __forceinline__ void normals6(uint4 w, float* e) { normals6_v<float>(&w, e); }

// The 12 force normals of step (or knot) j: draws 1 + 2j and 2 + 2j, counter
// (k, draw, iter lo, iter hi), key (seed, ctrl).
__device__ __forceinline__ void normals12(uint32_t k, int j, uint64_t iter, uint32_t seed, uint32_t ctrl,
                                          float e[12])
{
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const uint4 w = philox4x32_10(
            make_uint4(k, 1u + 2u * (uint32_t)j + (uint32_t)d, (uint32_t)iter, (uint32_t)(iter >> 32)), seed, ctrl);
        normals6(w, e + 6 * d);
    }
}

// The same 12 normals from a sample's precomputed Philox state.
__device__ __forceinline__ void normals12(const PhiloxPre& pp, int j, float e[12])
{
#pragma unroll
    for (int d = 0; d < 2; ++d) normals6(philox_draw(pp, 1u + 2u * (uint32_t)j + (uint32_t)d), e + 6 * d);
}

// Regeneration of the sampled deviations sigma * eps (for readers of a solve that
// did not store them): the same draws and the same operations as the rollout,
// so the same bits.  Force normal c of step (or knot) j comes from draw
// 1 + 2 j + (c >= 6), slot s = c mod 6: Box-Muller pair s / 2 of that draw's six
// 21-bit integers, its cosine output for even s and sine output for odd s.
__device__ __forceinline__ float2 draw_pair(uint4 w, int p)
{
    uint32_t a, b;
    if (p == 0) {
        a = w.x >> 11;
        b = w.y >> 11;
    } else if (p == 1) {
        a = w.z >> 11;
        b = w.w >> 11;
    } else {
        a = ((w.x & 0x7ffu) << 10) | (w.y & 0x3ffu);
        b = ((w.z & 0x7ffu) << 10) | (w.w & 0x3ffu);
    }
    return box_muller21(a, b);
}

// Deviations 4 qd .. 4 qd + 3 of sample k at step j (sd4: their standard
// deviations).  Quads 0 and 2 lie in one draw each, quad 1 spans both.
__device__ __forceinline__ float4 regen_quad(uint32_t k, int j, int qd, uint64_t iter, uint32_t seed, uint32_t ctrl,
                                             float4 sd4)
{
    const uint32_t dA = 1u + 2u * (uint32_t)j;
    const uint4 ctr = make_uint4(k, qd == 2 ? dA + 1u : dA, (uint32_t)iter, (uint32_t)(iter >> 32));
    const uint4 w0 = philox4x32_10(ctr, seed, ctrl);
    float2 p0, p1;
    if (qd == 0) {
        p0 = draw_pair(w0, 0);
        p1 = draw_pair(w0, 1);
    } else if (qd == 2) {
        p0 = draw_pair(w0, 1);
        p1 = draw_pair(w0, 2);
    } else {
        const uint4 w1 = philox4x32_10(make_uint4(k, dA + 1u, (uint32_t)iter, (uint32_t)(iter >> 32)), seed, ctrl);
        p0 = draw_pair(w0, 2);
        p1 = draw_pair(w1, 0);
    }
    return make_float4(__fmul_rn(sd4.x, p0.x), __fmul_rn(sd4.y, p0.y), __fmul_rn(sd4.z, p1.x),
                       __fmul_rn(sd4.w, p1.y));
}

// All 12 deviations of sample k at step (or knot) j (sd12: their standard deviations).
__device__ __forceinline__ void regen_row(uint32_t k, int j, uint64_t iter, uint32_t seed, uint32_t ctrl,
                                          const float* sd12, float d[12])
{
    float e[12];
    normals12(k, j, iter, seed, ctrl, e);
#pragma unroll
    for (int c = 0; c < 12; ++c) d[c] = __fmul_rn(sd12[c], e[c]);
}

// Step frequency of sample k (Sec. IV-C): clip(mu_f + sigma_f z, f_min, f_max)
// quantised to integer mHz.  The exact single-precision sequence (one fused
// multiply-add, one multiply, one add, floor) defines the rounding.
__device__ __forceinline__ uint32_t sample_freq(uint32_t k, uint64_t iter, uint32_t seed, uint32_t ctrl,
                                                float mu_f, float sig_f, float f_min, float f_max)
{
    const uint4 w = philox4x32_10(make_uint4(k, 0u, (uint32_t)iter, (uint32_t)(iter >> 32)), seed, ctrl);
    const float z = box_muller(w.x, w.y).x;
    float f = __fmaf_rn(sig_f, z, mu_f);
    if (f < f_min) f = f_min;
    if (f > f_max) f = f_max;
    const float t = __fmul_rn(1000.0f, f);
    return (uint32_t)floorf(__fadd_rn(t, 0.5f));
}

// Entry of a discrete step-frequency set of n values drawn by sample k (Sec. V:
// uniform over the set): floor(n u / 2^24), u the top 24 bits of the frequency
// draw's first Philox word.
__device__ __forceinline__ int freq_block(uint32_t k, uint64_t iter, uint32_t seed, uint32_t ctrl, int n)
{
    const uint4 w = philox4x32_10(make_uint4(k, 0u, (uint32_t)iter, (uint32_t)(iter >> 32)), seed, ctrl);
    return (int)(((w.x >> 8) * (uint32_t)n) >> 24);
}

__device__ __forceinline__ uint32_t quantise_mhz(float f, float f_min, float f_max)
{
    if (f < f_min) f = f_min;
    if (f > f_max) f = f_max;
    return (uint32_t)floorf(__fadd_rn(__fmul_rn(1000.0f, f), 0.5f));
}

// Contact flag of one leg at step j for frequency q (mHz); 64-bit exact phase.
__device__ __forceinline__ int stance_at(const TickArgs& t, int leg, uint32_t q, uint32_t dt_us, int j)
{
    const uint64_t ph = ((uint64_t)t.phase0 + t.offset[leg] + (uint64_t)j * q * dt_us) % kPhaseOne;
    return ph < (uint64_t)t.duty ? 1 : 0;
}

// Kahan-compensated accumulation.
template <class V>
__device__ __forceinline__ void kahan_add_v(V& s, V& c, V v)
{
    using L = Lane<V>;
    const V y = L::sub(v, c);
    const V t = L::add(s, y);
    c = L::sub(L::sub(t, s), y);
    s = t;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) { kahan_add_v<float>(s, c, v); }

// ---------------------------------------------------------------------------
// One explicit-Euler step of Eq. (1) plus the stage cost of the pre-step state
// (Alg. 2 charges r(u_i, x_i, x^r_i) before x_{i+1} = f(x_i, u_i)).
// G: world-frame forces already zeroed on swing legs.  fe: f_ext / m.
// live: bit i clear when leg i swings on every lane of the warp; its terms are
// then skipped (a +0 force contributes +0 to every sum, so the result is
// unchanged for finite states).
// ---------------------------------------------------------------------------
// Rows of 12 lane values from 16-byte aligned shared memory (one sample per
// thread: 3 vector loads; two: 6, each holding two duplicated pairs).
template <class V>
__device__ __forceinline__ void load_row12(const V* p, V out[12])
{
    const float4* p4 = reinterpret_cast<const float4*>(p);
    if constexpr (Lane<V>::N == 1) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 a = p4[q];
            out[4 * q] = a.x;
            out[4 * q + 1] = a.y;
            out[4 * q + 2] = a.z;
            out[4 * q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 a = p4[q];
            out[2 * q] = make_float2(a.x, a.y);
            out[2 * q + 1] = make_float2(a.z, a.w);
        }
    }
}

// The state part of the stage cost, sum_c Q_c (x_c - x^r_c)^2 (Sec. V).  It reads
// the state only, so a rollout may form it ahead of the step's draws.
template <class V>
__device__ __forceinline__ V stage_state_cost_v(const Consts<V>& K, const V x[12], const V* xr)
{
    using L = Lane<V>;
    V xrr[12];
    load_row12<V>(xr, xrr);
    V r = L::bc(0.0f);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const V e = L::sub(x[c], xrr[c]);
        r = L::fma(L::mul(K.Q(c), e), e, r);
    }
    return r;
}

// The force part added to r: R-weighted squared forces and, with penalty, the
// friction-cone penalty of the stance legs.
// The same from a reference row of single floats, broadcast to both lanes.
__device__ __forceinline__ float2 stage_state_cost_bc(const Consts<float2>& K, const float2 x[12], const float* xr)
{
    using L = Lane<float2>;
    const float4* r4 = reinterpret_cast<const float4*>(xr);
    float xs[12];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 a = r4[q];
        xs[4 * q] = a.x;
        xs[4 * q + 1] = a.y;
        xs[4 * q + 2] = a.z;
        xs[4 * q + 3] = a.w;
    }
    float2 r = L::bc(0.0f);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float2 e = L::sub(x[c], L::bc(xs[c]));
        r = L::fma(L::mul(K.Q(c), e), e, r);
    }
    return r;
}

template <class V>
__device__ __forceinline__ V stage_force_cost_v(const Consts<V>& K, V r, const V G[12], unsigned live, bool penalty)
{
    using L = Lane<V>;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!(live & (1u << i))) continue;  // zero force on every lane: adds exactly nothing
        const V gx = G[3 * i], gy = G[3 * i + 1], gz = G[3 * i + 2];
        r = L::fma(L::mul(K.R(0), gx), gx, r);
        r = L::fma(L::mul(K.R(1), gy), gy, r);
        r = L::fma(L::mul(K.R(2), gz), gz, r);
        if (!penalty) continue;  // forces already projected onto the cone
        // friction cone on stance legs; a swing leg's zero force adds nothing
        // (|G_xy| by sqrt_hw, exact zero for a zero force)
        const V t2 = L::fma(gx, gx, L::mul(gy, gy));
        V sq, sp, gn;
#pragma unroll
        for (int l = 0; l < L::N; ++l) L::set(sq, l, sqrt_hw(L::get(t2, l)));
        const V slip = L::fma(K.nmu(), gz, sq);
#pragma unroll
        for (int l = 0; l < L::N; ++l) {
            L::set(sp, l, fmaxf(L::get(slip, l), 0.0f));
            L::set(gn, l, fminf(L::get(gz, l), 0.0f));
        }
        const V pen = L::fma(gn, gn, L::mul(sp, sp));
        r = L::fma(K.w_fc(), pen, r);
    }
    return r;
}

template <class V>
__device__ __forceinline__ V stage_cost_v(const Consts<V>& K, const V x[12], const V* xr, const V G[12],
                                          unsigned live, bool penalty)
{
    return stage_force_cost_v<V>(K, stage_state_cost_v<V>(K, x, xr), G, live, penalty);
}

__device__ __forceinline__ float stage_cost(const InstParams& P, const float x[12], const float* xr,
                                            const float G[12], unsigned live = 0xfu, bool penalty = true)
{
    return stage_cost_v<float>(Consts<float>{P}, x, xr, G, live, penalty);
}

// Orthogonal projection of one force onto the friction cone |G_xy| <= mu G_z
// (Sec. IV-B): unchanged inside, zero in the polar cone (mu |G_xy| <= -G_z),
// otherwise the nearest point of the boundary, G_z' = lambda = (mu |G_xy| + G_z)
// / (1 + mu^2) and |G_xy'| = mu lambda.  A swing leg's zero force stays zero.
__device__ __forceinline__ void cone_project(float mu, float inv_1pmu2, float& gx, float& gy, float& gz)
{
    const float s2 = fmaf(gx, gx, gy * gy);
    const float s = sqrt_hw(s2);
    if (s <= mu * gz) return;
    if (mu * s <= -gz) {
        gx = gy = gz = 0.0f;
        return;
    }
    const float lam = fmaf(mu, s, gz) * inv_1pmu2;
    const float k = mu * lam / s;
    gx *= k;
    gy *= k;
    gz = lam;
}

// sin and cos of attitude angles, written here rather than taken from the math
// library so that two samples' reduction and polynomials issue as packed
// instructions.  Cody-Waite reduction (Cody & Waite, 1980): j = rint(2 x / pi)
// from the low bits of fma(x, 2/pi, 1.5 2^23), r = x - j pi/2 with pi/2 in three
// single-precision parts subtracted one fused multiply-add at a time (the first
// step is exact: j P1 and x lie within a factor of two); on |r| <= pi/4,
// sin r = r + r^3 (s1 + s2 r^2 + s3 r^4) and cos r = 1 + r^2 (c1 + .. + c4 r^6)
// by Horner; the quadrant j mod 4 swaps and negates.  Constants from
// paper_2403_11383_b300/sincos_coefficients.py (least-squares fits on Chebyshev
// nodes; fit error 1.3e-8 relative for sin, 7.5e-10 for cos).  Beyond
// |x| = kSinCosMax (a rollout that has long left any meaningful attitude: its
// cost is infinite or ungated) and for non-finite x the lane takes the hardware
// approximation, which costs a few instructions where the accurate library
// routine would take its slow reduction path.  Both are formed on every lane and
// the lane selects (2.4 % off the batched tick against a per-lane branch).
constexpr float kSinCosMax = 65536.0f;

template <class V>
__device__ __forceinline__ void sincos_v(V x, V& s, V& c)
{
    using L = Lane<V>;
    const float magic = 12582912.0f;  // 1.5 2^23
    const V jm = L::fma(x, L::bc(0x1.45f306p-1f), L::bc(magic));
    const V j = L::sub(jm, L::bc(magic));
    V r = L::fma(j, L::bc(-0x1.921fb6p+0f), x);
    r = L::fma(j, L::bc(0x1.777a5cp-25f), r);
    r = L::fma(j, L::bc(0x1.ee59dap-50f), r);
    const V u = L::mul(r, r);
    V ps = L::fma(u, L::bc(-0x1.9aca02p-13f), L::bc(0x1.110c2ap-7f));
    ps = L::fma(u, ps, L::bc(-0x1.555552p-3f));
    const V sn = L::fma(L::mul(u, r), ps, r);
    V pc = L::fma(u, L::bc(0x1.9a6f60p-16f), L::bc(-0x1.6c0e0ap-10f));
    pc = L::fma(u, pc, L::bc(0x1.55554cp-5f));
    pc = L::fma(u, pc, L::bc(-0.5f));
    const V cs = L::fma(u, pc, L::bc(1.0f));
#pragma unroll
    for (int l = 0; l < L::N; ++l) {
        const float xl = L::get(x, l);
        const int q = __float_as_int(L::get(jm, l));
        const float a = L::get(sn, l), b = L::get(cs, l);
        float sl = (q & 1) ? b : a, cl = (q & 1) ? a : b;
        sl = __int_as_float(__float_as_int(sl) ^ ((q & 2) << 30));
        cl = __int_as_float(__float_as_int(cl) ^ (((q + 1) & 2) << 30));
        float hs, hc;  // formed on every lane and selected: a per-lane branch splits the step's code
        __sincosf(xl, &hs, &hc);
        const bool big = !(fabsf(xl) <= kSinCosMax);
        sl = big ? hs : sl;
        cl = big ? hc : cl;
        L::set(s, l, sl);
        L::set(c, l, cl);
    }
}

template <class V>
__device__ __forceinline__ void angle_sincos_v(V a, V& s, V& c)
{
    sincos_v<V>(a, s, c);
}

// The rotational and translational rates of Eq. (1) from the net force F and
// body-frame moment t, then the explicit Euler step of all 12 states.
template <class V>
__device__ __forceinline__ void srbd_integrate_v(const Consts<V>& K, V x[12], V sr, V cr, V sp, V cp, V F0, V F1,
                                                 V F2, V t0, V t1, V t2, const V fe[3])
{
    using L = Lane<V>;
    const V w0 = x[9], w1 = x[10], w2 = x[11];
    // I^{-1} (t - omega x I omega) with a diagonal I: component a is
    // t_a / I_a + omega_{a+1} omega_{a+2} (I_{a+1} - I_{a+2}) / I_a
    const V wd0 = L::fma(L::mul(w1, w2), K.gyro(0), L::mul(t0, K.inv_inertia(0)));
    const V wd1 = L::fma(L::mul(w2, w0), K.gyro(1), L::mul(t1, K.inv_inertia(1)));
    const V wd2 = L::fma(L::mul(w0, w1), K.gyro(2), L::mul(t2, K.inv_inertia(2)));
    // E'^{-1}(Phi) omega for the ZYX angles
    V ic;
#pragma unroll
    for (int l = 0; l < L::N; ++l) L::set(ic, l, __fdividef(1.0f, L::get(cp, l)));
    const V a = L::fma(sr, w1, L::mul(cr, w2));
    const V rd = L::fma(L::mul(sp, ic), a, w0);
    const V pd = L::fma(cr, w1, L::mul(L::neg(sr), w2));
    const V yd = L::mul(a, ic);
    const V dt = K.dt();
    const V vd0 = L::fma(L::add(F0, fe[0]), K.inv_mass(), K.gravity(0));
    const V vd1 = L::fma(L::add(F1, fe[1]), K.inv_mass(), K.gravity(1));
    const V vd2 = L::fma(L::add(F2, fe[2]), K.inv_mass(), K.gravity(2));
    x[0] = L::fma(dt, x[6], x[0]);
    x[1] = L::fma(dt, x[7], x[1]);
    x[2] = L::fma(dt, x[8], x[2]);
    x[3] = L::fma(dt, rd, x[3]);
    x[4] = L::fma(dt, pd, x[4]);
    x[5] = L::fma(dt, yd, x[5]);
    x[6] = L::fma(dt, vd0, x[6]);
    x[7] = L::fma(dt, vd1, x[7]);
    x[8] = L::fma(dt, vd2, x[8]);
    x[9] = L::fma(dt, wd0, w0);
    x[10] = L::fma(dt, wd1, w1);
    x[11] = L::fma(dt, wd2, w2);
}

__device__ __forceinline__ void srbd_integrate(const InstParams& P, float x[12], float sr, float cr, float sp,
                                               float cp, float F0, float F1, float F2, float t0, float t1,
                                               float t2, const float fe[3])
{
    srbd_integrate_v<float>(Consts<float>{P}, x, sr, cr, sp, cp, F0, F1, F2, t0, t1, t2, fe);
}

// Body-to-world rotation R = Rz(yaw) Ry(pitch) Rx(roll) from the attitude's
// sines and cosines; R20 = -sin(pitch) is left to the caller.
template <class V>
struct Rot {
    V R00, R01, R02, R10, R11, R12, R21, R22;
};

template <class V>
__device__ __forceinline__ Rot<V> rotation_v(V sr, V cr, V sp, V cp, V sy, V cy)
{
    using L = Lane<V>;
    Rot<V> R;
    const V t = L::mul(cy, sp), u = L::mul(sy, sp);
    R.R00 = L::mul(cy, cp);
    R.R01 = L::fma(t, sr, L::mul(L::neg(sy), cr));
    R.R02 = L::fma(t, cr, L::mul(sy, sr));
    R.R10 = L::mul(sy, cp);
    R.R11 = L::fma(u, sr, L::mul(cy, cr));
    R.R12 = L::fma(u, cr, L::mul(L::neg(cy), sr));
    R.R21 = L::mul(cp, sr);
    R.R22 = L::mul(cp, cr);
    return R;
}

// The attitude's sines and cosines and the body-to-world rotation of the
// pre-step state: they read the state only, so a rollout may form them ahead of
// the step's draws.
template <class V>
struct Attitude {
    V sr, cr, sp, cp, sy, cy;
    Rot<V> R;
};

template <class V>
__device__ __forceinline__ Attitude<V> attitude_v(const V x[12])
{
    Attitude<V> A;
    angle_sincos_v<V>(x[3], A.sr, A.cr);
    angle_sincos_v<V>(x[4], A.sp, A.cp);
    angle_sincos_v<V>(x[5], A.sy, A.cy);
    A.R = rotation_v<V>(A.sr, A.cr, A.sp, A.cp, A.sy, A.cy);
    return A;
}

// One explicit Euler step of Eq. (1) from the pre-step attitude A.
template <class V>
__device__ __forceinline__ void srbd_step_att_v(const Consts<V>& K, V x[12], const V G[12], const V fe[3],
                                                unsigned live, const Attitude<V>& A)
{
    using L = Lane<V>;
    const V sr = A.sr, cr = A.cr, sp = A.sp, cp = A.cp;
    const Rot<V>& R = A.R;
    const V nsp = L::neg(sp);  // R20
    V F0 = L::bc(0.0f), F1 = F0, F2 = F0, t0 = F0, t1 = F0, t2 = F0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!(live & (1u << i))) continue;  // zero force on every lane: adds exactly nothing
        const V gx = G[3 * i], gy = G[3 * i + 1], gz = G[3 * i + 2];
        F0 = L::add(F0, gx);
        F1 = L::add(F1, gy);
        F2 = L::add(F2, gz);
        // body-frame force R^T Gamma_i, then the lever arm cross product
        const V bx = L::fma(R.R00, gx, L::fma(R.R10, gy, L::mul(nsp, gz)));
        const V by = L::fma(R.R01, gx, L::fma(R.R11, gy, L::mul(R.R21, gz)));
        const V bz = L::fma(R.R02, gx, L::fma(R.R12, gy, L::mul(R.R22, gz)));
        t0 = L::fma(K.nfoot(3 * i + 2), by, L::fma(K.foot(3 * i + 1), bz, t0));
        t1 = L::fma(K.nfoot(3 * i), bz, L::fma(K.foot(3 * i + 2), bx, t1));
        t2 = L::fma(K.nfoot(3 * i + 1), bx, L::fma(K.foot(3 * i), by, t2));
    }
    srbd_integrate_v<V>(K, x, sr, cr, sp, cp, F0, F1, F2, t0, t1, t2, fe);
}

template <class V>
__device__ __forceinline__ void srbd_step_v(const Consts<V>& K, V x[12], const V G[12], const V fe[3],
                                            unsigned live = 0xfu)
{
    srbd_step_att_v<V>(K, x, G, fe, live, attitude_v<V>(x));
}

__device__ __forceinline__ void srbd_step(const InstParams& P, float x[12], const float G[12],
                                          const float fe[3], unsigned live = 0xfu)
{
    srbd_step_v<float>(Consts<float>{P}, x, G, fe, live);
}

// The same step with stance feet fixed on the ground z = 0: the lever arm of leg
// i is p_f,i - p_c, so the body moment is R^T sum_i (p_f,i - p_c) x Gamma_i
// (fx, fy: the feet's ground positions).  Legs in touch land at this step: they
// first take the foothold of the pre-step state (Sec. IV-D), the hip R (foot x,
// foot y, 0) from the CoM plus tsh v^d + sqrt(p_c,z / g) (v_c - v^d), with
// tsh = T_st / 2 and (vdx, vdy) the desired planar velocity.
__device__ __forceinline__ void srbd_step_world(const InstParams& P, float x[12], const float G[12],
                                                const float fe[3], unsigned live, float fx[4], float fy[4],
                                                unsigned touch, float vdx, float vdy, float tsh)
{
    float sr, cr, sp, cp, sy, cy;
    sincos_v<float>(x[3], sr, cr);
    sincos_v<float>(x[4], sp, cp);
    sincos_v<float>(x[5], sy, cy);
    const Rot<float> Rm = rotation_v<float>(sr, cr, sp, cp, sy, cy);
    const float R00 = Rm.R00, R01 = Rm.R01, R02 = Rm.R02, R10 = Rm.R10, R11 = Rm.R11, R12 = Rm.R12;
    const float R20 = -sp, R21 = Rm.R21, R22 = Rm.R22;
    if (touch) {
        const float s = sqrtf(fmaxf(x[2], 0.0f) * P.inv_g);
        const float ax = fmaf(s, x[6] - vdx, tsh * vdx), ay = fmaf(s, x[7] - vdy, tsh * vdy);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (touch & (1u << i)) {
                const float hx = P.foot[3 * i], hy = P.foot[3 * i + 1];
                fx[i] = x[0] + (R00 * hx + R01 * hy) + ax;
                fy[i] = x[1] + (R10 * hx + R11 * hy) + ay;
            }
        }
    }
    float F0 = 0.f, F1 = 0.f, F2 = 0.f, u0 = 0.f, u1 = 0.f, u2 = 0.f;  // u: world moment
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!(live & (1u << i))) continue;
        const float gx = G[3 * i], gy = G[3 * i + 1], gz = G[3 * i + 2];
        F0 += gx;
        F1 += gy;
        F2 += gz;
        const float dx = fx[i] - x[0], dy = fy[i] - x[1], dz = -x[2];
        u0 += dy * gz - dz * gy;
        u1 += dz * gx - dx * gz;
        u2 += dx * gy - dy * gx;
    }
    const float t0 = R00 * u0 + R10 * u1 + R20 * u2;
    const float t1 = R01 * u0 + R11 * u1 + R21 * u2;
    const float t2 = R02 * u0 + R12 * u1 + R22 * u2;
    srbd_integrate(P, x, sr, cr, sp, cp, F0, F1, F2, t0, t1, t2, fe);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Sum of 12 per-lane values over a warp.  On return, lane l holds the warp
// totals of components c0 + 0..2 with c0 = 6 (l & 16 ? 1 : 0) + 3 (l & 8 ? 1 : 0);
// lanes with (l & 7) == 0 are the designated writers.  18 shuffles in place of
// 60 for twelve independent butterflies.
__device__ __forceinline__ int warp_sum12(const float v[12], float out[3])
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    float a[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float send = h16 ? v[i] : v[i + 6];
        const float keep = h16 ? v[i + 6] : v[i];
        a[i] = keep + __shfl_xor_sync(kFull, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float send = h8 ? a[i] : a[i + 3];
        const float keep = h8 ? a[i + 3] : a[i];
        out[i] = keep + __shfl_xor_sync(kFull, send, 8);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) out[i] += __shfl_xor_sync(kFull, out[i], o);
    }
    return (h16 ? 6 : 0) + (h8 ? 3 : 0);
}

// Order-preserving map of a float cost to an unsigned key (NaN never occurs:
// non-finite costs are stored as +inf).
__device__ __forceinline__ uint32_t cost_key(float J)
{
    const uint32_t b = __float_as_uint(J);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

}  // namespace sbs
