// Device helpers shared by the RRS kernels: the direction stream (Philox4x32-10
// and the Alg. S1 / Alg. S4 direction maps) and the exact sign test behind
// exact halfspace counts.
//
// Direction stream formula (both this file and the independent CPU checker
// implement it from the same written definition):
//   key = (seed mod 2^32, seed >> 32), counter = (block, j, l-1, q).
//   unif(w) = float(2*(w >> 9) + 1) * 2^-24.
//   Gaussian i uses block i/4 and the word pair p = (i/2) mod 2:
//     R = sqrt(-2 ln unif(w_2p)), angle = 2*pi*unif(w_2p+1),
//     g = R cos(angle) for even i, R sin(angle) for odd i.
//   ln: exponent split, mantissa f in [sqrt(1/2), sqrt(2)], 2*atanh((f-1)/(f+1))
//       by its odd series to the s^13 term; sin/cos: exact quarter-turn
//       reduction to [-pi/4, pi/4] and Taylor series to x^9 / x^10.
//   Round 1 (Alg. S1): u = g / |g|.
//   Round l >= 2 (Alg. S4): theta = (pi/2) * unif(w_0 of block 0xFFFFFFFF) * alpha^(l-1);
//       u~ = (cos theta, sin theta * g'/|g'|) with g' the first d-1 Gaussians;
//       u = u~ - (2 v'u~ / v'v) v with v = e1 - pole (identity if v = 0).
//   Every operation is one IEEE-754 FP32 operation with round-to-nearest;
//   the _rn intrinsics below keep the compiler from fusing or reordering, so
//   the stream is bit-identical to any other faithful implementation.
#pragma once

#include <stdint.h>

namespace rrsdev {

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t a0 = c0, a2 = c2;
        const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ float unif01(uint32_t w)
{
    return __fmul_rn(__uint2float_rn(2u * (w >> 9) + 1u), 5.9604644775390625e-08f /* 2^-24 */);
}

// natural log on (0, 1]
__device__ __forceinline__ float stream_log(float a)
{
    const uint32_t bits = __float_as_uint(a);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float f = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (f > 1.41421356f) {
        f = __fmul_rn(f, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float z = __fmul_rn(s, s);
    float p = 1.0f / 13.0f;
    p = __fadd_rn(__fmul_rn(p, z), 1.0f / 11.0f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f / 9.0f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f / 7.0f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f / 5.0f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f / 3.0f);
    const float t = __fmul_rn(2.0f, s);
    const float w = __fmul_rn(t, __fmul_rn(z, p));
    const float lnf = __fadd_rn(t, w);
    const float ef = __int2float_rn(e);
    const float hi = __fmul_rn(ef, 0.693145751953125f);
    const float lo = __fmul_rn(ef, 1.42860682e-06f);
    return __fadd_rn(hi, __fadd_rn(lo, lnf));
}

// sin and cos of (pi/2) * a for a in [0, 4)
__device__ __forceinline__ void stream_sincos_qturn(float a, float& s_out, float& c_out)
{
    int q = __float2int_rz(a);
    float r = __fsub_rn(a, __int2float_rn(q));
    if (r > 0.5f) {
        r = __fsub_rn(r, 1.0f);
        q += 1;
    }
    const float x = __fmul_rn(r, 1.57079637f);
    const float z = __fmul_rn(x, x);
    float ps = 1.0f / 362880.0f;
    ps = __fadd_rn(__fmul_rn(ps, z), -(1.0f / 5040.0f));
    ps = __fadd_rn(__fmul_rn(ps, z), 1.0f / 120.0f);
    ps = __fadd_rn(__fmul_rn(ps, z), -(1.0f / 6.0f));
    const float sx = __fadd_rn(x, __fmul_rn(x, __fmul_rn(z, ps)));
    float pc = -(1.0f / 3628800.0f);
    pc = __fadd_rn(__fmul_rn(pc, z), 1.0f / 40320.0f);
    pc = __fadd_rn(__fmul_rn(pc, z), -(1.0f / 720.0f));
    pc = __fadd_rn(__fmul_rn(pc, z), 1.0f / 24.0f);
    pc = __fadd_rn(__fmul_rn(pc, z), -0.5f);
    const float cx = __fadd_rn(1.0f, __fmul_rn(z, pc));
    switch (q & 3) {
    case 0: s_out = sx;  c_out = cx;  break;
    case 1: s_out = cx;  c_out = -sx; break;
    case 2: s_out = -sx; c_out = -cx; break;
    default: s_out = -cx; c_out = sx; break;
    }
}

struct StreamKey {
    uint32_t k0, k1, j, round0, q;
};

__device__ __forceinline__ void stream_block(const StreamKey& key, uint32_t b, uint32_t w[4])
{
    uint32_t c0 = b, c1 = key.j, c2 = key.round0, c3 = key.q;
    philox4x32_10(c0, c1, c2, c3, key.k0, key.k1);
    w[0] = c0; w[1] = c1; w[2] = c2; w[3] = c3;
}

// Both Gaussians of the Box-Muller pair built from words (wa, wb).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& g_even, float& g_odd)
{
    const float U = unif01(wa), V = unif01(wb);
    const float R = __fsqrt_rn(__fmul_rn(-2.0f, stream_log(U)));
    float s, c;
    stream_sincos_qturn(__fmul_rn(4.0f, V), s, c);
    g_even = __fmul_rn(R, c);
    g_odd = __fmul_rn(R, s);
}

// Fill g[0..cnt) with the stream's Gaussians 0..cnt-1 (g has stride gs).
__device__ __forceinline__ void stream_gaussians(const StreamKey& key, int cnt, float* g, int gs)
{
    for (int b = 0; 4 * b < cnt; ++b) {
        uint32_t w[4];
        stream_block(key, (uint32_t)b, w);
        float g0, g1, g2, g3;
        box_muller(w[0], w[1], g0, g1);
        box_muller(w[2], w[3], g2, g3);
        const int i = 4 * b;
        if (i + 0 < cnt) g[(i + 0) * gs] = g0;
        if (i + 1 < cnt) g[(i + 1) * gs] = g1;
        if (i + 2 < cnt) g[(i + 2) * gs] = g2;
        if (i + 3 < cnt) g[(i + 3) * gs] = g3;
    }
}

// Direction j of round round0 (0-based) for query counter q, written to
// u[0..d) (stride us).  alpha_pow = alpha^round0 formed by repeated FP32
// products; pole has stride 1 (ignored in round 0).
__device__ __forceinline__ void stream_direction(uint64_t seed, uint32_t q, uint32_t round0, uint32_t j,
                                                 int d, float alpha_pow, const float* pole, float* u,
                                                 int us)
{
    StreamKey key{(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), j, round0, q};
    if (round0 == 0) {
        stream_gaussians(key, d, u, us);
        float s2 = 0.0f;
        for (int i = 0; i < d; ++i) s2 = __fadd_rn(s2, __fmul_rn(u[i * us], u[i * us]));
        const float nrm = __fsqrt_rn(s2);
        for (int i = 0; i < d; ++i) u[i * us] = __fdiv_rn(u[i * us], nrm);
        return;
    }
    uint32_t wc[4];
    stream_block(key, 0xFFFFFFFFu, wc);
    const float t = __fmul_rn(unif01(wc[0]), alpha_pow);
    float st, ct;
    stream_sincos_qturn(t, st, ct);
    if (d > 1) {
        stream_gaussians(key, d - 1, u + us, us);
        float s2 = 0.0f;
        for (int i = 1; i < d; ++i) s2 = __fadd_rn(s2, __fmul_rn(u[i * us], u[i * us]));
        const float nrm = __fsqrt_rn(s2);
        for (int i = 1; i < d; ++i) u[i * us] = __fmul_rn(st, __fdiv_rn(u[i * us], nrm));
    }
    u[0] = ct;
    // reflection e1 -> pole
    const float v0 = __fsub_rn(1.0f, pole[0]);
    float vv = __fmul_rn(v0, v0);
    for (int i = 1; i < d; ++i) vv = __fadd_rn(vv, __fmul_rn(pole[i], pole[i]));
    if (vv == 0.0f) return;
    float vu = __fmul_rn(v0, u[0]);
    for (int i = 1; i < d; ++i) vu = __fadd_rn(vu, __fmul_rn(-pole[i], u[i * us]));
    const float lam = __fdiv_rn(__fmul_rn(2.0f, vu), vv);
    u[0] = __fsub_rn(u[0], __fmul_rn(lam, v0));
    for (int i = 1; i < d; ++i) u[i * us] = __fsub_rn(u[i * us], __fmul_rn(lam, -pole[i]));
}

__device__ __forceinline__ float alpha_power(float alpha, int round0)
{
    float a = 1.0f;
    for (int t = 0; t < round0; ++t) a = __fmul_rn(a, alpha);
    return a;
}

// ---------------------------------------------------------------------------
// Exact sign of u'(x - z): FP64 evaluation with a forward error bound, then
// (rarely) an error-free expansion sum.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    const double bv = __dsub_rn(s, a);
    const double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// Renormalise the nonoverlapping expansion h[0..len) (increasing magnitude)
// into a shorter nonadjacent one (Shewchuk 1997, "Compress"); returns the
// new length.
static __device__ __noinline__ int expansion_compress(double* h, int len)
{
    if (len <= 1) return len;
    // top-down pass: sweep from the largest component, keeping the partial
    // sum Q and emitting a component whenever the sum cannot absorb the next
    int bottom = len - 1;
    double Q = h[len - 1];
    for (int i = len - 2; i >= 0; --i) {
        const double sum = __dadd_rn(Q, h[i]);
        const double err = __dsub_rn(h[i], __dsub_rn(sum, Q));
        if (err != 0.0) {
            h[bottom--] = sum;
            Q = err;
        } else {
            Q = sum;
        }
    }
    // bottom-up pass over the emitted components
    int top = 0;
    for (int i = bottom + 1; i < len; ++i) {
        const double sum = __dadd_rn(h[i], Q);
        const double err = __dsub_rn(Q, __dsub_rn(sum, h[i]));
        if (err != 0.0) h[top++] = err;
        Q = sum;
    }
    h[top++] = Q;
    return top;
}

template <typename TX>
__device__ __noinline__ int exact_sign_slow(const float* u, int us, const TX* x, const double* z, int d,
                                            int* err_flag)
{
    constexpr int CAP = 64;
    double h[CAP];
    int len = 0;
    auto grow = [&](double b) {
        if (b == 0.0) return;
        if (len == CAP) {
            len = expansion_compress(h, len);
            if (len == CAP) {
                atomicOr(err_flag, 4);
                return;
            }
        }
        double q = b;
        int out = 0;
        for (int i = 0; i < len; ++i) {
            double s, e;
            two_sum(q, h[i], s, e);
            if (e != 0.0) h[out++] = e;
            q = s;
        }
        if (q != 0.0) h[out++] = q;
        len = out;
    };
    for (int l = 0; l < d; ++l) {
        const double ul = (double)u[l * us];
        const double xl = (double)x[l];
        const double p = __dmul_rn(ul, xl);
        grow(p);
        grow(__fma_rn(ul, xl, -p));
        const double pz = __dmul_rn(ul, z[l]);
        grow(-pz);
        grow(-__fma_rn(ul, z[l], -pz));
    }
    if (len == 0) return 0;
    const double top = h[len - 1];
    return top > 0.0 ? 1 : (top < 0.0 ? -1 : 0);
}

template <typename TX>
__device__ __forceinline__ int exact_sign(const float* u, int us, const TX* x, const double* z, int d,
                                          int* err_flag)
{
    double a = 0.0, b = 0.0, mag = 0.0;
    for (int l = 0; l < d; ++l) {
        const double ul = (double)u[l * us];
        const double xl = (double)x[l];
        a = __fma_rn(ul, xl, a);
        b = __fma_rn(ul, z[l], b);
        mag = __dadd_rn(mag, __dmul_rn(fabs(ul), __dadd_rn(fabs(xl), fabs(z[l]))));
    }
    const double t = __dsub_rn(a, b);
    const double bound = (double)(2 * d + 8) * 1.1102230246251565e-16 /* 2^-53 */ * mag * (1.0 + 1e-12);
    if (t > bound) return 1;
    if (t < -bound) return -1;
    return exact_sign_slow<TX>(u, us, x, z, d, err_flag);
}

}  // namespace rrsdev
