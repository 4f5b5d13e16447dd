// noise.cuh -- the channel noise of the sampling kernels: Philox4x32-10
// (Salmon et al., SC'11) keyed by the job with counter (quad, sample low,
// sample high, 0); four uniforms u = (2 (x >> 9) + 1) 2^-24 per call; two
// single-precision Box-Muller pairs (Box and Muller 1958) computed with
// IEEE-rounded operations only: log by frexp and the atanh series of log,
// sin/cos of 2 pi u by quadrant reduction and their Taylor series on
// [0, pi/4].  Included by each sampling translation unit (after
// decode_impl.cuh, whose rounded-operation helpers it uses).
#pragma once
#include "decode_impl.cuh"

namespace tsx {
namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

__device__ __forceinline__ float uniform24(uint32_t x) { return hmul((float)(2u * (x >> 9) + 1u), 0x1p-24f); }

__device__ __forceinline__ float series_logf(float u) {
    int e;
    float m = frexpf(u, &e);
    if (m < 0x1.6a09e6p-1f) {
        m = hadd(m, m);
        e = e - 1;
    }
    const float s = hdiv(hsub(m, 1.0f), hadd(m, 1.0f));
    const float s2 = hmul(s, s);
    float q = 0x1.3b13b2p-4f;  // 1/13
    q = hadd(hmul(q, s2), 0x1.745d18p-4f);
    q = hadd(hmul(q, s2), 0x1.c71c72p-4f);
    q = hadd(hmul(q, s2), 0x1.24924ap-3f);
    q = hadd(hmul(q, s2), 0x1.99999ap-3f);
    q = hadd(hmul(q, s2), 0x1.555556p-2f);
    q = hadd(hmul(q, s2), 1.0f);
    return hadd(hmul((float)e, 0x1.62e43p-1f), hmul(hadd(s, s), q));
}

__device__ __forceinline__ float sin_poly(float a) {
    const float a2 = hmul(a, a);
    float p = 0x1.71de3ap-19f;                  // 1/9!
    p = hsub(hmul(p, a2), 0x1.a01a02p-13f);     // 1/7!
    p = hadd(hmul(p, a2), 0x1.111112p-7f);      // 1/5!
    p = hsub(hmul(p, a2), 0x1.555556p-3f);      // 1/3!
    p = hadd(hmul(p, a2), 1.0f);
    return hmul(p, a);
}
__device__ __forceinline__ float cos_poly(float a) {
    const float a2 = hmul(a, a);
    float p = -0x1.27e4fcp-22f;                 // -1/10!
    p = hadd(hmul(p, a2), 0x1.a01a02p-16f);     // 1/8!
    p = hsub(hmul(p, a2), 0x1.6c16c2p-10f);     // 1/6!
    p = hadd(hmul(p, a2), 0x1.555556p-5f);      // 1/4!
    p = hsub(hmul(p, a2), 0.5f);
    p = hadd(hmul(p, a2), 1.0f);
    return p;
}
__device__ __forceinline__ void sincos2pi(float t, float &s, float &c) {
    const float t4 = hmul(t, 4.0f);
    const float kf = floorf(t4);
    const int k = (int)kf;
    const float f = hsub(t4, kf);
    const float HALF_PI = 0x1.921fb6p+0f;
    float sa, ca;
    if (f <= 0.5f) {
        const float a = hmul(f, HALF_PI);
        sa = sin_poly(a);
        ca = cos_poly(a);
    } else {
        const float a = hmul(hsub(1.0f, f), HALF_PI);
        sa = cos_poly(a);
        ca = sin_poly(a);
    }
    switch (k & 3) {
        case 0: s = sa; c = ca; break;
        case 1: s = ca; c = -sa; break;
        case 2: s = -sa; c = -ca; break;
        default: s = -ca; c = sa; break;
    }
}

__device__ __forceinline__ void normals4(unsigned long long job, unsigned long long s, uint32_t q, float g[4]) {
    uint32_t c0 = q, c1 = (uint32_t)s, c2 = (uint32_t)(s >> 32), c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)job, (uint32_t)(job >> 32));
    const uint32_t x[4] = {c0, c1, c2, c3};
#pragma unroll
    for (int pr = 0; pr < 2; pr++) {
        const float ua = uniform24(x[2 * pr]), ub = uniform24(x[2 * pr + 1]);
        const float r = __fsqrt_rn(hmul(-2.0f, series_logf(ua)));
        float sn, cs;
        sincos2pi(ub, sn, cs);
        g[2 * pr] = hmul(r, cs);
        g[2 * pr + 1] = hmul(r, sn);
    }
}

}  // namespace
}  // namespace tsx
