// FP32 complex arithmetic, Fresnel reflection coefficient and antenna patterns shared by the
// field kernels (Eqs. 5-8): the per-element, per-path terms whose amplitudes need FP32 only.
#pragma once

#include "internal.cuh"

namespace risrt {

struct cf { float re, im; };
__device__ __forceinline__ cf cmulf(cf a, cf b) { return cf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Single special-function-unit instructions (PTX .approx forms: square root to about 1 ulp,
// reciprocal to 1 ulp; denormal inputs flush to zero), for the per-element terms whose FP32
// tolerance is far above a few ulp. sqrt_approx(0) = 0.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Fresnel coefficient of a lossless dielectric (real eps_r >= sin^2, TE or TM) with one square root
// and one reciprocal: R_TE = (c - s) / (c + s), R_TM = (eps c - s) / (eps c + s), s = sqrt(eps - sin^2).
__device__ __forceinline__ float fresnel_real_fast(float c, float er, bool tm)
{
    const float s = sqrt_approx(fmaxf(er - fmaxf(1.f - c * c, 0.f), 0.f));
    const float a = tm ? er * c : c;
    return (a - s) * rcp_approx(a + s);
}

// principal complex square root in FP32
__device__ __forceinline__ cf csqrtf_(float x, float y)
{
    float r = hypotf(x, y);
    if (r == 0.f) return cf{0.f, 0.f};
    if (x >= 0.f) {
        float s = sqrtf(0.5f * (r + x));
        return cf{s, y / (2.f * s)};
    }
    float s = copysignf(sqrtf(0.5f * (r - x)), y);
    return cf{y / (2.f * s), s};
}

// Fresnel coefficient at incidence cos_i for permittivity (er, ei); TE or TM (Collin).
__device__ __forceinline__ cf fresnel_f(float c, float er, float ei, bool tm)
{
    float s2 = fmaxf(1.f - c * c, 0.f);
    if (!tm && ei == 0.f && er >= s2) {      // lossless dielectric: real coefficient
        float root = sqrtf(er - s2);
        return cf{(c - root) / (c + root), 0.f};
    }
    cf root = csqrtf_(er - s2, ei);
    cf a, b;
    if (!tm) {
        a = cf{c - root.re, -root.im};
        b = cf{c + root.re, root.im};
    } else {
        a = cf{er * c - root.re, ei * c - root.im};
        b = cf{er * c + root.re, ei * c + root.im};
    }
    float inv = 1.f / (b.re * b.re + b.im * b.im);
    return cf{(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}

// Antenna pattern F(cos theta) (Sec. III-B) with the pattern chosen at run time: isotropic,
// cos^(G/2-1) in front of the antenna, quarter-wave monopole cos(pi/2 cos theta)^2 / sin^2 theta.
__device__ __forceinline__ float pattern_f(int pat, float gain, float c)
{
    if (pat == RISRT_PATTERN_COS_POW) return c > 0.f ? powf(c, 0.5f * gain - 1.f) : 0.f;
    if (pat == RISRT_PATTERN_MONOPOLE_QW) {
        float s2 = 1.f - c * c;
        if (s2 <= 0.f) return 0.f;
        float v = cospif(0.5f * c) * rsqrtf(s2);
        return v * v;
    }
    return 1.f;
}

}  // namespace risrt
