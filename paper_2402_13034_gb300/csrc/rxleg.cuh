// The Rx-leg term b_mq of one (path record, element) pair (Eq. 7's F_out, Eq. 8, Fresnel per bounce) as
// the field kernels evaluate it, shared by the field evaluation, the channel matrix and the fused
// sweep: from the RIS-frame receiver image w = I_q - c of the record, L = |w - u_m|,
// cos(theta_out) = (w - u_m).n / L, per-bounce cos(theta_i) = |(w - u_m).n'_j| / L, and the phase
// 2 pi frac(frac(D0/lambda) + dL/lambda) with D0 = |w| from FP64 and dL = (|u|^2 - 2 u.w)/(L + D0).
#pragma once

#include "cplx32.cuh"

namespace risrt {

template <int PAT>
__device__ __forceinline__ float rx_pattern(float c, float gain)
{
    if (PAT == RISRT_PATTERN_COS_POW) return c > 0.f ? __powf(c, 0.5f * gain - 1.f) : 0.f;
    if (PAT == RISRT_PATTERN_MONOPOLE_QW) {
        float s2 = 1.f - c * c;
        if (s2 <= 0.f) return 0.f;
        float v = cospif(0.5f * c) * rsqrtf(s2);
        return v * v;
    }
    return 1.f;
}

// Fresnel factor of one bounce at incidence cosine c: one square root and one reciprocal for a
// lossless dielectric, the complex form otherwise.
__device__ __forceinline__ cf bounce_factor(float c, float er, float ei, bool tm)
{
    if (ei == 0.f && er >= 1.f) return cf{fresnel_real_fast(c, er, tm), 0.f};
    return fresnel_f(c, er, ei, tm);
}

// b_mq for one (path record, element) pair, with the record's bounce count K and its lossless-TE flag
// LT fixed at compile time (straight-line code). Paths whose bounces are all lossless dielectrics
// under the TE coefficient (kRecLosslessTE) keep R real: per bounce c = |(w - u).n'| / L,
// s = sqrt(eps_r - 1 + c^2), R *= (c - s)^2 / (1 - eps_r), which equals (c - s) / (c + s) since
// c^2 - s^2 = 1 - eps_r.
template <int PAT, int K, bool LT>
__device__ __forceinline__ cf rx_leg_term_k(const PathRec& p, float4 e, float inv_lam, float gr, bool tm)
{
    const float dx = p.w.x - e.x, dy = p.w.y - e.y, dz = p.w.z;
    const float L2 = dx * dx + dy * dy + dz * dz;
    const float iL = rsqrtf(L2);
    const float L = L2 * iL;
    const float cos_out = dz * iL;
    float amp = sqrt_approx(fmaxf(cos_out, 0.f)) * iL;
    if (PAT != RISRT_PATTERN_ISO) {
        float cr = -(dx * p.v.x + dy * p.v.y + dz * p.v.z) * iL;
        amp *= sqrt_approx(gr * rx_pattern<PAT>(cr, gr));
    } else {
        amp *= sqrt_approx(gr);
    }
    cf R = cf{amp, 0.f};
    if (LT) {
        const float c1 = fabsf(dx * p.n1.x + dy * p.n1.y + dz * p.n1.z) * iL;
        const float d1 = c1 - sqrt_approx(fmaxf(fmaf(c1, c1, p.a.z), 0.f));
        R.re *= d1 * d1 * p.a.w;
        if (K == 2) {
            const float c2 = fabsf(dx * p.n2.x + dy * p.n2.y + dz * p.n2.z) * iL;
            const float d2 = c2 - sqrt_approx(fmaxf(fmaf(c2, c2, p.n1.w), 0.f));
            R.re *= d2 * d2 * p.n2.w;
        }
    } else if (K >= 1) {
        float c1 = fabsf(dx * p.n1.x + dy * p.n1.y + dz * p.n1.z) * iL;
        R = cmulf(R, bounce_factor(c1, p.a.z, p.a.w, tm));
        if (K == 2) {
            float c2 = fabsf(dx * p.n2.x + dy * p.n2.y + dz * p.n2.z) * iL;
            R = cmulf(R, bounce_factor(c2, p.n1.w, p.n2.w, tm));
        }
    }
    const float dL = (e.z - 2.f * (e.x * p.w.x + e.y * p.w.y)) * rcp_approx(L + p.w.w);
    float x = p.a.x + dL * inv_lam;
    x -= rintf(x);
    float sn, cs;
    __sincosf(6.28318530717958647f * x, &sn, &cs);
    if (LT || K == 0) return cf{R.re * cs, -R.re * sn};   // e^{-j 2 pi x}, R real
    return cmulf(R, cf{cs, -sn});
}

// b_mq for one (path record, element) pair: the specialised term for the record's bounce count and
// lossless-TE flag (the branch is uniform across a warp whose lanes share the record).
template <int PAT>
__device__ __forceinline__ cf rx_leg_term(const PathRec& p, float4 e, float inv_lam, float gr, bool tm)
{
    const int kk = __float_as_int(p.a.y);
    const int k = kk & 3;
    if (kk & kRecLosslessTE)
        return k == 2 ? rx_leg_term_k<PAT, 2, true>(p, e, inv_lam, gr, tm) : rx_leg_term_k<PAT, 1, true>(p, e, inv_lam, gr, tm);
    if (k == 0) return rx_leg_term_k<PAT, 0, false>(p, e, inv_lam, gr, tm);
    return k == 1 ? rx_leg_term_k<PAT, 1, false>(p, e, inv_lam, gr, tm) : rx_leg_term_k<PAT, 2, false>(p, e, inv_lam, gr, tm);
}

}  // namespace risrt
