// Field accumulation (Eqs. 7-10): for every receiver, E = E0 + sum_m Gamma_m c_m sum_q b_mq with the
// Rx-leg term of element m on path q
//   b_mq = sqrt(F(theta_out)) R_q sqrt(Gr Fr(theta_r)) e^{-j k L} / L        (Eq. 7 F_out, Eq. 8)
// evaluated in the RIS frame from the unfolded receiver image I_q: w = I_q - c, L = |w - u_m|,
// cos(theta_out) = (w - u_m).n / L, per-bounce cos(theta_i) = |(w - u_m).n'_j| / L, and the phase
// 2 pi frac(frac(D0/lambda) + dL/lambda) with D0 = |w| from FP64 and dL = (|u|^2 - 2 u.w)/(L + D0).
#include "rxleg.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// The same term as a plain FP32 program: unfolded length L = |w - u_m| from the RIS-frame image,
// absolute phase 2 pi L / lambda reduced by sincosf itself, IEEE square roots and divisions, Fresnel in
// its general complex form.
template <int PAT>
__device__ __forceinline__ cf rx_leg_term_plain(const PathRec& p, float4 e, float k0, float gr, bool tm)
{
    const float dx = p.w.x - e.x, dy = p.w.y - e.y, dz = p.w.z;
    const float L = sqrtf(dx * dx + dy * dy + dz * dz);
    const float cos_out = dz / L;
    float amp = sqrtf(fmaxf(cos_out, 0.f)) / L;
    if (PAT != RISRT_PATTERN_ISO) {
        float cr = -(dx * p.v.x + dy * p.v.y + dz * p.v.z) / L;
        amp *= sqrtf(gr * pattern_f(PAT, gr, cr));
    } else {
        amp *= sqrtf(gr);
    }
    cf R = cf{amp, 0.f};
    const int kk = __float_as_int(p.a.y);
    const int k = kk & 3;
    if (k >= 1) {          // a lossless-TE record holds eps_r - 1 in place of eps_r and no imaginary part
        const bool lt = (kk & kRecLosslessTE) != 0;
        const float er1 = lt ? p.a.z + 1.f : p.a.z, ei1 = lt ? 0.f : p.a.w;
        R = cmulf(R, fresnel_f(fabsf(dx * p.n1.x + dy * p.n1.y + dz * p.n1.z) / L, er1, ei1, tm));
        if (k == 2) {
            const float er2 = lt ? p.n1.w + 1.f : p.n1.w, ei2 = lt ? 0.f : p.n2.w;
            R = cmulf(R, fresnel_f(fabsf(dx * p.n2.x + dy * p.n2.y + dz * p.n2.z) / L, er2, ei2, tm));
        }
    }
    float sn, cs;
    sincosf(k0 * L, &sn, &cs);
    return cmulf(R, cf{cs, -sn});
}

constexpr int kEvalWarps = 8;
#ifndef RISRT_EVAL_EPL
#define RISRT_EVAL_EPL 2
#endif
// elements per lane per pass of the element-major kernel (measured on the room: 3 and 4 take 6% and 2%
// longer than 2)
constexpr int kEvalEpl = RISRT_EVAL_EPL;
constexpr int kMaxCfgPerPass = 4;
constexpr int kElemMajorMin = 64;   // arrays of at least this many elements: lanes own elements

// b_mq of one record for the lane's two elements (those with `on` set), added to their sums.
template <int PAT, int K, bool LT>
__device__ __forceinline__ void add_terms(const PathRec& p, const float4 (&e)[kEvalEpl], const bool (&on)[kEvalEpl],
                                          cf (&sum)[kEvalEpl], float inv_lam, float gr, bool tm)
{
#pragma unroll
    for (int h = 0; h < kEvalEpl; ++h) {
        if (!on[h]) continue;
        const cf b = rx_leg_term_k<PAT, K, LT>(p, e[h], inv_lam, gr, tm);
        sum[h].re += b.re;
        sum[h].im += b.im;
    }
}

// One warp per receiver, lanes own elements, kEvalEpl per pass (m = m0 + 32 h + lane): each
// lane keeps its elements' data in registers and sums b_mq over the receiver's paths, whose records
// every lane of the warp reads at the same address (one broadcast load per path serves kEvalEpl elements);
// then c_m and the NC configurations' Gamma_m scale the sums. For arrays of kElemMajorMin elements or
// more.
template <int PAT, int NC>
__global__ void __launch_bounds__(32 * kEvalWarps)
k_eval_em(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W,
          const float4* __restrict__ elem, const float2* __restrict__ cm, const float2* __restrict__ gamma,
          int M, int64_t n_rx, int cfg0, int n_cfg, const float2* __restrict__ E0, float2* __restrict__ E,
          float* __restrict__ P, float inv_lam, float gr, int tm, float inv_2eta0)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)kEvalWarps + (threadIdx.x >> 5);
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int nq = (int)(off[r + 1] - o);
    cf acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = cf{0.f, 0.f};
    for (int m0 = 0; m0 < M; m0 += 32 * kEvalEpl) {
        int mm[kEvalEpl];
        bool valid[kEvalEpl], direct[kEvalEpl];
        float4 e[kEvalEpl];
        cf sum[kEvalEpl];
#pragma unroll
        for (int h = 0; h < kEvalEpl; ++h) {
            mm[h] = m0 + 32 * h + lane;
            valid[h] = mm[h] < M;
            e[h] = valid[h] ? elem[mm[h]] : make_float4(0.f, 0.f, 0.f, 0.f);
            direct[h] = valid[h] && ((vis[r * W + (mm[h] >> 5)] >> (mm[h] & 31)) & 1u);
            sum[h] = cf{0.f, 0.f};
        }
        for (int q = 0; q < nq; ++q) {
            const PathRec p = rec[o + q];
            // one branch per record (uniform across the warp) into straight-line code for both elements
            const int kk = __float_as_int(p.a.y), k = kk & 3;
            if (kk & kRecLosslessTE) {
                if (k == 2) add_terms<PAT, 2, true>(p, e, valid, sum, inv_lam, gr, tm != 0);
                else add_terms<PAT, 1, true>(p, e, valid, sum, inv_lam, gr, tm != 0);
            } else if (k == 0) {
                add_terms<PAT, 0, false>(p, e, direct, sum, inv_lam, gr, tm != 0);   // the direct leg
            } else if (k == 1) {
                add_terms<PAT, 1, false>(p, e, valid, sum, inv_lam, gr, tm != 0);
            } else {
                add_terms<PAT, 2, false>(p, e, valid, sum, inv_lam, gr, tm != 0);
            }
        }
#pragma unroll
        for (int h = 0; h < kEvalEpl; ++h) {
            if (!valid[h]) continue;
            const float2 c2 = cm[mm[h]];
            const cf cb = cmulf(sum[h], cf{c2.x, c2.y});
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (c < n_cfg) {
                    const float2 g = gamma[(int64_t)(cfg0 + c) * M + mm[h]];
                    acc[c].re += g.x * cb.re - g.y * cb.im;
                    acc[c].im += g.x * cb.im + g.y * cb.re;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            acc[c].re += __shfl_down_sync(0xffffffffu, acc[c].re, s);
            acc[c].im += __shfl_down_sync(0xffffffffu, acc[c].im, s);
        }
    }
    if (lane == 0) {
        const float2 e0 = E0[r];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (c < n_cfg) {
                float er = e0.x + acc[c].re, ei = e0.y + acc[c].im;
                int64_t oi = (int64_t)(cfg0 + c) * n_rx + r;
                E[oi] = make_float2(er, ei);
                if (P) P[oi] = (er * er + ei * ei) * inv_2eta0;
            }
        }
    }
}

// One warp per receiver; lanes walk the flattened (path, element) index space so small arrays keep
// every lane busy. NC configurations share each b_mq. Configuration c's Gamma_m is gamma[c gstride + m];
// with accum the RIS sum is added to E (E0 and P untouched).
template <int PAT, int NC>
__global__ void __launch_bounds__(32 * kEvalWarps)
k_eval(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W,
       const float4* __restrict__ elem, const float2* __restrict__ cm, const float2* __restrict__ gamma,
       int M, int64_t n_rx, int cfg0, int n_cfg, const float2* __restrict__ E0, float2* __restrict__ E,
       float* __restrict__ P, float inv_lam, float gr, int tm, float inv_2eta0, int gstride, bool accum)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)kEvalWarps + (threadIdx.x >> 5);
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int64_t total = (off[r + 1] - o) * (int64_t)M;
    cf acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = cf{0.f, 0.f};
    int q = lane / M, m = lane % M;
    for (int64_t idx = lane; idx < total; idx += 32) {
        const PathRec p = rec[o + q];
        const int k = __float_as_int(p.a.y);
        bool on = k > 0 || ((vis[r * W + (m >> 5)] >> (m & 31)) & 1u);
        if (on) {
            const float4 e = elem[m];
            const cf b = rx_leg_term<PAT>(p, e, inv_lam, gr, tm != 0);
            const float2 c2 = cm[m];
            const cf cb = cmulf(b, cf{c2.x, c2.y});
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (c < n_cfg) {
                    const float2 g = gamma[(int64_t)(cfg0 + c) * gstride + m];
                    acc[c].re += g.x * cb.re - g.y * cb.im;
                    acc[c].im += g.x * cb.im + g.y * cb.re;
                }
            }
        }
        m += 32;
        while (m >= M) {
            m -= M;
            ++q;
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            acc[c].re += __shfl_down_sync(0xffffffffu, acc[c].re, s);
            acc[c].im += __shfl_down_sync(0xffffffffu, acc[c].im, s);
        }
    }
    if (lane == 0) {
        const float2 e0 = accum ? make_float2(0.f, 0.f) : E0[r];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (c < n_cfg) {
                const int64_t oi = (int64_t)(cfg0 + c) * n_rx + r;
                if (accum) {
                    const float2 prev = E[oi];
                    E[oi] = make_float2(prev.x + acc[c].re, prev.y + acc[c].im);
                    continue;
                }
                float er = e0.x + acc[c].re, ei = e0.y + acc[c].im;
                E[oi] = make_float2(er, ei);
                if (P) P[oi] = (er * er + ei * ei) * inv_2eta0;
            }
        }
    }
}

// Plain FP32 baseline: one thread per receiver, every (element, path) term in turn.
template <int PAT, int NC>
__global__ void __launch_bounds__(128)
k_eval_plain(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W,
             const float4* __restrict__ elem, const float2* __restrict__ cm, const float2* __restrict__ gamma,
             int M, int64_t n_rx, int cfg0, int n_cfg, const float2* __restrict__ E0, float2* __restrict__ E,
             float* __restrict__ P, float k0, float gr, int tm, float inv_2eta0)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int nq = (int)(off[r + 1] - o);
    cf acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = cf{0.f, 0.f};
    for (int m = 0; m < M; ++m) {
        const float4 e = elem[m];
        const bool direct = (vis[r * W + (m >> 5)] >> (m & 31)) & 1u;
        cf sum = cf{0.f, 0.f};
        for (int q = 0; q < nq; ++q) {
            const PathRec p = rec[o + q];
            if (__float_as_int(p.a.y) == 0 && !direct) continue;
            const cf b = rx_leg_term_plain<PAT>(p, e, k0, gr, tm != 0);
            sum.re += b.re;
            sum.im += b.im;
        }
        const float2 c2 = cm[m];
        const cf cb = cmulf(sum, cf{c2.x, c2.y});
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (c < n_cfg) {
                const float2 g = gamma[(int64_t)(cfg0 + c) * M + m];
                acc[c].re += g.x * cb.re - g.y * cb.im;
                acc[c].im += g.x * cb.im + g.y * cb.re;
            }
        }
    }
    const float2 e0 = E0[r];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c < n_cfg) {
            float er = e0.x + acc[c].re, ei = e0.y + acc[c].im;
            int64_t oi = (int64_t)(cfg0 + c) * n_rx + r;
            E[oi] = make_float2(er, ei);
            if (P) P[oi] = (er * er + ei * ei) * inv_2eta0;
        }
    }
}

// Channel impulse response of the RIS part: one warp per receiver, lanes own elements; for every Rx-leg
// entry q and Tx-leg path p the tap sum_m g[m][p] b_mq (g = Gamma_m K c_mp), written at (entry, p),
// and the entry's delay from the RIS centre D0 / c0.
template <int PAT>
__global__ void __launch_bounds__(32 * kEvalWarps)
k_cir(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W,
      const float4* __restrict__ elem, const float2* __restrict__ g, int M, int P, int64_t n_rx,
      float2* __restrict__ taps, double* __restrict__ rx_delay, float inv_lam, float gr, int tm)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)kEvalWarps + (threadIdx.x >> 5);
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int nq = (int)(off[r + 1] - o);
    for (int q = 0; q < nq; ++q) {
        const PathRec pr = rec[o + q];
        const bool reflected = __float_as_int(pr.a.y) > 0;
        if (lane == 0) rx_delay[o + q] = (double)pr.w.w / kC0;
        for (int p = 0; p < P; ++p) {
            cf acc = cf{0.f, 0.f};
            for (int m0 = 0; m0 < M; m0 += 32) {
                const int m = m0 + lane;
                if (m >= M) break;
                if (!reflected && !((vis[r * W + (m >> 5)] >> (m & 31)) & 1u)) continue;
                const cf b = rx_leg_term<PAT>(pr, elem[m], inv_lam, gr, tm != 0);
                const float2 gg = g[(int64_t)m * P + p];
                const cf v = cmulf(b, cf{gg.x, gg.y});
                acc.re += v.re;
                acc.im += v.im;
            }
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                acc.re += __shfl_down_sync(0xffffffffu, acc.re, s);
                acc.im += __shfl_down_sync(0xffffffffu, acc.im, s);
            }
            if (lane == 0) taps[(o + q) * P + p] = make_float2(acc.re, acc.im);
        }
    }
}

// A[r][m] = c_m sum_q b_mq: one warp per receiver, lanes own elements, paths broadcast.
template <int PAT>
__global__ void __launch_bounds__(32 * kEvalWarps)
k_build_A(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W,
          const float4* __restrict__ elem, const float2* __restrict__ cm, int M, int64_t n_rx,
          float2* __restrict__ A, float inv_lam, float gr, int tm)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)kEvalWarps + (threadIdx.x >> 5);
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int nq = (int)(off[r + 1] - o);
    for (int m0 = 0; m0 < M; m0 += 32) {
        const int m = m0 + lane;
        const bool valid = m < M;
        const float4 e = valid ? elem[m] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool direct = valid && ((vis[r * W + (m >> 5)] >> (m & 31)) & 1u);
        cf acc = cf{0.f, 0.f};
        for (int q = 0; q < nq; ++q) {
            const PathRec p = rec[o + q];
            if (!valid || (q == 0 && !direct)) continue;   // entry 0 is the direct path
            const cf b = rx_leg_term<PAT>(p, e, inv_lam, gr, tm != 0);
            acc.re += b.re;
            acc.im += b.im;
        }
        if (valid) {
            const float2 c2 = cm[m];
            const cf a = cmulf(acc, cf{c2.x, c2.y});
            A[r * (int64_t)M + m] = make_float2(a.re, a.im);
        }
    }
}

}  // namespace

int eval_field(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, int n_cfg, float2* E, float* P)
{
    const float inv_lam = (float)(ps->freq / kC0);
    const float inv_2eta0 = (float)(1.0 / (2.0 * kEta0));
    const int tm = (ps->flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
    const unsigned grid = nblk(ps->n_rx, kEvalWarps);
    for (int c0 = 0; c0 < n_cfg; c0 += kMaxCfgPerPass) {
        const int nc = std::min(kMaxCfgPerPass, n_cfg - c0);
#define RISRT_EVAL(PAT, NCV)                                                                                  \
    do {                                                                                                      \
        if (ps->M >= kElemMajorMin)                                                                           \
            RISRT_KERNEL(ctx, "k_eval", (k_eval_em<PAT, NCV><<<grid, 32 * kEvalWarps, 0, ctx->stream>>>(       \
                                            ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, ps->cm, gamma, ps->M, \
                                            ps->n_rx, c0, nc, ps->E0, E, P, inv_lam, ps->rx_gain, tm, inv_2eta0))); \
        else                                                                                                  \
            RISRT_KERNEL(ctx, "k_eval", (k_eval<PAT, NCV><<<grid, 32 * kEvalWarps, 0, ctx->stream>>>(          \
                                            ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, ps->cm, gamma, ps->M, \
                                            ps->n_rx, c0, nc, ps->E0, E, P, inv_lam, ps->rx_gain, tm, inv_2eta0, \
                                            ps->M, false)));                                                  \
    } while (0)
#define RISRT_EVAL_NC(PAT)           \
    do {                             \
        if (nc == 1) RISRT_EVAL(PAT, 1); \
        else if (nc == 2) RISRT_EVAL(PAT, 2); \
        else RISRT_EVAL(PAT, 4);     \
    } while (0)
        switch (ps->rx_pattern) {
            case RISRT_PATTERN_COS_POW: RISRT_EVAL_NC(RISRT_PATTERN_COS_POW); break;
            case RISRT_PATTERN_MONOPOLE_QW: RISRT_EVAL_NC(RISRT_PATTERN_MONOPOLE_QW); break;
            default: RISRT_EVAL_NC(RISRT_PATTERN_ISO); break;
        }
#undef RISRT_EVAL_NC
#undef RISRT_EVAL
    }
    return RISRT_OK;
}

int eval_field_accum(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, int gstride, int n_cfg, float2* E)
{
    const float inv_lam = (float)(ps->freq / kC0);
    const int tm = (ps->flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
    const unsigned grid = nblk(ps->n_rx, kEvalWarps);
    for (int c0 = 0; c0 < n_cfg; c0 += kMaxCfgPerPass) {
        const int nc = std::min(kMaxCfgPerPass, n_cfg - c0);
        auto launch = [&](auto kern) -> int {
            RISRT_KERNEL(ctx, "k_eval", (kern<<<grid, 32 * kEvalWarps, 0, ctx->stream>>>(
                                            ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, ps->cm, gamma, ps->M, ps->n_rx,
                                            c0, nc, ps->E0, E, nullptr, inv_lam, ps->rx_gain, tm, 0.f, gstride, true)));
            return RISRT_OK;
        };
        int rc;
#define RISRT_ACC_NC(PAT) (nc == 1 ? launch(k_eval<PAT, 1>) : nc == 2 ? launch(k_eval<PAT, 2>) : launch(k_eval<PAT, 4>))
        switch (ps->rx_pattern) {
            case RISRT_PATTERN_COS_POW: rc = RISRT_ACC_NC(RISRT_PATTERN_COS_POW); break;
            case RISRT_PATTERN_MONOPOLE_QW: rc = RISRT_ACC_NC(RISRT_PATTERN_MONOPOLE_QW); break;
            default: rc = RISRT_ACC_NC(RISRT_PATTERN_ISO); break;
        }
#undef RISRT_ACC_NC
        if (rc) return rc;
    }
    return RISRT_OK;
}

int eval_field_plain(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, int n_cfg, float2* E, float* P)
{
    const float k0 = (float)(2.0 * kPi * ps->freq / kC0);
    const float inv_2eta0 = (float)(1.0 / (2.0 * kEta0));
    const int tm = (ps->flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
    const unsigned grid = nblk(ps->n_rx, 128);
    for (int c0 = 0; c0 < n_cfg; c0 += kMaxCfgPerPass) {
        const int nc = std::min(kMaxCfgPerPass, n_cfg - c0);
#define RISRT_PLAIN(PAT, NCV)                                                                                 \
    RISRT_KERNEL(ctx, "k_eval_plain", (k_eval_plain<PAT, NCV><<<grid, 128, 0, ctx->stream>>>(                   \
                                         ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, ps->cm, gamma, ps->M,   \
                                         ps->n_rx, c0, nc, ps->E0, E, P, k0, ps->rx_gain, tm, inv_2eta0)))
#define RISRT_PLAIN_NC(PAT)                  \
    do {                                     \
        if (nc == 1) RISRT_PLAIN(PAT, 1);    \
        else if (nc == 2) RISRT_PLAIN(PAT, 2); \
        else RISRT_PLAIN(PAT, 4);            \
    } while (0)
        switch (ps->rx_pattern) {
            case RISRT_PATTERN_COS_POW: RISRT_PLAIN_NC(RISRT_PATTERN_COS_POW); break;
            case RISRT_PATTERN_MONOPOLE_QW: RISRT_PLAIN_NC(RISRT_PATTERN_MONOPOLE_QW); break;
            default: RISRT_PLAIN_NC(RISRT_PATTERN_ISO); break;
        }
#undef RISRT_PLAIN_NC
#undef RISRT_PLAIN
    }
    return RISRT_OK;
}

int eval_cir(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, float2* taps, double* rx_delay, double* tx_delay)
{
    const int P = (int)ps->tx_seq_host.size() + 1;
    void* g = nullptr;
    RISRT_CUDA(ctx, ctx_malloc(ctx, &g, sizeof(float2) * (size_t)ps->M * P));
    int rc = cir_tx_coef(ctx, ps, gamma, (float2*)g, tx_delay);
    if (!rc) {
        const float inv_lam = (float)(ps->freq / kC0);
        const int tm = (ps->flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
        const unsigned grid = nblk(ps->n_rx, kEvalWarps);
        auto launch = [&](auto kern) -> int {
            RISRT_KERNEL(ctx, "k_cir", (kern<<<grid, 32 * kEvalWarps, 0, ctx->stream>>>(
                                           ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, (const float2*)g, ps->M, P,
                                           ps->n_rx, taps, rx_delay, inv_lam, ps->rx_gain, tm)));
            return RISRT_OK;
        };
        switch (ps->rx_pattern) {
            case RISRT_PATTERN_COS_POW: rc = launch(k_cir<RISRT_PATTERN_COS_POW>); break;
            case RISRT_PATTERN_MONOPOLE_QW: rc = launch(k_cir<RISRT_PATTERN_MONOPOLE_QW>); break;
            default: rc = launch(k_cir<RISRT_PATTERN_ISO>); break;
        }
    }
    ctx_free(ctx, g);    // later users of the block are ordered after this work on the context's stream
    return rc;
}

int build_A(risrt_ctx* ctx, const risrt_pathset* ps, float2* A, float2* E0)
{
    const float inv_lam = (float)(ps->freq / kC0);
    const int tm = (ps->flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
    const unsigned grid = nblk(ps->n_rx, kEvalWarps);
#define RISRT_BUILD_A(PAT)                                                                                  \
    RISRT_KERNEL(ctx, "k_build_A", (k_build_A<PAT><<<grid, 32 * kEvalWarps, 0, ctx->stream>>>(                       \
                                       ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, ps->cm, ps->M, ps->n_rx, A,   \
                                       inv_lam, ps->rx_gain, tm)))
    switch (ps->rx_pattern) {
        case RISRT_PATTERN_COS_POW: RISRT_BUILD_A(RISRT_PATTERN_COS_POW); break;
        case RISRT_PATTERN_MONOPOLE_QW: RISRT_BUILD_A(RISRT_PATTERN_MONOPOLE_QW); break;
        default: RISRT_BUILD_A(RISRT_PATTERN_ISO); break;
    }
#undef RISRT_BUILD_A
    if (E0) RISRT_CUDA(ctx, cudaMemcpyAsync(E0, ps->E0, sizeof(float2) * ps->n_rx, cudaMemcpyDeviceToDevice, ctx->stream));
    return RISRT_OK;
}

}  // namespace risrt
