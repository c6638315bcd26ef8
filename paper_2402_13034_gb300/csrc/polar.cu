// Vector field with polarisation: the extension of Eq. 6 that Sec. II-A names without giving a model.
// Every path keeps the scalar model's factors (Eqs. 4-8) except the Fresnel products and carries a
// field vector instead:
//   launch      e = unit(P(d0) a_t), P(k) = I - k k^T, a_t the Tx polarisation axis, d0 the departure
//   bounce      e <- R_TE (e.s) s + R_TM (e.p_in) p_out, s = unit(k_in x n), p = s x k (TE and TM)
//   RIS         e <- P(k_out) (e - 2 (e.n) n)   (normal component reversed, outgoing wavefront)
//   reception   received = unit(P(k_arr) a_r) . e;  E3 = sum of the terms' e (amplitudes included)
// so that E = E0 + sum_m Gamma_m (received values) and E3 = E03 + sum_m Gamma_m (field vectors).
//
// Factorisation: the Tx leg and the RIS transform do not depend on the receiver, so each element's
// incident field, summed over its Tx-leg paths, becomes one complex vector c_m (RIS frame, normal
// component reversed, K included). The Rx leg of (receiver, element m, path q) is evaluated on the
// unfolded straight line d from e_m to the receiver image I_q, in the RIS frame of the path record:
// unfolding turns every bounce into D = R_TE s s^T - R_TM p p^T with s = unit(d x n'), p = s x d and
// n' the record's (unfolded) bounce normal, and the Rx axis into a' = H_n2' H_n1 a_r (the mirrors the
// record's pattern axis also took), so that
//   received = b_mq (D1 D2 unit(P(d) a')) . c_m,   field vector = b_mq H_n1 H_n2' D2 D1 P(d) c_m
// with b_mq the scalar Rx-leg term without its Fresnel product.
#include "cplx32.cuh"
#include "frame.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

constexpr int kVecWarps = 8;
constexpr int kVecCfg = 4;          // configurations per pass of the field kernel

// complex 3-vectors
struct cv3 { cf x, y, z; };

__device__ __forceinline__ cf cadd(cf a, cf b) { return cf{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf cscl(cf a, float s) { return cf{a.re * s, a.im * s}; }
__device__ __forceinline__ cv3 cv_of(float3 a) { return cv3{cf{a.x, 0.f}, cf{a.y, 0.f}, cf{a.z, 0.f}}; }
__device__ __forceinline__ cv3 cv_mul(cv3 a, cf s) { return cv3{cmulf(a.x, s), cmulf(a.y, s), cmulf(a.z, s)}; }
__device__ __forceinline__ cv3 cv_add(cv3 a, cv3 b) { return cv3{cadd(a.x, b.x), cadd(a.y, b.y), cadd(a.z, b.z)}; }
__device__ __forceinline__ cf cv_dot(cv3 a, float3 b)                  // bilinear, no conjugate
{
    return cf{a.x.re * b.x + a.y.re * b.y + a.z.re * b.z, a.x.im * b.x + a.y.im * b.y + a.z.im * b.z};
}
__device__ __forceinline__ cf cv_dotc(cv3 a, cv3 b)                    // bilinear complex . complex
{
    return cadd(cadd(cmulf(a.x, b.x), cmulf(a.y, b.y)), cmulf(a.z, b.z));
}
// a + s b (b real)
__device__ __forceinline__ cv3 cv_axpy(cv3 a, cf s, float3 b)
{
    return cv3{cf{a.x.re + s.re * b.x, a.x.im + s.im * b.x}, cf{a.y.re + s.re * b.y, a.y.im + s.im * b.y},
               cf{a.z.re + s.re * b.z, a.z.im + s.im * b.z}};
}
// mirror across the plane with unit normal n
__device__ __forceinline__ cv3 cv_mirror(cv3 a, float3 n) { return cv_axpy(a, cscl(cv_dot(a, n), -2.f), n); }

// unit(P(k) a): the field direction of an antenna with axis a for propagation direction k (zero when
// a lies along k)
__device__ __forceinline__ float3 pol_dir(float3 a, float3 k)
{
    const float3 p = a - k * dot(a, k);
    const float l2 = dot(p, p);
    return l2 > 1e-20f ? p * rsqrtf(l2) : f3(0.f, 0.f, 0.f);
}

// One bounce in real coordinates: incoming kin, outgoing kout, unit normal n, permittivity eps.
__device__ __forceinline__ cv3 bounce_real(cv3 e, float3 kin, float3 kout, float3 n, float2 eps)
{
    const float c = fabsf(dot(kin, n));
    const cf rte = fresnel_f(c, eps.x, eps.y, false), rtm = fresnel_f(c, eps.x, eps.y, true);
    float3 s = cross(kin, n);
    const float l2 = dot(s, s);
    if (l2 < 1e-20f) return cv_mul(e, rte);            // normal incidence: R_TM = -R_TE, p_out = -p_in
    s = s * rsqrtf(l2);
    const float3 pin = cross(s, kin), pout = cross(s, kout);
    cv3 r = cv_mul(cv_of(s), cmulf(rte, cv_dot(e, s)));
    return cv_axpy(r, cmulf(rtm, cv_dot(e, pin)), pout);
}

// One bounce on the unfolded line d (unit) of a field transverse to d: D = R_TE s s^T - R_TM p p^T.
__device__ __forceinline__ cv3 bounce_unfolded(cv3 e, float3 d, float3 n, cf rte, cf rtm)
{
    float3 s = cross(d, n);
    const float l2 = dot(s, s);
    if (l2 < 1e-20f) return cv_mul(e, rte);            // normal incidence: D = R_TE P(d)
    s = s * rsqrtf(l2);
    const float3 p = cross(s, d);
    cv3 r = cv_mul(cv_of(s), cmulf(rte, cv_dot(e, s)));
    return cv_axpy(r, cscl(cmulf(rtm, cv_dot(e, p)), -1.f), p);
}

// Tx leg of element m (one warp per element, lanes over its Tx-leg paths, LOS first): the incident
// field vector sum_p sqrt(2 eta0 Pt Gt Ft) sqrt(F_in) e^{-jkL} / L e_p (Eq. 4, Eq. 5, the Fresnel
// products inside e_p), then the RIS transform's normal reversal, K, and the RIS frame:
// cvec[m] = K (e.t1, e.t2, -e.n). FP64 for L and frac(L / lambda), FP32 otherwise.
__global__ void k_cm_vec(const float4* __restrict__ elem, int M, Frame fr, AntD tx, WaveD wv, double K, float3 a_t,
                         const uint8_t* __restrict__ tx_vis, const TxPathD* __restrict__ paths, int n_tx,
                         float2* __restrict__ cvec)
{
    const int lane = threadIdx.x & 31;
    const int m = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (m >= M) return;
    const d3 e = elem_pos(fr, elem[m]);
    const float3 z = f3((float)tx.z[0], (float)tx.z[1], (float)tx.z[2]);
    const float3 nr = f3((float)fr.n[0], (float)fr.n[1], (float)fr.n[2]);
    const float gt = (float)tx.gain;
    const float amp0 = (float)sqrt(2.0 * kEta0 * tx.power * tx.gain);
    cv3 acc = cv_of(f3(0.f, 0.f, 0.f));
    for (int p = lane - 1; p < n_tx; p += 32) {
        d3 Ts = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
        int k = 0;
        float3 nf[2] = {f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f)};
        float2 ef[2] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f)};
        if (p < 0) {
            if (!tx_vis[m]) continue;
        } else {
            const TxPathD t = paths[p];
            k = t.k;
            Ts = ld3(t.img);
            for (int j = 0; j < 2; ++j) {
                nf[j] = f3(t.n[j].x, t.n[j].y, t.n[j].z);
                ef[j] = t.eps[j];
            }
        }
        const d3 d = e - Ts;
        const double L = sqrt(dot(d, d));
        const double x = L * wv.inv_lam;
        const float ph = (float)(x - floor(x));
        float3 dir[3];
        float3 u = to_f(d);
        dir[k] = u * rsqrtf(dot(u, u));                // the last segment is real
        for (int j = k; j >= 1; --j) dir[j - 1] = mirror_dir_f(dir[j], nf[j - 1]);
        const float Ft = pattern_f(tx.pattern, gt, dot(dir[0], z));
        const float Fin = fmaxf(-dot(dir[k], nr), 0.f);
        const float amp = amp0 * sqrtf(Ft * Fin) / (float)L;
        cv3 v = cv_of(pol_dir(a_t, dir[0]));
        for (int j = 1; j <= k; ++j) v = bounce_real(v, dir[j - 1], dir[j], nf[j - 1], ef[j - 1]);
        float sn, cs;
        sincospif(2.f * ph, &sn, &cs);                 // e^{-j 2 pi frac(L / lambda)}
        acc = cv_add(acc, cv_mul(v, cf{amp * cs, -amp * sn}));
    }
    float w[6] = {acc.x.re, acc.x.im, acc.y.re, acc.y.im, acc.z.re, acc.z.im};
#pragma unroll
    for (int i = 0; i < 6; ++i)
        for (int o = 16; o > 0; o >>= 1) w[i] += __shfl_down_sync(0xffffffffu, w[i], o);
    if (lane == 0) {
        const cv3 s = cv3{cf{w[0], w[1]}, cf{w[2], w[3]}, cf{w[4], w[5]}};
        const float3 t1 = f3((float)fr.t1[0], (float)fr.t1[1], (float)fr.t1[2]);
        const float3 t2 = f3((float)fr.t2[0], (float)fr.t2[1], (float)fr.t2[2]);
        const float kk = (float)K;
        const cf c1 = cscl(cv_dot(s, t1), kk), c2 = cscl(cv_dot(s, t2), kk), c3 = cscl(cv_dot(s, nr), -kk);
        cvec[3 * m] = make_float2(c1.re, c1.im);
        cvec[3 * m + 1] = make_float2(c2.re, c2.im);
        cvec[3 * m + 2] = make_float2(c3.re, c3.im);
    }
}

// E0 of the vector field per receiver (one thread each): LOS (if unblocked) and the environment paths
// of the path set, each from its FP64 Tx image, with the received value (E0v) and the field vector
// (E03, global frame).
__global__ void k_e0_vec(DeviceScene S, const float* __restrict__ rx, int64_t n_rx, AntD tx, AntD rxa, WaveD wv,
                         float3 a_t, float3 a_r, const uint8_t* __restrict__ los, const int64_t* __restrict__ env_off,
                         const int64_t* __restrict__ env_seq, float2* __restrict__ E0v, float2* __restrict__ E03)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rx) return;
    const d3 R = D3((double)rx[3 * r], (double)rx[3 * r + 1], (double)rx[3 * r + 2]);
    const float3 zt = f3((float)tx.z[0], (float)tx.z[1], (float)tx.z[2]);
    const float3 zr = f3((float)rxa.z[0], (float)rxa.z[1], (float)rxa.z[2]);
    const float gt = (float)tx.gain, gr = (float)rxa.gain;
    const float amp0 = (float)(sqrt(2.0 * kEta0 * tx.power * tx.gain) * sqrt(rxa.gain) * wv.lam / (4.0 * kPi));
    const int F = S.n_faces;
    const int64_t e0 = env_off[r], n_env = env_off[r + 1] - e0;
    cf rec = cf{0.f, 0.f};
    cv3 vec = cv_of(f3(0.f, 0.f, 0.f));
    for (int64_t q = -1; q < n_env; ++q) {              // q = -1: LOS
        d3 Ts = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
        int k = 0, fa[2] = {-1, -1};
        if (q < 0) {
            if (!los[r]) continue;
        } else {
            const int64_t id = env_seq[e0 + q];
            if (id < F) {
                k = 1;
                fa[0] = (int)id;
            } else {
                k = 2;
                fa[0] = (int)((id - F) / F);
                fa[1] = (int)((id - F) % F);
            }
            for (int j = 0; j < k; ++j) {
                const dv4 pl = S.faces[fa[j]].plane;
                Ts = mirror_pt(Ts, ld3(pl), pl.w);
            }
        }
        const d3 d = R - Ts;
        const double L = sqrt(dot(d, d));
        const double x = L * wv.inv_lam;
        const float ph = (float)(x - floor(x));
        float3 dir[3];
        float3 u = to_f(d);
        dir[k] = u * rsqrtf(dot(u, u));
        for (int j = k; j >= 1; --j) dir[j - 1] = mirror_dir_f(dir[j], face_n32(S, fa[j - 1]));
        const float Ft = pattern_f(tx.pattern, gt, dot(dir[0], zt));
        const float Fr = pattern_f(rxa.pattern, gr, -dot(dir[k], zr));
        const float amp = amp0 * sqrtf(Ft * Fr) / (float)L;
        cv3 v = cv_of(pol_dir(a_t, dir[0]));
        for (int j = 1; j <= k; ++j)
            v = bounce_real(v, dir[j - 1], dir[j], face_n32(S, fa[j - 1]), face_eps32(S, fa[j - 1], wv));
        float sn, cs;
        sincospif(2.f * ph, &sn, &cs);
        v = cv_mul(v, cf{amp * cs, -amp * sn});
        rec = cadd(rec, cv_dot(v, pol_dir(a_r, dir[k])));
        vec = cv_add(vec, v);
    }
    E0v[r] = make_float2(rec.re, rec.im);
    E03[3 * r] = make_float2(vec.x.re, vec.x.im);
    E03[3 * r + 1] = make_float2(vec.y.re, vec.y.im);
    E03[3 * r + 2] = make_float2(vec.z.re, vec.z.im);
}

template <int PAT>
__device__ __forceinline__ float rx_pat(float c, float gain)
{
    if (PAT == RISRT_PATTERN_ISO) return 1.f;
    return pattern_f(PAT, gain, c);
}

// Sums over the Rx-leg entries of one receiver for element e (RIS frame, c its Tx-leg vector):
// a = sum_q b_mq (received value), V = sum_q b_mq (field vector, RIS frame) when V3.
template <int PAT, bool V3>
__device__ __forceinline__ void rx_leg_sums(const PathRec* __restrict__ rec, int64_t o, int nq, bool direct, float4 e,
                                            const cv3& c, float3 a_r, float inv_lam, float gr, cf& a, cv3& V)
{
    a = cf{0.f, 0.f};
    V = cv_of(f3(0.f, 0.f, 0.f));
    for (int q = 0; q < nq; ++q) {
        const PathRec p = rec[o + q];
        const int kk = __float_as_int(p.a.y);
        const int k = kk & 3;
        if (k == 0 && !direct) continue;               // entry 0: the direct leg, if unblocked
        const float3 w = f3(p.w.x, p.w.y, p.w.z);
        const float3 n1 = f3(p.n1.x, p.n1.y, p.n1.z), n2 = f3(p.n2.x, p.n2.y, p.n2.z);
        // the Rx polarisation axis unfolded like the record's pattern axis
        float3 ar = a_r;
        if (k >= 1) ar = mirror_dir_f(ar, n1);
        if (k == 2) ar = mirror_dir_f(ar, n2);
        const float dx = w.x - e.x, dy = w.y - e.y, dz = w.z;
        const float L2 = dx * dx + dy * dy + dz * dz;
        const float iL = rsqrtf(L2);
        const float L = L2 * iL;
        const float3 d = f3(dx * iL, dy * iL, dz * iL);
        float amp = sqrtf(fmaxf(d.z, 0.f)) * iL;          // sqrt(F_out) / L
        amp *= sqrtf(gr * rx_pat<PAT>(-dot(d, f3(p.v.x, p.v.y, p.v.z)), gr));
        const float dL = (e.z - 2.f * (e.x * w.x + e.y * w.y)) / (L + p.w.w);
        float x = p.a.x + dL * inv_lam;
        x -= rintf(x);
        float sn, cs;
        __sincosf(6.28318530717958647f * x, &sn, &cs);
        const cf b = cf{amp * cs, -amp * sn};
        // Fresnel coefficients of the bounces (a lossless-TE record holds eps_r - 1, no imaginary part)
        cf te1 = cf{1.f, 0.f}, tm1 = te1, te2 = te1, tm2 = te1;
        const bool lt = (kk & kRecLosslessTE) != 0;
        if (k >= 1) {
            const float er = lt ? p.a.z + 1.f : p.a.z, ei = lt ? 0.f : p.a.w;
            const float c1 = fabsf(dot(d, n1));
            te1 = fresnel_f(c1, er, ei, false);
            tm1 = fresnel_f(c1, er, ei, true);
        }
        if (k == 2) {
            const float er = lt ? p.n1.w + 1.f : p.n1.w, ei = lt ? 0.f : p.n2.w;
            const float c2 = fabsf(dot(d, n2));
            te2 = fresnel_f(c2, er, ei, false);
            tm2 = fresnel_f(c2, er, ei, true);
        }
        // received: (D1 D2 unit(P(d) a')) . c
        cv3 u = cv_of(pol_dir(ar, d));
        if (k == 2) u = bounce_unfolded(u, d, n2, te2, tm2);
        if (k >= 1) u = bounce_unfolded(u, d, n1, te1, tm1);
        a = cadd(a, cmulf(b, cv_dotc(u, c)));
        if (V3) {                                      // field vector: H_n1 H_n2' D2 D1 P(d) c
            cv3 f = cv_axpy(c, cscl(cv_dot(c, d), -1.f), d);
            if (k >= 1) f = bounce_unfolded(f, d, n1, te1, tm1);
            if (k == 2) f = bounce_unfolded(f, d, n2, te2, tm2);
            if (k == 2) f = cv_mirror(f, n2);
            if (k >= 1) f = cv_mirror(f, n1);
            V = cv_add(V, cv_mul(f, b));
        }
    }
}

// Field of NC configurations per pass: one warp per receiver, one element per lane per step; the
// received values (E, P) and, with V3, the field vectors E3 [cfg][n_rx][3] in the global frame.
template <int PAT, bool V3>
__global__ void __launch_bounds__(32 * kVecWarps)
k_eval_vec(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W,
           const float4* __restrict__ elem, const float2* __restrict__ cvec, const float2* __restrict__ gamma, int M,
           int64_t n_rx, int cfg0, int n_cfg, const float2* __restrict__ E0v, const float2* __restrict__ E03, Frame fr,
           float3 a_r, float inv_lam, float gr, float inv_2eta0, float2* __restrict__ E, float2* __restrict__ E3,
           float* __restrict__ P)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)kVecWarps + (threadIdx.x >> 5);
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int nq = (int)(off[r + 1] - o);
    cf acc[kVecCfg];
    cv3 acc3[kVecCfg];
#pragma unroll
    for (int c = 0; c < kVecCfg; ++c) {
        acc[c] = cf{0.f, 0.f};
        acc3[c] = cv_of(f3(0.f, 0.f, 0.f));
    }
    for (int m = lane; m < M; m += 32) {
        const float4 e = elem[m];
        const bool direct = (vis[r * W + (m >> 5)] >> (m & 31)) & 1u;
        const cv3 c = cv3{cf{cvec[3 * m].x, cvec[3 * m].y}, cf{cvec[3 * m + 1].x, cvec[3 * m + 1].y},
                          cf{cvec[3 * m + 2].x, cvec[3 * m + 2].y}};
        cf a;
        cv3 V;
        rx_leg_sums<PAT, V3>(rec, o, nq, direct, e, c, a_r, inv_lam, gr, a, V);
#pragma unroll
        for (int cc = 0; cc < kVecCfg; ++cc) {
            if (cc < n_cfg) {
                const float2 g2 = gamma[(int64_t)(cfg0 + cc) * M + m];
                const cf g = cf{g2.x, g2.y};
                acc[cc] = cadd(acc[cc], cmulf(g, a));
                if (V3) acc3[cc] = cv_add(acc3[cc], cv_mul(V, g));
            }
        }
    }
#pragma unroll
    for (int cc = 0; cc < kVecCfg; ++cc) {
        float w[8] = {acc[cc].re, acc[cc].im, acc3[cc].x.re, acc3[cc].x.im, acc3[cc].y.re, acc3[cc].y.im,
                      acc3[cc].z.re, acc3[cc].z.im};
#pragma unroll
        for (int i = 0; i < (V3 ? 8 : 2); ++i)
            for (int s = 16; s > 0; s >>= 1) w[i] += __shfl_down_sync(0xffffffffu, w[i], s);
        if (lane == 0 && cc < n_cfg) {
            const int64_t oi = (int64_t)(cfg0 + cc) * n_rx + r;
            const float2 e0 = E0v[r];
            const float er = e0.x + w[0], ei = e0.y + w[1];
            E[oi] = make_float2(er, ei);
            if (P) P[oi] = (er * er + ei * ei) * inv_2eta0;
            if (V3) {
                // RIS frame -> global: x t1 + y t2 + z n
                const cf vx = cf{w[2], w[3]}, vy = cf{w[4], w[5]}, vz = cf{w[6], w[7]};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float a1 = (float)fr.t1[j], a2 = (float)fr.t2[j], a3 = (float)fr.n[j];
                    const float2 b = E03[3 * r + j];
                    E3[3 * oi + j] = make_float2(b.x + vx.re * a1 + vy.re * a2 + vz.re * a3,
                                                 b.y + vx.im * a1 + vy.im * a2 + vz.im * a3);
                }
            }
        }
    }
}

// Received-value channel rows of the vector field: A[r][m] = sum_q b_mq (received), so that the
// received E = E0v + A . Gamma.
template <int PAT>
__global__ void __launch_bounds__(32 * kVecWarps)
k_build_A_vec(const PathRec* __restrict__ rec, const int64_t* __restrict__ off, const uint32_t* __restrict__ vis,
              int W, const float4* __restrict__ elem, const float2* __restrict__ cvec, int M, int64_t n_rx, float3 a_r,
              float inv_lam, float gr, float2* __restrict__ A)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)kVecWarps + (threadIdx.x >> 5);
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int nq = (int)(off[r + 1] - o);
    for (int m = lane; m < M; m += 32) {
        const float4 e = elem[m];
        const bool direct = (vis[r * W + (m >> 5)] >> (m & 31)) & 1u;
        const cv3 c = cv3{cf{cvec[3 * m].x, cvec[3 * m].y}, cf{cvec[3 * m + 1].x, cvec[3 * m + 1].y},
                          cf{cvec[3 * m + 2].x, cvec[3 * m + 2].y}};
        cf a;
        cv3 V;
        rx_leg_sums<PAT, false>(rec, o, nq, direct, e, c, a_r, inv_lam, gr, a, V);
        A[r * (int64_t)M + m] = make_float2(a.re, a.im);
    }
}

// unit axis in the frame's coordinates (t1, t2, n)
float3 to_frame(const Frame& fr, const float* a)
{
    double v[3] = {0, 0, 0};
    for (int j = 0; j < 3; ++j) {
        v[0] += fr.t1[j] * a[j];
        v[1] += fr.t2[j] * a[j];
        v[2] += fr.n[j] * a[j];
    }
    return f3((float)v[0], (float)v[1], (float)v[2]);
}

}  // namespace

// The receiver-independent parts: the elements' Tx-leg vectors and E0's received values and field
// vectors, into blocks of the context (freed by the caller after its last kernel).
static int vec_prepare(risrt_ctx* ctx, const risrt_scene* sc, const risrt_rxset* rxs, const risrt_pathset* ps,
                       void** cvec, void** e0v, void** e03)
{
    cudaStream_t s = ctx->stream;
    const int M = ps->M;
    const int64_t n_rx = ps->n_rx;
    RISRT_CUDA(ctx, ctx_malloc(ctx, cvec, sizeof(float2) * 3 * (size_t)M));
    RISRT_CUDA(ctx, ctx_malloc(ctx, e0v, sizeof(float2) * (size_t)n_rx));
    RISRT_CUDA(ctx, ctx_malloc(ctx, e03, sizeof(float2) * 3 * (size_t)n_rx));
    const float3 a_t = f3(ctx->pol[RISRT_TX][0], ctx->pol[RISRT_TX][1], ctx->pol[RISRT_TX][2]);
    const float3 a_r = f3(ctx->pol[RISRT_RX][0], ctx->pol[RISRT_RX][1], ctx->pol[RISRT_RX][2]);
    const int n_tx = (int)ps->tx_seq_host.size();
    RISRT_KERNEL(ctx, "k_cm_vec", (k_cm_vec<<<nblk((int64_t)M * 32, 128), 128, 0, s>>>(
                                      ps->elem, M, ps->fr, ps->txa, ps->wv, ps->K, a_t, ps->tx_vis_dev, ps->tx_paths,
                                      n_tx, (float2*)*cvec)));
    RISRT_KERNEL(ctx, "k_e0_vec", (k_e0_vec<<<nblk(n_rx, 128), 128, 0, s>>>(
                                      sc->dev(), rxs->xyz, n_rx, ps->txa, ps->rxa, ps->wv, a_t, a_r, ps->los, ps->env_off,
                                      ps->env_seq, (float2*)*e0v, (float2*)*e03)));
    return RISRT_OK;
}

int eval_field_vec(risrt_ctx* ctx, const risrt_scene* sc, const risrt_rxset* rxs, const risrt_pathset* ps,
                   const float2* gamma, int n_cfg, float2* E, float2* E3, float* P)
{
    void *cvec = nullptr, *e0v = nullptr, *e03 = nullptr;
    int rc = vec_prepare(ctx, sc, rxs, ps, &cvec, &e0v, &e03);
    if (!rc) {
        const float3 a_r = to_frame(ps->fr, ctx->pol[RISRT_RX]);
        const float inv_lam = (float)(ps->freq / kC0);
        const float inv_2eta0 = (float)(1.0 / (2.0 * kEta0));
        const unsigned grid = nblk(ps->n_rx, kVecWarps);
        for (int c0 = 0; c0 < n_cfg && !rc; c0 += kVecCfg) {
            const int nc = std::min(kVecCfg, n_cfg - c0);
            auto launch = [&](auto kern) -> int {
                RISRT_KERNEL(ctx, "k_eval_vec", (kern<<<grid, 32 * kVecWarps, 0, ctx->stream>>>(
                                                    ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, (const float2*)cvec,
                                                    gamma, ps->M, ps->n_rx, c0, nc, (const float2*)e0v,
                                                    (const float2*)e03, ps->fr, a_r, inv_lam, ps->rx_gain, inv_2eta0, E,
                                                    E3, P)));
                return RISRT_OK;
            };
#define RISRT_VEC(PAT) (E3 ? launch(k_eval_vec<PAT, true>) : launch(k_eval_vec<PAT, false>))
            switch (ps->rx_pattern) {
                case RISRT_PATTERN_COS_POW: rc = RISRT_VEC(RISRT_PATTERN_COS_POW); break;
                case RISRT_PATTERN_MONOPOLE_QW: rc = RISRT_VEC(RISRT_PATTERN_MONOPOLE_QW); break;
                default: rc = RISRT_VEC(RISRT_PATTERN_ISO); break;
            }
#undef RISRT_VEC
        }
    }
    ctx_free(ctx, cvec);    // later users of the blocks are ordered after this work on the context's stream
    ctx_free(ctx, e0v);
    ctx_free(ctx, e03);
    return rc;
}

int build_A_vec(risrt_ctx* ctx, const risrt_scene* sc, const risrt_rxset* rxs, const risrt_pathset* ps, float2* A,
                float2* E0)
{
    void *cvec = nullptr, *e0v = nullptr, *e03 = nullptr;
    int rc = vec_prepare(ctx, sc, rxs, ps, &cvec, &e0v, &e03);
    if (!rc) {
        const float3 a_r = to_frame(ps->fr, ctx->pol[RISRT_RX]);
        const float inv_lam = (float)(ps->freq / kC0);
        const unsigned grid = nblk(ps->n_rx, kVecWarps);
        auto launch = [&](auto kern) -> int {
            RISRT_KERNEL(ctx, "k_build_A_vec", (kern<<<grid, 32 * kVecWarps, 0, ctx->stream>>>(
                                                   ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, (const float2*)cvec,
                                                   ps->M, ps->n_rx, a_r, inv_lam, ps->rx_gain, A)));
            return RISRT_OK;
        };
        switch (ps->rx_pattern) {
            case RISRT_PATTERN_COS_POW: rc = launch(k_build_A_vec<RISRT_PATTERN_COS_POW>); break;
            case RISRT_PATTERN_MONOPOLE_QW: rc = launch(k_build_A_vec<RISRT_PATTERN_MONOPOLE_QW>); break;
            default: rc = launch(k_build_A_vec<RISRT_PATTERN_ISO>); break;
        }
        if (!rc && E0)
            RISRT_CUDA(ctx, cudaMemcpyAsync(E0, e0v, sizeof(float2) * (size_t)ps->n_rx, cudaMemcpyDeviceToDevice,
                                            ctx->stream));
    }
    ctx_free(ctx, cvec);
    ctx_free(ctx, e0v);
    ctx_free(ctx, e03);
    return rc;
}

}  // namespace risrt
