// Adjoint of the received power with respect to every element's phase (from Eq. 9 and Eq. 10):
//   Gamma_bm = amp_m e^{j phi_bm},  E_b(r) = E0(r) + sum_m A[r][m] Gamma_bm,  P = |E|^2 / (2 eta0)
//   J_b = sum_{r in T} log P_b(r)
//   dJ_b/dphi_bm = -2 Im( Gamma_bm sum_{r in T} A[r][m] conj(E_b(r)) / |E_b(r)|^2 )
// |E|^2 is clamped from below at 1e-30 max_r |E_b(r)|^2 on both sides of the comparison.
// Three passes, all FP32 on the CUDA cores: forward GEMM over the target rows (E), the per-config
// clamp, log and weights w = conj(E)/|E|^2, and the backward GEMM A^T w with the phase epilogue.
#include <cuda_bf16.h>

#include <algorithm>

#include "sweep.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void k_check_targets(const int* __restrict__ target, int n_t, int64_t n_rx, int* __restrict__ bad)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_t && (target[t] < 0 || target[t] >= n_rx)) atomicExch(bad, 1);
}

constexpr int kFR = 64, kFB = 64, kFK = 16;   // forward tile: 64 target rows x 64 configs

// E[b][t] = E0[r_t] + sum_m A[r_t][m] Gamma_bm for target t (row r_t).
__global__ void __launch_bounds__(256)
k_adj_forward(const float2* __restrict__ A, const float2* __restrict__ E0, int M, const int* __restrict__ target,
              int n_t, const float* __restrict__ phases, const float* __restrict__ amp, int B, int k_chunk,
              float2* __restrict__ E)
{
    __shared__ float2 sA[kFK][kFR + 1];
    __shared__ float2 sG[kFK][kFB + 1];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tb = tid % 16;    // 4 rows x 4 configs per thread
    const int t0 = blockIdx.x * kFR, b0 = blockIdx.y * kFB;
    const int k_begin = blockIdx.z * k_chunk, k_end = min(M, k_begin + k_chunk);
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = k_begin; k0 < k_end; k0 += kFK) {
        for (int i = tid; i < kFR * kFK; i += 256) {
            const int rr = i / kFK, kk = i % kFK;
            const int t = t0 + rr, k = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (t < n_t && k < k_end) {
                const int64_t r = target ? target[t] : t;
                v = A[r * M + k];
            }
            sA[kk][rr] = v;
        }
        for (int i = tid; i < kFB * kFK; i += 256) {
            const int bb = i / kFK, kk = i % kFK;
            const int b = b0 + bb, k = k0 + kk;
            float2 g = make_float2(0.f, 0.f);
            if (b < B && k < k_end) {
                float sn, cs;
                sincosf(phases[(int64_t)b * M + k], &sn, &cs);
                const float a = amp ? amp[k] : 1.f;
                g = make_float2(a * cs, a * sn);
            }
            sG[kk][bb] = g;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kFK; ++kk) {
            float2 a[4], g[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j] = sG[kk][tb + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(a[i].x, g[j].x, fmaf(-a[i].y, g[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, g[j].y, fmaf(a[i].y, g[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int t = t0 + tr + 16 * i;
        if (t >= n_t) continue;
        const int64_t r = target ? target[t] : t;
        const float2 e0 = (E0 && blockIdx.z == 0) ? E0[r] : make_float2(0.f, 0.f);
        float2* Ez = E + (int64_t)blockIdx.z * B * n_t;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + tb + 16 * j;
            if (b < B) Ez[(int64_t)b * n_t + t] = make_float2(acc[i][j].x + e0.x, acc[i][j].y + e0.y);
        }
    }
}

// Per configuration (one block): clamp floor, J_b = sum log(|E|^2 / (2 eta0)), w = conj(E)/|E|^2.
// Fixed-order reductions (block tree) keep J deterministic. Each term's logarithm in FP32 (about
// 1e-7 absolute), summed in FP64: J_b = sum_t log|E_t|^2 + n_t log(1 / (2 eta0)).
__global__ void __launch_bounds__(512)
k_adj_weights(float2* __restrict__ E, int n_t, int B, int splits, float* __restrict__ J, float inv_2eta0)
{
    __shared__ double red[512];
    const int b = blockIdx.x;
    float2* e = E + (int64_t)b * n_t;
    float mx = 0.f;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
        float2 v = e[t];
        for (int z = 1; z < splits; ++z) {          // fixed-order sum of the split-K partials
            const float2 u = E[((int64_t)z * B + b) * n_t + t];
            v.x += u.x;
            v.y += u.y;
        }
        e[t] = v;
        mx = fmaxf(mx, v.x * v.x + v.y * v.y);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    const float floor_ = (float)(red[0] * 1e-30);
    __syncthreads();
    double acc = 0.0;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
        const float2 v = e[t];
        const float p = fmaxf(v.x * v.x + v.y * v.y, floor_);
        acc += (double)logf(p);
        e[t] = make_float2(v.x / p, -v.y / p);      // w = conj(E) / |E|^2 (E is overwritten)
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) J[b] = (float)(red[0] + (double)n_t * log((double)inv_2eta0));
}

constexpr int kBM = 64, kBB = 64, kBK = 16;   // backward tile: 64 elements x 64 configs

// g[b][m] = sum_t A[r_t][m] w[b][t];  grad[b][m] = -2 Im(Gamma_bm g[b][m]).
__global__ void __launch_bounds__(256)
k_adj_backward(const float2* __restrict__ A, int M, const int* __restrict__ target, int n_t,
               const float2* __restrict__ W, int B, int t_chunk, float2* __restrict__ Gp)
{
    __shared__ float2 sA[kBK][kBM + 1];
    __shared__ float2 sW[kBK][kBB + 1];
    const int tid = threadIdx.x;
    const int tm = tid % 16, tb = tid / 16;   // 4 elements x 4 configs per thread
    const int m0 = blockIdx.x * kBM, b0 = blockIdx.y * kBB;
    const int t_begin = blockIdx.z * t_chunk, t_end = min(n_t, t_begin + t_chunk);
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = t_begin; k0 < t_end; k0 += kBK) {
        for (int i = tid; i < kBM * kBK; i += 256) {        // coalesced along elements
            const int kk = i / kBM, mm = i % kBM;
            const int t = k0 + kk, m = m0 + mm;
            float2 v = make_float2(0.f, 0.f);
            if (t < t_end && m < M) {
                const int64_t r = target ? target[t] : t;
                v = A[r * M + m];
            }
            sA[kk][mm] = v;
        }
        for (int i = tid; i < kBB * kBK; i += 256) {
            const int bb = i / kBK, kk = i % kBK;
            const int b = b0 + bb, t = k0 + kk;
            sW[kk][bb] = (b < B && t < t_end) ? W[(int64_t)b * n_t + t] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float2 a[4], w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][tm + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = sW[kk][tb + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(a[i].x, w[j].x, fmaf(-a[i].y, w[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, w[j].y, fmaf(a[i].y, w[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
    float2* Gz = Gp + (int64_t)blockIdx.z * B * M;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tm + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + tb + 16 * j;
            if (b < B) Gz[(int64_t)b * M + m] = acc[i][j];
        }
    }
}

// grad[b][m] = -2 Im(Gamma_bm g[b][m]), g summed over the split partials in a fixed order.
__global__ void k_adj_grad(const float2* __restrict__ Gp, int splits, const float* __restrict__ phases,
                           const float* __restrict__ amp, int B, int M, float* __restrict__ grad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * M) return;
    const int m = (int)(i % M);
    float2 g = Gp[i];
    for (int z = 1; z < splits; ++z) {
        const float2 u = Gp[(int64_t)z * B * M + i];
        g.x += u.x;
        g.y += u.y;
    }
    float sn, cs;
    sincosf(phases[i], &sn, &cs);
    const float a = amp ? amp[m] : 1.f;
    grad[i] = -2.f * a * (cs * g.y + sn * g.x);     // Im(Gamma g), Gamma = a (cs + j sn)
}

// ---- tensor-core path: both GEMMs as real BF16 GEMMs with split operands ------------------------
// A complex product is one real GEMM over [Re | Im] blocks. Every real factor x is split as
// hi = bf16(x), lo = bf16(x - hi); the large operand (A, read once per GEMM) carries [hi | lo] of its
// real and imaginary parts (four K blocks, 8 bytes per complex entry, as many as FP32), and every
// configuration b of the small operand gives two virtual configurations: 2b pairs hi(g) with both
// blocks of A (hi(A) hi(g) + lo(A) hi(g)), 2b + 1 pairs lo(g) with hi(A) only. Their sum is the
// three-term product (the lo.lo term, below 2^-16 of the product, is dropped), about 1e-5 relative.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Forward operand X [n_t][Kf]: row t = [hi(Re A) | hi(Im A) | lo(Re A) | lo(Im A)] of A's target row
// (M columns each; columns past 4M are cleared separately); E0t[t] = E0 of that row.
__global__ void k_gpack_xf(const float2* __restrict__ A, const float2* __restrict__ E0, int M, const int* __restrict__ target,
                           int n_t, int Kf, __nv_bfloat16* __restrict__ X, float2* __restrict__ E0t)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int t = blockIdx.y; t < n_t; t += gridDim.y) {
        const int64_t r = target ? target[t] : t;
        const float2 a = A[r * M + m];
        __nv_bfloat16 rh, rl, ih, il;
        split_bf16(a.x, rh, rl);
        split_bf16(a.y, ih, il);
        __nv_bfloat16* row = X + (int64_t)t * Kf;
        row[m] = rh;
        row[M + m] = ih;
        row[2 * M + m] = rl;
        row[3 * M + m] = il;
        if (m == 0) E0t[t] = E0 ? E0[r] : make_float2(0.f, 0.f);
    }
}

// Backward operand X [M][Kb] (A transposed): row m = [hi(Re A) | hi(Im A) | lo(Re A) | lo(Im A)] over
// the targets t (n_t columns each). 32 x 32 tiles through shared memory.
__global__ void k_gpack_xb(const float2* __restrict__ A, int M, const int* __restrict__ target, int n_t, int Kb,
                           __nv_bfloat16* __restrict__ X)
{
    __shared__ float2 tile[32][33];
    const int m0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int t = t0 + y, m = m0 + threadIdx.x;
        float2 v = make_float2(0.f, 0.f);
        if (t < n_t && m < M) v = A[(int64_t)(target ? target[t] : t) * M + m];
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int m = m0 + y, t = t0 + threadIdx.x;
        if (m >= M || t >= n_t) continue;
        const float2 v = tile[threadIdx.x][y];
        __nv_bfloat16* row = X + (int64_t)m * Kb;
        __nv_bfloat16 rh, rl, ih, il;
        split_bf16(v.x, rh, rl);
        split_bf16(v.y, ih, il);
        row[t] = rh;
        row[n_t + t] = ih;
        row[2 * n_t + t] = rl;
        row[3 * n_t + t] = il;
    }
}

// Zero columns [c0, K) of every row of a [rows][K] operand.
__global__ void k_gpack_pad(int64_t rows, int c0, int K, __nv_bfloat16* __restrict__ X)
{
    const int pad = K - c0;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pad <= 0 || i >= rows * pad) return;
    X[(i / pad) * K + c0 + i % pad] = __float2bfloat16_rn(0.f);
}

// The small operand Y [Np][K] (rows past 4B cleared separately) from complex coefficients v[b][k],
// k < n (n columns per block of the large operand): virtual configuration 2b (rows 4b, 4b + 1 = Re,
// Im) with hi(v) against all four blocks, 2b + 1 (rows 4b + 2, 4b + 3) with lo(v) against the hi
// blocks. Re: [Re v, -Im v] against [Re A, Im A]; Im: [Im v, Re v].
__device__ __forceinline__ void put_small_operand(__nv_bfloat16* __restrict__ Y, int K, int n, int b, int k, float vr, float vi)
{
    __nv_bfloat16 rh, rl, ih, il;
    split_bf16(vr, rh, rl);
    split_bf16(vi, ih, il);
    const __nv_bfloat16 nih = __hneg(ih), nil = __hneg(il), z = __float2bfloat16_rn(0.f);
    __nv_bfloat16* r0 = Y + (int64_t)(4 * b) * K;    // hi, Re
    __nv_bfloat16* r1 = r0 + K;                      // hi, Im
    __nv_bfloat16* r2 = r1 + K;                      // lo, Re
    __nv_bfloat16* r3 = r2 + K;                      // lo, Im
    r0[k] = rh; r0[n + k] = nih; r0[2 * n + k] = rh; r0[3 * n + k] = nih;
    r1[k] = ih; r1[n + k] = rh;  r1[2 * n + k] = ih; r1[3 * n + k] = rh;
    r2[k] = rl; r2[n + k] = nil; r2[2 * n + k] = z;  r2[3 * n + k] = z;
    r3[k] = il; r3[n + k] = rl;  r3[2 * n + k] = z;  r3[3 * n + k] = z;
}

// Forward small operand from Gamma_bm = amp_m e^{j phi_bm}.
__global__ void k_gpack_yf(const float* __restrict__ phases, const float* __restrict__ amp, int M, int B, int Kf,
                           __nv_bfloat16* __restrict__ Y)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const float a = amp ? amp[m] : 1.f;
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        float sn, cs;
        sincosf(phases[(int64_t)b * M + m], &sn, &cs);
        put_small_operand(Y, Kf, M, b, m, a * cs, a * sn);
    }
}

// Backward small operand from the weights w[b][t].
__global__ void k_gpack_yb(const float2* __restrict__ W, int n_t, int B, int Kb, __nv_bfloat16* __restrict__ Y)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_t) return;
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const float2 w = W[(int64_t)b * n_t + t];
        put_small_operand(Y, Kb, n_t, b, t, w.x, w.y);
    }
}

// Tensor-core path, weights in three passes over (target chunk, configuration) blocks, every sum in a
// fixed order: (1) E_b = E0 + the split-K partials of both virtual configurations into W, and the
// maximum of |E_b|^2 (an integer atomic max on the float's bits: the order does not matter);
// (2) clamp floor, per-block sums of log|E|^2 (FP32 logarithms, FP64 sums) and w = conj(E)/|E|^2 in
// place; (3) J_b = sum of the blocks' sums + n_t log(1 / (2 eta0)).
constexpr int kWT = 256;    // targets per block of the weights passes

__global__ void __launch_bounds__(kWT)
k_adj_sum_tc(const float2* __restrict__ Ep, const float2* __restrict__ E0t, int n_t, int B, int splits, int chunks,
             float2* __restrict__ W, unsigned* __restrict__ maxbits)
{
    __shared__ float red[kWT / 32];
    const int b = (int)(blockIdx.x / chunks), t = (int)(blockIdx.x % chunks) * kWT + threadIdx.x;
    float p2 = 0.f;
    if (t < n_t) {
        float2 v = E0t[t];
        for (int z = 0; z < splits; ++z) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 u = Ep[((int64_t)z * 2 * B + 2 * b + h) * n_t + t];
                v.x += u.x;
                v.y += u.y;
            }
        }
        W[(int64_t)b * n_t + t] = v;
        p2 = v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) p2 = fmaxf(p2, __shfl_down_sync(0xffffffffu, p2, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = red[0];
        for (int i = 1; i < kWT / 32; ++i) mx = fmaxf(mx, red[i]);
        atomicMax(maxbits + b, __float_as_uint(mx));      // non-negative floats order like their bits
    }
}

__global__ void __launch_bounds__(kWT)
k_adj_w_tc(float2* __restrict__ W, int n_t, int chunks, const unsigned* __restrict__ maxbits, double* __restrict__ Jpart)
{
    __shared__ float red[kWT / 32];
    const int b = (int)(blockIdx.x / chunks), c = (int)(blockIdx.x % chunks), t = c * kWT + threadIdx.x;
    const float floor_ = __uint_as_float(maxbits[b]) * 1e-30f;   // (a denormal floor is exact enough)
    float lg = 0.f;
    if (t < n_t) {
        const float2 v = W[(int64_t)b * n_t + t];
        const float p = fmaxf(v.x * v.x + v.y * v.y, floor_);
        lg = logf(p);
        W[(int64_t)b * n_t + t] = make_float2(v.x / p, -v.y / p);
    }
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_down_sync(0xffffffffu, lg, o);   // 32 terms in FP32
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int i = 0; i < kWT / 32; ++i) acc += (double)red[i];
        Jpart[(int64_t)b * chunks + c] = acc;
    }
}

// One warp per configuration: lanes take chunks lane, lane + 32, ..., then a shuffle tree (fixed order).
__global__ void k_adj_J_tc(const double* __restrict__ Jpart, int chunks, int n_t, int B, float* __restrict__ J,
                           float inv_2eta0)
{
    const int lane = threadIdx.x & 31;
    const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (b >= B) return;
    double acc = 0.0;
    for (int c = lane; c < chunks; c += 32) acc += Jpart[(int64_t)b * chunks + c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) J[b] = (float)(acc + (double)n_t * log((double)inv_2eta0));
}

// grad[b][m] = -2 Im(Gamma_bm g[b][m]), g summed over the split partials of both virtual
// configurations in a fixed order.
__global__ void k_adj_grad_tc(const float2* __restrict__ Gp, int splits, const float* __restrict__ phases,
                              const float* __restrict__ amp, int B, int M, float* __restrict__ grad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * M) return;
    const int b = (int)(i / M), m = (int)(i % M);
    float2 g = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int z = 0; z < splits; ++z) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 u = Gp[((int64_t)z * 2 * B + 2 * b + h) * M + m];
            g.x += u.x;
            g.y += u.y;
        }
    }
    float sn, cs;
    sincosf(phases[i], &sn, &cs);
    const float a = amp ? amp[m] : 1.f;
    grad[i] = -2.f * a * (cs * g.y + sn * g.x);     // Im(Gamma g), Gamma = a (cs + j sn)
}

}  // namespace

struct GradSplits {
    int fwd, bwd, k_chunk, t_chunk;
};

GradSplits grad_splits(int n_t, int B, int M)
{
    GradSplits g;
    const int target_blocks = 4 * 152;
    const int fw_tiles = (int)(nblk(n_t, kFR) * nblk(B, kFB));
    g.fwd = std::max(1, std::min(16, (target_blocks + fw_tiles - 1) / fw_tiles));
    g.k_chunk = (int)((nblk(M, g.fwd) + kFK - 1) / kFK * kFK);
    g.fwd = (int)nblk(M, g.k_chunk);
    const int bw_tiles = (int)(nblk(M, kBM) * nblk(B, kBB));
    g.bwd = std::max(1, std::min(64, (target_blocks + bw_tiles - 1) / bw_tiles));
    g.t_chunk = (int)((nblk(n_t, g.bwd) + kBK - 1) / kBK * kBK);
    g.bwd = (int)nblk(n_t, g.t_chunk);
    return g;
}

// Layout of the tensor-core workspace (byte offsets, 256-aligned) and its split-K part counts: both
// large operands ([hi | lo] of Re and Im: 4M and 4 n_t columns), both small ones (4 rows per
// configuration), E0 of the target rows, the partial sums of the 2B virtual configurations, w.
struct GradTcLayout {
    int Kf, Kb, Np, sf, sb;
    size_t xf, yf, e0t, ep, w, xb, yb, gp, jm, end;
};

GradTcLayout grad_tc_layout(int n_t, int B, int M)
{
    GradTcLayout L;
    auto up = [](int64_t v, int64_t a) { return (v + a - 1) / a * a; };
    L.Kf = (int)up(4LL * M, kTcBK);
    L.Kb = (int)up(4LL * n_t, kTcBK);
    L.Np = (int)up(4LL * B, kTcBN);
    // about 128 (tile, part) items per GEMM over the 76 SM pairs (measured on 16,384 targets x 4,096
    // elements x 64 configurations: 2 forward and 8 backward parts, 0.241 ms for both GEMMs against
    // 0.266 ms with 3 and 10)
    const int items = 128;
    const int tf = (int)(up(n_t, 2 * kTcBM) / (2 * kTcBM)) * (L.Np / kTcBN);
    const int tb = (int)(up(M, 2 * kTcBM) / (2 * kTcBM)) * (L.Np / kTcBN);
    L.sf = std::max(1, std::min(8, (items + tf / 2) / tf));
    L.sb = std::max(1, std::min(16, (items + tb / 2) / tb));
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t a = o;
        o = (size_t)up((int64_t)(o + bytes), 256);
        return a;
    };
    L.xf = take((size_t)n_t * L.Kf * 2);
    L.yf = take((size_t)L.Np * L.Kf * 2);
    L.e0t = take((size_t)n_t * sizeof(float2));
    L.ep = take((size_t)L.sf * 2 * B * n_t * sizeof(float2));
    L.w = take((size_t)B * n_t * sizeof(float2));
    L.xb = take((size_t)M * L.Kb * 2);
    L.yb = take((size_t)L.Np * L.Kb * 2);
    L.gp = take((size_t)L.sb * 2 * B * M * sizeof(float2));
    L.jm = take((size_t)B * sizeof(unsigned) + (size_t)B * ((n_t + kWT - 1) / kWT) * sizeof(double));
    L.end = o;
    return L;
}

size_t grad_workspace_bytes(int n_t, int B, int M, int precision)
{
    if (precision == RISRT_PREC_BF16X2) return grad_tc_layout(n_t, B, M).end + 256;
    GradSplits g = grad_splits(n_t, B, M);
    return sizeof(float2) * ((size_t)g.fwd * n_t * B + (size_t)g.bwd * B * M) + 256;
}

int check_targets(risrt_ctx* ctx, const int* target, int n_t, int64_t n_rx, void* ws, size_t ws_bytes)
{
    int* bad = (int*)((char*)ws + ws_bytes - 16);
    RISRT_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    RISRT_KERNEL(ctx, "k_check_targets", (k_check_targets<<<nblk(n_t, 256), 256, 0, ctx->stream>>>(target, n_t, n_rx, bad)));
    int h = 0;
    RISRT_CUDA(ctx, cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RISRT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return fail(ctx, RISRT_ERR_INVALID_ARG, "a target row is outside [0, n_rx)");
    return RISRT_OK;
}

// Tensor-core adjoint: both GEMMs on SM pairs (split-K), the packing of A into its forward and
// transposed operands done per call unless keep_a (A and the targets may change between calls). The
// GEMMs' pipeline-timeout flag is read once, after the last kernel, or left for grad_check (defer).
static int grad_phases_tc(risrt_ctx* ctx, const float2* A, const float2* E0, int M, const int* target, int n_t,
                          const float* phases, const float* amp, int B, float* J, float* grad, void* ws, size_t ws_bytes,
                          bool keep_a, bool defer)
{
    cudaStream_t s = ctx->stream;
    const GradTcLayout L = grad_tc_layout(n_t, B, M);
    char* w = (char*)ws;
    __nv_bfloat16* Xf = (__nv_bfloat16*)(w + L.xf);
    __nv_bfloat16* Yf = (__nv_bfloat16*)(w + L.yf);
    float2* E0t = (float2*)(w + L.e0t);
    float2* Ep = (float2*)(w + L.ep);
    float2* W = (float2*)(w + L.w);
    __nv_bfloat16* Xb = (__nv_bfloat16*)(w + L.xb);
    __nv_bfloat16* Yb = (__nv_bfloat16*)(w + L.yb);
    float2* Gp = (float2*)(w + L.gp);
    unsigned* maxbits = (unsigned*)(w + L.jm);
    double* Jpart = (double*)(w + L.jm + ((B * sizeof(unsigned) + 7) & ~(size_t)7));
    const int chunks = (int)nblk(n_t, kWT);
    unsigned* err = (unsigned*)(w + ws_bytes - 32);
    const unsigned gy_t = (unsigned)std::min(n_t, 65535), gy_b = (unsigned)std::min(B, 65535);
    RISRT_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    if (!keep_a) {              // A's target rows into both operands (kept in the workspace for KEEP_A calls)
        RISRT_KERNEL(ctx, "k_gpack_xf", (k_gpack_xf<<<dim3(nblk(M, 256), gy_t), 256, 0, s>>>(A, E0, M, target, n_t, L.Kf, Xf, E0t)));
        if (L.Kf > 4 * M)
            RISRT_KERNEL(ctx, "k_gpack_pad", (k_gpack_pad<<<nblk((int64_t)n_t * (L.Kf - 4 * M), 256), 256, 0, s>>>(n_t, 4 * M, L.Kf, Xf)));
        RISRT_KERNEL(ctx, "k_gpack_xb", (k_gpack_xb<<<dim3(nblk(M, 32), nblk(n_t, 32)), dim3(32, 8), 0, s>>>(A, M, target, n_t, L.Kb, Xb)));
        if (L.Kb > 4 * n_t)
            RISRT_KERNEL(ctx, "k_gpack_pad", (k_gpack_pad<<<nblk((int64_t)M * (L.Kb - 4 * n_t), 256), 256, 0, s>>>(M, 4 * n_t, L.Kb, Xb)));
    }
    // small operands: rows past the 4B used ones and columns past 4M / 4 n_t are zero (nothing to clear
    // when every row and column is written)
    const bool y_full = L.Np == 4 * B;
    if (!y_full || L.Kf > 4 * M) RISRT_CUDA(ctx, cudaMemsetAsync(Yf, 0, (size_t)L.Np * L.Kf * 2, s));
    RISRT_KERNEL(ctx, "k_gpack_yf", (k_gpack_yf<<<dim3(nblk(M, 256), gy_b), 256, 0, s>>>(phases, amp, M, B, L.Kf, Yf)));
    int pf = 0, pb = 0, rc;
    if ((rc = gemm_tc_complex(ctx, Xf, n_t, Yf, L.Np, L.Kf, nullptr, 2 * B, Ep, L.sf, &pf, err))) return rc;
    RISRT_CUDA(ctx, cudaMemsetAsync(maxbits, 0, B * sizeof(unsigned), s));
    RISRT_KERNEL(ctx, "k_adj_weights", (k_adj_sum_tc<<<(unsigned)((int64_t)chunks * B), kWT, 0, s>>>(Ep, E0t, n_t, B, pf, chunks, W, maxbits)));
    RISRT_KERNEL(ctx, "k_adj_weights", (k_adj_w_tc<<<(unsigned)((int64_t)chunks * B), kWT, 0, s>>>(W, n_t, chunks, maxbits, Jpart)));
    RISRT_KERNEL(ctx, "k_adj_weights", (k_adj_J_tc<<<nblk((int64_t)B * 32, 128), 128, 0, s>>>(Jpart, chunks, n_t, B, J, (float)(1.0 / (2.0 * kEta0)))));
    if (!y_full || L.Kb > 4 * n_t) RISRT_CUDA(ctx, cudaMemsetAsync(Yb, 0, (size_t)L.Np * L.Kb * 2, s));
    RISRT_KERNEL(ctx, "k_gpack_yb", (k_gpack_yb<<<dim3(nblk(n_t, 256), gy_b), 256, 0, s>>>(W, n_t, B, L.Kb, Yb)));
    if ((rc = gemm_tc_complex(ctx, Xb, M, Yb, L.Np, L.Kb, nullptr, 2 * B, Gp, L.sb, &pb, err))) return rc;
    RISRT_KERNEL(ctx, "k_adj_grad", (k_adj_grad_tc<<<nblk((int64_t)B * M, 256), 256, 0, s>>>(Gp, pb, phases, amp, B, M, grad)));
    if (defer) return RISRT_OK;
    return grad_check(ctx, ws, ws_bytes);
}

int grad_check(risrt_ctx* ctx, const void* ws, size_t ws_bytes)
{
    const unsigned* err = (const unsigned*)((const char*)ws + ws_bytes - 32);   // as in grad_phases_tc
    unsigned h = 0;
    RISRT_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    RISRT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return fail(ctx, RISRT_ERR_TIMEOUT, "tensor-core GEMM: a pipeline wait expired");
    return RISRT_OK;
}

int grad_phases(risrt_ctx* ctx, const float2* A, const float2* E0, int M, const int* target, int n_t,
                const float* phases, const float* amp, int B, float* J, float* grad, void* ws, size_t ws_bytes,
                int precision, bool keep_a, bool defer)
{
    if (precision == RISRT_PREC_BF16X2)
        return grad_phases_tc(ctx, A, E0, M, target, n_t, phases, amp, B, J, grad, ws, ws_bytes, keep_a, defer);
    cudaStream_t s = ctx->stream;
    const GradSplits g = grad_splits(n_t, B, M);
    RISRT_CUDA(ctx, cudaMemsetAsync((char*)ws + ws_bytes - 32, 0, sizeof(unsigned), s));   // no timeout flag here
    float2* E = (float2*)ws;                               // [fwd][B][n_t] partials, then w in split 0
    float2* Gp = E + (size_t)g.fwd * n_t * B;              // [bwd][B][M]
    RISRT_KERNEL(ctx, "k_adj_forward", (k_adj_forward<<<dim3(nblk(n_t, kFR), nblk(B, kFB), g.fwd), 256, 0, s>>>(
                                           A, E0, M, target, n_t, phases, amp, B, g.k_chunk, E)));
    RISRT_KERNEL(ctx, "k_adj_weights", (k_adj_weights<<<B, 512, 0, s>>>(E, n_t, B, g.fwd, J, (float)(1.0 / (2.0 * kEta0)))));
    RISRT_KERNEL(ctx, "k_adj_backward", (k_adj_backward<<<dim3(nblk(M, kBM), nblk(B, kBB), g.bwd), 256, 0, s>>>(
                                            A, M, target, n_t, E, B, g.t_chunk, Gp)));
    RISRT_KERNEL(ctx, "k_adj_grad", (k_adj_grad<<<nblk((int64_t)B * M, 256), 256, 0, s>>>(Gp, g.bwd, phases, amp, B, M, grad)));
    return RISRT_OK;
}

}  // namespace risrt
