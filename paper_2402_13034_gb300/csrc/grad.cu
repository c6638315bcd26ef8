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
// Fixed-order reductions (block tree) keep J deterministic.
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
        acc += log((double)p * (double)inv_2eta0);
        e[t] = make_float2(v.x / p, -v.y / p);      // w = conj(E) / |E|^2 (E is overwritten)
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) J[b] = (float)red[0];
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

// ---- tensor-core path: both GEMMs as real BF16 GEMMs with three-term splits ----------------------
// A complex product is one real GEMM over [Re | Im] blocks (rows of the second operand interleave
// [Re g, -Im g] and [Im g, Re g]); each real factor x is split as hi = bf16(x), lo = bf16(x - hi),
// and the reduction runs over three blocks pairing hi.hi, hi.lo and lo.hi (the lo.lo term, below
// 2^-16 of the product, is dropped), which keeps the products to about 1e-5 relative.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Forward operand X [n_t][Kf]: row t holds [hi(Re A), hi(Im A) | hi(Re A), hi(Im A) | lo(Re A), lo(Im A)]
// of A's target row (columns past 6M zero); E0t[t] = E0 of that row.
__global__ void k_gpack_xf(const float2* __restrict__ A, const float2* __restrict__ E0, int M, const int* __restrict__ target,
                           int n_t, int Kf, __nv_bfloat16* __restrict__ X, float2* __restrict__ E0t)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int wide = max(2 * M, Kf - 6 * M);
    if (i >= (int64_t)n_t * wide) return;
    const int t = (int)(i / wide), k2 = (int)(i % wide);
    const int64_t r = target ? target[t] : t;
    __nv_bfloat16* row = X + (int64_t)t * Kf;
    if (k2 < 2 * M) {
        const float2 a = A[r * M + (k2 % M)];
        __nv_bfloat16 hi, lo;
        split_bf16(k2 < M ? a.x : a.y, hi, lo);
        row[k2] = hi;
        row[2 * M + k2] = hi;
        row[4 * M + k2] = lo;
        if (k2 == 0) E0t[t] = E0 ? E0[r] : make_float2(0.f, 0.f);
    }
    if (k2 < Kf - 6 * M) row[6 * M + k2] = __float2bfloat16_rn(0.f);
}

// Forward operand Y [Np][Kf] from Gamma_bm = amp_m e^{j phi_bm}: rows 2b / 2b + 1 give Re / Im E_b.
__global__ void k_gpack_yf(const float* __restrict__ phases, const float* __restrict__ amp, int M, int B, int Np, int Kf,
                           __nv_bfloat16* __restrict__ Y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)Np * Kf) return;
    const int n = (int)(i / Kf), k = (int)(i % Kf);
    const int b = n >> 1, seg = k / (2 * M), k2 = k % (2 * M), part = k2 / M, m = k2 % M;
    float v = 0.f;
    bool use_lo = false;
    if (b < B && seg < 3) {
        float sn, cs;
        sincosf(phases[(int64_t)b * M + m], &sn, &cs);
        const float a = amp ? amp[m] : 1.f;
        const float gre = a * cs, gim = a * sn;
        // Re E = sum Re A Re g - Im A Im g;  Im E = sum Re A Im g + Im A Re g
        v = (n & 1) ? (part == 0 ? gim : gre) : (part == 0 ? gre : -gim);
        use_lo = seg == 1;
    }
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    Y[i] = use_lo ? lo : hi;
}

// Backward operand X [M][Kb] (A transposed): row m holds, for segments hi, hi, lo, [Re A[t][m] | Im A[t][m]]
// over the targets t (columns past 6 n_t zero). 32 x 32 tiles through shared memory.
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
        row[2 * n_t + t] = rh;
        row[3 * n_t + t] = ih;
        row[4 * n_t + t] = rl;
        row[5 * n_t + t] = il;
    }
}

__global__ void k_gpack_xb_pad(int M, int n_t, int Kb, __nv_bfloat16* __restrict__ X)
{
    const int pad = Kb - 6 * n_t;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pad <= 0 || i >= (int64_t)M * pad) return;
    X[(i / pad) * Kb + 6 * n_t + i % pad] = __float2bfloat16_rn(0.f);
}

// Backward operand Y [Np][Kb] from the weights w[b][t]: rows 2b / 2b + 1 give Re / Im of sum_t A w.
__global__ void k_gpack_yb(const float2* __restrict__ W, int n_t, int B, int Np, int Kb, __nv_bfloat16* __restrict__ Y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)Np * Kb) return;
    const int n = (int)(i / Kb), k = (int)(i % Kb);
    const int b = n >> 1, seg = k / (2 * n_t), k2 = k % (2 * n_t), part = k2 / n_t, t = k2 % n_t;
    float v = 0.f;
    bool use_lo = false;
    if (b < B && seg < 3) {
        const float2 w = W[(int64_t)b * n_t + t];
        v = (n & 1) ? (part == 0 ? w.y : w.x) : (part == 0 ? w.x : -w.y);
        use_lo = seg == 1;
    }
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    Y[i] = use_lo ? lo : hi;
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

// Layout of the tensor-core workspace (byte offsets, 256-aligned) and its split-K part counts.
struct GradTcLayout {
    int Kf, Kb, Np, sf, sb;
    size_t xf, yf, e0t, ep, xb, yb, gp, end;
};

GradTcLayout grad_tc_layout(int n_t, int B, int M)
{
    GradTcLayout L;
    auto up = [](int64_t v, int64_t a) { return (v + a - 1) / a * a; };
    L.Kf = (int)up(6LL * M, kTcBK);
    L.Kb = (int)up(6LL * n_t, kTcBK);
    L.Np = (int)up(2LL * B, kTcBN);
    const int clusters = 152;           // enough parts to give every SM pair about one tile
    const int tf = (int)(up(n_t, 2 * kTcBM) / (2 * kTcBM)) * (L.Np / kTcBN);
    const int tb = (int)(up(M, 2 * kTcBM) / (2 * kTcBM)) * (L.Np / kTcBN);
    L.sf = std::max(1, std::min(8, (clusters + tf - 1) / tf));
    L.sb = std::max(1, std::min(16, (clusters + tb - 1) / tb));
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t a = o;
        o = (size_t)up((int64_t)(o + bytes), 256);
        return a;
    };
    L.xf = take((size_t)n_t * L.Kf * 2);
    L.yf = take((size_t)L.Np * L.Kf * 2);
    L.e0t = take((size_t)n_t * sizeof(float2));
    L.ep = take((size_t)L.sf * B * n_t * sizeof(float2));
    L.xb = take((size_t)M * L.Kb * 2);
    L.yb = take((size_t)L.Np * L.Kb * 2);
    L.gp = take((size_t)L.sb * B * M * sizeof(float2));
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
// transposed operands done per call (A and the targets may change between calls).
static int grad_phases_tc(risrt_ctx* ctx, const float2* A, const float2* E0, int M, const int* target, int n_t,
                          const float* phases, const float* amp, int B, float* J, float* grad, void* ws, size_t ws_bytes,
                          bool keep_a)
{
    cudaStream_t s = ctx->stream;
    const GradTcLayout L = grad_tc_layout(n_t, B, M);
    char* w = (char*)ws;
    __nv_bfloat16* Xf = (__nv_bfloat16*)(w + L.xf);
    __nv_bfloat16* Yf = (__nv_bfloat16*)(w + L.yf);
    float2* E0t = (float2*)(w + L.e0t);
    float2* Ep = (float2*)(w + L.ep);
    __nv_bfloat16* Xb = (__nv_bfloat16*)(w + L.xb);
    __nv_bfloat16* Yb = (__nv_bfloat16*)(w + L.yb);
    float2* Gp = (float2*)(w + L.gp);
    unsigned* err = (unsigned*)(w + ws_bytes - 32);
    const int wide = std::max(2 * M, L.Kf - 6 * M);
    if (!keep_a) {              // A's target rows into both operands (kept in the workspace for KEEP_A calls)
        RISRT_KERNEL(ctx, "k_gpack_xf", (k_gpack_xf<<<nblk((int64_t)n_t * wide, 256), 256, 0, s>>>(A, E0, M, target, n_t, L.Kf, Xf, E0t)));
        RISRT_KERNEL(ctx, "k_gpack_xb", (k_gpack_xb<<<dim3(nblk(M, 32), nblk(n_t, 32)), dim3(32, 8), 0, s>>>(A, M, target, n_t, L.Kb, Xb)));
        if (L.Kb > 6 * n_t)
            RISRT_KERNEL(ctx, "k_gpack_xb_pad", (k_gpack_xb_pad<<<nblk((int64_t)M * (L.Kb - 6 * n_t), 256), 256, 0, s>>>(M, n_t, L.Kb, Xb)));
    }
    RISRT_KERNEL(ctx, "k_gpack_yf", (k_gpack_yf<<<nblk((int64_t)L.Np * L.Kf, 256), 256, 0, s>>>(phases, amp, M, B, L.Np, L.Kf, Yf)));
    int pf = 0, pb = 0, rc;
    if ((rc = gemm_tc_complex(ctx, Xf, n_t, Yf, L.Np, L.Kf, E0t, B, Ep, L.sf, &pf, err))) return rc;
    RISRT_KERNEL(ctx, "k_adj_weights", (k_adj_weights<<<B, 512, 0, s>>>(Ep, n_t, B, pf, J, (float)(1.0 / (2.0 * kEta0)))));
    RISRT_KERNEL(ctx, "k_gpack_yb", (k_gpack_yb<<<nblk((int64_t)L.Np * L.Kb, 256), 256, 0, s>>>(Ep, n_t, B, L.Np, L.Kb, Yb)));
    if ((rc = gemm_tc_complex(ctx, Xb, M, Yb, L.Np, L.Kb, nullptr, B, Gp, L.sb, &pb, err))) return rc;
    RISRT_KERNEL(ctx, "k_adj_grad", (k_adj_grad<<<nblk((int64_t)B * M, 256), 256, 0, s>>>(Gp, pb, phases, amp, B, M, grad)));
    return RISRT_OK;
}

int grad_phases(risrt_ctx* ctx, const float2* A, const float2* E0, int M, const int* target, int n_t,
                const float* phases, const float* amp, int B, float* J, float* grad, void* ws, size_t ws_bytes,
                int precision, bool keep_a)
{
    if (precision == RISRT_PREC_BF16X2)
        return grad_phases_tc(ctx, A, E0, M, target, n_t, phases, amp, B, J, grad, ws, ws_bytes, keep_a);
    cudaStream_t s = ctx->stream;
    const GradSplits g = grad_splits(n_t, B, M);
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
