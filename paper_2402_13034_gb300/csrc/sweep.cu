// Configuration sweep (Eq. 9 is linear in Gamma, Eq. 10): for every receiver r and configuration c,
//   P[r][c] = |E0[r] + sum_m A[r][m] Gamma[c][m]|^2 / (2 eta0).
// FP32 SIMT path (complex GEMM on the CUDA cores) and the packing kernels of the tensor-core paths,
// which run the complex product as one real GEMM D = X . Y^T with
//   X = [Re A | Im A]                       (receivers x 2M, K-major)
//   Y[2c]   = [ Re G_c | -Im G_c ],  Y[2c+1] = [ Im G_c | Re G_c ]   (2C x 2M, K-major)
// so that D[r][2c] = Re E, D[r][2c+1] = Im E and the epilogue squares adjacent columns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"
#include "sweep.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------------------------------------
// FP32 SIMT complex GEMM with fused |E|^2 epilogue: 128 receivers x 64 configurations per block,
// K chunks of 16 elements staged in shared memory, 8 x 4 complex accumulators per thread.
// ------------------------------------------------------------------------------------------------
constexpr int kSB_R = 128, kSB_C = 64, kSB_K = 16;

__global__ void __launch_bounds__(256)
k_sweep_fp32(const float2* __restrict__ A, const float2* __restrict__ E0, int64_t n_rx, int M,
             GammaSrc G, int C, float* __restrict__ P, float scale, float2* __restrict__ Eout)
{
    __shared__ float2 sA[kSB_K][kSB_R + 1];
    __shared__ float2 sG[kSB_K][kSB_C + 1];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;           // 16 x 16 threads, 8 rows x 4 configs each
    const int64_t r0 = (int64_t)blockIdx.x * kSB_R;
    const int c0 = blockIdx.y * kSB_C;
    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < M; k0 += kSB_K) {
        // A tile: 128 x 16 complex (coalesced along k)
        for (int i = tid; i < kSB_R * kSB_K; i += 256) {
            const int rr = i / kSB_K, kk = i % kSB_K;
            const int64_t r = r0 + rr;
            const int k = k0 + kk;
            sA[kk][rr] = (r < n_rx && k < M) ? A[r * M + k] : make_float2(0.f, 0.f);
        }
        for (int i = tid; i < kSB_C * kSB_K; i += 256) {
            const int cc = i / kSB_K, kk = i % kSB_K;
            const int c = c0 + cc, k = k0 + kk;
            sG[kk][cc] = (c < C && k < M) ? G.at(c, k, M) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kSB_K; ++kk) {
            float2 a[8], g[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = sA[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j] = sG[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(a[i].x, g[j].x, fmaf(-a[i].y, g[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, g[j].y, fmaf(a[i].y, g[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + tr + 16 * i;
        if (r >= n_rx) continue;
        const float2 e0 = E0 ? E0[r] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tc + 16 * j;
            if (c >= C) continue;
            const float er = acc[i][j].x + e0.x, ei = acc[i][j].y + e0.y;
            if (P) P[r * C + c] = (er * er + ei * ei) * scale;
            if (Eout) Eout[r * C + c] = make_float2(er, ei);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// packing for the tensor-core paths
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T to_t(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_t<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_t<__half>(float v) { return __float2half_rn(v); }
template <typename T>
__device__ __forceinline__ float from_t(T v);
template <>
__device__ __forceinline__ float from_t<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float from_t<__half>(__half v) { return __half2float(v); }

// X rows (receivers) of length Kp: [Re A | Im A] (split: then [Re lo | Im lo] of the residual),
// scaled by `scale`, zero padded up to Kp.
template <typename T>
__global__ void k_pack_X(const float2* __restrict__ A, int64_t n_rx, int M, int Kp, bool split, float scale,
                         T* __restrict__ X)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = i / Kp;
    const int k = (int)(i % Kp);
    if (r >= n_rx) return;
    const int part = k / M, m = k % M;       // 0: Re hi, 1: Im hi, 2: Re lo, 3: Im lo
    float v = 0.f;
    if (k < (split ? 4 : 2) * M) {
        const float2 a = A[r * M + m];
        const float x = ((part & 1) ? a.y : a.x) * scale;
        const T hi = to_t<T>(x);
        v = part < 2 ? from_t<T>(hi) : x - from_t<T>(hi);
    }
    X[i] = to_t<T>(v);
}

// Y rows (2C + padding up to Np) of length Kp; the split layout repeats the 2M block for the residual.
template <typename T>
__global__ void k_pack_Y(GammaSrc G, int C, int M, int Np, int Kp, bool split, T* __restrict__ Y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int n = (int)(i / Kp);
    const int k = (int)(i % Kp);
    if (n >= Np) return;
    float v = 0.f;
    const int c = n >> 1;
    if (c < C && k < (split ? 4 : 2) * M) {
        const int kk = k % (2 * M);
        const int m = kk % M;
        const bool second = kk >= M;              // multiplies Im A
        const float2 g = G.at(c, m, M);
        if (!(n & 1)) v = second ? -g.y : g.x;   // Re E = Re A Re G - Im A Im G
        else v = second ? g.x : g.y;             // Im E = Re A Im G + Im A Re G
    }
    Y[i] = to_t<T>(v);
}

__global__ void k_absmax(const float2* __restrict__ A, int64_t n, unsigned* __restrict__ out)
{
    unsigned m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = A[i];
        m = max(m, __float_as_uint(fmaxf(fabsf(a.x), fabsf(a.y))));
    }
    atomicMax(out, m);
}

}  // namespace

SweepShape sweep_shape(int64_t n_rx, int M, int C, int precision)
{
    SweepShape s;
    s.split = precision == RISRT_PREC_BF16X2;
    s.Kp = (int)(((int64_t)(s.split ? 4 : 2) * M + kTcBK - 1) / kTcBK * kTcBK);
    s.Np = (int)(((int64_t)2 * C + kTcBN - 1) / kTcBN * kTcBN);
    s.Mp = (n_rx + kTcBM - 1) / kTcBM * kTcBM;
    s.x_bytes = (size_t)s.Mp * s.Kp * 2;
    s.y_bytes = (size_t)s.Np * s.Kp * 2;
    return s;
}

size_t sweep_workspace_bytes(int64_t n_rx, int M, int C, int precision)
{
    if (precision == RISRT_PREC_FP32) return 0;
    SweepShape s = sweep_shape(n_rx, M, C, precision);
    return s.x_bytes + s.y_bytes + 4096;
}

int sweep_configs(risrt_ctx* ctx, const float2* A, const float2* E0, int64_t n_rx, int M, GammaSrc G, int C,
                  int precision, float* P, float2* Eout, void* ws, size_t ws_bytes, bool keep_a, bool defer)
{
    cudaStream_t s = ctx->stream;
    const float inv2eta = (float)(1.0 / (2.0 * kEta0));
    if (precision == RISRT_PREC_FP32) {
        dim3 grid(nblk(n_rx, kSB_R), nblk(C, kSB_C));
        RISRT_KERNEL(ctx, "k_sweep_fp32", (k_sweep_fp32<<<grid, 256, 0, s>>>(A, E0, n_rx, M, G, C, P, inv2eta, Eout)));
        return RISRT_OK;
    }
    SweepShape sh = sweep_shape(n_rx, M, C, precision);
    if (ws_bytes < sh.x_bytes + sh.y_bytes + 4096 || !ws)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "workspace smaller than risrt_sweep_workspace_size");
    char* base = (char*)(((uintptr_t)ws + 1023) & ~(uintptr_t)1023);
    void* X = base;
    void* Y = base + ((sh.x_bytes + 1023) & ~(size_t)1023);
    unsigned* d_max = (unsigned*)((char*)ws + ws_bytes - 16);
    float xscale = 1.f;
    if (precision == RISRT_PREC_FP16) {
        // power-of-two scale that brings max |A| near 2^14 (FP16 keeps 11 bits over a wide range)
        RISRT_CUDA(ctx, cudaMemsetAsync(d_max, 0, sizeof(unsigned), s));
        RISRT_KERNEL(ctx, "k_absmax", (k_absmax<<<std::min<unsigned>(nblk(n_rx * M, 256), 2048u), 256, 0, s>>>(A, n_rx * M, d_max)));
        unsigned hm = 0;
        RISRT_CUDA(ctx, cudaMemcpyAsync(&hm, d_max, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        float amax;
        memcpy(&amax, &hm, 4);
        if (amax > 0.f) xscale = ldexpf(1.f, 14 - (int)ceilf(log2f(amax)));
    }
    const int64_t nx = (int64_t)sh.Mp * sh.Kp, ny = (int64_t)sh.Np * sh.Kp;
    if (precision == RISRT_PREC_FP16) {
        RISRT_KERNEL(ctx, "k_pack_X", (k_pack_X<__half><<<nblk(nx, 256), 256, 0, s>>>(A, n_rx, M, sh.Kp, false, xscale, (__half*)X)));
        RISRT_KERNEL(ctx, "k_pack_Y", (k_pack_Y<__half><<<nblk(ny, 256), 256, 0, s>>>(G, C, M, sh.Np, sh.Kp, false, (__half*)Y)));
    } else {
        if (!keep_a)   // with keep_a the workspace already holds A packed by an earlier call
            RISRT_KERNEL(ctx, "k_pack_X", (k_pack_X<__nv_bfloat16><<<nblk(nx, 256), 256, 0, s>>>(A, n_rx, M, sh.Kp, sh.split, 1.f,
                                                                                                (__nv_bfloat16*)X)));
        RISRT_KERNEL(ctx, "k_pack_Y", (k_pack_Y<__nv_bfloat16><<<nblk(ny, 256), 256, 0, s>>>(G, C, M, sh.Np, sh.Kp, sh.split,
                                                                                            (__nv_bfloat16*)Y)));
    }
    return sweep_tc(ctx, X, Y, sh, precision == RISRT_PREC_FP16, E0, n_rx, C, P, inv2eta / (xscale * xscale), xscale,
                    d_max + 1, defer, Eout);
}

int sweep_check(risrt_ctx* ctx, const void* ws, size_t ws_bytes)
{
    const unsigned* err_dev = (const unsigned*)((const char*)ws + ws_bytes - 16) + 1;   // as in sweep_configs
    unsigned h = 0;
    RISRT_CUDA(ctx, cudaMemcpyAsync(&h, err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    RISRT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return fail(ctx, RISRT_ERR_TIMEOUT, "tensor-core sweep: a pipeline wait expired");
    return RISRT_OK;
}

}  // namespace risrt
