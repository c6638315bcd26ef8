// Issue-rate microbenchmarks of the pipes the field kernels use: FP32 fused multiply-add, the
// special-function unit (sine, cosine, reciprocal square root, reciprocal, square root, base-2
// exponential, each as the single-instruction approximation) and FP64 fused multiply-add. They give
// the measured denominators of the field kernels' roofline (min over pipes of peak / ops per unit).
//
// Each thread runs kChains independent dependency chains, so the pipe, not the latency of one
// chain, bounds the rate; every block size and grid is a whole number of resident blocks per SM.
#include "internal.cuh"

namespace risrt {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;      // 2048 resident threads per SM

__device__ __forceinline__ float mufu(int kind, float x)
{
    float y;
    switch (kind) {
        case RISRT_MB_MUFU_SIN: asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
        case RISRT_MB_MUFU_COS: asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
        case RISRT_MB_MUFU_RSQ: asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
        case RISRT_MB_MUFU_RCP: asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
        case RISRT_MB_MUFU_SQRT: asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
        default: asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    }
    return y;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float* __restrict__ out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak_mufu(float* __restrict__ out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 0.25f + (float)(threadIdx.x + k) * 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            x[k] = mufu(KIND, x[k]);
            // a reciprocal of a reciprocal may be folded away; an add (on the FP32 pipe) keeps the chain
            if (KIND == RISRT_MB_MUFU_RCP) x[k] += 0.5f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(double* __restrict__ out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int microbench(risrt_ctx* ctx, int kind, int iters, double* ops_per_s, double* ms_out)
{
    const unsigned blocks = (unsigned)ctx->sm_count * kPeakBlocksPerSm;
    const size_t n_threads = (size_t)blocks * kPeakThreads;
    void* buf = nullptr;
    RISRT_CUDA(ctx, ctx_malloc(ctx, &buf, n_threads * sizeof(double)));
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = RISRT_OK;
    auto launch = [&]() -> int {
        cudaStream_t s = ctx->stream;
        switch (kind) {
            case RISRT_MB_FFMA:
                RISRT_KERNEL(ctx, "k_peak_ffma", (k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>((float*)buf, iters, 0.999f, 1e-3f)));
                break;
#define RISRT_MB_CASE(K)                                                                                         \
    case K: RISRT_KERNEL(ctx, "k_peak_mufu", (k_peak_mufu<K><<<blocks, kPeakThreads, 0, s>>>((float*)buf, iters))); break;
            RISRT_MB_CASE(RISRT_MB_MUFU_SIN)
            RISRT_MB_CASE(RISRT_MB_MUFU_COS)
            RISRT_MB_CASE(RISRT_MB_MUFU_RSQ)
            RISRT_MB_CASE(RISRT_MB_MUFU_RCP)
            RISRT_MB_CASE(RISRT_MB_MUFU_SQRT)
            RISRT_MB_CASE(RISRT_MB_MUFU_EX2)
#undef RISRT_MB_CASE
            case RISRT_MB_DFMA:
                RISRT_KERNEL(ctx, "k_peak_dfma", (k_peak_dfma<<<blocks, kPeakThreads, 0, s>>>((double*)buf, iters, 0.999, 1e-3)));
                break;
            default: return fail(ctx, RISRT_ERR_INVALID_ARG, "unknown microbenchmark");
        }
        return RISRT_OK;
    };
    double best = 1e30;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = fail(ctx, RISRT_ERR_CUDA, "cudaEventCreate failed");
    } else if (!(rc = launch())) {                       // warm-up launch
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            cudaEventRecord(a, ctx->stream);
            rc = launch();
            cudaEventRecord(b, ctx->stream);
            if (!rc && cudaEventSynchronize(b) == cudaSuccess) {
                float t = 0.f;
                cudaEventElapsedTime(&t, a, b);
                best = std::min(best, (double)t);
            }
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaStreamSynchronize(ctx->stream);
    ctx_free(ctx, buf);
    if (rc) return rc;
    const double ops = (double)n_threads * (double)iters * kChains;
    *ops_per_s = ops / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return RISRT_OK;
}

}  // namespace risrt
