// Shapes shared by the sweep packing kernels and the tensor-core GEMM.
#pragma once

#include "internal.cuh"

namespace risrt {

constexpr int kTcBM = 128;   // receivers per tile (TMEM lanes)
constexpr int kTcBN = 256;   // real output columns per tile (128 configurations, re/im interleaved)
constexpr int kTcBK = 64;    // 16-bit elements per stage row (128 B, one swizzle atom)
constexpr int kTcStages = 4;

struct SweepShape {
    bool split;        // split-BF16: X carries hi and lo parts, K doubles
    int Kp;            // padded K (multiple of kTcBK)
    int Np;            // padded 2C (multiple of kTcBN)
    int64_t Mp;        // padded receiver count (multiple of kTcBM)
    size_t x_bytes, y_bytes;
};

SweepShape sweep_shape(int64_t n_rx, int M, int C, int precision);
size_t sweep_workspace_bytes(int64_t n_rx, int M, int C, int precision);
// Configurations as given: complex G [C][M], or 2-bit codes q (4 per byte, element m at bits 2 (m % 4) of
// byte m / 4 of row c, ceil(M/4) bytes per row) meaning Gamma = amp j^q.
struct GammaSrc {
    const float2* G = nullptr;
    const uint8_t* g2 = nullptr;
    float amp = 1.f;
    __device__ __forceinline__ float2 at(int64_t c, int m, int M) const
    {
        if (G) return G[c * M + m];
        const int q = (g2[c * ((M + 3) >> 2) + (m >> 2)] >> (2 * (m & 3))) & 3;
        return q == 0 ? make_float2(amp, 0.f) : q == 1 ? make_float2(0.f, amp) : q == 2 ? make_float2(-amp, 0.f)
                                                                                        : make_float2(0.f, -amp);
    }
};

int sweep_configs(risrt_ctx* ctx, const float2* A, const float2* E0, int64_t n_rx, int M, GammaSrc G, int C,
                  int precision, float* P, float2* Eout, void* ws, size_t ws_bytes, bool keep_a = false,
                  bool defer = false);
// Fused channel tile -> tensor-core sweep over a path set (A computed in shared memory, BF16): at most
// sweep_fused_max_configs() configurations; P and/or Eout receiver-major [n_rx][C]. Synchronises.
int sweep_fused(risrt_ctx* ctx, const risrt_pathset* ps, GammaSrc G, int C, float* P, float2* Eout);
int sweep_fused_max_configs();
// The deferred wait-timeout flag of the last sweep on this workspace (waits for the stream).
int sweep_check(risrt_ctx* ctx, const void* ws, size_t ws_bytes);
// D = X . Y^T on tcgen05 (X: [n_rx][Kp], Y: [Np][Kp], 16-bit, K-major), then
// P[r][c] = ((D[r][2c] + e0s Re E0[r])^2 + (D[r][2c+1] + e0s Im E0[r])^2) * pscale.
// With Eout (receiver-major [n_rx][C]) also E = (D + e0s E0) / e0s; P may then be NULL.
int sweep_tc(risrt_ctx* ctx, const void* X, const void* Y, const SweepShape& sh, bool fp16, const float2* E0,
             int64_t n_rx, int C, float* P, float pscale, float e0scale, unsigned* err_dev, bool defer = false,
             float2* Eout = nullptr);

// D = X . Y^T on SM pairs with split-K, complex partial sums out; enqueued only, the caller clears
// and reads err_dev (see sweep_tc.cu).
int gemm_tc_complex(risrt_ctx* ctx, const void* X, int64_t rows, const void* Y, int Np, int Kp, const float2* E0rows, int C,
                    float2* out, int splits, int* parts, unsigned* err_dev);

}  // namespace risrt
