// Strict per-element validation of reflected paths. The paper validates every face sequence once
// between the RIS centre and the Rx (and between the Tx and the RIS centre) and then applies it to
// every element (Sec. II-B); in strict mode each element's reflected legs are validated at the element
// itself. The Rx legs of element m are those of a one-element RIS centred exactly (FP64) at e_m, traced
// with the regular path search; its Tx legs are decided in FP64 per (element, sequence); the field is
//   E = E0 + sum_m Gamma_m K c_m^strict sum_{q valid for m} b_mq
// with E0 (LOS and environment paths) from one trace of the whole RIS.
#include <cmath>

#include "internal.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void k_e_init(const float2* __restrict__ E0, int64_t n_rx, int n_cfg, float2* __restrict__ E)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_rx * n_cfg) E[i] = E0[i % n_rx];
}

__global__ void k_power(const float2* __restrict__ E, int64_t n, float s, float* __restrict__ P)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 e = E[i];
        P[i] = (e.x * e.x + e.y * e.y) * s;
    }
}

}  // namespace

int eval_field_strict(risrt_ctx* ctx, const risrt_scene* sc, const risrt_ris* ris, const risrt_rxset* rxs, double freq,
                      int max_tx, int max_rx, uint32_t flags, const float2* gamma, int n_cfg, float2* E, float* P)
{
    cudaStream_t s = ctx->stream;
    const int M = ris->M;
    const int64_t n_rx = rxs->n;
    risrt_pathset* ps0 = new (std::nothrow) risrt_pathset();
    risrt_pathset* psm = new (std::nothrow) risrt_pathset();
    void* cmb = nullptr;
    void* elem1 = nullptr;
    int rc = RISRT_OK;
    if (!ps0 || !psm) rc = fail(ctx, RISRT_ERR_OOM, "host allocation failed");
    if (!rc) {
        ps0->owner = ctx;
        psm->owner = ctx;
        cudaError_t e = ctx_malloc(ctx, &cmb, sizeof(float2) * M);
        if (e == cudaSuccess) e = ctx_malloc(ctx, &elem1, sizeof(float4));
        if (e == cudaSuccess) e = cudaMemsetAsync(elem1, 0, sizeof(float4), s);   // one element at the centre
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "strict-mode buffers");
    }
    // E0 (LOS and environment paths) and E = E0 for every configuration
    if (!rc) rc = trace_paths(ctx, sc, ris, rxs, freq, 0, max_rx, flags, ps0);
    auto e_init = [&]() -> int {       // launch failures return here, so the clean-up below still runs
        RISRT_KERNEL(ctx, "k_e_init", (k_e_init<<<nblk(n_rx * n_cfg, 256), 256, 0, s>>>(ps0->E0, n_rx, n_cfg, E)));
        return RISRT_OK;
    };
    if (!rc) rc = e_init();
    // every element's K c_m with its own Tx-leg validity
    if (!rc) rc = strict_tx_cm(ctx, sc, ris, freq, max_tx, flags, (float2*)cmb);
    // every element's Rx legs: a one-element RIS centred exactly at the element
    if (!rc) {
        risrt_ris r1;
        r1.owner = ctx;
        r1.M = 1;
        for (int k = 0; k < 3; ++k) {
            r1.t1[k] = ris->t1[k];
            r1.t2[k] = ris->t2[k];
        }
        r1.dy = ris->dy;
        r1.dz = ris->dz;
        r1.elem_gain = ris->elem_gain;
        r1.host_face = ris->host_face;
        r1.elem = (float4*)elem1;
        r1.uv_host = {0.f, 0.f};
        r1.exact_center = true;
        for (int m = 0; m < M && !rc; ++m) {
            const double a = ris->uv_host[2 * m], b = ris->uv_host[2 * m + 1];
            for (int k = 0; k < 3; ++k) {
                r1.center_d[k] = (double)ris->center[k] + a * (double)ris->t1[k] + b * (double)ris->t2[k];
                r1.center[k] = (float)r1.center_d[k];
            }
            rc = trace_paths(ctx, sc, &r1, rxs, freq, 0, max_rx, flags & ~(uint32_t)RISRT_FLAG_ENV_PATHS, psm);
            if (rc) break;
            // the trace's c_m holds only the direct Tx leg: take the strict one
            cudaError_t e = cudaMemcpyAsync(psm->cm, (float2*)cmb + m, sizeof(float2), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) {
                rc = cuda_fail(ctx, e, "cudaMemcpyAsync(c_m)");
                break;
            }
            rc = eval_field_accum(ctx, psm, gamma + m, M, n_cfg, E);
        }
    }
    auto power = [&]() -> int {
        RISRT_KERNEL(ctx, "k_power", (k_power<<<nblk(n_rx * n_cfg, 256), 256, 0, s>>>(E, n_rx * n_cfg, (float)(1.0 / (2.0 * kEta0)), P)));
        return RISRT_OK;
    };
    if (!rc && P) rc = power();
    cudaStreamSynchronize(s);
    if (ps0) risrt_pathset_destroy(ctx, ps0);
    if (psm) risrt_pathset_destroy(ctx, psm);
    ctx_free(ctx, cmb);
    ctx_free(ctx, elem1);
    return rc;
}

}  // namespace risrt
