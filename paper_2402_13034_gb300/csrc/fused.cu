// Fused channel tile -> tensor-core sweep (Eq. 9 is linear in Gamma, Eq. 10 on its result): the
// channel matrix A[r][m] = c_m sum_q b_mq(r) is computed tile by tile straight into shared memory and
// consumed there by tcgen05.mma; A never goes to HBM. One CTA per 128 receivers, one 256-column FP32
// accumulator in tensor memory (128 configurations, Re/Im interleaved):
//   warp 0      TMA producer of the configuration operand Y (128B-swizzled, 64 K columns per stage)
//   warp 1      allocates the accumulator; one thread issues tcgen05.mma (M = 128, N = 256, K = 16)
//   warps 2-31  A producers: per stage 32 elements of 128 receivers, one element per lane, a warp per
//               receiver row at a time (the row's path records broadcast to the warp; rows claimed
//               from a per-stage counter, so warps with short rows take more), BF16 values written in
//               the MMA's swizzled K-major layout; then warps 2-5 run the epilogue
//               (E = D + E0, P = |E|^2 / (2 eta0))
// K is ordered by blocks of 32 elements, [Re A | Im A] within a block, and Y's rows follow the same
// order: D[r][2c] = sum Re A Re G - Im A Im G = Re E_c, D[r][2c + 1] = sum Re A Im G + Im A Re G.
// Every mbarrier wait has a clock deadline; on expiry the kernel records an error and returns after
// draining its own copies and MMAs.
#include <cuda_bf16.h>

#include "rxleg.cuh"
#include "tc.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

#ifndef RISRT_FUSE_PROD
#define RISRT_FUSE_PROD 30
#endif
constexpr int kFuseProd = RISRT_FUSE_PROD;             // producer warps
constexpr int kFuseThreads = 64 + 32 * kFuseProd;
constexpr int kFuseStages = 4;
constexpr int kFStageA = kTcBM * kTcBK * 2;            // 16 KB: 128 rows x 64 BF16
constexpr int kFStageB = kTcBN * kTcBK * 2;            // 32 KB: 256 rows x 64 BF16
constexpr int kFuseSmem = kFuseStages * (kFStageA + kFStageB) + 1024 + 256;
constexpr int kFuseCfg = kTcBN / 2;                    // configurations per call
constexpr long long kFuseWait = 4000000000LL;          // ~2 s at 2 GHz

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// Byte offset of K column k (0..63) of row r in a 128B-swizzled K-major stage (rows 128 B apart, the
// 16-byte chunk index XORed with r mod 8), the layout a SWIZZLE_128B TMA load writes.
__device__ __forceinline__ uint32_t swz(int r, int k)
{
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

template <int PAT>
__global__ void __launch_bounds__(kFuseThreads, 1)
k_sweep_fused(const __grid_constant__ CUtensorMap tmY, int nkb, uint32_t idesc, const PathRec* __restrict__ rec,
              const int64_t* __restrict__ off, const uint32_t* __restrict__ vis, int W, const float4* __restrict__ elem,
              const float2* __restrict__ cm, int M, int64_t n_rx, const float2* __restrict__ E0, int C,
              float* __restrict__ P, float pscale, float2* __restrict__ Eout, float inv_lam, float gr, int tm,
              unsigned* __restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kFuseStages * kFStageA;
    uint64_t* full = (uint64_t*)(sB + kFuseStages * kFStageB);
    uint64_t* empty = full + kFuseStages;
    uint64_t* tfull = empty + kFuseStages;
    uint32_t* tmem_slot = (uint32_t*)(tfull + 1);
    __shared__ int abort_flag;
    __shared__ unsigned row_ctr[kFuseStages];   // rows claimed from each stage over all its uses

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * kTcBM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFuseStages; ++s) {
            row_ctr[s] = 0;
            mbar_init(smem_u32(&full[s]), 1 + kFuseProd);   // the TMA's arrive.expect_tx + one per producer warp
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(tfull), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long deadline = clock64() + kFuseWait;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer of Y
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kFuseStages;
                if (!mbar_wait(smem_u32(&empty[s]), ((kb / kFuseStages) & 1) ^ 1, deadline) ||
                    *(volatile int*)&abort_flag) {
                    atomicExch(err, 1u);
                    *(volatile int*)&abort_flag = 1;
                    break;
                }
                mbar_expect_tx(smem_u32(&full[s]), kFStageB);
                tma_load_2d(smem_u32(sB + s * kFStageB), &tmY, smem_u32(&full[s]), kb * kTcBK, 0);
                ++issued;
            }
            if (*(volatile int*)&abort_flag) {   // let this CTA's copies land before the shared memory is released
                const long long d2 = clock64() + kFuseWait;
                for (int kb = (issued > kFuseStages ? issued - kFuseStages : 0); kb < issued; ++kb)
                    mbar_wait(smem_u32(&full[kb % kFuseStages]), (kb / kFuseStages) & 1, d2);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kFuseStages;
                if (!mbar_wait(smem_u32(&full[s]), (kb / kFuseStages) & 1, deadline) || *(volatile int*)&abort_flag) {
                    atomicExch(err, 1u);
                    *(volatile int*)&abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t a0 = smem_u32(sA + s * kFStageA), b0 = smem_u32(sB + s * kFStageB);
#pragma unroll
                for (int k = 0; k < kTcBK / 16; ++k)
                    mma_f16(tmem, smem_desc(a0 + k * 32), smem_desc(b0 + k * 32), idesc, (kb | k) != 0);
                mma_commit(smem_u32(&empty[s]));   // frees the stage once these MMAs have read it
            }
            mma_commit(smem_u32(tfull));           // accumulator complete (or issued work drained)
        }
    } else {   // A producers (warps 2 and up), then the epilogue (warps 2..5)
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kFuseStages;
            bool ok = true;
            if (lane == 0)
                ok = mbar_wait(smem_u32(&empty[s]), ((kb / kFuseStages) & 1) ^ 1, deadline) &&
                     !*(volatile int*)&abort_flag;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(err, 1u);
                    *(volatile int*)&abort_flag = 1;
                }
                break;
            }
            const int m = kb * 32 + lane;
            const bool valid = m < M;
            const float4 e = valid ? elem[m] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float2 c2 = valid ? cm[m] : make_float2(0.f, 0.f);
            uint8_t* stage = sA + s * kFStageA;
            // every warp claims rows until one past the last: kTcBM + kFuseProd claims per use of a stage
            const unsigned base = (unsigned)(kb / kFuseStages) * (kTcBM + kFuseProd);
            while (true) {
                unsigned claim = 0;
                if (lane == 0) claim = atomicAdd(&row_ctr[s], 1u);
                const int rr = (int)(__shfl_sync(0xffffffffu, claim, 0) - base);
                if (rr >= kTcBM) break;
                const int64_t row = m0 + rr;
                cf a = cf{0.f, 0.f};
                if (row < n_rx) {
                    const int64_t o = off[row];
                    const int nq = (int)(off[row + 1] - o);
                    const bool direct = valid && ((vis[row * W + kb] >> lane) & 1u);
                    cf acc = cf{0.f, 0.f};
                    for (int q = 0; q < nq; ++q) {
                        const PathRec p = rec[o + q];
                        if (!valid || (q == 0 && !direct)) continue;   // entry 0 is the direct path
                        const cf b = rx_leg_term<PAT>(p, e, inv_lam, gr, tm != 0);
                        acc.re += b.re;
                        acc.im += b.im;
                    }
                    if (valid) a = cmulf(acc, cf{c2.x, c2.y});
                }
                *(__nv_bfloat16*)(stage + swz(rr, lane)) = __float2bfloat16_rn(a.re);
                *(__nv_bfloat16*)(stage + swz(rr, 32 + lane)) = __float2bfloat16_rn(a.im);
            }
            // make the generic-proxy writes visible to the tensor core's (async-proxy) reads, then arrive
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full[s]));
        }
        if (warp < 6) {   // then the epilogue, warps 2..5: TMEM lanes 32*(warp%4) .. +31
            const bool ok = mbar_wait(smem_u32(tfull), 0, deadline + kFuseWait);
            if (!ok) {
                atomicExch(err, 1u);
                *(volatile int*)&abort_flag = 1;
            }
            fence_after();
            const int lane_base = 32 * (warp & 3);
            const int64_t row = m0 + lane_base + lane;
            const bool live = ok && !*(volatile int*)&abort_flag && row < n_rx;
            const float2 e0 = live ? E0[row] : make_float2(0.f, 0.f);
            for (int j = 0; j < kTcBN / 16; ++j) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(j * 16), v);
                if (!live) continue;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int c = j * 8 + q;
                    if (c < C) {
                        const float er = v[2 * q] + e0.x, ei = v[2 * q + 1] + e0.y;
                        if (P) P[row * C + c] = (er * er + ei * ei) * pscale;
                        if (Eout) Eout[row * C + c] = make_float2(er, ei);
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcBN) : "memory");
    }
}

// Y [256][Kp] BF16 in the fused K order (block j: elements 32j..32j+31, Re then Im columns): rows 2c and
// 2c + 1 give Re and Im of E_c; rows past 2C and columns of elements past M stay zero (cleared first).
__global__ void k_pack_y_fused(GammaSrc G, int C, int M, int Kp, __nv_bfloat16* __restrict__ Y)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (m >= M || c >= C) return;
    const float2 g = G.at(c, m, M);
    const int k = (m >> 5) * 64 + (m & 31);
    __nv_bfloat16* re = Y + (int64_t)(2 * c) * Kp;
    __nv_bfloat16* im = re + Kp;
    re[k] = __float2bfloat16_rn(g.x);
    re[k + 32] = __float2bfloat16_rn(-g.y);
    im[k] = __float2bfloat16_rn(g.y);
    im[k + 32] = __float2bfloat16_rn(g.x);
}

}  // namespace

int sweep_fused(risrt_ctx* ctx, const risrt_pathset* ps, GammaSrc G, int C, float* P, float2* Eout)
{
    cudaStream_t s = ctx->stream;
    const int M = ps->M;
    const int nkb = (M + 31) / 32;
    const int Kp = nkb * kTcBK;
    const size_t ybytes = (size_t)kTcBN * Kp * 2;
    void* blk = nullptr;
    RISRT_CUDA(ctx, ctx_malloc(ctx, &blk, ybytes + 256));
    __nv_bfloat16* Y = (__nv_bfloat16*)blk;
    unsigned* err = (unsigned*)((char*)blk + ybytes);
    auto body = [&]() -> int {
        RISRT_CUDA(ctx, cudaMemsetAsync(blk, 0, ybytes + 256, s));   // Y's unused rows and columns, the error flag
        RISRT_KERNEL(ctx, "k_pack_y_fused", (k_pack_y_fused<<<dim3(nblk(M, 256), C), 256, 0, s>>>(G, C, M, Kp, Y)));
        CUtensorMap mY;
        if (!make_map(&mY, Y, false, kTcBN, Kp, kTcBN)) return fail(ctx, RISRT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        const uint32_t idesc = make_idesc(false, kTcBM, kTcBN);
        const float inv_lam = (float)(ps->freq / kC0);
        const int tm = (ps->flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
        const float pscale = (float)(1.0 / (2.0 * kEta0));
        const unsigned grid = nblk(ps->n_rx, kTcBM);
        auto launch = [&](auto kern) -> int {
            const cudaError_t ae = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kFuseSmem);
            if (ae != cudaSuccess) return cuda_fail(ctx, ae, "cudaFuncSetAttribute(k_sweep_fused)");
            RISRT_KERNEL(ctx, "k_sweep_fused", (kern<<<grid, kFuseThreads, kFuseSmem, s>>>(
                                                   mY, nkb, idesc, ps->rec, ps->rx_off, ps->vis, ps->W, ps->elem, ps->cm, M,
                                                   ps->n_rx, ps->E0, C, P, pscale, Eout, inv_lam, ps->rx_gain, tm, err)));
            return RISRT_OK;
        };
        int rc;
        switch (ps->rx_pattern) {
            case RISRT_PATTERN_COS_POW: rc = launch(k_sweep_fused<RISRT_PATTERN_COS_POW>); break;
            case RISRT_PATTERN_MONOPOLE_QW: rc = launch(k_sweep_fused<RISRT_PATTERN_MONOPOLE_QW>); break;
            default: rc = launch(k_sweep_fused<RISRT_PATTERN_ISO>); break;
        }
        if (rc) return rc;
        unsigned h = 0;
        RISRT_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        if (h) return fail(ctx, RISRT_ERR_TIMEOUT, "fused sweep: a pipeline wait expired");
        return RISRT_OK;
    };
    const int rc = body();
    ctx_free(ctx, blk);
    return rc;
}

int sweep_fused_max_configs() { return kFuseCfg; }

}  // namespace risrt
