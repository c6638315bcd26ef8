// Tensor-core sweep GEMM for sm_103a: D = X . Y^T with X [receivers][K], Y [2C][K] in BF16 or FP16
// (both K-major), FP32 accumulation in tensor memory, and the |E|^2 / (2 eta0) epilogue fused.
//
// One CTA computes a 128 x 256 tile (128 receivers x 128 configurations):
//   warp 0     TMA producer: 128B-swizzled X and Y tiles of 64 K elements into a 4-stage ring
//   warp 1     allocates 256 TMEM columns; one thread issues tcgen05.mma (M=128, N=256, K=16)
//   warps 2-5  epilogue: tcgen05.ld of their 32 TMEM lanes, square re/im pairs, store P
// Every mbarrier wait has a clock deadline; on expiry the kernel records an error, waits (again
// bounded) for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "sweep.cuh"
#include "tc.cuh"

namespace risrt {
namespace {

constexpr int kStageA = kTcBM * kTcBK * 2;   // 16 KB
constexpr int kStageB = kTcBN * kTcBK * 2;   // 32 KB
constexpr int kTmemCols = kTcBN;             // FP32 accumulator, one column per output column
constexpr int kSmemBytes = kTcStages * (kStageA + kStageB) + 1024 + 256;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__global__ void __launch_bounds__(192, 1)
k_sweep_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int num_kb, uint32_t idesc,
           const float2* __restrict__ E0, int64_t n_rx, int C, float* __restrict__ P, float pscale, float e0scale,
           unsigned* __restrict__ err, float2* __restrict__ Eout, float escale)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kTcStages * kStageA;
    uint64_t* full = (uint64_t*)(sB + kTcStages * kStageB);
    uint64_t* empty = full + kTcStages;
    uint64_t* tfull = empty + kTcStages;
    uint32_t* tmem_slot = (uint32_t*)(tfull + 1);
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * kTcBM;
    const int n0 = blockIdx.y * kTcBN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(tfull), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long deadline = clock64() + kWaitCycles;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            int issued = 0;
            for (int kb = 0; kb < num_kb; ++kb) {
                const int s = kb % kTcStages;
                const uint32_t ph = (kb / kTcStages) & 1;
                if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, deadline) || *(volatile int*)&abort_flag) {
                    atomicExch(err, 1u);
                    *(volatile int*)&abort_flag = 1;
                    break;
                }
                mbar_expect_tx(smem_u32(&full[s]), kStageA + kStageB);
                tma_load_2d(smem_u32(sA + s * kStageA), &tmX, smem_u32(&full[s]), kb * kTcBK, (int)m0);
                tma_load_2d(smem_u32(sB + s * kStageB), &tmY, smem_u32(&full[s]), kb * kTcBK, n0);
                ++issued;
            }
            if (*(volatile int*)&abort_flag) {   // let this CTA's own copies land before the shared memory is released
                const long long d2 = clock64() + kWaitCycles;
                for (int kb = (issued > kTcStages ? issued - kTcStages : 0); kb < issued; ++kb)
                    mbar_wait(smem_u32(&full[kb % kTcStages]), (kb / kTcStages) & 1, d2);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            bool ok = true;
            for (int kb = 0; kb < num_kb && ok; ++kb) {
                const int s = kb % kTcStages;
                if (!mbar_wait(smem_u32(&full[s]), (kb / kTcStages) & 1, deadline) || *(volatile int*)&abort_flag) {
                    atomicExch(err, 1u);
                    *(volatile int*)&abort_flag = 1;
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t a0 = smem_u32(sA + s * kStageA), b0 = smem_u32(sB + s * kStageB);
#pragma unroll
                for (int k = 0; k < kTcBK / 16; ++k)
                    mma_f16(tmem, smem_desc(a0 + k * 32), smem_desc(b0 + k * 32), idesc, (kb | k) != 0);
                mma_commit(smem_u32(&empty[s]));   // frees the stage once these MMAs have read it
            }
            mma_commit(smem_u32(tfull));           // accumulator complete (or issued work drained)
        }
    } else {   // epilogue warps 2..5: TMEM lanes 32*(warp%4) .. +31
        const bool ok = mbar_wait(smem_u32(tfull), 0, deadline + kWaitCycles);
        if (!ok) {
            atomicExch(err, 1u);
            *(volatile int*)&abort_flag = 1;
        }
        fence_after();
        const int lane_base = 32 * (warp & 3);
        const int64_t row = m0 + lane_base + lane;
        const bool live = ok && !*(volatile int*)&abort_flag && row < n_rx;
        float2 e0 = make_float2(0.f, 0.f);
        if (live && E0) {
            e0 = E0[row];
            e0.x *= e0scale;
            e0.y *= e0scale;
        }
        for (int j = 0; j < kTcBN / 16; ++j) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(j * 16), v);
            if (!live) continue;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = (n0 >> 1) + j * 8 + q;
                if (c < C) {
                    const float er = v[2 * q] + e0.x, ei = v[2 * q + 1] + e0.y;
                    if (P) P[row * C + c] = (er * er + ei * ei) * pscale;
                    if (Eout) Eout[row * C + c] = make_float2(er * escale, ei * escale);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---- Persistent pair kernel (cta_group::2) ---------------------------------------------------------
// Two CTAs of a cluster share one 256 x 256 tile: each stages its own 128 receiver rows of X and one
// half (128 rows) of the Y tile, the even CTA issues tcgen05.mma with M = 256 reading both CTAs'
// shared memory, and each CTA's tensor memory receives its 128 rows. Per k-block the pair moves 64 KB
// for 8.4 MFLOP (128 flop/B), against 48 KB for 4.2 MFLOP (85 flop/B) with one CTA per 128 x 256 tile.
// Clusters loop over tiles (receiver-block major); two 256-column accumulators let the epilogue of
// one tile run under the main loop of the next.
constexpr int kPairStages = 6;
constexpr int kPairStageB = (kTcBN / 2) * kTcBK * 2;   // 16 KB: this CTA's half of the Y tile
constexpr int kPairSmemBytes = kPairStages * (kStageA + kPairStageB) + 1024 + 256;
constexpr long long kPairWait = 2000000000LL;         // per wait, ~1 s at 2 GHz

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Remote (or local) arrive on an mbarrier addressed in the cluster window.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool wait_for(uint32_t a, uint32_t parity, bool cluster_scope)
{
    const long long until = clock64() + kPairWait;
    for (;;) {
        if (cluster_scope ? mbar_try_cluster(a, parity) : mbar_try(a, parity)) return true;
        if (clock64() > until) return false;
    }
}
// TMA load into this CTA's shared memory that signals an mbarrier of either CTA of the pair.
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t mbar_cluster, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(mbar_cluster), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void mma_f16_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on the mbarrier at the same offset in both CTAs of the pair once the issued MMAs complete.
__device__ __forceinline__ void mma_commit_pair(uint32_t mbar)
{
    const uint16_t mask = 0x3;
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(mbar),
                 "h"(mask)
                 : "memory");
}

__global__ void __launch_bounds__(192, 1)
k_sweep_tc_pair(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int num_kb, int tiles_n,
                int num_tiles, uint32_t idesc, const float2* __restrict__ E0, int64_t n_rx, int C,
                float* __restrict__ P, float pscale, float e0scale, unsigned* __restrict__ err, int num_kb_total,
                float2* __restrict__ Cout, float2* __restrict__ Eout, float escale)
{
    // split-K (num_kb k-blocks per split, num_kb_total in all): tile t covers split z = t / tiles_mn;
    // with Cout the epilogue writes the complex partial sums D[row][2c] + j D[row][2c + 1] (+ E0 in
    // split 0) to Cout[(z C + c) n_rx + row] instead of the power
    const int tiles_mn = num_tiles / max(1, (num_kb_total + num_kb - 1) / num_kb);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kPairStages * kStageA;
    uint64_t* full = (uint64_t*)(sB + kPairStages * kPairStageB);   // used in the even CTA only
    uint64_t* empty = full + kPairStages;
    uint64_t* tfull = empty + kPairStages;    // [2] accumulator ready (both CTAs)
    uint64_t* tempty = tfull + 2;             // [2] accumulator drained by all 8 epilogue warps (even CTA)
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    __shared__ int abort_flag;
    volatile int* abort_v = &abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();     // 0: issues the MMAs, 1: peer
    int cluster, n_clusters;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cluster));
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(n_clusters));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPairStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), 8);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // both CTAs allocate together: 2 x 256 accumulator columns
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    cluster_sync_all();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer (both CTAs)
            long long g = 0;
            bool ok = true;
            for (int t = cluster; t < num_tiles && ok; t += n_clusters) {
                const int tt = t % tiles_mn, kb0 = (t / tiles_mn) * num_kb, kb1 = min(num_kb_total, kb0 + num_kb);
                const int xrow = (tt / tiles_n) * (2 * kTcBM) + (int)rank * kTcBM;
                const int yrow = (tt % tiles_n) * kTcBN + (int)rank * (kTcBN / 2);
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int s = (int)(g % kPairStages);
                    const uint32_t ph = (uint32_t)((g / kPairStages) & 1);
                    if (!wait_for(smem_u32(&empty[s]), ph ^ 1, false) || *abort_v) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_expect_tx(smem_u32(&full[s]), 2 * (kStageA + kPairStageB));
                    const uint32_t fb = map_to_rank(smem_u32(&full[s]), 0);   // even CTA's barrier
                    tma_load_2d_pair(smem_u32(sA + s * kStageA), &tmX, fb, kb * kTcBK, xrow);
                    tma_load_2d_pair(smem_u32(sB + s * kPairStageB), &tmY, fb, kb * kTcBK, yrow);
                }
            }
            if (!ok) {
                atomicExch(err, 1u);
                *abort_v = 1;
            }
            // Every stage released: all MMA-completion arrivals aimed at this CTA have landed.
            for (long long q = g; q < g + kPairStages; ++q)
                if (!wait_for(smem_u32(&empty[q % kPairStages]), (uint32_t)(((q / kPairStages) & 1) ^ 1), false)) {
                    atomicExch(err, 1u);
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {   // MMA issuer
            long long g = 0;
            int i = 0;
            bool ok = true;
            for (int t = cluster; t < num_tiles && ok; t += n_clusters, ++i) {
                const int acc = i & 1;
                if (!wait_for(smem_u32(&tempty[acc]), (uint32_t)(((i >> 1) & 1) ^ 1), true) || *abort_v) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * kTmemCols);
                const int kb0 = (t / tiles_mn) * num_kb, kb1 = min(num_kb_total, kb0 + num_kb);
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int s = (int)(g % kPairStages);
                    if (!wait_for(smem_u32(&full[s]), (uint32_t)((g / kPairStages) & 1), false) || *abort_v) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kStageA), b0 = smem_u32(sB + s * kPairStageB);
#pragma unroll
                    for (int k = 0; k < kTcBK / 16; ++k)
                        mma_f16_pair(d, smem_desc(a0 + k * 32), smem_desc(b0 + k * 32), idesc, kb != kb0 || k != 0);
                    mma_commit_pair(smem_u32(&empty[s]));
                }
                if (ok) mma_commit_pair(smem_u32(&tfull[acc]));
            }
            if (!ok) {
                atomicExch(err, 1u);
                *abort_v = 1;
            }
            // Both accumulators drained: every epilogue arrival aimed at this CTA has landed.
            for (int j = i; j < i + 2; ++j)
                if (!wait_for(smem_u32(&tempty[j & 1]), (uint32_t)(((j >> 1) & 1) ^ 1), true)) {
                    atomicExch(err, 1u);
                    break;
                }
        }
    } else {   // epilogue warps 2..5 (both CTAs): TMEM lanes 32*(warp%4) .. +31 of this CTA
        const int lane_base = 32 * (warp & 3);
        const bool vec = (C & 3) == 0 && ((uintptr_t)P & 15) == 0;
        int i = 0;
        for (int t = cluster; t < num_tiles; t += n_clusters, ++i) {
            const int acc = i & 1;
            bool ok = wait_for(smem_u32(&tfull[acc]), (uint32_t)((i >> 1) & 1), false) && !*abort_v;
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(err, 1u);
                    *abort_v = 1;
                }
                break;
            }
            fence_after();
            const int z = t / tiles_mn, tt = t % tiles_mn;
            const int64_t row = (int64_t)(tt / tiles_n) * (2 * kTcBM) + rank * kTcBM + lane_base + lane;
            const int cbase = (tt % tiles_n) * (kTcBN / 2);
            const bool live = row < n_rx;
            float2 e0 = make_float2(0.f, 0.f);
            if (live && E0 && z == 0) {
                e0 = E0[row];
                e0.x *= e0scale;
                e0.y *= e0scale;
            }
            const uint32_t tbase = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * kTmemCols);
            for (int j = 0; j < kTcBN / 16; ++j) {
                float v[16], p[8];
                tmem_ld16(tbase + (uint32_t)(j * 16), v);
                if (Cout) {                          // complex partial sums, coalesced over rows
                    if (!live) continue;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int c = cbase + j * 8 + q;
                        if (c < C) Cout[((int64_t)z * C + c) * n_rx + row] = make_float2(v[2 * q] + e0.x, v[2 * q + 1] + e0.y);
                    }
                    continue;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float er = v[2 * q] + e0.x, ei = v[2 * q + 1] + e0.y;
                    p[q] = (er * er + ei * ei) * pscale;
                }
                if (!live) continue;
                const int c0 = cbase + j * 8;
                if (Eout) {                          // complex field, receiver-major like P
                    float2* edst = Eout + row * C + c0;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c0 + q < C) edst[q] = make_float2((v[2 * q] + e0.x) * escale, (v[2 * q + 1] + e0.y) * escale);
                }
                if (!P) continue;
                float* dst = P + row * C + c0;
                if (vec && c0 + 8 <= C) {
                    reinterpret_cast<float4*>(dst)[0] = make_float4(p[0], p[1], p[2], p[3]);
                    reinterpret_cast<float4*>(dst)[1] = make_float4(p[4], p[5], p[6], p[7]);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c0 + q < C) dst[q] = p[q];
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(map_to_rank(smem_u32(&tempty[acc]), 0));
        }
    }
    __syncwarp();
    fence_before();
    cluster_sync_all();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace

bool make_map(CUtensorMap* map, const void* base, bool fp16, int64_t rows, int cols, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Clusters of two CTAs that can be resident at once (0 if the pair kernel cannot be placed).
int pair_clusters(risrt_ctx* ctx)
{
    static int cached[64];
    static bool have[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (have[dev]) return cached[dev];
    int n = 0;
    if (cudaFuncSetAttribute(k_sweep_tc_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmemBytes) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(192, 1, 1);
        cfg.dynamicSmemBytes = kPairSmemBytes;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, k_sweep_tc_pair, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    cached[dev] = n;
    have[dev] = true;
    (void)ctx;
    return n;
}

// RISRT_SWEEP_PAIR=0 selects the one-CTA-per-tile kernel (kept as the reference design and fallback).
bool pair_enabled()
{
    const char* e = getenv("RISRT_SWEEP_PAIR");
    return !(e && e[0] == '0');
}

uint32_t make_idesc(bool fp16, int m, int n)
{
    // instruction descriptor (kind::f16): D = F32, A = B = BF16 or F16, both K-major, N/8, M/16
    const uint32_t fmt = fp16 ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

int sweep_tc(risrt_ctx* ctx, const void* X, const void* Y, const SweepShape& sh, bool fp16, const float2* E0,
             int64_t n_rx, int C, float* P, float pscale, float e0scale, unsigned* err_dev, bool defer, float2* Eout)
{
    const float escale = 1.f / e0scale;
    cudaStream_t s = ctx->stream;
    CUtensorMap mX, mY;
    if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15)) return fail(ctx, RISRT_ERR_INVALID_ARG, "operands not 16-byte aligned");
    const int ncl = pair_enabled() ? pair_clusters(ctx) : 0;
    const bool pair = ncl > 0;
    if (!make_map(&mX, X, fp16, n_rx, sh.Kp, kTcBM) || !make_map(&mY, Y, fp16, sh.Np, sh.Kp, pair ? kTcBN / 2 : kTcBN))
        return fail(ctx, RISRT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    RISRT_CUDA(ctx, cudaMemsetAsync(err_dev, 0, sizeof(unsigned), s));
    if (pair) {
        const int tiles_m = (int)((n_rx + 2 * kTcBM - 1) / (2 * kTcBM)), tiles_n = sh.Np / kTcBN;
        const int num_tiles = tiles_m * tiles_n;
        const int nc = num_tiles < ncl ? num_tiles : ncl;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(2 * nc), 1, 1);
        cfg.blockDim = dim3(192, 1, 1);
        cfg.dynamicSmemBytes = kPairSmemBytes;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const uint32_t idesc = make_idesc(fp16, 2 * kTcBM, kTcBN);
        cudaError_t le = cudaSuccess;
        RISRT_KERNEL(ctx, "k_sweep_tc_pair",
                     (le = cudaLaunchKernelEx(&cfg, k_sweep_tc_pair, mX, mY, sh.Kp / kTcBK, tiles_n, num_tiles, idesc, E0,
                                              n_rx, C, P, pscale, e0scale, err_dev, sh.Kp / kTcBK, (float2*)nullptr,
                                              Eout, escale)));
        if (le != cudaSuccess) return cuda_fail(ctx, le, "k_sweep_tc_pair");
    } else {
        RISRT_CUDA(ctx, cudaFuncSetAttribute(k_sweep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        dim3 grid((unsigned)(sh.Mp / kTcBM), (unsigned)(sh.Np / kTcBN));
        const uint32_t idesc = make_idesc(fp16, kTcBM, kTcBN);
        RISRT_KERNEL(ctx, "k_sweep_tc", (k_sweep_tc<<<grid, 192, kSmemBytes, s>>>(mX, mY, sh.Kp / kTcBK, idesc, E0, n_rx,
                                                                                C, P, pscale, e0scale, err_dev, Eout, escale)));
    }
    if (defer) return RISRT_OK;          // the flag stays in the workspace (risrt_sweep_check)
    unsigned h = 0;
    RISRT_CUDA(ctx, cudaMemcpyAsync(&h, err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    if (h) return fail(ctx, RISRT_ERR_TIMEOUT, "tensor-core sweep: a pipeline wait expired");
    return RISRT_OK;
}

// D = X . Y^T on SM pairs (BF16, both K-major: X [rows][Kp], Y [Np][Kp]) with the reduction split
// into about `splits` parts; writes the complex partial sums D[row][2c] + j D[row][2c + 1] (+ E0rows[row]
// in part 0) to out[(z C + c) rows + row] and the number of parts to *parts. RISRT_ERR_NOT_READY when
// the pair kernel cannot be placed on this device. Enqueued only: the caller clears *err_dev before
// and reads it after its last GEMM (an expired pipeline wait sets it).
int gemm_tc_complex(risrt_ctx* ctx, const void* X, int64_t rows, const void* Y, int Np, int Kp, const float2* E0rows, int C,
                    float2* out, int splits, int* parts, unsigned* err_dev)
{
    cudaStream_t s = ctx->stream;
    const int ncl = pair_clusters(ctx);
    if (ncl <= 0) return fail(ctx, RISRT_ERR_NOT_READY, "the paired tensor-core kernel cannot run on this device");
    if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15) || (Kp % kTcBK) || (Np % kTcBN))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "tensor-core operands: 16-byte alignment, K multiple of 64, N of 256");
    CUtensorMap mX, mY;
    if (!make_map(&mX, X, false, rows, Kp, kTcBM) || !make_map(&mY, Y, false, Np, Kp, kTcBN / 2))
        return fail(ctx, RISRT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    const int kb_total = Kp / kTcBK;
    const int kb_per = (kb_total + std::max(1, splits) - 1) / std::max(1, splits);
    const int z = (kb_total + kb_per - 1) / kb_per;
    const int tiles_m = (int)((rows + 2 * kTcBM - 1) / (2 * kTcBM)), tiles_n = Np / kTcBN;
    const int num_tiles = tiles_m * tiles_n * z;
    const int nc = num_tiles < ncl ? num_tiles : ncl;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * nc), 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = kPairSmemBytes;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const uint32_t idesc = make_idesc(false, 2 * kTcBM, kTcBN);
    cudaError_t le = cudaSuccess;
    RISRT_KERNEL(ctx, "k_sweep_tc_pair",
                 (le = cudaLaunchKernelEx(&cfg, k_sweep_tc_pair, mX, mY, kb_per, tiles_n, num_tiles, idesc, E0rows, rows, C,
                                          (float*)nullptr, 0.f, 1.f, err_dev, kb_total, out, (float2*)nullptr, 1.f)));
    if (le != cudaSuccess) return cuda_fail(ctx, le, "k_sweep_tc_pair");
    *parts = z;
    return RISRT_OK;
}

}  // namespace risrt
