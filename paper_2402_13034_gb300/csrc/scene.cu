// Scene upload: face table and linear BVH (Morton codes -> stable radix sort -> binary radix tree
// after Karras 2012 -> bottom-up box refit), plus the device-wide scan and sort they use.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

namespace risrt {

// ================================================================================================
// Exclusive scan of int64 (three launches: block sums, scan of the sums, apply)
// ================================================================================================
namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* sh_warp, int64_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = lane < nw ? sh_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh_warp[lane] = s;
    }
    __syncthreads();
    int64_t base = warp > 0 ? sh_warp[warp - 1] : 0;
    *total = sh_warp[nw - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void k_scan_reduce(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc = 0;
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
        if (i < n) acc += in[i];
    }
    int64_t tot;
    block_exclusive_scan(acc, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nb)
{
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
    }
}

__global__ void k_scan_apply(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             const int64_t* __restrict__ sums)
{
    __shared__ int64_t sh[32];
    // blocked arrangement: thread t owns items [t*kScanItems, (t+1)*kScanItems) of the tile
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t acc = 0;
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? in[base + j] : 0;
        acc += v[j];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(acc, sh, &tot) + sums[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = ex;
        ex += v[j];
    }
}
}  // namespace

size_t scan_temp_bytes(int64_t n) { return sizeof(int64_t) * (size_t)((n + kScanTile - 1) / kScanTile + 1); }

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t* sums = (int64_t*)temp;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    g_launches.fetch_add(3, std::memory_order_relaxed);
    return cudaGetLastError();
}

// ================================================================================================
// Stable LSD radix sort of (uint32 key, uint32 value), 8-bit digits
// ================================================================================================
namespace {
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 4;
constexpr int kSortTile = kSortThreads * kSortRounds;

__global__ void k_sort_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t n_tiles,
                            int64_t* __restrict__ hist)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = 0; j < kSortRounds; ++j) {
        int64_t i = base + (int64_t)j * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];   // digit-major
}

__global__ void k_sort_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                               int shift, int64_t n_tiles, const int64_t* __restrict__ offs)
{
    __shared__ int wcnt[kSortThreads / 32][256];
    __shared__ int running[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    running[threadIdx.x] = 0;
    int64_t tile_off = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
    __shared__ int64_t toff[256];
    toff[threadIdx.x] = tile_off;
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = 0; j < kSortRounds; ++j) {
        for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)j * kSortThreads + threadIdx.x;
        bool ok = i < n;
        uint32_t key = ok ? kin[i] : 0u;
        uint32_t val = ok ? vin[i] : 0u;
        uint32_t dig = ok ? (key >> shift) & 255u : 256u;   // 256 = padding, never written
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over warps, continuing from earlier rounds
            int d = threadIdx.x;
            int run = running[d];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                int c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            running[d] = run;
        }
        __syncthreads();
        if (ok) {
            int64_t pos = toff[dig] + wcnt[warp][dig] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}
}  // namespace

size_t sort_temp_bytes(int64_t n)
{
    int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    size_t hist = sizeof(int64_t) * 256 * (size_t)n_tiles;
    return 2 * sizeof(uint32_t) * (size_t)n + 2 * hist + scan_temp_bytes(256 * n_tiles) + 256;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, void* temp, cudaStream_t s)
{
    if (n <= 1) return cudaSuccess;
    int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    char* p = (char*)temp;
    uint32_t* k2 = (uint32_t*)p; p += sizeof(uint32_t) * n;
    uint32_t* v2 = (uint32_t*)p; p += sizeof(uint32_t) * n;
    p = (char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    int64_t* hist = (int64_t*)p; p += sizeof(int64_t) * 256 * n_tiles;
    int64_t* offs = (int64_t*)p; p += sizeof(int64_t) * 256 * n_tiles;
    void* scan_tmp = p;
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    int passes = (bits + 7) / 8;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = 8 * pass;
        k_sort_hist<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(ka, n, shift, n_tiles, hist);
        cudaError_t e = exclusive_scan_i64(hist, offs, 256 * n_tiles, scan_tmp, s);
        if (e != cudaSuccess) return e;
        k_sort_scatter<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, n_tiles, offs);
        g_launches.fetch_add(2, std::memory_order_relaxed);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

// ================================================================================================
// BVH build
// ================================================================================================
namespace {

__device__ __forceinline__ unsigned ordered_bits(float f)
{
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(unsigned o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

inline float from_ordered_host(unsigned o)
{
    const unsigned b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
    memcpy(&f, &b, sizeof(f));
    return f;
}

__global__ void k_bounds(const float* __restrict__ verts, int64_t nv, unsigned* __restrict__ bb)
{
    // bb[0..2] = ordered min, bb[3..5] = ordered max, bb[6] = max |coord| bits
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0}, ext = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            float v = verts[3 * i + k];
            unsigned o = ordered_bits(v);
            lo[k] = min(lo[k], o);
            hi[k] = max(hi[k], o);
            ext = max(ext, __float_as_uint(fabsf(v)));
        }
    }
    for (int k = 0; k < 3; ++k) {
        atomicMin(&bb[k], lo[k]);
        atomicMax(&bb[3 + k], hi[k]);
    }
    atomicMax(&bb[6], ext);
}

__device__ __forceinline__ unsigned spread10(unsigned x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Triangle references: a triangle whose box is longer than a cell (1/8 of the scene's largest
// span) in some axis is split into a grid of references, each bounded by the triangle's box
// intersected with one grid cell, so large walls do not inflate the boxes of the tree above them.
// Every point of the triangle lies in one reference's box, so traversal still finds every hit.
struct RefGrid {
    int n[3];
};

__device__ __forceinline__ void tri_box(const float* verts, const int32_t* tris, int64_t t, float lo[3], float hi[3])
{
    for (int k = 0; k < 3; ++k) {
        float a = verts[3 * tris[3 * t] + k], b = verts[3 * tris[3 * t + 1] + k], c = verts[3 * tris[3 * t + 2] + k];
        lo[k] = fminf(a, fminf(b, c));
        hi[k] = fmaxf(a, fmaxf(b, c));
    }
}

__device__ __forceinline__ RefGrid ref_grid(const float lo[3], const float hi[3], float cell)
{
    RefGrid g;
    for (int k = 0; k < 3; ++k) {
        int n = (int)ceilf((hi[k] - lo[k]) / cell);
        g.n[k] = max(1, min(n, 16));
    }
    return g;
}

// Box of the part of triangle t inside [blo, bhi] (Sutherland-Hodgman against the box's six planes,
// the box grown by e to absorb rounding); false if the triangle misses the box. Explicit rounding
// (no contraction): the counting and the emitting kernels must take the same decisions.
__device__ bool clip_tri_box(const float* verts, const int32_t* tris, int64_t t, const float blo[3], const float bhi[3],
                             float e, float olo[3], float ohi[3])
{
    float P[9][3], Q[9][3];
    int n = 3;
    for (int v = 0; v < 3; ++v)
        for (int k = 0; k < 3; ++k) P[v][k] = verts[3 * tris[3 * t + v] + k];
    for (int pl = 0; pl < 6 && n > 0; ++pl) {
        const int k = pl >> 1;
        const bool upper = pl & 1;
        const float lim = upper ? __fadd_rn(bhi[k], e) : __fsub_rn(blo[k], e);
        int m = 0;
        for (int i = 0; i < n; ++i) {
            const float* a = P[i];
            const float* b = P[(i + 1) % n];
            const float da = upper ? __fsub_rn(lim, a[k]) : __fsub_rn(a[k], lim);
            const float db = upper ? __fsub_rn(lim, b[k]) : __fsub_rn(b[k], lim);
            if (da >= 0.f && m < 9) {
                for (int c = 0; c < 3; ++c) Q[m][c] = a[c];
                ++m;
            }
            if ((da >= 0.f) != (db >= 0.f) && m < 9) {
                const float u = __fdiv_rn(da, __fsub_rn(da, db));
                for (int c = 0; c < 3; ++c) Q[m][c] = __fadd_rn(a[c], __fmul_rn(u, __fsub_rn(b[c], a[c])));
                Q[m][k] = lim;
                ++m;
            }
        }
        n = m;
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) P[i][c] = Q[i][c];
    }
    if (n == 0) return false;
    for (int c = 0; c < 3; ++c) {
        olo[c] = P[0][c];
        ohi[c] = P[0][c];
    }
    for (int i = 1; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            olo[c] = fminf(olo[c], P[i][c]);
            ohi[c] = fmaxf(ohi[c], P[i][c]);
        }
    for (int c = 0; c < 3; ++c) {         // stay inside the grown cell
        olo[c] = fmaxf(olo[c], __fsub_rn(blo[c], e));
        ohi[c] = fminf(ohi[c], __fadd_rn(bhi[c], e));
    }
    return true;
}

// Cell (i, j, l) of the reference grid of a triangle's box.
__device__ __forceinline__ void ref_cell(const float lo[3], const float hi[3], const RefGrid& g, const int c[3], float blo[3],
                                         float bhi[3])
{
    for (int k = 0; k < 3; ++k) {
        const float w = __fdiv_rn(__fsub_rn(hi[k], lo[k]), (float)g.n[k]);
        blo[k] = c[k] == 0 ? lo[k] : __fadd_rn(lo[k], __fmul_rn(w, (float)c[k]));
        bhi[k] = c[k] == g.n[k] - 1 ? hi[k] : __fadd_rn(lo[k], __fmul_rn(w, (float)(c[k] + 1)));
    }
}

__device__ __forceinline__ float clip_eps(const float lo[3], const float hi[3])
{
    return 1e-6f * (1.f + fmaxf(fmaxf(fabsf(lo[0]), fabsf(hi[0])), fmaxf(fmaxf(fabsf(lo[1]), fabsf(hi[1])),
                                                                            fmaxf(fabsf(lo[2]), fabsf(hi[2])))));
}

__device__ __forceinline__ float scene_cell(const unsigned* bb)
{
    float span = 0.f;
    for (int k = 0; k < 3; ++k) span = fmaxf(span, from_ordered(bb[3 + k]) - from_ordered(bb[k]));
    return fmaxf(span * 0.125f, 1e-6f);
}

// One warp per triangle, lanes over the cells of its reference grid (cell c = (i, j, l) with
// c = (i n1 + j) n2 + l): the number of cells the triangle meets (at least 1).
__global__ void k_ref_count(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t nt,
                            const unsigned* __restrict__ bb, int64_t* __restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nt) return;                              // whole warps leave together
    float lo[3], hi[3];
    tri_box(verts, tris, t, lo, hi);
    RefGrid g = ref_grid(lo, hi, scene_cell(bb));
    const int nc = g.n[0] * g.n[1] * g.n[2];
    if (nc == 1) {
        if (lane == 0) cnt[t] = 1;
        return;
    }
    const float e = clip_eps(lo, hi);
    int n = 0;
    for (int cc = lane; cc < nc; cc += 32) {
        const int c[3] = {cc / (g.n[1] * g.n[2]), (cc / g.n[2]) % g.n[1], cc % g.n[2]};
        float blo[3], bhi[3], olo[3], ohi[3];
        ref_cell(lo, hi, g, c, blo, bhi);
        n += clip_tri_box(verts, tris, t, blo, bhi, e, olo, ohi) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[t] = n > 0 ? n : 1;            // a triangle always keeps at least one reference
}

// Shell triangle: its plane has the whole scene box (bb) on one closed side, so no segment with both
// ends in the box crosses it (a wall, the floor or the ceiling of a box-shaped room, or a face lying
// in one of them). The tolerance only absorbs the rounding of the FP64 plane.
__device__ bool shell_tri(const float* verts, const int32_t* tris, int64_t t, const unsigned* bb)
{
    d3 v[3];
    for (int j = 0; j < 3; ++j) {
        const float* p = verts + 3 * (int64_t)tris[3 * t + j];
        v[j] = D3((double)p[0], (double)p[1], (double)p[2]);
    }
    d3 n = cross(v[1] - v[0], v[2] - v[0]);
    const double nn = norm(n);
    if (!(nn > 0.0)) return false;
    n = n * (1.0 / nn);
    const double d = dot(n, v[0]);
    double lo[3], hi[3], ext = 0.0;
    for (int k = 0; k < 3; ++k) {
        lo[k] = (double)from_ordered(bb[k]);
        hi[k] = (double)from_ordered(bb[3 + k]);
        ext = fmax(ext, fmax(fabs(lo[k]), fabs(hi[k])));
    }
    const double tol = 1e-12 * (1.0 + ext);
    double smin = 1e300, smax = -1e300;
    for (int c = 0; c < 8; ++c) {
        const d3 q = D3((c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]);
        const double sd = dot(n, q) - d;
        smin = fmin(smin, sd);
        smax = fmax(smax, sd);
    }
    return smin >= -tol || smax <= tol;
}

// References of every triangle with their boxes; 30-bit Morton code of each box centre. One warp per
// triangle: one reference per grid cell the triangle meets, in cell order, boxed tightly around the
// part inside the cell (a triangle in a single cell keeps its own box); never more references than
// counted, and any shortfall filled with the triangle's whole box (conservative). With `shell` set,
// the keys of shell triangles' references carry bit 30, so they sort after all others and the
// root's first child covers exactly the rest; shell_refs counts them.
__global__ void k_ref_emit(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t nt,
                           const unsigned* __restrict__ bb, const int64_t* __restrict__ off,
                           const int64_t* __restrict__ cnt,
                           uint32_t* __restrict__ ref_tri, float4* __restrict__ ref_lo, float4* __restrict__ ref_hi,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int shell,
                           unsigned long long* __restrict__ shell_refs)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nt) return;                              // whole warps leave together
    const unsigned shell_bit = shell && shell_tri(verts, tris, t, bb) ? (1u << 30) : 0u;
    if (shell_bit && lane == 0) atomicAdd(shell_refs, (unsigned long long)cnt[t]);
    float lo[3], hi[3];
    tri_box(verts, tris, t, lo, hi);
    RefGrid g = ref_grid(lo, hi, scene_cell(bb));
    float slo[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        slo[k] = from_ordered(bb[k]);
        float span = from_ordered(bb[3 + k]) - slo[k];
        inv[k] = span > 0.f ? 1.f / span : 0.f;
    }
    auto emit = [&](int64_t r, const float* olo, const float* ohi) {
        unsigned code = 0;
        for (int k = 0; k < 3; ++k) {
            float u = (0.5f * (olo[k] + ohi[k]) - slo[k]) * inv[k];
            unsigned q = (unsigned)fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
            code |= spread10(q) << (2 - k);
        }
        ref_tri[r] = (uint32_t)t;
        ref_lo[r] = make_float4(olo[0], olo[1], olo[2], 0.f);
        ref_hi[r] = make_float4(ohi[0], ohi[1], ohi[2], 0.f);
        keys[r] = code | shell_bit;
        vals[r] = (uint32_t)r;
    };
    const int nc = g.n[0] * g.n[1] * g.n[2];
    const int64_t r0 = off[t], r_end = r0 + cnt[t];
    if (nc == 1) {
        if (lane == 0) emit(r0, lo, hi);
        return;
    }
    const float e = clip_eps(lo, hi);
    int64_t r = r0;
    for (int c0 = 0; c0 < nc; c0 += 32) {
        const int cc = c0 + lane;
        float olo[3], ohi[3];
        bool in = false;
        if (cc < nc) {
            const int c[3] = {cc / (g.n[1] * g.n[2]), (cc / g.n[2]) % g.n[1], cc % g.n[2]};
            float blo[3], bhi[3];
            ref_cell(lo, hi, g, c, blo, bhi);
            in = clip_tri_box(verts, tris, t, blo, bhi, e, olo, ohi);
        }
        const unsigned b = __ballot_sync(0xffffffffu, in);
        const int64_t mine = r + __popc(b & ((1u << lane) - 1u));
        if (in && mine < r_end) emit(mine, olo, ohi);
        r += __popc(b);
    }
    for (int64_t q = r + lane; q < r_end; q += 32) emit(q, lo, hi);
}

// Per leaf (sorted reference order): exact float vertices of the referenced triangle, FP32 plane and
// edge planes computed in FP64, and the reference box for the refit. leaf_of_orig[t] receives one
// leaf of triangle t (all leaves of a triangle carry identical triangle data).
__global__ void k_leaves(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                         const int32_t* __restrict__ face, const uint32_t* __restrict__ order, int64_t n_ref,
                         const uint32_t* __restrict__ ref_tri, const float4* __restrict__ ref_lo,
                         const float4* __restrict__ ref_hi, TriVerts* __restrict__ tv, TriGeom* __restrict__ tg,
                         int* __restrict__ tf, float4* __restrict__ leaf_lo, float4* __restrict__ leaf_hi,
                         int* __restrict__ leaf_of_orig)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_ref) return;
    const int64_t ref = order[i];
    const int64_t t = ref_tri[ref];
    leaf_lo[i] = ref_lo[ref];
    leaf_hi[i] = ref_hi[ref];
    leaf_of_orig[t] = (int)i;
    float3 v[3];
    for (int j = 0; j < 3; ++j) {
        const float* p = verts + 3 * (int64_t)tris[3 * t + j];
        v[j] = f3(p[0], p[1], p[2]);
    }
    int f = face[t];
    TriVerts o;
    o.v0 = make_float4(v[0].x, v[0].y, v[0].z, __int_as_float(f));
    o.v1 = make_float4(v[1].x, v[1].y, v[1].z, 0.f);
    o.v2 = make_float4(v[2].x, v[2].y, v[2].z, 0.f);
    tv[i] = o;
    tf[i] = f;
    d3 a = D3(v[0]), b = D3(v[1]), c = D3(v[2]);
    d3 n = cross(b - a, c - a);
    double nn = norm(n);
    TriGeom g;
    if (nn > 0) {
        n = n * (1.0 / nn);
        g.plane = make_float4((float)n.x, (float)n.y, (float)n.z, (float)dot(n, a));
        d3 P[3] = {a, b, c};
        for (int k = 0; k < 3; ++k) {   // edge opposite vertex k runs P[k+1] -> P[k+2]
            d3 p = P[(k + 1) % 3], q = P[(k + 2) % 3];
            d3 e = q - p;
            d3 m = cross(n, e);          // in-plane, points to the interior for a CCW triangle about n
            double mn = norm(m);
            m = m * (1.0 / mn);
            g.edge[k] = make_float4((float)m.x, (float)m.y, (float)m.z, (float)dot(m, p));
        }
    } else {   // degenerate triangle: never hit
        g.plane = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < 3; ++k) g.edge[k] = make_float4(0.f, 0.f, 0.f, 1.f);
    }
    tg[i] = g;
}

__device__ __forceinline__ unsigned long long ckey(const uint32_t* keys, int i) {
    return ((unsigned long long)keys[i] << 32) | (unsigned)i;
}
__device__ __forceinline__ int delta(const uint32_t* keys, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    return __clzll(ckey(keys, i) ^ ckey(keys, j));
}

// Binary radix tree over n sorted keys (Karras, "Maximizing parallelism in the construction of
// BVHs, octrees, and k-d trees", HPG 2012): internal node i covers a key range found by an
// exponential + binary search on the common-prefix length, split at the highest differing bit.
__global__ void k_karras(const uint32_t* __restrict__ keys, int n, BvhNode* __restrict__ nodes,
                         int* __restrict__ parent_int, int* __restrict__ parent_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int left = (min(i, j) == gamma) ? ~gamma : gamma;
    int right = (max(i, j) == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    nodes[i].l_lo.w = __int_as_float(left);
    nodes[i].l_hi.w = __int_as_float(right);
    if (left < 0) parent_leaf[~left] = i; else parent_int[left] = i;
    if (right < 0) parent_leaf[~right] = i; else parent_int[right] = i;
}

__device__ __forceinline__ void store_slot(BvhNode* node, bool right, float3 lo, float3 hi, int face)
{
    float* base = right ? &node->r_lo.x : &node->l_lo.x;
    float* baseh = right ? &node->r_hi.x : &node->l_hi.x;
    volatile float* vl = base;
    volatile float* vh = baseh;
    vl[0] = lo.x; vl[1] = lo.y; vl[2] = lo.z;
    vh[0] = hi.x; vh[1] = hi.y; vh[2] = hi.z;
    *(volatile float*)(right ? &node->r_hi.w : &node->r_lo.w) = __int_as_float(face);
}

// Bottom-up refit: the second child to finish a node merges both boxes and moves up.
// Each child slot also records the one face all leaves below it belong to, or -1 when they mix
// faces (r_lo.w: left child, r_hi.w: right child), so a traversal can skip subtrees of ignored faces.
__global__ void k_refit(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi, int n, BvhNode* nodes,
                        const int* __restrict__ parent_int, const int* __restrict__ parent_leaf,
                        const int* __restrict__ leaf_face, int* flags, float pad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 lo = xyz(leaf_lo[i]), hi = xyz(leaf_hi[i]);
    lo = lo - f3(pad, pad, pad);
    hi = hi + f3(pad, pad, pad);
    int face = leaf_face[i];
    int child = ~i;
    int p = parent_leaf[i];
    while (p >= 0) {
        BvhNode* node = nodes + p;
        bool right = __float_as_int(((volatile float*)&node->l_hi.w)[0]) == child;
        store_slot(node, right, lo, hi, face);
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;
        __threadfence();
        volatile float* q = &node->l_lo.x;
        float3 a_lo = f3(q[0], q[1], q[2]), a_hi = f3(q[4], q[5], q[6]);
        float3 b_lo = f3(q[8], q[9], q[10]), b_hi = f3(q[12], q[13], q[14]);
        lo = f3(fminf(a_lo.x, b_lo.x), fminf(a_lo.y, b_lo.y), fminf(a_lo.z, b_lo.z));
        hi = f3(fmaxf(a_hi.x, b_hi.x), fmaxf(a_hi.y, b_hi.y), fmaxf(a_hi.z, b_hi.z));
        const int fa = __float_as_int(q[11]), fb = __float_as_int(q[15]);
        face = fa == fb ? fa : -1;
        child = p;
        p = parent_int[p];
    }
}

// Four-wide nodes: the slots of binary node i are its children, each internal child replaced by its
// own two children (tighter boxes, half the levels).
__global__ void k_bvh4(const BvhNode* __restrict__ nodes, int n_int, Bvh4Node* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const BvhNode nd = nodes[i];
    Bvh4Node o;
    int k = 0;
    auto put = [&](float4 lo, float4 hi, int code, float face) {
        o.lo[k] = make_float4(lo.x, lo.y, lo.z, __int_as_float(code));
        o.hi[k] = make_float4(hi.x, hi.y, hi.z, face);
        ++k;
    };
    for (int side = 0; side < 2; ++side) {
        const float4 lo = side ? nd.r_lo : nd.l_lo, hi = side ? nd.r_hi : nd.l_hi;
        const int code = __float_as_int(side ? nd.l_hi.w : nd.l_lo.w);
        const float face = side ? nd.r_hi.w : nd.r_lo.w;
        if (code < 0) {
            put(lo, hi, code, face);
        } else {
            const BvhNode c = nodes[code];
            put(c.l_lo, c.l_hi, __float_as_int(c.l_lo.w), c.r_lo.w);
            put(c.r_lo, c.r_hi, __float_as_int(c.l_hi.w), c.r_hi.w);
        }
    }
    for (; k < 4; ++k) {
        o.lo[k] = make_float4(1e30f, 1e30f, 1e30f, __int_as_float(kNoChild));
        o.hi[k] = make_float4(-1e30f, -1e30f, -1e30f, __int_as_float(-1));
    }
    out[i] = o;
}

// Compact four-wide tree. A walk that starts at a node of the binary tree and follows the four-wide
// views visits the nodes of one depth parity only: depth 1 (the roots of the main and the shell
// subtree) when the root splits them, else depth 0 (the root). Those nodes get a sort key that orders
// them by depth, then by index, so the compact array starts with the top levels (which the
// validation keeps in shared memory); the others sort last. parent_int[root] = -1.
__global__ void k_node_keys(const int* __restrict__ parent_int, int n_int, int parity, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals, unsigned* __restrict__ n_sel)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int d = 0;
    for (int p = parent_int[i]; p >= 0 && d < n_int; p = parent_int[p]) ++d;
    const bool sel = (d & 1) == parity;
    keys[i] = sel ? ((uint32_t)min(d >> 1, 31) << 27) | (uint32_t)i : 0xffffffffu;
    vals[i] = (uint32_t)i;
    if (sel) atomicAdd(n_sel, 1u);
}

__global__ void k_compact_index(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int n_int,
                                int* __restrict__ cidx)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_int && keys[j] != 0xffffffffu) cidx[vals[j]] = j;
}

// Entry j of the compact tree: the four-wide view of binary node vals[j], its internal child codes
// (nodes of the same parity) replaced by their compact positions.
__global__ void k_bvh4_compact(const Bvh4Node* __restrict__ nodes4, const uint32_t* __restrict__ vals,
                               const int* __restrict__ cidx, int n4c, Bvh4Node* __restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n4c) return;
    Bvh4Node nd = nodes4[vals[j]];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = __float_as_int(nd.lo[k].w);
        if (c >= 0 && c != kNoChild) nd.lo[k].w = __int_as_float(cidx[c]);
    }
    out[j] = nd;
}

// ------------------------------------------------------------------------------------------------
// faces
// ------------------------------------------------------------------------------------------------
__global__ void k_face_first(const int32_t* __restrict__ face, int64_t nt, int* __restrict__ first,
                             int* __restrict__ count)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    atomicMin(&first[face[t]], (int)t);
    atomicAdd(&count[face[t]], 1);
}

__global__ void k_face_fill(const int32_t* __restrict__ face, int64_t nt, const int* __restrict__ leaf_of_orig,
                            const int64_t* __restrict__ start, int* __restrict__ cursor, int* __restrict__ face_tris)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int f = face[t];
    int k = atomicAdd(&cursor[f], 1);
    face_tris[start[f] + k] = leaf_of_orig[t];
}

// Per face: an orthonormal frame in its plane (origin at a vertex, u along an edge of the first
// triangle, v = normal x u), the bounds of its vertices in (u, v), and a grid of cells of side about
// h (1 to 128 per axis). cnt[f] = cells of face f (exclusive-scan input, cnt[F] = 0).
__global__ void k_face_grid(const Face* __restrict__ faces, const int* __restrict__ face_tris,
                            const TriVerts* __restrict__ tri_verts, int F, double h, FaceGrid* __restrict__ grid,
                            int64_t* __restrict__ cnt)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > F) return;
    if (f == F) {
        cnt[F] = 0;
        return;
    }
    const Face fc = faces[f];
    if (fc.tri_end <= fc.tri_begin) {      // a face id without triangles: one cell, never looked up
        FaceGrid g = {};
        g.o.w = 1.f;
        g.dv = 1.f;
        g.nu = g.nv = 1;
        grid[f] = g;
        cnt[f] = 1;
        return;
    }
    const d3 n = D3(fc.plane.x, fc.plane.y, fc.plane.z);
    const TriVerts t0 = tri_verts[face_tris[fc.tri_begin]];
    const d3 o = D3(t0.v0.x, t0.v0.y, t0.v0.z);
    d3 e = D3(t0.v1.x, t0.v1.y, t0.v1.z) - o;
    e = e - n * dot(n, e);
    double el = norm(e);
    if (!(el > 0.0)) {            // degenerate first edge: any direction in the plane
        e = fabs(n.x) < 0.9 ? cross(n, D3(1, 0, 0)) : cross(n, D3(0, 1, 0));
        el = norm(e);
    }
    const d3 u = e * (1.0 / el);
    const d3 v = cross(n, u);
    double a0 = 1e300, a1 = -1e300, b0 = 1e300, b1 = -1e300;
    for (int j = fc.tri_begin; j < fc.tri_end; ++j) {
        const TriVerts tv = tri_verts[face_tris[j]];
        const float4 q[3] = {tv.v0, tv.v1, tv.v2};
        for (int k = 0; k < 3; ++k) {
            const d3 p = D3(q[k].x, q[k].y, q[k].z) - o;
            const double a = dot(p, u), b = dot(p, v);
            a0 = fmin(a0, a); a1 = fmax(a1, a);
            b0 = fmin(b0, b); b1 = fmax(b1, b);
        }
    }
    const int nu = (int)fmin(fmax(ceil((a1 - a0) / h), 1.0), 128.0);
    const int nv = (int)fmin(fmax(ceil((b1 - b0) / h), 1.0), 128.0);
    FaceGrid g;
    g.o = make_float4((float)o.x, (float)o.y, (float)o.z, (float)fmax((a1 - a0) / nu, 1e-6));
    g.u = make_float4((float)u.x, (float)u.y, (float)u.z, (float)a0);
    g.v = make_float4((float)v.x, (float)v.y, (float)v.z, (float)b0);
    g.nu = nu;
    g.nv = nv;
    g.off = 0;
    g.dv = (float)fmax((b1 - b0) / nv, 1e-6);
    grid[f] = g;
    cnt[f] = (int64_t)nu * nv;
}

__global__ void k_cell_face(FaceGrid* __restrict__ grid, const int64_t* __restrict__ off, int F, int* __restrict__ cell_face)
{
    const int f = blockIdx.x;
    if (f >= F) return;
    const int64_t o = off[f];
    const int n = grid[f].nu * grid[f].nv;
    if (threadIdx.x == 0) grid[f].off = (int)o;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cell_face[o + i] = f;
}

// Face plane in FP64 from the face's first triangle (lowest input index), as the image method's
// mirror plane (Sec. II-B).
__global__ void k_face_plane(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                             const int32_t* __restrict__ mat, const int* __restrict__ first,
                             const int64_t* __restrict__ start, const int* __restrict__ count, int F,
                             Face* __restrict__ faces)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    int t = first[f];
    d3 v[3];
    for (int j = 0; j < 3; ++j) {
        const float* p = verts + 3 * (int64_t)tris[3 * (int64_t)t + j];
        v[j] = D3((double)p[0], (double)p[1], (double)p[2]);
    }
    d3 n = cross(v[1] - v[0], v[2] - v[0]);
    n = n * (1.0 / norm(n));
    double d = dot(n, v[0]);
    Face fc;
    fc.plane = mk_dv4(n.x, n.y, n.z, d);
    fc.plane32 = make_float4((float)n.x, (float)n.y, (float)n.z, (float)d);
    fc.tri_begin = (int)start[f];
    fc.tri_end = (int)(start[f] + count[f]);
    fc.mat = mat[t];
    fc.pad = 0;
    faces[f] = fc;
}

__device__ __forceinline__ bool same3(float4 a, float4 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

// Outline of each face for the FP32 in-face filter: a single triangle keeps its three edges; two
// triangles sharing an edge keep their four outer edges when the quad is convex.
__global__ void k_face_test(const Face* __restrict__ faces, const int* __restrict__ face_tris,
                            const TriVerts* __restrict__ tv, const TriGeom* __restrict__ tg, int F,
                            FaceTest* __restrict__ out)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const Face fc = faces[f];
    FaceTest t;
    t.n = 0;
    t.pad[0] = t.pad[1] = t.pad[2] = 0;
    for (int i = 0; i < 4; ++i) t.e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int cnt = fc.tri_end - fc.tri_begin;
    if (cnt == 1) {
        const TriGeom g = tg[face_tris[fc.tri_begin]];
        for (int i = 0; i < 3; ++i) t.e[i] = g.edge[i];
        t.e[3] = make_float4(0.f, 0.f, 0.f, -1e30f);   // never the closest edge
        t.n = 3;
    } else if (cnt == 2) {
        const int a = face_tris[fc.tri_begin], b = face_tris[fc.tri_begin + 1];
        const float4 va[3] = {tv[a].v0, tv[a].v1, tv[a].v2};
        const float4 vb[3] = {tv[b].v0, tv[b].v1, tv[b].v2};
        // vertex of each triangle that is not on the shared edge (edge i is opposite vertex i)
        int oa = -1, ob = -1;
        for (int i = 0; i < 3; ++i) {
            int hits = 0;
            for (int j = 0; j < 3; ++j) hits += same3(va[i], vb[j]);
            if (!hits) oa = i;
        }
        for (int j = 0; j < 3; ++j) {
            int hits = 0;
            for (int i = 0; i < 3; ++i) hits += same3(va[i], vb[j]);
            if (!hits) ob = j;
        }
        if (oa >= 0 && ob >= 0) {
            const TriGeom ga = tg[a], gb = tg[b];
            int n = 0;
            for (int i = 0; i < 3; ++i) if (i != oa) t.e[n++] = ga.edge[i];
            for (int j = 0; j < 3; ++j) if (j != ob) t.e[n++] = gb.edge[j];
            // convex if every vertex lies on the inner side of every outer edge
            bool convex = true;
            for (int i = 0; i < 4 && convex; ++i)
                for (int j = 0; j < 3; ++j) {
                    float4 v = va[j];
                    if (t.e[i].x * v.x + t.e[i].y * v.y + t.e[i].z * v.z - t.e[i].w < -1e-5f) convex = false;
                    v = vb[j];
                    if (t.e[i].x * v.x + t.e[i].y * v.y + t.e[i].z * v.z - t.e[i].w < -1e-5f) convex = false;
                }
            t.n = convex ? 4 : 0;
        }
    }
    out[f] = t;
}

__global__ void k_i32_to_i64(const int* __restrict__ a, int64_t* __restrict__ b, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

template <typename T>
int dmalloc(risrt_ctx* ctx, T** p, size_t count)
{
    cudaError_t e = ctx_malloc(ctx, (void**)p, sizeof(T) * (count > 0 ? count : 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, RISRT_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    return RISRT_OK;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int build_scene(risrt_ctx* ctx, risrt_scene* sc, const float* verts_host, int64_t n_verts,
                const int32_t* tris_host, const int32_t* face_host, const int32_t* mat_host,
                const float* mats_host, int n_mat)
{
    cudaStream_t s = ctx->stream;
    const int64_t nt = sc->n_tris;
    const int F = sc->n_faces;
    sc->n_mat = n_mat;
    int rc;
    if ((rc = dmalloc(ctx, &sc->mats, n_mat))) return rc;
    RISRT_CUDA(ctx, cudaMemcpyAsync(sc->mats, mats_host, sizeof(float2) * n_mat, cudaMemcpyHostToDevice, s));
    if (nt == 0) {
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        return RISRT_OK;
    }
    // inputs on the device
    float* d_verts;
    int32_t *d_tris, *d_face, *d_mat;
    if ((rc = dmalloc(ctx, &d_verts, 3 * n_verts))) return rc;
    if ((rc = dmalloc(ctx, &d_tris, 3 * nt))) return rc;
    if ((rc = dmalloc(ctx, &d_face, nt))) return rc;
    if ((rc = dmalloc(ctx, &d_mat, nt))) return rc;
    RISRT_CUDA(ctx, cudaMemcpyAsync(d_verts, verts_host, sizeof(float) * 3 * n_verts, cudaMemcpyHostToDevice, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(d_tris, tris_host, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(d_face, face_host, sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(d_mat, mat_host, sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));

    // scene bounds
    // bb[0..6] bounds (k_bounds), bb[8..9] the number of shell references (64-bit), bb[10] the number
    // of four-wide nodes
    unsigned* d_bb;
    if ((rc = dmalloc(ctx, &d_bb, 12))) return rc;
    unsigned bb_init[12] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const char* shell_env = getenv("RISRT_SHELL");      // "0": shell triangles stay in the main tree
    const int shell_on = !(shell_env && shell_env[0] == '0');
    RISRT_CUDA(ctx, cudaMemcpyAsync(d_bb, bb_init, sizeof(bb_init), cudaMemcpyHostToDevice, s));
    RISRT_KERNEL(ctx, "k_bounds", (k_bounds<<<std::min<int64_t>(nblk(n_verts, 256), 1024), 256, 0, s>>>(d_verts, n_verts, d_bb)));

    // triangle references (large triangles split over a grid), Morton codes, stable sort
    int64_t *ref_cnt, *ref_off;
    if ((rc = dmalloc(ctx, &ref_cnt, nt + 1))) return rc;
    if ((rc = dmalloc(ctx, &ref_off, nt + 1))) return rc;
    void* tmp0;
    if ((rc = dmalloc(ctx, (char**)&tmp0, scan_temp_bytes(nt + 1) + 64))) return rc;
    RISRT_CUDA(ctx, cudaMemsetAsync(ref_cnt + nt, 0, sizeof(int64_t), s));
    RISRT_KERNEL(ctx, "k_ref_count", (k_ref_count<<<nblk(nt * 32, 256), 256, 0, s>>>(d_verts, d_tris, nt, d_bb, ref_cnt)));
    RISRT_CUDA(ctx, exclusive_scan_i64(ref_cnt, ref_off, nt + 1, tmp0, s));
    int64_t nr = 0;
    RISRT_CUDA(ctx, cudaMemcpyAsync(&nr, ref_off + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    if (nr > ((int64_t)1 << 27)) return fail(ctx, RISRT_ERR_CAPACITY, "too many BVH references");
    sc->n_refs = nr;
    uint32_t *keys, *vals, *ref_tri;
    float4 *ref_lo, *ref_hi, *leaf_lo, *leaf_hi;
    void* tmp;
    if ((rc = dmalloc(ctx, &keys, nr))) return rc;
    if ((rc = dmalloc(ctx, &vals, nr))) return rc;
    if ((rc = dmalloc(ctx, &ref_tri, nr))) return rc;
    if ((rc = dmalloc(ctx, &ref_lo, nr))) return rc;
    if ((rc = dmalloc(ctx, &ref_hi, nr))) return rc;
    if ((rc = dmalloc(ctx, &leaf_lo, nr))) return rc;
    if ((rc = dmalloc(ctx, &leaf_hi, nr))) return rc;
    size_t tmp_bytes = std::max(sort_temp_bytes(nr), scan_temp_bytes(F) + 64);
    if ((rc = dmalloc(ctx, (char**)&tmp, tmp_bytes))) return rc;
    RISRT_KERNEL(ctx, "k_ref_emit", (k_ref_emit<<<nblk(nt * 32, 256), 256, 0, s>>>(d_verts, d_tris, nt, d_bb, ref_off, ref_cnt, ref_tri,
                                                                            ref_lo, ref_hi, keys, vals, shell_on,
                                                                            (unsigned long long*)(d_bb + 8))));
    RISRT_CUDA(ctx, radix_sort_pairs(keys, vals, nr, 31, tmp, s));

    // leaves, hierarchy, refit
    int* leaf_of_orig;
    if ((rc = dmalloc(ctx, &sc->tri_verts, nr))) return rc;
    if ((rc = dmalloc(ctx, &sc->tri_leaf, nt))) return rc;
    if ((rc = dmalloc(ctx, &sc->tri_geom, nr))) return rc;
    if ((rc = dmalloc(ctx, &sc->tri_face, nr))) return rc;
    if ((rc = dmalloc(ctx, &leaf_of_orig, nt))) return rc;
    RISRT_KERNEL(ctx, "k_leaves", (k_leaves<<<nblk(nr, 256), 256, 0, s>>>(d_verts, d_tris, d_face, vals, nr, ref_tri, ref_lo,
                                                                        ref_hi, sc->tri_verts, sc->tri_geom, sc->tri_face,
                                                                        leaf_lo, leaf_hi, leaf_of_orig)));

    unsigned bb_host[10];
    RISRT_CUDA(ctx, cudaMemcpyAsync(bb_host, d_bb, sizeof(bb_host), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    float ext;
    memcpy(&ext, &bb_host[6], 4);
    sc->scene_extent = ext;
    for (int k = 0; k < 3; ++k) {
        sc->box_lo[k] = from_ordered_host(bb_host[k]);
        sc->box_hi[k] = from_ordered_host(bb_host[3 + k]);
    }
    uint64_t n_shell = 0;
    memcpy(&n_shell, &bb_host[8], sizeof(n_shell));
    sc->n_shell_refs = (int64_t)n_shell;
    const float pad = 1e-4f * (1.f + ext);

    int n_int = (int)std::max<int64_t>(nr - 1, 1);
    int *parent_int, *parent_leaf, *flags;
    if ((rc = dmalloc(ctx, &sc->nodes, n_int))) return rc;
    if ((rc = dmalloc(ctx, &sc->nodes4, n_int))) return rc;
    if ((rc = dmalloc(ctx, &parent_int, n_int))) return rc;
    if ((rc = dmalloc(ctx, &parent_leaf, nr))) return rc;
    if ((rc = dmalloc(ctx, &flags, n_int))) return rc;
    RISRT_CUDA(ctx, cudaMemsetAsync(sc->nodes, 0, sizeof(BvhNode) * n_int, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(flags, 0, sizeof(int) * n_int, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(parent_int, 0xff, sizeof(int) * n_int, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(parent_leaf, 0xff, sizeof(int) * nr, s));
    // The shell references sort last (key bit 30), so when both kinds exist the root splits at that
    // bit: its first child (leaf 0 or internal node n_main - 1, the radix tree's split position) covers
    // the others, its second (leaf n_main or internal node n_main) the shell.
    const int64_t n_shell_refs = sc->n_shell_refs, n_main = nr - n_shell_refs;
    const bool split = n_shell_refs > 0 && n_main > 0;
    int* cidx = nullptr;
    if ((rc = dmalloc(ctx, &cidx, n_int))) return rc;
    if (nr > 1) {
        RISRT_KERNEL(ctx, "k_karras", (k_karras<<<nblk(nr - 1, 256), 256, 0, s>>>(keys, (int)nr, sc->nodes, parent_int, parent_leaf)));
        RISRT_KERNEL(ctx, "k_refit", (k_refit<<<nblk(nr, 256), 256, 0, s>>>(leaf_lo, leaf_hi, (int)nr, sc->nodes, parent_int, parent_leaf, sc->tri_face, flags, pad)));
        RISRT_KERNEL(ctx, "k_bvh4", (k_bvh4<<<nblk(n_int, 256), 256, 0, s>>>(sc->nodes, n_int, sc->nodes4)));
        // compact four-wide tree in breadth-first order (the reference keys and values are free now)
        RISRT_KERNEL(ctx, "k_node_keys", (k_node_keys<<<nblk(n_int, 256), 256, 0, s>>>(parent_int, n_int, split ? 1 : 0, keys, vals,
                                                                                     d_bb + 10)));
        RISRT_CUDA(ctx, radix_sort_pairs(keys, vals, n_int, 32, tmp, s));
        RISRT_CUDA(ctx, cudaMemsetAsync(cidx, 0xff, sizeof(int) * n_int, s));
        RISRT_KERNEL(ctx, "k_compact_index", (k_compact_index<<<nblk(n_int, 256), 256, 0, s>>>(keys, vals, n_int, cidx)));
        unsigned n4c = 0;
        RISRT_CUDA(ctx, cudaMemcpyAsync(&n4c, d_bb + 10, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        Bvh4Node* compact;
        if ((rc = dmalloc(ctx, &compact, std::max<unsigned>(n4c, 1u)))) return rc;
        RISRT_KERNEL(ctx, "k_bvh4_compact", (k_bvh4_compact<<<nblk(n4c, 128), 128, 0, s>>>(sc->nodes4, vals, cidx, (int)n4c, compact)));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        ctx_free(ctx, sc->nodes4);
        sc->nodes4 = compact;
        sc->n_nodes4 = (int)n4c;
        // walk starts: the depth-1 nodes sort first, the main subtree's root before the shell's
        if (split) {
            sc->root_main = n_main > 1 ? 0 : ~0;
            sc->root_shell = n_shell_refs > 1 ? (n_main > 1 ? 1 : 0) : ~(int)n_main;
        } else if (n_shell_refs == 0) {
            sc->root_main = 0;
        } else {
            sc->root_shell = 0;
        }
    } else if (n_shell_refs == 0) {
        sc->root_main = ~0;
    } else {
        sc->root_shell = ~0;
    }

    // faces: first triangle, triangle lists, FP64 planes
    int *first, *count, *cursor;
    int64_t *count64, *start;
    if ((rc = dmalloc(ctx, &first, F))) return rc;
    if ((rc = dmalloc(ctx, &count, F))) return rc;
    if ((rc = dmalloc(ctx, &cursor, F))) return rc;
    if ((rc = dmalloc(ctx, &count64, F))) return rc;
    if ((rc = dmalloc(ctx, &start, F))) return rc;
    if ((rc = dmalloc(ctx, &sc->face_tris, nt))) return rc;
    if ((rc = dmalloc(ctx, &sc->faces, F))) return rc;
    if ((rc = dmalloc(ctx, &sc->face_test, F))) return rc;
    RISRT_CUDA(ctx, cudaMemsetAsync(first, 0x7f, sizeof(int) * F, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int) * F, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(cursor, 0, sizeof(int) * F, s));
    RISRT_KERNEL(ctx, "k_face_first", (k_face_first<<<nblk(nt, 256), 256, 0, s>>>(d_face, nt, first, count)));
    RISRT_KERNEL(ctx, "k_i32_to_i64", (k_i32_to_i64<<<nblk(F, 256), 256, 0, s>>>(count, count64, F)));
    RISRT_CUDA(ctx, exclusive_scan_i64(count64, start, F, tmp, s));
    RISRT_KERNEL(ctx, "k_face_fill", (k_face_fill<<<nblk(nt, 256), 256, 0, s>>>(d_face, nt, leaf_of_orig, start, cursor, sc->face_tris)));
    RISRT_KERNEL(ctx, "k_face_plane", (k_face_plane<<<nblk(F, 128), 128, 0, s>>>(d_verts, d_tris, d_mat, first, start, count, F, sc->faces)));
    RISRT_KERNEL(ctx, "k_face_test", (k_face_test<<<nblk(F, 128), 128, 0, s>>>(sc->faces, sc->face_tris, sc->tri_verts,
                                                                               sc->tri_geom, F, sc->face_test)));

    // cell grids of the faces for the per-source visibility maps (cells of about 1/96 of the extent)
    {
        int64_t *gcnt, *goff;
        if ((rc = dmalloc(ctx, &gcnt, F + 1))) return rc;
        if ((rc = dmalloc(ctx, &goff, F + 1))) return rc;
        if ((rc = dmalloc(ctx, &sc->face_grid, F))) return rc;
        const double h = fmax((double)sc->scene_extent, 1e-3) / 96.0;
        RISRT_KERNEL(ctx, "k_face_grid", (k_face_grid<<<nblk(F + 1, 128), 128, 0, s>>>(sc->faces, sc->face_tris, sc->tri_verts,
                                                                                    F, h, sc->face_grid, gcnt)));
        RISRT_CUDA(ctx, exclusive_scan_i64(gcnt, goff, F + 1, tmp, s));
        int64_t n_cells = 0;
        RISRT_CUDA(ctx, cudaMemcpyAsync(&n_cells, goff + F, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        sc->n_cells = n_cells;
        if ((rc = dmalloc(ctx, &sc->cell_face, n_cells > 0 ? n_cells : 1))) return rc;
        RISRT_KERNEL(ctx, "k_cell_face", (k_cell_face<<<F, 256, 0, s>>>(sc->face_grid, goff, F, sc->cell_face)));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        ctx_free(ctx, gcnt);
        ctx_free(ctx, goff);
    }

    RISRT_CUDA(ctx, cudaMemcpyAsync(sc->tri_leaf, leaf_of_orig, sizeof(int) * nt, cudaMemcpyDeviceToDevice, s));
    RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    for (void* p : {(void*)d_verts, (void*)d_tris, (void*)d_face, (void*)d_mat, (void*)d_bb, (void*)keys, (void*)vals, tmp,
                    (void*)leaf_of_orig, tmp0, (void*)ref_cnt, (void*)ref_off, (void*)ref_tri, (void*)ref_lo, (void*)ref_hi,
                    (void*)leaf_lo, (void*)leaf_hi, (void*)parent_int, (void*)parent_leaf, (void*)flags, (void*)cidx,
                    (void*)first, (void*)count, (void*)cursor, (void*)count64, (void*)start})
        ctx_free(ctx, p);
    return RISRT_OK;
}

}  // namespace risrt
