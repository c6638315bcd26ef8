// Path finding (Sec. II-B): image trees of the Tx and the RIS centre over face sequences of length
// <= 2, per-destination candidate search, BVH occlusion of every segment, per-element direct-leg
// visibility (one ray per element, Sec. IV-A), and the resident path set with FP64 phase references.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "cplx32.cuh"
#include "frame.cuh"
#include "geom.cuh"

namespace risrt {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------------------------------------
// sequence tables
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool coplanar_d(const Face& a, const Face& b)
{
    d3 na = ld3(a.plane), nb = ld3(b.plane);
    if (norm(cross(na, nb)) > 1e-9) return false;
    double s = dot(na, nb) > 0 ? 1.0 : -1.0;
    return fabs(a.plane.w - s * b.plane.w) < 1e-9;
}
__device__ __forceinline__ bool contains_point(const Face& a, d3 p) { return fabs(dot(ld3(a.plane), p) - a.plane.w) < 1e-6; }

// Can face f2 hold the second reflection point of a path src -> f1 -> f2 -> (anything)? The point
// must lie strictly on the source's side of plane f1 and inside the cone from the source image S1
// through f1 (the union over f1's triangles of the trihedral cones with apex S1). Returns false only
// when every vertex of f2 is separated by more than 1e-9 m, so no destination can make the sequence
// valid; the test is independent of the receiver.
// Can a path from src reflect on f1 and then reach face f2? f2 must have a point in front of f1 (on
// the source side) and inside the beam from the image S1 of src through f1. Decided in FP32 with a
// margin far above its rounding: a sequence is dropped only when the separation is certain (every
// vertex of f2 behind f1, or outside one side plane of each of f1's triangles, by more than m);
// sequences kept in doubt are settled exactly by the candidate tests later.
__device__ bool beam_reaches(const DeviceScene& S, d3 src, int f1, int f2, float m)
{
    const Face F1 = S.faces[f1], F2 = S.faces[f2];
    const float3 n1 = xyz(F1.plane32);
    const float s0 = dot(n1, to_f(src)) - F1.plane32.w;
    const float sgn = s0 > 0.f ? 1.f : -1.f;
    bool any_front = false;
    for (int j = F2.tri_begin; j < F2.tri_end && !any_front; ++j) {
        const TriVerts tv = S.tri_verts[S.face_tris[j]];
        const float3 v[3] = {xyz(tv.v0), xyz(tv.v1), xyz(tv.v2)};
        for (int i = 0; i < 3; ++i)
            if (sgn * (dot(n1, v[i]) - F1.plane32.w) > -m) any_front = true;
    }
    if (!any_front) return false;
    const float3 S1 = to_f(mirror_pt(src, ld3(F1.plane), F1.plane.w));
    for (int a = F1.tri_begin; a < F1.tri_end; ++a) {
        const TriVerts ta = S.tri_verts[S.face_tris[a]];
        const float3 P[3] = {xyz(ta.v0), xyz(ta.v1), xyz(ta.v2)};
        bool separated = false;
        for (int e = 0; e < 3 && !separated; ++e) {
            const float3 p = P[e], q = P[(e + 1) % 3], r = P[(e + 2) % 3];
            float3 nn = cross(p - S1, q - S1);
            const float l2 = dot(nn, nn);
            if (!(l2 > 0.f)) continue;
            nn = nn * rsqrtf(l2);
            if (dot(nn, r - S1) < 0.f) nn = nn * -1.f;
            bool all_out = true;
            for (int j = F2.tri_begin; j < F2.tri_end && all_out; ++j) {
                const TriVerts tv = S.tri_verts[S.face_tris[j]];
                const float3 v[3] = {xyz(tv.v0), xyz(tv.v1), xyz(tv.v2)};
                for (int i = 0; i < 3; ++i)
                    if (dot(nn, v[i] - S1) >= -m) all_out = false;
            }
            separated = all_out;
        }
        if (!separated) return true;
    }
    return false;
}

// mode 0: Tx leg (last face may not contain the RIS centre); 1: Rx leg (first face may not);
// 2: Tx -> Rx environment paths. Order-2 sequences whose second face is outside the beam of the
// first are dropped (beam_reaches).
__global__ void k_seq_allowed(DeviceScene S, int64_t n_ids, int mode, Frame fr, d3 src, float margin,
                              int64_t* __restrict__ flag)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= n_ids) return;
    const int F = S.n_faces;
    int f1, f2 = -1, k = 1;
    if (id < F) f1 = (int)id;
    else {
        int64_t r = id - F;
        f1 = (int)(r / F);
        f2 = (int)(r % F);
        k = 2;
    }
    bool ok = true;
    if (k == 2 && (f1 == f2 || coplanar_d(S.faces[f1], S.faces[f2]))) ok = false;
    d3 c = fr_c(fr);
    if (mode == 0 && contains_point(S.faces[k == 2 ? f2 : f1], c)) ok = false;
    if (mode == 1 && contains_point(S.faces[f1], c)) ok = false;
    if (ok && k == 2 && fabs(dot(ld3(S.faces[f1].plane), src) - S.faces[f1].plane.w) > 0.0 && !beam_reaches(S, src, f1, f2, margin))
        ok = false;
    flag[id] = ok ? 1 : 0;
}

// Number of allowed sequences: last exclusive-scan position + last flag.
__global__ void k_seq_count(const int64_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t n_ids,
                            int64_t* __restrict__ out)
{
    if (threadIdx.x == 0) *out = pos[n_ids - 1] + flag[n_ids - 1];
}

__global__ void k_seq_build(DeviceScene S, int64_t n_ids, const int64_t* __restrict__ flag,
                            const int64_t* __restrict__ pos, d3 src, SeqEntry* __restrict__ out,
                            SeqEntryD* __restrict__ outd)
{
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= n_ids || !flag[id]) return;
    const int F = S.n_faces;
    int f1, f2 = -1, k = 1;
    if (id < F) f1 = (int)id;
    else {
        int64_t r = id - F;
        f1 = (int)(r / F);
        f2 = (int)(r % F);
        k = 2;
    }
    const dv4 p1 = S.faces[f1].plane;
    d3 S1 = mirror_pt(src, ld3(p1), p1.w);
    d3 S2 = S1;
    dv4 pl = p1;
    if (k == 2) {
        pl = S.faces[f2].plane;
        S2 = mirror_pt(S1, ld3(pl), pl.w);
    }
    SeqEntry e;
    const d3 prev = k == 2 ? S1 : src;
    e.sL = make_float4((float)S2.x, (float)S2.y, (float)S2.z, (float)(dot(ld3(pl), prev) - pl.w));
    e.pL = make_float4((float)pl.x, (float)pl.y, (float)pl.z, (float)pl.w);
    e.s1 = make_float4((float)S1.x, (float)S1.y, (float)S1.z, (float)(dot(ld3(p1), src) - p1.w));
    e.p1 = make_float4((float)p1.x, (float)p1.y, (float)p1.z, (float)p1.w);
    e.info = make_int4(f1, f2, (int)id, k);
    int64_t o = pos[id];
    out[o] = e;
    SeqEntryD d;
    d.S1 = mk_dv4(S1.x, S1.y, S1.z, 0.0);
    d.S2 = mk_dv4(S2.x, S2.y, S2.z, 0.0);
    outd[o] = d;
}

// ------------------------------------------------------------------------------------------------
// candidate search: for each destination and each allowed sequence, back-trace the reflection
// points and keep the sequence if every point lies in its face and on the correct sides.
// ------------------------------------------------------------------------------------------------
constexpr int kCandThreads = 128;
constexpr int kCandChunk = 2048;

// Candidate filter in FP32 with exact conditions (Sec. II-B image method):
//  (A) the destination and the previous image lie strictly on the same side of the last plane
//      (equivalently the back-trace parameter lies in (0,1));
//  (B) the last reflection point lies in its face;
//  (C) order 2: the source and the last reflection point lie on the same side of the first plane;
//  (D) order 2: the first reflection point lies in its face.
// Each test is decided in FP32 when its margin exceeds the FP32 error bound, otherwise the whole
// candidate is settled by the FP64 check.
#ifndef RISRT_MAX_SMEM_FACES
#define RISRT_MAX_SMEM_FACES 1024
#endif
constexpr int kMaxSmemFaces = RISRT_MAX_SMEM_FACES;

template <bool SMEM_FACES>
__device__ __forceinline__ int face_class(const DeviceScene& S, const FaceTest* sh_faces, int f, float3 q, float tol)
{
    const FaceTest& t = SMEM_FACES ? sh_faces[f] : S.face_test[f];
    if (t.n) return in_outline_fp32(t, q, tol);
    return in_face_fp32(S, f, q, tol);
}

// Does the box [lo, hi] reach into the pyramid from apex `ap` through one of face f's triangles
// (optionally mirrored across the plane (mn, md))? False only when, for every triangle, one side
// plane of its pyramid has all eight corners outside by more than `margin`.
__device__ bool box_meets_pyramid(const DeviceScene& S, float3 ap, int f, bool mirror, float3 mn, float md, float3 lo,
                                  float3 hi, float margin)
{
    const Face fc = S.faces[f];
    for (int j = fc.tri_begin; j < fc.tri_end; ++j) {
        const TriVerts tv = S.tri_verts[S.face_tris[j]];
        float3 v[3] = {xyz(tv.v0), xyz(tv.v1), xyz(tv.v2)};
        if (mirror)
#pragma unroll
            for (int k = 0; k < 3; ++k) v[k] = v[k] - mn * (2.f * (dot(mn, v[k]) - md));
        bool separated = false;
        for (int k = 0; k < 3 && !separated; ++k) {
            float3 n = cross(v[k] - ap, v[(k + 1) % 3] - ap);
            const float l2 = dot(n, n);
            if (!(l2 > 0.f)) continue;
            n = n * rsqrtf(l2);
            if (dot(n, v[(k + 2) % 3] - ap) < 0.f) n = n * -1.f;
            bool all_out = true;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float3 q = f3((c & 1) ? hi.x : lo.x, (c & 2) ? hi.y : lo.y, (c & 4) ? hi.z : lo.z);
                if (dot(n, q - ap) >= -margin) all_out = false;
            }
            separated = all_out;
        }
        if (!separated) return true;
    }
    return false;
}

// Can any destination inside the box [lo, hi] make sequence e geometrically valid? It must lie on
// the previous image's side of the last plane, inside the pyramid from the last image S_L through the
// last face, and for order 2 also inside the pyramid from S_L through the first face mirrored across
// the last plane (unfolded, the straight line from S_2 to the destination crosses the mirror image of
// the first reflection point). False only when the whole box is separated by more than `margin`, far
// beyond FP32 error, so skipping it for every destination in the box changes no decision.
__device__ bool box_in_beam(const DeviceScene& S, const SeqEntry& e, float3 lo, float3 hi, float margin)
{
    const float3 nL = xyz(e.pL);
    const float sp = e.sL.w;
    bool same = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float3 q = f3((c & 1) ? hi.x : lo.x, (c & 2) ? hi.y : lo.y, (c & 4) ? hi.z : lo.z);
        const float sR = dot(nL, q) - e.pL.w;
        if (sp > 0.f ? sR > -margin : sR < margin) same = true;
    }
    if (!same) return false;
    const float3 ap = xyz(e.sL);
    const bool two = e.info.w == 2;
    if (!box_meets_pyramid(S, ap, two ? e.info.y : e.info.x, false, nL, e.pL.w, lo, hi, margin)) return false;
    return !two || box_meets_pyramid(S, ap, e.info.x, true, nL, e.pL.w, lo, hi, margin);
}

// Deferred FP64 settlements. A warp settles one too-close-to-call FP32 decision with all its FP64
// instructions even when one lane needs it, and FP64 issues at a small fraction of the FP32 rate, so
// the filters queue such cases and a dense kernel settles them afterwards, 32 per warp. q == nullptr,
// or a full queue, settles inline instead.
struct RefineQ {
    int4* q;
    int cap;
    unsigned* cnt;
};

// The validation work list written by the candidate search itself: every warp's 32 lanes are
// Morton-adjacent destinations testing one sequence at a time, so the lanes that pass form a run of
// one sequence over neighbouring destinations; a warp stages its runs in shared memory and appends
// them in chunks (one atomic per chunk). r == nullptr: no list (it is built afterwards).
struct DenseOut {
    int* r;
    int* slot;
    int* seq;                    // the candidate's sequence index (its slot's content)
    unsigned long long* cnt;
};
#ifndef RISRT_DENSE_BUF
#define RISRT_DENSE_BUF 192
#endif
constexpr int kDenseBuf = RISRT_DENSE_BUF;   // staged work-list entries per warp (must be >= 32)

// Margin of the beam culling for a box: far beyond the FP32 error of the plane and corner arithmetic.
__device__ __forceinline__ float cull_margin(float3 lo, float3 hi)
{
    return 1e-3f + 1e-5f * (fabsf(lo.x) + fabsf(lo.y) + fabsf(lo.z) + fabsf(hi.x) + fabsf(hi.y) + fabsf(hi.z));
}

// Super-patches: kSuperRx destinations consecutive in Morton order. Their bounding boxes (one block each).
constexpr int kSuperRx = 1024;
__global__ void k_patch_boxes(const float* __restrict__ dst_xyz, const int* __restrict__ order, int64_t n_dst,
                              float4* __restrict__ boxes)
{
    __shared__ float3 wlo[8], whi[8];
    const float inf = __int_as_float(0x7f800000);
    float3 lo = f3(inf, inf, inf), hi = f3(-inf, -inf, -inf);
    const int64_t b0 = blockIdx.x * (int64_t)kSuperRx;
    for (int i = threadIdx.x; i < kSuperRx && b0 + i < n_dst; i += blockDim.x) {
        const int64_t r = order[b0 + i];
        const float3 q = f3(dst_xyz[3 * r], dst_xyz[3 * r + 1], dst_xyz[3 * r + 2]);
        lo = f3(fminf(lo.x, q.x), fminf(lo.y, q.y), fminf(lo.z, q.z));
        hi = f3(fmaxf(hi.x, q.x), fmaxf(hi.y, q.y), fmaxf(hi.z, q.z));
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = f3(fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o)), fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o)),
                fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o)));
        hi = f3(fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o)), fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o)),
                fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o)));
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        wlo[warp] = lo;
        whi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = f3(fminf(lo.x, wlo[w].x), fminf(lo.y, wlo[w].y), fminf(lo.z, wlo[w].z));
            hi = f3(fmaxf(hi.x, whi[w].x), fmaxf(hi.y, whi[w].y), fmaxf(hi.z, whi[w].z));
        }
        boxes[2 * blockIdx.x] = make_float4(lo.x, lo.y, lo.z, 0.f);
        boxes[2 * blockIdx.x + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
    }
}

// Groups of kGroupSuper consecutive super-patches: the union of their boxes, and in lo.w a margin
// above every member's (plus a slack far beyond FP32 error), so that a sequence culled for the group
// is culled for each member: box_in_beam only rejects a box wholly separated by more than the margin,
// and a separation of the group's box by a larger margin separates every member box too.
constexpr int kGroupSuper = 16;
__global__ void k_group_boxes(const float4* __restrict__ sp_box, int64_t n_super, int64_t n_groups, float4* __restrict__ g_box)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    const float inf = __int_as_float(0x7f800000);
    float3 lo = f3(inf, inf, inf), hi = f3(-inf, -inf, -inf);
    float m = 0.f;
    for (int64_t sp = g * kGroupSuper; sp < min(n_super, (g + 1) * kGroupSuper); ++sp) {
        const float3 a = xyz(sp_box[2 * sp]), b = xyz(sp_box[2 * sp + 1]);
        lo = f3(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, a.z));
        hi = f3(fmaxf(hi.x, b.x), fmaxf(hi.y, b.y), fmaxf(hi.z, b.z));
        m = fmaxf(m, cull_margin(a, b));
    }
    g_box[2 * g] = make_float4(lo.x, lo.y, lo.z, m + 1e-4f);
    g_box[2 * g + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
}

// One bit per (box, sequence): can a destination in the box make the sequence valid (box_in_beam)?
// Word w of box p covers sequences 32w .. 32w + 31. margin_in_w: the boxes carry their margin in
// lo.w (group boxes), else cull_margin of the box.
__global__ void k_seq_cull(DeviceScene S, const SeqEntry* __restrict__ seqs, int n_seq, const float4* __restrict__ boxes,
                           int64_t n_super, int words, unsigned* __restrict__ mask, const int64_t* __restrict__ n_dev,
                           bool margin_in_w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (n_dev) n_seq = (int)min((int64_t)n_seq, *n_dev);   // the table's size on the device (asynchronous traces)
    for (int64_t sp = blockIdx.y; sp < n_super; sp += gridDim.y) {
        bool k = false;
        if (i < n_seq) {
            const float4 l4 = boxes[2 * sp];
            const float3 lo = xyz(l4), hi = xyz(boxes[2 * sp + 1]);
            k = box_in_beam(S, seqs[i], lo, hi, margin_in_w ? l4.w : cull_margin(lo, hi));
        }
        const unsigned b = __ballot_sync(0xffffffffu, k);
        if ((threadIdx.x & 31) == 0 && (i >> 5) < words) mask[sp * words + (i >> 5)] = b;
    }
}

// Second level: one bit per (super-patch, position in its group's survivor list): box_in_beam of the
// survivor on the super-patch box. Blocks past the group's count exit at once (k_mask_compact reads
// only the words its count covers).
__global__ void k_seq_cull2(DeviceScene S, const SeqEntry* __restrict__ seqs, const float4* __restrict__ boxes,
                            int64_t n_super, const int* __restrict__ g_list, const int* __restrict__ g_cnt,
                            int64_t stride, int words, unsigned* __restrict__ mask)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t sp = blockIdx.y; sp < n_super; sp += gridDim.y) {
        const int64_t g = sp / kGroupSuper;
        const int n = g_cnt[g];
        if ((int)(blockIdx.x * blockDim.x) >= n) continue;        // uniform per block
        bool k = false;
        if (i < n) {
            const float3 lo = xyz(boxes[2 * sp]), hi = xyz(boxes[2 * sp + 1]);
            k = box_in_beam(S, seqs[g_list[g * stride + i]], lo, hi, cull_margin(lo, hi));
        }
        const unsigned b = __ballot_sync(0xffffffffu, k);
        if ((threadIdx.x & 31) == 0 && (i >> 5) < words) mask[sp * words + (i >> 5)] = b;
    }
}

// Indices of the set bits of each super-patch's sequence mask, in increasing order (one block of 256
// threads per super-patch): list[p * stride + i] for i < cnt[p].
constexpr int kCompactThreads = 1024;
__global__ void __launch_bounds__(kCompactThreads) k_mask_compact(const unsigned* __restrict__ mask, int words, int64_t n_super,
                                                                  int64_t stride, int* __restrict__ list,
                                                                  int* __restrict__ cnt, const int* __restrict__ g_list,
                                                                  const int* __restrict__ g_cnt)
{
    __shared__ int wsum[kCompactThreads / 32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t sp = blockIdx.x; sp < n_super; sp += gridDim.x) {
        const unsigned* m = mask + sp * words;
        // second level: bits are positions in the group's survivor list, valid up to its count
        const int nw = g_list ? min(words, (g_cnt[sp / kGroupSuper] + 31) / 32) : words;
        const int* remap = g_list ? g_list + (sp / kGroupSuper) * stride : nullptr;
        int* out = list + sp * stride;
        int total = 0;
        for (int r0 = 0; r0 < nw; r0 += kCompactThreads) {   // rounds of one word per thread
            const int wi = r0 + (int)threadIdx.x;
            const unsigned mw = wi < nw ? m[wi] : 0u;
            const int c = __popc(mw);
            int x = c;                                        // inclusive scan over the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            if (warp == 0) {                                  // inclusive scan of the warp totals
                int v = wsum[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, v, o);
                    if (lane >= o) v += y;
                }
                wsum[lane] = v;
            }
            __syncthreads();
            const int wbase = total + (warp > 0 ? wsum[warp - 1] : 0);
            // the warp's 32 words in order, each word's set bits written by the lanes they name
            for (int j = 0; j < 32; ++j) {
                const unsigned wj = __shfl_sync(FULL, mw, j);
                const int oj = __shfl_sync(FULL, x - c, j);
                if ((wj >> lane) & 1u) {
                    const int idx = (r0 + warp * 32 + j) * 32 + lane;
                    out[wbase + oj + __popc(wj & ((1u << lane) - 1u))] = remap ? remap[idx] : idx;
                }
            }
            total += wsum[kCompactThreads / 32 - 1];
            __syncthreads();
        }
        if (threadIdx.x == 0) cnt[sp] = total;
    }
}

template <bool SMEM_FACES>
__global__ void __launch_bounds__(kCandThreads)
k_candidates(DeviceScene S, const float* __restrict__ dst_xyz, int64_t n_dst, const int* __restrict__ order, d3 src,
             const SeqEntry* __restrict__ seqs, const SeqEntryD* __restrict__ seqd, int n_seq,
             float tol_base, int* __restrict__ cand, int* __restrict__ cand_cnt, int cap,
             int* __restrict__ overflow, unsigned long long* __restrict__ refines, const int* __restrict__ slist,
             const int* __restrict__ slist_cnt, int64_t slist_stride, RefineQ rq, DenseOut dl,
             const int64_t* __restrict__ n_dev)
{
    if (n_dev) n_seq = (int)min((int64_t)n_seq, *n_dev);   // the table's size on the device (asynchronous traces)
    __shared__ int2 dbuf[kCandThreads / 32][kDenseBuf];
    __shared__ int dseq[kCandThreads / 32][kDenseBuf];
    __shared__ SeqEntry sh[kCandThreads];
    __shared__ int sh_idx[kCandThreads];
    __shared__ unsigned char kept[kCandThreads];
    __shared__ int wcnt[kCandThreads / 32];
    __shared__ float3 sh_R[kCandThreads];
    __shared__ float3 box[2];
    extern __shared__ FaceTest sh_faces[];
    if (SMEM_FACES)
        for (int f = threadIdx.x; f < S.n_faces; f += blockDim.x) sh_faces[f] = S.face_test[f];
    // destinations in spatial (Morton) order, so a block covers a compact patch
    const int64_t ri = blockIdx.x * (int64_t)kCandThreads + threadIdx.x;
    const bool active = ri < n_dst;
    const int64_t r = active ? (order ? (int64_t)order[ri] : ri) : 0;
    const float3 R = active ? f3(dst_xyz[3 * r], dst_xyz[3 * r + 1], dst_xyz[3 * r + 2]) : f3(0.f, 0.f, 0.f);
    sh_R[threadIdx.x] = R;
    __syncthreads();
    if (threadIdx.x < 2) {
        const int64_t rem = n_dst - blockIdx.x * (int64_t)kCandThreads;
        const int n_act = rem < kCandThreads ? (int)rem : kCandThreads;
        float3 b = sh_R[0];
        for (int i = 1; i < n_act; ++i) {
            const float3 q = sh_R[i];
            b = threadIdx.x == 0 ? f3(fminf(b.x, q.x), fminf(b.y, q.y), fminf(b.z, q.z))
                                 : f3(fmaxf(b.x, q.x), fmaxf(b.y, q.y), fmaxf(b.z, q.z));
        }
        box[threadIdx.x] = b;
    }
    __syncthreads();
    const float3 blo = box[0], bhi = box[1];
    const float margin = cull_margin(blo, bhi);
    // the sequences that may reach this block's super-patch (kSuperRx / kCandThreads blocks per
    // super-patch), or all of them without a list; rounds of kCandThreads staged and beam-tested
    // against this block's box, then the survivors compacted so every thread loops over them only
    const int64_t spi = blockIdx.x / (kSuperRx / kCandThreads);
    const int* lst = slist ? slist + spi * slist_stride : nullptr;
    const int lcnt = slist ? slist_cnt[spi] : n_seq;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this warp's box over its active destinations
    const float inf = __int_as_float(0x7f800000);
    float3 wlo = active ? R : f3(inf, inf, inf), whi = active ? R : f3(-inf, -inf, -inf);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wlo = f3(fminf(wlo.x, __shfl_xor_sync(0xffffffffu, wlo.x, o)), fminf(wlo.y, __shfl_xor_sync(0xffffffffu, wlo.y, o)),
                 fminf(wlo.z, __shfl_xor_sync(0xffffffffu, wlo.z, o)));
        whi = f3(fmaxf(whi.x, __shfl_xor_sync(0xffffffffu, whi.x, o)), fmaxf(whi.y, __shfl_xor_sync(0xffffffffu, whi.y, o)),
                 fmaxf(whi.z, __shfl_xor_sync(0xffffffffu, whi.z, o)));
    }
    const bool warp_any = __any_sync(0xffffffffu, active);
    const float wmargin = warp_any ? cull_margin(wlo, whi) : 0.f;
    int wn = 0;                                      // staged work-list entries of this warp (uniform)
    auto flush = [&]() {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0 && wn > 0) base = atomicAdd(dl.cnt, (unsigned long long)wn);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int k = lane; k < wn; k += 32) {
            const int2 v = dbuf[warp][k];
            dl.r[base + k] = v.x;
            dl.slot[base + k] = v.y;
            dl.seq[base + k] = dseq[warp][k];
        }
        __syncwarp();
        wn = 0;
    };
    for (int p0 = blockIdx.y * kCandThreads; p0 < lcnt; p0 += gridDim.y * kCandThreads) {
        __syncthreads();
        const int pi = p0 + threadIdx.x;
        bool k = false;
        if (pi < lcnt) {
            const int si = lst ? lst[pi] : pi;
            const SeqEntry e = seqs[si];
            sh[threadIdx.x] = e;
            sh_idx[threadIdx.x] = si;
            k = box_in_beam(S, e, blo, bhi, margin);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, k);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int base = 0, n_kept = 0;
#pragma unroll
        for (int w = 0; w < kCandThreads / 32; ++w) {
            base += w < warp ? wcnt[w] : 0;
            n_kept += wcnt[w];
        }
        if (k) kept[base + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)threadIdx.x;
        __syncthreads();
        // a third level for first-order sequences: each warp's own box (32 Morton-adjacent
        // destinations) against the kept ones, 32 at a time; the warp's destinations then test only the
        // sequences that pass (second-order sequences, whose beam test costs two pyramids and whose
        // beams are wide against a block in the scenes measured, are not culled again)
        for (int c0 = 0; c0 < n_kept && warp_any; c0 += 32) {
            bool wk = c0 + lane < n_kept;
            if (wk) {
                const SeqEntry& q = sh[kept[c0 + lane]];
                wk = q.info.w != 1 || box_in_beam(S, q, wlo, whi, wmargin);
            }
            for (unsigned bits = __ballot_sync(0xffffffffu, wk); bits; bits &= bits - 1) {
                const int j = kept[c0 + __ffs(bits) - 1];
                const int sidx = sh_idx[j];
                const SeqEntry& e = sh[j];
                // the geometric tests (A)-(D); false when they reject, or when the decision is queued
                auto passes = [&]() -> bool {
                    // (A)
                    const float sR = dot(xyz(e.pL), R) - e.pL.w;
                    const float sp = e.sL.w;
                    const bool clearA = fabsf(sR) > tol_base && fabsf(sp) > tol_base;
                    if (clearA && sp * sR < 0.f) return false;
                    bool unsure = !clearA;
                    // (B) last reflection point P = R + t (S_L - R), t = sR / (sR + sp)
                    const float den = sR + sp;
                    const float3 d = xyz(e.sL) - R;
                    const float iden = __frcp_rn(den);
                    const float t = sR * iden;
                    const float3 P = R + d * t;
                    const float d2 = dot(d, d);
                    const float cond = d2 * rsqrtf(d2) * fabsf(iden);   // |d| / |den| (a few ulps suffice: tol has margin)
                    const float tol = tol_base * fminf(cond, 1e6f);
                    const int k = e.info.w;
                    const int cB = face_class<SMEM_FACES>(S, sh_faces, k == 2 ? e.info.y : e.info.x, P, tol);
                    if (cB == 0) return false;
                    unsure |= cB == 2;
                    if (k == 2) {
                        // (C)
                        const float s1P = dot(xyz(e.p1), P) - e.p1.w;
                        const float ssrc = e.s1.w;
                        const bool clearC = fabsf(s1P) > tol && fabsf(ssrc) > tol_base;
                        if (clearC && s1P * ssrc < 0.f) return false;
                        unsure |= !clearC;
                        // (D) P1 = P + t1 (S1 - P), t1 = s1P / (s1P + ssrc)
                        const float den1 = s1P + ssrc;
                        const float3 d1 = xyz(e.s1) - P;
                        const float iden1 = __frcp_rn(den1);
                        const float3 P1 = P + d1 * (s1P * iden1);
                        const float d12 = dot(d1, d1);
                        const float cond1 = d12 * rsqrtf(d12) * fabsf(iden1);
                        const float tol1 = tol * fminf(cond1, 1e6f) + tol_base;
                        const int cD = face_class<SMEM_FACES>(S, sh_faces, e.info.x, P1, tol1);
                        if (cD == 0) return false;
                        unsure |= cD == 2;
                    }
                    if (unsure) {
                        if (rq.q) {
                            const unsigned pos = atomicAdd(rq.cnt, 1u);
                            if (pos < (unsigned)rq.cap) {
                                rq.q[pos] = make_int4((int)r, sidx, 0, 0);
                                return false;
                            }
                        }
                        atomicAdd(refines, 1ull);
                        d3 pts[4];
                        const d3 Rd = D3((double)R.x, (double)R.y, (double)R.z);
                        if (!seq_geom_fp64(S, src, Rd, e.info, seqd[sidx], pts)) return false;
                    }
                    return true;
                };
                bool pass = active && passes();
                int slot = -1;
                if (pass) {
                    slot = atomicAdd(&cand_cnt[r], 1);
                    if (slot < cap) {
                        cand[r * (int64_t)cap + slot] = sidx;
                    } else {
                        atomicExch(overflow, 1);
                        pass = false;
                    }
                }
                if (dl.r) {                              // this warp's run of sequence sidx
                    const unsigned b = __ballot_sync(0xffffffffu, pass);
                    const int nb = __popc(b);
                    if (nb) {
                        if (wn + nb > kDenseBuf) flush();
                        if (pass) {
                            const int k = wn + __popc(b & ((1u << lane) - 1u));
                            dbuf[warp][k] = make_int2((int)r, slot);
                            dseq[warp][k] = sidx;
                        }
                        wn += nb;
                    }
                }
            }
        }
    }
    if (dl.r) flush();
}

// Settle the queued candidate decisions in FP64 (seq_geom_fp64, the same check as the inline path).
__global__ void k_refine_cand(DeviceScene S, const float* __restrict__ dst_xyz, d3 src, const SeqEntry* __restrict__ seqs,
                              const SeqEntryD* __restrict__ seqd, RefineQ rq, int* __restrict__ cand,
                              int* __restrict__ cand_cnt, int cap, int* __restrict__ overflow,
                              unsigned long long* __restrict__ refines, DenseOut dl)
{
    const unsigned n = min(*rq.cnt, (unsigned)rq.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(refines, (unsigned long long)n);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 q = rq.q[i];
        const int64_t r = q.x;
        const float3 R = f3(dst_xyz[3 * r], dst_xyz[3 * r + 1], dst_xyz[3 * r + 2]);
        d3 pts[4];
        if (!seq_geom_fp64(S, src, D3((double)R.x, (double)R.y, (double)R.z), seqs[q.y].info, seqd[q.y], pts)) continue;
        const int slot = atomicAdd(&cand_cnt[r], 1);
        if (slot < cap) {
            cand[r * (int64_t)cap + slot] = q.y;
            if (dl.r) {                              // appended to the work list as well
                const unsigned long long pos = atomicAdd(dl.cnt, 1ull);
                dl.r[pos] = (int)r;
                dl.slot[pos] = slot;
                dl.seq[pos] = q.y;
            }
        } else {
            atomicExch(overflow, 1);
        }
    }
}

// Dense list of the (destination, slot) pairs holding a geometric candidate, receiver-major.
__global__ void k_cand_counts(const int* __restrict__ cand_cnt, int64_t n_dst, int cap, int64_t* __restrict__ out)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n_dst) out[r] = min(cand_cnt[r], cap);
    if (r == n_dst) out[r] = 0;
}

__global__ void k_dense_list(const int* __restrict__ cand_cnt, const int* __restrict__ cand, const int64_t* __restrict__ off,
                             int64_t n_dst, int cap, int* __restrict__ dense_r, int* __restrict__ dense_slot,
                             int* __restrict__ dense_seq)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= n_dst) return;
    const int n = min(cand_cnt[r], cap);
    const int64_t o = off[r];
    for (int slot = lane; slot < n; slot += 32) {
        dense_r[o + slot] = (int)r;
        dense_slot[o + slot] = slot;
        dense_seq[o + slot] = cand[r * (int64_t)cap + slot];
    }
}

// FP32 reflection points of a candidate (the same back-trace as the candidate filter): q0 = the last
// point P (next to the destination R), q1 = the first point P1 (order 2; P for order 1); w holds a
// first-order bound on each point's error from the FP32 roundings of the inputs (images, planes and
// signed distances are FP32 copies of FP64 values) and of these operations, doubled.
__device__ __forceinline__ void path_points(const SeqEntry& e, float3 R, float4& q0, float4& q1)
{
    const float sR = dot(xyz(e.pL), R) - e.pL.w;
    const float den = sR + e.sL.w;
    const float t = sR / den;
    const float3 d = xyz(e.sL) - R;
    const float3 P = R + d * t;
    const float eps = 5.9604645e-8f;
    auto l1 = [](float3 a) { return fabsf(a.x) + fabsf(a.y) + fabsf(a.z); };
    const float mag = l1(R) + l1(xyz(e.sL)) + fabsf(e.pL.w);
    const float e_s = 8.f * eps * mag;
    const float e_den = e_s + 2.f * eps * fabsf(e.sL.w) + eps * fabsf(den);
    const float e_t = (e_s + fabsf(t) * e_den) / fabsf(den) + 2.f * eps * fabsf(t);
    const float errP = l1(d) * e_t + (fabsf(t) + 1.f) * 4.f * eps * mag;
    float3 P1 = P;
    float errP1 = errP;
    if (e.info.w == 2) {
        const float s1P = dot(xyz(e.p1), P) - e.p1.w;
        const float den1 = s1P + e.s1.w;
        const float t1 = s1P / den1;
        const float3 d1 = xyz(e.s1) - P;
        P1 = P + d1 * t1;
        const float mag1 = l1(P) + l1(xyz(e.s1)) + fabsf(e.p1.w);
        const float e_s1 = l1(xyz(e.p1)) * errP + 8.f * eps * mag1;
        const float e_den1 = e_s1 + 2.f * eps * fabsf(e.s1.w) + eps * fabsf(den1);
        const float e_t1 = (e_s1 + fabsf(t1) * e_den1) / fabsf(den1) + 2.f * eps * fabsf(t1);
        errP1 = errP + l1(d1) * e_t1 + fabsf(t1) * (errP + 4.f * eps * l1(xyz(e.s1))) + 4.f * eps * mag1;
    }
    q0 = make_float4(P.x, P.y, P.z, 2.f * errP);
    q1 = make_float4(P1.x, P1.y, P1.z, 2.f * errP1);
}

// ------------------------------------------------------------------------------------------------
// Visibility maps from a fixed source S (the RIS centre for the Rx leg, the Tx for environment
// paths): every path's first segment runs from S to its first reflection point on face f1. Per cell
// of f1's grid, enlarged by kMapDelta, the pyramid from S through the cell contains all those
// segments; 1 = no triangle (other than of src_face and f1) can meet the pyramid, so every such
// segment is unblocked; 2 = one triangle meets every ray of the pyramid inside it, at least
// kSegEps + margin from both ends, so every such segment is blocked; 0 = undecided (traverse). The
// walk stops at the first triangle that may meet the pyramid: it either covers the whole pyramid
// (2) or leaves the cell undecided, which bounds the work per cell.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool box_outside(float4 lo, float4 hi, float3 n, float3 q, float m)
{
    const float3 c = f3(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z));
    const float3 h = f3(0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z));
    return dot(n, c - q) - (fabsf(n.x) * h.x + fabsf(n.y) * h.y + fabsf(n.z) * h.z) > m;
}

// Does triangle (V0, V1, V2) meet every ray S -> C_k (k < 4) of the pyramid inside itself, by at
// least m from its edges, with hit parameters t such that t D and (1 - t) D stay above kSegEps + m,
// D the distance of S to the cell's plane? Then, by convexity of the central projection of the cell,
// it blocks every segment from S to a point of the cell. FP32: m is far above its rounding.
__device__ bool tri_covers(const float3* C, float3 Sf, const TriVerts& tv, float D, float m)
{
    const float3 V[3] = {xyz(tv.v0), xyz(tv.v1), xyz(tv.v2)};
    float3 nT = cross(V[1] - V[0], V[2] - V[0]);
    const float nn2 = dot(nT, nT);
    if (!(nn2 > 0.f)) return false;
    nT = nT * rsqrtf(nn2);
    float tmin = 3e38f, tmax = -3e38f, sgn = 0.f;
    for (int k = 0; k < 4; ++k) {
        const float3 dk = C[k] - Sf;
        const float den = dot(nT, dk);
        if (fabsf(den) <= 1e-3f * sqrtf(dot(dk, dk))) return false;
        if (sgn != 0.f && (den > 0.f) != (sgn > 0.f)) return false;
        sgn = den;
        const float t = dot(nT, V[0] - Sf) / den;
        tmin = fminf(tmin, t);
        tmax = fmaxf(tmax, t);
        const float3 X = Sf + dk * t;
        for (int e = 0; e < 3; ++e) {
            const float3 ed = V[(e + 1) % 3] - V[e];
            if (dot(cross(ed, X - V[e]), nT) < m * sqrtf(dot(ed, ed))) return false;
        }
    }
    return tmin * D >= kSegEps + m && (1.f - tmax) * D >= kSegEps + m;
}

// The same for a face with a convex outline (one triangle or a convex two-triangle quad): every ray
// S -> C_k meets the face plane inside the outline by at least m, so every segment from S to the
// cell meets one of the face's triangles (the outline is their union).
__device__ bool face_covers(const DeviceScene& S, int ft, const float3* C, float3 Sf, float D, float m)
{
    const FaceTest ot = S.face_test[ft];
    if (ot.n == 0) return false;
    const float4 pl = S.faces[ft].plane32;
    const float3 nT = xyz(pl);
    float tmin = 3e38f, tmax = -3e38f, sgn = 0.f;
    for (int k = 0; k < 4; ++k) {
        const float3 dk = C[k] - Sf;
        const float den = dot(nT, dk);
        if (fabsf(den) <= 1e-3f * sqrtf(dot(dk, dk))) return false;
        if (sgn != 0.f && (den > 0.f) != (sgn > 0.f)) return false;
        sgn = den;
        const float t = (pl.w - dot(nT, Sf)) / den;
        tmin = fminf(tmin, t);
        tmax = fmaxf(tmax, t);
        const float3 X = Sf + dk * t;
        for (int i = 0; i < ot.n; ++i)
            if (dot(xyz(ot.e[i]), X) - ot.e[i].w < m) return false;
    }
    return tmin * D >= kSegEps + m && (1.f - tmax) * D >= kSegEps + m;
}

constexpr int kMapLeafBudget = 8;    // triangles that may meet a cell's pyramid examined before giving up
#ifndef RISRT_MAP_NODE_BUDGET
#define RISRT_MAP_NODE_BUDGET 32     // four-wide BVH nodes visited per cell before giving up (measured: bounds the slowest cells)
#endif

// Classify the pyramid with apex A and base quad C[0..3] (a convex quad on a plane with unit normal
// nb pointing away from A, at distance D from A), ignoring triangles of faces ig0 and ig1: 1 = no
// triangle can meet it, 2 = one face (or triangle) meets every ray from A to the base with the
// margins of face_covers / tri_covers, 0 = undecided. The walk visits children entered first along
// the centre ray first and gives up after kMapLeafBudget candidate triangles or
// RISRT_MAP_NODE_BUDGET nodes.
__device__ uint8_t classify_pyramid(const DeviceScene& S, bool in_box, float3 A, const float3* C, float3 nb, float D,
                                    int ig0, int ig1, float margin)
{
    int stack[64];
    int sp = 0;
    int cur = occ_start(S, in_box, stack, sp);
    if (cur == kNoRoot) return 1;
    // the pyramid's planes, outside = positive side: four through A, the fifth the base plane, the
    // sixth across the axis at A (or behind A by as much as a base corner lies behind it), which
    // culls what lies behind the apex: boxes there straddle the side planes one by one
    const float3 cdir = (C[0] + C[2]) * 0.5f - A;
    const float3 ax = cdir * rsqrtf(fmaxf(dot(cdir, cdir), 1e-30f));
    float3 pn[6];
    float pmin = 0.f;
    for (int k = 0; k < 4; ++k) {
        float3 n = cross(C[k] - A, C[(k + 1) % 4] - A);
        n = n * rsqrtf(fmaxf(dot(n, n), 1e-30f));
        if (dot(n, C[(k + 2) % 4] - A) > 0.f) n = n * -1.f;
        pn[k] = n;
        pmin = fminf(pmin, dot(ax, C[k] - A));
    }
    pn[4] = nb;
    pn[5] = ax * -1.f;
    const float3 Acap = A + ax * pmin;
    auto pq = [&](int k) { return k < 4 ? A : (k == 4 ? C[0] : Acap); };
    const int g0 = ig0 >= 0 ? ig0 : -3, g1 = ig1 >= 0 ? ig1 : -3;
    bool mixed = false, covered = false;
    int budget = 0, visits = 0;
    const float3 cinv = f3(safe_inv(cdir.x), safe_inv(cdir.y), safe_inv(cdir.z));
    while (true) {
        if (cur < 0) {
            const int L = ~cur;
            const int ft = S.tri_face[L];
            if (ft != ig0 && ft != ig1) {
                const TriVerts tv = S.tri_verts[L];
                const float3 V[3] = {xyz(tv.v0), xyz(tv.v1), xyz(tv.v2)};
                bool sep = false;
                for (int k = 0; k < 6 && !sep; ++k) {
                    const float3 q = pq(k);
                    sep = dot(pn[k], V[0] - q) > margin && dot(pn[k], V[1] - q) > margin && dot(pn[k], V[2] - q) > margin;
                }
                if (!sep) {                     // the pyramid's five corners on one side of the triangle's plane
                    float3 nT = cross(V[1] - V[0], V[2] - V[0]);
                    nT = nT * rsqrtf(fmaxf(dot(nT, nT), 1e-30f));
                    const float s0 = dot(nT, A - V[0]);
                    bool pos = s0 > margin, neg = s0 < -margin;
                    for (int k = 0; k < 4; ++k) {
                        const float sk = dot(nT, C[k] - V[0]);
                        pos = pos && sk > margin;
                        neg = neg && sk < -margin;
                    }
                    sep = pos || neg;
                }
                if (!sep) {                     // a covering face decides; a few misses leave it undecided
                    mixed = true;
                    covered = face_covers(S, ft, C, A, D, margin) || tri_covers(C, A, tv, D, margin);
                    if (covered || ++budget >= kMapLeafBudget) break;
                }
            }
            if (sp == 0) break;
            cur = stack[--sp];
            continue;
        }
        if (++visits > RISRT_MAP_NODE_BUDGET) {
            mixed = true;
            covered = false;
            break;
        }
        if (sp + 3 > 64) {                      // never expected; undecided
            mixed = true;
            covered = false;
            break;
        }
        const Bvh4Node nd = S.nodes4[cur];
        float t[4];
        int ch[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ch[q] = __float_as_int(nd.lo[q].w);
            const int fq = __float_as_int(nd.hi[q].w);
            bool in = ch[q] != kNoChild && fq != g0 && fq != g1;
            for (int k = 0; k < 6 && in; ++k) in = !box_outside(nd.lo[q], nd.hi[q], pn[k], pq(k), margin);
            // entered children in the order the centre ray meets them (boxes it misses last)
            t[q] = in ? fminf(box_entry(nd.lo[q], nd.hi[q], A, cinv), 1e30f) : 3e38f;
        }
        auto cs = [&](int i, int j) {
            if (t[j] < t[i]) {
                const float tt = t[i]; t[i] = t[j]; t[j] = tt;
                const int cc = ch[i]; ch[i] = ch[j]; ch[j] = cc;
            }
        };
        cs(0, 1); cs(2, 3); cs(0, 2); cs(1, 3); cs(1, 2);
        for (int q = 3; q >= 1; --q)
            if (t[q] < 2e38f) stack[sp++] = ch[q];
        if (t[0] < 2e38f) {
            cur = ch[0];
        } else {
            if (sp == 0) break;
            cur = stack[--sp];
        }
    }
    return covered ? 2 : (mixed ? 0 : 1);
}

__global__ void __launch_bounds__(128) k_src_map(DeviceScene S, d3 src, int src_face, float margin, uint8_t* __restrict__ map)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= S.n_cells) return;
    const int f = S.cell_face[c];
    const FaceGrid g = S.face_grid[f];
    const int idx = (int)(c - g.off);
    const int ci = idx / g.nv, cj = idx % g.nv;
    const Face fc = S.faces[f];
    const double sd = dot(ld3(fc.plane), src) - fc.plane.w;   // signed distance of S to the face plane
    uint8_t state = 0;
    if (fabs(sd) > 1e-2 && fc.tri_end > fc.tri_begin && f != src_face) {
        const float3 o = xyz(g.o), u = xyz(g.u), v = xyz(g.v);
        const float a0 = g.u.w + ci * g.o.w - kMapDelta, a1 = g.u.w + (ci + 1) * g.o.w + kMapDelta;
        const float b0 = g.v.w + cj * g.dv - kMapDelta, b1 = g.v.w + (cj + 1) * g.dv + kMapDelta;
        const float3 C[4] = {o + u * a0 + v * b0, o + u * a1 + v * b0, o + u * a1 + v * b1, o + u * a0 + v * b1};
        const float3 nb = sd > 0.0 ? f3(-(float)fc.plane.x, -(float)fc.plane.y, -(float)fc.plane.z)
                                   : f3((float)fc.plane.x, (float)fc.plane.y, (float)fc.plane.z);
        // the map answers segments from the source to points of face f, which lie in the scene box
        state = classify_pyramid(S, in_scene_box(S, src), to_f(src), C, nb, (float)fabs(sd), src_face, f, margin);
    }
    map[c] = state;
}

// Bounds (a_min, a_max, b_min, b_max) of the element centres in the RIS frame (one block).
__global__ void k_elem_bounds(const float4* __restrict__ elem, int M, float4* __restrict__ out)
{
    __shared__ float4 red[256];
    float4 b = make_float4(3e38f, -3e38f, 3e38f, -3e38f);
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 e = elem[m];
        b = make_float4(fminf(b.x, e.x), fmaxf(b.y, e.x), fminf(b.z, e.y), fmaxf(b.w, e.y));
    }
    red[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const float4 q = red[threadIdx.x + o];
            b = make_float4(fminf(b.x, q.x), fmaxf(b.y, q.y), fminf(b.z, q.z), fmaxf(b.w, q.w));
            red[threadIdx.x] = b;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Per tile: the corners of its rectangle (element-centre bounds enlarged by kMapDelta) computed in
// FP64 and rounded to FP32, and in c[0].w whether all four lie in the scene box (1) or not (0).
struct TileGeom {
    float4 c[4];
};
constexpr int kTileDeferCap = 1 << 20;   // tile rays queued for the FP64 settlement (more settle in place)
__global__ void k_tile_geom(DeviceScene S, Frame fr, const float4* __restrict__ tile_bb, int T, TileGeom* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const d3 c = fr_c(fr), t1 = fr_t1(fr), t2 = fr_t2(fr);
    const float4 b = tile_bb[t];
    const double a0 = b.x - kMapDelta, a1 = b.y + kMapDelta, b0 = b.z - kMapDelta, b1 = b.w + kMapDelta;
    const d3 Cd[4] = {c + t1 * a0 + t2 * b0, c + t1 * a1 + t2 * b0, c + t1 * a1 + t2 * b1, c + t1 * a0 + t2 * b1};
    bool in_box = true;
    TileGeom g;
    for (int k = 0; k < 4; ++k) {
        const float3 q = to_f(Cd[k]);
        g.c[k] = make_float4(q.x, q.y, q.z, 0.f);
        in_box = in_box && in_scene_box(S, Cd[k]);
    }
    g.c[0].w = in_box ? 1.f : 0.f;
    out[t] = g;
}

// The class of the pyramid from receiver R through a rectangle of the RIS plane (g: its FP32 corners
// and in-box flag): 1 all visible, 2 all blocked, 0 undecided; in_box: R and the rectangle lie in the
// scene box, so every segment from R to the rectangle does too. The distance to the RIS plane is
// taken in FP32: the classification works with margins, so its decisions are sound either way.
__device__ __forceinline__ uint8_t rect_class(const DeviceScene& S, float3 R, float3 c32, float3 n32, const TileGeom& g,
                                              int host_face, float margin, bool& in_box)
{
    in_box = g.c[0].w != 0.f && in_scene_box(S, R);
    const float sd = dot(n32, R - c32);
    if (!(fabsf(sd) > 1e-2f)) return 0;
    const float3 C[4] = {xyz(g.c[0]), xyz(g.c[1]), xyz(g.c[2]), xyz(g.c[3])};
    return classify_pyramid(S, in_box, R, C, sd > 0.f ? n32 * -1.f : n32, fabsf(sd), host_face, -1, margin);
}

// Append the lanes whose `add` is set to list (one atomic per warp); every lane of the warp calls it.
__device__ __forceinline__ void warp_append(bool add, uint32_t value, uint32_t* list, unsigned* count)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(FULL, add);
    if (bal == 0u) return;
    unsigned base = 0;
    if (lane == __ffs(bal) - 1) base = atomicAdd(count, (unsigned)__popc(bal));
    base = __shfl_sync(FULL, base, __ffs(bal) - 1);
    if (add) list[base + __popc(bal & ((1u << lane) - 1u))] = value;
}

// Per receiver: the pyramid from R through the RIS aperture (ag: the element centres' bounding
// rectangle in the RIS plane, enlarged by kMapDelta) contains every element -> R segment, so its class
// decides all of them at once (1 all visible, 2 all blocked, 0 trace each element or tile). With und
// set, the undecided receivers are appended to und (order unspecified; *und_n counts them).
__global__ void __launch_bounds__(128) k_rx_aperture(DeviceScene S, const float* __restrict__ rx, int64_t n_rx, Frame fr,
                                                     const TileGeom* __restrict__ ag, int host_face, float margin,
                                                     uint8_t* __restrict__ state, uint32_t* __restrict__ und,
                                                     unsigned* __restrict__ und_n)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    uint8_t st = 0;
    if (r < n_rx) {
        bool in_box;
        st = rect_class(S, f3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]), to_f(fr_c(fr)), to_f(fr_n(fr)), *ag, host_face,
                        margin, in_box);
        state[r] = st;
    }
    if (und) warp_append(r < n_rx && st == 0, (uint32_t)r, und, und_n);
}

// Visibility words of the receivers whose aperture pyramid is decided, four words per thread (one
// 16-byte store when rows are multiples of four words and the array is 16-byte aligned); the
// undecided receivers' words come from k_vis_tiles and k_direct_tiles.
__global__ void k_vis_decided(int64_t n_rx, int W, int M, const uint8_t* __restrict__ state, uint32_t* __restrict__ vis)
{
    const int W4 = (W + 3) >> 2;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_rx * W4) return;
    const int64_t r = i / W4;
    const uint8_t st = state[r];
    if (st == 0) return;
    const int w0 = (int)(i % W4) * 4;
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int left = M - 32 * (w0 + k);
        v[k] = st == 2 || left <= 0 ? 0u : (left >= 32 ? 0xffffffffu : ((1u << left) - 1u));
    }
    uint32_t* row = vis + r * W;
    if ((W & 3) == 0 && ((uintptr_t)vis & 15) == 0) {
        *reinterpret_cast<uint4*>(row + w0) = make_uint4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (w0 + k < W) row[w0 + k] = v[k];
    }
}

// Per (undecided receiver u, super-tile s of four consecutive tiles): the class of the pyramid from
// the receiver through the super-tile's rectangle -> sstate[u * ST + s] (bits 0-1: the class of
// rect_class; bit 2: its in_box); undecided super-tiles are appended to swork as u * ST + s.
// Grid-stride over the device count of undecided receivers.
__global__ void __launch_bounds__(128) k_super_aperture(DeviceScene S, const float* __restrict__ rx, Frame fr,
                                                        const TileGeom* __restrict__ sg, int ST, int host_face,
                                                        float margin, const uint32_t* __restrict__ und,
                                                        const unsigned* __restrict__ und_n, uint8_t* __restrict__ sstate,
                                                        uint32_t* __restrict__ swork, unsigned* __restrict__ swork_n)
{
    const int64_t total = (int64_t)*und_n * ST;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float3 c32 = to_f(fr_c(fr)), n32 = to_f(fr_n(fr));
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total; base += stride) {   // uniform per block
        const int64_t i = base + threadIdx.x;
        uint8_t st = 0;
        if (i < total) {
            const int64_t r = und[i / ST];
            bool in_box;
            st = rect_class(S, f3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]), c32, n32, sg[i % ST], host_face, margin, in_box);
            sstate[i] = st | (in_box ? 4 : 0);
        }
        warp_append(i < total && st == 0, (uint32_t)i, swork, swork_n);
    }
}

// Per tile of an undecided super-tile (four threads per swork entry): the class of the pyramid from
// the receiver through the tile's rectangle -> tstate[u * T + t] (as sstate); undecided tiles are
// appended to work as u * T + t. Tiles of decided super-tiles are never classified (their state is
// the super-tile's). swork == nullptr: one super-tile (at most four tiles), not classified on its own
// (its rectangle is the aperture's): entry u of the undecided receivers stands for (u, 0).
__global__ void __launch_bounds__(128) k_tile_aperture(DeviceScene S, const float* __restrict__ rx, Frame fr,
                                                       const TileGeom* __restrict__ tg, int T, int ST, int host_face,
                                                       float margin, const uint32_t* __restrict__ und,
                                                       const uint32_t* __restrict__ swork, const unsigned* __restrict__ swork_n,
                                                       uint8_t* __restrict__ tstate, uint32_t* __restrict__ work,
                                                       unsigned* __restrict__ work_n)
{
    const int64_t total = (int64_t)*swork_n * 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float3 c32 = to_f(fr_c(fr)), n32 = to_f(fr_n(fr));
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total; base += stride) {   // uniform per block
        const int64_t k = base + threadIdx.x;
        uint8_t st = 0;
        bool live = false;
        int64_t i = 0;
        if (k < total) {
            const uint32_t e = swork ? swork[k >> 2] : (uint32_t)(k >> 2);
            const int64_t u = e / ST;
            const int t = (int)(e % ST) * 4 + (int)(k & 3);
            if (t < T) {
                live = true;
                i = u * T + t;
                const int64_t r = und[u];
                bool in_box;
                st = rect_class(S, f3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]), c32, n32, tg[t], host_face, margin, in_box);
                tstate[i] = st | (in_box ? 4 : 0);
            }
        }
        warp_append(live && st == 0, (uint32_t)i, work, work_n);
    }
}

// Visibility words of the undecided receivers from their tiles' classes (a decided super-tile's class,
// else the tile's own): bits of the elements whose tile is all visible (elements of undecided tiles
// are added by k_direct_tiles).
__global__ void k_vis_tiles(int W, int T, int ST, const uint32_t* __restrict__ und, const unsigned* __restrict__ und_n,
                            const int* __restrict__ word_ofs, const int2* __restrict__ word_tile,
                            const uint8_t* __restrict__ sstate, const uint8_t* __restrict__ tstate, uint32_t* __restrict__ vis)
{
    const int64_t total = (int64_t)*und_n * W;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t u = i / W;
        const int w = (int)(i % W);
        uint32_t v = 0u;
        for (int p = word_ofs[w]; p < word_ofs[w + 1]; ++p) {
            const int2 q = word_tile[p];
            int st = sstate ? sstate[u * ST + (q.x >> 2)] & 3 : 0;
            if (st == 0) st = tstate[u * T + q.x] & 3;
            if (st == 1) v |= (uint32_t)q.y;
        }
        vis[(int64_t)und[u] * W + w] = v;
    }
}

// One element -> receiver ray of an undecided tile: its FP32 end points (the element from the FP32
// frame, within a few ulps of the exact point) and whether both exact ends lie in the scene box.
struct TileRay {
    float3 a, b;
    bool in_box;
};
__device__ __forceinline__ TileRay tile_ray(const DeviceScene& S, const float* rx, int64_t r, float4 el, const Frame& fr,
                                            float3 c32, float3 t1, float3 t2, bool tile_in_box)
{
    TileRay q;
    q.a = f3(fmaf(t2.x, el.y, fmaf(t1.x, el.x, c32.x)), fmaf(t2.y, el.y, fmaf(t1.y, el.x, c32.y)),
             fmaf(t2.z, el.y, fmaf(t1.z, el.x, c32.z)));
    q.b = f3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    q.in_box = tile_in_box || (in_scene_box(S, elem_pos(fr, el)) && in_scene_box(S, q.b));
    return q;
}

// OR the bits of the lanes whose `visible` is set into their visibility words of receiver r (one
// atomic per word touched); every lane of the warp calls it.
__device__ __forceinline__ void or_visible_bits(bool visible, int m, uint32_t* vis, int64_t row)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(FULL, visible);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int word = __shfl_sync(FULL, m >> 5, leader);
        const bool mine = visible && (m >> 5) == word;
        const unsigned bits = __reduce_or_sync(FULL, mine ? 1u << (m & 31) : 0u);
        todo &= ~__ballot_sync(FULL, mine);
        if (lane == leader) atomicOr(&vis[row + word], bits);
    }
}

// Element -> receiver rays for the undecided tiles, one warp per work entry (lanes over the tile's
// elements); the visible elements' bits are OR-ed into their words. A ray with a triangle too close
// to call in FP32 and no certain hit is queued (work entry, lane) for k_direct_settle, which settles
// such rays 32 to a warp in FP64 (a full queue settles in place).
__global__ void __launch_bounds__(128) k_direct_tiles(DeviceScene S, const float* __restrict__ rx, const float4* __restrict__ elem,
                                                      int W, int T, Frame fr, int host_face, float tol_base,
                                                      const uint32_t* __restrict__ und, const int* __restrict__ tile_elem,
                                                      const uint8_t* __restrict__ tstate,
                                                      const uint32_t* __restrict__ work, const unsigned* __restrict__ work_n,
                                                      uint32_t* __restrict__ vis, int4* __restrict__ dq, int dq_cap,
                                                      unsigned* __restrict__ dq_n, unsigned long long* refines, int* err)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = *work_n;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float3 c32 = to_f(fr_c(fr)), t1 = to_f(fr_t1(fr)), t2 = to_f(fr_t2(fr));
    for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {   // uniform per warp
        const uint32_t i = work[k];
        const int64_t r = und[i / T];
        const int m = tile_elem[(int64_t)(i % T) * 32 + lane];
        bool visible = false;
        if (m >= 0) {
            const float4 el = elem[m];
            const TileRay q = tile_ray(S, rx, r, el, fr, c32, t1, t2, (tstate[i] & 4) != 0);
            auto exact = [&](d3& x, d3& y) { x = elem_pos(fr, el); y = D3(q.b.x, q.b.y, q.b.z); };
            int un[3] = {0, -1, -1};
            const bool blocked = seg_blocked_f(S, q.a, q.b, q.in_box, host_face, -1, tol_base, nullptr, err, exact,
                                               nullptr, un);
            visible = !blocked && un[0] == 0;
            if (!blocked && un[0] > 0) {
                const unsigned pos = atomicAdd(dq_n, 1u);
                if (pos < (unsigned)dq_cap)     // up to two triangles to settle, else the whole ray (-1)
                    dq[pos] = make_int4((int)i, lane, un[0] <= 2 ? un[1] : -1, un[0] <= 2 ? un[2] : -1);
                else
                    visible = !seg_blocked_f(S, q.a, q.b, q.in_box, host_face, -1, tol_base, refines, err, exact);
            }
        }
        or_visible_bits(visible, m, vis, r * W);
    }
}

// The queued rays of k_direct_tiles, one per thread: the (at most two) triangles left too close to
// call tested in FP64, or, for a ray that met more of them, the ray walked again with each settled in
// FP64; visible bits OR-ed into their words.
__global__ void k_direct_settle(DeviceScene S, const float* __restrict__ rx, const float4* __restrict__ elem, int W, int T,
                                Frame fr, int host_face, float tol_base, const uint32_t* __restrict__ und,
                                const int* __restrict__ tile_elem, const uint8_t* __restrict__ tstate,
                                const int4* __restrict__ dq, int dq_cap, const unsigned* __restrict__ dq_n,
                                uint32_t* __restrict__ vis, unsigned long long* refines, int* err)
{
    const unsigned n = min(*dq_n, (unsigned)dq_cap);
    const float3 c32 = to_f(fr_c(fr)), t1 = to_f(fr_t1(fr)), t2 = to_f(fr_t2(fr));
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int4 e = dq[j];
        const uint32_t i = (uint32_t)e.x;
        const int64_t r = und[i / T];
        const int m = tile_elem[(int64_t)(i % T) * 32 + e.y];
        const float4 el = elem[m];
        const TileRay q = tile_ray(S, rx, r, el, fr, c32, t1, t2, (tstate[i] & 4) != 0);
        bool blocked;
        if (e.z >= 0) {
            atomicAdd(refines, e.w >= 0 ? 2ull : 1ull);
            const d3 A = elem_pos(fr, el), B = D3(q.b.x, q.b.y, q.b.z), dD = B - A;
            const double L = norm(dD);
            blocked = tri_hit_fp64(S.tri_verts[e.z], A, dD, L) || (e.w >= 0 && tri_hit_fp64(S.tri_verts[e.w], A, dD, L));
        } else {
            blocked = seg_blocked_f(S, q.a, q.b, q.in_box, host_face, -1, tol_base, refines, err,
                                    [&](d3& x, d3& y) { x = elem_pos(fr, el); y = D3(q.b.x, q.b.y, q.b.z); });
        }
        if (!blocked) atomicOr(&vis[r * W + (m >> 5)], 1u << (m & 31));
    }
}

// Occlusion of every segment of every candidate (segments in propagation order, early exit on the
// first block); blocked candidates are set to -1. Persistent while-while traversal: each lane pulls
// the next work-list entry (receiver, slot, sequence) from a warp-aggregated atomic counter as soon
// as its current one is finished, computes the candidate's FP32 path points and their error bounds
// (path_points), and every loop iteration advances each busy lane by at most kSteps BVH visits,
// moving on to the candidate's next segment within them, so lanes stay busy while traversal lengths
// differ. A first segment whose point lies in a decided cell
// of the source's visibility map takes the map's answer; a segment with both ends in the scene box
// does not walk the shell subtree. Triangles too close to call in FP32 are queued for an FP64
// settlement after the kernel. ctr[0..3]: candidates, segments, nodes, triangle tests.
constexpr int kValThreads = 128;
#ifndef RISRT_VALIDATE_STEPS
#define RISRT_VALIDATE_STEPS 64    // BVH visits per lane between refills (measured on the room workload)
#endif
constexpr int kSteps = RISRT_VALIDATE_STEPS;

#ifndef RISRT_VALIDATE_MINB
#define RISRT_VALIDATE_MINB 5      // blocks per SM the register budget targets (measured)
#endif
__global__ void __launch_bounds__(kValThreads, RISRT_VALIDATE_MINB)
k_validate(DeviceScene S, const float* __restrict__ dst_xyz, d3 src, int src_face, int dst_face,
           const SeqEntry* __restrict__ seqs, const SeqEntryD* __restrict__ seqd, int* __restrict__ cand, int cap,
           const int* __restrict__ dense_r, const int* __restrict__ dense_slot, const int* __restrict__ dense_seq,
           const long long* __restrict__ d_total, unsigned long long* __restrict__ next, float tol_base,
           unsigned long long* refines,
           int* err, unsigned long long* ctr, RefineQ rq, const uint8_t* __restrict__ smap)
{
    const long long total = *d_total;
    const float3 srcf = to_f(src);
    const bool src_in = in_scene_box(S, src);   // with both ends in the scene box a segment skips the shell
    bool dst_in = false;
    float p1err = 0.f;                            // error bound of the first reflection point
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    TraceCounters tc{};
    long long item = -1;
    int r = 0, slot = 0, si = 0, j = 0;
    int js = 0;                  // segments walked so far; j = the segment walked now
    bool swap12 = false;         // order 2: the last segment walked before the middle one (it is longer)
    int4 info = make_int4(0, 0, 0, 0);
    float3 p[4] = {f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f)};
    float3 a = f3(0.f, 0.f, 0.f), dir = a, inv = a, ainv = a;
    float len = 0.f, tb = 0.f;
    int ign0 = -1, ign1 = -1, g0 = -3, g1 = -3;
    int stack[64];
    int sp = 0;
    constexpr int kNone = 0x7fffffff;
    int cur = kNone;             // current node in a register; the other entered children go on the stack
    bool blocked = false;

    auto start_segment = [&]() {
        a = p[j];
        dir = p[j + 1] - a;
        len = sqrtf(dot(dir, dir));
        inv = f3(safe_inv(dir.x), safe_inv(dir.y), safe_inv(dir.z));
        ainv = f3(a.x * inv.x, a.y * inv.y, a.z * inv.z);
        tb = tol_base + 2e-7f * (fabsf(a.x) + fabsf(a.y) + fabsf(a.z) + len);
        ign0 = j == 0 ? src_face : (j == 1 ? info.x : info.y);
        ign1 = j == info.w ? dst_face : (j == 0 ? info.x : info.y);
        g0 = ign0 >= 0 ? ign0 : -3;        // subtrees of one ignored face are skipped
        g1 = ign1 >= 0 ? ign1 : -3;
        {
            sp = 0;
            const int first = occ_start(S, (j > 0 || src_in) && (j < info.w || dst_in), stack, sp);   // path points
            cur = first == kNoRoot ? kNone : first;                                                   // lie on faces
            if (j == 0 && smap) {       // first segment: the source's visibility map of face f1
                if (p1err <= 0.5f * kMapDelta) {
                    const FaceGrid g = S.face_grid[info.x];
                    const float3 dq = p[1] - xyz(g.o);
                    // (a cell's entry holds up to kMapDelta outside it, far beyond the reciprocal's ulp)
                    const float fa = floorf((dot(dq, xyz(g.u)) - g.u.w) * rcp_slab(g.o.w));
                    const float fb = floorf((dot(dq, xyz(g.v)) - g.v.w) * rcp_slab(g.dv));
                    if (fa >= 0.f && fa < (float)g.nu && fb >= 0.f && fb < (float)g.nv) {
                        const uint8_t st = smap[g.off + (int)fa * g.nv + (int)fb];
                        if (st != 0) {
                            cur = kNone;
                            sp = 0;
                            blocked = st == 2;
                        }
                    }
                }
            }
        }
        ++tc.segs;
    };

    auto test_leaf = [&](int i) -> bool {
        const int f = S.tri_face[i];
        if (f == ign0 || f == ign1) return false;
        ++tc.tris;
        const int h = tri_hit_fp32(S.tri_geom[i], a, dir, len, tb);
        bool hit = h == 1;
        if (h == 2) {
            if (rq.q && item < 0x7fffffffLL) {   // settled later; the traversal goes on as if this triangle missed
                const unsigned pos = atomicAdd(rq.cnt, 1u);
                if (pos < (unsigned)rq.cap) {
                    rq.q[pos] = make_int4((int)item, j, i, 0);
                    return false;
                }
            }
            atomicAdd(refines, 1ull);
            const d3 R = D3((double)dst_xyz[3 * r], (double)dst_xyz[3 * r + 1], (double)dst_xyz[3 * r + 2]);
            d3 pts[4];
            seq_points_fp64(S, R, info, seqd[si], src, pts);
            const d3 dD = pts[j + 1] - pts[j];
            hit = tri_hit_fp64(S.tri_verts[i], pts[j], dD, norm(dD));
        }
        return hit;
    };

    while (true) {
        const bool need = item < 0;
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                item = (long long)(base + __popc(m & ((1u << lane) - 1u)));
                if (item < total) {
                    r = dense_r[item];
                    slot = dense_slot[item];
                    si = dense_seq[item];
                    const SeqEntry e = seqs[si];
                    info = e.info;
                    const float3 R = f3(dst_xyz[3 * r], dst_xyz[3 * r + 1], dst_xyz[3 * r + 2]);
                    dst_in = in_scene_box(S, R);
                    float4 q0, q1;
                    path_points(e, R, q0, q1);
                    p1err = q1.w;
                    const float3 PL = xyz(q0), P1 = xyz(q1);
                    p[0] = srcf;
                    if (info.w == 2) {
                        p[1] = P1;
                        p[2] = PL;
                        p[3] = R;
                    } else {
                        p[1] = PL;
                        p[2] = R;
                        p[3] = R;
                    }
                    j = 0;
                    js = 0;
                    // most candidates are blocked: after the first segment (often decided by the map),
                    // the longer of the other two first
                    swap12 = info.w == 2 && dot(p[3] - p[2], p[3] - p[2]) > dot(p[2] - p[1], p[2] - p[1]);
                    blocked = false;
                    ++tc.cand;
                    start_segment();
                }
            }
        }
        const bool active = item >= 0 && item < total;
        if (!__any_sync(FULL, active)) break;
        if (!active) continue;
        {
            for (int it = 0; it < kSteps; ++it) {
                if (cur == kNone) {          // segment done: the candidate's next segment right away
                    if (blocked || js >= info.w) break;
                    ++js;
                    j = swap12 && js > 0 ? 3 - js : js;
                    start_segment();
                    continue;
                }
                if (cur < 0) {
                    if (test_leaf(~cur)) {
                        blocked = true;
                        cur = kNone;
                        sp = 0;
                        break;
                    }
                    cur = sp > 0 ? stack[--sp] : kNone;
                    continue;
                }
                if (sp + 3 > 64) {           // never expected (stack depth ~ 3 x tree depth / 2)
                    atomicExch(err, 1);
                    blocked = true;
                    cur = kNone;
                    sp = 0;
                    break;
                }
                const Bvh4Node nd = S.nodes4[cur];
                ++tc.nodes;
                cur = bvh4_step(nd, inv, ainv, g0, g1, stack, sp);   // nearest entered child next
                if (cur == kNoChild) cur = sp > 0 ? stack[--sp] : kNone;
            }
        }
        if (cur == kNone) {
            if (blocked) {
                cand[(int64_t)r * cap + slot] = -1;
                item = -1;
            } else if (js < info.w) {
                ++js;
                j = swap12 && js > 0 ? 3 - js : js;
                start_segment();
            } else {
                item = -1;
            }
        }
    }
    flush_counters(tc, ctr);
}

// Settle the queued triangle tests of the validation in FP64: a hit blocks the candidate (the
// traversal treated the triangle as missed, so only a hit changes the outcome).
__global__ void k_refine_val(DeviceScene S, const float* __restrict__ dst_xyz, d3 src, const SeqEntry* __restrict__ seqs,
                             const SeqEntryD* __restrict__ seqd, int* __restrict__ cand, int cap,
                             const int* __restrict__ dense_r, const int* __restrict__ dense_slot, RefineQ rq,
                             unsigned long long* __restrict__ refines)
{
    const unsigned n = min(*rq.cnt, (unsigned)rq.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(refines, (unsigned long long)n);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 q = rq.q[i];
        const int r = dense_r[q.x], slot = dense_slot[q.x];
        const int si = cand[(int64_t)r * cap + slot];
        if (si < 0) continue;                    // already blocked
        const d3 R = D3((double)dst_xyz[3 * r], (double)dst_xyz[3 * r + 1], (double)dst_xyz[3 * r + 2]);
        d3 pts[4];
        seq_points_fp64(S, R, seqs[si].info, seqd[si], src, pts);
        const d3 dD = pts[q.y + 1] - pts[q.y];
        if (tri_hit_fp64(S.tri_verts[q.z], pts[q.y], dD, norm(dD))) cand[(int64_t)r * cap + slot] = -1;
    }
}

// Per destination (one warp): keep the valid candidates, sorted by sequence id (rank sort; ids are
// unique per destination), in the first slots; count -> cnt64.
__global__ void k_finalize(int* __restrict__ cand, const int* __restrict__ cand_cnt, int64_t n_dst, int cap,
                           const SeqEntry* __restrict__ seqs, int64_t* __restrict__ cnt64)
{
    extern __shared__ int sh_list[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (r >= n_dst) return;
    int* list = sh_list + warp * cap;
    int* row = cand + r * (int64_t)cap;
    int n = min(cand_cnt[r], cap);
    int m = 0;
    for (int b = 0; b < n; b += 32) {
        int v = b + lane < n ? row[b + lane] : -1;
        unsigned ball = __ballot_sync(0xffffffffu, v >= 0);
        if (v >= 0) list[m + __popc(ball & ((1u << lane) - 1u))] = v;
        m += __popc(ball);
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) {      // table index order is sequence-id order
        int v = list[i];
        int rank = 0;
        for (int j = 0; j < m; ++j) rank += list[j] < v;
        row[rank] = v;
    }
    __syncwarp();
    if (lane == 0) cnt64[r] = m;
}

// ------------------------------------------------------------------------------------------------
// direct legs
// ------------------------------------------------------------------------------------------------
// e_m -> Rx visibility bits, one warp per (Rx, 32 elements): coherent rays from a small aperture.
// Element -> receiver visibility, one warp per (receiver, 32 elements). A receiver whose aperture
// pyramid is decided (k_rx_aperture: 1 all visible, 2 all blocked) takes that answer for every element.
__global__ void k_direct_vis(DeviceScene S, const float* __restrict__ rx, int64_t n_rx, const float4* __restrict__ elem,
                             int M, int W, Frame fr, int host_face, float tol_base, uint32_t* __restrict__ vis,
                             unsigned long long* refines, int* err, const uint8_t* __restrict__ rx_state)
{
    const int lane = threadIdx.x & 31;
    int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t r = wid / W;
    int w = (int)(wid % W);
    if (r >= n_rx) return;
    int m = w * 32 + lane;
    bool blocked = true;
    const uint8_t st = rx_state ? rx_state[r] : 0;
    if (m < M) {
        if (st != 0) {
            blocked = st == 2;
        } else {
            d3 e = elem_pos(fr, elem[m]);
            d3 R = D3((double)rx[3 * r], (double)rx[3 * r + 1], (double)rx[3 * r + 2]);
            blocked = seg_blocked(S, e, R, host_face, -1, tol_base, refines, err);
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, !blocked);
    if (lane == 0) vis[r * W + w] = b;
}

__global__ void k_tx_vis(DeviceScene S, const float4* __restrict__ elem, int M, Frame fr, AntD tx, int host_face,
                         float tol_base, uint8_t* __restrict__ vis, unsigned long long* refines, int* err)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    d3 e = elem_pos(fr, elem[m]);
    vis[m] = !seg_blocked(S, D3(tx.pos[0], tx.pos[1], tx.pos[2]), e, -1, host_face, tol_base, refines, err);
}

// ------------------------------------------------------------------------------------------------
// Tx-leg element coefficients: K * c_m = K * sum_p sqrt(2 eta0 Pt Gt Ft) sqrt(F_in) R_p e^{-jkL}/L
// (Eq. 4, Eq. 5, Eq. 7; K = sqrt(G dy dz / 4 pi) lambda / 4 pi): FP64 for the unfolded length L and
// frac(L / lambda), FP32 for directions, Fresnel products and patterns (they enter amplitudes only).
// ------------------------------------------------------------------------------------------------


// One Tx-leg term of element e from the Tx image Ts across k faces (nf / ef: FP32 normals and complex
// permittivities of the faces in propagation order): sqrt(2 eta0 Pt Gt Ft) sqrt(F_in) R_p e^{-jkL} / L
// (Eq. 4, Eq. 5, Fresnel per bounce) with L and frac(L / lambda) in FP64, directions, Fresnel
// products and patterns in FP32 (they enter amplitudes only).
__device__ __forceinline__ cf tx_term(d3 e, d3 Ts, int k, const float3* nf, const float2* ef, float3 z, float3 nr,
                                      float gt, float amp0, int pattern, const WaveD& wv)
{
    const d3 d = e - Ts;
    const double L = sqrt(dot(d, d));
    const double x = L * wv.inv_lam;
    const float ph = (float)(x - floor(x));
    float3 u = to_f(d);                       // arrival direction at the element: the last segment is real
    u = u * rsqrtf(dot(u, u));
    cf Rp = cf{1.f, 0.f};
    if (k >= 1) {
        const float3 nl = nf[k - 1];
        Rp = fresnel_f(fabsf(dot(u, nl)), ef[k - 1].x, ef[k - 1].y, wv.tm);
        if (k == 2) {
            const float3 n1 = mirror_dir_f(nf[0], nl);
            Rp = cmulf(Rp, fresnel_f(fabsf(dot(u, n1)), ef[0].x, ef[0].y, wv.tm));
        }
    }
    float3 dep = u;
    for (int j = k - 1; j >= 0; --j) dep = mirror_dir_f(dep, nf[j]);
    const float Ft = pattern_f(pattern, gt, dot(dep, z));
    const float Fin = fmaxf(-dot(u, nr), 0.f);  // element pattern max(cos, 0) toward the Tx side
    const float amp = amp0 * sqrtf(Ft * Fin) / (float)L;
    float sn, cs;
    sincospif(2.f * ph, &sn, &cs);            // e^{-j 2 pi frac(L / lambda)}
    return cmulf(Rp, cf{amp * cs, -amp * sn});
}

// Tx-leg element coefficients: K * c_m = K * sum_p (the terms of tx_term), one warp per element, lanes
// over its Tx-leg paths (LOS first); fixed reduction order (lane-strided paths, shuffle tree).
__global__ void k_cm(DeviceScene S, const float4* __restrict__ elem, int M, Frame fr, AntD tx, WaveD wv, double K,
                     const uint8_t* __restrict__ tx_vis, const int* __restrict__ tx_seq,
                     const int64_t* __restrict__ n_tx_dev, const SeqEntry* __restrict__ seqs,
                     const SeqEntryD* __restrict__ seqd, float2* __restrict__ cm)
{
    const int n_tx = (int)*n_tx_dev;
    const int lane = threadIdx.x & 31;
    const int m = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (m >= M) return;
    const d3 e = elem_pos(fr, elem[m]);
    const d3 T = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
    const float3 z = f3((float)tx.z[0], (float)tx.z[1], (float)tx.z[2]);
    const float3 nr = f3((float)fr.n[0], (float)fr.n[1], (float)fr.n[2]);
    const float gt = (float)tx.gain;
    const float amp0 = (float)sqrt(2.0 * kEta0 * tx.power * tx.gain);
    float are = 0.f, aim = 0.f;
    for (int p = lane - 1; p < n_tx; p += 32) {
        d3 Ts = T;
        int k = 0;
        float3 nf[2] = {f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f)};
        float2 ef[2] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f)};
        if (p < 0) {
            if (!tx_vis[m]) continue;
        } else {
            const int si = tx_seq[p];
            const int4 info = seqs[si].info;
            k = info.w;
            for (int j = 0; j < k; ++j) {
                const int f = j == 0 ? info.x : info.y;
                nf[j] = face_n32(S, f);
                ef[j] = face_eps32(S, f, wv);
            }
            Ts = k == 2 ? ld3(seqd[si].S2) : ld3(seqd[si].S1);
        }
        const cf t = tx_term(e, Ts, k, nf, ef, z, nr, gt, amp0, tx.pattern, wv);
        are += t.re;
        aim += t.im;
    }
    for (int o = 16; o > 0; o >>= 1) {
        are += __shfl_down_sync(0xffffffffu, are, o);
        aim += __shfl_down_sync(0xffffffffu, aim, o);
    }
    if (lane == 0) cm[m] = make_float2((float)(K * are), (float)(K * aim));
}

// Sequence ids of the Tx-leg paths (for the host copy of the path set) and their table kept with the
// path set (image, face normals and permittivities), in id order.
__global__ void k_tx_ids(const int* __restrict__ cand, const int64_t* __restrict__ n_dev, int cap,
                         const SeqEntry* __restrict__ seqs, const SeqEntryD* __restrict__ seqd, DeviceScene S, WaveD wv,
                         int64_t* __restrict__ ids, TxPathD* __restrict__ paths)
{
    const int n = (int)min(*n_dev, (int64_t)cap);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int si = cand[i];
        const int4 info = seqs[si].info;
        ids[i] = info.z;
        TxPathD t;
        t.k = info.w;
        t.id = info.z;
        t.img = info.w == 2 ? seqd[si].S2 : seqd[si].S1;
        for (int j = 0; j < 2; ++j) {
            const int f = j == 0 ? info.x : info.y;
            const bool on = j < info.w;
            const float3 nv = on ? face_n32(S, f) : f3(0.f, 0.f, 0.f);
            t.n[j] = make_float4(nv.x, nv.y, nv.z, 0.f);
            t.eps[j] = on ? face_eps32(S, f, wv) : make_float2(1.f, 0.f);
        }
        paths[i] = t;
    }
}

// Per (element m, Tx-leg path p; p = 0 the direct leg, p >= 1 the kept reflected paths in id order):
// g[m][p] = Gamma_m K c_mp, the element coefficient restricted to one Tx-leg path (the terms k_cm sums),
// and the delay of each Tx-leg path at the RIS centre, |T_p - c| / c0 in FP64.
__global__ void k_cir_coef(const float4* __restrict__ elem, int M, Frame fr, AntD tx, WaveD wv, double K,
                           const uint8_t* __restrict__ tx_vis, const TxPathD* __restrict__ paths, int n_tx,
                           const float2* __restrict__ gamma, float2* __restrict__ g, double* __restrict__ tx_delay)
{
    const int P = n_tx + 1;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * P) return;
    const int m = (int)(i / P), p = (int)(i % P);
    d3 Ts = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
    int k = 0;
    float3 nf[2] = {f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f)};
    float2 ef[2] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f)};
    if (p > 0) {
        const TxPathD t = paths[p - 1];
        k = t.k;
        Ts = ld3(t.img);
        for (int j = 0; j < 2; ++j) {
            nf[j] = f3(t.n[j].x, t.n[j].y, t.n[j].z);
            ef[j] = t.eps[j];
        }
    }
    if (m == 0) {
        const d3 dc = fr_c(fr) - Ts;
        tx_delay[p] = sqrt(dot(dc, dc)) / kC0;
    }
    float2 out = make_float2(0.f, 0.f);
    if (p > 0 || tx_vis[m]) {
        const float3 z = f3((float)tx.z[0], (float)tx.z[1], (float)tx.z[2]);
        const float3 nr = f3((float)fr.n[0], (float)fr.n[1], (float)fr.n[2]);
        const float amp0 = (float)sqrt(2.0 * kEta0 * tx.power * tx.gain);
        const cf t = tx_term(elem_pos(fr, elem[m]), Ts, k, nf, ef, z, nr, (float)tx.gain, amp0, tx.pattern, wv);
        const cf c = cf{(float)(K * t.re), (float)(K * t.im)};
        const float2 gm = gamma[m];
        const cf v = cmulf(c, cf{gm.x, gm.y});
        out = make_float2(v.re, v.im);
    }
    g[i] = out;
}

// Strict mode, Tx leg: every (element m, allowed Tx-leg sequence si) decided in FP64 between the Tx and
// the element itself (reflection points in their faces, back-trace parameters in (0, 1), neighbours on
// the same side of each plane, every segment unblocked); the bounce next to the element may not lie on
// a plane through it. Elements run fastest, so the threads of a warp share a sequence.
__global__ void k_tx_strict(DeviceScene S, const float4* __restrict__ elem, int M, Frame fr, AntD tx, int host_face,
                            float tol_base, const SeqEntry* __restrict__ seqs, const SeqEntryD* __restrict__ seqd,
                            int n_seq, int W, uint32_t* __restrict__ mask, unsigned long long* refines, int* err)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_seq * M) return;
    const int m = (int)(i % M), si = (int)(i / M);
    const int4 info = seqs[si].info;
    const int k = info.w;
    const int fa[2] = {info.x, info.y};
    const d3 e = elem_pos(fr, elem[m]);
    if (contains_point(S.faces[fa[k - 1]], e)) return;
    const d3 T = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
    d3 pts[4];
    if (!seq_geom_fp64(S, T, e, info, seqd[si], pts)) return;
    for (int j = 0; j <= k; ++j) {
        const int ign0 = j == 0 ? -1 : fa[j - 1];
        const int ign1 = j == k ? host_face : fa[j];
        if (seg_blocked(S, pts[j], pts[j + 1], ign0, ign1, tol_base, refines, err)) return;
    }
    atomicOr(&mask[(int64_t)si * W + (m >> 5)], 1u << (m & 31));
}

// Strict mode's K c_m: the direct Tx leg if unblocked plus every Tx-leg sequence valid for element m
// (mask bit m), one warp per element, lanes over the sequences, fixed reduction order.
__global__ void k_cm_strict(DeviceScene S, const float4* __restrict__ elem, int M, Frame fr, AntD tx, WaveD wv, double K,
                            int host_face, float tol_base, const SeqEntry* __restrict__ seqs,
                            const SeqEntryD* __restrict__ seqd, int n_seq, int W, const uint32_t* __restrict__ mask,
                            float2* __restrict__ cm, unsigned long long* refines, int* err)
{
    const int lane = threadIdx.x & 31;
    const int m = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (m >= M) return;
    const d3 e = elem_pos(fr, elem[m]);
    const d3 T = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
    const float3 z = f3((float)tx.z[0], (float)tx.z[1], (float)tx.z[2]);
    const float3 nr = f3((float)fr.n[0], (float)fr.n[1], (float)fr.n[2]);
    const float gt = (float)tx.gain;
    const float amp0 = (float)sqrt(2.0 * kEta0 * tx.power * tx.gain);
    float are = 0.f, aim = 0.f;
    for (int p = lane - 1; p < n_seq; p += 32) {
        d3 Ts = T;
        int k = 0;
        float3 nf[2] = {f3(0.f, 0.f, 0.f), f3(0.f, 0.f, 0.f)};
        float2 ef[2] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f)};
        if (p < 0) {
            if (seg_blocked(S, T, e, -1, host_face, tol_base, refines, err)) continue;
        } else {
            if (!((mask[(int64_t)p * W + (m >> 5)] >> (m & 31)) & 1u)) continue;
            const int4 info = seqs[p].info;
            k = info.w;
            for (int j = 0; j < k; ++j) {
                const int f = j == 0 ? info.x : info.y;
                nf[j] = face_n32(S, f);
                ef[j] = face_eps32(S, f, wv);
            }
            Ts = k == 2 ? ld3(seqd[p].S2) : ld3(seqd[p].S1);
        }
        const cf t = tx_term(e, Ts, k, nf, ef, z, nr, gt, amp0, tx.pattern, wv);
        are += t.re;
        aim += t.im;
    }
    for (int o = 16; o > 0; o >>= 1) {
        are += __shfl_down_sync(0xffffffffu, are, o);
        aim += __shfl_down_sync(0xffffffffu, aim, o);
    }
    if (lane == 0) cm[m] = make_float2((float)(K * are), (float)(K * aim));
}

// ------------------------------------------------------------------------------------------------
// Path records (FP64 reference quantities per (Rx, path)) and E0 = LOS + environment paths.
// ------------------------------------------------------------------------------------------------
__global__ void k_count_total(const int64_t* __restrict__ cnt, int64_t n, int64_t* __restrict__ tot)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) tot[i] = cnt[i] + 1;    // + the direct entry
}

__device__ __forceinline__ float4 local4(const Frame& fr, d3 v, float w)
{
    return make_float4((float)dot(v, fr_t1(fr)), (float)dot(v, fr_t2(fr)), (float)dot(v, fr_n(fr)), w);
}


// Receivers have a handful of paths each: a group of 8 lanes per receiver keeps most lanes busy.
constexpr int kRecGroup = 8;

// Per (Rx, path) record for the field kernel. FP64 only where the phase needs it: the receiver image
// I (mirrored through the bounce planes in reverse order), w = I - c in the RIS frame, D0 = |w| and
// frac(D0 / lambda); the normals, pattern axis and permittivities are FP32 (they enter amplitudes only).
__global__ void k_records(DeviceScene S, const float* __restrict__ rx, int64_t n_rx, Frame fr, WaveD wv,
                          AntD rxa, const int* __restrict__ cand, int cap, const int64_t* __restrict__ off,
                          const SeqEntry* __restrict__ seqs, PathRec* __restrict__ rec, int64_t* __restrict__ rec_seq,
                          int64_t rec_cap, int* __restrict__ overflow)
{
    const int lane = threadIdx.x & (kRecGroup - 1);   // kRecGroup lanes per receiver, over its paths
    int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kRecGroup;
    if (r >= n_rx) return;
    const int64_t o = off[r];
    const int n = (int)(off[r + 1] - o);
    const d3 R = D3((double)rx[3 * r], (double)rx[3 * r + 1], (double)rx[3 * r + 2]);
    const d3 c = fr_c(fr);
    const float3 t1 = f3((float)fr.t1[0], (float)fr.t1[1], (float)fr.t1[2]);
    const float3 t2 = f3((float)fr.t2[0], (float)fr.t2[1], (float)fr.t2[2]);
    const float3 nn = f3((float)fr.n[0], (float)fr.n[1], (float)fr.n[2]);
    const float3 zr = f3((float)rxa.z[0], (float)rxa.z[1], (float)rxa.z[2]);
    auto local = [&](float3 v, float wv_) { return make_float4(dot(v, t1), dot(v, t2), dot(v, nn), wv_); };
    for (int q = lane; q < n; q += kRecGroup) {
        if (o + q >= rec_cap) {               // a workspace-bound path set is full
            atomicExch(overflow, 1);
            break;
        }
        int k = 0;
        int fa[2] = {-1, -1};
        int64_t id = -1;
        if (q > 0) {
            int4 info = seqs[cand[r * (int64_t)cap + q - 1]].info;
            k = info.w;
            fa[0] = info.x;
            fa[1] = info.y;
            id = info.z;
        }
        d3 I = R;
        for (int j = k - 1; j >= 0; --j) {
            dv4 pl = S.faces[fa[j]].plane;
            I = mirror_pt(I, ld3(pl), pl.w);
        }
        const d3 w = I - c;
        const double D0 = sqrt(dot(w, w));
        const double x = D0 * wv.inv_lam;
        const float fr0 = (float)(x - floor(x));
        // Rx pattern axis unfolded: v = L_f1 L_f2 z_r
        float3 v = zr;
        for (int j = k - 1; j >= 0; --j) v = mirror_dir_f(v, face_n32(S, fa[j]));
        float3 n1 = f3(0.f, 0.f, 0.f), n2 = n1;
        float2 e1 = make_float2(1.f, 0.f), e2 = e1;
        if (k >= 1) {
            n1 = face_n32(S, fa[0]);
            e1 = face_eps32(S, fa[0], wv);
        }
        if (k == 2) {
            n2 = mirror_dir_f(face_n32(S, fa[1]), n1);
            e2 = face_eps32(S, fa[1], wv);
        }
        // every bounce a lossless dielectric with the TE coefficient: the record carries eps_r - 1 and
        // 1 / (1 - eps_r) per bounce instead of the complex permittivities (bit 2 of the order field), so
        // the field kernel evaluates R = (c - s)^2 / (1 - eps_r) with s = sqrt(eps_r - 1 + c^2), real
        const bool fast = !wv.tm && k >= 1 && e1.y == 0.f && e1.x >= 1.f && (k < 2 || (e2.y == 0.f && e2.x >= 1.f));
        float az = e1.x, aw = e1.y, n1w = e2.x, n2w = e2.y;
        if (fast) {
            az = e1.x - 1.f;
            aw = e1.x == 1.f ? 0.f : (float)(1.0 / (1.0 - (double)e1.x));
            if (k == 2) {
                n1w = e2.x - 1.f;
                n2w = e2.x == 1.f ? 0.f : (float)(1.0 / (1.0 - (double)e2.x));
            }
        }
        PathRec pr;
        pr.w = local4(fr, w, (float)D0);   // FP64 projection: |w_local| must match D0 for the phase
        pr.a = make_float4(fr0, __int_as_float(k | (fast ? kRecLosslessTE : 0)), az, aw);
        pr.n1 = local(n1, n1w);
        pr.n2 = local(n2, n2w);
        pr.v = local(v, 0.f);
        rec[o + q] = pr;
        rec_seq[o + q] = id;
    }
}

// E0 per receiver (a group of kRecGroup lanes): LOS (if unblocked) + environment paths (Eqs. 2-3 of the direct and
// reflected Tx -> Rx rays), each from its unfolded image source Ts. FP64 for the unfolded length L and
// frac(L / lambda); FP32 for directions, Fresnel products, patterns and amplitudes. Fixed order: lane-
// strided paths, then a shuffle tree.
__global__ void k_e0(DeviceScene S, const float* __restrict__ rx, int64_t n_rx, AntD tx, AntD rxa, WaveD wv,
                     const uint8_t* __restrict__ los, const int* __restrict__ cand, int cap,
                     const int64_t* __restrict__ cnt, const SeqEntry* __restrict__ seqs,
                     const SeqEntryD* __restrict__ seqd, float2* __restrict__ E0)
{
    const int lane = threadIdx.x & (kRecGroup - 1);   // kRecGroup lanes per receiver, over its paths
    const int64_t r0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kRecGroup;
    const bool live = r0 < n_rx;                      // every lane reaches the shuffles below
    const int64_t r = live ? r0 : 0;
    const d3 R = D3((double)rx[3 * r], (double)rx[3 * r + 1], (double)rx[3 * r + 2]);
    const d3 T = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
    const float3 zt = f3((float)tx.z[0], (float)tx.z[1], (float)tx.z[2]);
    const float3 zr = f3((float)rxa.z[0], (float)rxa.z[1], (float)rxa.z[2]);
    const float gt = (float)tx.gain, gr = (float)rxa.gain;
    const float amp0 = (float)(sqrt(2.0 * kEta0 * tx.power * tx.gain) * sqrt(rxa.gain) * wv.lam / (4.0 * kPi));
    const int n = live ? (cnt ? (int)cnt[r] : 0) : -1;
    float are = 0.f, aim = 0.f;
    for (int q = lane - 1; q < n; q += kRecGroup) {   // q = -1: LOS
        d3 Ts = T;
        int fa[2] = {-1, -1};
        int k = 0;
        if (q < 0) {
            if (!los[r]) continue;
        } else {
            int si = cand[r * (int64_t)cap + q];
            int4 info = seqs[si].info;
            k = info.w;
            fa[0] = info.x;
            fa[1] = info.y;
            Ts = k == 2 ? ld3(seqd[si].S2) : ld3(seqd[si].S1);
        }
        const d3 d = R - Ts;
        const double L = sqrt(dot(d, d));
        const double x = L * wv.inv_lam;
        const float ph = (float)(x - floor(x));
        float3 u = to_f(d);                       // arrival direction: the last segment is real
        u = u * rsqrtf(dot(u, u));
        cf Rp = cf{1.f, 0.f};
        if (k >= 1) {                             // last bounce plane real, the earlier one mirrored across it
            const float3 nl = face_n32(S, fa[k - 1]);
            const float2 el = face_eps32(S, fa[k - 1], wv);
            Rp = fresnel_f(fabsf(dot(u, nl)), el.x, el.y, wv.tm);
            if (k == 2) {
                const float3 n1 = mirror_dir_f(face_n32(S, fa[0]), nl);
                const float2 e1 = face_eps32(S, fa[0], wv);
                Rp = cmulf(Rp, fresnel_f(fabsf(dot(u, n1)), e1.x, e1.y, wv.tm));
            }
        }
        float3 dep = u;                           // real first-segment direction: L_f1 L_f2 u
        for (int j = k - 1; j >= 0; --j) dep = mirror_dir_f(dep, face_n32(S, fa[j]));
        const float Ft = pattern_f(tx.pattern, gt, dot(dep, zt));
        const float Fr = pattern_f(rxa.pattern, gr, -dot(u, zr));
        const float amp = amp0 * sqrtf(Ft * Fr) / (float)L;
        float sn, cs;
        sincospif(2.f * ph, &sn, &cs);            // e^{-j 2 pi frac(L / lambda)}
        const cf t = cmulf(Rp, cf{amp * cs, -amp * sn});
        are += t.re;
        aim += t.im;
    }
    for (int o = kRecGroup / 2; o > 0; o >>= 1) {   // fixed order within the group
        are += __shfl_down_sync(0xffffffffu, are, o, kRecGroup);
        aim += __shfl_down_sync(0xffffffffu, aim, o, kRecGroup);
    }
    if (lane == 0 && live) E0[r] = make_float2(are, aim);
}

__global__ void k_los(DeviceScene S, const float* __restrict__ rx, int64_t n_rx, AntD tx, float tol_base,
                      uint8_t* __restrict__ los, unsigned long long* refines, int* err)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rx) return;
    d3 R = D3((double)rx[3 * r], (double)rx[3 * r + 1], (double)rx[3 * r + 2]);
    los[r] = !seg_blocked(S, D3(tx.pos[0], tx.pos[1], tx.pos[2]), R, -1, -1, tol_base, refines, err);
}

__global__ void k_env_ids(const int* __restrict__ cand, int cap, const int64_t* __restrict__ cnt,
                          const int64_t* __restrict__ off, int64_t n_rx, const SeqEntry* __restrict__ seqs,
                          int64_t* __restrict__ out, int64_t out_cap, int* __restrict__ overflow)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rx) return;
    for (int q = 0; q < cnt[r]; ++q) {
        if (off[r] + q >= out_cap) {          // a workspace-bound path set is full
            atomicExch(overflow, 1);
            return;
        }
        out[off[r] + q] = seqs[cand[r * (int64_t)cap + q]].info.z;
    }
}

__global__ void k_trace_init(float* __restrict__ c_xyz, float cx, float cy, float cz, unsigned* __restrict__ rx_bb,
                             unsigned long long* __restrict__ gen)
{
    const int t = threadIdx.x;
    if (t == 0 && gen) *gen += 1ull;
    if (t < 3) c_xyz[t] = t == 0 ? cx : (t == 1 ? cy : cz);
    if (t < 8) rx_bb[t] = t < 3 ? 0xffffffffu : 0u;
}

__global__ void k_abs_max(const float* __restrict__ v, int64_t n, unsigned* __restrict__ out)
{
    unsigned m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(v[i])));
    atomicMax(out, m);
}

__device__ __forceinline__ unsigned ord_bits(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ord(unsigned o) { return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o); }

__global__ void k_rx_bounds(const float* __restrict__ xyz, int64_t n, unsigned* __restrict__ bb)
{
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const unsigned o = ord_bits(xyz[3 * i + k]);
            lo[k] = min(lo[k], o);
            hi[k] = max(hi[k], o);
        }
    for (int k = 0; k < 3; ++k) {
        atomicMin(&bb[k], lo[k]);
        atomicMax(&bb[3 + k], hi[k]);
    }
}

__device__ __forceinline__ unsigned spread10b(unsigned x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// 30-bit Morton code of every receiver (spatial order for the candidate search).
__global__ void k_rx_morton(const float* __restrict__ xyz, int64_t n, const unsigned* __restrict__ bb,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned code = 0;
    for (int k = 0; k < 3; ++k) {
        const float lo = from_ord(bb[k]), span = from_ord(bb[3 + k]) - lo;
        const float u = span > 0.f ? (xyz[3 * i + k] - lo) / span : 0.f;
        code |= spread10b((unsigned)fminf(fmaxf(u * 1024.f, 0.f), 1023.f)) << (2 - k);
    }
    keys[i] = code;
    vals[i] = (uint32_t)i;
}

__global__ void k_units(const int64_t* __restrict__ off, int64_t n_rx, int M, unsigned long long* units)
{
    __shared__ unsigned long long s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n_rx) atomicAdd(&s, (unsigned long long)(off[r + 1] - off[r]) * M);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(units, s);
}

// ------------------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------------------
struct Arena {   // bump allocator over one device buffer; with base == nullptr it only measures
    char* base = nullptr;
    size_t used = 0;
    template <typename T>
    T* get(size_t n)
    {
        size_t a = (used + 255) & ~(size_t)255;
        used = a + sizeof(T) * (n > 0 ? n : 1);
        return base ? (T*)(base + a) : nullptr;
    }
};

// Device buffer of at least `need` elements, from (and returned to) the block cache of `pool`.
template <typename T>
int grow(risrt_ctx* ctx, risrt_ctx* pool, T** p, int64_t* cap, int64_t need)
{
    if (*p && *cap >= need) return RISRT_OK;
    if (*p) ctx_free(pool, *p);
    int64_t c = std::max<int64_t>(need, 1);
    cudaError_t e = ctx_malloc(pool, (void**)p, sizeof(T) * (size_t)c);
    if (e != cudaSuccess) {
        *p = nullptr;
        *cap = 0;
        return fail(ctx, RISRT_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    *cap = c;
    return RISRT_OK;
}

struct SeqTable {
    SeqEntry* e = nullptr;
    SeqEntryD* d = nullptr;
    int n = 0;
};

struct Candidates {
    int* cand = nullptr;
    int* cnt = nullptr;
    int64_t* cnt64 = nullptr;
    int64_t* cnt64_tmp = nullptr;
    int cap = 0;
};

// Scratch of one candidate search + validation: the work list (receiver, slot), its
// length, the queue of FP64 settlements, scan space and the validation's work counter. Searches that
// run concurrently on different streams each need their own.
struct LegBufs {
    int *dense_r = nullptr, *dense_slot = nullptr, *dense_seq = nullptr;
    int64_t* dense_off = nullptr;
    unsigned long long* dense_cnt = nullptr;
    int4* rq = nullptr;
    int rq_cap = 0;
    unsigned* rq_cnt = nullptr;
    void* scan_tmp = nullptr;
    unsigned long long* work = nullptr;
    float4* sp_box = nullptr;        // super-patch boxes [n_super][2]
    unsigned* sp_mask = nullptr;     // [n_super][ceil(n_seq / 32)] sequence survivors per super-patch
    int* sp_list = nullptr;          // [n_super][32 ceil(n_seq / 32)] the same as index lists
    int* sp_cnt = nullptr;           // [n_super]
    float4* g_box = nullptr;         // the same for groups of kGroupSuper super-patches
    unsigned* g_mask = nullptr;
    int* g_list = nullptr;
    int* g_cnt = nullptr;
};
constexpr int kTxLegQueue = 4096;   // settlements queued by the Tx leg (more are settled in place)

}  // namespace

// Dynamic shared memory is a per-function, per-device attribute shared by every context and thread of
// the process, so it is raised once per device to the largest size any launch uses and never lowered:
// k_candidates<true> holds up to kMaxSmemFaces face outlines, k_finalize up to kFinalizeSmemMax bytes
// (its launches take fewer warps per block when the candidate slab is wide).
constexpr int kFinalizeSmemMax = 128 * 1024;
constexpr int kAttrMaxDevices = 64;

static int trace_func_attrs(risrt_ctx* ctx)
{
    static std::mutex mu;
    static bool done[kAttrMaxDevices] = {};
    if (ctx->device < 0 || ctx->device >= kAttrMaxDevices)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "device index too large for the kernel attribute table");
    std::lock_guard<std::mutex> lock(mu);
    if (done[ctx->device]) return RISRT_OK;
    cudaError_t e = cudaFuncSetAttribute(k_candidates<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(FaceTest) * kMaxSmemFaces));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(k_candidates)");
    e = cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinalizeSmemMax);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(k_finalize)");
    done[ctx->device] = true;
    return RISRT_OK;
}

// Warps per k_finalize block for a candidate slab `cap` wide (each warp stages one row in shared
// memory); 0 if even one row does not fit.
static int finalize_warps(int cap)
{
    const size_t row = sizeof(int) * (size_t)cap;
    return (int)std::min<size_t>(4, kFinalizeSmemMax / row);
}

// The context's three side streams and the events that order them against its stream (created on first
// use, non-blocking, released with the context).
static int side_streams(risrt_ctx* ctx)
{
    if (ctx->side[0]) return RISRT_OK;
    for (cudaStream_t& st : ctx->side)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return fail(ctx, RISRT_ERR_CUDA, "cudaStreamCreateWithFlags failed");
    for (cudaEvent_t& ev : ctx->ev)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, RISRT_ERR_CUDA, "cudaEventCreateWithFlags failed");
    return RISRT_OK;
}

// Frame of the RIS (its exact FP64 centre when it has one), the antennas, the wave and the RIS
// constant K = sqrt(G dy dz / 4 pi) lambda / 4 pi (G from the element size unless given).
static void trace_params(const risrt_ctx* ctx, const risrt_ris* ris, double freq, uint32_t flags, Frame& fr, AntD& tx,
                         AntD& rxa, WaveD& wv, double& K)
{
    d3 t1 = D3(ris->t1[0], ris->t1[1], ris->t1[2]), t2 = D3(ris->t2[0], ris->t2[1], ris->t2[2]);
    d3 nn = cross(t1, t2);
    nn = nn * (1.0 / norm(nn));
    for (int k = 0; k < 3; ++k) {
        fr.c[k] = ris->exact_center ? ris->center_d[k] : (double)ris->center[k];
        fr.t1[k] = ris->t1[k];
        fr.t2[k] = ris->t2[k];
    }
    fr.n[0] = nn.x; fr.n[1] = nn.y; fr.n[2] = nn.z;
    auto mk_ant = [](const Antenna& a) {
        AntD o;
        double z[3] = {a.orient[6], a.orient[7], a.orient[8]};
        double zn = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
        for (int k = 0; k < 3; ++k) {
            o.pos[k] = a.pos[k];
            o.z[k] = z[k] / zn;
        }
        o.power = a.power_w;
        o.gain = a.gain_lin;
        o.pattern = a.pattern;
        return o;
    };
    tx = mk_ant(ctx->tx);
    rxa = mk_ant(ctx->rx);
    wv.lam = kC0 / freq;
    wv.k = 2.0 * kPi / wv.lam;
    wv.omega = 2.0 * kPi * freq;
    wv.inv_lam = 1.0 / wv.lam;
    wv.inv_we = (float)(1.0 / (wv.omega * kEps0));
    wv.tm = (flags & RISRT_FLAG_FRESNEL_TM) ? 1 : 0;
    double G = ris->elem_gain > 0 ? (double)ris->elem_gain : 4.0 * kPi * (double)ris->dy * (double)ris->dz / (wv.lam * wv.lam);
    K = sqrt(G * (double)ris->dy * (double)ris->dz / (4.0 * kPi)) * wv.lam / (4.0 * kPi);
}

int trace_paths(risrt_ctx* ctx, const risrt_scene* sc, const risrt_ris* ris, const risrt_rxset* rxs, double freq,
                int max_tx, int max_rx, uint32_t flags, risrt_pathset* ps, const AsyncTrace* at)
{
    cudaStream_t s = ctx->stream;
    if (int arc = trace_func_attrs(ctx)) return arc;
    const DeviceScene S = sc->dev();
    const int F = sc->n_faces;
    const int M = ris->M;
    const int64_t n_rx = rxs->n;
    const bool env = (flags & RISRT_FLAG_ENV_PATHS) != 0;
    if (sc->n_tris == 0) {
        max_tx = 0;
        max_rx = 0;
    }
    const int max_env = env ? max_rx : 0;

    // frame, antennas, wave
    Frame fr;
    AntD tx, rxa;
    WaveD wv;
    double K;
    trace_params(ctx, ris, freq, flags, fr, tx, rxa, wv, K);
    float ext = sc->scene_extent;
    for (int k = 0; k < 3; ++k) {
        ext = std::max(ext, std::fabs(ctx->tx.pos[k]));
        ext = std::max(ext, std::fabs(ris->center[k]));
    }
    {   // receivers' extent (max |coordinate|) enters the FP32 error bound; an uploaded set keeps it
        float rx_ext = rxs->ext;
        if (rx_ext < 0.f) {
            if (at) return fail(ctx, RISRT_ERR_INVALID_ARG, "receiver set without a known extent");
            if (!ctx->small) RISRT_CUDA(ctx, cudaMalloc(&ctx->small, 256));
            unsigned* d_ext = (unsigned*)ctx->small;
            RISRT_CUDA(ctx, cudaMemsetAsync(d_ext, 0, sizeof(unsigned), s));
            RISRT_KERNEL(ctx, "k_abs_max", (k_abs_max<<<std::min<unsigned>(nblk(3 * n_rx, 256), 1024u), 256, 0, s>>>(rxs->xyz, 3 * n_rx, d_ext)));
            unsigned h_ext = 0;
            RISRT_CUDA(ctx, cudaMemcpyAsync(&h_ext, d_ext, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            RISRT_CUDA(ctx, cudaStreamSynchronize(s));
            memcpy(&rx_ext, &h_ext, sizeof(float));
            rxs->ext = rx_ext;
        }
        ext = std::max(ext, rx_ext);
    }
    const float tol_base = 4e-6f * (1.f + 3.f * ext);

    ps->n_rx = n_rx;
    ps->M = M;
    ps->n_faces = F;
    ps->freq = freq;
    ps->flags = flags;
    ps->rx_pattern = ctx->rx.pattern;
    ps->rx_gain = ctx->rx.gain_lin;
    const int W = (M + 31) / 32;
    // tiled direct legs ((receiver, tile) entries numbered in 32 bits); RISRT_TILES=0 forces one ray
    // per element for every receiver whose aperture pyramid is undecided (both give the same bits)
    const int T_tiles = ris->n_tiles, ST_tiles = (T_tiles + 3) / 4;
    const char* tiles_env = getenv("RISRT_TILES");
    // sequence culling over groups of super-patches first; RISRT_CULL_LEVELS=1 culls each super-patch
    // against every sequence (both give the same candidates)
    const char* cull_env = getenv("RISRT_CULL_LEVELS");
    const bool two_level_cull = !(cull_env && cull_env[0] == '1');
    const bool tiled = T_tiles > 0 && (uint64_t)n_rx * (uint64_t)T_tiles < (1ull << 32) &&
                       !(tiles_env && tiles_env[0] == '0');
    ps->W = W;

    // --- resident per-Rx arrays
    int rc;
    // the path set's device memory comes from its owner's block cache (reused buffers are only
    // touched by work ordered after their earlier uses on this stream), or, for an asynchronous trace,
    // from the caller's workspace (WA), the scratch after the path set's arrays
    risrt_ctx* pool = ps->owner == ctx ? ctx : nullptr;
    Arena WA{at ? (char*)at->ws : nullptr, 0};
    if (at) {
        const int cap0 = at->cand_cap;
        const int64_t np = n_rx * (int64_t)at->max_paths, ne = std::max<int64_t>(n_rx * (int64_t)at->max_env, 1);
        ps->vis = WA.get<uint32_t>(n_rx * W);
        ps->E0 = WA.get<float2>(n_rx);
        ps->rx_off = WA.get<int64_t>(n_rx + 1);
        ps->los = WA.get<uint8_t>(n_rx);
        ps->env_off = WA.get<int64_t>(n_rx + 1);
        ps->cm = WA.get<float2>(M);
        ps->elem = WA.get<float4>(M);
        ps->tx_vis_dev = WA.get<uint8_t>(M);
        ps->tx_paths = WA.get<TxPathD>(cap0);
        ps->rec = WA.get<PathRec>(np);
        ps->rx_seq = WA.get<int64_t>(np);
        ps->env_seq = WA.get<int64_t>(ne);
        ps->ctr_dev = WA.get<unsigned long long>(7);
        ps->gen_dev = ps->ctr_dev + 6;
        ps->cap_rx = n_rx;
        ps->cap_m = M;
        ps->cap_tx_vis = M;
        ps->cap_tx_paths = cap0;
        ps->cap_paths = np;
        ps->cap_rx_seq = np;
        ps->cap_env = ne;
        ps->external = true;
    } else if (ps->cap_rx < n_rx || !ps->vis) {
        for (void* q : {(void*)ps->vis, (void*)ps->E0, (void*)ps->rx_off, (void*)ps->los, (void*)ps->env_off}) ctx_free(pool, q);
        ps->vis = nullptr; ps->E0 = nullptr; ps->rx_off = nullptr; ps->los = nullptr; ps->env_off = nullptr;
        int64_t c = 0;
        if ((rc = grow(ctx, pool, &ps->vis, &c, n_rx * W))) return rc;
        c = 0; if ((rc = grow(ctx, pool, &ps->E0, &c, n_rx))) return rc;
        c = 0; if ((rc = grow(ctx, pool, &ps->rx_off, &c, n_rx + 1))) return rc;
        c = 0; if ((rc = grow(ctx, pool, &ps->los, &c, n_rx))) return rc;
        c = 0; if ((rc = grow(ctx, pool, &ps->env_off, &c, n_rx + 1))) return rc;
        ps->cap_rx = n_rx;
    }
    if (!at) {
        int64_t c = ps->cm ? ps->cap_m : 0;
        if ((rc = grow(ctx, pool, &ps->cm, &c, M))) return rc;
        c = ps->elem ? ps->cap_m : 0;
        if ((rc = grow(ctx, pool, &ps->elem, &c, M))) return rc;
        ps->cap_m = std::max<int64_t>(ps->cap_m, M);
        if ((rc = grow(ctx, pool, &ps->tx_vis_dev, &ps->cap_tx_vis, M))) return rc;
    }
    ps->fr = fr;
    ps->txa = tx;
    ps->rxa = rxa;
    ps->wv = wv;
    ps->K = K;
    if (!at || at->ws) RISRT_CUDA(ctx, cudaMemcpyAsync(ps->elem, ris->elem, sizeof(float4) * M, cudaMemcpyDeviceToDevice, s));

    // --- scratch: sequence tables, candidates, counters
    const int64_t n_ids_tx = max_tx >= 2 ? (int64_t)F + (int64_t)F * F : (max_tx >= 1 ? F : 0);
    const int64_t n_ids_rx = max_rx >= 2 ? (int64_t)F + (int64_t)F * F : (max_rx >= 1 ? F : 0);
    const int64_t n_ids_env = max_env >= 2 ? (int64_t)F + (int64_t)F * F : (max_env >= 1 ? F : 0);
    const int64_t n_ids_max = std::max(n_ids_tx, std::max(n_ids_rx, n_ids_env));
    int cap = at ? at->cand_cap : (ps->cand_cap > 0 ? ps->cand_cap : 512);
    const int rq_cap = (int)std::min<int64_t>(16 * n_rx + 4096, (int64_t)1 << 22);

    // Streams of the concurrent parts (the trace's own stream when profiling every kernel, so that
    // each kernel's events bracket it alone, or when RISRT_OVERLAP=0)
    cudaStream_t sA = s, sB = s, sC = s;
    if (!at || at->ws) {
        const char* ov = getenv("RISRT_OVERLAP");
        const bool overlap = !(ov && ov[0] == '0') && !(ctx->profiling && ctx->prof_only.empty());
        if (overlap) {
            if ((rc = side_streams(ctx))) return rc;
            sA = ctx->side[0];
            sB = ctx->side[1];
            sC = ctx->side[2];
        }
    }
    auto fork = [&](cudaStream_t to, cudaEvent_t ev) {
        if (to == s) return;
        cudaEventRecord(ev, s);
        cudaStreamWaitEvent(to, ev, 0);
    };
    auto join = [&](cudaStream_t from, cudaEvent_t ev) {
        if (from == s) return;
        cudaEventRecord(ev, from);
        cudaStreamWaitEvent(s, ev, 0);
    };
    // work an earlier trace left on the side streams (one that returned early with an error) comes
    // before this trace's use of the path set's buffers
    // (skipped while the stream is being captured into a graph: a captured stream may not wait on work
    // outside the capture, and a trace captured after the context's earlier work has none pending)
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap_st);
    if (ctx->side[0] && (!at || at->ws) && cap_st == cudaStreamCaptureStatusNone) {
        join(ctx->side[0], ctx->ev[3]);
        join(ctx->side[1], ctx->ev[4]);
        join(ctx->side[2], ctx->ev[6]);
    }

    for (int attempt = 0; attempt < 6; ++attempt) {
        struct Layout {
            SeqTable tab[3];
            int64_t *flag, *pos, *tot, *env_cnt_tot;
            void* scan_tmp;
            Candidates crx, cenv, ctx_leg;
            uint8_t* tx_vis;
            unsigned long long* counters;
            int* flags_dev;
            float* c_xyz;
            int *dense_r, *dense_slot, *dense_seq;
            int64_t* dense_off;
            uint32_t *rx_keys, *rx_order_u;
            void* rx_sort_tmp;
            unsigned* rx_bb;
            int* rx_order;
            unsigned long long* dense_cnt;   // entries of the work list written by the candidate search
            int64_t* seq_n;                  // sizes of the three sequence tables
            int64_t* tx_ids;                 // [cap] sequence ids of the Tx-leg paths
            int4* rq;                // deferred FP64 settlements (candidates, then validation)
            unsigned* rq_cnt;
            uint8_t* smap[2];        // visibility maps of the face cells from the Tx and from the RIS centre
            float4* elem_bb;         // element centre bounds in the RIS frame
            uint8_t* rx_state;       // per receiver: class of its RIS-aperture pyramid
            uint32_t* und;           // tiled direct legs: receivers with an undecided aperture pyramid,
            unsigned* tile_n;        // their count and the count of undecided (receiver, tile) entries,
            uint8_t* tstate;         // the class of each (undecided receiver, tile) pyramid
            uint32_t* twork;         // and the undecided (receiver, tile) entries
            TileGeom* tgeom;         // per tile, then per super-tile: FP32 corners of its rectangle, in-box flag
            uint8_t* sstate;         // per (undecided receiver, super-tile): class and in-box flag
            uint32_t* swork;         // the undecided (receiver, super-tile) entries
            int4* tdq;               // tile rays left for the FP64 settlement (work entry, lane, triangles)
            TileGeom* ageom;         // the same for the whole aperture
            LegBufs main, env, tx;   // work lists, settlement queues and scan space of the Rx leg, of the
                                     // environment paths and of the Tx leg (they run on separate streams)
        };
        auto layout = [&](Arena& A, Layout& L) {
            for (int i = 0; i < 3; ++i) {
                L.tab[i].e = A.get<SeqEntry>(n_ids_max + 1);
                L.tab[i].d = A.get<SeqEntryD>(n_ids_max + 1);
            }
            L.flag = A.get<int64_t>(n_ids_max + 1);
            L.pos = A.get<int64_t>(n_ids_max + 1);
            L.scan_tmp = A.get<char>(scan_temp_bytes(std::max<int64_t>(n_ids_max, n_rx + 1)));
            L.crx.cand = A.get<int>((size_t)n_rx * cap); L.crx.cnt = A.get<int>(n_rx); L.crx.cnt64 = A.get<int64_t>(n_rx); L.crx.cap = cap;
            L.cenv.cand = A.get<int>(env ? (size_t)n_rx * cap : 1); L.cenv.cnt = A.get<int>(n_rx); L.cenv.cnt64 = A.get<int64_t>(n_rx); L.cenv.cap = cap;
            L.ctx_leg.cand = A.get<int>(cap); L.ctx_leg.cnt = A.get<int>(1); L.ctx_leg.cnt64 = A.get<int64_t>(1); L.ctx_leg.cap = cap;
            L.tot = A.get<int64_t>(n_rx + 1);
            L.env_cnt_tot = A.get<int64_t>(n_rx + 1);
            L.tx_vis = A.get<uint8_t>(M);
            L.counters = A.get<unsigned long long>(8);
            L.flags_dev = A.get<int>(4);
            L.c_xyz = A.get<float>(3);
            L.dense_r = A.get<int>((size_t)n_rx * cap);
            L.dense_slot = A.get<int>((size_t)n_rx * cap);
            L.dense_seq = A.get<int>((size_t)n_rx * cap);
            L.dense_off = A.get<int64_t>(n_rx + 1);
            L.crx.cnt64_tmp = A.get<int64_t>(n_rx + 1);
            L.cenv.cnt64_tmp = A.get<int64_t>(env ? n_rx + 1 : 1);
            L.ctx_leg.cnt64_tmp = A.get<int64_t>(2);
            L.rx_keys = A.get<uint32_t>(n_rx);
            L.rx_order_u = A.get<uint32_t>(n_rx);
            L.rx_sort_tmp = A.get<char>(sort_temp_bytes(n_rx));
            L.rx_bb = A.get<unsigned>(8);
            const int64_t n_super = (n_rx + kSuperRx - 1) / kSuperRx;
            L.dense_cnt = A.get<unsigned long long>(1);
            L.seq_n = A.get<int64_t>(3);
            L.tx_ids = A.get<int64_t>((size_t)cap);
            L.rq = A.get<int4>((size_t)rq_cap);
            L.rq_cnt = A.get<unsigned>(2);
            for (int q = 0; q < 2; ++q) L.smap[q] = A.get<uint8_t>((size_t)std::max<int64_t>(sc->n_cells, 1));
            L.elem_bb = A.get<float4>(1);
            L.rx_state = A.get<uint8_t>((size_t)n_rx);
            L.und = A.get<uint32_t>(tiled ? (size_t)n_rx : 1);
            L.tile_n = A.get<unsigned>(4);
            L.tdq = A.get<int4>(tiled ? (size_t)kTileDeferCap : 1);
            L.tstate = A.get<uint8_t>(tiled ? (size_t)n_rx * T_tiles : 1);
            L.twork = A.get<uint32_t>(tiled ? (size_t)n_rx * T_tiles : 1);
            L.tgeom = A.get<TileGeom>(tiled ? (size_t)(T_tiles + ST_tiles) : 1);
            L.sstate = A.get<uint8_t>(tiled ? (size_t)n_rx * ST_tiles : 1);
            L.swork = A.get<uint32_t>(tiled ? (size_t)n_rx * ST_tiles : 1);
            L.ageom = A.get<TileGeom>(1);
            L.main = LegBufs{L.dense_r, L.dense_slot, L.dense_seq, L.dense_off, L.dense_cnt, L.rq, rq_cap, L.rq_cnt,
                             L.scan_tmp, L.counters + 6};
            // the environment paths run beside the Rx leg: their own work list, queue and scan space
            const size_t n_env_rx = env ? (size_t)n_rx : 1;
            L.env.dense_r = A.get<int>(n_env_rx * cap);
            L.env.dense_slot = A.get<int>(n_env_rx * cap);
            L.env.dense_seq = A.get<int>(n_env_rx * cap);
            L.env.dense_off = A.get<int64_t>(n_env_rx + 1);
            L.env.dense_cnt = A.get<unsigned long long>(1);
            L.env.rq_cap = env ? rq_cap : 1;
            L.env.rq = A.get<int4>((size_t)L.env.rq_cap);
            L.env.rq_cnt = A.get<unsigned>(2);
            L.env.scan_tmp = A.get<char>(scan_temp_bytes((int64_t)n_env_rx + 1));
            L.env.work = A.get<unsigned long long>(1);
            for (LegBufs* lb : {&L.main, &L.env}) {
                const size_t ns = lb == &L.env && !env ? 1 : (size_t)n_super;
                lb->sp_box = A.get<float4>(ns * 2);
                lb->sp_mask = A.get<unsigned>(ns * ((n_ids_max + 31) / 32 + 1));
                lb->sp_list = A.get<int>(ns * ((n_ids_max + 31) / 32 + 1) * 32);
                lb->sp_cnt = A.get<int>(ns);
                const size_t ng = ns / kGroupSuper + 1;
                lb->g_box = A.get<float4>(ng * 2);
                lb->g_mask = A.get<unsigned>(ng * ((n_ids_max + 31) / 32 + 1));
                lb->g_list = A.get<int>(ng * ((n_ids_max + 31) / 32 + 1) * 32);
                lb->g_cnt = A.get<int>(ng);
            }
            L.tx.dense_r = A.get<int>((size_t)cap);
            L.tx.dense_slot = A.get<int>((size_t)cap);
            L.tx.dense_seq = A.get<int>((size_t)cap);
            L.tx.dense_off = A.get<int64_t>(2);
            L.tx.dense_cnt = A.get<unsigned long long>(1);
            L.tx.rq_cap = kTxLegQueue;
            L.tx.rq = A.get<int4>((size_t)kTxLegQueue);
            L.tx.rq_cnt = A.get<unsigned>(2);
            L.tx.scan_tmp = A.get<char>(scan_temp_bytes(2));
            L.tx.work = A.get<unsigned long long>(1);
        };
        if (at) {              // the scratch follows the path set's arrays in the workspace
            Arena probe = WA;
            Layout Lp;
            layout(probe, Lp);
            const size_t need_ws = probe.used + 256;
            if (at->need) *at->need = need_ws;
            if (!at->ws) return RISRT_OK;
            if (need_ws > at->bytes) return fail(ctx, RISRT_ERR_INVALID_ARG, "workspace smaller than risrt_trace_workspace_size");
        }
        Arena measure;
        Layout Lm;
        layout(measure, Lm);
        const size_t need = measure.used + 256;
        if (!at && ps->scratch_bytes < need) {
            ctx_free(pool, ps->scratch);
            ps->scratch = nullptr;
            ps->scratch_bytes = 0;
            cudaError_t e = ctx_malloc(pool, &ps->scratch, need);
            if (e != cudaSuccess) return fail(ctx, RISRT_ERR_OOM, "scratch allocation failed");
            ps->scratch_bytes = need;
        }
        Arena A = at ? WA : Arena{(char*)ps->scratch, 0};
        Layout L;
        layout(A, L);
        SeqTable* tab = L.tab;
        int64_t *flag = L.flag, *pos = L.pos, *tot = L.tot, *env_cnt_tot = L.env_cnt_tot;
        void* scan_tmp = L.scan_tmp;
        Candidates &crx = L.crx, &cenv = L.cenv, &ctx_leg = L.ctx_leg;
        uint8_t* tx_vis = ps->tx_vis_dev;       // kept with the path set (per-path outputs read it)
        if (!at && (rc = grow(ctx, pool, &ps->tx_paths, &ps->cap_tx_paths, cap))) return rc;
        unsigned long long* counters = L.counters;
        int* flags_dev = L.flags_dev;
        float* c_xyz = L.c_xyz;
        RISRT_CUDA(ctx, cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * 8, s));
        RISRT_CUDA(ctx, cudaMemsetAsync(flags_dev, 0, sizeof(int) * 4, s));
        // the RIS centre as the Tx leg's destination and the receivers' bounding-box seeds (a kernel, not a
        // copy from host memory, so a captured trace keeps no host address)
        RISRT_KERNEL(ctx, "k_trace_init", (k_trace_init<<<1, 32, 0, s>>>(c_xyz, ris->center[0], ris->center[1], ris->center[2],
                                                                           L.rx_bb, at ? ps->ctr_dev + 6 : nullptr)));
        const float* rxp = rxs->xyz;
        const d3 Tpos = D3(tx.pos[0], tx.pos[1], tx.pos[2]);
        const d3 Cpos = D3(fr.c[0], fr.c[1], fr.c[2]);

        // Work that needs only the inputs runs beside the sequence tables and the candidate search on
        // stream sB: the visibility maps (the receiver legs' validations wait for them) and the direct
        // legs. The Tx leg runs on sA, the environment paths on sC beside the Rx leg. All join the
        // trace's stream before the path offsets.
        fork(sB, ctx->ev[0]);
        // visibility maps of the face cells from the Tx (environment paths) and the RIS centre (Rx leg);
        // they cost a fixed pass over all cells, so only traces with more receivers than half the
        // cells use them (RISRT_MAPS=0 / 1 forces them off / on: both give the same decisions)
        const char* maps_env = getenv("RISRT_MAPS");
        const bool use_maps = sc->n_cells > 0 && n_rx > 1 &&
                              (maps_env && maps_env[0] ? maps_env[0] == '1' : 2 * n_rx >= sc->n_cells);
        if (use_maps) {
            const float mg = 1e-4f * (1.f + ext);
            if (max_env > 0)
                RISRT_KERNEL_ON(ctx, sB, "k_src_map", (k_src_map<<<nblk(sc->n_cells, 128), 128, 0, sB>>>(S, Tpos, -1, mg, L.smap[0])));
            if (max_rx > 0)
                RISRT_KERNEL_ON(ctx, sB, "k_src_map", (k_src_map<<<nblk(sc->n_cells, 128), 128, 0, sB>>>(S, Cpos, ris->host_face, mg,
                                                                                                L.smap[1])));
        }
        if (sB != s) RISRT_CUDA(ctx, cudaEventRecord(ctx->ev[1], sB));
        // direct legs: element -> receiver visibility (aperture pyramids, then rays where undecided), LOS
        {
            const float mg = 1e-4f * (1.f + ext);
            RISRT_KERNEL_ON(ctx, sB, "k_elem_bounds", (k_elem_bounds<<<1, 256, 0, sB>>>(ris->elem, M, L.elem_bb)));
            RISRT_KERNEL_ON(ctx, sB, "k_tile_geom", (k_tile_geom<<<1, 32, 0, sB>>>(S, fr, L.elem_bb, 1, L.ageom)));
            if (tiled) {
                // receivers, then spatial tiles of 32 elements, decided by pyramids; rays for the rest
                const unsigned grid = (unsigned)ctx->sm_count * 8;
                RISRT_CUDA(ctx, cudaMemsetAsync(L.tile_n, 0, sizeof(unsigned) * 4, sB));
                RISRT_KERNEL_ON(ctx, sB, "k_rx_aperture", (k_rx_aperture<<<nblk(n_rx, 128), 128, 0, sB>>>(S, rxp, n_rx, fr, L.ageom,
                                                                  ris->host_face, mg, L.rx_state, L.und, L.tile_n)));
                RISRT_KERNEL_ON(ctx, sB, "k_vis_decided", (k_vis_decided<<<nblk(n_rx * ((W + 3) / 4), 256), 256, 0, sB>>>(
                                                                  n_rx, W, M, L.rx_state, ps->vis)));
                // (receiver, super-tile) pyramids, then (receiver, tile) pyramids of undecided super-tiles
                RISRT_KERNEL_ON(ctx, sB, "k_tile_geom", (k_tile_geom<<<nblk(T_tiles + ST_tiles, 128), 128, 0, sB>>>(
                                                                  S, fr, ris->tile_bb, T_tiles + ST_tiles, L.tgeom)));
                // (one super-tile is the aperture itself: its tiles are classified directly)
                const bool supers = ST_tiles > 1;
                if (supers)
                    RISRT_KERNEL_ON(ctx, sB, "k_super_aperture", (k_super_aperture<<<grid, 128, 0, sB>>>(S, rxp, fr, L.tgeom + T_tiles,
                                                                      ST_tiles, ris->host_face, mg, L.und, L.tile_n, L.sstate,
                                                                      L.swork, L.tile_n + 3)));
                RISRT_KERNEL_ON(ctx, sB, "k_tile_aperture", (k_tile_aperture<<<grid, 128, 0, sB>>>(S, rxp, fr, L.tgeom, T_tiles,
                                                                  ST_tiles, ris->host_face, mg, L.und, supers ? L.swork : nullptr,
                                                                  supers ? L.tile_n + 3 : L.tile_n, L.tstate, L.twork, L.tile_n + 1)));
                RISRT_KERNEL_ON(ctx, sB, "k_vis_tiles", (k_vis_tiles<<<grid, 256, 0, sB>>>(W, T_tiles, ST_tiles, L.und, L.tile_n,
                                                                  ris->word_ofs, ris->word_tile, supers ? L.sstate : nullptr,
                                                                  L.tstate, ps->vis)));
                RISRT_KERNEL_ON(ctx, sB, "k_direct_tiles", (k_direct_tiles<<<grid, 128, 0, sB>>>(S, rxp, ris->elem, W, T_tiles, fr,
                                                                  ris->host_face, tol_base, L.und, ris->tile_elem, L.tstate,
                                                                  L.twork, L.tile_n + 1, ps->vis, L.tdq, kTileDeferCap,
                                                                  L.tile_n + 2, counters, flags_dev + 1)));
                RISRT_KERNEL_ON(ctx, sB, "k_direct_settle", (k_direct_settle<<<grid, 128, 0, sB>>>(S, rxp, ris->elem, W, T_tiles, fr,
                                                                  ris->host_face, tol_base, L.und, ris->tile_elem, L.tstate,
                                                                  L.tdq, kTileDeferCap, L.tile_n + 2, ps->vis, counters,
                                                                  flags_dev + 1)));
            } else {
                const int64_t nthreads = n_rx * W * 32;
                RISRT_KERNEL_ON(ctx, sB, "k_rx_aperture", (k_rx_aperture<<<nblk(n_rx, 128), 128, 0, sB>>>(S, rxp, n_rx, fr, L.ageom,
                                                                  ris->host_face, mg, L.rx_state, nullptr, nullptr)));
                RISRT_KERNEL_ON(ctx, sB, "k_direct_vis", (k_direct_vis<<<nblk(nthreads, 128), 128, 0, sB>>>(S, rxp, n_rx, ris->elem, M, W, fr,
                                                                  ris->host_face, tol_base, ps->vis, counters, flags_dev + 1,
                                                                  L.rx_state)));
            }
            RISRT_KERNEL_ON(ctx, sB, "k_los", (k_los<<<nblk(n_rx, 128), 128, 0, sB>>>(S, rxp, n_rx, tx, tol_base, ps->los, counters, flags_dev + 1)));
        }

        const int64_t n_ids_of[3] = {n_ids_tx, n_ids_rx, n_ids_env};
        const d3 src_of[3] = {Tpos, Cpos, Tpos};
        RISRT_CUDA(ctx, cudaMemsetAsync(L.seq_n, 0, sizeof(int64_t) * 3, s));
        for (int i = 0; i < 3; ++i) {
            int64_t nid = n_ids_of[i];
            if (nid == 0) continue;
            RISRT_KERNEL(ctx, "k_seq_allowed", (k_seq_allowed<<<nblk(nid, 256), 256, 0, s>>>(S, nid, i, fr, src_of[i], 1e-4f * (1.f + ext), flag)));
            RISRT_CUDA(ctx, exclusive_scan_i64(flag, pos, nid, scan_tmp, s));
            RISRT_KERNEL(ctx, "k_seq_build", (k_seq_build<<<nblk(nid, 256), 256, 0, s>>>(S, nid, flag, pos, src_of[i], tab[i].e, tab[i].d)));
            RISRT_KERNEL(ctx, "k_seq_count", (k_seq_count<<<1, 32, 0, s>>>(flag, pos, nid, L.seq_n + i)));
        }
        if (at) {   // no read-back: grids cover every sequence id, the kernels read the sizes on the device
            for (int i = 0; i < 3; ++i) tab[i].n = (int)n_ids_of[i];
        } else {    // the three table sizes in one read-back
            int64_t n_allowed[3];
            RISRT_CUDA(ctx, cudaMemcpyAsync(n_allowed, L.seq_n, sizeof(n_allowed), cudaMemcpyDeviceToHost, s));
            RISRT_CUDA(ctx, cudaStreamSynchronize(s));
            for (int i = 0; i < 3; ++i) tab[i].n = (int)n_allowed[i];
        }

        // receivers in Morton order for the candidate search
        {
            RISRT_KERNEL(ctx, "k_rx_bounds", (k_rx_bounds<<<std::min<unsigned>(nblk(n_rx, 256), 1024u), 256, 0, s>>>(
                                                 rxs->xyz, n_rx, L.rx_bb)));
            RISRT_KERNEL(ctx, "k_rx_morton", (k_rx_morton<<<nblk(n_rx, 256), 256, 0, s>>>(rxs->xyz, n_rx, L.rx_bb, L.rx_keys,
                                                                                          L.rx_order_u)));
            RISRT_CUDA(ctx, radix_sort_pairs(L.rx_keys, L.rx_order_u, n_rx, 30, L.rx_sort_tmp, s));
            L.rx_order = (int*)L.rx_order_u;
        }

        // One leg's candidate search and validation on stream st with scratch lb; the validation of a
        // many-destination leg first waits for maps_ready (the visibility maps, built on another stream).
        auto run_candidates = [&](const SeqTable& t, const float* dst, int64_t n_dst, d3 src, int src_face,
                                  int dst_face, Candidates& cs, int map_src, cudaStream_t st, const LegBufs& lb,
                                  cudaEvent_t maps_ready, const int64_t* n_dev) -> int {
            RISRT_CUDA(ctx, cudaMemsetAsync(cs.cnt, 0, sizeof(int) * n_dst, st));
            if (t.n > 0) {
                dim3 grid(nblk(n_dst, kCandThreads), std::min<unsigned>(nblk(t.n, kCandChunk), 32768u));
                const RefineQ rq{lb.rq, lb.rq_cap, lb.rq_cnt};
                RISRT_CUDA(ctx, cudaMemsetAsync(lb.rq_cnt, 0, sizeof(unsigned) * 2, st));
                // many destinations: the candidate search writes the validation work list itself
                const DenseOut dl = n_dst > 1 ? DenseOut{lb.dense_r, lb.dense_slot, lb.dense_seq, lb.dense_cnt}
                                              : DenseOut{nullptr, nullptr, nullptr, nullptr};
                if (dl.r) RISRT_CUDA(ctx, cudaMemsetAsync(lb.dense_cnt, 0, sizeof(unsigned long long), st));
                // sequences that can reach each super-patch of kSuperRx Morton-consecutive destinations
                const int words = (t.n + 31) / 32;
                const int* slist = nullptr;
                const int* slist_cnt = nullptr;
                int64_t slist_stride = 0;
                if (n_dst > kCandThreads) {
                    const int64_t n_super = (n_dst + kSuperRx - 1) / kSuperRx;
                    RISRT_KERNEL_ON(ctx, st, "k_patch_boxes", (k_patch_boxes<<<(unsigned)n_super, 256, 0, st>>>(dst, L.rx_order, n_dst,
                                                                                                       lb.sp_box)));
                    if (n_super > 16 * kGroupSuper && two_level_cull) {
                        // two levels (above 256 super-patches, where they pay: measured on the room
                        // and the hall): groups of super-patches against every sequence, then each
                        // super-patch against its group's survivors
                        const int64_t n_groups = (n_super + kGroupSuper - 1) / kGroupSuper;
                        RISRT_KERNEL_ON(ctx, st, "k_group_boxes", (k_group_boxes<<<nblk(n_groups, 128), 128, 0, st>>>(
                                                                  lb.sp_box, n_super, n_groups, lb.g_box)));
                        RISRT_KERNEL_ON(ctx, st, "k_seq_cull", (k_seq_cull<<<dim3(nblk(t.n, 256), (unsigned)std::min<int64_t>(n_groups, 65535)),
                                                                      256, 0, st>>>(S, t.e, t.n, lb.g_box, n_groups, words, lb.g_mask,
                                                                                    n_dev, true)));
                        RISRT_KERNEL_ON(ctx, st, "k_mask_compact", (k_mask_compact<<<(unsigned)std::min<int64_t>(n_groups, 4096), kCompactThreads, 0, st>>>(
                                                                lb.g_mask, words, n_groups, (int64_t)words * 32, lb.g_list, lb.g_cnt,
                                                                nullptr, nullptr)));
                        RISRT_KERNEL_ON(ctx, st, "k_seq_cull2", (k_seq_cull2<<<dim3(nblk(t.n, 256), (unsigned)std::min<int64_t>(n_super, 65535)),
                                                                 256, 0, st>>>(S, t.e, lb.sp_box, n_super, lb.g_list, lb.g_cnt,
                                                                               (int64_t)words * 32, words, lb.sp_mask)));
                        RISRT_KERNEL_ON(ctx, st, "k_mask_compact", (k_mask_compact<<<(unsigned)std::min<int64_t>(n_super, 4096), kCompactThreads, 0, st>>>(
                                                                lb.sp_mask, words, n_super, (int64_t)words * 32, lb.sp_list, lb.sp_cnt,
                                                                lb.g_list, lb.g_cnt)));
                    } else {
                        RISRT_KERNEL_ON(ctx, st, "k_seq_cull", (k_seq_cull<<<dim3(nblk(t.n, 256), (unsigned)std::min<int64_t>(n_super, 65535)),
                                                                      256, 0, st>>>(S, t.e, t.n, lb.sp_box, n_super, words, lb.sp_mask,
                                                                                    n_dev, false)));
                        RISRT_KERNEL_ON(ctx, st, "k_mask_compact", (k_mask_compact<<<(unsigned)std::min<int64_t>(n_super, 4096), kCompactThreads, 0, st>>>(
                                                                lb.sp_mask, words, n_super, (int64_t)words * 32, lb.sp_list, lb.sp_cnt,
                                                                nullptr, nullptr)));
                    }
                    slist = lb.sp_list;
                    slist_cnt = lb.sp_cnt;
                    slist_stride = (int64_t)words * 32;
                }
                const int* ord = n_dst > 1 ? L.rx_order : nullptr;
                if (F <= kMaxSmemFaces) {
                    const size_t shm = sizeof(FaceTest) * (size_t)F;
                    RISRT_KERNEL_ON(ctx, st, "k_candidates", (k_candidates<true><<<grid, kCandThreads, shm, st>>>(
                                                          S, dst, n_dst, ord, src, t.e, t.d, t.n, tol_base, cs.cand, cs.cnt,
                                                          cs.cap, flags_dev, counters, slist, slist_cnt, slist_stride, rq, dl, n_dev)));
                } else {
                    RISRT_KERNEL_ON(ctx, st, "k_candidates", (k_candidates<false><<<grid, kCandThreads, 0, st>>>(
                                                          S, dst, n_dst, ord, src, t.e, t.d, t.n, tol_base, cs.cand, cs.cnt,
                                                          cs.cap, flags_dev, counters, slist, slist_cnt, slist_stride, rq, dl, n_dev)));
                }
                RISRT_KERNEL_ON(ctx, st, "k_refine_cand", (k_refine_cand<<<ctx->sm_count * 2, 256, 0, st>>>(
                                                       S, dst, src, t.e, t.d, rq, cs.cand, cs.cnt, cs.cap, flags_dev, counters, dl)));
                // dense candidate list (written above for many destinations), then persistent validation;
                // its length stays on the device (no host round trip)
                const long long* d_total = (const long long*)lb.dense_cnt;
                if (!dl.r) {
                    RISRT_KERNEL_ON(ctx, st, "k_cand_counts", (k_cand_counts<<<nblk(n_dst + 1, 256), 256, 0, st>>>(cs.cnt, n_dst, cs.cap, cs.cnt64_tmp)));
                    RISRT_CUDA(ctx, exclusive_scan_i64(cs.cnt64_tmp, lb.dense_off, n_dst + 1, lb.scan_tmp, st));
                    RISRT_KERNEL_ON(ctx, st, "k_dense_list", (k_dense_list<<<nblk(n_dst * 32, 128), 128, 0, st>>>(
                                                                cs.cnt, cs.cand, lb.dense_off, n_dst, cs.cap, lb.dense_r,
                                                                lb.dense_slot, lb.dense_seq)));
                    d_total = (const long long*)(lb.dense_off + n_dst);
                }
                RISRT_CUDA(ctx, cudaMemsetAsync(lb.work, 0, sizeof(unsigned long long), st));
                const int *vr = lb.dense_r, *vs = lb.dense_slot;
                // the validation queue reuses the buffer (the candidate settlements are done)
                const RefineQ vq{lb.rq, lb.rq_cap, lb.rq_cnt + 1};
                const uint8_t* smap = n_dst > 1 && use_maps ? L.smap[map_src] : nullptr;   // 0: from the Tx, 1: from the RIS centre
                if (smap && maps_ready) RISRT_CUDA(ctx, cudaStreamWaitEvent(st, maps_ready, 0));
                const unsigned blocks = (unsigned)ctx->sm_count * RISRT_VALIDATE_MINB;
                RISRT_KERNEL_ON(ctx, st, "k_validate", (k_validate<<<blocks, kValThreads, 0, st>>>(
                                                    S, dst, src, src_face, dst_face, t.e, t.d, cs.cand, cs.cap, vr,
                                                    vs, lb.dense_seq, d_total, lb.work, tol_base, counters, flags_dev + 1,
                                                    counters + 2, vq, smap)));
                RISRT_KERNEL_ON(ctx, st, "k_refine_val", (k_refine_val<<<ctx->sm_count * 2, 256, 0, st>>>(
                                                      S, dst, src, t.e, t.d, cs.cand, cs.cap, vr, vs, vq, counters)));
            }
            const int warps = finalize_warps(cs.cap);
            if (warps < 1) return fail(ctx, RISRT_ERR_CAPACITY, "more geometric candidates per destination than k_finalize can sort");
            const size_t shm = sizeof(int) * (size_t)cs.cap * warps;
            RISRT_KERNEL_ON(ctx, st, "k_finalize", (k_finalize<<<nblk(n_dst, warps), 32 * warps, shm, st>>>(cs.cand, cs.cnt, n_dst, cs.cap, t.e, cs.cnt64)));
            return RISRT_OK;
        };

        // Tx leg (destination: RIS centre, mounted on host_face), its element visibility, c_m (its path
        // count stays on the device) and path ids, beside the receiver legs on stream sA
        fork(sA, ctx->ev[2]);
        const int64_t* nd0 = at ? L.seq_n + 0 : nullptr;
        const int64_t* nd1 = at ? L.seq_n + 1 : nullptr;
        const int64_t* nd2 = at ? L.seq_n + 2 : nullptr;
        if ((rc = run_candidates(tab[0], c_xyz, 1, Tpos, -1, ris->host_face, ctx_leg, 0, sA, L.tx, nullptr, nd0))) return rc;
        RISRT_KERNEL_ON(ctx, sA, "k_tx_vis", (k_tx_vis<<<nblk(M, 128), 128, 0, sA>>>(S, ris->elem, M, fr, tx, ris->host_face, tol_base, tx_vis, counters,
                                              flags_dev + 1)));
        RISRT_KERNEL_ON(ctx, sA, "k_cm", (k_cm<<<nblk((int64_t)M * 32, 128), 128, 0, sA>>>(S, ris->elem, M, fr, tx, wv, K, tx_vis, ctx_leg.cand,
                                                                                  ctx_leg.cnt64, tab[0].e, tab[0].d, ps->cm)));
        RISRT_KERNEL_ON(ctx, sA, "k_tx_ids", (k_tx_ids<<<1, 256, 0, sA>>>(ctx_leg.cand, ctx_leg.cnt64, cap, tab[0].e, tab[0].d, S,
                                                                         wv, L.tx_ids, ps->tx_paths)));
        // Rx leg (source: RIS centre) and environment paths (source: Tx); their validations use the maps
        const cudaEvent_t maps_ready = sB != s ? ctx->ev[1] : nullptr;
        fork(sC, ctx->ev[5]);
        if ((rc = run_candidates(tab[1], rxp, n_rx, Cpos, ris->host_face, -1, crx, 1, s, L.main, maps_ready, nd1))) return rc;
        if (env && (rc = run_candidates(tab[2], rxp, n_rx, Tpos, -1, -1, cenv, 0, sC, L.env, maps_ready, nd2))) return rc;
        join(sA, ctx->ev[3]);
        join(sB, ctx->ev[4]);
        join(sC, ctx->ev[6]);
        // Rx-leg and environment offsets
        RISRT_KERNEL(ctx, "k_count_total", (k_count_total<<<nblk(n_rx, 256), 256, 0, s>>>(crx.cnt64, n_rx, tot)));
        RISRT_CUDA(ctx, cudaMemsetAsync(tot + n_rx, 0, sizeof(int64_t), s));
        RISRT_CUDA(ctx, exclusive_scan_i64(tot, ps->rx_off, n_rx + 1, scan_tmp, s));
        if (env) {
            RISRT_CUDA(ctx, cudaMemcpyAsync(env_cnt_tot, cenv.cnt64, sizeof(int64_t) * n_rx, cudaMemcpyDeviceToDevice, s));
            RISRT_CUDA(ctx, cudaMemsetAsync(env_cnt_tot + n_rx, 0, sizeof(int64_t), s));
            RISRT_CUDA(ctx, exclusive_scan_i64(env_cnt_tot, ps->env_off, n_rx + 1, scan_tmp, s));
        } else {
            RISRT_CUDA(ctx, cudaMemsetAsync(ps->env_off, 0, sizeof(int64_t) * (n_rx + 1), s));
        }
        if (at) {
            // no read-back: records and ids go to the workspace's fixed-size arrays (a full array sets
            // flag 2), the counts and Tx-leg ids stay on the device for risrt_trace_check
            ps->n_paths = -1;
            ps->n_env = -1;
            ps->chk_flags = flags_dev;
            ps->chk_ntx = ctx_leg.cnt64;
            ps->chk_ids = L.tx_ids;
            ps->chk_cap = cap;
            ps->check_pending = true;
            fork(sB, ctx->ev[0]);
            RISRT_KERNEL_ON(ctx, sB, "k_e0", (k_e0<<<nblk(n_rx * kRecGroup, 128), 128, 0, sB>>>(S, rxp, n_rx, tx, rxa, wv, ps->los, cenv.cand,
                                                                                         cenv.cap, env ? cenv.cnt64 : nullptr,
                                                                                         tab[2].e, tab[2].d, ps->E0)));
            if (env)
                RISRT_KERNEL_ON(ctx, sB, "k_env_ids", (k_env_ids<<<nblk(n_rx, 128), 128, 0, sB>>>(cenv.cand, cenv.cap, cenv.cnt64,
                                                                                               ps->env_off, n_rx, tab[2].e,
                                                                                               ps->env_seq, ps->cap_env,
                                                                                               flags_dev + 2)));
            RISRT_KERNEL(ctx, "k_records", (k_records<<<nblk(n_rx * kRecGroup, 128), 128, 0, s>>>(S, rxp, n_rx, fr, wv, rxa, crx.cand, crx.cap, ps->rx_off,
                                                          tab[1].e, ps->rec, ps->rx_seq, ps->cap_paths, flags_dev + 2)));
            RISRT_KERNEL(ctx, "k_units", (k_units<<<nblk(n_rx, 256), 256, 0, s>>>(ps->rx_off, n_rx, M, counters + 1)));
            join(sB, ctx->ev[4]);
            RISRT_CUDA(ctx, cudaMemcpyAsync(ps->ctr_dev, counters, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToDevice, s));
            ps->stats_pending = true;
            ps->stream = s;
            return RISRT_OK;
        }
        // one read-back: error flags, path counts, Tx-leg ids and visibility
        int host_flags[2];
        int64_t n_tx64 = 0, n_paths = 0, n_env = 0;
        std::vector<int64_t> tx_ids_host(cap);
        ps->tx_vis_host.resize(M);
        RISRT_CUDA(ctx, cudaMemcpyAsync(host_flags, flags_dev, sizeof(host_flags), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(&n_tx64, ctx_leg.cnt64, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(&n_paths, ps->rx_off + n_rx, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(&n_env, ps->env_off + n_rx, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(tx_ids_host.data(), L.tx_ids, sizeof(int64_t) * cap, cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(ps->tx_vis_host.data(), tx_vis, M, cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        if (host_flags[1]) return fail(ctx, RISRT_ERR_CAPACITY, "BVH traversal stack overflow");
        if (host_flags[0]) {       // a destination had more geometric candidates than slots: retry
            cap *= 4;
            ps->cand_cap = cap;
            continue;
        }
        const int n_tx = (int)std::min<int64_t>(n_tx64, cap);
        ps->tx_seq_host.assign(tx_ids_host.begin(), tx_ids_host.begin() + n_tx);

        // Rx-leg records, E0, environment ids
        if ((rc = grow(ctx, pool, &ps->rec, &ps->cap_paths, n_paths))) return rc;
        if ((rc = grow(ctx, pool, &ps->rx_seq, &ps->cap_rx_seq, std::max<int64_t>(n_paths, 1)))) return rc;
        if ((rc = grow(ctx, pool, &ps->env_seq, &ps->cap_env, std::max<int64_t>(n_env, 1)))) return rc;
        ps->n_paths = n_paths;
        ps->n_env = n_env;
        // E0 and the environment ids (environment leg) beside the Rx-leg records
        fork(sB, ctx->ev[0]);
        RISRT_KERNEL_ON(ctx, sB, "k_e0", (k_e0<<<nblk(n_rx * kRecGroup, 128), 128, 0, sB>>>(S, rxp, n_rx, tx, rxa, wv, ps->los, cenv.cand,
                                                                                     cenv.cap, env ? cenv.cnt64 : nullptr,
                                                                                     tab[2].e, tab[2].d, ps->E0)));
        if (env && n_env > 0) {
            RISRT_KERNEL_ON(ctx, sB, "k_env_ids", (k_env_ids<<<nblk(n_rx, 128), 128, 0, sB>>>(cenv.cand, cenv.cap, cenv.cnt64, ps->env_off,
                                                                                           n_rx, tab[2].e, ps->env_seq, INT64_MAX,
                                                                                           flags_dev + 2)));
        }
        RISRT_KERNEL(ctx, "k_records", (k_records<<<nblk(n_rx * kRecGroup, 128), 128, 0, s>>>(S, rxp, n_rx, fr, wv, rxa, crx.cand, crx.cap, ps->rx_off,
                                                      tab[1].e, ps->rec, ps->rx_seq, INT64_MAX, flags_dev + 2)));
        RISRT_KERNEL(ctx, "k_units", (k_units<<<nblk(n_rx, 256), 256, 0, s>>>(ps->rx_off, n_rx, M, counters + 1)));
        join(sB, ctx->ev[4]);
        // statistics stay on the device until asked for (risrt_pathset_stats_get waits for them)
        if (!ps->ctr_dev) RISRT_CUDA(ctx, ctx_malloc(pool, (void**)&ps->ctr_dev, sizeof(unsigned long long) * 6));
        RISRT_CUDA(ctx, cudaMemcpyAsync(ps->ctr_dev, counters, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToDevice, s));
        ps->stats_pending = true;
        ps->stream = s;
        return RISRT_OK;
    }
    return fail(ctx, RISRT_ERR_CAPACITY, "too many geometric path candidates per receiver");
}

// Per-Tx-path element coefficients of a traced path set for one configuration (risrt_eval_cir):
// g [M][1 + n_tx] complex, tx_delay [1 + n_tx] seconds; on the context's stream.
int cir_tx_coef(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, float2* g, double* tx_delay)
{
    const int n_tx = (int)ps->tx_seq_host.size();
    const int64_t n = (int64_t)ps->M * (n_tx + 1);
    RISRT_KERNEL(ctx, "k_cir_coef", (k_cir_coef<<<nblk(n, 128), 128, 0, ctx->stream>>>(
                                         ps->elem, ps->M, ps->fr, ps->txa, ps->wv, ps->K, ps->tx_vis_dev, ps->tx_paths,
                                         n_tx, gamma, g, tx_delay)));
    return RISRT_OK;
}

// Strict mode's K c_m of every element (risrt_eval_field_strict): the Tx-leg sequence table from the Tx
// (no exclusion by the RIS centre; each element applies its own), every (element, sequence) decided in
// FP64 at the element, the valid terms summed. Synchronises the stream (the table size sizes the work).
int strict_tx_cm(risrt_ctx* ctx, const risrt_scene* sc, const risrt_ris* ris, double freq, int max_tx, uint32_t flags,
                 float2* cm)
{
    cudaStream_t s = ctx->stream;
    const DeviceScene S = sc->dev();
    const int F = sc->n_faces, M = ris->M, W = (M + 31) / 32;
    Frame fr;
    AntD tx, rxa;
    WaveD wv;
    double K;
    trace_params(ctx, ris, freq, flags, fr, tx, rxa, wv, K);
    float ext = sc->scene_extent;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, std::max(std::fabs(ctx->tx.pos[k]), std::fabs(ris->center[k])));
    const float tol_base = 4e-6f * (1.f + 3.f * ext);
    if (sc->n_tris == 0) max_tx = 0;
    const int64_t n_ids = max_tx >= 2 ? (int64_t)F + (int64_t)F * F : (max_tx >= 1 ? F : 0);
    void *flagb = nullptr, *posb = nullptr, *tmp = nullptr, *tab = nullptr, *tabd = nullptr, *maskb = nullptr, *small = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void* q : {flagb, posb, tmp, tab, tabd, maskb, small}) ctx_free(ctx, q);
    };
#define RISRT_STRICT_CUDA(call)                                   \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) {                                  \
            release();                                            \
            return cuda_fail(ctx, _e, #call);                     \
        }                                                         \
    } while (0)
    RISRT_STRICT_CUDA(ctx_malloc(ctx, &small, 64));
    unsigned long long* refines = (unsigned long long*)small;
    int* err = (int*)((char*)small + 16);
    RISRT_STRICT_CUDA(cudaMemsetAsync(small, 0, 64, s));
    int64_t n_seq = 0;
    if (n_ids > 0) {
        RISRT_STRICT_CUDA(ctx_malloc(ctx, &flagb, sizeof(int64_t) * n_ids));
        RISRT_STRICT_CUDA(ctx_malloc(ctx, &posb, sizeof(int64_t) * (n_ids + 1)));
        RISRT_STRICT_CUDA(ctx_malloc(ctx, &tmp, scan_temp_bytes(std::max<int64_t>(n_ids, 2))));
        int64_t* flag = (int64_t*)flagb;
        int64_t* pos = (int64_t*)posb;
        auto allowed = [&]() -> int {     // launch failures return here, so release() still runs
            RISRT_KERNEL(ctx, "k_seq_allowed", (k_seq_allowed<<<nblk(n_ids, 256), 256, 0, s>>>(S, n_ids, 2, fr, D3(tx.pos[0], tx.pos[1], tx.pos[2]),
                                                                                             1e-4f * (1.f + ext), flag)));
            return RISRT_OK;
        };
        auto count = [&]() -> int {
            RISRT_KERNEL(ctx, "k_seq_count", (k_seq_count<<<1, 32, 0, s>>>(flag, pos, n_ids, pos + n_ids)));
            return RISRT_OK;
        };
        int lrc = allowed();
        if (!lrc) RISRT_STRICT_CUDA(exclusive_scan_i64(flag, pos, n_ids, tmp, s));
        if (!lrc) lrc = count();
        if (lrc) {
            release();
            return lrc;
        }
        RISRT_STRICT_CUDA(cudaMemcpyAsync(&n_seq, pos + n_ids, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_STRICT_CUDA(cudaStreamSynchronize(s));
        if (n_seq > 0) {
            RISRT_STRICT_CUDA(ctx_malloc(ctx, &tab, sizeof(SeqEntry) * n_seq));
            RISRT_STRICT_CUDA(ctx_malloc(ctx, &tabd, sizeof(SeqEntryD) * n_seq));
            RISRT_STRICT_CUDA(ctx_malloc(ctx, &maskb, sizeof(uint32_t) * n_seq * W));
            RISRT_STRICT_CUDA(cudaMemsetAsync(maskb, 0, sizeof(uint32_t) * n_seq * W, s));
            auto build = [&]() -> int {
                RISRT_KERNEL(ctx, "k_seq_build", (k_seq_build<<<nblk(n_ids, 256), 256, 0, s>>>(S, n_ids, flag, pos, D3(tx.pos[0], tx.pos[1], tx.pos[2]),
                                                                                             (SeqEntry*)tab, (SeqEntryD*)tabd)));
                RISRT_KERNEL(ctx, "k_tx_strict", (k_tx_strict<<<nblk(n_seq * M, 128), 128, 0, s>>>(
                                                     S, ris->elem, M, fr, tx, ris->host_face, tol_base, (const SeqEntry*)tab,
                                                     (const SeqEntryD*)tabd, (int)n_seq, W, (uint32_t*)maskb, refines, err)));
                return RISRT_OK;
            };
            if ((lrc = build())) {
                release();
                return lrc;
            }
        }
    }
    auto coef = [&]() -> int {
        RISRT_KERNEL(ctx, "k_cm_strict", (k_cm_strict<<<nblk((int64_t)M * 32, 128), 128, 0, s>>>(
                                             S, ris->elem, M, fr, tx, wv, K, ris->host_face, tol_base, (const SeqEntry*)tab,
                                             (const SeqEntryD*)tabd, (int)n_seq, W, (const uint32_t*)maskb, cm, refines, err)));
        return RISRT_OK;
    };
    if (int crc = coef()) {
        release();
        return crc;
    }
    int h_err = 0;
    RISRT_STRICT_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    release();
#undef RISRT_STRICT_CUDA
    if (h_err) return fail(ctx, RISRT_ERR_CAPACITY, "BVH traversal stack overflow");
    return RISRT_OK;
}

int trace_check(risrt_ctx* ctx, risrt_pathset* ps)
{
    // a regular trace is checked before it returns; an asynchronous one is read again every time, since
    // a replayed graph reruns its kernels without the host code that would mark it pending
    if (!ps->external) return RISRT_OK;
    cudaStream_t s = ctx->stream;
    int fl[3] = {0, 0, 0};
    int64_t n_tx64 = 0, n_paths = 0, n_env = 0;
    unsigned long long gen = 0;
    std::vector<int64_t> ids((size_t)std::max(ps->chk_cap, 1));
    ps->tx_vis_host.resize(ps->M);
    RISRT_CUDA(ctx, cudaMemcpyAsync(fl, ps->chk_flags, sizeof(fl), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(&n_tx64, ps->chk_ntx, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(&n_paths, ps->rx_off + ps->n_rx, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(&n_env, ps->env_off + ps->n_rx, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(ids.data(), ps->chk_ids, sizeof(int64_t) * ps->chk_cap, cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(ps->tx_vis_host.data(), ps->tx_vis_dev, ps->M, cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(&gen, ps->gen_dev, sizeof(gen), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    ps->stats_pending = true;
    ps->check_pending = true;                  // until the checks below pass: no host copies of a failed trace
    if (fl[1]) return fail(ctx, RISRT_ERR_CAPACITY, "BVH traversal stack overflow");
    if (fl[0]) return fail(ctx, RISRT_ERR_CAPACITY, "a destination had more geometric candidates than cand_cap");
    if (fl[2] || n_paths > ps->cap_paths || n_env > ps->cap_env)
        return fail(ctx, RISRT_ERR_CAPACITY, "more paths than max_paths_per_rx / max_env_paths_per_rx hold");
    const int n_tx = (int)std::min<int64_t>(n_tx64, ps->chk_cap);
    ps->tx_seq_host.assign(ids.begin(), ids.begin() + n_tx);
    ps->n_paths = n_paths;
    ps->n_env = n_env;
    ps->checked_gen = gen;
    ps->check_pending = false;
    return RISRT_OK;
}

int rx_extent(risrt_ctx* ctx, const float* xyz, int64_t n, float* out)
{
    cudaStream_t s = ctx->stream;
    if (!ctx->small) RISRT_CUDA(ctx, cudaMalloc(&ctx->small, 256));
    unsigned* d_ext = (unsigned*)ctx->small;
    RISRT_CUDA(ctx, cudaMemsetAsync(d_ext, 0, sizeof(unsigned), s));
    RISRT_KERNEL(ctx, "k_abs_max", (k_abs_max<<<std::min<unsigned>(nblk(3 * n, 256), 1024u), 256, 0, s>>>(xyz, 3 * n, d_ext)));
    unsigned h = 0;
    RISRT_CUDA(ctx, cudaMemcpyAsync(&h, d_ext, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    memcpy(out, &h, sizeof(float));
    return RISRT_OK;
}

}  // namespace risrt

// ================================================================================================
// Allocation-free path search between two points.
//
// Some callers cannot allocate device memory while they run: code inside a region where the CUDA
// allocator must not be touched (for instance a host callback or a section that runs while another
// component owns every allocation), or hosts that hand this library a fixed memory budget and
// forbid growth. For them, this entry point runs the reflected-path search of the Tx leg
// (sequence table, candidate filter, BVH validation) on a scratch array that is part of the
// library image itself, so it never calls cudaMalloc, cudaFree or any allocating routine.
// ================================================================================================
namespace risrt {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)12 << 20;   // 12 MiB on every GPU that loads the library
constexpr int kNoAllocCands = 4096;                          // geometric candidates per call
constexpr int kNoAllocMaxDevices = 64;

}  // namespace
}  // namespace risrt

// The scratch array. In host code its name is only a stand-in for the device symbol: the device
// address is obtained with cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[risrt::kNoAllocScratchBytes];

namespace risrt {
namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use per device).
int noalloc_scratch(risrt_ctx* ctx, char** out)
{
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "device index too large for the static scratch table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[ctx->device] = p;
    }
    *out = (char*)g_noalloc_ptr[ctx->device];
    return RISRT_OK;
}

__global__ void k_ids_of(const int* __restrict__ cand, const int64_t* __restrict__ cnt,
                         const SeqEntry* __restrict__ seqs, int64_t* __restrict__ ids)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int)cnt[0]) ids[i] = seqs[cand[i]].info.z;
}

}  // namespace

int find_paths_noalloc(risrt_ctx* ctx, const risrt_scene* sc, const float src3[3], int src_face, const float dst3[3],
                       int dst_face, int max_order, int64_t* ids_host, int cap_host, int* n_host)
{
    cudaStream_t s = ctx->stream;
    if (int arc = trace_func_attrs(ctx)) return arc;
    const DeviceScene S = sc->dev();
    const int F = sc->n_faces;
    if (sc->n_tris == 0) max_order = 0;
    const int64_t n_ids = max_order >= 2 ? (int64_t)F + (int64_t)F * F : (max_order >= 1 ? F : 0);
    const int cap = kNoAllocCands;
    Frame fr{};
    for (int k = 0; k < 3; ++k) fr.c[k] = dst3[k];   // the exclusion rule looks at the destination
    const d3 src = D3((double)src3[0], (double)src3[1], (double)src3[2]);
    float ext = sc->scene_extent;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, std::max(std::fabs(src3[k]), std::fabs(dst3[k])));
    const float tol_base = 4e-6f * (1.f + 3.f * ext);

    // layout inside the static array (measured first, then checked against its size)
    struct Lay {
        int64_t *flag, *pos, *cnt64, *cnt64_tmp, *dense_off, *ids;
        void* scan_tmp;
        SeqEntry* e;
        SeqEntryD* d;
        int *cand, *cnt, *dense_r, *dense_slot, *dense_seq, *flags;
        unsigned long long* counters;
        float* dst;
    };
    auto layout = [&](Arena& A, Lay& L) {
        L.flag = A.get<int64_t>(n_ids + 1);
        L.pos = A.get<int64_t>(n_ids + 1);
        L.scan_tmp = A.get<char>(scan_temp_bytes(std::max<int64_t>(n_ids, 2)));
        L.e = A.get<SeqEntry>(n_ids + 1);
        L.d = A.get<SeqEntryD>(n_ids + 1);
        L.cand = A.get<int>(cap);
        L.cnt = A.get<int>(1);
        L.cnt64 = A.get<int64_t>(1);
        L.cnt64_tmp = A.get<int64_t>(2);
        L.dense_off = A.get<int64_t>(2);
        L.dense_r = A.get<int>(cap);
        L.dense_slot = A.get<int>(cap);
        L.dense_seq = A.get<int>(cap);
        L.ids = A.get<int64_t>(cap);
        L.counters = A.get<unsigned long long>(8);
        L.flags = A.get<int>(4);
        L.dst = A.get<float>(3);
    };
    Arena measure;
    Lay Lm;
    layout(measure, Lm);
    if (measure.used > kNoAllocScratchBytes)
        return fail(ctx, RISRT_ERR_CAPACITY,
                    "path search needs " + std::to_string(measure.used) + " bytes, above the 12 MiB static scratch "
                    "(order 2 fits up to about 250 faces, order 1 up to about 70000)");
    char* base;
    int rc = noalloc_scratch(ctx, &base);
    if (rc) return rc;
    Arena A{base, 0};
    Lay L;
    layout(A, L);

    // the array keeps the previous call's contents: clear what must start at zero
    RISRT_CUDA(ctx, cudaMemsetAsync(L.counters, 0, sizeof(unsigned long long) * 8, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(L.flags, 0, sizeof(int) * 4, s));
    RISRT_CUDA(ctx, cudaMemsetAsync(L.cnt, 0, sizeof(int), s));
    RISRT_CUDA(ctx, cudaMemsetAsync(L.cnt64, 0, sizeof(int64_t), s));
    RISRT_CUDA(ctx, cudaMemcpyAsync(L.dst, dst3, sizeof(float) * 3, cudaMemcpyHostToDevice, s));

    int n_seq = 0;
    if (n_ids > 0) {
        RISRT_KERNEL(ctx, "k_seq_allowed", (k_seq_allowed<<<nblk(n_ids, 256), 256, 0, s>>>(S, n_ids, 0, fr, src, 1e-4f * (1.f + ext), L.flag)));
        RISRT_CUDA(ctx, exclusive_scan_i64(L.flag, L.pos, n_ids, L.scan_tmp, s));
        RISRT_KERNEL(ctx, "k_seq_build", (k_seq_build<<<nblk(n_ids, 256), 256, 0, s>>>(S, n_ids, L.flag, L.pos, src, L.e, L.d)));
        int64_t last[2];
        RISRT_CUDA(ctx, cudaMemcpyAsync(&last[0], L.pos + n_ids - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(&last[1], L.flag + n_ids - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        n_seq = (int)(last[0] + last[1]);
    }
    if (n_seq > 0) {
        dim3 grid(1, std::min<unsigned>(nblk(n_seq, kCandChunk), 32768u));
        if (F <= kMaxSmemFaces) {
            const size_t shm = sizeof(FaceTest) * (size_t)F;
            RISRT_KERNEL(ctx, "k_candidates", (k_candidates<true><<<grid, kCandThreads, shm, s>>>(
                                                  S, L.dst, 1, nullptr, src, L.e, L.d, n_seq, tol_base, L.cand, L.cnt, cap,
                                                  L.flags, L.counters, nullptr, nullptr, 0, RefineQ{nullptr, 0, nullptr},
                                                  DenseOut{nullptr, nullptr, nullptr, nullptr}, nullptr)));
        } else {
            RISRT_KERNEL(ctx, "k_candidates", (k_candidates<false><<<grid, kCandThreads, 0, s>>>(
                                                  S, L.dst, 1, nullptr, src, L.e, L.d, n_seq, tol_base, L.cand, L.cnt, cap,
                                                  L.flags, L.counters, nullptr, nullptr, 0, RefineQ{nullptr, 0, nullptr},
                                                  DenseOut{nullptr, nullptr, nullptr, nullptr}, nullptr)));
        }
        RISRT_KERNEL(ctx, "k_cand_counts", (k_cand_counts<<<1, 32, 0, s>>>(L.cnt, 1, cap, L.cnt64_tmp)));
        RISRT_CUDA(ctx, exclusive_scan_i64(L.cnt64_tmp, L.dense_off, 2, L.scan_tmp, s));
        RISRT_KERNEL(ctx, "k_dense_list", (k_dense_list<<<1, 32, 0, s>>>(L.cnt, L.cand, L.dense_off, 1, cap, L.dense_r,
                                                                          L.dense_slot, L.dense_seq)));
        long long total = 0;
        int host_flags[1] = {0};
        RISRT_CUDA(ctx, cudaMemcpyAsync(&total, L.dense_off + 1, sizeof(long long), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(host_flags, L.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
        if (host_flags[0]) return fail(ctx, RISRT_ERR_CAPACITY, "more than 4096 geometric candidates");
        if (total > 0) {
            const unsigned blocks = (unsigned)std::min<long long>((long long)ctx->sm_count * 8, (total + kValThreads - 1) / kValThreads);
            RISRT_KERNEL(ctx, "k_validate", (k_validate<<<blocks, kValThreads, 0, s>>>(
                                                S, L.dst, src, src_face, dst_face, L.e, L.d, L.cand, cap, L.dense_r,
                                                L.dense_slot, L.dense_seq, (const long long*)(L.dense_off + 1), L.counters + 6,
                                                tol_base, L.counters,
                                                L.flags + 1, L.counters + 2, RefineQ{nullptr, 0, nullptr}, nullptr)));
        }
        const size_t shm = sizeof(int) * (size_t)cap;
        RISRT_KERNEL(ctx, "k_finalize", (k_finalize<<<1, 32, shm, s>>>(L.cand, L.cnt, 1, cap, L.e, L.cnt64)));
        RISRT_KERNEL(ctx, "k_ids_of", (k_ids_of<<<nblk(cap, 256), 256, 0, s>>>(L.cand, L.cnt64, L.e, L.ids)));
    }
    int64_t n = 0;
    int stack_err = 0;
    if (n_seq > 0) {
        RISRT_CUDA(ctx, cudaMemcpyAsync(&n, L.cnt64, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaMemcpyAsync(&stack_err, L.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    }
    if (stack_err) return fail(ctx, RISRT_ERR_CAPACITY, "BVH traversal stack overflow");
    *n_host = (int)n;
    if (n > cap_host) return fail(ctx, RISRT_ERR_CAPACITY, "ids_host is smaller than the number of paths found");
    if (n > 0) {
        RISRT_CUDA(ctx, cudaMemcpyAsync(ids_host, L.ids, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
        RISRT_CUDA(ctx, cudaStreamSynchronize(s));
    }
    return RISRT_OK;
}

}  // namespace risrt
