// Device geometry: segment occlusion by BVH traversal, point-in-face tests and the image-method
// back-trace (Sec. II-B). Decisions are filtered in FP32 and settled in FP64 when the FP32 margin
// does not decide them.
#pragma once

#include "frame.cuh"

namespace risrt {

// ------------------------------------------------------------------------------------------------
// triangle tests
// ------------------------------------------------------------------------------------------------

// Exact-in-FP64 decision: does segment a + s*dir, s in [0,1] (|dir| = len), hit the triangle at a
// distance in [kSegEps, len - kSegEps]? Inside is inclusive.
__device__ __forceinline__ bool tri_hit_fp64(const TriVerts& tv, d3 a, d3 dir, double len)
{
    d3 v0 = ldv(tv.v0), v1 = ldv(tv.v1), v2 = ldv(tv.v2);
    d3 nrm = cross(v1 - v0, v2 - v0);
    double nn = norm(nrm);
    double den = dot(nrm, dir);
    double num = dot(nrm, v0 - a);
    if (fabs(den) <= 1e-12 * nn * len) return false;
    double s = num / den;
    double dist = s * len;
    if (!(dist >= kSegEpsD && dist <= len - kSegEpsD)) return false;
    d3 q = a + dir * s;
    d3 nu = nrm * (1.0 / nn);
    d3 P[3] = {v0, v1, v2};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        d3 p = P[(i + 1) % 3], r = P[(i + 2) % 3];
        if (dot(cross(r - p, q - p), nu) < 0.0) return false;
    }
    return true;
}

// FP32 filter: 1 = certainly hit, 0 = certainly not, 2 = too close to call (settle in FP64).
__device__ __forceinline__ int tri_hit_fp32(const TriGeom& g, float3 a, float3 dir, float len, float tol_base)
{
    float3 n = xyz(g.plane);
    float den = dot(n, dir);
    float sa = dot(n, a) - g.plane.w;          // signed distance of the start
    float adn = fabsf(den);
    if (adn < 1e-3f * len) {                   // nearly parallel to the plane
        float sb = sa + den;
        float tol = tol_base;
        if ((sa > tol && sb > tol) || (sa < -tol && sb < -tol)) return 0;
        return 2;
    }
    float t = -sa / den;
    float dist = t * len;
    float tol = tol_base * (len / adn);
    if (dist < kSegEps - tol || dist > len - kSegEps + tol) return 0;
    float3 q = a + dir * t;
    float e0 = dot(xyz(g.edge[0]), q) - g.edge[0].w;
    float e1 = dot(xyz(g.edge[1]), q) - g.edge[1].w;
    float e2 = dot(xyz(g.edge[2]), q) - g.edge[2].w;
    float emin = fminf(e0, fminf(e1, e2));
    if (emin < -tol) return 0;
    if (emin > tol && dist > kSegEps + tol && dist < len - kSegEps - tol) return 1;
    return 2;
}

// ------------------------------------------------------------------------------------------------
// segment occlusion (any hit) by stack traversal of the binary BVH
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool box_overlap(float4 lo, float4 hi, float3 a, float3 inv)
{
    float tx0 = (lo.x - a.x) * inv.x, tx1 = (hi.x - a.x) * inv.x;
    float ty0 = (lo.y - a.y) * inv.y, ty1 = (hi.y - a.y) * inv.y;
    float tz0 = (lo.z - a.z) * inv.z, tz1 = (hi.z - a.z) * inv.z;
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), 1.f));
    return tmin <= tmax;
}

// Entry parameter of the segment into the box, or +inf when it misses.
__device__ __forceinline__ float box_entry(float4 lo, float4 hi, float3 a, float3 inv)
{
    float tx0 = (lo.x - a.x) * inv.x, tx1 = (hi.x - a.x) * inv.x;
    float ty0 = (lo.y - a.y) * inv.y, ty1 = (hi.y - a.y) * inv.y;
    float tz0 = (lo.z - a.z) * inv.z, tz1 = (hi.z - a.z) * inv.z;
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), 1.f));
    return tmin <= tmax ? tmin : __int_as_float(0x7f800000);
}

// Entry parameter with the segment's a * inv precomputed: one FMA per slab plane, t = lo inv - a inv.
__device__ __forceinline__ float box_entry_fma(float4 lo, float4 hi, float3 inv, float3 ainv)
{
    float tx0 = fmaf(lo.x, inv.x, -ainv.x), tx1 = fmaf(hi.x, inv.x, -ainv.x);
    float ty0 = fmaf(lo.y, inv.y, -ainv.y), ty1 = fmaf(hi.y, inv.y, -ainv.y);
    float tz0 = fmaf(lo.z, inv.z, -ainv.z), tz1 = fmaf(hi.z, inv.z, -ainv.z);
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), 1.f));
    return tmin <= tmax ? tmin : __int_as_float(0x7f800000);
}

// Reciprocal by one special-function instruction (about 1 ulp, denormal inputs flushed). Slab tests
// take it: every BVH box is padded by 1e-4 (1 + scene extent), many orders of magnitude above the
// position error an ulp of the inverse direction (or of a * inv) makes at the slab planes.
__device__ __forceinline__ float rcp_slab(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float safe_inv(float d) { return rcp_slab(fabsf(d) > 1e-20f ? d : copysignf(1e-20f, d)); }

struct TraceCounters {           // per thread (32 bits each; widened when flushed)
    unsigned cand, segs, nodes, tris;
};

// Warp-aggregated add of the per-thread counters (all lanes of the warp must call it).
__device__ __forceinline__ void flush_counters(const TraceCounters& t, unsigned long long* ctr)
{
    unsigned long long v[4] = {t.cand, t.segs, t.nodes, t.tris};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long x = v[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&ctr[i], x);
    }
}

// One step of a four-wide walk along the segment a + t dir, t in [0, 1] (inv = 1 / dir, ainv = a * inv):
// the children the segment enters, except subtrees made only of the faces g0 / g1, nearest entry
// first. Returns the nearest (kNoChild if none) and pushes the others farthest first; the caller keeps
// 3 free stack entries.
__device__ __forceinline__ int bvh4_step(const Bvh4Node& nd, float3 inv, float3 ainv, int g0, int g1, int* stack, int& sp)
{
    float t[4];
    int c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[k] = __float_as_int(nd.lo[k].w);
        const int f = __float_as_int(nd.hi[k].w);
        t[k] = (c[k] != kNoChild && f != g0 && f != g1) ? box_entry_fma(nd.lo[k], nd.hi[k], inv, ainv) : 3e38f;
    }
    auto cs = [&](int i, int j) {
        if (t[j] < t[i]) {
            const float tt = t[i]; t[i] = t[j]; t[j] = tt;
            const int cc = c[i]; c[i] = c[j]; c[j] = cc;
        }
    };
    cs(0, 1); cs(2, 3); cs(0, 2); cs(1, 3); cs(1, 2);
#pragma unroll
    for (int k = 3; k >= 1; --k)
        if (t[k] < 1e30f) stack[sp++] = c[k];
    return t[0] < 1e30f ? c[0] : kNoChild;
}

// Segment ends in the scene box (exact comparisons): a segment between two such points meets the plane
// of a shell triangle at most at an end or lies in it, and neither counts as a hit (hits closer than
// the tolerance to an end are ignored; a segment in a triangle's plane passes), so its traversal
// visits root_main only and never sees the shell.
__device__ __forceinline__ bool in_scene_box(const DeviceScene& S, float3 p)
{
    return p.x >= S.box_lo.x && p.y >= S.box_lo.y && p.z >= S.box_lo.z && p.x <= S.box_hi.x && p.y <= S.box_hi.y &&
           p.z <= S.box_hi.z;
}
__device__ __forceinline__ bool in_scene_box(const DeviceScene& S, d3 p)
{
    return p.x >= (double)S.box_lo.x && p.y >= (double)S.box_lo.y && p.z >= (double)S.box_lo.z &&
           p.x <= (double)S.box_hi.x && p.y <= (double)S.box_hi.y && p.z <= (double)S.box_hi.z;
}
// First node of an occlusion walk; a segment with an end outside the scene box also pushes the shell
// subtree onto the walk's stack. kNoRoot: nothing to visit.
__device__ __forceinline__ int occ_start(const DeviceScene& S, bool ends_in_box, int* stack, int& sp)
{
    int first = S.root_main;
    if (!ends_in_box && S.root_shell != kNoRoot) {
        if (first == kNoRoot) first = S.root_shell;
        else stack[sp++] = S.root_shell;
    }
    return first;
}

// Is segment a->b blocked (faces ign0 / ign1 skipped)? a, b: FP32 end points within a few ulps of
// the exact ones (the filter's tolerance covers that); in_box: both exact ends lie in the scene box
// (the shell subtree is then skipped); exact(A, B) gives the FP64 ends for the settlement of a
// triangle too close to call. `refines` counts FP64 settlements, `err` is set if the traversal stack
// would overflow (never expected; treated as blocked). With `unsure` set (int[3], zeroed by the
// caller), a triangle too close to call is not settled: unsure[0] counts them and unsure[1..2] keep
// the first two, and the walk goes on; a false return with unsure[0] > 0 means "unblocked unless one
// of those triangles is hit", for the caller to settle later (densely).
template <class Exact>
__device__ bool seg_blocked_f(const DeviceScene& S, float3 a, float3 b, bool in_box, int ign0, int ign1,
                              float tol_base, unsigned long long* refines, int* err, Exact exact,
                              TraceCounters* tc = nullptr, int* unsure = nullptr)
{
    int stack[64];
    int sp = 0;
    int c = occ_start(S, in_box, stack, sp);     // current node in a register;
    if (c == kNoRoot) return false;             // entered children go on the stack
    float3 dir = b - a;
    float len = sqrtf(dot(dir, dir));
    float3 inv = f3(safe_inv(dir.x), safe_inv(dir.y), safe_inv(dir.z));
    const float3 ainv = f3(a.x * inv.x, a.y * inv.y, a.z * inv.z);
    float tb = tol_base + 2e-7f * (fabsf(a.x) + fabsf(a.y) + fabsf(a.z) + len);
    const int g0 = ign0 >= 0 ? ign0 : -3, g1 = ign1 >= 0 ? ign1 : -3;   // subtrees of one ignored face are skipped
    while (true) {
        if (c < 0) {
            int i = ~c;
            int f = S.tri_face[i];
            if (f != ign0 && f != ign1) {
                if (tc) ++tc->tris;
                int r = tri_hit_fp32(S.tri_geom[i], a, dir, len, tb);
                if (r == 1) return true;
                if (r == 2) {
                    if (unsure) {
                        if (unsure[0] < 2) unsure[1 + unsure[0]] = i;
                        ++unsure[0];
                    } else {
                        if (refines) atomicAdd(refines, 1ull);
                        d3 A, B;
                        exact(A, B);
                        const d3 dirD = B - A;
                        if (tri_hit_fp64(S.tri_verts[i], A, dirD, norm(dirD))) return true;
                    }
                }
            }
            if (sp == 0) break;
            c = stack[--sp];
            continue;
        }
        if (sp + 3 > 64) {          // never expected (stack depth ~ 3 x tree depth / 2); treated as blocked
            if (err) atomicExch(err, 1);
            return true;
        }
        const Bvh4Node nd = S.nodes4[c];
        if (tc) ++tc->nodes;
        // any hit ends the query, so the children entered first along the segment are visited first
        c = bvh4_step(nd, inv, ainv, g0, g1, stack, sp);
        if (c == kNoChild) {
            if (sp == 0) break;
            c = stack[--sp];
        }
    }
    return false;
}

// The same for FP64 end points A, B (rounded to FP32 for the filter).
__device__ bool seg_blocked(const DeviceScene& S, d3 A, d3 B, int ign0, int ign1, float tol_base,
                           unsigned long long* refines, int* err, TraceCounters* tc = nullptr)
{
    return seg_blocked_f(S, to_f(A), to_f(B), in_scene_box(S, A) && in_scene_box(S, B), ign0, ign1, tol_base,
                         refines, err, [&](d3& x, d3& y) { x = A; y = B; }, tc);
}

// ------------------------------------------------------------------------------------------------
// point in face (union of the face's triangles, inclusive)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool in_face_fp64(const DeviceScene& S, int f, d3 q)
{
    const Face fc = S.faces[f];
    for (int j = fc.tri_begin; j < fc.tri_end; ++j) {
        const TriVerts tv = S.tri_verts[S.face_tris[j]];
        d3 v0 = ldv(tv.v0), v1 = ldv(tv.v1), v2 = ldv(tv.v2);
        d3 nrm = cross(v1 - v0, v2 - v0);
        double nn = norm(nrm);
        if (nn == 0.0) continue;
        d3 nu = nrm * (1.0 / nn);
        if (dot(cross(v2 - v1, q - v1), nu) < 0.0) continue;
        if (dot(cross(v0 - v2, q - v2), nu) < 0.0) continue;
        if (dot(cross(v1 - v0, q - v0), nu) < 0.0) continue;
        return true;
    }
    return false;
}

// FP32 classification: 1 inside, 0 outside, 2 too close to call.
__device__ __forceinline__ int in_face_fp32(const DeviceScene& S, int f, float3 q, float tol)
{
    const Face& fc = S.faces[f];
    int res = 0;
    for (int j = fc.tri_begin; j < fc.tri_end; ++j) {
        const TriGeom& g = S.tri_geom[S.face_tris[j]];
        float e0 = dot(xyz(g.edge[0]), q) - g.edge[0].w;
        float e1 = dot(xyz(g.edge[1]), q) - g.edge[1].w;
        float e2 = dot(xyz(g.edge[2]), q) - g.edge[2].w;
        float emin = fminf(e0, fminf(e1, e2));
        if (emin > tol) return 1;
        if (emin >= -tol) res = 2;
    }
    return res;
}

// FP32 classification against a convex face outline (4 edges; unused edges never bind).
__device__ __forceinline__ int in_outline_fp32(const FaceTest& t, float3 q, float tol)
{
    float emin = dot(xyz(t.e[0]), q) - t.e[0].w;
#pragma unroll
    for (int i = 1; i < 4; ++i) emin = fminf(emin, dot(xyz(t.e[i]), q) - t.e[i].w);
    if (emin > tol) return 1;
    if (emin < -tol) return 0;
    return 2;
}

// ------------------------------------------------------------------------------------------------
// face sequences
// ------------------------------------------------------------------------------------------------
struct SeqEntry {          // FP32 data for the candidate filter
    float4 sL;             // image of the source across every face of the sequence; w = signed
                           // distance to the last plane of the previous image (source for order 1)
    float4 pL;             // plane (n, d) of the last face (next to the destination)
    float4 s1;             // order 2: image across the first face only; w = signed distance of the
                           // source to the first plane
    float4 p1;             // order 2: plane of the first face
    int4 info;             // (f1, f2 or -1, id, order)
};
struct SeqEntryD {         // FP64 images for the settled decision and path points
    dv4 S1;            // image across the first face
    dv4 S2;            // order 2: image across both faces
};

// Full FP64 geometric check of a face sequence between src and dst (reflection points inside
// their faces, strictly same side at each bounce, back-trace parameter in (0,1)); pts gets
// src, P_1..P_k, dst.
__device__ __forceinline__ bool seq_geom_fp64(const DeviceScene& S, d3 src, d3 dst, const int4& info,
                                              const SeqEntryD& im, d3* pts)
{
    const int k = info.w;
    const int fa[2] = {info.x, info.y};
    d3 img[3] = {src, ld3(im.S1), ld3(im.S2)};
    pts[0] = src;
    pts[k + 1] = dst;
    d3 y = dst;
    bool ok = true;
    for (int j = k; j >= 1; --j) {
        const dv4 pl = S.faces[fa[j - 1]].plane;
        d3 n = ld3(pl);
        d3 d = img[j] - y;
        double den = dot(n, d);
        if (den == 0.0) return false;
        double t = (pl.w - dot(n, y)) / den;
        d3 p = y + d * t;
        pts[j] = p;
        if (!(t > 0.0 && t < 1.0)) ok = false;
        if (ok && !in_face_fp64(S, fa[j - 1], p)) ok = false;
        y = p;
    }
    if (!ok) return false;
    for (int j = 1; j <= k; ++j) {
        const dv4 pl = S.faces[fa[j - 1]].plane;
        d3 n = ld3(pl);
        double s1 = dot(n, pts[j - 1]) - pl.w, s2 = dot(n, pts[j + 1]) - pl.w;
        if (!(s1 * s2 > 0.0)) return false;
    }
    return true;
}

// Back-trace without checks (per-element geometry of an accepted sequence).
__device__ __forceinline__ void seq_points_fp64(const DeviceScene& S, d3 dst, const int4& info,
                                                const SeqEntryD& im, d3 src, d3* pts)
{
    const int k = info.w;
    const int fa[2] = {info.x, info.y};
    d3 img[3] = {src, ld3(im.S1), ld3(im.S2)};
    pts[0] = src;
    pts[k + 1] = dst;
    d3 y = dst;
    for (int j = k; j >= 1; --j) {
        const dv4 pl = S.faces[fa[j - 1]].plane;
        d3 n = ld3(pl);
        d3 d = img[j] - y;
        double t = (pl.w - dot(n, y)) / dot(n, d);
        pts[j] = y + d * t;
        y = pts[j];
    }
}

}  // namespace risrt
