// C ABI of the risrt library: argument validation, object lifetime and dispatch to the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>

#include "internal.cuh"
#include "sweep.cuh"

namespace risrt {

static thread_local std::string g_create_err;

int fail(risrt_ctx* ctx, int code, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return code;
}

std::atomic<long long> g_launches{0};

cudaError_t ctx_malloc(risrt_ctx* ctx, void** p, size_t bytes)
{
    if (bytes == 0) bytes = 1;
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->pool_mu);
        auto it = ctx->pool_free.lower_bound(bytes);
        if (it != ctx->pool_free.end() && it->first <= 2 * bytes + ((size_t)1 << 20)) {
            *p = it->second;
            ctx->pool_cached -= it->first;
            ctx->pool_free.erase(it);
            return cudaSuccess;
        }
    }
    // cached blocks count against the context's budget and may be what the device is missing: they are
    // released before a new block would exceed the budget, and before one more try after a failure
    auto release_cache = [&]() {
        std::lock_guard<std::mutex> lk(ctx->pool_mu);
        for (auto& kv : ctx->pool_free) {
            ctx->pool_size.erase(kv.second);
            ctx->allocated -= kv.first;
            cudaFree(kv.second);
        }
        ctx->pool_free.clear();
        ctx->pool_cached = 0;
    };
    if (ctx && ctx->budget) {
        bool over;
        {
            std::lock_guard<std::mutex> lk(ctx->pool_mu);
            over = ctx->allocated + bytes > ctx->budget;
        }
        if (over) release_cache();
        std::lock_guard<std::mutex> lk(ctx->pool_mu);
        if (ctx->allocated + bytes > ctx->budget) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        if (ctx) release_cache();
        cudaGetLastError();
        e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();                  // returned to the caller, not left for a launch check
            *p = nullptr;
            return e;
        }
    }
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->pool_mu);
        ctx->pool_size[*p] = bytes;
        ctx->allocated += bytes;
    }
    return cudaSuccess;
}

void ctx_free(risrt_ctx* ctx, void* p)
{
    if (!p) return;
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->pool_mu);
        auto it = ctx->pool_size.find(p);
        if (it != ctx->pool_size.end()) {
            if (ctx->pool_cached + it->second <= kPoolLimit) {
                ctx->pool_free.emplace(it->second, p);
                ctx->pool_cached += it->second;
                return;
            }
            ctx->allocated -= it->second;
            ctx->pool_size.erase(it);
        }
    }
    cudaFree(p);
}

void prof_begin(risrt_ctx* ctx, const char* name, cudaStream_t st)
{
    if (!ctx || !ctx->profiling) return;
    ctx->prof_skip = true;
    if (!ctx->prof_only.empty() && ctx->prof_only != name) return;
    KernelPending p;
    p.name = name;
    p.stream = st;
    int got = 0;
    for (cudaEvent_t* ev : {&p.a, &p.b}) {
        if (!ctx->event_pool.empty()) {
            *ev = ctx->event_pool.back();
            ctx->event_pool.pop_back();
        } else if (cudaEventCreate(ev) != cudaSuccess) {
            break;
        }
        ++got;
    }
    if (got < 2) {                       // no events: this launch goes unbracketed
        if (got == 1) ctx->event_pool.push_back(p.a);
        return;
    }
    ctx->prof_skip = false;
    cudaEventRecord(p.a, st);
    ctx->pending.push_back(p);
}

void prof_end(risrt_ctx* ctx)
{
    if (!ctx || !ctx->profiling || ctx->prof_skip || ctx->pending.empty()) return;
    cudaEventRecord(ctx->pending.back().b, ctx->pending.back().stream);
}

static void prof_collect(risrt_ctx* ctx)
{
    for (KernelPending& p : ctx->pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& slot = ctx->ktime[p.name];
        slot.first += ms;
        slot.second += 1;
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

int cuda_fail(risrt_ctx* ctx, cudaError_t e, const char* where)
{
    // the failure is returned here; clearing the thread's last-error state keeps a later launch
    // check from reporting it again (an error that breaks the context persists regardless)
    cudaGetLastError();
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? RISRT_ERR_OOM : RISRT_ERR_CUDA, m);
}

}  // namespace risrt

using namespace risrt;

namespace {

uint32_t spread16(uint32_t x)          // bits 0..15 of x to the even bits 0..30
{
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

struct TileLayout {
    size_t bb = 0, pairs = 0, elem = 0, ofs = 0, bytes = 0;
};

// Spatial tiles of a RIS for the direct legs: the elements in the Morton order of their (a, b)
// coordinates (quantised to 16 bits over the array's extent; ties by index), 32 consecutive ones per
// tile; per tile the bounds of its element centres, then per super-tile (four consecutive tiles) the
// bounds of its tiles; per visibility word (elements 32 w .. 32 w + 31)
// the tiles that hold its elements with the bits of those elements. One host buffer, laid out as
// tile bounds, word pairs, tile elements, word offsets.
TileLayout build_tiles(const float* uv, int M, std::vector<char>& buf, int& n_tiles)
{
    float amin = uv[0], amax = uv[0], bmin = uv[1], bmax = uv[1];
    for (int m = 1; m < M; ++m) {
        amin = std::min(amin, uv[2 * m]);
        amax = std::max(amax, uv[2 * m]);
        bmin = std::min(bmin, uv[2 * m + 1]);
        bmax = std::max(bmax, uv[2 * m + 1]);
    }
    const double sa = amax > amin ? 65535.0 / ((double)amax - amin) : 0.0;
    const double sb = bmax > bmin ? 65535.0 / ((double)bmax - bmin) : 0.0;
    std::vector<std::pair<uint32_t, int>> key(M);
    for (int m = 0; m < M; ++m) {
        const uint32_t qa = (uint32_t)std::llround(((double)uv[2 * m] - amin) * sa);
        const uint32_t qb = (uint32_t)std::llround(((double)uv[2 * m + 1] - bmin) * sb);
        key[m] = {spread16(qa) | (spread16(qb) << 1), m};
    }
    std::sort(key.begin(), key.end());
    const int T = (M + 31) / 32, W = (M + 31) / 32;
    n_tiles = T;
    std::vector<float4> bb(T, make_float4(3e38f, -3e38f, 3e38f, -3e38f));
    std::vector<int> elem((size_t)T * 32, -1);
    std::vector<std::vector<std::pair<int, unsigned>>> per_word(W);
    for (int i = 0; i < M; ++i) {
        const int t = i / 32, m = key[i].second;
        elem[(size_t)i] = m;
        float4& b = bb[t];
        b = make_float4(std::min(b.x, uv[2 * m]), std::max(b.y, uv[2 * m]), std::min(b.z, uv[2 * m + 1]),
                        std::max(b.w, uv[2 * m + 1]));
        auto& pw = per_word[m >> 5];
        if (pw.empty() || pw.back().first != t) pw.push_back({t, 0u});
        pw.back().second |= 1u << (m & 31);
    }
    // super-tiles: four consecutive tiles (128 elements consecutive in Morton order); their bounds
    // follow the tiles' in the same array
    for (int t = 0; t < T; t += 4) {
        float4 b = bb[t];
        for (int q = t + 1; q < std::min(T, t + 4); ++q)
            b = make_float4(std::min(b.x, bb[q].x), std::max(b.y, bb[q].y), std::min(b.z, bb[q].z), std::max(b.w, bb[q].w));
        bb.push_back(b);
    }
    std::vector<int> ofs(W + 1, 0);
    std::vector<int2> pairs;
    for (int w = 0; w < W; ++w) {
        std::sort(per_word[w].begin(), per_word[w].end());       // one pair per tile, tiles ascending
        std::vector<std::pair<int, unsigned>> merged;
        for (const auto& q : per_word[w]) {
            if (!merged.empty() && merged.back().first == q.first) merged.back().second |= q.second;
            else merged.push_back(q);
        }
        for (const auto& q : merged) pairs.push_back(make_int2(q.first, (int)q.second));
        ofs[w + 1] = (int)pairs.size();
    }
    TileLayout L;
    L.bb = 0;
    L.pairs = L.bb + sizeof(float4) * bb.size();
    L.elem = L.pairs + sizeof(int2) * pairs.size();
    L.ofs = L.elem + sizeof(int) * elem.size();
    L.bytes = L.ofs + sizeof(int) * ofs.size();
    buf.assign(L.bytes, 0);
    memcpy(buf.data() + L.bb, bb.data(), sizeof(float4) * bb.size());
    memcpy(buf.data() + L.pairs, pairs.data(), sizeof(int2) * pairs.size());
    memcpy(buf.data() + L.elem, elem.data(), sizeof(int) * elem.size());
    memcpy(buf.data() + L.ofs, ofs.data(), sizeof(int) * ofs.size());
    return L;
}

int set_device(risrt_ctx* ctx)
{
    // A non-sticky error that an earlier failed runtime call on this thread left behind (an
    // allocation another library retried, say) was returned to that call; discard it so the launch
    // checks of this call report only their own failures. A sticky error persists and shows again.
    cudaGetLastError();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return RISRT_OK;
}

#define RISRT_CHECK_CTX(ctx)                                   \
    do {                                                       \
        if (!(ctx)) return fail(nullptr, RISRT_ERR_INVALID_ARG, "null context"); \
        int _rc = set_device(ctx);                             \
        if (_rc) return _rc;                                   \
    } while (0)

}  // namespace

extern "C" {

int risrt_create(risrt_ctx** out, int device, void* stream, size_t hbm_budget_bytes)
{
    if (!out) return fail(nullptr, RISRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(nullptr, RISRT_ERR_INVALID_ARG, "device index out of range");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    risrt_ctx* c = new (std::nothrow) risrt_ctx();
    if (!c) return fail(nullptr, RISRT_ERR_OOM, "host allocation failed");
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->budget = hbm_budget_bytes;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return RISRT_OK;
}

int risrt_set_stream(risrt_ctx* ctx, void* stream)
{
    if (!ctx) return fail(nullptr, RISRT_ERR_INVALID_ARG, "null context");
    // blocks returned to the context's cache may still be in use by work on the old stream
    if ((cudaStream_t)stream != ctx->stream) RISRT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->stream = (cudaStream_t)stream;
    return RISRT_OK;
}

// Wait for everything the context enqueued: its stream and the side streams of its traces.
static void sync_ctx(risrt_ctx* ctx)
{
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (cudaStream_t st : ctx->side)
        if (st) cudaStreamSynchronize(st);
}

int risrt_destroy(risrt_ctx* ctx)
{
    if (!ctx) return RISRT_OK;
    sync_ctx(ctx);
    for (KernelPending& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (cudaStream_t st : ctx->side)
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (cudaEvent_t e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->small) cudaFree(ctx->small);
    for (auto& kv : ctx->pool_free) cudaFree(kv.second);   // blocks of live objects stay theirs
    delete ctx;
    return RISRT_OK;
}

int risrt_profile_enable(risrt_ctx* ctx, int on)
{
    RISRT_CHECK_CTX(ctx);
    ctx->profiling = on != 0;
    return RISRT_OK;
}

int risrt_profile_only(risrt_ctx* ctx, const char* name)
{
    RISRT_CHECK_CTX(ctx);
    ctx->prof_only = name ? name : "";
    return RISRT_OK;
}

int risrt_profile_query(risrt_ctx* ctx, const char* name, double* total_ms, int64_t* launches)
{
    RISRT_CHECK_CTX(ctx);
    prof_collect(ctx);
    double ms = 0.0;
    int64_t n = 0;
    for (auto& kv : ctx->ktime) {
        if (name && kv.first != name) continue;
        ms += kv.second.first;
        n += kv.second.second;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = n;
    return RISRT_OK;
}

int risrt_profile_names(risrt_ctx* ctx, char* buf, size_t cap, size_t* needed)
{
    RISRT_CHECK_CTX(ctx);
    prof_collect(ctx);
    std::string all;
    for (auto& kv : ctx->ktime) {
        if (!all.empty()) all += ",";
        all += kv.first;
    }
    if (needed) *needed = all.size() + 1;
    if (buf && cap > 0) {
        size_t n = std::min(cap - 1, all.size());
        memcpy(buf, all.data(), n);
        buf[n] = 0;
    }
    return RISRT_OK;
}

int risrt_profile_reset(risrt_ctx* ctx)
{
    RISRT_CHECK_CTX(ctx);
    prof_collect(ctx);
    ctx->ktime.clear();
    return RISRT_OK;
}

int risrt_launch_count(int64_t* out)
{
    if (!out) return RISRT_ERR_INVALID_ARG;
    *out = g_launches.load();
    return RISRT_OK;
}

const char* risrt_last_error(const risrt_ctx* ctx)
{
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

int risrt_scene_upload(risrt_ctx* ctx, const float* verts_host, int64_t n_verts, const int32_t* tris_host,
                       const int32_t* face_id_host, const int32_t* mat_id_host, int64_t n_tris,
                       const float* mats_host, int32_t n_mat, risrt_scene** out)
{
    RISRT_CHECK_CTX(ctx);
    if (!out) return fail(ctx, RISRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_tris < 0 || n_verts < 0 || n_mat < 1 || !mats_host) return fail(ctx, RISRT_ERR_INVALID_ARG, "bad sizes");
    if (n_tris > (int64_t)1 << 26) return fail(ctx, RISRT_ERR_INVALID_ARG, "n_tris above 2^26");
    if (n_tris > 0 && (!verts_host || !tris_host || !face_id_host || !mat_id_host))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL scene array");
    int F = 0;
    for (int64_t t = 0; t < n_tris; ++t) {
        for (int j = 0; j < 3; ++j)
            if (tris_host[3 * t + j] < 0 || tris_host[3 * t + j] >= n_verts)
                return fail(ctx, RISRT_ERR_INVALID_ARG, "triangle vertex index out of range");
        if (face_id_host[t] < 0) return fail(ctx, RISRT_ERR_INVALID_ARG, "negative face id");
        if (mat_id_host[t] < 0 || mat_id_host[t] >= n_mat) return fail(ctx, RISRT_ERR_INVALID_ARG, "material index out of range");
        F = std::max(F, face_id_host[t] + 1);
    }
    std::vector<char> used(F, 0);
    for (int64_t t = 0; t < n_tris; ++t) used[face_id_host[t]] = 1;
    for (int f = 0; f < F; ++f)
        if (!used[f]) return fail(ctx, RISRT_ERR_INVALID_ARG, "face ids must be 0..F-1 without gaps");
    for (int64_t i = 0; i < 3 * n_verts; ++i)
        if (!std::isfinite(verts_host[i])) return fail(ctx, RISRT_ERR_INVALID_ARG, "non-finite vertex");
    for (int i = 0; i < n_mat; ++i)
        if (!(mats_host[2 * i] >= 1.0f) || !(mats_host[2 * i + 1] >= 0.0f))
            return fail(ctx, RISRT_ERR_INVALID_ARG, "material needs eps_r >= 1 and sigma >= 0");
    risrt_scene* sc = new (std::nothrow) risrt_scene();
    if (sc) sc->owner = ctx;
    if (!sc) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
    sc->n_tris = n_tris;
    sc->n_faces = F;
    int rc = build_scene(ctx, sc, verts_host, n_verts, tris_host, face_id_host, mat_id_host, mats_host, n_mat);
    if (rc) {
        risrt_scene_destroy(ctx, sc);
        return rc;
    }
    *out = sc;
    return RISRT_OK;
}

int risrt_ris_upload(risrt_ctx* ctx, const float* elem_uv_host, int32_t M, const float center[3], const float t1[3],
                     const float t2[3], float dy, float dz, float elem_gain, int32_t host_face, risrt_ris** out)
{
    RISRT_CHECK_CTX(ctx);
    if (!out) return fail(ctx, RISRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (M < 1 || M > 65536 || !elem_uv_host || !center || !t1 || !t2)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "RIS needs 1 <= M <= 65536 and non-NULL arrays");
    if (!(dy > 0.f) || !(dz > 0.f)) return fail(ctx, RISRT_ERR_INVALID_ARG, "element size must be positive");
    double n1 = 0, n2 = 0, d12 = 0;
    for (int k = 0; k < 3; ++k) {
        n1 += (double)t1[k] * t1[k];
        n2 += (double)t2[k] * t2[k];
        d12 += (double)t1[k] * t2[k];
    }
    if (std::fabs(n1 - 1) > 1e-5 || std::fabs(n2 - 1) > 1e-5 || std::fabs(d12) > 1e-5)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "t1, t2 must be orthonormal");
    risrt_ris* r = new (std::nothrow) risrt_ris();
    if (!r) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
    r->owner = ctx;
    r->M = M;
    memcpy(r->center, center, sizeof(float) * 3);
    memcpy(r->t1, t1, sizeof(float) * 3);
    memcpy(r->t2, t2, sizeof(float) * 3);
    r->dy = dy;
    r->dz = dz;
    r->elem_gain = elem_gain;
    r->host_face = host_face;
    r->uv_host.assign(elem_uv_host, elem_uv_host + 2 * (size_t)M);
    std::vector<float4> e(M);
    for (int m = 0; m < M; ++m) {
        float a = elem_uv_host[2 * m], b = elem_uv_host[2 * m + 1];
        if (!std::isfinite(a) || !std::isfinite(b)) {
            delete r;
            return fail(ctx, RISRT_ERR_INVALID_ARG, "non-finite element coordinate");
        }
        e[m] = make_float4(a, b, a * a + b * b, 0.f);
    }
    cudaError_t err = ctx_malloc(ctx, (void**)&r->elem, sizeof(float4) * M);
    if (err != cudaSuccess) {
        delete r;
        return cuda_fail(ctx, err, "cudaMalloc");
    }
    err = cudaMemcpyAsync(r->elem, e.data(), sizeof(float4) * M, cudaMemcpyHostToDevice, ctx->stream);
    std::vector<char> tiles;
    if (err == cudaSuccess && M > kTileMinElems) {
        const TileLayout tl = build_tiles(elem_uv_host, M, tiles, r->n_tiles);
        err = ctx_malloc(ctx, &r->tile_buf, tiles.size());
        if (err == cudaSuccess) {
            char* b = (char*)r->tile_buf;
            r->tile_bb = (float4*)(b + tl.bb);
            r->word_tile = (int2*)(b + tl.pairs);
            r->tile_elem = (int*)(b + tl.elem);
            r->word_ofs = (int*)(b + tl.ofs);
            err = cudaMemcpyAsync(r->tile_buf, tiles.data(), tiles.size(), cudaMemcpyHostToDevice, ctx->stream);
        }
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
    if (err != cudaSuccess) {
        ctx_free(ctx, r->elem);
        ctx_free(ctx, r->tile_buf);
        delete r;
        return cuda_fail(ctx, err, "element upload");
    }
    *out = r;
    return RISRT_OK;
}

int risrt_antenna_set(risrt_ctx* ctx, int which, const float pos[3], const float orient3x3[9], float power_w,
                      float gain_lin, int pattern)
{
    RISRT_CHECK_CTX(ctx);
    if (which != RISRT_TX && which != RISRT_RX) return fail(ctx, RISRT_ERR_INVALID_ARG, "which must be RISRT_TX or RISRT_RX");
    if (!orient3x3) return fail(ctx, RISRT_ERR_INVALID_ARG, "orientation is NULL");
    if (pattern < RISRT_PATTERN_ISO || pattern > RISRT_PATTERN_MONOPOLE_QW) return fail(ctx, RISRT_ERR_INVALID_ARG, "unknown pattern");
    if (!(gain_lin > 0.f)) return fail(ctx, RISRT_ERR_INVALID_ARG, "gain must be positive");
    double zn = 0;
    for (int k = 6; k < 9; ++k) zn += (double)orient3x3[k] * orient3x3[k];
    if (!(zn > 0)) return fail(ctx, RISRT_ERR_INVALID_ARG, "orientation z axis is zero");
    Antenna a{};
    if (which == RISRT_TX) {
        if (!pos) return fail(ctx, RISRT_ERR_INVALID_ARG, "Tx position is NULL");
        if (!(power_w >= 0.f)) return fail(ctx, RISRT_ERR_INVALID_ARG, "power must be >= 0");
        memcpy(a.pos, pos, sizeof(float) * 3);
    }
    memcpy(a.orient, orient3x3, sizeof(float) * 9);
    a.power_w = power_w;
    a.gain_lin = gain_lin;
    a.pattern = pattern;
    a.set = true;
    if (which == RISRT_TX) ctx->tx = a;
    else ctx->rx = a;
    return RISRT_OK;
}

int risrt_rx_upload(risrt_ctx* ctx, const float* rx_xyz_host, int64_t n_rx, risrt_rxset** out)
{
    RISRT_CHECK_CTX(ctx);
    if (!out) return fail(ctx, RISRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_rx < 1 || n_rx > ((int64_t)1 << 26) || !rx_xyz_host) return fail(ctx, RISRT_ERR_INVALID_ARG, "need 1 <= n_rx <= 2^26");
    risrt_rxset* r = new (std::nothrow) risrt_rxset();
    if (!r) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
    r->owner = ctx;
    r->n = n_rx;
    r->owned = true;
    cudaError_t e = ctx_malloc(ctx, (void**)&r->xyz, sizeof(float) * 3 * n_rx);
    if (e != cudaSuccess) {
        delete r;
        return cuda_fail(ctx, e, "cudaMalloc");
    }
    e = cudaMemcpyAsync(r->xyz, rx_xyz_host, sizeof(float) * 3 * n_rx, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        ctx_free(ctx, r->xyz);
        delete r;
        return cuda_fail(ctx, e, "cudaMemcpyAsync");
    }
    float ext = 0.f;                  // largest |coordinate| (the traces' FP32 error bounds use it)
    for (int64_t i = 0; i < 3 * n_rx; ++i) ext = std::max(ext, std::fabs(rx_xyz_host[i]));
    r->ext = ext;
    *out = r;
    return RISRT_OK;
}

int risrt_rx_bind(risrt_ctx* ctx, const float* rx_xyz, int64_t n_rx, risrt_rxset** out)
{
    RISRT_CHECK_CTX(ctx);
    if (!out) return fail(ctx, RISRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_rx < 1 || n_rx > ((int64_t)1 << 26) || !rx_xyz) return fail(ctx, RISRT_ERR_INVALID_ARG, "need 1 <= n_rx <= 2^26");
    risrt_rxset* r = new (std::nothrow) risrt_rxset();
    if (!r) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
    r->owner = ctx;
    r->n = n_rx;
    r->xyz = const_cast<float*>(rx_xyz);
    r->owned = false;
    float ext = 0.f;
    int rc = rx_extent(ctx, rx_xyz, n_rx, &ext);
    if (rc) {
        delete r;
        return rc;
    }
    r->ext = ext;
    *out = r;
    return RISRT_OK;
}

int risrt_trace_paths(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                      double freq_hz, int32_t max_order_tx, int32_t max_order_rx, uint32_t flags, risrt_pathset** inout)
{
    RISRT_CHECK_CTX(ctx);
    if (!scene || !ris || !rxset || !inout) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->tx.set || !ctx->rx.set) return fail(ctx, RISRT_ERR_NOT_READY, "Tx and Rx antennas must be set");
    if (!(freq_hz > 0) || !std::isfinite(freq_hz)) return fail(ctx, RISRT_ERR_INVALID_ARG, "frequency must be positive");
    if (max_order_tx < 0 || max_order_tx > 2 || max_order_rx < 0 || max_order_rx > 2)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "orders must be in [0, 2]");
    if ((max_order_tx == 2 || max_order_rx == 2) && scene->n_faces > 40000)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "order 2 supports at most 40000 faces");
    if (ris->host_face >= scene->n_faces) return fail(ctx, RISRT_ERR_INVALID_ARG, "host_face out of range");
    if (flags & ~(uint32_t)(RISRT_FLAG_ENV_PATHS | RISRT_FLAG_FRESNEL_TM)) return fail(ctx, RISRT_ERR_INVALID_ARG, "unknown flag");
    risrt_pathset* ps = *inout;
    bool created = false;
    if (ps && ps->external) return fail(ctx, RISRT_ERR_INVALID_ARG, "the path set lives in a workspace: trace it with risrt_trace_paths_async");
    if (!ps) {
        ps = new (std::nothrow) risrt_pathset();
        if (ps) ps->owner = ctx;
        if (!ps) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
        created = true;
    }
    int rc = trace_paths(ctx, scene, ris, rxset, freq_hz, max_order_tx, max_order_rx, flags, ps);
    if (rc) {
        if (created) risrt_pathset_destroy(ctx, ps);
        return rc;
    }
    *inout = ps;
    return RISRT_OK;
}

static int check_trace_args(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                            int32_t max_order_tx, int32_t max_order_rx, uint32_t flags, const risrt_trace_limits* lim)
{
    if (!scene || !ris || !rxset || !lim) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->tx.set || !ctx->rx.set) return fail(ctx, RISRT_ERR_NOT_READY, "Tx and Rx antennas must be set");
    if (max_order_tx < 0 || max_order_tx > 2 || max_order_rx < 0 || max_order_rx > 2)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "orders must be in [0, 2]");
    if ((max_order_tx == 2 || max_order_rx == 2) && scene->n_faces > 40000)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "order 2 supports at most 40000 faces");
    if (ris->host_face >= scene->n_faces) return fail(ctx, RISRT_ERR_INVALID_ARG, "host_face out of range");
    if (flags & ~(uint32_t)(RISRT_FLAG_ENV_PATHS | RISRT_FLAG_FRESNEL_TM)) return fail(ctx, RISRT_ERR_INVALID_ARG, "unknown flag");
    if (lim->cand_cap < 1 || lim->cand_cap > (1 << 16) || lim->max_paths_per_rx < 1 || lim->max_env_paths_per_rx < 0)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "limits out of range");
    return RISRT_OK;
}

int risrt_trace_workspace_size(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                               int32_t max_order_tx, int32_t max_order_rx, uint32_t flags, const risrt_trace_limits* lim,
                               size_t* bytes)
{
    RISRT_CHECK_CTX(ctx);
    if (!bytes) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (int rc = check_trace_args(ctx, scene, ris, rxset, max_order_tx, max_order_rx, flags, lim)) return rc;
    risrt_pathset probe;
    AsyncTrace at;
    at.cand_cap = lim->cand_cap;
    at.max_paths = lim->max_paths_per_rx;
    at.max_env = lim->max_env_paths_per_rx;
    at.need = bytes;
    return trace_paths(ctx, scene, ris, rxset, 1e9, max_order_tx, max_order_rx, flags, &probe, &at);
}

int risrt_trace_paths_async(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                            double freq_hz, int32_t max_order_tx, int32_t max_order_rx, uint32_t flags,
                            const risrt_trace_limits* lim, void* workspace, size_t workspace_bytes, risrt_pathset** inout)
{
    RISRT_CHECK_CTX(ctx);
    if (!inout || !workspace) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (int rc = check_trace_args(ctx, scene, ris, rxset, max_order_tx, max_order_rx, flags, lim)) return rc;
    if (!(freq_hz > 0) || !std::isfinite(freq_hz)) return fail(ctx, RISRT_ERR_INVALID_ARG, "frequency must be positive");
    if ((uintptr_t)workspace & 255u) return fail(ctx, RISRT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    risrt_pathset* ps = *inout;
    bool created = false;
    if (ps && !ps->external) return fail(ctx, RISRT_ERR_INVALID_ARG, "the path set was filled by risrt_trace_paths");
    if (!ps) {
        ps = new (std::nothrow) risrt_pathset();
        if (!ps) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
        ps->owner = ctx;
        created = true;
    }
    AsyncTrace at;
    at.ws = workspace;
    at.bytes = workspace_bytes;
    at.cand_cap = lim->cand_cap;
    at.max_paths = lim->max_paths_per_rx;
    at.max_env = lim->max_env_paths_per_rx;
    int rc = trace_paths(ctx, scene, ris, rxset, freq_hz, max_order_tx, max_order_rx, flags, ps, &at);
    if (rc) {
        if (created) delete ps;
        return rc;
    }
    *inout = ps;
    return RISRT_OK;
}

int risrt_trace_check(risrt_ctx* ctx, risrt_pathset* ps)
{
    RISRT_CHECK_CTX(ctx);
    if (!ps) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL path set");
    return trace_check(ctx, ps);
}

// Waits for the trace that filled ps and brings its device-side statistics to the host (once per
// trace). An asynchronous trace's host copies are current only if no run of it (a graph replay
// included) came after its last risrt_trace_check: RISRT_ERR_NOT_READY otherwise.
static int pathset_sync(const risrt_pathset* ps)
{
    if (ps->check_pending) return RISRT_ERR_NOT_READY;       // an asynchronous trace not checked yet
    if (ps->stream && cudaStreamSynchronize(ps->stream) != cudaSuccess) return RISRT_ERR_CUDA;
    if (ps->external) {
        unsigned long long gen = 0;
        if (cudaMemcpy(&gen, ps->gen_dev, sizeof(gen), cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
        if (gen != ps->checked_gen) return RISRT_ERR_NOT_READY;
    }
    if (ps->stats_pending) {
        unsigned long long c[6];
        if (cudaMemcpy(c, ps->ctr_dev, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
        ps->fp64_refines = (int64_t)c[0];
        ps->units = (int64_t)c[1];
        ps->n_candidates = (int64_t)c[2];
        ps->n_segments = (int64_t)c[3];
        ps->node_visits = (int64_t)c[4];
        ps->tri_tests = (int64_t)c[5];
        ps->stats_pending = false;
    }
    return RISRT_OK;
}

int risrt_pathset_stats_get(const risrt_pathset* ps, risrt_pathset_stats* out)
{
    if (!ps || !out) return RISRT_ERR_INVALID_ARG;
    if (int rc = pathset_sync(ps)) return rc;
    out->n_rx = ps->n_rx;
    out->M = ps->M;
    out->n_faces = ps->n_faces;
    out->n_rx_paths = ps->n_paths;
    out->n_env_paths = ps->n_env;
    out->n_tx_paths = (int32_t)ps->tx_seq_host.size();
    out->units = ps->units;
    out->fp64_refines = ps->fp64_refines;
    out->n_candidates = ps->n_candidates;
    out->n_segments = ps->n_segments;
    out->node_visits = ps->node_visits;
    out->tri_tests = ps->tri_tests;
    return RISRT_OK;
}

int risrt_pathset_export(const risrt_pathset* ps, int32_t* rx_count_host, int64_t* rx_seq_host, int32_t* env_count_host,
                         int64_t* env_seq_host, uint8_t* los_host, uint32_t* vis_host, int64_t* tx_seq_host,
                         uint8_t* tx_vis_host)
{
    if (!ps) return RISRT_ERR_INVALID_ARG;
    if (int rc = pathset_sync(ps)) return rc;
    const int64_t n = ps->n_rx;
    std::vector<int64_t> off(n + 1), eoff(n + 1);
    if (cudaMemcpy(off.data(), ps->rx_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
    if (cudaMemcpy(eoff.data(), ps->env_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
    // the caller sized its arrays from the counts on the host: the offsets must agree with them
    if (off[n] != ps->n_paths || eoff[n] != ps->n_env) return RISRT_ERR_NOT_READY;
    if (rx_count_host)
        for (int64_t r = 0; r < n; ++r) rx_count_host[r] = (int32_t)(off[r + 1] - off[r] - 1);
    if (rx_seq_host && ps->n_paths > 0) {
        std::vector<int64_t> all(ps->n_paths);
        if (cudaMemcpy(all.data(), ps->rx_seq, sizeof(int64_t) * ps->n_paths, cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
        int64_t k = 0;
        for (int64_t r = 0; r < n; ++r)
            for (int64_t i = off[r] + 1; i < off[r + 1]; ++i) rx_seq_host[k++] = all[i];
    }
    if (env_count_host)
        for (int64_t r = 0; r < n; ++r) env_count_host[r] = (int32_t)(eoff[r + 1] - eoff[r]);
    if (env_seq_host && ps->n_env > 0)
        if (cudaMemcpy(env_seq_host, ps->env_seq, sizeof(int64_t) * ps->n_env, cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
    if (los_host)
        if (cudaMemcpy(los_host, ps->los, n, cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
    if (vis_host)
        if (cudaMemcpy(vis_host, ps->vis, sizeof(uint32_t) * n * ps->W, cudaMemcpyDeviceToHost) != cudaSuccess) return RISRT_ERR_CUDA;
    if (tx_seq_host)
        for (size_t i = 0; i < ps->tx_seq_host.size(); ++i) tx_seq_host[i] = ps->tx_seq_host[i];
    if (tx_vis_host)
        for (int m = 0; m < ps->M; ++m) tx_vis_host[m] = ps->tx_vis_host[m];
    return RISRT_OK;
}

int risrt_eval_field(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, int32_t n_cfg, float* E_out, float* P_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!ps || !gamma || !E_out) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (n_cfg < 1) return fail(ctx, RISRT_ERR_INVALID_ARG, "n_cfg must be >= 1");
    if (((uintptr_t)gamma | (uintptr_t)E_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    return eval_field(ctx, ps, (const float2*)gamma, n_cfg, (float2*)E_out, P_out);
}

int risrt_eval_field_plain(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, int32_t n_cfg, float* E_out,
                           float* P_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!ps || !gamma || !E_out) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (n_cfg < 1) return fail(ctx, RISRT_ERR_INVALID_ARG, "n_cfg must be >= 1");
    if (((uintptr_t)gamma | (uintptr_t)E_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    return eval_field_plain(ctx, ps, (const float2*)gamma, n_cfg, (float2*)E_out, P_out);
}

int risrt_eval_field_strict(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                            double freq_hz, int32_t max_order_tx, int32_t max_order_rx, uint32_t flags, const float* gamma,
                            int32_t n_cfg, float* E_out, float* P_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!scene || !ris || !rxset || !gamma || !E_out) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->tx.set || !ctx->rx.set) return fail(ctx, RISRT_ERR_NOT_READY, "antennas not set");
    if (!(freq_hz > 0) || max_order_tx < 0 || max_order_tx > 2 || max_order_rx < 0 || max_order_rx > 2 || n_cfg < 1 ||
        (flags & ~(uint32_t)(RISRT_FLAG_ENV_PATHS | RISRT_FLAG_FRESNEL_TM)))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "bad frequency, order, configuration count or flags");
    if (((uintptr_t)gamma | (uintptr_t)E_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    return eval_field_strict(ctx, scene, ris, rxset, freq_hz, max_order_tx, max_order_rx, flags, (const float2*)gamma,
                             n_cfg, (float2*)E_out, P_out);
}

int risrt_antenna_set_polarization(risrt_ctx* ctx, int which, const float axis[3])
{
    RISRT_CHECK_CTX(ctx);
    if (which != RISRT_TX && which != RISRT_RX) return fail(ctx, RISRT_ERR_INVALID_ARG, "which must be RISRT_TX or RISRT_RX");
    if (!axis) return fail(ctx, RISRT_ERR_INVALID_ARG, "axis is NULL");
    const double n = std::sqrt((double)axis[0] * axis[0] + (double)axis[1] * axis[1] + (double)axis[2] * axis[2]);
    if (!(n > 0) || !std::isfinite(n)) return fail(ctx, RISRT_ERR_INVALID_ARG, "axis must be a finite non-zero vector");
    for (int k = 0; k < 3; ++k) ctx->pol[which][k] = (float)(axis[k] / n);
    ctx->pol_set[which] = true;
    return RISRT_OK;
}

// Shared checks of the vector-field calls: the scene and receivers the path set was traced with, both
// polarisation axes set, and an asynchronous path set checked since its last run.
static int check_vec_args(risrt_ctx* ctx, const risrt_scene* scene, const risrt_rxset* rxset, const risrt_pathset* ps)
{
    if (!scene || !rxset || !ps) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->pol_set[RISRT_TX] || !ctx->pol_set[RISRT_RX])
        return fail(ctx, RISRT_ERR_NOT_READY, "set both polarisation axes (risrt_antenna_set_polarization)");
    if (rxset->n != ps->n_rx || scene->n_faces != ps->n_faces)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "scene and receivers must be those the path set was traced with");
    if (ps->external)
        if (int rc = pathset_sync(ps))
            return fail(ctx, rc, rc == RISRT_ERR_NOT_READY ? "call risrt_trace_check after an asynchronous trace" : "CUDA error");
    return RISRT_OK;
}

int risrt_eval_field_vec(risrt_ctx* ctx, const risrt_scene* scene, const risrt_rxset* rxset, const risrt_pathset* ps,
                         const float* gamma, int32_t n_cfg, float* E_out, float* E3_out, float* P_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!gamma || !E_out || n_cfg < 1) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument or n_cfg < 1");
    if (((uintptr_t)gamma | (uintptr_t)E_out | (uintptr_t)E3_out) & 7u)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    if (int rc = check_vec_args(ctx, scene, rxset, ps)) return rc;
    return eval_field_vec(ctx, scene, rxset, ps, (const float2*)gamma, n_cfg, (float2*)E_out, (float2*)E3_out, P_out);
}

int risrt_build_A_vec(risrt_ctx* ctx, const risrt_scene* scene, const risrt_rxset* rxset, const risrt_pathset* ps,
                      float* A_out, float* E0_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!A_out) return fail(ctx, RISRT_ERR_INVALID_ARG, "A_out is NULL");
    if (((uintptr_t)A_out | (uintptr_t)E0_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    if (int rc = check_vec_args(ctx, scene, rxset, ps)) return rc;
    return build_A_vec(ctx, scene, rxset, ps, (float2*)A_out, (float2*)E0_out);
}

int risrt_eval_cir(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, float* taps_out, double* rx_delay_out,
                   double* tx_delay_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!ps || !gamma || !taps_out || !rx_delay_out || !tx_delay_out) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)gamma | (uintptr_t)taps_out | (uintptr_t)rx_delay_out | (uintptr_t)tx_delay_out) & 7u)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "arrays must be 8-byte aligned");
    if (int rc = pathset_sync(ps))
        return fail(ctx, rc, rc == RISRT_ERR_NOT_READY ? "call risrt_trace_check after an asynchronous trace" : "CUDA error");
    return eval_cir(ctx, ps, (const float2*)gamma, (float2*)taps_out, rx_delay_out, tx_delay_out);
}

int risrt_microbench(risrt_ctx* ctx, int kind, int32_t iters, double* ops_per_s, double* ms)
{
    RISRT_CHECK_CTX(ctx);
    if (!ops_per_s || iters < 1 || kind < RISRT_MB_FFMA || kind > RISRT_MB_DFMA)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "bad microbenchmark arguments");
    return microbench(ctx, kind, iters, ops_per_s, ms);
}

int risrt_build_A(risrt_ctx* ctx, const risrt_pathset* ps, float* A_out, float* E0_out, risrt_amat** resident_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!ps || (!A_out && !resident_out)) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL path set, or neither A_out nor resident_out");
    if (((uintptr_t)A_out | (uintptr_t)E0_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    if (resident_out) *resident_out = nullptr;
    risrt_amat* h = nullptr;
    if (resident_out) {
        h = new (std::nothrow) risrt_amat();
        if (!h) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
        h->owner = ctx;
        h->n_rx = ps->n_rx;
        h->M = ps->M;
    }
    float2* A = (float2*)A_out;
    float2* E0 = (float2*)E0_out;
    if (!A_out) {               // resident: the library holds A and E0 in blocks of this context
        void* a = nullptr;
        void* e = nullptr;
        cudaError_t err = ctx_malloc(ctx, &a, sizeof(float2) * (size_t)ps->n_rx * ps->M);
        if (err == cudaSuccess) err = ctx_malloc(ctx, &e, sizeof(float2) * (size_t)ps->n_rx);
        if (err != cudaSuccess) {
            ctx_free(ctx, a);
            delete h;
            return cuda_fail(ctx, err, "channel matrix allocation");
        }
        A = (float2*)a;
        E0 = (float2*)e;
        h->owned = true;
    }
    int rc = build_A(ctx, ps, A, E0);
    if (rc) {
        if (h && h->owned) {
            sync_ctx(ctx);
            ctx_free(ctx, A);
            ctx_free(ctx, E0);
        }
        delete h;
        return rc;
    }
    if (h) {
        h->A = A;
        h->E0 = E0;
        *resident_out = h;
    }
    return RISRT_OK;
}

int risrt_amat_wrap(risrt_ctx* ctx, const float* A, const float* E0, int64_t n_rx, int32_t M, risrt_amat** out)
{
    RISRT_CHECK_CTX(ctx);
    if (!A || !out) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    if (n_rx < 1 || n_rx > ((int64_t)1 << 26) || M < 1 || M > 65536) return fail(ctx, RISRT_ERR_INVALID_ARG, "sizes out of range");
    if (((uintptr_t)A | (uintptr_t)E0) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    risrt_amat* h = new (std::nothrow) risrt_amat();
    if (!h) return fail(ctx, RISRT_ERR_OOM, "host allocation failed");
    h->owner = ctx;
    h->A = (const float2*)A;
    h->E0 = (const float2*)E0;
    h->n_rx = n_rx;
    h->M = M;
    *out = h;
    return RISRT_OK;
}

int risrt_amat_data(const risrt_amat* amat, const float** A, const float** E0, int64_t* n_rx, int32_t* M)
{
    if (!amat) return RISRT_ERR_INVALID_ARG;
    if (A) *A = (const float*)amat->A;
    if (E0) *E0 = (const float*)amat->E0;
    if (n_rx) *n_rx = amat->n_rx;
    if (M) *M = amat->M;
    return RISRT_OK;
}

int risrt_amat_destroy(risrt_ctx* ctx, risrt_amat* amat)
{
    if (!amat) return RISRT_OK;
    if (amat->owned) {
        if (ctx) sync_ctx(ctx);
        risrt_ctx* pc = ctx && ctx == amat->owner ? ctx : nullptr;
        ctx_free(pc, (void*)amat->A);
        ctx_free(pc, (void*)amat->E0);
    }
    delete amat;
    return RISRT_OK;
}

int risrt_sweep_workspace_size(int64_t n_rx, int32_t M, int32_t n_cfg, int precision, size_t* bytes)
{
    if (!bytes || n_rx < 1 || M < 1 || n_cfg < 1 || precision < RISRT_PREC_FP32 || precision > RISRT_PREC_FP16)
        return RISRT_ERR_INVALID_ARG;
    *bytes = sweep_workspace_bytes(n_rx, M, n_cfg, precision);
    return RISRT_OK;
}

int risrt_sweep_configs(risrt_ctx* ctx, const risrt_amat* amat, const float* gamma, const uint8_t* gamma_2bit, float amp,
                        int32_t n_cfg, int precision, float* P_out, float* E_out, void* workspace, size_t workspace_bytes)
{
    RISRT_CHECK_CTX(ctx);
    if (!amat || (!gamma == !gamma_2bit) || (!P_out && !E_out))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "need the channel matrix, exactly one of gamma / gamma_2bit, and P_out or E_out");
    if (n_cfg < 1 || n_cfg > (1 << 24)) return fail(ctx, RISRT_ERR_INVALID_ARG, "n_cfg out of range");
    if (gamma_2bit && !std::isfinite(amp)) return fail(ctx, RISRT_ERR_INVALID_ARG, "amp must be finite");
    const int opts = precision & ~0xff;
    precision &= 0xff;
    if (precision < RISRT_PREC_FP32 || precision > RISRT_PREC_FP16 || (opts & ~(RISRT_SWEEP_KEEP_A | RISRT_SWEEP_DEFER_CHECK)))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "unknown precision or option");
    if (opts && precision == RISRT_PREC_FP16)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "RISRT_SWEEP_KEEP_A / DEFER_CHECK need RISRT_PREC_BF16 or BF16X2");
    if (((uintptr_t)gamma | (uintptr_t)E_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    if (precision != RISRT_PREC_FP32 && ((uintptr_t)workspace & 15u))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    GammaSrc G;
    G.G = (const float2*)gamma;
    G.g2 = gamma_2bit;
    G.amp = amp;
    return sweep_configs(ctx, amat->A, amat->E0, amat->n_rx, amat->M, G, n_cfg, precision, P_out, (float2*)E_out,
                         workspace, workspace_bytes, (opts & RISRT_SWEEP_KEEP_A) != 0, (opts & RISRT_SWEEP_DEFER_CHECK) != 0);
}

int risrt_sweep_fused(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, const uint8_t* gamma_2bit, float amp,
                      int32_t n_cfg, float* P_out, float* E_out)
{
    RISRT_CHECK_CTX(ctx);
    if (!ps || (!gamma == !gamma_2bit) || (!P_out && !E_out))
        return fail(ctx, RISRT_ERR_INVALID_ARG, "need the path set, exactly one of gamma / gamma_2bit, and P_out or E_out");
    if (n_cfg < 1 || n_cfg > sweep_fused_max_configs()) return fail(ctx, RISRT_ERR_INVALID_ARG, "n_cfg must be in [1, 128]");
    if (gamma_2bit && !std::isfinite(amp)) return fail(ctx, RISRT_ERR_INVALID_ARG, "amp must be finite");
    if (((uintptr_t)gamma | (uintptr_t)E_out) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "complex arrays must be 8-byte aligned");
    GammaSrc G;
    G.G = (const float2*)gamma;
    G.g2 = gamma_2bit;
    G.amp = amp;
    return sweep_fused(ctx, ps, G, n_cfg, P_out, (float2*)E_out);
}

int risrt_sweep_check(risrt_ctx* ctx, const void* workspace, size_t workspace_bytes)
{
    RISRT_CHECK_CTX(ctx);
    if (!workspace || workspace_bytes < 64) return fail(ctx, RISRT_ERR_INVALID_ARG, "no workspace");
    return sweep_check(ctx, workspace, workspace_bytes);
}

int risrt_grad_workspace_size(int32_t n_target, int32_t B, int32_t M, int precision, size_t* bytes)
{
    if (!bytes || n_target < 1 || B < 1 || M < 1) return RISRT_ERR_INVALID_ARG;
    if (precision != RISRT_PREC_FP32 && precision != RISRT_PREC_BF16X2) return RISRT_ERR_INVALID_ARG;
    *bytes = grad_workspace_bytes(n_target, B, M, precision) + 64;
    return RISRT_OK;
}

int risrt_grad_phases(risrt_ctx* ctx, const risrt_amat* amat, const int32_t* target, int32_t n_target, const float* phases,
                      const float* amp, int32_t B, float* J_out, float* grad_out, void* workspace, size_t workspace_bytes,
                      int precision)
{
    RISRT_CHECK_CTX(ctx);
    if (!amat || !phases || !J_out || !grad_out || !workspace) return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument");
    const float* A = (const float*)amat->A;
    const float* E0 = (const float*)amat->E0;
    const int64_t n_rx = amat->n_rx;
    const int32_t M = amat->M;
    if (n_rx < 1 || M < 1 || M > 65536 || n_target < 1 || B < 1) return fail(ctx, RISRT_ERR_INVALID_ARG, "sizes out of range");
    const bool keep_a = (precision & RISRT_GRAD_KEEP_A) != 0;
    const bool defer = (precision & RISRT_GRAD_DEFER_CHECK) != 0;
    precision &= ~(RISRT_GRAD_KEEP_A | RISRT_GRAD_DEFER_CHECK);
    if (precision != RISRT_PREC_FP32 && precision != RISRT_PREC_BF16X2)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "precision must be RISRT_PREC_FP32 or RISRT_PREC_BF16X2");
    if (!target && n_target > n_rx) return fail(ctx, RISRT_ERR_INVALID_ARG, "n_target > n_rx without a target list");
    if (workspace_bytes < grad_workspace_bytes(n_target, B, M, precision) + 64) return fail(ctx, RISRT_ERR_INVALID_ARG, "workspace too small");
    if (((uintptr_t)workspace) & 255u) return fail(ctx, RISRT_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (((uintptr_t)A | (uintptr_t)E0 | (uintptr_t)workspace) & 7u) return fail(ctx, RISRT_ERR_INVALID_ARG, "misaligned array");
    if (target && !keep_a) {
        int rc = check_targets(ctx, target, n_target, n_rx, workspace, workspace_bytes);
        if (rc) return rc;
    }
    int rc = grad_phases(ctx, (const float2*)A, (const float2*)E0, M, target, n_target, phases, amp, B, J_out, grad_out,
                         workspace, workspace_bytes, precision, keep_a, defer);
    if (rc) return rc;
    if (!defer) RISRT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RISRT_OK;
}

int risrt_grad_check(risrt_ctx* ctx, const void* workspace, size_t workspace_bytes)
{
    RISRT_CHECK_CTX(ctx);
    if (!workspace || workspace_bytes < 64) return fail(ctx, RISRT_ERR_INVALID_ARG, "no workspace");
    return grad_check(ctx, workspace, workspace_bytes);
}

int risrt_find_paths_noalloc(risrt_ctx* ctx, const risrt_scene* scene, const float src[3], int32_t src_face,
                             const float dst[3], int32_t dst_face, int32_t max_order, int64_t* ids_host,
                             int32_t cap, int32_t* n_host)
{
    RISRT_CHECK_CTX(ctx);
    if (!scene || !src || !dst || !n_host || (cap > 0 && !ids_host) || cap < 0)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "NULL argument or negative capacity");
    if (max_order < 0 || max_order > 2) return fail(ctx, RISRT_ERR_INVALID_ARG, "order must be in [0, 2]");
    if (src_face >= scene->n_faces || dst_face >= scene->n_faces)
        return fail(ctx, RISRT_ERR_INVALID_ARG, "face index out of range");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(src[k]) || !std::isfinite(dst[k])) return fail(ctx, RISRT_ERR_INVALID_ARG, "non-finite point");
    *n_host = 0;
    return find_paths_noalloc(ctx, scene, src, src_face, dst, dst_face, max_order, ids_host, cap, n_host);
}

int risrt_scene_destroy(risrt_ctx* ctx, risrt_scene* sc)
{
    if (!sc) return RISRT_OK;
    if (ctx) sync_ctx(ctx);
    risrt_ctx* pc = ctx && ctx == sc->owner ? ctx : nullptr;
    for (void* p : {(void*)sc->nodes, (void*)sc->nodes4, (void*)sc->tri_geom, (void*)sc->tri_verts, (void*)sc->tri_face,
                    (void*)sc->faces, (void*)sc->face_tris, (void*)sc->face_test, (void*)sc->tri_leaf, (void*)sc->mats,
                    (void*)sc->face_grid, (void*)sc->cell_face})
        ctx_free(pc, p);
    delete sc;
    return RISRT_OK;
}

int risrt_ris_destroy(risrt_ctx* ctx, risrt_ris* r)
{
    if (!r) return RISRT_OK;
    if (ctx) sync_ctx(ctx);
    ctx_free(ctx && ctx == r->owner ? ctx : nullptr, r->elem);
    ctx_free(ctx && ctx == r->owner ? ctx : nullptr, r->tile_buf);
    delete r;
    return RISRT_OK;
}

int risrt_rxset_destroy(risrt_ctx* ctx, risrt_rxset* r)
{
    if (!r) return RISRT_OK;
    if (ctx) sync_ctx(ctx);
    if (r->owned) ctx_free(ctx && ctx == r->owner ? ctx : nullptr, r->xyz);
    delete r;
    return RISRT_OK;
}

int risrt_pathset_destroy(risrt_ctx* ctx, risrt_pathset* ps)
{
    if (!ps) return RISRT_OK;
    if (ctx) sync_ctx(ctx);
    if (ps->external) {             // its device arrays belong to the caller's workspace
        delete ps;
        return RISRT_OK;
    }
    risrt_ctx* pc = ctx && ctx == ps->owner ? ctx : nullptr;
    for (void* p : {(void*)ps->rec, (void*)ps->rx_off, (void*)ps->vis, (void*)ps->E0, (void*)ps->cm, (void*)ps->elem,
                    (void*)ps->rx_seq, (void*)ps->env_seq, (void*)ps->env_off, (void*)ps->los, ps->scratch,
                    (void*)ps->ctr_dev})
        ctx_free(pc, p);
    delete ps;
    return RISRT_OK;
}

}  // extern "C"
