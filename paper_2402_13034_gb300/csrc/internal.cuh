// Internal declarations of the risrt CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "risrt.h"

namespace risrt {

constexpr double kPi = 3.14159265358979323846;
constexpr double kC0 = 299792458.0;          // m/s
constexpr double kEta0 = 120.0 * kPi;        // Eq. 1: free-space impedance 120 pi ohm
constexpr double kEps0 = 8.8541878128e-12;   // F/m
constexpr float kSegEps = 1e-4f;             // occluder hits within this of a segment end are ignored
constexpr double kSegEpsD = 1e-4;
constexpr int kNoRoot = (int)0x80000000;   // BVH root of a scene without triangles

// ------------------------------------------------------------------------------------------------
// small vector helpers
// ------------------------------------------------------------------------------------------------
struct d3 { double x, y, z; };
struct __align__(32) dv4 { double x, y, z, w; };
__host__ __device__ __forceinline__ dv4 mk_dv4(double x, double y, double z, double w) { dv4 r = {x, y, z, w}; return r; }

__host__ __device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }

__host__ __device__ __forceinline__ d3 D3(double x, double y, double z) { d3 r = {x, y, z}; return r; }
__host__ __device__ __forceinline__ d3 D3(float3 a) { return D3(a.x, a.y, a.z); }
__host__ __device__ __forceinline__ d3 operator+(d3 a, d3 b) { return D3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ d3 operator-(d3 a, d3 b) { return D3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ d3 operator*(d3 a, double s) { return D3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return D3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double norm(d3 a) { return sqrt(dot(a, a)); }
__host__ __device__ __forceinline__ float3 to_f(d3 a) { return f3((float)a.x, (float)a.y, (float)a.z); }

// Mirror across the plane n.x = d (n unit): the image method's reflection of a point.
__host__ __device__ __forceinline__ d3 mirror_pt(d3 p, d3 n, double d) { return p - n * (2.0 * (dot(n, p) - d)); }
// Linear part of the mirror: reflects a direction.
__host__ __device__ __forceinline__ d3 mirror_dir(d3 v, d3 n) { return v - n * (2.0 * dot(n, v)); }

// ------------------------------------------------------------------------------------------------
// device-side object layouts
// ------------------------------------------------------------------------------------------------

// One triangle in BVH leaf order: FP32 plane and inward edge planes for the filtered test, plus the
// original float vertices (exact in FP64) for the FP64 decision.
struct TriGeom {
    float4 plane;        // unit normal n, offset d (n.x = d)
    float4 edge[3];      // inward in-plane unit normal m_i, offset c_i: distance to edge = m_i.q - c_i
};
struct TriVerts {
    float4 v0;           // xyz, w = face id (int bits)
    float4 v1;
    float4 v2;
};

// BVH node with both child boxes inline; child >= 0 is an internal node, child < 0 is leaf ~child.
struct BvhNode {
    float4 l_lo;         // xyz, w = left child (int bits)
    float4 l_hi;         // xyz, w = right child (int bits)
    float4 r_lo;         // xyz, w = the single face of every leaf under the left child, or -1 (int bits)
    float4 r_hi;         // xyz, w = the same for the right child
};

// Four-wide view of the binary BVH: entry i holds the children of binary node i's children (a leaf
// child stays as it is), so a walk that starts at the root and follows these codes visits every
// other level. Empty slots have code kNoChild and an inverted box.
struct Bvh4Node {
    float4 lo[4];        // xyz child box min, w = child code (binary internal index, ~leaf or kNoChild)
    float4 hi[4];        // xyz child box max, w = the single face under the child, or -1 (int bits)
};
constexpr int kNoChild = 0x7fffffff;

struct Face {
    dv4 plane;       // FP64 unit normal (from the face's first triangle) and offset
    float4 plane32;
    int tri_begin, tri_end;  // range in the face's triangle list (indices into leaf order)
    int mat;
    int pad;
};

// Convex outline of a face for the FP32 in-face filter: n inward edge planes (m, c), distance to
// edge i = m_i.q - c_i; n = 0 when the face is not a single triangle or a convex two-triangle quad.
struct FaceTest {
    float4 e[4];
    int n;
    int pad[3];
};

// Cell grid over a face's plane for the visibility maps from a fixed source point: cell (i, j) covers
// o + a u + b v with a in [a0 + i du, a0 + (i + 1) du], b in [b0 + j dv, b0 + (j + 1) dv]; its map
// entry sits at off + i * nv + j.
struct FaceGrid {
    float4 o;            // xyz origin (a vertex of the face), w = du
    float4 u;            // xyz unit in-plane axis, w = a0
    float4 v;            // xyz unit in-plane axis (normal x u), w = b0
    int nu, nv;
    int off;
    float dv;
};
constexpr float kMapDelta = 1e-3f;   // a cell's map entry holds for points up to this far outside it
constexpr int kTileMinElems = 64;    // RIS with more elements get spatial tiles for the direct legs

struct DeviceScene {
    int64_t n_tris;
    int n_faces;
    // Occlusion walks start at root_main: the subtree of the references that can stop a segment whose
    // two ends lie in the scene box [box_lo, box_hi]. The triangles whose plane has the whole box on one
    // closed side (the shell of a box-shaped room, or faces lying in it) sit in the subtree root_shell,
    // which only segments with an end outside the box visit. Codes index nodes4 (>= 0) or are ~leaf;
    // kNoRoot when a subtree is empty.
    int root_main, root_shell;
    int n_nodes4;                // compact four-wide nodes, top levels first
    float3 box_lo, box_hi;
    const BvhNode* nodes;
    const Bvh4Node* nodes4;      // [n_nodes4] compact four-wide tree used by the traversals
    const TriGeom* tri_geom;     // [n_refs] leaf (reference) order
    const TriVerts* tri_verts;   // [n_refs] leaf order
    const int* tri_face;         // [n_refs] leaf order
    const Face* faces;           // [n_faces]
    const int* face_tris;        // CSR: triangles (leaf order) of each face
    const FaceTest* face_test;   // [n_faces]
    const int* tri_leaf;         // [n_tris] one leaf (reference) of every input triangle
    const float2* mats;          // [n_mat] (eps_r, sigma)
    const FaceGrid* face_grid;   // [n_faces]
    const int* cell_face;        // [n_cells] face of every map cell
    int64_t n_cells;
};

}  // namespace risrt

// ------------------------------------------------------------------------------------------------
// ABI objects
// ------------------------------------------------------------------------------------------------
struct Antenna {
    float pos[3];
    float orient[9];
    float power_w;
    float gain_lin;
    int pattern;
    bool set;
};

struct KernelPending {
    const char* name;
    cudaEvent_t a, b;
    cudaStream_t stream;         // the launch's stream: both events are recorded on it
};

struct risrt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    void* small = nullptr;       // 256 B of device memory for per-call reductions (allocated on first use)
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // concurrent parts of a trace (created on first use)
    cudaEvent_t ev[7] = {};                               // their fork / join events
    // device blocks this context allocated (ctx_malloc) and those returned for reuse (ctx_free)
    std::mutex pool_mu;
    std::multimap<size_t, void*> pool_free;
    std::unordered_map<void*, size_t> pool_size;
    size_t pool_cached = 0;
    size_t budget = 0;           // cap on the device bytes this context holds (0: none)
    size_t allocated = 0;        // bytes of every block this context holds (in use or cached)
    std::string err;
    Antenna tx{}, rx{};
    float pol[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};   // unit polarisation axes (Tx, Rx) of the vector field
    bool pol_set[2] = {false, false};
    // tracing
    bool profiling = false;
    std::string prof_only;       // non-empty: only kernels of this name are bracketed
    bool prof_skip = false;      // the launch being bracketed is not one of them
    std::vector<KernelPending> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<double, int64_t>> ktime;
};

struct risrt_scene {
    risrt_ctx* owner = nullptr;      // context whose block cache holds this object's device memory
    int64_t n_tris = 0;
    int64_t n_refs = 0;              // BVH leaves (triangle references)
    int n_faces = 0;
    int n_mat = 0;
    int root_main = risrt::kNoRoot;
    int root_shell = risrt::kNoRoot;
    int n_nodes4 = 0;
    int64_t n_shell_refs = 0;        // references of shell triangles (planes with the scene box on one side)
    float box_lo[3] = {0.f, 0.f, 0.f}, box_hi[3] = {0.f, 0.f, 0.f};
    risrt::BvhNode* nodes = nullptr;
    risrt::Bvh4Node* nodes4 = nullptr;
    risrt::TriGeom* tri_geom = nullptr;
    risrt::TriVerts* tri_verts = nullptr;
    int* tri_face = nullptr;
    risrt::Face* faces = nullptr;
    int* face_tris = nullptr;
    risrt::FaceTest* face_test = nullptr;
    int* tri_leaf = nullptr;
    float2* mats = nullptr;
    float scene_extent = 0.f;     // max |coordinate| over vertices
    risrt::FaceGrid* face_grid = nullptr;
    int* cell_face = nullptr;
    int64_t n_cells = 0;
    risrt::DeviceScene dev() const {
        risrt::DeviceScene s;
        s.n_tris = n_tris; s.n_faces = n_faces; s.root_main = root_main; s.root_shell = root_shell; s.n_nodes4 = n_nodes4;
        s.nodes = nodes;
        s.box_lo = make_float3(box_lo[0], box_lo[1], box_lo[2]);
        s.box_hi = make_float3(box_hi[0], box_hi[1], box_hi[2]); s.nodes4 = nodes4; s.tri_geom = tri_geom;
        s.tri_verts = tri_verts; s.tri_face = tri_face; s.faces = faces; s.face_tris = face_tris; s.face_test = face_test; s.tri_leaf = tri_leaf; s.mats = mats;
        s.face_grid = face_grid; s.cell_face = cell_face; s.n_cells = n_cells;
        return s;
    }
};

struct risrt_ris {
    risrt_ctx* owner = nullptr;      // context whose block cache holds this object's device memory
    int M = 0;
    float center[3], t1[3], t2[3];
    float dy = 0, dz = 0, elem_gain = 0;
    int host_face = -1;
    float4* elem = nullptr;      // [M] (a_m, b_m, a^2 + b^2, 0)
    std::vector<float> uv_host;  // [M][2]
    // Spatial tiles of up to 32 elements (consecutive in the Morton order of (a, b)) for the direct
    // legs' visibility, built at upload for M > kTileMinElems; one device block holds all four arrays.
    int n_tiles = 0;
    void* tile_buf = nullptr;
    float4* tile_bb = nullptr;   // [n_tiles + ceil(n_tiles / 4)] (a_min, a_max, b_min, b_max) of the tile's
                                 // element centres, then of each super-tile (four consecutive tiles)
    int2* word_tile = nullptr;   // [n_pairs] (tile, bits of a visibility word's elements in that tile)
    int* tile_elem = nullptr;    // [n_tiles * 32] element indices, -1 past the tile's end
    int* word_ofs = nullptr;     // [W + 1] word w's pairs are word_tile[word_ofs[w] .. word_ofs[w + 1])
    // a RIS the library makes for one element (strict mode) is centred exactly at the element
    bool exact_center = false;
    double center_d[3] = {0.0, 0.0, 0.0};
};

struct risrt_rxset {
    risrt_ctx* owner = nullptr;      // context whose block cache holds this object's device memory
    int64_t n = 0;
    float* xyz = nullptr;        // [n][3] device
    bool owned = false;
    mutable float ext = -1.f;    // max |coordinate|, cached for uploaded (library-owned) sets; -1: unknown
};

// Rx-leg path record (structure of arrays, one entry per (rx, path)); see field.cu for use.
// With kRecLosslessTE set in the order field every bounce is a lossless dielectric under the TE
// coefficient and the eps fields hold (eps_r - 1, 1 / (1 - eps_r)) per bounce: a.z, a.w for bounce 1,
// n1.w, n2.w for bounce 2.
constexpr int kRecLosslessTE = 4;
struct PathRec {
    float4 w;        // w = I - c in the RIS frame (t1, t2, n), and D0 = |w|
    float4 a;        // frac(D0/lambda), order (int bits, low 2; kRecLosslessTE), eps1 (re, im)
    float4 n1;       // bounce-1 normal in the RIS frame, eps2.re
    float4 n2;       // bounce-2 normal (unfolded) in the RIS frame, eps2.im
    float4 v;        // Rx pattern axis, unfolded into the RIS frame
};

namespace risrt {
struct Frame {             // RIS frame, FP64
    double c[3], t1[3], t2[3], n[3];
};
struct AntD {
    double pos[3];
    double z[3];           // unit boresight (local z axis)
    double power, gain;
    int pattern;
};
struct WaveD {
    double lam, k, omega;
    double inv_lam;        // 1 / lambda
    float inv_we;          // 1 / (omega eps0): eps_c = eps_r - j sigma / (omega eps0)
    int tm;
};
// One valid reflected Tx-leg path kept with its path set: the Tx image across its faces (FP64) and,
// per face in propagation order, the FP32 unit normal and complex permittivity.
struct TxPathD {
    dv4 img;
    float4 n[2];
    float2 eps[2];
    int k;                 // order
    int id;                // sequence id
};
}  // namespace risrt

// A dense channel matrix A [n_rx][M] and E0 [n_rx] (complex64) on the device: either owned (built by
// the library into blocks of its context) or a view of caller memory.
struct risrt_amat {
    risrt_ctx* owner = nullptr;
    const float2* A = nullptr;
    const float2* E0 = nullptr;      // may be NULL (E0 = 0)
    int64_t n_rx = 0;
    int M = 0;
    bool owned = false;
};

struct risrt_pathset {
    risrt_ctx* owner = nullptr;      // context whose block cache holds this object's device memory
    int64_t n_rx = 0;
    int M = 0;
    int n_faces = 0;
    double freq = 0;
    uint32_t flags = 0;
    int rx_pattern = 0;
    float rx_gain = 1.f;
    // resident results
    PathRec* rec = nullptr;          // [n_paths]
    int64_t* rx_off = nullptr;       // [n_rx + 1] entry offsets per Rx (direct entry first)
    uint32_t* vis = nullptr;         // [n_rx][W] direct e_m -> Rx visibility
    int W = 0;
    float2* E0 = nullptr;            // [n_rx] LOS + environment field
    float2* cm = nullptr;            // [M] K * c_m (Tx leg, Eq. 4/5/7 factors)
    int64_t cap_m = 0;               // elements cm and elem hold
    float4* elem = nullptr;          // [M] copy of the RIS element table (a, b, |u|^2, 0)
    int64_t n_paths = 0, cap_paths = 0;
    // inspection data
    int64_t* rx_seq = nullptr;       // [n_paths] sequence id per entry (-1 for direct)
    int64_t* env_seq = nullptr;      // [n_env]
    int64_t* env_off = nullptr;      // [n_rx + 1]
    int64_t n_env = 0, cap_env = 0;
    uint8_t* los = nullptr;          // [n_rx]
    std::vector<int64_t> tx_seq_host;
    std::vector<uint8_t> tx_vis_host;
    // the Tx leg and the parameters of the trace, for per-path outputs (risrt_eval_cir)
    risrt::TxPathD* tx_paths = nullptr;   // [n_tx] valid reflected Tx-leg paths by ascending id
    int64_t cap_tx_paths = 0;
    uint8_t* tx_vis_dev = nullptr;        // [M] Tx -> e_m unblocked
    int64_t cap_tx_vis = 0;
    risrt::Frame fr{};
    risrt::AntD txa{};
    risrt::AntD rxa{};                    // the Rx antenna of the trace (gain, pattern, boresight)
    risrt::WaveD wv{};
    double K = 0.0;
    // asynchronous traces: every device array lives in the caller's workspace (external), and the
    // counts, flags and Tx-leg ids stay on the device until risrt_trace_check reads them
    bool external = false;
    bool check_pending = false;
    const int* chk_flags = nullptr;          // [0] candidate slab full, [1] traversal stack, [2] path arrays full
    const int64_t* chk_ntx = nullptr;
    const int64_t* chk_ids = nullptr;
    int chk_cap = 0;
    // generation of the asynchronous trace: advanced on the device by every run (a graph replay
    // included), recorded on the host by risrt_trace_check; the host copies are current when they agree
    const unsigned long long* gen_dev = nullptr;
    unsigned long long checked_gen = 0;
    // statistics: counted on the device, fetched when first asked for (the trace does not wait)
    mutable int64_t units = 0;
    mutable int64_t fp64_refines = 0;
    mutable int64_t n_candidates = 0, n_segments = 0, node_visits = 0, tri_tests = 0;
    unsigned long long* ctr_dev = nullptr;   // [6] copy of the trace's counters ([6] the generation, asynchronous)
    mutable bool stats_pending = false;
    cudaStream_t stream = nullptr;           // stream of the trace that filled this set
    int64_t cap_rx_seq = 0;
    int64_t cap_rx = 0;              // capacity of the per-Rx arrays
    // scratch (grown as needed, kept for reuse)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int cand_cap = 0;                // per-Rx geometric candidate capacity
};

// ------------------------------------------------------------------------------------------------
// cross-file entry points (implemented in scene.cu / trace.cu / field.cu)
// ------------------------------------------------------------------------------------------------
namespace risrt {
int fail(risrt_ctx* ctx, int code, const std::string& msg);
// Device memory of a context: ctx_malloc reuses a block that ctx_free returned (the smallest that
// holds the request and is at most twice its size plus 1 MiB) or calls cudaMalloc; ctx_free keeps the
// block for reuse up to kPoolLimit cached bytes per context, else frees it. A returned block may be
// handed out again at once: callers return blocks only when later uses on the context's stream are
// ordered after every earlier use (the destroy calls synchronise first). ctx == nullptr: plain
// cudaMalloc / cudaFree.
constexpr size_t kPoolLimit = (size_t)2 << 30;
cudaError_t ctx_malloc(risrt_ctx* ctx, void** p, size_t bytes);
void ctx_free(risrt_ctx* ctx, void* p);
int cuda_fail(risrt_ctx* ctx, cudaError_t e, const char* where);
#define RISRT_CUDA(ctx, call)                                           \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::risrt::cuda_fail(ctx, _e, #call); \
    } while (0)
#define RISRT_LAUNCH(ctx, what)                                          \
    do {                                                                 \
        cudaError_t _e = cudaGetLastError();                             \
        if (_e != cudaSuccess) return ::risrt::cuda_fail(ctx, _e, what); \
    } while (0)

extern std::atomic<long long> g_launches;
void prof_begin(risrt_ctx* ctx, const char* name, cudaStream_t st);   // events on the launch's stream st
void prof_end(risrt_ctx* ctx);
// Launch a kernel (the `launch` expression) with optional event timing and error check.
#define RISRT_KERNEL_ON(ctx, st, name, launch)                           \
    do {                                                                 \
        ::risrt::prof_begin(ctx, name, st);                              \
        launch;                                                          \
        ::risrt::g_launches.fetch_add(1, std::memory_order_relaxed);     \
        ::risrt::prof_end(ctx);                                          \
        RISRT_LAUNCH(ctx, name);                                         \
    } while (0)
#define RISRT_KERNEL(ctx, name, launch) RISRT_KERNEL_ON(ctx, ((ctx) ? (ctx)->stream : cudaStream_t(0)), name, launch)

int build_scene(risrt_ctx* ctx, risrt_scene* sc, const float* verts_host, int64_t n_verts,
                const int32_t* tris_host, const int32_t* face_host, const int32_t* mat_host,
                const float* mats_host, int n_mat);
// An asynchronous trace (risrt_trace_paths_async): all device memory from the workspace `ws` of `bytes`
// (nullptr: only store the bytes needed in *need), fixed capacities, no host synchronisation.
struct AsyncTrace {
    void* ws = nullptr;
    size_t bytes = 0;
    int cand_cap = 512;          // geometric candidates per destination and leg
    int max_paths = 64;          // Rx-leg entries per receiver (the direct one included)
    int max_env = 64;            // environment paths per receiver
    size_t* need = nullptr;
};
int trace_paths(risrt_ctx* ctx, const risrt_scene* sc, const risrt_ris* ris, const risrt_rxset* rx,
                double freq, int max_order_tx, int max_order_rx, uint32_t flags, risrt_pathset* ps,
                const AsyncTrace* at = nullptr);
// Reads the device-side results of an asynchronous trace (synchronises); RISRT_ERR_CAPACITY if one of
// its fixed capacities was exceeded.
int trace_check(risrt_ctx* ctx, risrt_pathset* ps);
// max |coordinate| of n points on the device (synchronises)
int rx_extent(risrt_ctx* ctx, const float* xyz, int64_t n, float* out);
int eval_field(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, int n_cfg, float2* E, float* P);
int build_A(risrt_ctx* ctx, const risrt_pathset* ps, float2* A, float2* E0);
int eval_field_plain(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, int n_cfg, float2* E, float* P);
int eval_cir(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, float2* taps, double* rx_delay, double* tx_delay);
int cir_tx_coef(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, float2* g, double* tx_delay);
int strict_tx_cm(risrt_ctx* ctx, const risrt_scene* sc, const risrt_ris* ris, double freq, int max_tx, uint32_t flags,
                 float2* cm);
int eval_field_accum(risrt_ctx* ctx, const risrt_pathset* ps, const float2* gamma, int gstride, int n_cfg, float2* E);
int eval_field_strict(risrt_ctx* ctx, const risrt_scene* sc, const risrt_ris* ris, const risrt_rxset* rxs, double freq,
                      int max_tx, int max_rx, uint32_t flags, const float2* gamma, int n_cfg, float2* E, float* P);
int microbench(risrt_ctx* ctx, int kind, int iters, double* ops_per_s, double* ms);
int eval_field_vec(risrt_ctx* ctx, const risrt_scene* sc, const risrt_rxset* rxs, const risrt_pathset* ps,
                   const float2* gamma, int n_cfg, float2* E, float2* E3, float* P);
int build_A_vec(risrt_ctx* ctx, const risrt_scene* sc, const risrt_rxset* rxs, const risrt_pathset* ps, float2* A,
                float2* E0);
size_t grad_workspace_bytes(int n_t, int B, int M, int precision);
int check_targets(risrt_ctx* ctx, const int* target, int n_t, int64_t n_rx, void* ws, size_t ws_bytes);
int grad_phases(risrt_ctx* ctx, const float2* A, const float2* E0, int M, const int* target, int n_t,
                const float* phases, const float* amp, int B, float* J, float* grad, void* ws, size_t ws_bytes,
                int precision, bool keep_a, bool defer = false);
// The deferred tensor-core timeout flag of the last grad_phases on this workspace (waits for the stream).
int grad_check(risrt_ctx* ctx, const void* ws, size_t ws_bytes);
int find_paths_noalloc(risrt_ctx* ctx, const risrt_scene* sc, const float src[3], int src_face, const float dst[3],
                       int dst_face, int max_order, int64_t* ids_host, int cap_host, int* n_host);

// device-wide exclusive scan (int64 in/out), n <= 2^31; temp from scan_temp_bytes
size_t scan_temp_bytes(int64_t n);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp, cudaStream_t s);
// stable LSD radix sort of (key, value) pairs on the low `bits` bits of key
size_t sort_temp_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, void* temp, cudaStream_t s);
}  // namespace risrt
