/*
 * risrt — GB300-native RIS ray-tracing field engine (C ABI).
 *
 * Implements the data-parallel hot path of "Ray Tracing Algorithm for Reconfigurable Intelligent
 * Surfaces" (Sandh et al., arXiv 2402.13034): for every receiver (Rx) point, the complex field summed
 * over every RIS element and every propagation path, with the paper's RIS path-loss model
 * (Sec. II-A, Eqs. 4-10) and specular wall reflections on the Tx->RIS and RIS->Rx legs found by
 * BVH ray-triangle traversal and the image method (Sec. II-B, Fig. 2).
 *
 * Conventions (all entry points):
 *  - Every function returns an int status (RISRT_OK = 0 or a RISRT_ERR_* code). No exception,
 *    longjmp or abort crosses the boundary. risrt_last_error(ctx) returns a message for the last
 *    failure on that context (valid until the next call on the context).
 *  - SI units: metres, Hz, W, V/m. Gains are linear. Angles in radians.
 *  - Pointer arguments whose name ends in _host are host memory; every other array pointer is
 *    CUDA device memory owned by the caller. Arrays are dense, row-major, with the stated layout.
 *    complex values are interleaved float pairs (re, im) ("float2"), 8-byte aligned.
 *  - Work is enqueued asynchronously on the context's stream unless a function says it
 *    synchronises. Outputs in caller memory are valid once that stream reaches the call's work.
 *  - Library-owned objects (scene, RIS, Rx set, path set) are opaque handles holding device memory;
 *    free them with the matching *_destroy. A handle may be used only with the context that
 *    created it. The context itself must outlive its handles.
 *  - Functions are not thread-safe on one context; distinct contexts are independent.
 */
#ifndef RISRT_H
#define RISRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct risrt_ctx risrt_ctx;
typedef struct risrt_scene risrt_scene;
typedef struct risrt_ris risrt_ris;
typedef struct risrt_rxset risrt_rxset;
typedef struct risrt_pathset risrt_pathset;
typedef struct risrt_amat risrt_amat;

enum {
    RISRT_OK = 0,
    RISRT_ERR_INVALID_ARG = 1, /* a size, pointer, index or value outside its documented range */
    RISRT_ERR_OOM = 2,         /* device allocation failed */
    RISRT_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    RISRT_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    RISRT_ERR_NOT_READY = 5,   /* an input object is missing (antenna not set) or an asynchronous trace is unchecked */
    RISRT_ERR_CAPACITY = 6     /* a fixed internal capacity would be exceeded */
};

enum { RISRT_TX = 0, RISRT_RX = 1 };

/* Antenna / radiation patterns F(theta), theta measured from the antenna's local z axis (Sec. II-A). */
enum {
    RISRT_PATTERN_ISO = 0,        /* F = 1 */
    RISRT_PATTERN_COS_POW = 1,    /* F = max(cos theta, 0)^(G/2 - 1), G linear (Sec. III-B, horn) */
    RISRT_PATTERN_MONOPOLE_QW = 2 /* F = ((cos(pi/2 cos theta) - cos(pi/2)) / sin theta)^2, h = lambda/4
                                     (Sec. III-B); 0 on the axis */
};

/* trace flags */
enum {
    RISRT_FLAG_ENV_PATHS = 1,  /* add Tx->Rx specular paths without the RIS (order <= max_order_rx) to E0 */
    RISRT_FLAG_FRESNEL_TM = 2  /* TM (parallel) Fresnel coefficient instead of TE (perpendicular) */
};

/* ------------------------------------------------------------------------------------------------
 * Context
 * ---------------------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`, enqueueing work on `stream` (a cudaStream_t; NULL means
 * the legacy default stream). Fails with RISRT_ERR_CUDA if the device cannot be used.
 * Scenes, RIS, receiver sets, path sets and resident channel matrices take their device memory from
 * a block cache of the context that creates them; destroying them with that context returns the
 * blocks to it (up to 2 GiB stay cached for reuse; an allocation that fails releases the cache and
 * retries). Destroy objects before their context: an object destroyed with another context or NULL
 * frees its memory with cudaFree.
 * hbm_budget_bytes: upper bound on the device bytes the context holds at once (objects in use plus
 * cached blocks; 0 = no bound). A request that would exceed it first releases the cache, then fails
 * with RISRT_ERR_OOM, so a host can give each context a share of the GPU (serving admission). */
int risrt_create(risrt_ctx** out, int device, void* stream, size_t hbm_budget_bytes);

/* Change the stream later calls enqueue on (synchronises the previous stream first, since cached
 * blocks may still be in use by its work). */
int risrt_set_stream(risrt_ctx* ctx, void* stream);

/* Synchronise the context's stream and release every device resource of the context, including
 * its cached blocks. */
int risrt_destroy(risrt_ctx* ctx);

/* Message describing the last failure on ctx (or on creation when ctx is NULL). Never NULL. */
const char* risrt_last_error(const risrt_ctx* ctx);

/* ------------------------------------------------------------------------------------------------
 * Inputs
 * ---------------------------------------------------------------------------------------------- */

/* Upload a triangle scene and build its bounding-volume hierarchy on the device (LBVH: Morton
 * codes, radix sort, binary radix tree, bottom-up box refit).
 *   verts_host   [n_verts][3] float   vertex positions
 *   tris_host    [n_tris][3]  int32   vertex indices, each in [0, n_verts)
 *   face_id_host [n_tris]     int32   planar face of each triangle, ids 0..F-1 all used; triangles of
 *                                     one face must be coplanar. The image method reflects on faces.
 *   mat_id_host  [n_tris]     int32   material index in [0, n_mat); one material per face
 *   mats_host    [n_mat][2]   float   (eps_r, sigma [S/m]) per material (Table 1 for metal)
 * n_tris may be 0 (free space). Synchronises the stream (the face count is validated on the host).
 * Errors: RISRT_ERR_INVALID_ARG on out-of-range indices or n_mat < 1; RISRT_ERR_OOM. */
int risrt_scene_upload(risrt_ctx* ctx, const float* verts_host, int64_t n_verts,
                       const int32_t* tris_host, const int32_t* face_id_host,
                       const int32_t* mat_id_host, int64_t n_tris,
                       const float* mats_host, int32_t n_mat, risrt_scene** out);

/* Upload a RIS (Sec. II, Fig. 1): M elements at e_m = center + a_m t1 + b_m t2 with normal
 * n = t1 x t2 (t1, t2 orthonormal within 1e-5), effective element size dy x dz (A_m = dy dz, Eq. 5),
 * element gain G (<= 0 selects G = 4 pi dy dz / lambda^2, the reading under which Eqs. 4-10 reduce to
 * Tang22), element pattern F(theta) = max(cos theta, 0) about n (Sec. III-C).
 *   elem_uv_host [M][2] float (a_m, b_m).  1 <= M <= 65536.
 *   host_face: face of the scene the RIS is mounted on (ignored for occlusion of rays leaving or
 *   reaching an element), or -1.
 * For M > 64 the call also stores spatial tiles of 32 elements (consecutive in the Morton order of
 * (a_m, b_m)) with which a trace decides element -> receiver visibility tile by tile; a trace over
 * such a RIS takes about 5 n_rx M / 32 bytes more scratch (included in risrt_trace_workspace_size).
 * The environment variable RISRT_TILES=0, read by each trace, makes it trace every element instead
 * (the same visibility bits). */
int risrt_ris_upload(risrt_ctx* ctx, const float* elem_uv_host, int32_t M, const float center[3],
                     const float t1[3], const float t2[3], float dy, float dz, float elem_gain,
                     int32_t host_face, risrt_ris** out);

/* Set the Tx or Rx antenna (Eq. 4, Eq. 8). orient3x3: rows are the antenna's local x, y, z axes in
 * global coordinates (theta from the local z axis). pos, power_w: Tx only (pos ignored for the Rx,
 * whose positions come from the Rx set). gain_lin > 0. */
int risrt_antenna_set(risrt_ctx* ctx, int which, const float pos[3], const float orient3x3[9],
                      float power_w, float gain_lin, int pattern);

/* Copy n_rx receiver positions [n_rx][3] float from host memory into a library-owned Rx set.
 * 1 <= n_rx <= 2^26. */
int risrt_rx_upload(risrt_ctx* ctx, const float* rx_xyz_host, int64_t n_rx, risrt_rxset** out);

/* Wrap caller-owned device memory [n_rx][3] float as an Rx set without copying. The caller keeps
 * the memory alive until risrt_rxset_destroy; its contents may change between traces only within the
 * largest |coordinate| measured here (the traces' FP32 error bounds use it). Synchronises the stream. */
int risrt_rx_bind(risrt_ctx* ctx, const float* rx_xyz, int64_t n_rx, risrt_rxset** out);

/* ------------------------------------------------------------------------------------------------
 * Path finding (Sec. II-B)
 * ---------------------------------------------------------------------------------------------- */

/* Find every propagation path for every receiver and keep it resident in a path set:
 *  - Tx leg: direct Tx->e_m per element with an occlusion ray each (Sec. IV-A), plus reflected face
 *    sequences of length 1..max_order_tx validated once between the Tx and the RIS centre;
 *  - Rx leg: direct e_m->Rx per (Rx, element) with an occlusion ray each, plus reflected face
 *    sequences of length 1..max_order_rx validated once between the RIS centre and each Rx
 *    (the per-element image method then uses each element's own unfolded geometry);
 *  - LOS Tx->Rx, and with RISRT_FLAG_ENV_PATHS the Tx->Rx specular paths, summed into E0 (FP64
 *    phase);
 *  - per-element Tx-leg coefficients c_m (Eq. 4, Eq. 5, Fresnel per bounce; FP64 phase).
 * A sequence is a list of faces; consecutive faces may not repeat or be coplanar, and a face whose
 * plane contains the RIS centre may not be the first Rx-leg or last Tx-leg bounce. A path is valid if
 * every reflection point lies inside its face (union of the face's triangles, inclusive), its two
 * neighbours lie strictly on the same side of each reflecting plane, and no triangle (faces at the
 * segment's ends excluded) is hit between 1e-4 m after a segment's start and 1e-4 m before its end.
 * Geometric decisions are filtered in FP32 and settled in FP64 when the FP32 margin is too small.
 * 0 <= max_order_tx, max_order_rx <= 2; order 2 needs F <= 40000 faces. freq_hz > 0.
 * *inout: NULL to create a new path set, or an existing path set of this context whose buffers are
 * reused (grown when needed). Synchronises the stream (path counts size the output). The Tx leg, the
 * environment paths and the visibility work run on three non-blocking streams the context creates
 * on its first trace, ordered after the work already on the context's stream and joined back into
 * it before the call returns (RISRT_OVERLAP=0 in the environment keeps everything on the context's
 * stream; so does per-kernel profiling without a name filter).
 * Errors: RISRT_ERR_NOT_READY if the Tx or Rx antenna is unset; RISRT_ERR_INVALID_ARG. */
int risrt_trace_paths(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris,
                      const risrt_rxset* rxset, double freq_hz, int32_t max_order_tx,
                      int32_t max_order_rx, uint32_t flags, risrt_pathset** inout);

/* Fixed capacities of an asynchronous trace. */
typedef struct {
    int32_t cand_cap;              /* geometric path candidates per destination and leg (1 .. 65536) */
    int32_t max_paths_per_rx;      /* Rx-leg entries per receiver, the direct one included (>= 1) */
    int32_t max_env_paths_per_rx;  /* environment (Tx -> Rx reflected) paths per receiver (>= 0) */
} risrt_trace_limits;

/* Bytes of device workspace risrt_trace_paths_async needs for these inputs, orders, flags and limits
 * (host arithmetic over the sizes; launches nothing). Errors as risrt_trace_paths. */
int risrt_trace_workspace_size(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris,
                               const risrt_rxset* rxset, int32_t max_order_tx, int32_t max_order_rx,
                               uint32_t flags, const risrt_trace_limits* limits, size_t* bytes);

/* The path search of risrt_trace_paths (same paths, bit for bit, when the limits hold them) that neither
 * synchronises nor allocates device memory: every array of the path set and all scratch live in
 * `workspace` (256-byte aligned, at least risrt_trace_workspace_size bytes, owned by the caller, not to
 * be reused until the path set is no longer needed), sequence-table sizes and path counts stay on the
 * device, and the work is only enqueued, so the call can be captured into a CUDA graph and replayed
 * (with new contents of the inputs: receiver coordinates must stay within the extent measured when the
 * receiver set was uploaded or bound). The first trace of a context, of either kind, creates its
 * side streams and sets kernel attributes: make it before any capture, and capture only after the
 * context's earlier work has completed (a capturing stream cannot wait on work outside the capture). Candidates, entries or
 * environment paths beyond the limits are dropped and flagged; risrt_trace_check reports them
 * (RISRT_ERR_CAPACITY) and must run, after the work completes and before the workspace is reused,
 * before risrt_pathset_stats_get, risrt_pathset_export or risrt_eval_cir; risrt_eval_field,
 * risrt_build_A and the sweeps can be enqueued right after this call. Grids span every sequence id, so
 * order 2 suits scenes of a few thousand faces. *inout: NULL, or a path set filled by this call before
 * (one created by risrt_trace_paths is refused). */
int risrt_trace_paths_async(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                            double freq_hz, int32_t max_order_tx, int32_t max_order_rx, uint32_t flags,
                            const risrt_trace_limits* limits, void* workspace, size_t workspace_bytes,
                            risrt_pathset** inout);

/* Waits for an asynchronous trace and reads its counts, flags and Tx-leg ids; RISRT_ERR_CAPACITY names
 * the limit that was exceeded (the path set is then incomplete), RISRT_OK otherwise. Call it after every
 * run of the trace, each replay of a CUDA graph that holds one included: every run advances a counter
 * on the device, and risrt_pathset_stats_get, risrt_pathset_export and risrt_eval_cir return
 * RISRT_ERR_NOT_READY while that counter is ahead of the one read here (the device-side consumers,
 * risrt_eval_field, risrt_build_A and the sweeps, need no check). A no-op for other path sets. */
int risrt_trace_check(risrt_ctx* ctx, risrt_pathset* ps);

/* Counts of a path set (host struct). */
typedef struct {
    int64_t n_rx;          /* receivers */
    int32_t M;             /* RIS elements */
    int32_t n_faces;       /* scene faces */
    int64_t n_rx_paths;    /* Rx-leg path entries, including one direct entry per receiver */
    int64_t n_env_paths;   /* Tx->Rx reflected paths (RISRT_FLAG_ENV_PATHS) */
    int32_t n_tx_paths;    /* valid reflected Tx-leg sequences */
    int64_t units;         /* field evaluation units: sum over receivers of M x (Rx-leg entries) */
    int64_t fp64_refines;  /* geometric decisions settled in FP64 in the last trace */
    int64_t n_candidates;  /* geometric path candidates whose segments were traced */
    int64_t n_segments;    /* candidate segments traced through the BVH (early exit on a block) */
    int64_t node_visits;   /* BVH nodes visited by those segments */
    int64_t tri_tests;     /* triangle tests of those segments */
} risrt_pathset_stats;

int risrt_pathset_stats_get(const risrt_pathset* ps, risrt_pathset_stats* out);

/* Export the path set to host memory for inspection and bit-exact comparison. Sequence ids:
 * id = f for the single face f; id = F + f1*F + f2 for (f1, f2) in propagation order (for the Rx
 * leg f1 is the first bounce after the RIS). Any pointer may be NULL to skip it. Synchronises.
 *   rx_count_host   [n_rx]            int32  reflected Rx-leg sequences per receiver
 *   rx_seq_host     [n_rx_paths - n_rx] int64 their ids, receiver-major, ascending per receiver
 *   env_count_host  [n_rx]            int32
 *   env_seq_host    [n_env_paths]     int64  Tx->Rx reflected ids, receiver-major, ascending
 *   los_host        [n_rx]            uint8  1 if the Tx->Rx segment is unblocked
 *   vis_host        [n_rx][ceil(M/32)] uint32 bit m%32 of word m/32: e_m->Rx unblocked
 *   tx_seq_host     [n_tx_paths]      int64  valid reflected Tx-leg ids, ascending
 *   tx_vis_host     [M]               uint8  1 if Tx->e_m is unblocked */
int risrt_pathset_export(const risrt_pathset* ps, int32_t* rx_count_host, int64_t* rx_seq_host,
                         int32_t* env_count_host, int64_t* env_seq_host, uint8_t* los_host,
                         uint32_t* vis_host, int64_t* tx_seq_host, uint8_t* tx_vis_host);

/* ------------------------------------------------------------------------------------------------
 * Field (Eqs. 7-10)
 * ---------------------------------------------------------------------------------------------- */

/* For n_cfg reflection-coefficient configurations gamma [n_cfg][M] (complex64), the received field
 * E [n_cfg][n_rx] (complex64) = E0 + sum_m Gamma_m c_m sum_q b_mq (Eq. 9 over every element and
 * Rx-leg path) and, if P_out is not NULL, P [n_cfg][n_rx] float = |E|^2 / (2 eta0) (Eq. 10).
 * The phase of each term is 2 pi frac(frac(D0/lambda) + dL/lambda) with D0 in FP64 per (Rx, path)
 * and the element offset dL = (|u|^2 - 2 u.w)/(L + D0) in FP32. 1 <= n_cfg. */
int risrt_eval_field(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, int32_t n_cfg,
                     float* E_out, float* P_out);

/* Plain FP32 baseline of risrt_eval_field (same arguments, same outputs): one thread per receiver
 * walks every (element, Rx-leg path) term with the phase computed in FP32 from the absolute unfolded
 * length (sincosf of 2 pi L / lambda, with its full range reduction), IEEE square roots and
 * divisions. It exists to measure what the FP64 per-path phase reference, the element-major warp
 * layout and the single-instruction approximations of risrt_eval_field buy, in time and accuracy. */
int risrt_eval_field_plain(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, int32_t n_cfg,
                           float* E_out, float* P_out);

/* Field with strict per-element validation of reflected paths. The paper validates each face sequence
 * once between the RIS centre and the Rx (and between the Tx and the RIS centre) and lets every element
 * use the accepted sequences (Sec. II-B); here every element's reflected legs are validated between
 * the element itself and each end, with the same conditions (reflection points in their faces,
 * neighbours strictly on the same side of each plane, every segment unblocked; the bounce next to the
 * element may not lie on a plane through it), and each element's field uses only its own valid legs:
 *   E = E0 + sum_m Gamma_m K c_m^strict sum_{q valid for m} b_mq,  P = |E|^2 / (2 eta0)   (Eqs. 9, 10)
 * Arguments as risrt_trace_paths followed by those of risrt_eval_field (gamma [n_cfg][M] complex64,
 * E_out [n_cfg][n_rx] complex64, P_out [n_cfg][n_rx] float or NULL). Costs about M traces (a one-element
 * trace per element plus one for E0) and synchronises the stream; it keeps no path set.
 * Errors as risrt_trace_paths. */
int risrt_eval_field_strict(risrt_ctx* ctx, const risrt_scene* scene, const risrt_ris* ris, const risrt_rxset* rxset,
                            double freq_hz, int32_t max_order_tx, int32_t max_order_rx, uint32_t flags,
                            const float* gamma, int32_t n_cfg, float* E_out, float* P_out);

/* Channel impulse response of the RIS part of the field (Sec. II-B: every multipath component that
 * goes through the RIS) for one configuration gamma [M] complex64. Let P = n_tx_paths + 1 (Tx-leg
 * paths: p = 0 the direct leg, p >= 1 the valid reflected Tx-leg sequences in ascending id, as in
 * risrt_pathset_export) and let the Rx-leg entries be those of the path set, receiver-major, each
 * receiver's direct entry first, then its reflected sequences in ascending id (n_rx_paths in all).
 *   taps_out     [n_rx_paths][P] complex64: tap (entry q, p) = sum_m Gamma_m K c_mp b_mq, the field of
 *                the multipath components that take Tx-leg path p and Rx-leg path q (a direct leg
 *                counts the elements it reaches unblocked); the taps of a receiver plus E0 add up to
 *                the field of risrt_eval_field
 *   rx_delay_out [n_rx_paths] double: |I_q - c| / c0, the Rx-leg travel time from the RIS centre c
 *                (seconds; the receiver image I_q from FP64, stored in FP32, about 1e-7 relative)
 *   tx_delay_out [P] double: |T_p - c| / c0 with T_p the Tx image of path p (FP64)
 * A tap's delay is tx_delay[p] + rx_delay[q]: the travel time through the RIS centre; the offsets of
 * the individual elements (at most the aperture over c0) stay in the tap's phase. LOS and environment
 * paths are not taps here (they are summed in E0). Enqueued on the context's stream. */
int risrt_eval_cir(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, float* taps_out, double* rx_delay_out,
                   double* tx_delay_out);

/* Polarisation axis (unit vector, global frame; normalised here) of the Tx or Rx antenna for the vector
 * field. A dipole or monopole's axis is its own; a horn's is the direction of its aperture field. The
 * axes in force when a vector-field call is made are used. Errors: RISRT_ERR_INVALID_ARG for a zero
 * or non-finite axis. */
int risrt_antenna_set_polarization(risrt_ctx* ctx, int which, const float axis[3]);

/* Vector field with polarisation (the extension of Eq. 6 named in Sec. II-A) over the paths of ps,
 * which must have been traced with `scene` and `rxset`. Every path keeps the scalar model's factors
 * (Eqs. 4-8) but the Fresnel products and carries a field vector: launched along the Tx axis projected
 * on the wavefront (unit length), split at every bounce into TE (along unit(k_in x n), R_TE) and TM
 * (R_TM, from s x k_in to s x k_out) parts with complex permittivities (RISRT_FLAG_FRESNEL_TM has no
 * effect here), re-radiated by the RIS as Gamma_m times the incident field with its normal component
 * reversed and restricted to the outgoing wavefront, and received on the Rx axis projected on the
 * arrival wavefront (unit length). Directions of every segment are those of each element's own path.
 *   gamma  [n_cfg][M] complex64 (device)
 *   E_out  [n_cfg][n_rx] complex64: received values (LOS and environment paths included); with every
 *          field TE and co-polarised they equal risrt_eval_field's (TE) values
 *   E3_out [n_cfg][n_rx][3] complex64 or NULL: the field vectors (global frame, Eq. 8 amplitudes)
 *   P_out  [n_cfg][n_rx] float or NULL: |E|^2 / (2 eta0) of the received value (Eq. 10)
 * Enqueued on the context's stream. Errors: RISRT_ERR_NOT_READY if an axis is unset or an asynchronous
 * path set is unchecked; RISRT_ERR_INVALID_ARG for another scene or receiver set (by size). */
int risrt_eval_field_vec(risrt_ctx* ctx, const risrt_scene* scene, const risrt_rxset* rxset, const risrt_pathset* ps,
                         const float* gamma, int32_t n_cfg, float* E_out, float* E3_out, float* P_out);

/* Channel matrix of the vector field's received values: A_out [n_rx][M] complex64 with the received
 * E = E0 + A . Gamma, E0_out [n_rx] complex64 or NULL (LOS and environment paths). A_out can feed the
 * sweeps through risrt_amat_wrap. Arguments and errors as risrt_eval_field_vec. */
int risrt_build_A_vec(risrt_ctx* ctx, const risrt_scene* scene, const risrt_rxset* rxset, const risrt_pathset* ps,
                      float* A_out, float* E0_out);

/* Dense channel matrix (Eq. 9 is linear in Gamma): A [n_rx][M] complex64 with A[r][m] = c_m sum_q b_mq(r),
 * so that E = E0 + A . Gamma, and E0 [n_rx] complex64.
 *  - A_out != NULL: written into caller memory (E0_out may be NULL). If resident_out != NULL,
 *    *resident_out receives a handle viewing A_out and E0_out (the caller keeps them alive).
 *  - A_out == NULL: resident_out must not be NULL; the library allocates A and E0 in blocks of this
 *    context (16 n_rx (M + 1) bytes, counted against its budget), builds them there and returns a
 *    handle that owns them (E0_out is ignored).
 * The handle feeds risrt_sweep_configs and risrt_grad_phases; free it with risrt_amat_destroy. */
int risrt_build_A(risrt_ctx* ctx, const risrt_pathset* ps, float* A_out, float* E0_out, risrt_amat** resident_out);

/* A handle viewing caller memory A [n_rx][M] and E0 [n_rx] (complex64; E0 may be NULL, meaning 0) for
 * risrt_sweep_configs and risrt_grad_phases; no copy, the caller keeps the memory alive and unchanged
 * while the handle is used. 1 <= n_rx <= 2^26, 1 <= M <= 65536. */
int risrt_amat_wrap(risrt_ctx* ctx, const float* A, const float* E0, int64_t n_rx, int32_t M, risrt_amat** out);

/* Device pointers and sizes of a channel matrix (any output may be NULL). */
int risrt_amat_data(const risrt_amat* amat, const float** A, const float** E0, int64_t* n_rx, int32_t* M);

/* Free a handle (synchronises the context; owned memory returns to the context's cache). */
int risrt_amat_destroy(risrt_ctx* ctx, risrt_amat* amat);

/* ------------------------------------------------------------------------------------------------
 * Configuration sweep (Eq. 9 is linear in Gamma; Eq. 10)
 * ---------------------------------------------------------------------------------------------- */

enum {
    RISRT_PREC_FP32 = 0,    /* complex GEMM on the CUDA cores, FP32 */
    RISRT_PREC_BF16 = 1,    /* tensor cores (tcgen05), BF16 operands, FP32 accumulation */
    RISRT_PREC_BF16X2 = 2,  /* tensor cores, A split into BF16 hi + lo (Gamma rounded to BF16) */
    RISRT_PREC_FP16 = 3     /* tensor cores, FP16 operands, A scaled by a power of two */
};

/* Bytes of device workspace risrt_sweep_configs needs for these sizes and precision (0 for FP32). */
int risrt_sweep_workspace_size(int64_t n_rx, int32_t M, int32_t n_cfg, int precision, size_t* bytes);

/* For every receiver r and configuration c of the channel matrix `amat` (risrt_build_A or
 * risrt_amat_wrap):
 *   E[r][c] = E0[r] + sum_m A[r][m] Gamma[c][m],   P[r][c] = |E[r][c]|^2 / (2 eta0)   (Eqs. 9, 10)
 * Configurations, exactly one of:
 *   gamma      [n_cfg][M] complex64, or
 *   gamma_2bit [n_cfg][ceil(M/4)] uint8: 2-bit phase codes q, element m in bits 2 (m % 4) of byte m / 4
 *              (the bits of a row's last byte beyond M are ignored), Gamma = amp j^q (q = 0..3: amp,
 *              j amp, -amp, -j amp: phases quantised to 2 bits with one common amplitude). Every
 *              value is exact in BF16 when amp is.
 * Outputs (at least one): P_out [n_rx][n_cfg] float, E_out [n_rx][n_cfg] complex64.
 * The tensor-core precisions run the complex product as one real GEMM ([Re A | Im A] against
 * interleaved [Re G, -Im G] / [Im G, Re G] rows) with the |E|^2 epilogue fused; they need a
 * workspace of risrt_sweep_workspace_size bytes (16-byte aligned) and synchronise the stream.
 * 1 <= n_cfg <= 2^24. Errors: RISRT_ERR_INVALID_ARG; RISRT_ERR_TIMEOUT if a pipeline wait in the
 * tensor-core kernel expired (the kernel then stops and the output is incomplete). */
int risrt_sweep_configs(risrt_ctx* ctx, const risrt_amat* amat, const float* gamma, const uint8_t* gamma_2bit,
                        float amp, int32_t n_cfg, int precision, float* P_out, float* E_out, void* workspace,
                        size_t workspace_bytes);

/* OR-ed into the precision of risrt_sweep_configs with RISRT_PREC_BF16 or RISRT_PREC_BF16X2
 * (RISRT_ERR_INVALID_ARG with RISRT_PREC_FP16; ignored with RISRT_PREC_FP32):
 * RISRT_SWEEP_KEEP_A: the caller states that A, n_rx, M, the precision, the workspace and its size
 *   are those of an earlier call, whose packed copy of A in the workspace is then reused (only gamma
 *   is packed); n_cfg may differ while it fits the workspace. Results are undefined if A changed.
 *   Calls sharing a workspace must not overlap in time.
 * RISRT_SWEEP_DEFER_CHECK: the call only enqueues work on the stream and does not synchronise, so it
 *   can be captured into a CUDA graph; the tensor-core kernel's wait-timeout flag is left in the
 *   workspace for risrt_sweep_check. */
#define RISRT_SWEEP_KEEP_A 0x100
#define RISRT_SWEEP_DEFER_CHECK 0x200

/* Fused channel tile -> tensor-core sweep over a path set (Eq. 9 linear in Gamma, Eq. 10): the channel
 * matrix A[r][m] = c_m sum_q b_mq(r) of risrt_build_A is computed, 128 receivers x 32 elements at a
 * time, straight into shared memory and consumed there by the tensor cores in BF16 (FP32
 * accumulation); A is never written to memory. At most 128 configurations per call (one tensor-memory
 * accumulator). Configurations as in risrt_sweep_configs: gamma [n_cfg][M] complex64 or gamma_2bit
 * [n_cfg][ceil(M/4)] codes with amp. P_out [n_rx][n_cfg] float (|E|^2 / (2 eta0)) and/or E_out
 * [n_rx][n_cfg] complex64, receiver-major. Arithmetic and accuracy as risrt_sweep_configs with
 * RISRT_PREC_BF16 on the same path set's channel matrix. Synchronises the stream. Errors:
 * RISRT_ERR_INVALID_ARG (n_cfg outside [1, 128], both or neither of gamma / gamma_2bit, no output),
 * RISRT_ERR_TIMEOUT (a pipeline wait expired; the call's outputs are then undefined). */
int risrt_sweep_fused(risrt_ctx* ctx, const risrt_pathset* ps, const float* gamma, const uint8_t* gamma_2bit, float amp,
                      int32_t n_cfg, float* P_out, float* E_out);

/* After sweeps with RISRT_SWEEP_DEFER_CHECK on this workspace: waits for the context's stream and
 * returns RISRT_ERR_TIMEOUT if a pipeline wait of the last such sweep expired (its output is then
 * incomplete), else RISRT_OK. The flag is cleared by every sweep. */
int risrt_sweep_check(risrt_ctx* ctx, const void* workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------------------------------------
 * Phase gradient (adjoint of Eq. 9 and Eq. 10)
 * ---------------------------------------------------------------------------------------------- */

/* Workspace bytes for risrt_grad_phases (n_target receivers, B configurations, M elements) at the
 * given precision (RISRT_PREC_FP32 or RISRT_PREC_BF16X2; anything else: RISRT_ERR_INVALID_ARG). */
int risrt_grad_workspace_size(int32_t n_target, int32_t B, int32_t M, int precision, size_t* bytes);

/* OR-ed into the precision of risrt_grad_phases with RISRT_PREC_BF16X2: the caller states that A, E0,
 * target and the sizes are those of the previous call with this workspace, whose packed copies of A
 * are then reused (only the phase-dependent operands are rebuilt). Results are undefined if they
 * changed. Ignored for RISRT_PREC_FP32. */
#define RISRT_GRAD_KEEP_A 0x100
/* OR-ed into the precision of risrt_grad_phases: the call only enqueues work on the stream and does not
 * synchronise, so successive steps overlap and a step can be captured into a CUDA graph; with
 * RISRT_GRAD_KEEP_A the target rows are not validated again (they are those of the earlier call). The
 * tensor-core GEMMs' wait-timeout flag is left in the workspace for risrt_grad_check (cleared by every
 * call); J_out and grad_out are ready in stream order. */
#define RISRT_GRAD_DEFER_CHECK 0x200

/* For B phase configurations Gamma_bm = amp_m e^{j phases[b][m]} on the channel matrix `amat`:
 *   J[b]       = sum_{t} log P_b(target[t]),  P = |E0 + A Gamma_b|^2 / (2 eta0)
 *   grad[b][m] = dJ[b]/dphases[b][m] = -2 Im(Gamma_bm sum_t A[target[t]][m] conj(E) / |E|^2)
 * with |E|^2 clamped below at 1e-30 of its maximum over the targets of configuration b.
 *   target [n_target] int32 rows of A (NULL: rows 0..n_target-1), phases [B][M] float, amp [M] float or
 *   NULL (1), J_out [B] float, grad_out [B][M] float, workspace of risrt_grad_workspace_size bytes. All
 *   device memory.
 * precision RISRT_PREC_FP32: FP32 arithmetic on the CUDA cores, A read twice (forward and adjoint
 * GEMM, each split over its reduction axis with the partial sums added in a fixed order, so results
 * do not depend on scheduling). RISRT_PREC_BF16X2: both GEMMs on the tensor cores as real BF16 GEMMs
 * in which every factor is split into a high and a low BF16 part (three products per pair, about
 * 1e-5 relative), FP32 accumulation, partial sums again added in a fixed order; A's target rows are
 * packed into the two operands on every call. The workspace must be 256-byte aligned. Synchronises
 * the stream (the target rows are validated on the device) unless RISRT_GRAD_DEFER_CHECK. Errors: RISRT_ERR_INVALID_ARG (sizes,
 * precision, a target row outside [0, n_rx)); RISRT_ERR_NOT_READY (the paired tensor-core kernel
 * cannot run on this device); RISRT_ERR_TIMEOUT (a pipeline wait in the tensor-core kernel expired). */
int risrt_grad_phases(risrt_ctx* ctx, const risrt_amat* amat, const int32_t* target, int32_t n_target,
                      const float* phases, const float* amp, int32_t B, float* J_out, float* grad_out,
                      void* workspace, size_t workspace_bytes, int precision);

/* After calls with RISRT_GRAD_DEFER_CHECK on this workspace: waits for the context's stream and returns
 * RISRT_ERR_TIMEOUT if a pipeline wait of the last such call's tensor-core GEMMs expired (its J and
 * gradient are then incomplete), else RISRT_OK. */
int risrt_grad_check(risrt_ctx* ctx, const void* workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------------------------------------
 * Allocation-free path search (this entry point has no counterpart in the paper; it exists for
 * callers that may not allocate device memory while they run, e.g. code executing where the CUDA
 * allocator must not be touched or hosts that give the library a fixed memory budget)
 * ---------------------------------------------------------------------------------------------- */

/* Valid reflected face sequences (length 1..max_order, ids as in risrt_pathset_export, ascending)
 * between the points src and dst: the same search trace_paths runs for the Tx leg (src = Tx with
 * src_face -1, dst = RIS centre with dst_face = the RIS host face), with the same validity rules
 * (a face whose plane contains dst may not be the last bounce). It calls no cudaMalloc, cudaFree or
 * allocating routine: its scratch is a 12 MiB array inside the library image, held by every GPU that
 * loads the library until the process exits. Sizes beyond it fail with RISRT_ERR_CAPACITY (order 2
 * fits scenes of up to about 250 faces, order 1 up to about 70000; at most 4096 geometric
 * candidates). The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. Every call uses the same array and clears what it
 * needs, so calls whose GPU work overlaps (other streams, other threads, other contexts on the same
 * device) race and must be serialised by the caller. Synchronises the context's stream.
 *   src, dst     host [3] float points
 *   ids_host     host [cap] int64, receives the ids; *n_host receives their number
 * Errors: RISRT_ERR_INVALID_ARG; RISRT_ERR_CAPACITY (also when cap < number found). */
int risrt_find_paths_noalloc(risrt_ctx* ctx, const risrt_scene* scene, const float src[3], int32_t src_face,
                             const float dst[3], int32_t dst_face, int32_t max_order, int64_t* ids_host,
                             int32_t cap, int32_t* n_host);

/* ------------------------------------------------------------------------------------------------
 * Tracing
 * ---------------------------------------------------------------------------------------------- */

/* on != 0: bracket every kernel this context launches with CUDA events on its stream and keep the
 * elapsed time per kernel name (adds two event records per launch; off by default). */
int risrt_profile_enable(risrt_ctx* ctx, int on);

/* Restrict the profiling of risrt_profile_enable to the kernels named `name` (NULL or "" for all),
 * so that a timed run brackets only the kernel it reports on. Returns RISRT_ERR_INVALID_ARG for a
 * NULL context. */
int risrt_profile_only(risrt_ctx* ctx, const char* name);

/* Total elapsed milliseconds and launch count of kernel `name` since the last reset, or of all
 * kernels when name is NULL. Synchronises the pending events. Unknown names give 0 and 0. */
int risrt_profile_query(risrt_ctx* ctx, const char* name, double* total_ms, int64_t* launches);

/* Comma-separated names of the kernels timed so far, written to buf (NUL-terminated, truncated to
 * cap). *needed receives the full length + 1 (may be NULL). */
int risrt_profile_names(risrt_ctx* ctx, char* buf, size_t cap, size_t* needed);

int risrt_profile_reset(risrt_ctx* ctx);

/* Issue-rate microbenchmarks of the pipes the field kernels use (the measured denominators of their
 * roofline). kind: RISRT_MB_FFMA (FP32 fused multiply-add), RISRT_MB_MUFU_* (the special-function
 * unit's single-instruction sine, cosine, reciprocal square root, reciprocal, square root and base-2
 * exponential), RISRT_MB_DFMA (FP64 fused multiply-add). Runs independent chains on every SM at full
 * occupancy for `iters` iterations per chain; *ops_per_s receives the lane operations per second of
 * the best of three timed launches (CUDA events on the context's stream), *ms (may be NULL) its
 * duration. Synchronises the stream. */
enum {
    RISRT_MB_FFMA = 0,
    RISRT_MB_MUFU_SIN = 1,
    RISRT_MB_MUFU_COS = 2,
    RISRT_MB_MUFU_RSQ = 3,
    RISRT_MB_MUFU_RCP = 4,
    RISRT_MB_MUFU_SQRT = 5,
    RISRT_MB_MUFU_EX2 = 6,
    RISRT_MB_DFMA = 7
};
int risrt_microbench(risrt_ctx* ctx, int kind, int32_t iters, double* ops_per_s, double* ms);

/* Number of kernels the library has launched in this process (all contexts), for accounting. */
int risrt_launch_count(int64_t* out);

/* ------------------------------------------------------------------------------------------------
 * Destruction (each synchronises the context stream first; NULL is accepted)
 * ---------------------------------------------------------------------------------------------- */
int risrt_scene_destroy(risrt_ctx* ctx, risrt_scene* scene);
int risrt_ris_destroy(risrt_ctx* ctx, risrt_ris* ris);
int risrt_rxset_destroy(risrt_ctx* ctx, risrt_rxset* rxset);
int risrt_pathset_destroy(risrt_ctx* ctx, risrt_pathset* ps);

#ifdef __cplusplus
}
#endif

#endif /* RISRT_H */
