/*
 * vafr.h -- C ABI of the GB300 (sm_103a) VaFR ray-casting library (libvafr.so).
 *
 * The library implements the data-parallel hot path of "Visual Acuity
 * Consistent Foveated Rendering towards Retinal Resolution" (Zhang, Gai, Li;
 * arXiv 2503.23410) for its ray-casting pipeline (Sec. 6.1): one primary ray
 * per texel of the constant-size log-polar (LP) buffer generated through the
 * inverse mapping (Eqs. 3, 10, 11 with the segmented mapping of Eq. 12),
 * closest-hit / miss shading into the LP buffer, and the inverse-mapping pass
 * that reconstructs the full-resolution display (Sec. 3.4).  The "GT" of the
 * paper's evaluation (one ray per display pixel, Sec. 5.2.1 and Table 1) is
 * provided as the baseline.
 *
 * Conventions (every entry point):
 *  - Return value: VAFR_OK (0) or a negative VAFR_ERR_* code.  No C++
 *    exception crosses this boundary: a failed host allocation returns
 *    VAFR_ERR_OOM.  vafr_last_error_message() gives a human-readable detail
 *    for the calling thread's last failure (a per-thread buffer, valid until
 *    that thread's next failure).
 *  - Work is asynchronous on the given CUDA stream (passed as void*, a
 *    cudaStream_t; NULL = legacy default stream).  Device-side faults of the
 *    method (traversal stack overflow, watchdog) set a per-object status word
 *    that vafr_session_check / vafr_scene_check read after a stream sync.
 *  - Ownership: the caller owns every buffer it passes (LP buffers, display
 *    buffers, hit-id buffers).  The library owns the scene's acceleration
 *    structure, each session's tables and each batch's graph.
 *  - Pointers documented "device" must be device memory of the current device.
 *    Pointers documented "host or device" are classified with
 *    cudaPointerGetAttributes.
 *  - Coordinates: display pixels, x right, y down, pixel (i, j) centred at
 *    (i + 0.5, j + 0.5).  Camera: x right, y up, z forward; a pose is a
 *    row-major 3x4 [R | t] taking camera to world coordinates.
 *  - Colours: RGBA, alpha = 1.  VAFR_FMT_RGBA32F = 4 x float (16 B),
 *    VAFR_FMT_RGBA16F = 4 x IEEE half, round-to-nearest-even (8 B).
 */
#ifndef VAFR_H
#define VAFR_H

#include <stdint.h>

#if defined(__GNUC__)
#define VAFR_API __attribute__((visibility("default")))
#else
#define VAFR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define VAFR_OK               0
#define VAFR_ERR_INVALID_ARG (-1) /* bad pointer, size, format, eye, NaN gaze  */
#define VAFR_ERR_OOM         (-2) /* device or host allocation failed          */
#define VAFR_ERR_CUDA        (-3) /* a CUDA runtime call failed                */
#define VAFR_ERR_TIMEOUT     (-4) /* a device watchdog (iteration limit) fired */
#define VAFR_ERR_BUDGET      (-5) /* request exceeds a configured memory budget */
#define VAFR_ERR_DEVICE      (-6) /* device status word reports a fault        */
#define VAFR_ERR_UNSUPPORTED (-7) /* no usable sm_103 device                   */

#define VAFR_FMT_RGBA32F 0
#define VAFR_FMT_RGBA16F 1

#define VAFR_MAX_PIVOTS 9
#define VAFR_MAX_BATCH  128   /* frame-eyes per batched launch */
#define VAFR_MAX_POINT_LIGHTS 256   /* vafr_scene_set_point_lights */

typedef struct vafr_scene vafr_scene;
typedef struct vafr_session vafr_session;
typedef struct vafr_batch vafr_batch;

/* Acuity pivots of the segmented mapping (Sec. 3.3, Eq. 12): MAR = 1/f is
 * piecewise linear through (pivot_ecc_deg[k], 1/pivot_cpd[k]);
 * pivot_ecc_deg[0] must be 0 and strictly increasing; e_max_deg is the
 * maximum perceivable eccentricity (Sec. 3.2.2).
 * Anisotropic acuity (Sec. 9, Eq. 19): with anisotropic != 0 the tangential
 * shading rate is Delta(e) times the radial one, Delta piecewise linear in e
 * through (pivot_ecc_deg[k], pivot_delta[k]) and constant past the last
 * pivot (every pivot_delta[k] > 0); column c then holds
 * max(1, round(Delta(e_c) l(e_c))) texels.  anisotropic = 0 ignores
 * pivot_delta (Delta = 1, the paper's default mapping). */
typedef struct {
    int32_t n_pivots;
    double  pivot_ecc_deg[VAFR_MAX_PIVOTS];
    double  pivot_cpd[VAFR_MAX_PIVOTS];
    double  e_max_deg;
    int32_t anisotropic;
    double  pivot_delta[VAFR_MAX_PIVOTS];
} vafr_acuity;

/* Fills the paper's pivots: f = 40, 10, 6, 5, 4 cpd at 0, 10, 20, 30, 60 deg
 * and e_max = 60 deg (Sec. 3.3 and Sec. 3.2.2); isotropic. */
VAFR_API void vafr_acuity_default(vafr_acuity* a);
/* The paper's pivots with the anisotropy of Sec. 9: tangential acuity equal
 * to radial at the fovea and half of it from 30 deg on (the factor of two at
 * 30 deg the paper takes from the literature), linear in between:
 * Delta = 1, 5/6, 2/3, 1/2, 1/2 at the five pivots. */
VAFR_API void vafr_acuity_anisotropic(vafr_acuity* a);
/* A curve for a display that resolves at most max_cpd cycles/deg (the
 * head-mounted-display curves of Sec. 3.3): the paper's pivots with every
 * pivot acuity capped at max_cpd, so the fovea is shaded at the display's
 * own density.  Errors: INVALID_ARG (NULL, max_cpd <= 0). */
VAFR_API int vafr_acuity_display_limited(vafr_acuity* a, double max_cpd);

/* A display + viewer.  n_eyes 1 (mono) or 2 (binocular, VaFR_Dup of Sec. 5.1:
 * each eye rendered independently).  fov_v_deg is the vertical field of view;
 * c_r = 2 tan(fov_v/2) / height (Sec. 3.2.1). */
typedef struct {
    int32_t     width, height;
    double      fov_v_deg;
    int32_t     n_eyes;
    double      eye_pose[2][12];
    int32_t     lp_format;       /* VAFR_FMT_* of the LP buffer             */
    int32_t     display_format;  /* VAFR_FMT_* of the reconstructed display */
    vafr_acuity acuity;
    int32_t     lp_fxaa;         /* 1: FXAA inside the LP buffer before the
                                    inverse mapping (Sec. 3.4), see
                                    vafr_fxaa_lp; 0: none                  */
} vafr_session_desc;

/* One frame-eye of a batched launch. */
typedef struct {
    vafr_session* session;
    int32_t       eye;
    void*         lp;        /* device, LP buffer of that eye (see vafr_render_lp) */
    void*         display;   /* device or page-locked host memory, height x width
                                pixels of display_format (host displays are written
                                through a device staging buffer of the batch and a
                                copy-engine transfer on the same stream)           */
    void*         lp_aa;     /* device, second LP buffer receiving the FXAA pass;
                                required when the session has lp_fxaa, else ignored */
} vafr_frame_desc;

/* ---- errors -------------------------------------------------------------- */
VAFR_API const char* vafr_error_string(int code);
VAFR_API const char* vafr_last_error_message(void);
/* Library version (major*10000 + minor*100 + patch) and the number of
 * kernels this library launched so far on this process (all devices). */
VAFR_API int32_t vafr_version(void);
VAFR_API int64_t vafr_kernel_launch_count(void);

/* ---- scene ---------------------------------------------------------------
 * vafr_build_scene: builds the ray-casting acceleration structure of a
 * triangle soup (the paper's closest-hit stage, Sec. 6.1, leaves the
 * acceleration structure to the API; this library builds an LBVH after
 * Karras 2012: 30-bit Morton codes of centroids, stable radix sort, binary
 * radix tree, bottom-up FP32 bounds).
 *   tri_xyz    host or device, n_tris x 3 vertices x 3 floats (xyz).
 *   albedo_rgb host or device, n_tris x 3 floats in [0, 1]; NULL = 0.8 grey.
 *   n_tris     0 <= n_tris < 2^30 (0 gives an empty scene: every ray misses).
 *   light_dir  host, 3 floats, direction the light travels (normalised here).
 *   stream     stream for the build; the scene is usable on any stream after
 *              the build's work on `stream` completes.
 *   out        receives the handle (library-owned; vafr_scene_destroy).
 * Errors: INVALID_ARG (NULL tri_xyz with n_tris > 0, n_tris out of range,
 * non-finite light), OOM, CUDA. */
VAFR_API int vafr_build_scene(const float* tri_xyz, const float* albedo_rgb, int64_t n_tris,
                     const float light_dir[3], void* stream, vafr_scene** out);
/* Point lights for the direct-shading pipelines (ray-cast LP and GT, the
 * deferred path): each adds albedo * rgb * max(0, n . l) / |x - p|^2 at a
 * hit point p (l the unit vector to the light at x, n the geometric normal
 * facing the ray), unshadowed, on top of the Lambert + ambient directional
 * light -- the many-light scenes the paper's deferred tests use (Sec. 5.2).
 * Path tracing ignores them.  Replaces any previous set; n = 0 removes them.
 *   pos_xyz, rgb  host, n x 3 floats; rgb >= 0.
 * Errors: INVALID_ARG (n outside [0, VAFR_MAX_POINT_LIGHTS], NULL arrays,
 * non-finite values), OOM, CUDA. */
VAFR_API int vafr_scene_set_point_lights(vafr_scene* scene, int32_t n, const float* pos_xyz,
                                         const float* rgb);
VAFR_API int vafr_scene_destroy(vafr_scene* scene);
/* Triangle count and device bytes held by the scene. */
VAFR_API int vafr_scene_info(const vafr_scene* scene, int64_t* n_tris, int64_t* device_bytes);
/* Copies the tree the rays traverse to HOST buffers (either may be NULL; call
 * with both NULL to learn n_nodes first).  It is built by PLOC over the
 * Morton-sorted leaves (Meister and Bittner 2018) and collapsed into 4-wide
 * nodes; the paper's acceleration structure is the driver's own (Sec. 6.1),
 * so this is the build's choice, checked by its invariants.
 *   n_nodes  number of 4-wide nodes; node 0 is the root.
 *   nodes    n_nodes x 32 floats: per axis the lo then hi planes of the four
 *            children (lo.x[4], hi.x[4], lo.y[4], hi.y[4], lo.z[4], hi.z[4]),
 *            then four int32 child references (>= 0 node, < 0 leaf ~k,
 *            INT32_MIN unused), then four uint32 slot keys (q for an internal
 *            child in slot q, 0xFFFFFFFF otherwise).  Internal children take
 *            the first slots and are consecutive nodes (slot q's reference is
 *            slot 0's + q); leaves follow; unused slots come last.
 *   leaves   n_tris x 12 floats, sorted (leaf) order: v0.xyz | id bits,
 *            v1.xyz | 0, v2.xyz | 0, vertices in lexicographic order.
 * A scene of fewer than two triangles has no nodes.  Synchronises the
 * device.  Errors: INVALID_ARG, CUDA. */
VAFR_API int vafr_scene_export_tree4(const vafr_scene* scene, int64_t* n_nodes, float* nodes,
                                     float* leaves);
/* Copies the LBVH build products to HOST buffers (any may be NULL):
 *   codes      n     uint32 Morton codes, input triangle order
 *   sorted_ids n     int32 triangle ids in sorted (leaf) order
 *   child      n-1 x 2 int32: >= 0 internal node, < 0 leaf ~k (k = leaf index)
 *   node_box   n-1 x 6 float (lo xyz, hi xyz) of internal nodes
 *   leaf_box   n   x 6 float of leaves (sorted order)
 * Synchronises the device.  Errors: INVALID_ARG, CUDA. */
VAFR_API int vafr_scene_export_lbvh(const vafr_scene* scene, uint32_t* codes, int32_t* sorted_ids,
                           int32_t* child, float* node_box, float* leaf_box);
/* Synchronises `stream` and reads + clears the scene's device status word.
 * Returns VAFR_OK, VAFR_ERR_DEVICE or VAFR_ERR_TIMEOUT. */
VAFR_API int vafr_scene_check(const vafr_scene* scene, void* stream);

/* Failure injection for tests of the device status words, made on the host:
 * rewrites the child references and slot keys of the root of the scene's
 * 4-wide tree in device memory (the node boxes stay), so that the traversal's own checks
 * stop the affected rays and report the fault through the session status word
 * of the launch (vafr_session_check) instead of touching memory out of range.
 *   VAFR_INJECT_NONE        restore the references and keys saved by the first
 *                           injection
 *   VAFR_INJECT_BAD_CHILD   every used slot becomes an internal child from
 *                           the first index past the last 4-wide node on: the
 *                           node check fails (VAFR_ERR_DEVICE)
 *   VAFR_INJECT_LOOP        slot 0 names the root itself, the other slots are
 *                           emptied: a ray entering slot 0's box cycles without
 *                           growing its stack until the iteration limit of
 *                           4 n_tris + 64 node visits (VAFR_ERR_TIMEOUT)
 *   VAFR_INJECT_STACK       every used slot names the root: a ray entering two
 *                           or more of the root's boxes pushes at every visit
 *                           until the 128-entry stack would overflow (status
 *                           bit 1); a ray entering one box cycles as above
 *                           (bit 2, which takes precedence: VAFR_ERR_TIMEOUT)
 * The check's error message ("session status 0x..") carries the bits:
 * 1 stack, 2 iteration limit, 4 child reference out of range.
 * The scene must have at least two triangles.  Synchronises the device.
 * Errors: INVALID_ARG (NULL, unknown kind, one triangle), CUDA. */
#define VAFR_INJECT_NONE      0
#define VAFR_INJECT_BAD_CHILD 1
#define VAFR_INJECT_LOOP      2
#define VAFR_INJECT_STACK     3
VAFR_API int vafr_scene_inject_fault(vafr_scene* scene, int32_t kind);
/* Host-side fault injection for tests of error recovery (no counterpart in
 * the paper).  Arms a per-thread countdown: the batch entry points
 * (vafr_batch_create, _render, _capture, _autotune) pass a checkpoint before
 * each host allocation they make, and the checkpoint reached when the
 * countdown is 0 fails as a failed allocation does: the call returns
 * VAFR_ERR_OOM and leaves the batch as it was before the call (a captured
 * graph, its parameters and frames stay consistent; a graph whose staging
 * buffer had to be replaced is dropped, so vafr_batch_replay then returns
 * INVALID_ARG instead of copying from freed memory).  The countdown then
 * stays off until armed again.  countdown = -1 disarms it.
 * Errors: INVALID_ARG (countdown < -1). */
VAFR_API int vafr_debug_fail_host_alloc(int32_t countdown);

/* ---- session --------------------------------------------------------------
 * vafr_session_create: validates the description and builds, in FP64 on the
 * host, the discrete LP layout of the acuity model: columns c at
 * u = c + 0.5 < u(e_max) (Eq. 12), eccentricity e_c by the inverse mapping
 * (Eq. 10), n_c = max(1, round(l(e_c))) texels per column (Eq. 9), texel
 * (c, j) at angle (j + 0.5) 360/n_c (Eq. 11).  The layout does not depend on
 * the display size (Sec. 3.2.2).
 * Errors: INVALID_ARG (size <= 0 or > 32768, fov outside (0, 170), n_eyes
 * not 1 or 2, bad pivots, non-finite pose, unknown format), OOM, CUDA. */
VAFR_API int vafr_session_create(const vafr_session_desc* desc, vafr_session** out);
VAFR_API int vafr_session_destroy(vafr_session* session);
/* Copies the LP layout to HOST buffers (any may be NULL): n_cols, n_texels
 * (texels = rays per eye), col_counts[n_cols], col_offsets[n_cols],
 * col_ecc_deg[n_cols] (FP32 eccentricity of each column centre).
 * LP buffer layout: columns are stored one after another, texel (c, j) in
 * slot col_offsets[c] + j; each column is framed by two guard slots,
 * col_offsets[c] - 1 holding a copy of texel (c, n_c - 1) and
 * col_offsets[c] + n_c a copy of texel (c, 0) (the angular wrap), so one
 * eye's buffer holds n_texels + 2 n_cols slots (vafr_session_sizes).
 * Errors: INVALID_ARG. */
VAFR_API int vafr_lp_layout(const vafr_session* session, int32_t* n_cols, int64_t* n_texels,
                   int32_t* col_counts, int64_t* col_offsets, float* col_ecc_deg);
/* Bytes of one eye's LP buffer and of one eye's display in the session's formats. */
VAFR_API int vafr_session_sizes(const vafr_session* session, int64_t* lp_bytes_per_eye,
                       int64_t* display_bytes_per_eye);
/* Reads (set = 0) or writes (set = 1) the kernel variants used by this
 * session's single-session calls: cfg[0] render variant, cfg[1] reconstruct
 * tile shape (see vafr_tuning_space).  Render variants 6 and 7 take the LP
 * work in chunks of 32 rays and render the chunks that were slowest in the
 * session's previous frame first, so a launch does not end waiting for slow
 * chunks that happened to come last (7 keeps fewer registers, 7 blocks per
 * SM).  Results do not depend on the choice.
 * Errors: INVALID_ARG (NULL, variant out of range). */
VAFR_API int vafr_session_tuning(vafr_session* session, int32_t set, int32_t cfg[2]);
/* Picks the session's kernel variants by timing whole frames at the current
 * gaze: every render variant renders `warm` untimed frames (variants 6 and 7,
 * the longest-first order, need two frames of history) and then `iters` timed
 * frames (render_lp of all eyes + reconstruct of every eye, CUDA events on
 * `stream`); then every reconstruct variant is timed the same way with the
 * chosen render variant.  The fastest pair is kept and written to cfg_out
 * (may be NULL).
 *   lp       device, n_eyes x vafr_session_sizes lp bytes, 16-byte aligned.
 *   display  device, n_eyes x display bytes, 16-byte aligned.
 * Synchronises `stream`.  Errors: INVALID_ARG (NULL, unaligned, gaze not set),
 * CUDA. */
VAFR_API int vafr_session_autotune(const vafr_scene* scene, vafr_session* session, void* lp, void* display,
                                   int32_t warm, int32_t iters, int32_t cfg_out[2], void* stream);
/* Sets the gaze point (x0, y0) in display pixels of one eye (Eq. 3).  Any
 * finite value with |x0|, |y0| <= 1e7 is accepted (gaze outside the display
 * is legal; with displays of at most 32768 pixels a side every pixel offset
 * from the gaze is then an exact FP32 integer plus fraction).  The FP64
 * per-frame set-up (c_r, gaze tangent offsets, the integer/fraction split of
 * the gaze used by reconstruction) is done here on the host; the next render
 * or reconstruct call on the session uses it.  Errors: INVALID_ARG (eye out
 * of range, NaN/inf, |gaze| > 1e7). */
VAFR_API int vafr_set_gaze(vafr_session* session, int32_t eye, double x0, double y0);
/* Synchronises `stream` and reads + clears the session's device status word. */
VAFR_API int vafr_session_check(vafr_session* session, void* stream);

/* ---- the hot path ----------------------------------------------------------
 * vafr_render_lp: for every texel of the eyes in eye_mask (bit e = eye e),
 * casts the primary ray through the texel's screen point (Eqs. 3, 10, 11),
 * finds the closest hit (two-sided watertight test, closest t > 0, equal t ->
 * lower triangle id) and shades it (Lambert, ambient 0.1; sky gradient on a
 * miss) -- the ray-generation / closest-hit / miss shaders of Sec. 6.1.
 *   lp_out      device, [popcount(eye_mask)][slots] pixels of lp_format,
 *               eyes in increasing order, in the layout of vafr_lp_layout
 *               (guard slots included; slots = lp_bytes_per_eye / pixel size).
 *   hit_ids_out device or NULL, [popcount(eye_mask)][slots] int32 triangle
 *               id of the hit, -1 on a miss, same layout.
 * Errors: INVALID_ARG (NULL lp_out, eye_mask not a subset of the session's
 * eyes or empty, gaze never set), CUDA. */
VAFR_API int vafr_render_lp(const vafr_scene* scene, vafr_session* session, int32_t eye_mask,
                   void* lp_out, int32_t* hit_ids_out, void* stream);
/* vafr_render_lp_pt: the path-traced LP buffer (Sec. 8: the LP texels are
 * rendered by a path tracer at one sample each, next-event estimation on, no
 * Russian roulette, at most max_diffuse diffuse bounces; 3 is the paper's
 * setting).  Every surface is Lambertian with the scene's albedo; lights are
 * the scene's directional light (radiance scale 1, through shadow rays) and
 * the sky gradient of vafr_render_lp's miss shading (seen by escaping rays).
 * Rays leaving a surface start 1e-5 max(1, |p|_inf) off it along the normal
 * facing the incoming ray and ignore the triangle they leave; bounce
 * directions are cosine-distributed (basis of Duff et al. 2017).  Random
 * numbers: uniform = top 24 bits of SplitMix64's output function applied to
 * seed, the texel's index in column order (texels only, no guard slots) and
 * 2 k + dim (k = bounce, dim 0/1) in turn, / 2^24.
 *   lp_out        as vafr_render_lp; alpha 1.
 *   path_sig_out  device or NULL, [popcount(eye_mask)][slots][max_diffuse + 2]
 *                 int32: hit triangle id of each segment (-1 miss, -2 not
 *                 traced), then a mask: bit k = segment k's shadow ray
 *                 reached the light, bit 16 + k = a shadow ray was cast there
 *                 (n . -L > 0); written for texel slots only.
 * Errors: INVALID_ARG (as vafr_render_lp, max_diffuse outside [0, 15]), CUDA. */
VAFR_API int vafr_render_lp_pt(const vafr_scene* scene, vafr_session* session, int32_t eye_mask,
                               void* lp_out, uint64_t seed, int32_t max_diffuse,
                               int32_t* path_sig_out, void* stream);
/* vafr_render_full_gt_pt: the path-traced GT: one path per display pixel
 * centre with vafr_render_lp_pt's estimator (random numbers keyed by the
 * pixel index y width + x), written to display_out (display_format).
 * Errors: INVALID_ARG, CUDA. */
VAFR_API int vafr_render_full_gt_pt(const vafr_scene* scene, vafr_session* session, int32_t eye,
                                    void* display_out, uint64_t seed, int32_t max_diffuse,
                                    void* stream);
/* VaFR_Rep (Sec. 5.1): the right eye's LP buffer by forward grid warping of
 * the left eye's (the reprojection of Wissmann et al. 2020, directly from the
 * LP buffer), disocclusions ray cast.  Each left texel's hit point (a miss:
 * the point at infinity along its ray) is mapped through the right eye's
 * forward map to (U, F) = (u - 1/2, angle fraction); each pair of
 * neighbouring LP rings is zipped by angle into triangles; triangles with a
 * vertex behind the right eye, mixing hits and misses, spread over more than
 * 1.1x in depth, or spanning more than 64 columns or a quarter turn are
 * dropped; the rest are rasterised at the right texel centres with a
 * nearest-depth test (ties: lower triangle id) and their three left colours
 * interpolated.  Needs a binocular session with both gazes set; session-owned
 * scratch (~62 MB at the default acuity) is allocated on first use, so calls
 * on one session must not overlap.
 * vafr_render_lp_rep: the whole mode: casts the left eye (eye 0) into
 *   lp_out[0], warps it into lp_out[1] and casts the right eye's holes.
 *   lp_out as vafr_render_lp with both eyes; right_tri_out (device or NULL,
 *   one int32 per slot) receives the warp's winning triangle per right texel
 *   as in vafr_reproject_lp, -1 where the texel was a hole and was cast.
 * vafr_reproject_lp: the warp alone, from a caller's left LP buffer and hit
 *   distances (left_depth: device, one float per slot, +inf on a miss; only
 *   texel slots are read); holes are left unwritten in right_lp_out and
 *   marked -1 in right_tri_out (device or NULL, one int32 per slot: the
 *   winning left triangle, 2 t + {0: towards the next column, 1: towards the
 *   previous one} for left texel t in column order).
 * vafr_rep_hole_count: holes of the last warp on this session (synchronises
 *   `stream`).
 * Errors: INVALID_ARG (NULL, unaligned, not binocular, gaze not set), OOM, CUDA. */
VAFR_API int vafr_render_lp_rep(const vafr_scene* scene, vafr_session* session, void* lp_out,
                                int32_t* right_tri_out, void* stream);
VAFR_API int vafr_reproject_lp(vafr_session* session, const void* left_lp, const float* left_depth,
                               void* right_lp_out, int32_t* right_tri_out, void* stream);
VAFR_API int vafr_rep_hole_count(vafr_session* session, int64_t* holes, void* stream);
/* Deferred pipeline (Sec. 3.4, Sec. 5: the G-buffer pass runs at native
 * resolution and the lighting in the LP buffer).  The G-buffer here is a
 * visibility buffer rasterised in CUDA: per display pixel the 64-bit key
 * (FP32 hit distance bits << 32) | triangle id of the closest triangle,
 * ~0 for the sky.  Its coverage test is the watertight test of the pixel-
 * centre ray and the depth test keeps the smallest (distance, id), so the
 * buffer equals the GT cast's closest hits (triangle parts closer than 1e-4
 * scene units to the camera plane are not drawn).  Triangles are clipped to
 * the view frustum; boxes of at most 128 pixels are rasterised one thread per
 * triangle, larger ones as 16 x 8 pixel tiles spread evenly over all warps.
 * Scene-owned scratch (~32 B per triangle) is allocated on first use, so
 * deferred calls on one scene must not overlap.
 * vafr_render_vbuffer: the G-buffer pass of one eye into vbuf_out (device,
 *   height x width uint64, 8-byte aligned).
 * vafr_shade_lp_deferred: LP lighting: each LP texel takes the shading of the
 *   display pixel under its screen point (clamped to the display); lp_out as
 *   one eye of vafr_render_lp.
 * vafr_shade_full_deferred: full-resolution lighting of every pixel (the
 *   deferred GT) into display_out.
 * Shading is vafr_render_lp's (Lambert + ambient, point lights, sky).
 * Errors: INVALID_ARG (NULL, bad eye, unaligned, gaze not set for the LP
 * pass), OOM, CUDA. */
VAFR_API int vafr_render_vbuffer(const vafr_scene* scene, vafr_session* session, int32_t eye,
                                 uint64_t* vbuf_out, void* stream);
/* vafr_vbuffer_stats: vafr_render_vbuffer through an instrumented copy of the
 * rasteriser (never the timed one), then out[0] = pre-filter evaluations
 * (pixels of triangle boxes outside culled tiles), out[1] = pixels past the
 * screen-space pre-filter, out[2] = exact pixel-ray tests run (past the depth
 * pre-test), out[3] = atomic minima issued.  The counts after the depth
 * pre-test depend on the order the GPU runs triangles in.  Synchronises
 * `stream`.  Errors: as vafr_render_vbuffer. */
VAFR_API int vafr_vbuffer_stats(const vafr_scene* scene, vafr_session* session, int32_t eye,
                                uint64_t* vbuf_out, int64_t out[4], void* stream);
VAFR_API int vafr_shade_lp_deferred(const vafr_scene* scene, vafr_session* session, int32_t eye,
                                    const uint64_t* vbuf, void* lp_out, void* stream);
VAFR_API int vafr_shade_full_deferred(const vafr_scene* scene, vafr_session* session, int32_t eye,
                                      const uint64_t* vbuf, void* display_out, void* stream);
/* vafr_reconstruct: inverse-mapping pass (Sec. 3.4): every display pixel
 * (x + 0.5, y + 0.5) maps forward to (u, angle) with r = |p - gaze|,
 * e = atan(c_r r) clamped to e_max (Eq. 3), u = u(e) (Eq. 12), angle =
 * atan2(y - y0, x - x0) in [0, 360); the colour is the bilinear blend of
 * columns floor(u - 0.5), +1 (clamped) and, in each, of rows
 * floor(angle n_c/360 - 0.5), +1 wrapped modulo n_c.  FP32 arithmetic.
 *   lp       device, one eye's LP buffer (vafr_lp_layout, guard slots filled
 *            as vafr_render_lp writes them).
 *   display  device, height x width pixels of display_format, row-major.
 * Errors: INVALID_ARG, CUDA. */
VAFR_API int vafr_reconstruct(vafr_session* session, int32_t eye, const void* lp, void* display_out,
                     void* stream);
/* vafr_fxaa_lp: FXAA inside one eye's LP buffer (Sec. 3.4: the paper
 * anti-aliases the LP buffer with FXAA before the inverse mapping; Sec. 7
 * ablates it).  FXAA (Lottes 2009) on the LP grid: angular neighbours are
 * the rows j -+ 1 of a column (wrapping), radial neighbours the texel of
 * column c -+ 1 (clamped) whose angular interval holds the same angle; luma
 * 0.299 R + 0.587 G + 0.114 B; texels whose 5-neighbourhood luma range is
 * below max(1/12, max/6) are copied; the others are blended towards one
 * neighbour by the larger of the edge offset (from a 12-step search along
 * the edge) and the subpixel term (weight 3/4).  FP32.
 *   lp      device, the eye's LP buffer as vafr_render_lp writes it.
 *   lp_out  device, another buffer of the same size (not overlapping lp);
 *           receives every texel and its guard copies.
 * The pass keeps the lumas of the eye's texels in session-owned scratch
 * (allocated by vafr_session_create when lp_fxaa is set, else by the first
 * call), so FXAA calls for one session and eye must not overlap in time.
 * Errors: INVALID_ARG (NULL, bad eye, unaligned, lp == lp_out), OOM, CUDA. */
VAFR_API int vafr_fxaa_lp(vafr_session* session, int32_t eye, const void* lp, void* lp_out,
                          void* stream);
/* vafr_render_full_gt: the paper's GT (Sec. 5.2.1, Table 1): one ray per
 * display pixel centre, same traversal and shading, written straight to the
 * display (display_format).  hit_ids_out: device or NULL, height x width int32.
 * Errors: INVALID_ARG, CUDA. */
VAFR_API int vafr_render_full_gt(const vafr_scene* scene, vafr_session* session, int32_t eye,
                        void* display_out, int32_t* hit_ids_out, void* stream);
/* vafr_render_frame: one whole frame of the session (render_lp of every eye
 * into a session-owned LP buffer, the FXAA pass when the session has
 * lp_fxaa, then reconstruct every eye).
 *   display_out  host or device, [n_eyes][height][width] of display_format,
 *                16-byte aligned.  Pinned host memory (page-locked or
 *                registered) is written directly by the reconstruction kernel
 *                through its device alias; pageable host memory is filled by a
 *                device->host copy.  For host memory the call synchronises
 *                `stream` before returning.
 * Errors: as vafr_render_lp / vafr_reconstruct, OOM. */
VAFR_API int vafr_render_frame(const vafr_scene* scene, vafr_session* session, void* display_out,
                      void* stream);
/* Traversal statistics of one eye's LP render (an instrumented copy of the
 * render kernel's 4-wide traversal, never the timed one): out[0] = rays,
 * out[1] = 4-wide nodes visited, out[2] = child boxes tested, out[3] =
 * triangle tests, out[4] = hits, out[5] = most nodes visited by one ray.
 * Host out[6]. */
VAFR_API int vafr_traversal_stats(const vafr_scene* scene, vafr_session* session, int32_t eye,
                         int64_t out[6], void* stream);

/* FP32 issue rate of the current device, the denominator of the traversal
 * kernels' ALU roofline: out[0] = FMAs per second with scalar FFMA, out[1] =
 * FMAs per second with paired FFMA2 (two FMAs per instruction), each the
 * best of three timed launches of 8 independent FMA chains per thread,
 * 2,048 threads per SM, after one warm-up launch.  Synchronises `stream`
 * (allocates and frees a few KB of device memory).  Errors: INVALID_ARG
 * (NULL out), CUDA. */
VAFR_API int vafr_measure_fp32_peak(double out[2], void* stream);

/* ---- batching --------------------------------------------------------------
 * A batch renders many frame-eyes (any mix of sessions, eyes and display
 * sizes, all on one scene) with ONE persistent render launch over all LP
 * texels and ONE persistent reconstruct launch over all display tiles.  The
 * LP and reconstruct work of a frame-eye is the same as vafr_render_lp /
 * vafr_reconstruct on its session.
 *   vafr_batch_create   max_frames <= VAFR_MAX_BATCH.
 *   vafr_batch_render   launches the two kernels directly (no graph).
 *   vafr_batch_capture  records the two launches for `frames` into a CUDA
 *                       graph (replaces any earlier graph of the batch).
 *   vafr_batch_replay   re-reads every captured session's current gaze,
 *                       patches the graph's kernel parameters and launches it.
 *   vafr_batch_autotune times the candidate render block shapes and
 *                       reconstruct tile shapes on `frames` (iters launches
 *                       each, CUDA events) and keeps the fastest.
 *   vafr_batch_tuning   reads (set = 0) or writes (set = 1) the choice:
 *                       cfg[0] render variant, cfg[1] reconstruct variant.
 * With render variant 6 or 7 (longest-first order) vafr_batch_render keeps one
 * order state per frame position of the batch (the first render at a
 * position, or one whose session has more LP texels than before, allocates
 * it and synchronises the device); captured graphs and the autotuner's
 * timings run variants 6 and 7 without an order (chunks in work order).
 * A batch owns device state that its launches use: the render's work
 * counter, the order states and one staging buffer per host display.  Keep
 * at most one render or replay of a batch in flight at a time (for frames in
 * flight on several streams, create one batch per stream); a session may take
 * part in several batches, but not with the same eye in two batches in flight.
 * Errors: INVALID_ARG (n out of range, frame with a NULL buffer, eye out of
 * range, session never given a gaze, display in pageable host memory), CUDA. */
VAFR_API int vafr_batch_create(const vafr_scene* scene, int32_t max_frames, vafr_batch** out);
VAFR_API int vafr_batch_destroy(vafr_batch* batch);
VAFR_API int vafr_batch_render(vafr_batch* batch, const vafr_frame_desc* frames, int32_t n, void* stream);
VAFR_API int vafr_batch_capture(vafr_batch* batch, const vafr_frame_desc* frames, int32_t n, void* stream);
VAFR_API int vafr_batch_replay(vafr_batch* batch, void* stream);
VAFR_API int vafr_batch_autotune(vafr_batch* batch, const vafr_frame_desc* frames, int32_t n,
                        void* stream, int32_t iters);
VAFR_API int vafr_batch_tuning(vafr_batch* batch, int32_t set, int32_t cfg[2]);
/* Number of render / reconstruct variants the autotuner chooses between. */
VAFR_API int vafr_tuning_space(int32_t* n_render, int32_t* n_reconstruct);

/* ---- allocation-free entry point ---------------------------------------------
 * vafr_morton_sort_noalloc: the Morton codes and the stable (code, id) order
 * of a triangle soup -- the first stages of vafr_build_scene -- computed
 * without allocating any memory.  The paper has no counterpart; it exists for
 * callers that may not allocate device memory: code whose GPU memory all
 * belongs to the caller's own pool allocator, or that runs on a
 * latency-critical thread where cudaMalloc's implicit device synchronisation
 * is not acceptable.  The caller passes inputs and outputs; the scratch is a
 * fixed 6.3 MB file-scope device array that every GPU loading the library
 * holds until the process exits.
 *   tri_xyz         device, n_tris x 9 floats.
 *   n_tris          0 <= n_tris <= VAFR_NOALLOC_MAX_TRIS (larger: INVALID_ARG).
 *   codes_out       device, n_tris uint32, Morton codes in input order (the
 *                   same values vafr_scene_export_lbvh reports).
 *   sorted_ids_out  device, n_tris int32, triangle ids sorted by (code, id).
 *   err, err_len    optional host buffer for a message (NULL allowed).
 * The three buffers must not share any byte (INVALID_ARG otherwise: the
 * sort reads keys while it writes ids).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept per device and context: after cudaDeviceReset the
 * next call looks it up again, so it too should come before any capture.
 * Every call shares the one array: calls that overlap on the GPU (other
 * streams, other threads) race and corrupt each other's results; serialise
 * them.  No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: INVALID_ARG (size, NULL, non-device or overlapping pointers), CUDA. */
#define VAFR_NOALLOC_MAX_TRIS 524288
VAFR_API int vafr_morton_sort_noalloc(const float* tri_xyz, int64_t n_tris, uint32_t* codes_out,
                                      int32_t* sorted_ids_out, void* stream, char* err,
                                      int32_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* VAFR_H */
