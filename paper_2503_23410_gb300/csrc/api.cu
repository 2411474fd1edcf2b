// api.cu -- the C ABI of libvafr.so (declared in include/vafr.h): object
// lifetimes, argument checking, the FP64 host set-up of the log-polar layout
// (Sec. 3.2.2, Eqs. 9, 10, 12) and of each frame's gaze parameters (Eq. 3),
// batching, CUDA-graph capture and the tile-shape autotuner.
#include "layout.h"
#include "vafr_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits.h>
#include <memory>
#include <new>
#include <string>
#include <vector>

using namespace vafr;

namespace vafr {
static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace vafr

namespace {

// the calling thread's last failure, formatted in place (no allocation, so
// reporting an out-of-memory failure cannot fail itself)
thread_local char g_msg[512];

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

// Host-allocation fault injection (vafr_debug_fail_host_alloc): the batch
// entry points call host_alloc_point() before each host allocation they make;
// the countdown-th call throws std::bad_alloc, exactly as a failed allocation
// would.  Per thread, off (-1) unless a test arms it.
thread_local int g_alloc_countdown = -1;

void host_alloc_point() {
    if (g_alloc_countdown < 0) return;
    if (g_alloc_countdown-- == 0) throw std::bad_alloc();
}

// Entry points that allocate host memory run their body through this, so a
// failed host allocation returns VAFR_ERR_OOM and no C++ exception leaves the
// library.  Their bodies change caller-visible state only after the last step
// that can throw, so a failed call leaves every object as it was.
template <class F>
int guarded(F&& body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return fail(VAFR_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(VAFR_ERR_CUDA, "unexpected host-side exception");
    }
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? VAFR_ERR_OOM : VAFR_ERR_CUDA,  \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Two timing events destroyed on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int check_device(int* sms) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp p;
    CUDA_TRY(cudaGetDeviceProperties(&p, dev));
    if (!(p.major == 10 && p.minor == 3))
        return fail(VAFR_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a",
                    dev, p.major, p.minor);
    if (sms) *sms = p.multiProcessorCount;
    return VAFR_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int bytes_per_px(int fmt) { return fmt == VAFR_FMT_RGBA16F ? 8 : 16; }

}  // namespace

// ---- objects ----------------------------------------------------------------------
struct vafr_scene {
    int device = 0;
    int sms = 0;
    int64_t n = 0;
    std::vector<void*> allocs;
    int64_t bytes = 0;
    LbvhBuffers buf{};
    SceneDev dev{};
    unsigned* status = nullptr;
    int n_nodes4 = 0;              // 4-wide nodes of the traversal tree
    bool injected = false;         // vafr_scene_inject_fault: root references and keys saved
    int4 root_refs{}, root_keys{};
    float4* d_plights = nullptr;   // point lights (vafr_scene_set_point_lights)
    // deferred path scratch (first use): triangle id -> leaf, large-triangle list
    int* d_leaf_of = nullptr;
    int4* d_big = nullptr;
    int* d_big_leaf = nullptr;
    long long* d_big_first = nullptr;
    unsigned long long* d_n_big = nullptr;

    template <class T>
    int alloc(T** p, size_t count) {
        const size_t b = sizeof(T) * (count ? count : 1);
        void* q = nullptr;
        allocs.reserve(allocs.size() + 1);   // may throw; the push_back below cannot
        CUDA_TRY(cudaMalloc(&q, b));
        allocs.push_back(q);
        bytes += (int64_t)b;
        *p = reinterpret_cast<T*>(q);
        return VAFR_OK;
    }
    ~vafr_scene() {
        for (void* p : allocs) cudaFree(p);
    }
};

struct vafr_session {
    int device = 0;
    int sms = 0;
    vafr_session_desc desc{};
    std::shared_ptr<const LayoutTables> lay;   // shared by sessions with the same acuity
    int n_cols = 0;
    int64_t n_texels = 0;   // rays per eye
    int64_t n_slots = 0;    // LP buffer texels per eye (texels + 2 guard slots per column)
    unsigned* d_status = nullptr;
    unsigned long long* d_counter = nullptr;
    unsigned long long* d_stats = nullptr;
    bool gaze_set[2] = {false, false};
    FrameDesc fd[2]{};
    void* lp_internal = nullptr;       // render_frame's LP buffer
    void* lp_aa_internal = nullptr;    // render_frame's FXAA output
    float* d_luma = nullptr;           // FXAA scratch: [n_eyes][n_slots] lumas
    // VaFR_Rep scratch (first use): left depth, warped vertices, right z-buffer, holes
    float* d_rep_depth = nullptr;
    float4* d_rep_vert = nullptr;
    unsigned long long* d_rep_zbuf = nullptr;
    int2* d_rep_holes = nullptr;
    unsigned* d_rep_count = nullptr;
    void* disp_internal = nullptr;     // render_frame's device display for host output
    int recon_variant = 0;
    int render_variant = 0;
    LptState* d_lpt[2] = {nullptr, nullptr};   // longest-first order state per eye
    unsigned lpt_frames[2] = {0u, 0u};          // frames rendered with it (parity)

    ~vafr_session() {
        cudaFree(d_lpt[0]);
        cudaFree(d_lpt[1]);
        cudaFree(d_status);
        cudaFree(d_counter);
        cudaFree(d_stats);
        cudaFree(lp_internal);
        cudaFree(lp_aa_internal);
        cudaFree(d_luma);
        cudaFree(d_rep_depth);
        cudaFree(d_rep_vert);
        cudaFree(d_rep_zbuf);
        cudaFree(d_rep_holes);
        cudaFree(d_rep_count);
        cudaFree(disp_internal);
    }
};

struct vafr_batch {
    const vafr_scene* scene = nullptr;
    int max_frames = 0;
    int render_variant = 0;
    int recon_variant = 0;
    unsigned long long* d_counter = nullptr;
    // captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // kernel nodes in launch order: render (scene + batch), then the FXAA pass
    // if any and reconstruct (batch only)
    std::vector<cudaGraphNode_t> kernel_nodes;
    std::vector<cudaKernelNodeParams> kernel_params;
    std::vector<vafr_frame_desc> captured;
    BigBatch* host_batch = nullptr;  // parameters of the captured launches
    // longest-first order state per frame slot (the batch's own, so batches in
    // flight on different streams never share one)
    struct LptSlot {
        LptState* state;
        int cap;           // chunks the state holds
        unsigned frames;   // frames rendered with it (parity)
    };
    std::vector<LptSlot> lpt;
    // displays in page-locked host memory: the reconstruction writes a device
    // staging buffer per frame position, which the copy engine then moves to
    // the host (faster over the CPU-GPU link than the kernel's own stores)
    struct HostCopy {
        void* dst;
        const void* src;
        size_t bytes;
    };
    struct StageSlot {
        void* buf;
        size_t cap;
    };
    std::vector<StageSlot> stage;
    std::vector<HostCopy> copies;   // of the last built batch

    ~vafr_batch() {
        for (const LptSlot& q : lpt) cudaFree(q.state);
        for (const StageSlot& q : stage) cudaFree(q.buf);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_counter);
        delete host_batch;
    }
};

namespace {

// One device block: the LptState, then hot[2] and flag[2] for `chunks` chunks.
cudaError_t lpt_alloc(LptState** out, int chunks) {
    *out = nullptr;
    const size_t head = (sizeof(LptState) + 255) & ~(size_t)255;
    const size_t arr = (size_t)chunks * sizeof(int);
    char* q = nullptr;
    cudaError_t e = cudaMalloc(&q, head + 2 * arr + 2 * (size_t)chunks);
    if (e != cudaSuccess) return e;
    LptState h{};
    h.hot[0] = reinterpret_cast<int*>(q + head);
    h.hot[1] = reinterpret_cast<int*>(q + head + arr);
    h.flag[0] = reinterpret_cast<unsigned char*>(q + head + 2 * arr);
    h.flag[1] = reinterpret_cast<unsigned char*>(q + head + 2 * arr + chunks);
    h.capacity = chunks;
    e = cudaMemcpy(q, &h, sizeof(h), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(q); return e; }
    *out = reinterpret_cast<LptState*>(q);
    return cudaSuccess;
}

// The state pointer for the next frame of `st` (frame parity in bit 0), after
// clearing the counters of the half that frame collects into.
cudaError_t lpt_next(LptState* st, unsigned& frames, cudaStream_t s, LptState** tagged) {
    const int p = (int)(frames & 1u);
    cudaError_t e = cudaMemsetAsync(&st->ctr[p ^ 1], 0, sizeof(LptCounters), s);
    if (e != cudaSuccess) return e;
    ++frames;
    *tagged = reinterpret_cast<LptState*>(reinterpret_cast<uintptr_t>(st) | (uintptr_t)p);
    return cudaSuccess;
}

int lpt_chunks(int64_t n_texels) { return (int)((n_texels + kLptChunk - 1) / kLptChunk); }

// FP64 per-frame set-up of one eye (Eq. 3): c_r, gaze offsets, gaze split.
void setup_gaze(vafr_session* s, int eye, double x0, double y0) {
    const vafr_session_desc& d = s->desc;
    const double cr = 2.0 * std::tan(0.5 * d.fov_v_deg * M_PI / 180.0) / d.height;
    FrameDesc& f = s->fd[eye];
    f.gx = (float)(cr * (x0 - 0.5 * d.width));
    f.gy = (float)(cr * (0.5 * d.height - y0));
    const double fx = std::floor(x0), fy = std::floor(y0);
    f.gxi = (int)fx;
    f.gyi = (int)fy;
    f.gxf = (float)(0.5 - (x0 - fx));
    f.gyf = (float)(0.5 - (y0 - fy));
    s->gaze_set[eye] = true;
}

void fill_static(vafr_session* s, int eye) {
    const vafr_session_desc& d = s->desc;
    FrameDesc& f = s->fd[eye];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) f.R[3 * r + c] = (float)d.eye_pose[eye][4 * r + c];
        f.org[r] = (float)d.eye_pose[eye][4 * r + 3];
    }
    const double cr = 2.0 * std::tan(0.5 * d.fov_v_deg * M_PI / 180.0) / d.height;
    f.cr = (float)cr;
    f.px0 = (float)(cr * (0.5 - 0.5 * d.width));
    f.py0 = (float)(cr * (0.5 * d.height - 0.5));
    f.W = d.width;
    f.H = d.height;
    f.lp_fmt = d.lp_format;
    f.disp_fmt = d.display_format;
    const LayoutTables& L = *s->lay;
    f.tan_e = L.d_tan_e;
    f.col = L.d_col;
    f.col_pair = L.d_col_pair + 1;   // valid for c = -1 .. C - 1
    f.u_tab = L.d_u_tab;
    f.work = L.d_work;
    f.u_n = kUTable;
    f.u_inv_h = (float)L.u_inv_h;
    f.n_cols = s->n_cols;
    f.n_texels = (int)s->n_texels;
    f.status = s->d_status;
    f.lp = nullptr;
    f.lp_aa = nullptr;
    f.luma = nullptr;
    f.depth = nullptr;
    f.disp = nullptr;
    f.hit_ids = nullptr;
    f.lpt = nullptr;   // set per render (frame parity) when the longest-first order is used
}

long long recon_tiles(const FrameDesc& f, int variant) {
    const ReconShape sh = recon_shape(variant);
    return (long long)((f.W + sh.tw - 1) / sh.tw) * ((f.H + sh.th - 1) / sh.th);
}

long long gt_items(const FrameDesc& f) {
    return (long long)((f.W + 7) / 8) * ((f.H + 3) / 4) * 32;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// =====================================================================================
extern "C" {

const char* vafr_error_string(int code) {
    switch (code) {
        case VAFR_OK: return "ok";
        case VAFR_ERR_INVALID_ARG: return "invalid argument";
        case VAFR_ERR_OOM: return "out of memory";
        case VAFR_ERR_CUDA: return "CUDA error";
        case VAFR_ERR_TIMEOUT: return "device watchdog fired";
        case VAFR_ERR_BUDGET: return "memory budget exceeded";
        case VAFR_ERR_DEVICE: return "device fault reported";
        case VAFR_ERR_UNSUPPORTED: return "unsupported device";
        default: return "unknown error";
    }
}

const char* vafr_last_error_message(void) { return g_msg; }

int32_t vafr_version(void) { return 10000; }

int64_t vafr_kernel_launch_count(void) { return g_launches.load(); }

void vafr_acuity_default(vafr_acuity* a) {
    if (!a) return;
    std::memset(a, 0, sizeof(*a));
    const double E[5] = {0, 10, 20, 30, 60}, f[5] = {40, 10, 6, 5, 4};
    a->n_pivots = 5;
    for (int k = 0; k < 5; ++k) {
        a->pivot_ecc_deg[k] = E[k];
        a->pivot_cpd[k] = f[k];
        a->pivot_delta[k] = 1.0;
    }
    a->e_max_deg = 60.0;
}

void vafr_acuity_anisotropic(vafr_acuity* a) {
    if (!a) return;
    vafr_acuity_default(a);
    const double d[5] = {1.0, 5.0 / 6.0, 2.0 / 3.0, 0.5, 0.5};
    for (int k = 0; k < 5; ++k) a->pivot_delta[k] = d[k];
    a->anisotropic = 1;
}

int vafr_acuity_display_limited(vafr_acuity* a, double max_cpd) {
    if (!a || !(max_cpd > 0.0) || !std::isfinite(max_cpd))
        return fail(VAFR_ERR_INVALID_ARG, "max_cpd must be finite and > 0");
    vafr_acuity_default(a);
    for (int k = 0; k < a->n_pivots; ++k) a->pivot_cpd[k] = std::min(a->pivot_cpd[k], max_cpd);
    return VAFR_OK;
}

// ---- scene ---------------------------------------------------------------------------
static int vafr_build_scene_impl(const float* tri_xyz, const float* albedo_rgb, int64_t n_tris,
                     const float light_dir[3], void* stream, vafr_scene** out) {
    if (!out) return fail(VAFR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_tris < 0 || n_tris >= (1ll << 30)) return fail(VAFR_ERR_INVALID_ARG, "n_tris out of range");
    if (n_tris > 0 && !tri_xyz) return fail(VAFR_ERR_INVALID_ARG, "tri_xyz is NULL");
    if (!light_dir) return fail(VAFR_ERR_INVALID_ARG, "light_dir is NULL");
    const double ll = std::sqrt((double)light_dir[0] * light_dir[0] + (double)light_dir[1] * light_dir[1] +
                                (double)light_dir[2] * light_dir[2]);
    if (!std::isfinite(ll) || !(ll > 0.0)) return fail(VAFR_ERR_INVALID_ARG, "light_dir not finite/non-zero");
    int sms = 0;
    int rc = check_device(&sms);
    if (rc) return rc;
    cudaStream_t s = as_stream(stream);
    std::unique_ptr<vafr_scene> sc(new vafr_scene());
    cudaGetDevice(&sc->device);
    sc->sms = sms;
    sc->n = n_tris;
    const int n = (int)n_tris;
    LbvhBuffers& b = sc->buf;
    b.n = n;
    float* tris = nullptr;
    float* alb = nullptr;
    const size_t nb = lbvh_sort_blocks(n);
#define ALLOC(p, c)                              \
    do {                                         \
        int r_ = sc->alloc(&(p), (size_t)(c));   \
        if (r_) return r_;                       \
    } while (0)
    ALLOC(sc->status, 1);
    if (n > 0) {
        ALLOC(tris, 9ll * n);
        if (albedo_rgb) ALLOC(alb, 3ll * n);
        ALLOC(b.codes, n);
        ALLOC(b.keys_tmp, n);
        ALLOC(b.ids, n);
        ALLOC(b.ids_tmp, n);
        ALLOC(b.keys_sorted, n);
        ALLOC(b.hist, 256 * nb);
        ALLOC(b.part_bounds, 6 * 304);
        ALLOC(b.scene_bounds, 6);
        ALLOC(b.child, n > 1 ? n - 1 : 1);
        ALLOC(b.parent, 2ll * n);
        ALLOC(b.flags, n > 1 ? n - 1 : 1);
        ALLOC(b.node_box, 6ll * (n > 1 ? n - 1 : 1));
        ALLOC(b.leaf_box, 6ll * n);
        ALLOC(b.nodes, 4ll * (n > 1 ? n - 1 : 1));
        ALLOC(b.head_flag, n > 1 ? n - 1 : 1);
        ALLOC(b.head_idx, n > 1 ? n - 1 : 1);
        ALLOC(b.leaves, 3ll * n);
        ALLOC(b.albedo4, n);
    }
#undef ALLOC
    auto bail = [&](int code) { return code; };   // sc frees everything it holds
    if (cudaMemsetAsync(sc->status, 0, sizeof(unsigned), s) != cudaSuccess)
        return bail(fail(VAFR_ERR_CUDA, "memset status"));
    if (n > 0) {
        const cudaMemcpyKind k1 = is_device_ptr(tri_xyz) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaError_t e = cudaMemcpyAsync(tris, tri_xyz, sizeof(float) * 9ull * n, k1, s);
        if (e == cudaSuccess && albedo_rgb) {
            const cudaMemcpyKind k2 = is_device_ptr(albedo_rgb) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            e = cudaMemcpyAsync(alb, albedo_rgb, sizeof(float) * 3ull * n, k2, s);
        }
        if (e != cudaSuccess) return bail(fail(VAFR_ERR_CUDA, "input copy: %s", cudaGetErrorString(e)));
        b.tris = tris;
        b.albedo = alb;
        e = lbvh_build(b, s);
        if (e != cudaSuccess) return bail(fail(VAFR_ERR_CUDA, "lbvh build: %s", cudaGetErrorString(e)));
        if (n > 1) {
            struct Scratch {   // freed on every way out, a thrown bad_alloc included
                void* p = nullptr;
                ~Scratch() { if (p) cudaFree(p); }
            } scratch;
            e = cudaMalloc(&scratch.p, tree4_scratch_bytes(n));
            if (e != cudaSuccess) return bail(fail(VAFR_ERR_OOM, "traversal tree scratch"));
            e = tree4_build(b, scratch.p, kPlocRadius, s, &sc->n_nodes4);
            if (e != cudaSuccess)
                return bail(fail(VAFR_ERR_CUDA, "traversal tree build: %s", cudaGetErrorString(e)));
            const int r4 = sc->alloc(&b.nodes4, 16ll * sc->n_nodes4);
            if (r4) return r4;
            e = tree4_pack(b, scratch.p, sc->n_nodes4, s);
            if (e != cudaSuccess)
                return bail(fail(VAFR_ERR_CUDA, "traversal tree build: %s", cudaGetErrorString(e)));
        }
    }
    SceneDev& d = sc->dev;
    d.nodes = b.nodes;
    d.nodes4 = b.nodes4;
    d.n_nodes4 = sc->n_nodes4;
    d.leaves = b.leaves;
    d.albedo = b.albedo4;
    d.n_tris = n;
    d.root = n == 0 ? INT_MIN : (n == 1 ? ~0 : 0);
    for (int k = 0; k < 3; ++k) d.light[k] = (float)(light_dir[k] / ll);
    d.status = sc->status;
    *out = sc.release();
    return VAFR_OK;
}

int vafr_build_scene(const float* tri_xyz, const float* albedo_rgb, int64_t n_tris,
                     const float light_dir[3], void* stream, vafr_scene** out) {
    return guarded([&] { return vafr_build_scene_impl(tri_xyz, albedo_rgb, n_tris, light_dir, stream, out); });
}

static int vafr_scene_set_point_lights_impl(vafr_scene* scene, int32_t n, const float* pos_xyz, const float* rgb) {
    if (!scene) return fail(VAFR_ERR_INVALID_ARG, "scene is NULL");
    if (n < 0 || n > VAFR_MAX_POINT_LIGHTS || (n > 0 && (!pos_xyz || !rgb)))
        return fail(VAFR_ERR_INVALID_ARG, "point light count %d out of [0, %d] or NULL arrays", n, VAFR_MAX_POINT_LIGHTS);
    std::vector<float4> h(2 * (size_t)(n > 0 ? n : 1));
    for (int q = 0; q < n; ++q) {
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(pos_xyz[3 * q + k]) || !std::isfinite(rgb[3 * q + k]) || rgb[3 * q + k] < 0.0f)
                return fail(VAFR_ERR_INVALID_ARG, "point light %d: non-finite position or negative colour", q);
        h[2 * q] = make_float4(pos_xyz[3 * q], pos_xyz[3 * q + 1], pos_xyz[3 * q + 2], 0.0f);
        h[2 * q + 1] = make_float4(rgb[3 * q], rgb[3 * q + 1], rgb[3 * q + 2], 0.0f);
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(scene->device);
    int rc = VAFR_OK;
    if (!scene->d_plights) {
        if (scene->alloc(&scene->d_plights, 2 * VAFR_MAX_POINT_LIGHTS) != VAFR_OK) rc = VAFR_ERR_OOM;
    }
    if (!rc && n > 0 &&
        cudaMemcpy(scene->d_plights, h.data(), sizeof(float4) * 2 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(VAFR_ERR_CUDA, "point lights upload failed");
    if (!rc) {
        scene->dev.plights = scene->d_plights;
        scene->dev.n_plights = n;
    }
    cudaSetDevice(cur);
    return rc;
}

int vafr_scene_set_point_lights(vafr_scene* scene, int32_t n, const float* pos_xyz, const float* rgb) {
    return guarded([&] { return vafr_scene_set_point_lights_impl(scene, n, pos_xyz, rgb); });
}

int vafr_scene_destroy(vafr_scene* scene) {
    if (!scene) return VAFR_OK;
    cudaDeviceSynchronize();
    delete scene;
    return VAFR_OK;
}

int vafr_scene_info(const vafr_scene* scene, int64_t* n_tris, int64_t* device_bytes) {
    if (!scene) return fail(VAFR_ERR_INVALID_ARG, "scene is NULL");
    if (n_tris) *n_tris = scene->n;
    if (device_bytes) *device_bytes = scene->bytes;
    return VAFR_OK;
}

int vafr_scene_export_lbvh(const vafr_scene* scene, uint32_t* codes, int32_t* sorted_ids,
                           int32_t* child, float* node_box, float* leaf_box) {
    if (!scene) return fail(VAFR_ERR_INVALID_ARG, "scene is NULL");
    const int64_t n = scene->n;
    CUDA_TRY(cudaDeviceSynchronize());
    if (n == 0) return VAFR_OK;
    const LbvhBuffers& b = scene->buf;
    if (codes) CUDA_TRY(cudaMemcpy(codes, b.codes, 4ull * n, cudaMemcpyDeviceToHost));
    if (sorted_ids) CUDA_TRY(cudaMemcpy(sorted_ids, b.ids, 4ull * n, cudaMemcpyDeviceToHost));
    if (n > 1 && child) CUDA_TRY(cudaMemcpy(child, b.child, 8ull * (n - 1), cudaMemcpyDeviceToHost));
    if (n > 1 && node_box) CUDA_TRY(cudaMemcpy(node_box, b.node_box, 24ull * (n - 1), cudaMemcpyDeviceToHost));
    if (leaf_box) CUDA_TRY(cudaMemcpy(leaf_box, b.leaf_box, 24ull * n, cudaMemcpyDeviceToHost));
    return VAFR_OK;
}

int vafr_scene_export_tree4(const vafr_scene* scene, int64_t* n_nodes, float* nodes, float* leaves) {
    if (!scene || !n_nodes) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = scene->n;
    CUDA_TRY(cudaDeviceSynchronize());
    const int64_t n4 = n > 1 ? scene->n_nodes4 : 0;
    *n_nodes = n4;
    if (nodes && n4 > 0) {   // device nodes hold each axis as lo, hi, hi, lo: export lo, hi
        std::vector<float4> dev((size_t)n4 * 16);
        CUDA_TRY(cudaMemcpy(dev.data(), scene->buf.nodes4, 256ull * (size_t)n4, cudaMemcpyDeviceToHost));
        float4* o = reinterpret_cast<float4*>(nodes);
        for (int64_t j = 0; j < n4; ++j) {
            const float4* d = dev.data() + 16 * j;
            for (int a = 0; a < 3; ++a) {
                o[8 * j + 2 * a] = d[4 * a];
                o[8 * j + 2 * a + 1] = d[4 * a + 1];
            }
            o[8 * j + 6] = d[12];
            o[8 * j + 7] = d[13];
        }
    }
    if (leaves && n > 0)
        CUDA_TRY(cudaMemcpy(leaves, scene->buf.leaves, 48ull * (size_t)n, cudaMemcpyDeviceToHost));
    return VAFR_OK;
}

int vafr_scene_check(const vafr_scene* scene, void* stream) {
    if (!scene) return fail(VAFR_ERR_INVALID_ARG, "scene is NULL");
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    unsigned st = 0;
    CUDA_TRY(cudaMemcpy(&st, scene->status, sizeof(st), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(scene->status, 0, sizeof(unsigned)));
    if (st & kFaultWatchdog) return fail(VAFR_ERR_TIMEOUT, "scene status 0x%x", st);
    if (st) return fail(VAFR_ERR_DEVICE, "scene status 0x%x", st);
    return VAFR_OK;
}

int vafr_debug_fail_host_alloc(int32_t countdown) {
    if (countdown < -1) return fail(VAFR_ERR_INVALID_ARG, "countdown %d < -1", countdown);
    g_alloc_countdown = countdown;
    return VAFR_OK;
}

int vafr_scene_inject_fault(vafr_scene* scene, int32_t kind) {
    if (!scene) return fail(VAFR_ERR_INVALID_ARG, "scene is NULL");
    if (kind < VAFR_INJECT_NONE || kind > VAFR_INJECT_STACK) return fail(VAFR_ERR_INVALID_ARG, "unknown kind %d", kind);
    if (scene->n < 2) return fail(VAFR_ERR_INVALID_ARG, "a one-triangle scene has no tree");
    // the root is 4-wide node 0; its child references are the node's 7th float4
    // and its slot keys the 8th (slot q's internal child is reference 0 + key)
    int4* refs = reinterpret_cast<int4*>(scene->buf.nodes4 + 12);
    int4* keys = reinterpret_cast<int4*>(scene->buf.nodes4 + 13);
    CUDA_TRY(cudaDeviceSynchronize());
    if (!scene->injected) {
        if (kind == VAFR_INJECT_NONE) return VAFR_OK;
        CUDA_TRY(cudaMemcpy(&scene->root_refs, refs, sizeof(int4), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(&scene->root_keys, keys, sizeof(int4), cudaMemcpyDeviceToHost));
        scene->injected = true;
    }
    int4 v = scene->root_refs, w = scene->root_keys;
    int* c = &v.x;
    int* q = &w.x;
    const int bad = scene->n_nodes4;   // one past the last 4-wide node
    for (int k = 0; k < 4; ++k) {
        const bool used = c[k] != kEmptyRef;
        if (kind == VAFR_INJECT_BAD_CHILD && used) {   // every used slot an internal child out of range
            c[k] = bad;
            q[k] = k;
        }
        if (kind == VAFR_INJECT_LOOP) {   // the root's only child is the root
            c[k] = k == 0 ? 0 : kEmptyRef;
            q[k] = k == 0 ? 0 : -1;
        }
        if (kind == VAFR_INJECT_STACK && used) {   // every used slot leads back to the root
            c[k] = 0;
            q[k] = 0;
        }
    }
    CUDA_TRY(cudaMemcpy(refs, &v, sizeof(int4), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(keys, &w, sizeof(int4), cudaMemcpyHostToDevice));
    if (kind == VAFR_INJECT_NONE) scene->injected = false;
    return VAFR_OK;
}

// ---- session -------------------------------------------------------------------------
static int vafr_session_create_impl(const vafr_session_desc* desc, vafr_session** out) {
    if (!desc || !out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const vafr_session_desc& d = *desc;
    if (d.width <= 0 || d.height <= 0 || d.width > 32768 || d.height > 32768)
        return fail(VAFR_ERR_INVALID_ARG, "display size %dx%d out of range", d.width, d.height);
    if (!(d.fov_v_deg > 0.0 && d.fov_v_deg < 170.0)) return fail(VAFR_ERR_INVALID_ARG, "fov out of range");
    if (d.n_eyes != 1 && d.n_eyes != 2) return fail(VAFR_ERR_INVALID_ARG, "n_eyes must be 1 or 2");
    if ((d.lp_format != VAFR_FMT_RGBA32F && d.lp_format != VAFR_FMT_RGBA16F) ||
        (d.display_format != VAFR_FMT_RGBA32F && d.display_format != VAFR_FMT_RGBA16F))
        return fail(VAFR_ERR_INVALID_ARG, "unknown format");
    for (int e = 0; e < d.n_eyes; ++e)
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(d.eye_pose[e][k])) return fail(VAFR_ERR_INVALID_ARG, "pose not finite");
    int sms = 0;
    int rc = check_device(&sms);
    if (rc) return rc;
    std::shared_ptr<const LayoutTables> lay;
    std::string why;
    rc = get_layout(d.acuity, &lay, &why);
    if (rc) return fail(rc, "%s", why.c_str());
    std::unique_ptr<vafr_session> s(new vafr_session());
    cudaGetDevice(&s->device);
    s->sms = sms;
    s->desc = d;
    s->lay = lay;
    s->n_cols = lay->n_cols;
    s->n_texels = lay->n_texels;
    s->n_slots = lay->n_slots;
    auto bail = [&](cudaError_t e) {   // s frees what it holds
        return fail(e == cudaErrorMemoryAllocation ? VAFR_ERR_OOM : VAFR_ERR_CUDA, "session: %s",
                    cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&s->d_status, sizeof(unsigned))) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&s->d_counter, 2 * sizeof(unsigned long long))) != cudaSuccess) return bail(e);
    for (int eye = 0; eye < d.n_eyes; ++eye)
        if ((e = lpt_alloc(&s->d_lpt[eye], lpt_chunks(s->n_texels))) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&s->d_stats, 6 * sizeof(unsigned long long))) != cudaSuccess) return bail(e);
    if ((e = cudaMemset(s->d_status, 0, sizeof(unsigned))) != cudaSuccess) return bail(e);
    if (d.lp_fxaa && (e = cudaMalloc(&s->d_luma, sizeof(float) * s->n_slots * d.n_eyes)) != cudaSuccess)
        return bail(e);
    for (int eye = 0; eye < d.n_eyes; ++eye) fill_static(s.get(), eye);
    *out = s.release();
    return VAFR_OK;
}

int vafr_session_create(const vafr_session_desc* desc, vafr_session** out) {
    return guarded([&] { return vafr_session_create_impl(desc, out); });
}

int vafr_session_destroy(vafr_session* session) {
    if (!session) return VAFR_OK;
    cudaDeviceSynchronize();
    delete session;
    return VAFR_OK;
}

int vafr_lp_layout(const vafr_session* s, int32_t* n_cols, int64_t* n_texels, int32_t* col_counts,
                   int64_t* col_offsets, float* col_ecc_deg) {
    if (!s) return fail(VAFR_ERR_INVALID_ARG, "session is NULL");
    if (n_cols) *n_cols = s->n_cols;
    if (n_texels) *n_texels = s->n_texels;
    const LayoutTables& L = *s->lay;
    for (int c = 0; c < s->n_cols; ++c) {
        if (col_counts) col_counts[c] = L.n_col[c];
        if (col_offsets) col_offsets[c] = L.off_col[c];
        if (col_ecc_deg) col_ecc_deg[c] = (float)L.e_col[c];
    }
    return VAFR_OK;
}

int vafr_session_sizes(const vafr_session* s, int64_t* lp_bytes, int64_t* disp_bytes) {
    if (!s) return fail(VAFR_ERR_INVALID_ARG, "session is NULL");
    if (lp_bytes) *lp_bytes = s->n_slots * bytes_per_px(s->desc.lp_format);
    if (disp_bytes) *disp_bytes = (int64_t)s->desc.width * s->desc.height * bytes_per_px(s->desc.display_format);
    return VAFR_OK;
}

int vafr_session_tuning(vafr_session* s, int32_t set, int32_t cfg[2]) {
    if (!s || !cfg) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (set) {
        if (cfg[0] < 0 || cfg[0] >= kNumRenderVariants || cfg[1] < 0 || cfg[1] >= kNumReconVariants)
            return fail(VAFR_ERR_INVALID_ARG, "variant out of range");
        s->render_variant = cfg[0];
        s->recon_variant = cfg[1];
    } else {
        cfg[0] = s->render_variant;
        cfg[1] = s->recon_variant;
    }
    return VAFR_OK;
}

int vafr_set_gaze(vafr_session* s, int32_t eye, double x0, double y0) {
    if (!s) return fail(VAFR_ERR_INVALID_ARG, "session is NULL");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (!std::isfinite(x0) || !std::isfinite(y0) || std::fabs(x0) > 1e7 || std::fabs(y0) > 1e7)
        return fail(VAFR_ERR_INVALID_ARG, "gaze must be finite and |gaze| <= 1e7");
    setup_gaze(s, eye, x0, y0);
    return VAFR_OK;
}

int vafr_session_check(vafr_session* s, void* stream) {
    if (!s) return fail(VAFR_ERR_INVALID_ARG, "session is NULL");
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    unsigned st = 0;
    CUDA_TRY(cudaMemcpy(&st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(s->d_status, 0, sizeof(unsigned)));
    if (st & kFaultWatchdog) return fail(VAFR_ERR_TIMEOUT, "session status 0x%x", st);
    if (st) return fail(VAFR_ERR_DEVICE, "session status 0x%x", st);
    return VAFR_OK;
}

// ---- hot path ---------------------------------------------------------------------------
int vafr_render_lp(const vafr_scene* scene, vafr_session* s, int32_t eye_mask, void* lp_out,
                   int32_t* hit_ids_out, void* stream) {
    if (!scene || !s || !lp_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    const int all = (1 << s->desc.n_eyes) - 1;
    if (eye_mask <= 0 || (eye_mask & ~all)) return fail(VAFR_ERR_INVALID_ARG, "bad eye_mask %d", eye_mask);
    if (!aligned(lp_out, 16) || !aligned(hit_ids_out, 4)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    SmallBatch b{};
    b.work_counter = s->d_counter;
    const int bpp = bytes_per_px(s->desc.lp_format);
    for (int eye = 0; eye < s->desc.n_eyes; ++eye) {
        if (!(eye_mask & (1 << eye))) continue;
        if (!s->gaze_set[eye]) return fail(VAFR_ERR_INVALID_ARG, "gaze of eye %d never set", eye);
        FrameDesc f = s->fd[eye];
        f.lp = static_cast<char*>(lp_out) + (size_t)b.n * s->n_slots * bpp;
        f.hit_ids = hit_ids_out ? hit_ids_out + (size_t)b.n * s->n_slots : nullptr;
        f.work_begin = b.total_work;
        if (is_lpt_variant(s->render_variant))
            CUDA_TRY(lpt_next(s->d_lpt[eye], s->lpt_frames[eye], as_stream(stream), &f.lpt));
        b.total_work += s->n_texels;
        b.d[b.n++] = f;
    }
    CUDA_TRY(launch_render_lp(scene->dev, b, s->render_variant, as_stream(stream), s->sms));
    return VAFR_OK;
}

int vafr_render_lp_pt(const vafr_scene* scene, vafr_session* s, int32_t eye_mask, void* lp_out,
                      uint64_t seed, int32_t max_diffuse, int32_t* path_sig_out, void* stream) {
    if (!scene || !s || !lp_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    const int all = (1 << s->desc.n_eyes) - 1;
    if (eye_mask <= 0 || (eye_mask & ~all)) return fail(VAFR_ERR_INVALID_ARG, "bad eye_mask %d", eye_mask);
    if (max_diffuse < 0 || max_diffuse > 15) return fail(VAFR_ERR_INVALID_ARG, "max_diffuse %d out of [0, 15]", max_diffuse);
    if (!aligned(lp_out, 16) || !aligned(path_sig_out, 4)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    SmallBatch b{};
    b.work_counter = s->d_counter;
    const int bpp = bytes_per_px(s->desc.lp_format);
    for (int eye = 0; eye < s->desc.n_eyes; ++eye) {
        if (!(eye_mask & (1 << eye))) continue;
        if (!s->gaze_set[eye]) return fail(VAFR_ERR_INVALID_ARG, "gaze of eye %d never set", eye);
        FrameDesc f = s->fd[eye];
        f.lp = static_cast<char*>(lp_out) + (size_t)b.n * s->n_slots * bpp;
        f.hit_ids = path_sig_out ? path_sig_out + (size_t)b.n * s->n_slots * (max_diffuse + 2) : nullptr;
        f.work_begin = b.total_work;
        b.total_work += s->n_texels;
        b.d[b.n++] = f;
    }
    CUDA_TRY(launch_path_lp(scene->dev, b, (unsigned long long)seed, max_diffuse, as_stream(stream), s->sms));
    return VAFR_OK;
}

// ---- VaFR_Rep ------------------------------------------------------------------------
static int rep_scratch(vafr_session* s) {
    if (s->d_rep_vert) return VAFR_OK;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rep_depth, sizeof(float) * s->n_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rep_vert, sizeof(float4) * s->n_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rep_zbuf, sizeof(unsigned long long) * s->n_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rep_holes, sizeof(int2) * s->n_texels);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rep_count, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaFree(s->d_rep_depth); cudaFree(s->d_rep_vert); cudaFree(s->d_rep_zbuf);
        cudaFree(s->d_rep_holes); cudaFree(s->d_rep_count);
        s->d_rep_depth = nullptr; s->d_rep_vert = nullptr; s->d_rep_zbuf = nullptr;
        s->d_rep_holes = nullptr; s->d_rep_count = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? VAFR_ERR_OOM : VAFR_ERR_CUDA, "reprojection scratch: %s",
                    cudaGetErrorString(e));
    }
    return VAFR_OK;
}

static int rep_check(vafr_session* s) {
    if (s->desc.n_eyes != 2) return fail(VAFR_ERR_INVALID_ARG, "reprojection needs a binocular session");
    if (!s->gaze_set[0] || !s->gaze_set[1]) return fail(VAFR_ERR_INVALID_ARG, "gaze of both eyes must be set");
    return rep_scratch(s);
}

int vafr_reproject_lp(vafr_session* s, const void* left_lp, const float* left_depth, void* right_lp_out,
                      int32_t* right_tri_out, void* stream) {
    if (!s || !left_lp || !left_depth || !right_lp_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (!aligned(left_lp, 16) || !aligned(right_lp_out, 16) || !aligned(left_depth, 4) || !aligned(right_tri_out, 4))
        return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (int rc = rep_check(s)) return rc;
    SmallBatch b{};
    b.d[0] = s->fd[0];
    b.d[0].lp = const_cast<void*>(left_lp);
    b.d[0].depth = const_cast<float*>(left_depth);
    b.d[1] = s->fd[1];
    b.d[1].lp = right_lp_out;
    b.n = 2;
    RepScratch r{s->d_rep_vert, s->d_rep_zbuf, s->d_rep_holes, s->d_rep_count, right_tri_out};
    CUDA_TRY(launch_reproject(b, r, as_stream(stream), s->sms));
    return VAFR_OK;
}

int vafr_render_lp_rep(const vafr_scene* scene, vafr_session* s, void* lp_out, int32_t* right_tri_out,
                       void* stream) {
    if (!scene || !s || !lp_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (!aligned(lp_out, 16)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (int rc = rep_check(s)) return rc;
    cudaStream_t st = as_stream(stream);
    const size_t eye_bytes = (size_t)s->n_slots * bytes_per_px(s->desc.lp_format);
    void* right = static_cast<char*>(lp_out) + eye_bytes;
    // 1. the left eye cast, with hit distances
    SmallBatch b{};
    b.work_counter = s->d_counter;
    b.d[0] = s->fd[0];
    b.d[0].lp = lp_out;
    b.d[0].depth = s->d_rep_depth;
    b.d[0].work_begin = 0;
    b.n = 1;
    b.total_work = s->n_texels;
    CUDA_TRY(launch_render_lp(scene->dev, b, s->render_variant, st, s->sms));
    // 2. warp into the right eye
    SmallBatch w{};
    w.d[0] = b.d[0];
    w.d[1] = s->fd[1];
    w.d[1].lp = right;
    w.n = 2;
    RepScratch r{s->d_rep_vert, s->d_rep_zbuf, s->d_rep_holes, s->d_rep_count, right_tri_out};
    CUDA_TRY(launch_reproject(w, r, st, s->sms));
    // 3. cast the right eye's holes
    SmallBatch h{};
    h.work_counter = s->d_counter;
    h.d[0] = s->fd[1];
    h.d[0].lp = right;
    h.d[0].work = s->d_rep_holes;
    h.n = 1;
    CUDA_TRY(launch_render_list(scene->dev, h, s->d_rep_count, st, s->sms));
    return VAFR_OK;
}

int vafr_rep_hole_count(vafr_session* s, int64_t* holes, void* stream) {
    if (!s || !holes) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (!s->d_rep_count) { *holes = 0; return VAFR_OK; }
    unsigned h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, s->d_rep_count, sizeof(h), cudaMemcpyDeviceToHost, as_stream(stream)));
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    *holes = h;
    return VAFR_OK;
}

// ---- deferred path -----------------------------------------------------------------
static int deferred_scratch(const vafr_scene* scene_c, cudaStream_t st) {
    auto* scene = const_cast<vafr_scene*>(scene_c);
    if (scene->d_leaf_of) return VAFR_OK;
    const size_t n = (size_t)(scene->n > 0 ? scene->n : 1);
    int rc = scene->alloc(&scene->d_leaf_of, n);
    if (!rc) rc = scene->alloc(&scene->d_big, n);
    if (!rc) rc = scene->alloc(&scene->d_big_leaf, n);
    if (!rc) rc = scene->alloc(&scene->d_big_first, n);
    if (!rc) rc = scene->alloc(&scene->d_n_big, 1);
    if (rc) return fail(VAFR_ERR_OOM, "deferred scratch");
    CUDA_TRY(launch_leaf_of(scene->dev, scene->d_leaf_of, st, scene->sms));
    return VAFR_OK;
}

static int render_vbuffer(const vafr_scene* scene, vafr_session* s, int32_t eye, uint64_t* vbuf_out, void* stream,
                          unsigned long long* stats) {
    if (!scene || !s || !vbuf_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (!aligned(vbuf_out, 8)) return fail(VAFR_ERR_INVALID_ARG, "vbuf must be 8-byte aligned");
    cudaStream_t st = as_stream(stream);
    if (int rc = deferred_scratch(scene, st)) return rc;
    SmallBatch b{};
    b.d[0] = s->fd[eye];
    b.n = 1;
    VbufScratch v{reinterpret_cast<unsigned long long*>(vbuf_out), scene->d_big, scene->d_big_leaf,
                  scene->d_big_first, scene->d_n_big, (unsigned)(scene->n > 0 ? scene->n : 1)};
    CUDA_TRY(launch_vbuffer(scene->dev, b, v, st, scene->sms, stats));
    return VAFR_OK;
}

int vafr_render_vbuffer(const vafr_scene* scene, vafr_session* s, int32_t eye, uint64_t* vbuf_out, void* stream) {
    return render_vbuffer(scene, s, eye, vbuf_out, stream, nullptr);
}

int vafr_vbuffer_stats(const vafr_scene* scene, vafr_session* s, int32_t eye, uint64_t* vbuf_out, int64_t out[4],
                       void* stream) {
    if (!s || !out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaMemsetAsync(s->d_stats, 0, 4 * sizeof(unsigned long long), st));
    if (int rc = render_vbuffer(scene, s, eye, vbuf_out, stream, s->d_stats)) return rc;
    unsigned long long h[4];
    CUDA_TRY(cudaMemcpyAsync(h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k) out[k] = (int64_t)h[k];
    return VAFR_OK;
}

static int shade_deferred(const vafr_scene* scene, vafr_session* s, int32_t eye, const uint64_t* vbuf, void* out,
                          bool full_res, void* stream) {
    if (!scene || !s || !vbuf || !out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (!aligned(vbuf, 8) || !aligned(out, 16)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be aligned");
    if (!full_res && !s->gaze_set[eye]) return fail(VAFR_ERR_INVALID_ARG, "gaze of eye %d never set", eye);
    cudaStream_t st = as_stream(stream);
    if (int rc = deferred_scratch(scene, st)) return rc;
    SmallBatch b{};
    b.d[0] = s->fd[eye];
    if (full_res) b.d[0].disp = out; else b.d[0].lp = out;
    b.n = 1;
    CUDA_TRY(launch_shade_vbuf(scene->dev, b, reinterpret_cast<const unsigned long long*>(vbuf), scene->d_leaf_of,
                               full_res, st, scene->sms));
    return VAFR_OK;
}

int vafr_shade_lp_deferred(const vafr_scene* scene, vafr_session* s, int32_t eye, const uint64_t* vbuf,
                           void* lp_out, void* stream) {
    return shade_deferred(scene, s, eye, vbuf, lp_out, false, stream);
}

int vafr_shade_full_deferred(const vafr_scene* scene, vafr_session* s, int32_t eye, const uint64_t* vbuf,
                             void* display_out, void* stream) {
    return shade_deferred(scene, s, eye, vbuf, display_out, true, stream);
}

int vafr_reconstruct(vafr_session* s, int32_t eye, const void* lp, void* display_out, void* stream) {
    if (!s || !lp || !display_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (!s->gaze_set[eye]) return fail(VAFR_ERR_INVALID_ARG, "gaze of eye %d never set", eye);
    if (!aligned(lp, 16) || !aligned(display_out, 16)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    SmallBatch b{};
    FrameDesc f = s->fd[eye];
    f.lp = const_cast<void*>(lp);
    f.lp_aa = nullptr;
    f.disp = display_out;
    f.tile_begin = 0;
    b.d[0] = f;
    b.n = 1;
    b.total_tiles = recon_tiles(f, s->recon_variant);
    CUDA_TRY(launch_reconstruct(b, s->recon_variant, as_stream(stream)));
    return VAFR_OK;
}

int vafr_fxaa_lp(vafr_session* s, int32_t eye, const void* lp, void* lp_out, void* stream) {
    if (!s || !lp || !lp_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (!aligned(lp, 16) || !aligned(lp_out, 16)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (lp == lp_out) return fail(VAFR_ERR_INVALID_ARG, "lp_out must not be lp");
    // luma scratch: allocated with the session when it has lp_fxaa, else on first use
    if (!s->d_luma) CUDA_TRY(cudaMalloc(&s->d_luma, sizeof(float) * s->n_slots * s->desc.n_eyes));
    SmallBatch b{};
    FrameDesc f = s->fd[eye];   // the layout tables only: no gaze needed
    f.lp = const_cast<void*>(lp);
    f.lp_aa = lp_out;
    f.luma = s->d_luma + (size_t)eye * s->n_slots;
    f.aa_begin = 0;
    b.d[0] = f;
    b.n = 1;
    b.total_aa = s->n_texels;
    CUDA_TRY(launch_fxaa(b, as_stream(stream), s->sms));
    return VAFR_OK;
}

int vafr_render_full_gt(const vafr_scene* scene, vafr_session* s, int32_t eye, void* display_out,
                        int32_t* hit_ids_out, void* stream) {
    if (!scene || !s || !display_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (!aligned(display_out, 16) || !aligned(hit_ids_out, 4)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    SmallBatch b{};
    b.work_counter = s->d_counter;
    FrameDesc f = s->fd[eye];   // GT needs no gaze: c_r and the pose only
    f.disp = display_out;
    f.hit_ids = hit_ids_out;
    f.work_begin = 0;
    b.d[0] = f;
    b.n = 1;
    b.total_work = gt_items(f);
    CUDA_TRY(launch_render_gt(scene->dev, b, s->render_variant, as_stream(stream), s->sms));
    return VAFR_OK;
}

int vafr_render_full_gt_pt(const vafr_scene* scene, vafr_session* s, int32_t eye, void* display_out,
                           uint64_t seed, int32_t max_diffuse, void* stream) {
    if (!scene || !s || !display_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "eye %d out of range", eye);
    if (max_diffuse < 0 || max_diffuse > 15) return fail(VAFR_ERR_INVALID_ARG, "max_diffuse %d out of [0, 15]", max_diffuse);
    if (!aligned(display_out, 16)) return fail(VAFR_ERR_INVALID_ARG, "display must be 16-byte aligned");
    SmallBatch b{};
    b.work_counter = s->d_counter;
    FrameDesc f = s->fd[eye];
    f.disp = display_out;
    f.hit_ids = nullptr;
    f.work_begin = 0;
    b.d[0] = f;
    b.n = 1;
    b.total_work = gt_items(f);
    CUDA_TRY(launch_path_gt(scene->dev, b, (unsigned long long)seed, max_diffuse, as_stream(stream), s->sms));
    return VAFR_OK;
}

int vafr_render_frame(const vafr_scene* scene, vafr_session* s, void* display_out, void* stream) {
    if (!scene || !s || !display_out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    const int eyes = s->desc.n_eyes;
    int64_t lpb = 0, dpb = 0;
    vafr_session_sizes(s, &lpb, &dpb);
    if (!s->lp_internal) CUDA_TRY(cudaMalloc(&s->lp_internal, (size_t)lpb * eyes));
    // Where the display goes: device memory as is; pinned (page-locked or
    // registered) host memory through its device alias, so the reconstruction
    // kernel writes it directly over the CPU-GPU link (for one synchronous
    // frame this beats a device display plus a copy, which cannot overlap);
    // pageable host memory through a device buffer and one device-to-host copy.
    cudaPointerAttributes pa;
    void* target = nullptr;
    bool copy_out = false;
    if (cudaPointerGetAttributes(&pa, display_out) != cudaSuccess) {
        cudaGetLastError();
        pa.type = cudaMemoryTypeUnregistered;
    }
    if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) {
        target = display_out;
    } else if (pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr) {
        target = pa.devicePointer;
    } else {
        if (!s->disp_internal) CUDA_TRY(cudaMalloc(&s->disp_internal, (size_t)dpb * eyes));
        target = s->disp_internal;
        copy_out = true;
    }
    if (!aligned(target, 16)) return fail(VAFR_ERR_INVALID_ARG, "display must be 16-byte aligned");
    int rc = vafr_render_lp(scene, s, (1 << eyes) - 1, s->lp_internal, nullptr, stream);
    if (rc) return rc;
    void* lp_final = s->lp_internal;
    if (s->desc.lp_fxaa) {
        if (!s->lp_aa_internal) CUDA_TRY(cudaMalloc(&s->lp_aa_internal, (size_t)lpb * eyes));
        for (int e = 0; e < eyes; ++e) {
            rc = vafr_fxaa_lp(s, e, static_cast<char*>(s->lp_internal) + (size_t)e * lpb,
                              static_cast<char*>(s->lp_aa_internal) + (size_t)e * lpb, stream);
            if (rc) return rc;
        }
        lp_final = s->lp_aa_internal;
    }
    for (int e = 0; e < eyes; ++e) {
        rc = vafr_reconstruct(s, e, static_cast<char*>(lp_final) + (size_t)e * lpb,
                              static_cast<char*>(target) + (size_t)e * dpb, stream);
        if (rc) return rc;
    }
    if (copy_out)
        CUDA_TRY(cudaMemcpyAsync(display_out, target, (size_t)dpb * eyes, cudaMemcpyDeviceToHost,
                                 as_stream(stream)));
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
        CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    return VAFR_OK;
}

int vafr_traversal_stats(const vafr_scene* scene, vafr_session* s, int32_t eye, int64_t out[6],
                         void* stream) {
    if (!scene || !s || !out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (eye < 0 || eye >= s->desc.n_eyes || !s->gaze_set[eye])
        return fail(VAFR_ERR_INVALID_ARG, "bad eye or gaze not set");
    SmallBatch b{};
    FrameDesc f = s->fd[eye];
    f.work_begin = 0;
    b.d[0] = f;
    b.n = 1;
    b.total_work = s->n_texels;
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(launch_render_stats(scene->dev, b, s->d_stats, st, s->sms));
    unsigned long long h[6];
    CUDA_TRY(cudaMemcpyAsync(h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < 6; ++k) out[k] = (int64_t)h[k];
    return VAFR_OK;
}

int vafr_measure_fp32_peak(double out[2], void* stream) {
    if (!out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    CUDA_TRY(cudaMalloc(&sink, sizeof(float) * (size_t)sms * 8));
    double ffma = 0.0, ffma2 = 0.0;
    const cudaError_t e = measure_fp32_peak(sms, sink, as_stream(stream), &ffma, &ffma2);
    cudaFree(sink);
    CUDA_TRY(e);
    out[0] = ffma;
    out[1] = ffma2;
    return VAFR_OK;
}

// ---- batching ----------------------------------------------------------------------------
// graph = true: for a captured graph, which replays fixed launches, so frames
// take no longest-first state (its frame parity alternates).
static int build_batch(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, BigBatch* b,
                       cudaStream_t st, bool graph) {
    if (!frames || n <= 0 || n > bt->max_frames)
        return fail(VAFR_ERR_INVALID_ARG, "frame count %d out of range (max %d)", n, bt->max_frames);
    std::memset(b, 0, sizeof(*b));
    b->work_counter = bt->d_counter;
    bt->copies.clear();
    for (int i = 0; i < n; ++i) {
        const vafr_frame_desc& fr = frames[i];
        vafr_session* s = fr.session;
        if (!s || !fr.lp || !fr.display) return fail(VAFR_ERR_INVALID_ARG, "frame %d: NULL session/buffer", i);
        if (fr.eye < 0 || fr.eye >= s->desc.n_eyes) return fail(VAFR_ERR_INVALID_ARG, "frame %d: bad eye", i);
        if (!s->gaze_set[fr.eye]) return fail(VAFR_ERR_INVALID_ARG, "frame %d: gaze never set", i);
        if (!aligned(fr.lp, 16) || !aligned(fr.display, 16)) return fail(VAFR_ERR_INVALID_ARG, "frame %d: unaligned buffer", i);
        FrameDesc f = s->fd[fr.eye];
        f.lp = fr.lp;
        f.lp_aa = nullptr;
        f.lpt = nullptr;
        if (is_lpt_variant(bt->render_variant) && !graph) {
            if ((int)bt->lpt.size() <= i) {
                host_alloc_point();
                bt->lpt.resize(i + 1, vafr_batch::LptSlot{nullptr, 0, 0u});   // all or nothing
            }
            vafr_batch::LptSlot& q = bt->lpt[i];
            const int need = lpt_chunks(s->n_texels);
            if (q.cap < need) {   // grows only (a state in use is never freed mid-flight)
                LptState* nq = nullptr;
                CUDA_TRY(lpt_alloc(&nq, need));
                cudaError_t e = cudaDeviceSynchronize();   // the old state may still be in use
                if (e != cudaSuccess) {
                    cudaFree(nq);
                    CUDA_TRY(e);
                }
                cudaFree(q.state);
                q = vafr_batch::LptSlot{nq, need, 0u};
            }
            CUDA_TRY(lpt_next(q.state, q.frames, st, &f.lpt));
        }
        if (s->desc.lp_fxaa) {
            if (!fr.lp_aa || !aligned(fr.lp_aa, 16) || fr.lp_aa == fr.lp)
                return fail(VAFR_ERR_INVALID_ARG, "frame %d: FXAA session needs a separate aligned lp_aa", i);
            f.lp_aa = fr.lp_aa;
            f.luma = s->d_luma + (size_t)fr.eye * s->n_slots;
        }
        f.disp = fr.display;
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, fr.display) != cudaSuccess) {
            cudaGetLastError();
            pa.type = cudaMemoryTypeUnregistered;
        }
        if (pa.type == cudaMemoryTypeUnregistered)
            return fail(VAFR_ERR_INVALID_ARG, "frame %d: display must be device or page-locked host memory", i);
        if (pa.type == cudaMemoryTypeHost) {
            int64_t lpb = 0, dpb = 0;
            vafr_session_sizes(s, &lpb, &dpb);
            if ((int)bt->stage.size() <= i) {
                host_alloc_point();
                bt->stage.resize(i + 1, vafr_batch::StageSlot{nullptr, 0});   // all or nothing
            }
            vafr_batch::StageSlot& q = bt->stage[i];
            if (q.cap < (size_t)dpb) {   // grows only
                void* nq = nullptr;
                CUDA_TRY(cudaMalloc(&nq, (size_t)dpb));
                cudaError_t e = cudaDeviceSynchronize();   // the old buffer may still be in use
                if (e != cudaSuccess) {
                    cudaFree(nq);
                    CUDA_TRY(e);
                }
                cudaFree(q.buf);
                q = vafr_batch::StageSlot{nq, (size_t)dpb};
            }
            f.disp = q.buf;
            host_alloc_point();
            bt->copies.push_back({fr.display, q.buf, (size_t)dpb});
        }
        f.hit_ids = nullptr;
        f.work_begin = b->total_work;
        f.tile_begin = b->total_tiles;
        f.aa_begin = b->total_aa;
        b->total_work += s->n_texels;
        b->total_tiles += recon_tiles(f, bt->recon_variant);
        if (f.lp_aa) b->total_aa += s->n_texels;
        b->d[i] = f;
    }
    b->n = n;
    return VAFR_OK;
}

static int launch_batch(vafr_batch* bt, const BigBatch& b, cudaStream_t st) {
    CUDA_TRY(launch_render_lp(bt->scene->dev, b, bt->render_variant, st, bt->scene->sms));
    CUDA_TRY(launch_fxaa(b, st, bt->scene->sms));
    CUDA_TRY(launch_reconstruct(b, bt->recon_variant, st));
    for (const auto& c : bt->copies)
        CUDA_TRY(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, st));
    return VAFR_OK;
}

static int vafr_batch_create_impl(const vafr_scene* scene, int32_t max_frames, vafr_batch** out) {
    if (!scene || !out) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (max_frames <= 0 || max_frames > VAFR_MAX_BATCH)
        return fail(VAFR_ERR_INVALID_ARG, "max_frames out of range");
    std::unique_ptr<vafr_batch> bt(new vafr_batch());
    bt->scene = scene;
    bt->max_frames = max_frames;
    if (cudaMalloc(&bt->d_counter, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(VAFR_ERR_OOM, "batch counter");
    host_alloc_point();
    bt->host_batch = new BigBatch();
    *out = bt.release();
    return VAFR_OK;
}

int vafr_batch_create(const vafr_scene* scene, int32_t max_frames, vafr_batch** out) {
    return guarded([&] { return vafr_batch_create_impl(scene, max_frames, out); });
}

int vafr_batch_destroy(vafr_batch* batch) {
    if (!batch) return VAFR_OK;
    cudaDeviceSynchronize();
    delete batch;
    return VAFR_OK;
}

static int vafr_batch_render_impl(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, void* stream) {
    if (!bt) return fail(VAFR_ERR_INVALID_ARG, "batch is NULL");
    host_alloc_point();
    std::unique_ptr<BigBatch> b(new BigBatch());
    int rc = build_batch(bt, frames, n, b.get(), as_stream(stream), false);
    if (!rc) rc = launch_batch(bt, *b, as_stream(stream));
    return rc;
}

int vafr_batch_render(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, void* stream) {
    return guarded([&] { return vafr_batch_render_impl(bt, frames, n, stream); });
}

// Owner of a graph and its executable while a capture is being built; the
// batch takes them over only when every step has succeeded.
struct GraphParts {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~GraphParts() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

static int vafr_batch_capture_impl(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, void* stream) {
    if (!bt) return fail(VAFR_ERR_INVALID_ARG, "batch is NULL");
    // everything is built in locals first: a failure at any step (including a
    // host allocation) leaves the batch's previous graph, parameters and
    // captured frames as they were, still consistent with one another
    host_alloc_point();
    std::unique_ptr<BigBatch> hb(new BigBatch());
    // build_batch may replace a staging buffer the current graph copies from;
    // if this capture then fails, that graph must not be replayed any more
    host_alloc_point();
    std::vector<void*> old_stage;
    old_stage.reserve(bt->stage.size());
    for (const vafr_batch::StageSlot& q : bt->stage) old_stage.push_back(q.buf);
    struct StaleGraph {
        vafr_batch* bt;
        const std::vector<void*>& old;
        bool committed = false;
        ~StaleGraph() {
            if (committed || !bt->exec) return;
            for (size_t i = 0; i < old.size(); ++i)
                if (i >= bt->stage.size() || bt->stage[i].buf != old[i]) {
                    cudaGraphExecDestroy(bt->exec);
                    bt->exec = nullptr;
                    return;
                }
        }
    } stale{bt, old_stage};
    int rc = build_batch(bt, frames, n, hb.get(), as_stream(stream), true);
    if (rc) return rc;
    GraphParts gp;
    cudaStream_t cs = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = launch_batch(bt, *hb, cs);
        e = cudaStreamEndCapture(cs, &gp.graph);
    }
    cudaStreamDestroy(cs);
    if (rc) return rc;
    CUDA_TRY(e);
    CUDA_TRY(cudaGraphInstantiate(&gp.exec, gp.graph, 0));
    // the kernel nodes, ordered along the captured chain (memset -> render ->
    // [FXAA ->] reconstruct): a node's rank is its number of kernel ancestors
    size_t nn = 0;
    CUDA_TRY(cudaGraphGetNodes(gp.graph, nullptr, &nn));
    host_alloc_point();
    std::vector<cudaGraphNode_t> nodes(nn);
    CUDA_TRY(cudaGraphGetNodes(gp.graph, nodes.data(), &nn));
    auto kernel_ancestors = [&](cudaGraphNode_t nd, auto&& self) -> int {
        size_t ndep = 0;
        if (cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &ndep) != cudaSuccess) return -1;
        std::vector<cudaGraphNode_t> deps(ndep);
        if (ndep && cudaGraphNodeGetDependencies(nd, deps.data(), nullptr, &ndep) != cudaSuccess) return -1;
        int k = 0;
        for (cudaGraphNode_t dn : deps) {
            cudaGraphNodeType dt;
            if (cudaGraphNodeGetType(dn, &dt) != cudaSuccess) return -1;
            const int up = self(dn, self);
            if (up < 0) return -1;
            k = std::max(k, up + (dt == cudaGraphNodeTypeKernel ? 1 : 0));
        }
        return k;
    };
    std::vector<std::pair<int, cudaGraphNode_t>> ranked;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeKernel) continue;
        const int r = kernel_ancestors(nd, kernel_ancestors);
        if (r < 0) return fail(VAFR_ERR_CUDA, "graph: dependency query failed");
        host_alloc_point();
        ranked.push_back({r, nd});
    }
    std::sort(ranked.begin(), ranked.end(),
              [](const std::pair<int, cudaGraphNode_t>& a, const std::pair<int, cudaGraphNode_t>& b) {
                  return a.first < b.first;
              });
    std::vector<cudaGraphNode_t> knodes;
    std::vector<cudaKernelNodeParams> kparams;
    for (size_t k = 0; k < ranked.size(); ++k) {
        if (ranked[k].first != (int)k) return fail(VAFR_ERR_CUDA, "graph: kernel nodes are not a chain");
        cudaKernelNodeParams p{};
        CUDA_TRY(cudaGraphKernelNodeGetParams(ranked[k].second, &p));
        host_alloc_point();
        knodes.push_back(ranked[k].second);
        kparams.push_back(p);
    }
    if (knodes.size() < 2) return fail(VAFR_ERR_CUDA, "graph: kernel nodes not found");
    host_alloc_point();
    std::vector<vafr_frame_desc> cap(frames, frames + n);
    // commit: nothing below can fail
    stale.committed = true;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    bt->exec = gp.exec;
    bt->graph = gp.graph;
    gp.exec = nullptr;
    gp.graph = nullptr;
    *bt->host_batch = *hb;
    bt->kernel_nodes.swap(knodes);
    bt->kernel_params.swap(kparams);
    bt->captured.swap(cap);
    return VAFR_OK;
}

int vafr_batch_capture(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, void* stream) {
    return guarded([&] { return vafr_batch_capture_impl(bt, frames, n, stream); });
}

int vafr_batch_replay(vafr_batch* bt, void* stream) {
    if (!bt || !bt->exec) return fail(VAFR_ERR_INVALID_ARG, "batch has no captured graph");
    // refresh the per-frame gaze fields from the sessions (FP64 set-up already
    // done by vafr_set_gaze), keep everything else as captured
    BigBatch* b = bt->host_batch;
    for (int i = 0; i < b->n; ++i) {
        const vafr_frame_desc& fr = bt->captured[i];
        const FrameDesc& src = fr.session->fd[fr.eye];
        FrameDesc& f = b->d[i];
        f.gx = src.gx; f.gy = src.gy;
        f.gxi = src.gxi; f.gyi = src.gyi; f.gxf = src.gxf; f.gyf = src.gyf;
    }
    SceneDev sc = bt->scene->dev;
    void* rargs[2] = {&sc, b};
    void* bargs[1] = {b};
    for (size_t k = 0; k < bt->kernel_nodes.size(); ++k) {
        cudaKernelNodeParams p = bt->kernel_params[k];
        p.kernelParams = k == 0 ? rargs : bargs;   // render takes (scene, batch), the rest (batch)
        p.extra = nullptr;
        CUDA_TRY(cudaGraphExecKernelNodeSetParams(bt->exec, bt->kernel_nodes[k], &p));
    }
    CUDA_TRY(cudaGraphLaunch(bt->exec, as_stream(stream)));
    count_launch((int)bt->kernel_nodes.size());
    return VAFR_OK;
}

int vafr_tuning_space(int32_t* n_render, int32_t* n_reconstruct) {
    if (n_render) *n_render = kNumRenderVariants;
    if (n_reconstruct) *n_reconstruct = kNumReconVariants;
    return VAFR_OK;
}

int vafr_batch_tuning(vafr_batch* bt, int32_t set, int32_t cfg[2]) {
    if (!bt || !cfg) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (set) {
        if (cfg[0] < 0 || cfg[0] >= kNumRenderVariants || cfg[1] < 0 || cfg[1] >= kNumReconVariants)
            return fail(VAFR_ERR_INVALID_ARG, "variant out of range");
        bt->render_variant = cfg[0];
        bt->recon_variant = cfg[1];
    } else {
        cfg[0] = bt->render_variant;
        cfg[1] = bt->recon_variant;
    }
    return VAFR_OK;
}

int vafr_session_autotune(const vafr_scene* scene, vafr_session* s, void* lp, void* display, int32_t warm,
                          int32_t iters, int32_t cfg_out[2], void* stream) {
    if (!scene || !s || !lp || !display) return fail(VAFR_ERR_INVALID_ARG, "NULL argument");
    if (!aligned(lp, 16) || !aligned(display, 16)) return fail(VAFR_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    const int eyes = s->desc.n_eyes;
    for (int e = 0; e < eyes; ++e)
        if (!s->gaze_set[e]) return fail(VAFR_ERR_INVALID_ARG, "gaze of eye %d never set", e);
    if (warm < 0) warm = 0;
    if (iters <= 0) iters = 3;
    int64_t lpb = 0, dpb = 0;
    vafr_session_sizes(s, &lpb, &dpb);
    cudaStream_t st = as_stream(stream);
    auto frame = [&]() -> int {
        int rc = vafr_render_lp(scene, s, (1 << eyes) - 1, lp, nullptr, stream);
        for (int e = 0; e < eyes && !rc; ++e)
            rc = vafr_reconstruct(s, e, static_cast<char*>(lp) + (size_t)e * lpb,
                                  static_cast<char*>(display) + (size_t)e * dpb, stream);
        return rc;
    };
    EventPair ev;
    CUDA_TRY(cudaEventCreate(&ev.a));
    CUDA_TRY(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    int rc = VAFR_OK;
    const int keep_render = s->render_variant;
    auto time_frames = [&](float& ms) {
        for (int i = 0; i < warm && !rc; ++i) rc = frame();
        cudaEventRecord(e0, st);
        for (int i = 0; i < iters && !rc; ++i) rc = frame();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        ms = INFINITY;
        if (!rc) cudaEventElapsedTime(&ms, e0, e1);
    };
    const int keep_recon = s->recon_variant;
    float best = INFINITY;
    int best_r = s->render_variant;
    for (int v = 0; v < kNumRenderVariants && !rc; ++v) {
        s->render_variant = v;
        float ms;
        time_frames(ms);
        if (ms < best) { best = ms; best_r = v; }
    }
    s->render_variant = best_r;
    best = INFINITY;
    int best_c = keep_recon;
    for (int v = 0; v < kNumReconVariants && !rc; ++v) {
        s->recon_variant = v;
        float ms;
        time_frames(ms);
        if (ms < best) { best = ms; best_c = v; }
    }
    s->recon_variant = best_c;
    if (rc) {   // a failed tuning run leaves the session's variants as they were
        s->render_variant = keep_render;
        s->recon_variant = keep_recon;
        return rc;
    }
    if (cfg_out) { cfg_out[0] = best_r; cfg_out[1] = best_c; }
    return VAFR_OK;
}

static int vafr_batch_autotune_impl(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, void* stream,
                        int32_t iters) {
    if (!bt) return fail(VAFR_ERR_INVALID_ARG, "batch is NULL");
    if (iters <= 0) iters = 3;
    cudaStream_t st = as_stream(stream);
    EventPair ev;
    CUDA_TRY(cudaEventCreate(&ev.a));
    CUDA_TRY(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    host_alloc_point();
    std::unique_ptr<BigBatch> holder(new BigBatch());
    BigBatch* b = holder.get();
    int rc = VAFR_OK;
    // restores the batch's variants unless the tuning completes
    struct Restore {
        vafr_batch* bt;
        int render, recon;
        bool done = false;
        ~Restore() {
            if (!done) { bt->render_variant = render; bt->recon_variant = recon; }
        }
    } restore{bt, bt->render_variant, bt->recon_variant};
    auto time_it = [&](auto&& launch) -> float {
        if (launch() != cudaSuccess) return INFINITY;
        cudaEventRecord(e0, st);
        for (int i = 0; i < iters; ++i) launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    float best = INFINITY;
    int best_v = 0;
    const int keep_recon = bt->recon_variant;
    for (int v = 0; v < kNumRenderVariants && !rc; ++v) {
        rc = build_batch(bt, frames, n, b, st, true);
        if (rc) break;
        const float ms = time_it([&] { return launch_render_lp(bt->scene->dev, *b, v, st, bt->scene->sms); });
        if (ms < best) { best = ms; best_v = v; }
    }
    bt->render_variant = best_v;
    best = INFINITY;
    best_v = keep_recon;
    for (int v = 0; v < kNumReconVariants && !rc; ++v) {
        bt->recon_variant = v;
        rc = build_batch(bt, frames, n, b, st, true);
        if (rc) break;
        const float ms = time_it([&] { return launch_reconstruct(*b, v, st); });
        if (ms < best) { best = ms; best_v = v; }
    }
    bt->recon_variant = best_v;
    if (!rc) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(VAFR_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    restore.done = rc == VAFR_OK;
    return rc;
}

int vafr_batch_autotune(vafr_batch* bt, const vafr_frame_desc* frames, int32_t n, void* stream,
                        int32_t iters) {
    return guarded([&] { return vafr_batch_autotune_impl(bt, frames, n, stream, iters); });
}

}  // extern "C"
