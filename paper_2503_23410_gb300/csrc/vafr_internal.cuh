// vafr_internal.cuh -- device data layouts and launch interfaces shared by the
// CUDA translation units of libvafr.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/vafr.h"

namespace vafr {

// ---- device status words --------------------------------------------------
enum DeviceFault : unsigned {
    kFaultStack = 1u,     // traversal stack would overflow
    kFaultWatchdog = 2u,  // traversal iteration limit reached
    kFaultBadNode = 4u,   // child reference out of range
};

constexpr int kStackSize = 128;   // entries; a descent pushes at most 3 per 4-wide level above the last: depth <= 43
constexpr int kEmptyRef = (int)0x80000000;   // unused slot of a 4-wide node
constexpr int kMaxSeg = VAFR_MAX_PIVOTS - 1;

// ---- scene (LBVH) in traversal layout ----------------------------------------
// Internal node i (64 B, four float4), children L and R:
//   n[0] = (L.lo.x, R.lo.x, L.hi.x, R.hi.x)
//   n[1] = (L.lo.y, R.lo.y, L.hi.y, R.hi.y)
//   n[2] = (L.lo.z, R.lo.z, L.hi.z, R.hi.z)
//   n[3] = (L ref, R ref, -, -) as int bits; ref >= 0 internal, < 0 leaf ~k
// Leaf k (sorted order): three float4 (v0.xyz | id), (v1.xyz | 0), (v2.xyz | 0).
// 4-wide node j (256 B, sixteen float4): per axis the planes lo, hi, hi, lo of
// children 0..3 (so the (near, far) pair of either ray direction is one
// 32-byte aligned load), then their refs (>= 0 4-wide node, < 0 leaf ~k,
// kEmptyRef unused), then the slot keys (q for an internal child in slot q,
// all ones otherwise), then padding.  Internal children take the first slots
// and consecutive indices (slot q's node = slot 0's + q); leaves follow,
// unused slots last.  4-wide node 0 is the root.
struct SceneDev {
    const float4* nodes;
    const float4* nodes4;
    int n_nodes4;           // 4-wide nodes (the traversal's bound on a child index)
    const float4* leaves;
    const float4* albedo;   // original triangle order (rgb, 0)
    int root;               // 0 (internal), ~0 (single leaf) or INT_MIN (empty)
    int n_tris;
    float light[3];         // unit light travel direction
    unsigned* status;       // device status word
    const float4* plights;  // [2 n_plights]: (position, 0), (rgb, 0) of each point light
    int n_plights;
};

// ---- per session: forward-map table ------------------------------------------
// u - 1/2 as a function of z = tan(e) = c_r r on [0, tan(e_max)] (Eqs. 3, 12):
// kUTable uniform intervals, interval i holding the cubic Hermite piece
// c.x + t (c.y + t (c.z + t c.w)), t in [0, 1]; entry kUTable is the constant
// u(e_max) - 1/2 used for z >= tan(e_max).
constexpr int kUTable = 2048;

// ---- longest-first LP render: per frame-eye state kept from frame to frame ----
// The LP render takes its work in chunks of 32 consecutive work items (one per
// lane of a warp).  While a frame renders, every chunk whose traversal time
// (the slowest lane's clock cycles) is at least twice the previous frame's
// mean is listed, and the next frame renders the listed chunks before all
// others.  Only the order changes: every chunk is still rendered exactly once,
// so the results are those of the plain order.  Without it the slowest chunks,
// wherever they fall in the work order, decide when the launch ends.  The
// state has two halves used alternately (frame parity): the half being read
// holds this frame's list, the other collects the next frame's; the host
// clears the collecting half's counters before each frame.
struct LptCounters {
    unsigned long long cyc_sum;   // sum of the chunk costs of the frame
    unsigned chunks_done;         // chunks costed
    unsigned hot_count;           // entries of the list
};
struct LptState {
    LptCounters ctr[2];
    int* hot[2];                  // [capacity] listed chunks
    unsigned char* flag[2];       // [capacity] 1 = listed
    int capacity;                 // chunks the arrays hold
};
constexpr int kLptChunk = 32;

// ---- one frame-eye of work (kernel parameter; filled on the host in FP64,
// rounded to FP32) ------------------------------------------------------------
struct FrameDesc {
    float R[9];             // camera -> world rotation, row-major
    float org[3];           // eye position
    float gx, gy;           // gaze tangent offsets: c_r (x0 - W/2), c_r (H/2 - y0)
    float cr;               // c_r
    float px0, py0;         // c_r (0.5 - W/2), c_r (H/2 - 0.5): GT ray of pixel (0,0)
    int gxi, gyi;           // floor of the gaze point
    float gxf, gyf;         // 0.5 - fractional part of the gaze point
    int W, H;
    int lp_fmt, disp_fmt;
    const float* tan_e;     // device [C] tan(e_c) of the column centres
    const int2* col;        // device [C] (first texel, texel count)
    const int4* col_pair;   // device [-1 .. C-1] (slot, FP32 bits of count) of c and of min(c + 1, C - 1); [-1] = column 0 twice
    const float4* u_tab;    // device [u_n + 1] cubic pieces of u(z)
    const int2* work;       // device [n_texels] (texel, column) in processing order
    int u_n;                // number of pieces
    float u_inv_h;          // u_n / tan(e_max)
    int n_cols;
    int n_texels;
    void* lp;
    void* lp_aa;            // FXAA output (read by reconstruct) or nullptr: no FXAA
    float* luma;            // FXAA scratch: luma of every LP slot
    float* depth;           // hit distance per LP slot (inf on a miss) or nullptr
    void* disp;
    int* hit_ids;
    unsigned* status;
    long long work_begin;   // first global work item (render) of this frame
    long long tile_begin;   // first global tile (reconstruct) of this frame
    long long aa_begin;     // first global FXAA texel of this frame
    LptState* lpt;          // longest-first state | frame parity (bit 0), or nullptr
};

template <int MAXD>
struct Batch {
    int n;
    long long total_work;   // sum of render work items
    long long total_tiles;  // sum of reconstruct tiles
    long long total_aa;     // sum of FXAA texels (frames with lp_aa)
    unsigned long long* work_counter;  // device counters (persistent fetch; [1]: longest-first list)
    FrameDesc d[MAXD];
};

using SmallBatch = Batch<2>;
using BigBatch = Batch<VAFR_MAX_BATCH>;
// kernel parameters (scene + batch) must fit the 32,764-byte parameter space
static_assert(sizeof(BigBatch) + sizeof(SceneDev) <= 32764, "batch too large for kernel params");

// ---- launch interfaces ---------------------------------------------------------
// Render variants: threads per block, tree width, child order, register cap;
// variants 6 and 7 are the longest-first LP order (7: the ray regenerated for
// shading and at most 72 registers, 7 blocks per SM); the GT keeps variant 0's
// kernel for both.
constexpr int kNumRenderVariants = 8;
constexpr int kLptVariant = 6;
constexpr int kLptVariantLean = 7;
__host__ __device__ constexpr bool is_lpt_variant(int v) { return v == kLptVariant || v == kLptVariantLean; }
// Reconstruct variants: column-run tiles (0-3), row tiles (4-7) and the
// column-run tile with its LP footprint staged in shared memory (8).
constexpr int kNumReconVariants = 9;

// tile width/height in pixels; pixels per thread along a row (row tiles), or 0
// for a column-run tile (one thread per display column, `th` rows)
struct ReconShape { int tw, th; int px; };
ReconShape recon_shape(int variant);

template <class B>
cudaError_t launch_render_lp(const SceneDev& scene, const B& batch, int variant,
                             cudaStream_t s, int num_sms);
template <class B>
cudaError_t launch_render_gt(const SceneDev& scene, const B& batch, int variant,
                             cudaStream_t s, int num_sms);
template <class B>
cudaError_t launch_reconstruct(const B& batch, int variant, cudaStream_t s);
// Path-traced LP buffers (pathtrace.cu): one path per texel, `depth` diffuse
// bounces; FrameDesc.hit_ids, when set, receives depth + 2 ints per slot.
template <class B>
cudaError_t launch_path_lp(const SceneDev& scene, const B& batch, unsigned long long seed, int depth,
                           cudaStream_t s, int num_sms);
template <class B>
cudaError_t launch_path_gt(const SceneDev& scene, const B& batch, unsigned long long seed, int depth,
                           cudaStream_t s, int num_sms);
// Ray casting of an explicit list of (slot, column) work items whose count
// is read from device memory (render.cu): the reprojection's holes.
cudaError_t launch_render_list(const SceneDev& scene, const SmallBatch& batch, const unsigned* count,
                               cudaStream_t s, int num_sms);
// VaFR_Rep reprojection (reproject.cu): left frame d[0] (lp, depth) warped into
// right frame d[1] (lp written, holes appended to `holes` / `count`).
struct RepScratch {
    float4* vert;                 // [left slots] (U, F, depth, flags) seen from the right eye
    unsigned long long* zbuf;     // [right slots] (depth bits << 32) | triangle id
    int2* holes;                  // [right texels] (slot, column) left uncovered
    unsigned* count;              // number of holes
    int* tri_out;                 // [right slots] winning triangle id / -1, or nullptr
};
cudaError_t launch_reproject(const SmallBatch& batch, const RepScratch& r, cudaStream_t s, int num_sms);
// Deferred path (raster.cu): visibility buffer of frame d[0] at display
// resolution, then LP or full-resolution lighting from it.
struct VbufScratch {
    unsigned long long* vbuf;   // [H][W] (hit distance bits << 32) | triangle id, ~0 = sky
    int4* big;                  // large triangles' pixel boxes
    int* big_leaf;              // ... their leaves
    long long* big_first;       // ... and first tiles
    unsigned long long* counter;  // (records << 34) | tiles
    unsigned big_cap;
};
// stats (device, 4 counters, zeroed by the caller) selects an instrumented
// copy of the rasteriser that counts pre-filter evaluations, pixels past the
// pre-filter, exact tests and atomic minima; nullptr = the plain kernels.
cudaError_t launch_vbuffer(const SceneDev& sc, const SmallBatch& b, const VbufScratch& v, cudaStream_t s,
                           int num_sms, unsigned long long* stats = nullptr);
cudaError_t launch_leaf_of(const SceneDev& sc, int* leaf_of, cudaStream_t s, int num_sms);
cudaError_t launch_shade_vbuf(const SceneDev& sc, const SmallBatch& b, const unsigned long long* vbuf,
                              const int* leaf_of, bool full_res, cudaStream_t s, int num_sms);
// FXAA inside the LP buffer of every frame with lp_aa set (fxaa.cu).
template <class B>
cudaError_t launch_fxaa(const B& batch, cudaStream_t s, int num_sms);
cudaError_t launch_render_stats(const SceneDev& scene, const SmallBatch& batch,
                                unsigned long long* counters, cudaStream_t s, int num_sms);

// LBVH build (lbvh.cu).  All device pointers are owned by the caller.
struct LbvhBuffers {
    const float* tris;      // n x 9 input (device)
    const float* albedo;    // n x 3 (device) or nullptr
    int n;
    uint32_t* codes;        // n  Morton codes, input order
    uint32_t* keys_tmp;     // n  sort scratch
    int32_t* ids;           // n  sorted triangle ids
    int32_t* ids_tmp;       // n  sort scratch
    uint32_t* keys_sorted;  // n
    unsigned* hist;         // 256 * blocks
    float* part_bounds;     // 6 * blocks
    float* scene_bounds;    // 6
    int2* child;            // n-1
    int32_t* parent;        // (n-1) + n: parents of internal nodes then leaves
    unsigned* flags;        // n-1 refit arrival counters
    float* node_box;        // (n-1) x 6
    float* leaf_box;        // n x 6
    float4* nodes;          // (n-1) x 4
    unsigned* head_flag;    // n-1: internal node at even depth
    unsigned* head_idx;     // n-1: its 4-wide node index (each node's internal children consecutive)
    float4* nodes4;         // n_nodes4 x 16 (allocated once tree4_build has counted them)
    float4* leaves;         // n x 3
    float4* albedo4;        // n
};
size_t lbvh_sort_blocks(int n);
cudaError_t lbvh_build(const LbvhBuffers& b, cudaStream_t s);
// Traversal tree (tree4.cu): PLOC over the sorted leaves, collapsed to
// 4-wide nodes.  tree4_build clusters, numbers the nodes and returns their
// count; the caller allocates b.nodes4 (16 float4 per node) and tree4_pack
// writes them.  `scratch` holds tree4_scratch_bytes(n) device bytes, carries
// the binary tree from the first call to the second and may be freed after
// it (both synchronise `s`).
constexpr int kPlocRadius = 8;
size_t tree4_scratch_bytes(int n);
cudaError_t tree4_build(const LbvhBuffers& b, void* scratch, int radius, cudaStream_t s, int* n_nodes4);
cudaError_t tree4_pack(const LbvhBuffers& b, void* scratch, int n_nodes4, cudaStream_t s);

// FP32 issue rate (peak.cu): FMAs per second of scalar FFMA and of paired
// FFMA2 (two FMAs each) over the whole device; `sink` holds num_sms * 8 floats.
cudaError_t measure_fp32_peak(int num_sms, float* sink, cudaStream_t s, double* ffma, double* ffma2);

void count_launch(int k = 1);

}  // namespace vafr
