// render.cu -- ray generation, LBVH traversal and shading (the ray-casting
// pipeline of Sec. 6.1: ray-generation shader dispatched over the LP buffer,
// closest-hit shader, miss shader; and the GT dispatch over display pixels).
//
// Kernels are persistent: a grid of (SMs x resident blocks) whose warps pull
// chunks of work items from one global atomic counter until the batch is done,
// so uneven frames and uneven rays balance dynamically.  The traversal and
// shading they share with the other pipelines live in trace.cuh.
#include "trace.cuh"

namespace vafr {
namespace {

template <int TPB, int FETCH, int WIDE, int ORDER, int MINB, class B>
__global__ void __launch_bounds__(TPB, MINB)
k_render_lp(const SceneDev sc, const __grid_constant__ B b) {
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long base = 0ull;
        if (lane == 0) base = atomicAdd(b.work_counter, (unsigned long long)FETCH);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= b.total_work) break;
#pragma unroll 1
        for (int k = 0; k < FETCH; k += 32) {
            const long long w = (long long)base + k + lane;
            if (w >= b.total_work) break;
            const int fi = find_frame(b, w, false);
            const FrameDesc& f = b.d[fi];
            Ray r;
            int glo, ghi;
            const int t = lp_ray(f, (int)(w - f.work_begin), r, glo, ghi);
            ray_setup(r);
            Hit h;
            const unsigned fault = traverse<WIDE, false, ORDER>(sc, r, h, nullptr, nullptr, nullptr);
            if (fault) { atomicOr(f.status, fault); h.leaf = -1; h.id = -1; }
            // shading regenerates the ray (same bits) instead of keeping its
            // direction in registers through the traversal: with it the
            // 64-register variants run without spills
            lp_ray(f, (int)(w - f.work_begin), r, glo, ghi);
            store_lp(f, t, glo, ghi, shade(sc, r, h), h.leaf >= 0 ? h.id : -1);
            if (f.depth) f.depth[t] = h.leaf >= 0 ? h.t : INFINITY;
        }
    }
}

// Ray casting of the work items listed in frame 0's work table, as many as
// *count says (a device-side count: the reprojection's holes).
__global__ void __launch_bounds__(128)
k_render_list(const SceneDev sc, const __grid_constant__ SmallBatch b, const unsigned* count) {
    const int lane = threadIdx.x & 31;
    const long long total = (long long)*count;
    const FrameDesc& f = b.d[0];
    while (true) {
        unsigned long long base = 0ull;
        if (lane == 0) base = atomicAdd(b.work_counter, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= total) break;
        const long long w = (long long)base + lane;
        if (w < total) {
            Ray r;
            int glo, ghi;
            const int t = lp_ray(f, (int)w, r, glo, ghi);
            ray_setup(r);
            Hit h;
            const unsigned fault = traverse<4, false, 1>(sc, r, h, nullptr, nullptr, nullptr);
            if (fault) { atomicOr(f.status, fault); h.leaf = -1; h.id = -1; }
            store_lp(f, t, glo, ghi, shade(sc, r, h), h.leaf >= 0 ? h.id : -1);
        }
    }
}

// ---- longest-first LP render -----------------------------------------------------
// FrameDesc.lpt carries the frame parity p in bit 0: half p of the state holds
// this frame's list (built while the previous frame rendered), half 1 - p
// collects the next frame's.  A chunk is listed when it took at least twice
// the previous frame's mean; before any valid mean exists nothing is listed.
__device__ __forceinline__ LptState* lpt_state(const FrameDesc& f, int& p) {
    const uintptr_t v = reinterpret_cast<uintptr_t>(f.lpt);
    p = (int)(v & 1u);
    return reinterpret_cast<LptState*>(v & ~(uintptr_t)1);
}

// The LP render in chunks of 32 work items: first the listed chunks of every
// frame (counter [1]), then all chunks in work order (counter [0]) except the
// listed ones.
// REGEN: the shading regenerates the ray (same bits) instead of keeping it
// through the traversal, which with MINB = 7 fits 7 blocks per SM.
template <int TPB, int ORDER, class B, bool REGEN = false, int MINB = 1>
__global__ void __launch_bounds__(TPB, MINB)
k_render_lp_lpt(const SceneDev sc, const __grid_constant__ B b) {
    // Everything the fetch needs lives in shared memory and is re-read there,
    // so the traversal keeps the registers of the plain kernel (a register cap
    // on this kernel costs more than the order gains).
    constexpr int MAXD = sizeof(b.d) / sizeof(b.d[0]);
    __shared__ int cbeg[MAXD + 1];         // first chunk of each frame
    __shared__ unsigned hbeg[MAXD + 1];    // first listed chunk of each frame
    __shared__ unsigned thr[MAXD];         // listing threshold of each frame (~0 = none)
    // this block's chunk costs per frame, added to the state once at the end
    // (one global atomic per block instead of one per chunk on a single address)
    __shared__ unsigned long long bsum[MAXD];
    __shared__ unsigned bcnt[MAXD];
    for (int f = threadIdx.x; f < b.n; f += blockDim.x) {
        bsum[f] = 0ull;
        bcnt[f] = 0u;
    }
    if (threadIdx.x == 0) {
        int c = 0;
        unsigned h = 0;
        for (int f = 0; f < b.n; ++f) {
            int p;
            const LptState* S = lpt_state(b.d[f], p);
            const int nch = (b.d[f].n_texels + kLptChunk - 1) / kLptChunk;
            cbeg[f] = c;
            hbeg[f] = h;
            thr[f] = 0xffffffffu;
            // the half is valid when the previous frame costed exactly this
            // frame's chunks: then its list and flags cover every chunk
            if (S && nch <= S->capacity && S->ctr[p].chunks_done == (unsigned)nch &&
                S->ctr[p].hot_count <= (unsigned)nch) {
                h += S->ctr[p].hot_count;
                thr[f] = (unsigned)min(2ull * (S->ctr[p].cyc_sum / (unsigned)nch), 0xffffffffull);
            }
            c += nch;
        }
        cbeg[b.n] = c;
        hbeg[b.n] = h;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    bool listed = true;
    while (true) {
        unsigned idx = 0u;
        if (lane == 0) idx = (unsigned)atomicAdd(b.work_counter + (listed ? 1 : 0), 1ull);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        int fi, c;
        if (listed) {
            if (idx >= hbeg[b.n]) {
                listed = false;
                continue;
            }
            int lo = 0, hi = b.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (hbeg[mid] <= idx) lo = mid; else hi = mid - 1;
            }
            fi = lo;
            int p;
            const LptState* S = lpt_state(b.d[fi], p);
            c = S->hot[p][idx - hbeg[fi]];
            if (c < 0 || c >= S->capacity) continue;
        } else {
            if (idx >= (unsigned)cbeg[b.n]) break;
            int lo = 0, hi = b.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((unsigned)cbeg[mid] <= idx) lo = mid; else hi = mid - 1;
            }
            fi = lo;
            c = (int)idx - cbeg[fi];
            int p;
            const LptState* S = lpt_state(b.d[fi], p);
            if (S && c < S->capacity && thr[fi] != 0xffffffffu && S->flag[p][c]) continue;   // listed
        }
        const FrameDesc& f = b.d[fi];
        const unsigned t0 = (unsigned)clock();
        const int local = c * kLptChunk + lane;
        if (local < f.n_texels) {
            Ray r;
            int glo, ghi;
            const int t = lp_ray(f, local, r, glo, ghi);
            ray_setup(r);
            Hit h;
            const unsigned fault = traverse<4, false, ORDER>(sc, r, h, nullptr, nullptr, nullptr);
            if (fault) { atomicOr(f.status, fault); h.leaf = -1; h.id = -1; }
            if (REGEN) lp_ray(f, local, r, glo, ghi);
            store_lp(f, t, glo, ghi, shade(sc, r, h), h.leaf >= 0 ? h.id : -1);
            if (f.depth) f.depth[t] = h.leaf >= 0 ? h.t : INFINITY;
        }
        const unsigned cmax = __reduce_max_sync(0xffffffffu, (unsigned)clock() - t0);
        int p;
        LptState* S = lpt_state(f, p);
        if (lane == 0 && S && c < S->capacity) {
            const int q = p ^ 1;
            const bool hot = cmax >= thr[fi];
            S->flag[q][c] = (unsigned char)hot;
            if (hot) {
                const unsigned pos = atomicAdd(&S->ctr[q].hot_count, 1u);
                if (pos < (unsigned)S->capacity) S->hot[q][pos] = c;
            }
            atomicAdd(&bsum[fi], (unsigned long long)cmax);
            atomicAdd(&bcnt[fi], 1u);
        }
    }
    __syncthreads();
    for (int f = threadIdx.x; f < b.n; f += blockDim.x) {
        int p;
        LptState* S = lpt_state(b.d[f], p);
        if (S && bcnt[f]) {
            atomicAdd(&S->ctr[p ^ 1].cyc_sum, bsum[f]);
            atomicAdd(&S->ctr[p ^ 1].chunks_done, bcnt[f]);
        }
    }
}

// GT: work item = (tile of 8 x 4 pixels, lane); pixel centre rays.
template <int TPB, int FETCH, int WIDE, int ORDER, int MINB, class B>
__global__ void __launch_bounds__(TPB, MINB)
k_render_gt(const SceneDev sc, const __grid_constant__ B b) {
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long base = 0ull;
        if (lane == 0) base = atomicAdd(b.work_counter, (unsigned long long)FETCH);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= b.total_work) break;
#pragma unroll 1
        for (int k = 0; k < FETCH; k += 32) {
            const long long w = (long long)base + k + lane;
            if (w >= b.total_work) break;
            const int fi = find_frame(b, w, false);
            const FrameDesc& f = b.d[fi];
            const long long local = w - f.work_begin;
            const long long tile = local >> 5;
            const int tiles_x = (f.W + 7) >> 3;
            const int x = (int)(tile % tiles_x) * 8 + (lane & 7);
            const int y = (int)(tile / tiles_x) * 4 + (lane >> 3);
            if (x >= f.W || y >= f.H) continue;
            const float cx = f.cr * ((float)x + 0.5f - 0.5f * (float)f.W);
            const float cy = f.cr * (0.5f * (float)f.H - ((float)y + 0.5f));
            Ray r;
            world_ray(f, cx, cy, r);
            ray_setup(r);
            Hit h;
            const unsigned fault = traverse<WIDE, false, ORDER>(sc, r, h, nullptr, nullptr, nullptr);
            if (fault) { atomicOr(f.status, fault); h.leaf = -1; h.id = -1; }
            const long long p = (long long)y * f.W + x;
            store_px(f.disp, p, f.disp_fmt, shade(sc, r, h));
            if (f.hit_ids) f.hit_ids[p] = h.leaf >= 0 ? h.id : -1;
        }
    }
}

// Instrumented copy (never timed): counts rays, node visits, box tests,
// triangle tests and hits of the 4-wide traversal the render kernels use.
__global__ void __launch_bounds__(128)
k_render_stats(const SceneDev sc, const __grid_constant__ SmallBatch b, unsigned long long* out) {
    unsigned long long nodes = 0, boxes = 0, tris = 0, rays = 0, hits = 0, worst = 0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < b.total_work;
         w += (long long)gridDim.x * blockDim.x) {
        const FrameDesc& f = b.d[find_frame(b, w, false)];
        Ray r;
        int glo, ghi;
        lp_ray(f, (int)(w - f.work_begin), r, glo, ghi);
        ray_setup(r);
        Hit h;
        unsigned long long n0 = nodes;
        traverse<4, true>(sc, r, h, &nodes, &boxes, &tris);
        worst = max(worst, nodes - n0);
        ++rays;
        hits += h.leaf >= 0;
    }
    atomicAdd(out + 0, rays);
    atomicAdd(out + 1, nodes);
    atomicAdd(out + 2, boxes);
    atomicAdd(out + 3, tris);
    atomicAdd(out + 4, hits);
    atomicMax(out + 5, worst);
}

template <int TPB, int FETCH, int WIDE, int ORDER, int MINB, bool GT, class B>
cudaError_t launch_one(const SceneDev& sc, const B& b, cudaStream_t s, int num_sms) {
    auto kern = GT ? k_render_gt<TPB, FETCH, WIDE, ORDER, MINB, B>
                   : k_render_lp<TPB, FETCH, WIDE, ORDER, MINB, B>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    e = cudaMemsetAsync(b.work_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long want_warps = (b.total_work + FETCH - 1) / FETCH;
    long long grid = (long long)per_sm * num_sms;
    const long long need = (want_warps * 32 + TPB - 1) / TPB;
    if (need < grid) grid = need < 1 ? 1 : need;
    kern<<<(unsigned)grid, TPB, 0, s>>>(sc, b);
    count_launch(1);
    return cudaGetLastError();
}

template <int TPB, int ORDER, bool REGEN = false, int MINB = 1, class B>
cudaError_t launch_lpt(const SceneDev& sc, const B& b, cudaStream_t s, int num_sms) {
    auto kern = k_render_lp_lpt<TPB, ORDER, B, REGEN, MINB>;
    // the kernel's few bytes of shared memory must not shrink the L1 the
    // traversal lives in: ask for the smallest shared-memory carveout
    static const cudaError_t carve =
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    if (carve != cudaSuccess) return carve;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    e = cudaMemsetAsync(b.work_counter, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long grid = (long long)per_sm * num_sms;
    const long long need = (b.total_work + TPB - 1) / TPB;
    if (need < grid) grid = need < 1 ? 1 : need;
    kern<<<(unsigned)grid, TPB, 0, s>>>(sc, b);
    count_launch(1);
    return cudaGetLastError();
}

template <bool GT, class B>
cudaError_t launch_variant(const SceneDev& sc, const B& b, int variant, cudaStream_t s, int sms) {
    if (b.total_work <= 0) return cudaSuccess;
    if (is_lpt_variant(variant)) {
        if (GT) return launch_one<128, 32, 4, 1, 1, GT>(sc, b, s, sms);
        return variant == kLptVariant ? launch_lpt<128, 0>(sc, b, s, sms) : launch_lpt<128, 0, true, 7>(sc, b, s, sms);
    }
    // (threads per block, rays per warp fetch, tree width, child order, min blocks/SM)
    switch (variant) {
        case 0: return launch_one<128, 32, 4, 1, 1, GT>(sc, b, s, sms);
        case 1: return launch_one<256, 32, 4, 0, 1, GT>(sc, b, s, sms);
        case 2: return launch_one<128, 32, 4, 0, 1, GT>(sc, b, s, sms);
        case 3: return launch_one<128, 32, 2, 0, 1, GT>(sc, b, s, sms);
        case 4: return launch_one<128, 32, 4, 0, 8, GT>(sc, b, s, sms);
        default: return launch_one<128, 32, 4, 1, 8, GT>(sc, b, s, sms);
    }
}
}  // namespace

template <class B>
cudaError_t launch_render_lp(const SceneDev& scene, const B& batch, int variant, cudaStream_t s,
                             int num_sms) {
    return launch_variant<false>(scene, batch, variant, s, num_sms);
}
template <class B>
cudaError_t launch_render_gt(const SceneDev& scene, const B& batch, int variant, cudaStream_t s,
                             int num_sms) {
    return launch_variant<true>(scene, batch, variant, s, num_sms);
}

template cudaError_t launch_render_lp<SmallBatch>(const SceneDev&, const SmallBatch&, int, cudaStream_t, int);
template cudaError_t launch_render_lp<BigBatch>(const SceneDev&, const BigBatch&, int, cudaStream_t, int);
template cudaError_t launch_render_gt<SmallBatch>(const SceneDev&, const SmallBatch&, int, cudaStream_t, int);
template cudaError_t launch_render_gt<BigBatch>(const SceneDev&, const BigBatch&, int, cudaStream_t, int);

cudaError_t launch_render_list(const SceneDev& scene, const SmallBatch& batch, const unsigned* count,
                               cudaStream_t s, int num_sms) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_list, 128, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    e = cudaMemsetAsync(batch.work_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_render_list<<<(unsigned)(per_sm * num_sms), 128, 0, s>>>(scene, batch, count);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_render_stats(const SceneDev& scene, const SmallBatch& batch,
                                unsigned long long* counters, cudaStream_t s, int num_sms) {
    cudaError_t e = cudaMemsetAsync(counters, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_render_stats<<<num_sms * 4, 128, 0, s>>>(scene, batch, counters);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace vafr
