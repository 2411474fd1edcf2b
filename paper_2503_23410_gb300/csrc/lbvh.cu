// lbvh.cu -- LBVH construction on the GPU (Karras 2012, "Maximizing Parallelism
// in the Construction of BVHs, Octrees, and k-d Trees"):
//   1. scene bounds of the triangle centroid sums s = (v0 + v1) + v2,
//   2. 30-bit Morton codes of s on a cubic grid of 1024 cells along the
//      largest extent of the bounds,
//   3. stable LSD radix sort of (code, triangle id), 4 passes of 8 bits,
//   4. binary radix tree: one thread per internal node,
//   5. bottom-up FP32 bounds with one arrival counter per internal node,
//   6. packing into the 64-byte two-child traversal node + 48-byte leaves.
// The quantisation uses explicitly rounded intrinsics (no FMA contraction) so
// the codes are bit-identical to any IEEE FP32 evaluation of the same sequence.
// No kernel here waits on another thread: there is nothing that can spin.
#include "vafr_internal.cuh"

#include <float.h>

#include <cuda.h>

#include <cstring>
#include <mutex>

namespace vafr {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kBoundsBlocks = 304;

__device__ __forceinline__ float centroid_sum(const float* t, int k) {
    return __fadd_rn(__fadd_rn(t[k], t[3 + k]), t[6 + k]);
}

__global__ void k_bounds_partial(const float* __restrict__ tris, int n, float* __restrict__ part) {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float* t = tris + 9ll * i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float s = centroid_sum(t, k);
            lo[k] = fminf(lo[k], s);
            hi[k] = fmaxf(hi[k], s);
        }
    }
    __shared__ float red[6][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) { red[k][warp] = lo[k]; red[3 + k][warp] = hi[k]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        float v = red[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            v = k < 3 ? fminf(v, red[k][w]) : fmaxf(v, red[k][w]);
        part[6 * blockIdx.x + k] = v;
    }
}

__global__ void k_bounds_final(const float* __restrict__ part, int nb, float* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 6) return;
    float v = part[k];
    for (int b = 1; b < nb; ++b) v = k < 3 ? fminf(v, part[6 * b + k]) : fmaxf(v, part[6 * b + k]);
    out[k] = v;
}

// 10 bits spread to every third bit position (bit b -> bit 3b).
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(const float* __restrict__ tris, int n, const float* __restrict__ bounds,
                         uint32_t* __restrict__ codes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* t = tris + 9ll * i;
    // cubic grid: every axis is scaled by the largest extent of the bounds
    const float ext = fmaxf(fmaxf(__fsub_rn(bounds[3], bounds[0]), __fsub_rn(bounds[4], bounds[1])),
                            __fsub_rn(bounds[5], bounds[2]));
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = bounds[k];
        if (!(ext > 0.0f)) { q[k] = 0u; continue; }
        const float s = centroid_sum(t, k);
        const float u = __fdiv_rn(__fsub_rn(s, lo), ext);
        const uint32_t c = __float2uint_rz(__fmul_rn(u, 1024.0f));
        q[k] = c > 1023u ? 1023u : c;
    }
    codes[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
}

// ---- stable LSD radix sort ----------------------------------------------------
// Pass = histogram (per tile) -> exclusive scan in (digit, tile) order ->
// scatter.  The scatter ranks keys of a tile stably with warp multi-split:
// every warp owns a contiguous run of the tile and walks it 32 keys at a time
// in index order; __match_any_sync groups equal digits, and a per-(warp,
// digit) counter accumulates ranks; a prefix over warps then orders warps.

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int n, int shift,
                             unsigned* __restrict__ hist, int nblocks) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` counters by one block of 1024 threads.
__global__ void k_radix_scan(unsigned* __restrict__ hist, int total) {
    __shared__ unsigned part[1024];
    const int per = (total + 1023) / 1024;
    const int b = threadIdx.x * per;
    unsigned s = 0;
    for (int i = 0; i < per; ++i)
        if (b + i < total) s += hist[b + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = part[threadIdx.x] - s;   // exclusive prefix of this chunk
    for (int i = 0; i < per; ++i) {
        if (b + i < total) {
            unsigned v = hist[b + i];
            hist[b + i] = run;
            run += v;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int n, int shift,
                const unsigned* __restrict__ hist, int nblocks) {
    __shared__ unsigned cnt[kSortWarps][256];
    __shared__ unsigned gbase[256];
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&cnt[0][0])[i] = 0u;
    gbase[threadIdx.x] = hist[threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kSortTile + (long long)warp * (32 * kSortItems);
    uint32_t key[kSortItems];
    int32_t val[kSortItems];
    unsigned rank[kSortItems], dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const long long i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? (vin ? vin[i] : (int32_t)i) : 0;
        const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u + lane;
        dig[r] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned before = 0u;
        if (valid) before = cnt[warp][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;   // kSortThreads == 256 digits
        unsigned run = 0u;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const unsigned c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const long long i = base + r * 32 + lane;
        if (i < n) {
            const unsigned d = dig[r];
            const unsigned dst = gbase[d] + cnt[warp][d] + rank[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
    }
}

// ---- Karras hierarchy -----------------------------------------------------------
// delta(i, j): common prefix length of the keys (code, index); -1 out of range.
__device__ __forceinline__ int delta(const uint32_t* __restrict__ k, int n, int i, int j, uint32_t ki) {
    if (j < 0 || j >= n) return -1;
    const uint32_t kj = k[j];
    if (kj == ki) return 32 + __clz((unsigned)(i ^ j));
    return __clz(ki ^ kj);
}

__global__ void k_karras(const uint32_t* __restrict__ keys, int n, int2* __restrict__ child,
                         int32_t* __restrict__ parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const uint32_t ki = keys[i];
    const int d = (delta(keys, n, i, i + 1, ki) - delta(keys, n, i, i - 1, ki)) >= 0 ? 1 : -1;
    const int dmin = delta(keys, n, i, i - d, ki);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d, ki) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d, ki) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(keys, n, i, j, ki);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d, ki) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int L = (lo == gamma) ? ~gamma : gamma;
    const int R = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    child[i] = make_int2(L, R);
    parent[L >= 0 ? L : (n - 1) + ~L] = i;
    parent[R >= 0 ? R : (n - 1) + ~R] = i;
    if (i == 0) parent[0] = -1;
}

__device__ __forceinline__ void load_box(const float* p, float b[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k] = __ldcg(p + k);
}

// Bottom-up bounds: each leaf thread writes its box and climbs; at every
// internal node the first arrival stops and the second (which then sees both
// children's boxes) writes the union and continues.
__global__ void k_refit(const float* __restrict__ tris, const int32_t* __restrict__ ids, int n,
                        const int2* __restrict__ child, const int32_t* __restrict__ parent,
                        unsigned* __restrict__ flags, float* __restrict__ node_box,
                        float* __restrict__ leaf_box) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float* t = tris + 9ll * ids[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        leaf_box[6ll * k + a] = fminf(fminf(t[a], t[3 + a]), t[6 + a]);
        leaf_box[6ll * k + 3 + a] = fmaxf(fmaxf(t[a], t[3 + a]), t[6 + a]);
    }
    if (n == 1) return;
    int node = parent[(n - 1) + k];
    // a binary radix tree over 30-bit codes + 32-bit positions is at most 64
    // levels deep; the bound only guards against a malformed parent array
    for (int climb = 0; node >= 0 && climb < 96; ++climb) {
        __threadfence();
        if (atomicAdd(&flags[node], 1u) == 0u) return;
        __threadfence();
        const int2 c = child[node];
        float a[6], b[6];
        load_box(c.x >= 0 ? node_box + 6ll * c.x : leaf_box + 6ll * ~c.x, a);
        load_box(c.y >= 0 ? node_box + 6ll * c.y : leaf_box + 6ll * ~c.y, b);
        float* o = node_box + 6ll * node;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            __stcg(o + q, fminf(a[q], b[q]));
            __stcg(o + 3 + q, fmaxf(a[3 + q], b[3 + q]));
        }
        node = parent[node];
    }
}

__global__ void k_pack_nodes(const int2* __restrict__ child, const float* __restrict__ node_box,
                             const float* __restrict__ leaf_box, int n, float4* __restrict__ nodes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int2 c = child[i];
    const float* a = c.x >= 0 ? node_box + 6ll * c.x : leaf_box + 6ll * ~c.x;
    const float* b = c.y >= 0 ? node_box + 6ll * c.y : leaf_box + 6ll * ~c.y;
    // per axis: (left lo, right lo, left hi, right hi), so both children's slabs
    // are computed with paired FP32 instructions
    nodes[4ll * i + 0] = make_float4(a[0], b[0], a[3], b[3]);
    nodes[4ll * i + 1] = make_float4(a[1], b[1], a[4], b[4]);
    nodes[4ll * i + 2] = make_float4(a[2], b[2], a[5], b[5]);
    nodes[4ll * i + 3] = make_float4(__int_as_float(c.x), __int_as_float(c.y), 0.0f, 0.0f);
}

__device__ __forceinline__ bool lex_less(float ax, float ay, float az, float bx, float by, float bz) {
    return ax < bx || (ax == bx && (ay < by || (ay == by && az < bz)));
}

// Leaves store their vertices in lexicographic (x, y, z) order.  The
// intersection test is two-sided, so the order carries no meaning, and
// identical triangles given with different vertex orders then evaluate to
// bit-identical t: the lower-id rule, not rounding, decides between them.
__global__ void k_pack_leaves(const float* __restrict__ tris, const float* __restrict__ albedo,
                              const int32_t* __restrict__ ids, int n, float4* __restrict__ leaves,
                              float4* __restrict__ albedo4) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int id = ids[k];
    const float* t = tris + 9ll * id;
    float v[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[a][c] = t[3 * a + c];
    // three-element sorting network
#define VAFR_CSWAP(i, j)                                                                      \
    if (lex_less(v[j][0], v[j][1], v[j][2], v[i][0], v[i][1], v[i][2])) {                     \
        for (int c = 0; c < 3; ++c) { const float q = v[i][c]; v[i][c] = v[j][c]; v[j][c] = q; } \
    }
    VAFR_CSWAP(0, 1)
    VAFR_CSWAP(1, 2)
    VAFR_CSWAP(0, 1)
#undef VAFR_CSWAP
    leaves[3ll * k + 0] = make_float4(v[0][0], v[0][1], v[0][2], __int_as_float(id));
    leaves[3ll * k + 1] = make_float4(v[1][0], v[1][1], v[1][2], 0.0f);
    leaves[3ll * k + 2] = make_float4(v[2][0], v[2][1], v[2][2], 0.0f);
    // albedo in original order (thread k writes triangle k's albedo)
    if (albedo)
        albedo4[k] = make_float4(albedo[3ll * k], albedo[3ll * k + 1], albedo[3ll * k + 2], 0.0f);
    else
        albedo4[k] = make_float4(0.8f, 0.8f, 0.8f, 0.0f);
}

inline int blocks_for(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

}  // namespace

size_t lbvh_sort_blocks(int n) { return (size_t)((n + kSortTile - 1) / kSortTile); }

cudaError_t lbvh_build(const LbvhBuffers& b, cudaStream_t s) {
    const int n = b.n;
    if (n <= 0) return cudaSuccess;
    const int nb_bounds = min(kBoundsBlocks, blocks_for(n, 256));
    k_bounds_partial<<<nb_bounds, 256, 0, s>>>(b.tris, n, b.part_bounds);
    k_bounds_final<<<1, 32, 0, s>>>(b.part_bounds, nb_bounds, b.scene_bounds);
    k_morton<<<blocks_for(n, 256), 256, 0, s>>>(b.tris, n, b.scene_bounds, b.codes);
    count_launch(3);
    const int nblocks = (int)lbvh_sort_blocks(n);
    // ping-pong: codes -> tmp -> sorted -> tmp -> sorted
    const uint32_t* kin = b.codes;
    const int32_t* vin = nullptr;
    for (int pass = 0; pass < 4; ++pass) {
        uint32_t* kout = (pass & 1) ? b.keys_sorted : b.keys_tmp;
        int32_t* vout = (pass & 1) ? b.ids : b.ids_tmp;
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, n, 8 * pass, b.hist, nblocks);
        k_radix_scan<<<1, 1024, 0, s>>>(b.hist, 256 * nblocks);
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * pass,
                                                         b.hist, nblocks);
        count_launch(3);
        kin = kout;
        vin = vout;
    }
    if (n > 1) {
        cudaMemsetAsync(b.flags, 0, sizeof(unsigned) * (size_t)(n - 1), s);
        k_karras<<<blocks_for(n - 1, 256), 256, 0, s>>>(b.keys_sorted, n, b.child, b.parent);
        count_launch(1);
    }
    k_refit<<<blocks_for(n, 256), 256, 0, s>>>(b.tris, b.ids, n, b.child, b.parent, b.flags,
                                               b.node_box, b.leaf_box);
    count_launch(1);
    if (n > 1) {
        k_pack_nodes<<<blocks_for(n - 1, 256), 256, 0, s>>>(b.child, b.node_box, b.leaf_box, n,
                                                            b.nodes);
        count_launch(1);
    }
    k_pack_leaves<<<blocks_for(n, 256), 256, 0, s>>>(b.tris, b.albedo, b.ids, n, b.leaves,
                                                     b.albedo4);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace vafr

// ---- allocation-free Morton codes + sort ---------------------------------------
// vafr_morton_sort_noalloc serves callers that may not allocate device memory:
// code running where the whole GPU's memory belongs to the caller's own pool
// allocator, or on a latency-critical thread where cudaMalloc's implicit
// device synchronisation is not acceptable.  All of its scratch lives in one
// file-scope __device__ array; it launches the same kernels as the build.
namespace vafr {
namespace {

constexpr int kNoAllocMaxTris = VAFR_NOALLOC_MAX_TRIS;
constexpr int kNoAllocBlocks = (kNoAllocMaxTris + kSortTile - 1) / kSortTile;

struct NoAllocScratch {
    uint32_t keys_tmp[kNoAllocMaxTris];
    int32_t ids_tmp[kNoAllocMaxTris];
    uint32_t keys_sorted[kNoAllocMaxTris];
    unsigned hist[256 * kNoAllocBlocks];
    float part_bounds[6 * kBoundsBlocks];
    float scene_bounds[8];
};

// Held by every GPU that loads the library until the process exits
// (sizeof(NoAllocScratch) = 6.3 MB).  Every call shares it; nothing in it has
// to start at zero (each pass overwrites what it reads).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocSlot {
    NoAllocScratch* ptr;         // device address of the array, or nullptr
    unsigned long long ctx_id;   // context it was looked up in (0: unknown)
};
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices] = {};

// Process-unique id of the calling thread's current context, or 0 if the
// driver cannot say.  A device reset destroys the context and the module with
// the array; the context that replaces it has a new id, which tells the cache
// below to look the address up again.  The two driver calls are found
// through the runtime, so the library needs no link against the driver.
unsigned long long current_context_id() {
    using GetCur = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<GetCur>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// that device current: once per device, and again after a device reset.
cudaError_t noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocSlot& slot = g_noalloc_slot[dev];
    if (!slot.ptr || slot.ctx_id != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot = NoAllocSlot{static_cast<NoAllocScratch*>(p), ctx};
    }
    *out = slot.ptr;
    return cudaSuccess;
}

// Whether byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace
}  // namespace vafr

extern "C" VAFR_API int vafr_morton_sort_noalloc(const float* tri_xyz, int64_t n_tris,
                                                 uint32_t* codes_out, int32_t* sorted_ids_out,
                                                 void* stream, char* err, int32_t err_len) {
    using namespace vafr;
    auto report = [&](int code, const char* msg) {
        if (err && err_len > 0) {
            std::strncpy(err, msg, (size_t)err_len - 1);
            err[err_len - 1] = '\0';
        }
        return code;
    };
    if (n_tris < 0) return report(VAFR_ERR_INVALID_ARG, "n_tris is negative");
    if (n_tris > kNoAllocMaxTris)
        return report(VAFR_ERR_INVALID_ARG, "n_tris exceeds VAFR_NOALLOC_MAX_TRIS (524288)");
    if (n_tris == 0) return VAFR_OK;
    if (!tri_xyz || !codes_out || !sorted_ids_out) return report(VAFR_ERR_INVALID_ARG, "NULL pointer");
    for (const void* p : {(const void*)tri_xyz, (const void*)codes_out, (const void*)sorted_ids_out}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return report(VAFR_ERR_INVALID_ARG, "every buffer must be device memory");
        }
    }
    // the sort reads its input keys while writing the output ids: any shared
    // byte between the three buffers would corrupt the result silently
    const size_t nt = (size_t)n_tris;
    if (overlaps(codes_out, 4 * nt, sorted_ids_out, 4 * nt) || overlaps(tri_xyz, 36 * nt, codes_out, 4 * nt) ||
        overlaps(tri_xyz, 36 * nt, sorted_ids_out, 4 * nt))
        return report(VAFR_ERR_INVALID_ARG, "tri_xyz, codes_out and sorted_ids_out must not overlap");
    NoAllocScratch* sc = nullptr;
    cudaError_t e = noalloc_scratch(&sc);
    if (e != cudaSuccess) return report(VAFR_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n = (int)n_tris;
    const int nb_bounds = min(kBoundsBlocks, blocks_for(n, 256));
    k_bounds_partial<<<nb_bounds, 256, 0, s>>>(tri_xyz, n, sc->part_bounds);
    k_bounds_final<<<1, 32, 0, s>>>(sc->part_bounds, nb_bounds, sc->scene_bounds);
    k_morton<<<blocks_for(n, 256), 256, 0, s>>>(tri_xyz, n, sc->scene_bounds, codes_out);
    count_launch(3);
    const int nblocks = (int)lbvh_sort_blocks(n);
    const uint32_t* kin = codes_out;
    const int32_t* vin = nullptr;
    for (int pass = 0; pass < 4; ++pass) {
        uint32_t* kout = (pass & 1) ? sc->keys_sorted : sc->keys_tmp;
        int32_t* vout = (pass & 1) ? sorted_ids_out : sc->ids_tmp;
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, n, 8 * pass, sc->hist, nblocks);
        k_radix_scan<<<1, 1024, 0, s>>>(sc->hist, 256 * nblocks);
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * pass,
                                                         sc->hist, nblocks);
        count_launch(3);
        kin = kout;
        vin = vout;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(VAFR_ERR_CUDA, cudaGetErrorString(e));
    return VAFR_OK;
}
