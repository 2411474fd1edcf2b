// tree4.cu -- the traversal tree: a binary tree of the scene's leaves built by
// PLOC (Meister and Bittner 2018, "Parallel Locally-Ordered Clustering for
// Bounding Volume Hierarchy Construction"), collapsed into 4-wide nodes.
//
// PLOC starts from the leaves in Morton order (the LBVH sort) and repeats:
//   1. every cluster finds the cluster within +-radius positions whose
//      merged box has the smallest surface area (ties: the nearer position,
//      then the partner i ^ 1, so runs of equal boxes pair up);
//   2. mutual nearest neighbours merge into a new internal node, which takes
//      the lower position; the other position is dropped;
//   3. the cluster array is compacted (exclusive scans; no atomics, so the
//      tree is deterministic).
// The pair of mutual neighbours with the smallest distance (lowest position on
// ties) always exists, so every round merges at least once.  The tree is then
// renumbered so its root is node 0 and collapsed two levels at a time: every
// internal node at even depth becomes a 4-wide node whose children are its
// children, internal children replaced by their own two children.  All boxes
// are exact FP32 unions of the triangles' boxes.
#include "vafr_internal.cuh"

#include <utility>

namespace vafr {
namespace {

constexpr int kPlocRadiusMax = 16;
constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

inline int blocks_for(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

// ---- multi-block exclusive scan of unsigned counters ----------------------------
__global__ void k_scan_tiles(unsigned* __restrict__ v, int n, unsigned* __restrict__ sums) {
    __shared__ unsigned part[kScanThreads];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned x[kScanItems];
    unsigned acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        x[k] = base + k < n ? v[base + k] : 0u;
        acc += x[k];
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const unsigned t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    unsigned run = part[threadIdx.x] - acc;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) v[base + k] = run;
        run += x[k];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = part[threadIdx.x];
}

__global__ void k_scan_add(unsigned* __restrict__ v, int n, const unsigned* __restrict__ sums) {
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) v[i] += sums[i / kScanTile];
}

// Scratch `sums` needs scan_scratch_elems(n) entries.
int scan_scratch_elems(int n) {
    int total = 0;
    for (int m = n; m > 1;) {
        m = blocks_for(m, kScanTile);
        total += m;
    }
    return total + 1;
}

cudaError_t exclusive_scan(unsigned* v, int n, unsigned* sums, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = blocks_for(n, kScanTile);
    k_scan_tiles<<<nb, kScanThreads, 0, s>>>(v, n, sums);
    count_launch(1);
    if (nb > 1) {
        cudaError_t e = exclusive_scan(sums, nb, sums + nb, s);   // scan the tile sums
        if (e != cudaSuccess) return e;
        k_scan_add<<<blocks_for(n, kThreads), kThreads, 0, s>>>(v, n, sums);
        count_launch(1);
    }
    return cudaGetLastError();
}

// ---- PLOC ---------------------------------------------------------------------------
__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return fmaf(dx, dy, fmaf(dy, dz, dz * dx));
}

__global__ void k_ploc_init(const float* __restrict__ leaf_box, int n, int* __restrict__ C,
                            float4* __restrict__ lo, float4* __restrict__ hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* b = leaf_box + 6ll * i;
    C[i] = ~i;
    lo[i] = make_float4(b[0], b[1], b[2], 0.0f);
    hi[i] = make_float4(b[3], b[4], b[5], 0.0f);
}

__global__ void __launch_bounds__(kThreads)
k_ploc_nn(const float4* __restrict__ lo, const float4* __restrict__ hi, int m, int radius,
          int* __restrict__ nbr) {
    constexpr int R = kPlocRadiusMax;
    __shared__ float4 slo[kThreads + 2 * R], shi[kThreads + 2 * R];
    const int base = blockIdx.x * kThreads;
    for (int k = threadIdx.x; k < kThreads + 2 * R; k += kThreads) {
        const int j = base - R + k;
        if (j >= 0 && j < m) {
            slo[k] = lo[j];
            shi[k] = hi[j];
        }
    }
    __syncthreads();
    const int i = base + threadIdx.x;
    if (i >= m) return;
    const float4 a = slo[threadIdx.x + R], A = shi[threadIdx.x + R];
    // Equal costs (identical boxes, e.g. duplicated geometry) go to the nearer
    // position, then to the partner i ^ 1: a run of equal boxes then pairs up
    // as (0,1) (2,3) ... in every round and halves, where "lower position
    // first" would merge one pair per round and chain the tree.
    const int pref = (i & 1) ? -1 : 1;
    float best = INFINITY;
    int bj = -1, bd = 0;
    for (int d = -radius; d <= radius; ++d) {
        const int j = i + d;
        if (d == 0 || j < 0 || j >= m) continue;
        const float4 b = slo[threadIdx.x + R + d], B = shi[threadIdx.x + R + d];
        const float c = half_area(make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.0f),
                                  make_float4(fmaxf(A.x, B.x), fmaxf(A.y, B.y), fmaxf(A.z, B.z), 0.0f));
        const int ad = d < 0 ? -d : d, abd = bd < 0 ? -bd : bd;
        if (c < best || (c == best && (ad < abd || (ad == abd && d == pref)))) {
            best = c;
            bj = j;
            bd = d;
        }
    }
    nbr[i] = bj;
}

__global__ void k_ploc_flags(const int* __restrict__ nbr, int m, unsigned* __restrict__ keep,
                             unsigned* __restrict__ merge) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j = nbr[i];
    const bool mutual = j >= 0 && nbr[j] == i;
    keep[i] = (mutual && i > j) ? 0u : 1u;
    merge[i] = (mutual && i < j) ? 1u : 0u;
}

__global__ void k_ploc_compact(const int* __restrict__ C, const float4* __restrict__ lo,
                               const float4* __restrict__ hi, const int* __restrict__ nbr,
                               const unsigned* __restrict__ keep_flag, const unsigned* __restrict__ pos,
                               const unsigned* __restrict__ merge_flag, const unsigned* __restrict__ moff,
                               int m, int node_base, int* __restrict__ C2, float4* __restrict__ lo2,
                               float4* __restrict__ hi2, int2* __restrict__ child,
                               float* __restrict__ node_box) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !keep_flag[i]) return;
    const unsigned p = pos[i];
    if (merge_flag[i]) {
        const int j = nbr[i];
        const int id = node_base + (int)moff[i];
        const float4 a = lo[i], b = lo[j], A = hi[i], B = hi[j];
        const float4 l = make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.0f);
        const float4 h = make_float4(fmaxf(A.x, B.x), fmaxf(A.y, B.y), fmaxf(A.z, B.z), 0.0f);
        child[id] = make_int2(C[i], C[j]);
        float* nb = node_box + 6ll * id;
        nb[0] = l.x; nb[1] = l.y; nb[2] = l.z; nb[3] = h.x; nb[4] = h.y; nb[5] = h.z;
        C2[p] = id;
        lo2[p] = l;
        hi2[p] = h;
    } else {
        C2[p] = C[i];
        lo2[p] = lo[i];
        hi2[p] = hi[i];
    }
}

// creation order puts the root last: node id -> n_inner - 1 - id puts it first
__global__ void k_renumber(const int2* __restrict__ child, const float* __restrict__ node_box,
                           int n_inner, int2* __restrict__ child2, float* __restrict__ node_box2,
                           int32_t* __restrict__ parent2) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_inner) return;
    const int nid = n_inner - 1 - id;
    int2 c = child[id];
    c.x = c.x >= 0 ? n_inner - 1 - c.x : c.x;
    c.y = c.y >= 0 ? n_inner - 1 - c.y : c.y;
    child2[nid] = c;
    if (c.x >= 0) parent2[c.x] = nid;
    if (c.y >= 0) parent2[c.y] = nid;
    if (nid == 0) parent2[0] = -1;
#pragma unroll
    for (int k = 0; k < 6; ++k) node_box2[6ll * nid + k] = node_box[6ll * id + k];
}

// ---- collapse to 4-wide -------------------------------------------------------------
__global__ void k_depth_heads(const int32_t* __restrict__ parent, int n_inner,
                              unsigned* __restrict__ head) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inner) return;
    int d = 0;
    // a PLOC tree of 2^30 leaves can be deeper than a radix tree; the bound only
    // guards against a malformed parent array
    for (int p = parent[i]; p >= 0 && d < 4096; p = parent[p]) ++d;
    head[i] = (d & 1) == 0 ? 1u : 0u;
}

__device__ __forceinline__ void box_of(int ref, const float* __restrict__ node_box,
                                       const float* __restrict__ leaf_box, float b[6]) {
    const float* p = ref >= 0 ? node_box + 6ll * ref : leaf_box + 6ll * ~ref;
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k] = p[k];
}

// The 4-wide children of head i: its binary children that are leaves and the
// two children of each internal one (heads, at the next even depth, or
// leaves).  Internal children come first (ni of them), then the leaves: m in
// all.  Each head's internal children get consecutive 4-wide indices, so the
// child in slot q < ni is the slot-0 child + q.
__device__ __forceinline__ void children4(const int2* __restrict__ child, int i, int ref[4], int& m, int& ni) {
    int tmp[4];
    m = 0;
    const int2 c = child[i];
    const int cs[2] = {c.x, c.y};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (cs[a] < 0) {
            tmp[m++] = cs[a];
        } else {
            const int2 g = child[cs[a]];
            tmp[m++] = g.x;
            tmp[m++] = g.y;
        }
    }
    ni = 0;
    for (int q = 0; q < m; ++q)
        if (tmp[q] >= 0) ref[ni++] = tmp[q];
    int k = ni;
    for (int q = 0; q < m; ++q)
        if (tmp[q] < 0) ref[k++] = tmp[q];
}

// Internal-child count of every head (0 elsewhere).
__global__ void k_count4(const int2* __restrict__ child, const unsigned* __restrict__ flag, int n_inner,
                         unsigned* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inner) return;
    int ref[4], m = 0, ni = 0;
    if (flag[i]) children4(child, i, ref, m, ni);
    cnt[i] = (unsigned)ni;
}

// 4-wide index of every head: 0 for the root, 1 + off[h] + k for the k-th
// internal child of head h (off: exclusive scan of the counts).
__global__ void k_number4(const int2* __restrict__ child, const unsigned* __restrict__ flag,
                          const unsigned* __restrict__ off, int n_inner, unsigned* __restrict__ idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inner || !flag[i]) return;
    if (i == 0) idx[0] = 0u;
    int ref[4], m, ni;
    children4(child, i, ref, m, ni);
    for (int k = 0; k < ni; ++k)
        if ((unsigned)ref[k] < (unsigned)n_inner) idx[ref[k]] = 1u + off[i] + (unsigned)k;
}

// Node of head i at idx[i]: six planes of the four child boxes, the child
// references (internal 4-wide indices, ~leaf, kEmptyRef for unused slots with
// a zero box) and the slot keys: q for an internal child in slot q, all ones
// for the others (the traversal sorts (entry distance | key) as integers).
__global__ void k_pack_nodes4(const int2* __restrict__ child, const float* __restrict__ node_box,
                              const float* __restrict__ leaf_box, const unsigned* __restrict__ flag,
                              const unsigned* __restrict__ off, const unsigned* __restrict__ idx, int n_inner,
                              int n_nodes4, float4* __restrict__ nodes4) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inner || !flag[i]) return;
    const unsigned self = idx[i];
    if (self >= (unsigned)n_nodes4) return;   // unnumbered: a malformed binary tree
    int ref[4], m, ni;
    children4(child, i, ref, m, ni);
    float box[4][6];
    int out[4];
    unsigned key[4];
    for (int k = 0; k < 4; ++k) {
        if (k < m) {
            box_of(ref[k], node_box, leaf_box, box[k]);
            out[k] = k < ni ? (int)(1u + off[i] + (unsigned)k) : ref[k];
        } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) box[k][q] = 0.0f;
            out[k] = kEmptyRef;
        }
        key[k] = k < ni ? (unsigned)k : 0xffffffffu;
    }
    float4* o = nodes4 + 16ll * self;
#pragma unroll
    for (int a = 0; a < 3; ++a) {   // per axis: lo, hi, hi, lo of the four children
        const float4 lo = make_float4(box[0][a], box[1][a], box[2][a], box[3][a]);
        const float4 hi = make_float4(box[0][a + 3], box[1][a + 3], box[2][a + 3], box[3][a + 3]);
        o[4 * a] = lo;
        o[4 * a + 1] = hi;
        o[4 * a + 2] = hi;
        o[4 * a + 3] = lo;
    }
    o[12] = make_float4(__int_as_float(out[0]), __int_as_float(out[1]), __int_as_float(out[2]),
                        __int_as_float(out[3]));
    o[13] = make_float4(__uint_as_float(key[0]), __uint_as_float(key[1]), __uint_as_float(key[2]),
                        __uint_as_float(key[3]));
    o[14] = o[15] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

}  // namespace

size_t tree4_scratch_bytes(int n) {
    const size_t N = (size_t)(n > 1 ? n : 1);
    return N * (2 * sizeof(int) + 4 * sizeof(float4) + sizeof(int) + 4 * sizeof(unsigned)) +
           (size_t)(n > 1 ? n - 1 : 1) * (sizeof(int2) * 2 + 12 * sizeof(float) + sizeof(int32_t)) +
           (size_t)scan_scratch_elems((int)N) * sizeof(unsigned) + 20 * 256;
}

// The scratch block's arrays.  tree4_build leaves the binary tree in child2 /
// nbox2 (root = 0) and the heads' internal-child offsets in pos for
// tree4_pack.
struct Tree4Scratch {
    int *C, *C2;
    float4 *lo, *hi, *lo2, *hi2;
    int* nbr;
    unsigned *keep, *pos, *merge, *moff;
    int2 *child, *child2;
    float *nbox, *nbox2;
    int32_t* parent;
    unsigned* sums;
};

static Tree4Scratch carve(void* scratch, int n) {
    const int n_inner = n - 1;
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    Tree4Scratch t;
    t.C = reinterpret_cast<int*>(take(sizeof(int) * n));
    t.C2 = reinterpret_cast<int*>(take(sizeof(int) * n));
    t.lo = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    t.hi = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    t.lo2 = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    t.hi2 = reinterpret_cast<float4*>(take(sizeof(float4) * n));
    t.nbr = reinterpret_cast<int*>(take(sizeof(int) * n));
    t.keep = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * n));
    t.pos = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * n));
    t.merge = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * n));
    t.moff = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * n));
    t.child = reinterpret_cast<int2*>(take(sizeof(int2) * n_inner));
    t.child2 = reinterpret_cast<int2*>(take(sizeof(int2) * n_inner));
    t.nbox = reinterpret_cast<float*>(take(sizeof(float) * 6 * n_inner));
    t.nbox2 = reinterpret_cast<float*>(take(sizeof(float) * 6 * n_inner));
    t.parent = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n_inner));
    t.sums = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * scan_scratch_elems(n)));
    return t;
}

cudaError_t tree4_build(const LbvhBuffers& b, void* scratch, int radius, cudaStream_t s, int* n_nodes4) {
    if (radius < 1 || radius > kPlocRadiusMax) return cudaErrorInvalidValue;
    const int n = b.n;
    *n_nodes4 = 0;
    if (n <= 1) return cudaSuccess;
    const int n_inner = n - 1;
    const Tree4Scratch sc = carve(scratch, n);
    int* C = sc.C;
    int* C2 = sc.C2;
    float4* lo = sc.lo;
    float4* hi = sc.hi;
    float4* lo2 = sc.lo2;
    float4* hi2 = sc.hi2;
    int* nbr = sc.nbr;
    unsigned* keep = sc.keep;
    unsigned* pos = sc.pos;
    unsigned* merge = sc.merge;
    unsigned* moff = sc.moff;
    int2* child = sc.child;
    int2* child2 = sc.child2;
    float* nbox = sc.nbox;
    float* nbox2 = sc.nbox2;
    int32_t* parent = sc.parent;
    unsigned* sums = sc.sums;
    unsigned* hostv = nullptr;
    cudaError_t e = cudaMallocHost(&hostv, 4 * sizeof(unsigned));
    if (e != cudaSuccess) return e;

    k_ploc_init<<<blocks_for(n, kThreads), kThreads, 0, s>>>(b.leaf_box, n, C, lo, hi);
    count_launch(1);
    int m = n, node_base = 0, rounds = 0;
    while (m > 1 && e == cudaSuccess) {
        if (++rounds > 100000) { e = cudaErrorUnknown; break; }
        const int g = blocks_for(m, kThreads);
        k_ploc_nn<<<g, kThreads, 0, s>>>(lo, hi, m, radius, nbr);
        k_ploc_flags<<<g, kThreads, 0, s>>>(nbr, m, keep, merge);
        count_launch(2);
        e = cudaMemcpyAsync(pos, keep, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(moff, merge, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = exclusive_scan(pos, m, sums, s);
        if (e == cudaSuccess) e = exclusive_scan(moff, m, sums, s);
        if (e != cudaSuccess) break;
        k_ploc_compact<<<g, kThreads, 0, s>>>(C, lo, hi, nbr, keep, pos, merge, moff, m, node_base, C2,
                                              lo2, hi2, child, nbox);
        count_launch(1);
        e = cudaMemcpyAsync(hostv + 0, pos + (m - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hostv + 1, keep + (m - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hostv + 2, moff + (m - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hostv + 3, merge + (m - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        const int m2 = (int)(hostv[0] + hostv[1]);
        const int merged = (int)(hostv[2] + hostv[3]);
        if (merged <= 0 || m2 != m - merged) { e = cudaErrorUnknown; break; }
        node_base += merged;
        m = m2;
        std::swap(C, C2);
        std::swap(lo, lo2);
        std::swap(hi, hi2);
    }
    if (e == cudaSuccess && node_base != n_inner) e = cudaErrorUnknown;
    if (e != cudaSuccess) {
        cudaFreeHost(hostv);
        return e;
    }
    // collapse: heads at even depth, their internal-child counts (in `pos`,
    // free after the rounds) scanned into offsets, then the numbering; the
    // caller allocates the nodes and tree4_pack writes them
    const int g = blocks_for(n_inner, kThreads);
    k_renumber<<<g, kThreads, 0, s>>>(child, nbox, n_inner, child2, nbox2, parent);
    k_depth_heads<<<g, kThreads, 0, s>>>(parent, n_inner, b.head_flag);
    k_count4<<<g, kThreads, 0, s>>>(child2, b.head_flag, n_inner, pos);
    count_launch(3);
    e = cudaMemcpyAsync(hostv + 0, pos + (n_inner - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = exclusive_scan(pos, n_inner, sums, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hostv + 1, pos + (n_inner - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.head_idx, 0xff, sizeof(unsigned) * (size_t)n_inner, s);
    if (e == cudaSuccess) {
        k_number4<<<g, kThreads, 0, s>>>(child2, b.head_flag, pos, n_inner, b.head_idx);
        count_launch(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the count is read next
    if (e == cudaSuccess) {
        const long long n4 = 1ll + hostv[0] + hostv[1];   // the root and every head's internal children
        if (n4 > n_inner) e = cudaErrorUnknown;
        else *n_nodes4 = (int)n4;
    }
    cudaFreeHost(hostv);
    return e;
}

cudaError_t tree4_pack(const LbvhBuffers& b, void* scratch, int n_nodes4, cudaStream_t s) {
    const int n = b.n;
    if (n <= 1) return cudaSuccess;
    const int n_inner = n - 1;
    const Tree4Scratch sc = carve(scratch, n);
    k_pack_nodes4<<<blocks_for(n_inner, kThreads), kThreads, 0, s>>>(sc.child2, sc.nbox2, b.leaf_box, b.head_flag,
                                                                      sc.pos, b.head_idx, n_inner, n_nodes4,
                                                                      b.nodes4);
    count_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the caller frees the scratch next
    return e;
}

}  // namespace vafr
