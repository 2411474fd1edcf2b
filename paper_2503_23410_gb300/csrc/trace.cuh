// trace.cuh -- the ray-casting core shared by the ray-cast (render.cu),
// path-traced (pathtrace.cu) and deferred (raster.cu) pipelines: rays, the
// robust box and watertight triangle tests, LBVH / 4-wide traversal, shading,
// LP ray generation and LP stores.  Everything is inline (or internal to each
// translation unit), so each pipeline's kernels are compiled on their own.
//
// Traversal: single-triangle leaves.  Each binary node holds both child boxes
// and each 4-wide node four, laid out per axis so the slabs run on paired FP32
// instructions.  Box tests follow Ize 2013 ("Robust BVH Ray Traversal"): slab
// distances (b - o) (1/d) and the far distance scaled by 1 + 2 gamma_3, so no
// box the ray touches is culled by rounding.  Triangle test: Woop, Benthin,
// Wald 2013 ("Watertight Ray/Triangle Intersection"), two-sided, with the
// 2-D edge functions evaluated without FMA contraction so that a shared edge
// gets exactly opposite values in the two neighbouring triangles.
// Hit rule: closest t > 0; equal t -> lower triangle id.
#pragma once

#include "vafr_internal.cuh"

#include <float.h>
#include <limits.h>

namespace vafr {
namespace {

constexpr float kAmbient = 0.1f;
constexpr float kFarScale = 1.0000003576278687f;   // 1 + 2 gamma_3 in FP32 (gamma_3 = 3u/(1-3u))
constexpr float kDirEps = 1e-30f;

struct Ray {
    float ox, oy, oz;
    float dx, dy, dz;
    float ix, iy, iz;            // 1/d with zero components clamped (box tests only)
    int nx, ny, nz;              // float4 index of each axis's near plane in a 4-wide node
    float mx0, mx1, mx2;         // shear rows: A'x = Mx . A, A'y = My . A, A'z = Mz . A
    float my0, my1, my2;
    float mz0, mz1, mz2;
    int skip;                    // triangle id the ray ignores (the surface it leaves), or -1
};

__device__ __forceinline__ float safe_inv(float d) {
    if (fabsf(d) < kDirEps) d = copysignf(kDirEps, d);
    return 1.0f / d;
}

__device__ __forceinline__ void ray_setup(Ray& r) {
    r.ix = safe_inv(r.dx);
    r.iy = safe_inv(r.dy);
    r.iz = safe_inv(r.dz);
    // a 4-wide node stores lo, hi, hi, lo per axis: (near, far) is (hi, lo)
    // from the axis's third float4 when 1/d < 0, (lo, hi) from its first otherwise
    r.nx = r.ix < 0.0f ? 2 : 0;
    r.ny = r.iy < 0.0f ? 6 : 4;
    r.nz = r.iz < 0.0f ? 10 : 8;
    const float ax = fabsf(r.dx), ay = fabsf(r.dy), az = fabsf(r.dz);
    const int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = kz == 0 ? r.dx : (kz == 1 ? r.dy : r.dz);
    if (dkz < 0.0f) { const int s = kx; kx = ky; ky = s; }
    const float dkx = kx == 0 ? r.dx : (kx == 1 ? r.dy : r.dz);
    const float dky = ky == 0 ? r.dx : (ky == 1 ? r.dy : r.dz);
    const float Sx = dkx / dkz, Sy = dky / dkz, Sz = 1.0f / dkz;
    // Mx has 1 at kx and -Sx at kz; My has 1 at ky and -Sy at kz; Mz has Sz at kz.
    r.mx0 = kx == 0 ? 1.0f : (kz == 0 ? -Sx : 0.0f);
    r.mx1 = kx == 1 ? 1.0f : (kz == 1 ? -Sx : 0.0f);
    r.mx2 = kx == 2 ? 1.0f : (kz == 2 ? -Sx : 0.0f);
    r.my0 = ky == 0 ? 1.0f : (kz == 0 ? -Sy : 0.0f);
    r.my1 = ky == 1 ? 1.0f : (kz == 1 ? -Sy : 0.0f);
    r.my2 = ky == 2 ? 1.0f : (kz == 2 ? -Sy : 0.0f);
    r.mz0 = kz == 0 ? Sz : 0.0f;
    r.mz1 = kz == 1 ? Sz : 0.0f;
    r.mz2 = kz == 2 ? Sz : 0.0f;
}

// Both child boxes of a node at once (paired FP32).  Slab distances are
// (b - o) (1/d) as in Ize 2013 ("Robust BVH Ray Traversal"): the subtraction
// keeps the sign of b - o exact even for rays parallel to an axis, and the far
// end is scaled by 1 + 2 gamma_3 so a box the ray touches is never culled by
// rounding.  Returns the entry distances (left, right), +inf for a miss.
__device__ __forceinline__ float2 sub2(float a, float b, float o) {
    return __fadd2_rn(make_float2(a, b), make_float2(-o, -o));
}

__device__ __forceinline__ float2 slab2(float4 nx, float4 ny, float4 nz, const Ray& r, float tmax) {
    const float2 ix = make_float2(r.ix, r.ix), iy = make_float2(r.iy, r.iy), iz = make_float2(r.iz, r.iz);
    const float2 x0 = __fmul2_rn(sub2(nx.x, nx.y, r.ox), ix), x1 = __fmul2_rn(sub2(nx.z, nx.w, r.ox), ix);
    const float2 y0 = __fmul2_rn(sub2(ny.x, ny.y, r.oy), iy), y1 = __fmul2_rn(sub2(ny.z, ny.w, r.oy), iy);
    const float2 z0 = __fmul2_rn(sub2(nz.x, nz.y, r.oz), iz), z1 = __fmul2_rn(sub2(nz.z, nz.w, r.oz), iz);
    const float tnl = fmaxf(fmaxf(fminf(x0.x, x1.x), fminf(y0.x, y1.x)), fmaxf(fminf(z0.x, z1.x), 0.0f));
    const float tnr = fmaxf(fmaxf(fminf(x0.y, x1.y), fminf(y0.y, y1.y)), fmaxf(fminf(z0.y, z1.y), 0.0f));
    const float tfl = fminf(fminf(fmaxf(x0.x, x1.x), fmaxf(y0.x, y1.x)), fminf(fmaxf(z0.x, z1.x), tmax));
    const float tfr = fminf(fminf(fmaxf(x0.y, x1.y), fmaxf(y0.y, y1.y)), fminf(fmaxf(z0.y, z1.y), tmax));
    return make_float2(tnl <= tfl * kFarScale ? tnl : INFINITY, tnr <= tfr * kFarScale ? tnr : INFINITY);
}

// Two float4 from one 32-byte aligned address (one 256-bit load).
__device__ __forceinline__ void ldg256(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Three-input FP32 minimum / maximum (one PTX instruction on sm_100 and later;
// same NaN rule as fminf / fmaxf).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The four child boxes of a 4-wide node (two pairs of paired-FP32 slabs), with
// the same robust evaluation as slab2.  Each axis's near and far planes are
// chosen per ray by the sign of 1/d (the near plane of every box is then its
// lo side, or its hi side, for all four children at once), so each child needs
// only the max of three near distances and the min of three far ones.  The
// node stores each axis as lo, hi, hi, lo: the ray's (near, far) pair is one
// 256-bit load at a 32-byte offset fixed per ray.
// Returns the entry distances, +inf for a miss.
__device__ __forceinline__ float4 slab4(const float4* __restrict__ nd, const Ray& r, float tmax) {
    float4 nxp, fxp, nyp, fyp, nzp, fzp;
    ldg256(nd + r.nx, nxp, fxp);
    ldg256(nd + r.ny, nyp, fyp);
    ldg256(nd + r.nz, nzp, fzp);
    const float2 ix = make_float2(r.ix, r.ix), iy = make_float2(r.iy, r.iy), iz = make_float2(r.iz, r.iz);
    const float2 xna = __fmul2_rn(sub2(nxp.x, nxp.y, r.ox), ix), xnb = __fmul2_rn(sub2(nxp.z, nxp.w, r.ox), ix);
    const float2 xfa = __fmul2_rn(sub2(fxp.x, fxp.y, r.ox), ix), xfb = __fmul2_rn(sub2(fxp.z, fxp.w, r.ox), ix);
    const float2 yna = __fmul2_rn(sub2(nyp.x, nyp.y, r.oy), iy), ynb = __fmul2_rn(sub2(nyp.z, nyp.w, r.oy), iy);
    const float2 yfa = __fmul2_rn(sub2(fyp.x, fyp.y, r.oy), iy), yfb = __fmul2_rn(sub2(fyp.z, fyp.w, r.oy), iy);
    const float2 zna = __fmul2_rn(sub2(nzp.x, nzp.y, r.oz), iz), znb = __fmul2_rn(sub2(nzp.z, nzp.w, r.oz), iz);
    const float2 zfa = __fmul2_rn(sub2(fzp.x, fzp.y, r.oz), iz), zfb = __fmul2_rn(sub2(fzp.z, fzp.w, r.oz), iz);
#define VAFR_CHILD(XN, XF, YN, YF, ZN, ZF)                                        \
    ([&]() {                                                                      \
        const float tn = max3f(XN, YN, fmaxf(ZN, 0.0f));                          \
        const float tf = min3f(XF, YF, fminf(ZF, tmax));                          \
        return tn <= tf * kFarScale ? tn : INFINITY;                              \
    }())
    const float t0 = VAFR_CHILD(xna.x, xfa.x, yna.x, yfa.x, zna.x, zfa.x);
    const float t1 = VAFR_CHILD(xna.y, xfa.y, yna.y, yfa.y, zna.y, zfa.y);
    const float t2 = VAFR_CHILD(xnb.x, xfb.x, ynb.x, yfb.x, znb.x, zfb.x);
    const float t3 = VAFR_CHILD(xnb.y, xfb.y, ynb.y, yfb.y, znb.y, zfb.y);
#undef VAFR_CHILD
    return make_float4(t0, t1, t2, t3);
}

// Watertight test; returns t or +inf.
__device__ __forceinline__ float tri_test(const Ray& r, float4 a, float4 b, float4 c) {
    const float Ax0 = __fsub_rn(a.x, r.ox), Ax1 = __fsub_rn(a.y, r.oy), Ax2 = __fsub_rn(a.z, r.oz);
    const float Bx0 = __fsub_rn(b.x, r.ox), Bx1 = __fsub_rn(b.y, r.oy), Bx2 = __fsub_rn(b.z, r.oz);
    const float Cx0 = __fsub_rn(c.x, r.ox), Cx1 = __fsub_rn(c.y, r.oy), Cx2 = __fsub_rn(c.z, r.oz);
    const float Ax = fmaf(r.mx0, Ax0, fmaf(r.mx1, Ax1, __fmul_rn(r.mx2, Ax2)));
    const float Ay = fmaf(r.my0, Ax0, fmaf(r.my1, Ax1, __fmul_rn(r.my2, Ax2)));
    const float Bx = fmaf(r.mx0, Bx0, fmaf(r.mx1, Bx1, __fmul_rn(r.mx2, Bx2)));
    const float By = fmaf(r.my0, Bx0, fmaf(r.my1, Bx1, __fmul_rn(r.my2, Bx2)));
    const float Cx = fmaf(r.mx0, Cx0, fmaf(r.mx1, Cx1, __fmul_rn(r.mx2, Cx2)));
    const float Cy = fmaf(r.my0, Cx0, fmaf(r.my1, Cx1, __fmul_rn(r.my2, Cx2)));
    const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return INFINITY;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return INFINITY;
    const float Az = fmaf(r.mz0, Ax0, fmaf(r.mz1, Ax1, __fmul_rn(r.mz2, Ax2)));
    const float Bz = fmaf(r.mz0, Bx0, fmaf(r.mz1, Bx1, __fmul_rn(r.mz2, Bx2)));
    const float Cz = fmaf(r.mz0, Cx0, fmaf(r.mz1, Cx1, __fmul_rn(r.mz2, Cx2)));
    const float T = fmaf(U, Az, fmaf(V, Bz, __fmul_rn(W, Cz)));
    const float t = __fdiv_rn(T, det);
    return t > 0.0f ? t : INFINITY;
}

struct Hit {
    float t;
    int leaf;   // sorted leaf index, -1 = miss
    int id;     // triangle id
};

template <bool STATS, bool SKIP = false>
__device__ __forceinline__ void test_leaf(const SceneDev& sc, const Ray& r, int k, Hit& h,
                                          unsigned long long* tri_tests) {
    const float4 a = __ldg(sc.leaves + 3ll * k);
    const float4 b = __ldg(sc.leaves + 3ll * k + 1);
    const float4 c = __ldg(sc.leaves + 3ll * k + 2);
    if (STATS) ++*tri_tests;
    const float t = tri_test(r, a, b, c);
    const int id = __float_as_int(a.w);
    if (SKIP && id == r.skip) return;
    if (t < h.t || (t == h.t && t < INFINITY && id < h.id)) {
        h.t = t;
        h.leaf = k;
        h.id = id;
    }
}

// Closest hit through the binary LBVH.  Returns a fault bit (0 = fine).
template <bool STATS>
__device__ unsigned traverse2(const SceneDev& sc, const Ray& r, Hit& h,
                              unsigned long long* node_visits, unsigned long long* box_tests,
                              unsigned long long* tri_tests) {
    h.t = INFINITY;
    h.leaf = -1;
    h.id = INT_MAX;
    if (sc.n_tris <= 0) return 0u;
    if (sc.root < 0) {   // single triangle
        test_leaf<STATS>(sc, r, 0, h, tri_tests);
        return 0u;
    }
    int stack[kStackSize];
    float stack_t[kStackSize];
    int sp = 0;
    int node = sc.root;
    const int n_inner = sc.n_tris - 1;
    unsigned budget = 4u * (unsigned)sc.n_tris + 64u;
    while (true) {
        if (--budget == 0u) return kFaultWatchdog;
        if ((unsigned)node >= (unsigned)n_inner) return kFaultBadNode;
        if (STATS) { ++*node_visits; *box_tests += 2; }
        const float4* nd = sc.nodes + 4ll * node;
        const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        const int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
        const float2 tt = slab2(n0, n1, n2, r, h.t);
        float tl = tt.x, tr = tt.y;
        if (tl < INFINITY && cl < 0) {
            if ((unsigned)~cl >= (unsigned)sc.n_tris) return kFaultBadNode;
            test_leaf<STATS>(sc, r, ~cl, h, tri_tests);
            tl = INFINITY;
        }
        if (tr < INFINITY && cr < 0) {
            if ((unsigned)~cr >= (unsigned)sc.n_tris) return kFaultBadNode;
            test_leaf<STATS>(sc, r, ~cr, h, tri_tests);
            tr = INFINITY;
        }
        const bool hl = tl < INFINITY, hr = tr < INFINITY;
        if (hl && hr) {
            if (sp >= kStackSize) return kFaultStack;
            const bool left_first = tl <= tr;
            stack[sp] = left_first ? cr : cl;
            stack_t[sp] = left_first ? tr : tl;
            ++sp;
            node = left_first ? cl : cr;
        } else if (hl) {
            node = cl;
        } else if (hr) {
            node = cr;
        } else {
            // pop, skipping entries that start beyond the current closest hit
            while (true) {
                if (sp == 0) return 0u;
                --sp;
                if (stack_t[sp] <= h.t * kFarScale) break;
            }
            node = stack[sp];
        }
    }
}

// Ascending order of two sort keys (one integer minimum and one maximum).
__device__ __forceinline__ void sort2(unsigned& a, unsigned& b) {
    const unsigned lo = min(a, b);
    b = max(a, b);
    a = lo;
}

// Sort key of child slot q: its entry distance t >= 0 (+inf for a miss) as
// bits without the sign (a -0 entry is 0), whose unsigned order is the order
// of t, with the two low bits replaced by q for an internal child (key word
// q); a leaf or unused slot has key word all ones and sorts after every miss.
// Keys below kKeyMiss are hit internal children; dropping two bits of t only
// reorders children whose distances agree within 4 ulp, and a stack entry's
// distance, rounded down, only culls later.
constexpr unsigned kKeyMiss = 0x7f800000u;
__device__ __forceinline__ unsigned child_key(float t, unsigned word) {
    return (__float_as_uint(t) & 0x7ffffffcu) | word;
}

// Closest hit through the 4-wide tree: test the four child boxes, test the
// leaf children that were hit, then continue with the nearest internal child
// and push the others far-to-near.  Internal children are ordered by integer
// keys (entry distance bits and slot); they are consecutive nodes, so the
// slot in a key's low bits gives the child's index.  The hit leaf children of
// a node form a bit mask that one loop consumes, so a warp runs as many
// triangle tests per node as its busiest lane needs (not one pass per child
// slot that any lane needs); the closest-hit rule (t, then id) makes the
// result independent of the order.
// Returns a fault bit (0 = fine).
template <bool STATS, int ORDER, bool ANY = false, bool SKIP = false>
__device__ unsigned traverse4(const SceneDev& sc, const Ray& r, Hit& h,
                              unsigned long long* node_visits, unsigned long long* box_tests,
                              unsigned long long* tri_tests) {
    h.t = INFINITY;
    h.leaf = -1;
    h.id = INT_MAX;
    if (sc.n_tris <= 0) return 0u;
    if (sc.root < 0) {   // single triangle
        test_leaf<STATS, SKIP>(sc, r, 0, h, tri_tests);
        return 0u;
    }
    unsigned long long stack[kStackSize];
    int sp = 0;
    int node = 0;
    unsigned budget = 4u * (unsigned)sc.n_tris + 64u;
    while (true) {
        if (--budget == 0u) return kFaultWatchdog;
        if ((unsigned)node >= (unsigned)sc.n_nodes4) return kFaultBadNode;   // the nodes are allocated at their count
        const float4* nd = sc.nodes4 + 16ll * node;
        float4 t = slab4(nd, r, h.t);
        float4 rf, kwf;
        ldg256(nd + 12, rf, kwf);
        const uint4 kw = make_uint4(__float_as_uint(kwf.x), __float_as_uint(kwf.y), __float_as_uint(kwf.z),
                                    __float_as_uint(kwf.w));
        const int c0 = __float_as_int(rf.x), c1 = __float_as_int(rf.y), c2 = __float_as_int(rf.z),
                  c3 = __float_as_int(rf.w);
        if (STATS) {
            ++*node_visits;
            *box_tests += (c0 != kEmptyRef) + (c1 != kEmptyRef) + (c2 != kEmptyRef) + (c3 != kEmptyRef);
        }
        // hit children that are leaves (bit q for child q): references below 0
        // other than kEmptyRef (INT_MIN: an unused slot with a zero box)
        static_assert(kEmptyRef == INT_MIN, "the leaf test below relies on kEmptyRef");
        unsigned lm = 0u;
#define VAFR_LEAF_BIT(T, C, Q)                                                            \
        if (T < INFINITY && (unsigned)C > (unsigned)kEmptyRef) lm |= 1u << Q;
        VAFR_LEAF_BIT(t.x, c0, 0)
        VAFR_LEAF_BIT(t.y, c1, 1)
        VAFR_LEAF_BIT(t.z, c2, 2)
        VAFR_LEAF_BIT(t.w, c3, 3)
#undef VAFR_LEAF_BIT
        const float t_entry = h.t;
        while (lm) {
            const int q = __ffs(lm) - 1;
            lm &= lm - 1u;
            const int C = q == 0 ? c0 : (q == 1 ? c1 : (q == 2 ? c2 : c3));
            if ((unsigned)~C >= (unsigned)sc.n_tris) return kFaultBadNode;
            test_leaf<STATS, SKIP>(sc, r, ~C, h, tri_tests);
        }
        if (ANY && h.leaf >= 0) return 0u;   // occlusion query: any hit ends it
        // children entering beyond a closest hit found at this node are dropped
        // (the box tests already clipped against the hit known before it)
        if (h.t != t_entry) {
            const float lim = h.t * kFarScale;
            if (t.x > lim) t.x = INFINITY;
            if (t.y > lim) t.y = INFINITY;
            if (t.z > lim) t.z = INFINITY;
            if (t.w > lim) t.w = INFINITY;
        }
        unsigned k0 = child_key(t.x, kw.x), k1 = child_key(t.y, kw.y), k2 = child_key(t.z, kw.z),
                 k3 = child_key(t.w, kw.w);
        if (ORDER == 0) {
            // ascending: sorting network (0,1) (2,3) (0,2) (1,3) (1,2)
            sort2(k0, k1);
            sort2(k2, k3);
            sort2(k0, k2);
            sort2(k1, k3);
            sort2(k1, k2);
        } else {
            // nearest first, the rest in slot order: (0,1) (2,3) (0,2)
            sort2(k0, k1);
            sort2(k2, k3);
            sort2(k0, k2);
        }
        if (k0 < kKeyMiss) {
            // a stack entry: the child's entry distance (key bits) high, its index low
#define VAFR_PUSH(K)                                                                      \
            if (K < kKeyMiss) {                                                           \
                if (sp >= kStackSize) return kFaultStack;                                 \
                stack[sp++] = ((unsigned long long)(K & ~3u) << 32) | (unsigned)(c0 + (int)(K & 3u)); \
            }
            VAFR_PUSH(k3)
            VAFR_PUSH(k2)
            VAFR_PUSH(k1)
#undef VAFR_PUSH
            node = c0 + (int)(k0 & 3u);
        } else {
            // pop, skipping entries that start beyond the current closest hit
            const float lim2 = h.t * kFarScale;
            unsigned long long e;
            while (true) {
                if (sp == 0) return 0u;
                e = stack[--sp];
                if (__uint_as_float((unsigned)(e >> 32)) <= lim2) break;
            }
            node = (int)(unsigned)e;
        }
    }
}

// WIDE: 4 (4-wide PLOC tree) or 2 (binary LBVH); ORDER (4-wide only): 0 pushes
// children far-to-near after a full sort, 1 only puts the nearest first.
template <int WIDE, bool STATS, int ORDER = 0>
__device__ __forceinline__ unsigned traverse(const SceneDev& sc, const Ray& r, Hit& h,
                                             unsigned long long* nv, unsigned long long* bt,
                                             unsigned long long* tt) {
    if (WIDE == 4) return traverse4<STATS, ORDER>(sc, r, h, nv, bt, tt);
    return traverse2<STATS>(sc, r, h, nv, bt, tt);
}

// Unshadowed inverse-square point lights added to acc: rgb max(0, n . l) / |x - p|^2
// for each light at x, hit point p.  Kept out of line so that scenes without
// point lights run the traversal kernels' code unchanged.
__device__ __noinline__ float3 point_lights(const float4* plights, int n, float px, float py, float pz, float nx,
                                            float ny, float nz, float3 acc) {
    for (int q = 0; q < n; ++q) {
        const float4 lp = __ldg(plights + 2 * q), lc = __ldg(plights + 2 * q + 1);
        const float lx = lp.x - px, ly = lp.y - py, lz = lp.z - pz;
        const float d2 = fmaf(lx, lx, fmaf(ly, ly, lz * lz));
        const float c = fmaf(nx, lx, fmaf(ny, ly, nz * lz)) * rsqrtf(d2);
        if (c > 0.0f) {
            const float g = c / d2;
            acc.x = fmaf(lc.x, g, acc.x);
            acc.y = fmaf(lc.y, g, acc.y);
            acc.z = fmaf(lc.z, g, acc.z);
        }
    }
    return acc;
}

__device__ __forceinline__ float4 shade(const SceneDev& sc, const Ray& r, const Hit& h) {
    if (h.leaf < 0) {
        const float inv = rsqrtf(fmaf(r.dx, r.dx, fmaf(r.dy, r.dy, r.dz * r.dz)));
        const float s = 0.5f * fmaf(r.dy, inv, 1.0f);
        return make_float4(1.0f - 0.5f * s, 1.0f - 0.3f * s, 1.0f, 1.0f);
    }
    const float4 a = __ldg(sc.leaves + 3ll * h.leaf);
    const float4 b = __ldg(sc.leaves + 3ll * h.leaf + 1);
    const float4 c = __ldg(sc.leaves + 3ll * h.leaf + 2);
    const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    float nx = e1y * e2z - e1z * e2y;
    float ny = e1z * e2x - e1x * e2z;
    float nz = e1x * e2y - e1y * e2x;
    const float inv = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    nx *= inv; ny *= inv; nz *= inv;
    if (fmaf(nx, r.dx, fmaf(ny, r.dy, nz * r.dz)) > 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
    const float lam = fmaxf(0.0f, -fmaf(nx, sc.light[0], fmaf(ny, sc.light[1], nz * sc.light[2])));
    const float s = fmaf(1.0f - kAmbient, lam, kAmbient);
    const float4 al = __ldg(sc.albedo + h.id);
    float3 acc = make_float3(s, s, s);
    if (sc.n_plights > 0)
        acc = point_lights(sc.plights, sc.n_plights, fmaf(h.t, r.dx, r.ox), fmaf(h.t, r.dy, r.oy), fmaf(h.t, r.dz, r.oz), nx, ny, nz, acc);
    return make_float4(al.x * acc.x, al.y * acc.y, al.z * acc.z, 1.0f);
}

__device__ __forceinline__ void store_px(void* base, long long idx, int fmt, float4 v) {
    if (fmt == VAFR_FMT_RGBA16F) {
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        uint2 p;
        p.x = *reinterpret_cast<const unsigned*>(&lo);
        p.y = *reinterpret_cast<const unsigned*>(&hi);
        reinterpret_cast<uint2*>(base)[idx] = p;
    } else {
        reinterpret_cast<float4*>(base)[idx] = v;
    }
}

__device__ __forceinline__ void world_ray(const FrameDesc& f, float cx, float cy, Ray& r) {
    // camera direction (cx, cy, 1) -> world
    r.dx = fmaf(f.R[0], cx, fmaf(f.R[1], cy, f.R[2]));
    r.dy = fmaf(f.R[3], cx, fmaf(f.R[4], cy, f.R[5]));
    r.dz = fmaf(f.R[6], cx, fmaf(f.R[7], cy, f.R[8]));
    r.ox = f.org[0];
    r.oy = f.org[1];
    r.oz = f.org[2];
    r.skip = -1;
}

template <class B>
__device__ __forceinline__ int find_frame(const B& b, long long w, bool tiles) {
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long beg = tiles ? b.d[mid].tile_begin : b.d[mid].work_begin;
        if (beg <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// LP ray of the frame's work item k (Eqs. 3, 10, 11): work items visit the
// texels in screen-space Hilbert order; texel t = (c, j) sits at distance
// r = tan(e_c)/c_r from the gaze at angle phi = (j + 0.5) 360/n_c, so its
// camera direction is (tan(e_c) cos(phi) + gx, -tan(e_c) sin(phi) + gy, 1).
// Returns the texel's slot; `guard_lo` / `guard_hi` get the guard slots that
// copy it (texel n_c - 1 -> slot before the column, texel 0 -> slot after),
// or -1.
__device__ __forceinline__ int lp_ray(const FrameDesc& f, int k, Ray& r, int& guard_lo, int& guard_hi) {
    const int2 tc = __ldg(f.work + k);
    const int2 cc = __ldg(&f.col[tc.y]);
    const int j = tc.x - cc.x;
    const float te = __ldg(&f.tan_e[tc.y]);
    float sp, cp;
    sincospif(__fdiv_rn((float)(2 * j + 1), (float)cc.y), &sp, &cp);
    world_ray(f, fmaf(te, cp, f.gx), fmaf(-te, sp, f.gy), r);
    guard_lo = j == cc.y - 1 ? tc.x - cc.y : -1;
    guard_hi = j == 0 ? tc.x + cc.y : -1;
    return tc.x;
}

// Shaded LP texel (and hit id) into its slot and the guard slots that copy it.
__device__ __forceinline__ void store_lp(const FrameDesc& f, int t, int glo, int ghi, float4 c, int id) {
    store_px(f.lp, t, f.lp_fmt, c);
    if (glo >= 0) store_px(f.lp, glo, f.lp_fmt, c);
    if (ghi >= 0) store_px(f.lp, ghi, f.lp_fmt, c);
    if (f.hit_ids) {
        f.hit_ids[t] = id;
        if (glo >= 0) f.hit_ids[glo] = id;
        if (ghi >= 0) f.hit_ids[ghi] = id;
    }
}

}  // namespace
}  // namespace vafr
