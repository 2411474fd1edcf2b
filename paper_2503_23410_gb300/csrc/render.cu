// render.cu -- ray generation, LBVH traversal and shading (the ray-casting
// pipeline of Sec. 6.1: ray-generation shader dispatched over the LP buffer,
// closest-hit shader, miss shader; and the GT dispatch over display pixels).
//
// Kernels are persistent: a grid of (SMs x resident blocks) whose warps pull
// chunks of work items from one global atomic counter until the batch is done,
// so uneven frames and uneven rays balance dynamically.
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
    // a 4-wide node stores lo then hi per axis: the near plane is hi when 1/d < 0
    r.nx = r.ix < 0.0f ? 1 : 0;
    r.ny = r.iy < 0.0f ? 3 : 2;
    r.nz = r.iz < 0.0f ? 5 : 4;
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

// The four child boxes of a 4-wide node (two pairs of paired-FP32 slabs), with
// the same robust evaluation as slab2.  Each axis's near and far planes are
// chosen per ray by the sign of 1/d (the near plane of every box is then its
// lo side, or its hi side, for all four children at once), so each child needs
// only the max of three near distances and the min of three far ones.
// Returns the entry distances, +inf for a miss.
__device__ __forceinline__ float4 slab4(const float4* __restrict__ nd, const Ray& r, float tmax) {
    const float4 nxp = __ldg(nd + r.nx), fxp = __ldg(nd + (r.nx ^ 1));
    const float4 nyp = __ldg(nd + r.ny), fyp = __ldg(nd + (r.ny ^ 1));
    const float4 nzp = __ldg(nd + r.nz), fzp = __ldg(nd + (r.nz ^ 1));
    const float2 ix = make_float2(r.ix, r.ix), iy = make_float2(r.iy, r.iy), iz = make_float2(r.iz, r.iz);
    const float2 xna = __fmul2_rn(sub2(nxp.x, nxp.y, r.ox), ix), xnb = __fmul2_rn(sub2(nxp.z, nxp.w, r.ox), ix);
    const float2 xfa = __fmul2_rn(sub2(fxp.x, fxp.y, r.ox), ix), xfb = __fmul2_rn(sub2(fxp.z, fxp.w, r.ox), ix);
    const float2 yna = __fmul2_rn(sub2(nyp.x, nyp.y, r.oy), iy), ynb = __fmul2_rn(sub2(nyp.z, nyp.w, r.oy), iy);
    const float2 yfa = __fmul2_rn(sub2(fyp.x, fyp.y, r.oy), iy), yfb = __fmul2_rn(sub2(fyp.z, fyp.w, r.oy), iy);
    const float2 zna = __fmul2_rn(sub2(nzp.x, nzp.y, r.oz), iz), znb = __fmul2_rn(sub2(nzp.z, nzp.w, r.oz), iz);
    const float2 zfa = __fmul2_rn(sub2(fzp.x, fzp.y, r.oz), iz), zfb = __fmul2_rn(sub2(fzp.z, fzp.w, r.oz), iz);
#define VAFR_CHILD(XN, XF, YN, YF, ZN, ZF)                                        \
    ([&]() {                                                                      \
        const float tn = fmaxf(fmaxf(XN, YN), fmaxf(ZN, 0.0f));                   \
        const float tf = fminf(fminf(XF, YF), fminf(ZF, tmax));                   \
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
    const int id = __float_as_int(a.w);
    if (SKIP && id == r.skip) return;
    const float t = tri_test(r, a, b, c);
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

__device__ __forceinline__ void sort2(float& ta, int& ra, float& tb, int& rb) {
    const bool sw = tb < ta;
    const float t = sw ? tb : ta;
    const int q = sw ? rb : ra;
    tb = sw ? ta : tb;
    rb = sw ? ra : rb;
    ta = t;
    ra = q;
}

// Closest hit through the 4-wide tree: test the four child boxes, test leaf
// children at once, then continue with the nearest internal child and push the
// others far-to-near.  Returns a fault bit (0 = fine).
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
    int stack[kStackSize];
    float stack_t[kStackSize];
    int sp = 0;
    int node = 0;
    const int n_inner = sc.n_tris - 1;
    unsigned budget = 4u * (unsigned)sc.n_tris + 64u;
    while (true) {
        if (--budget == 0u) return kFaultWatchdog;
        if ((unsigned)node >= (unsigned)n_inner) return kFaultBadNode;
        const float4* nd = sc.nodes4 + 8ll * node;
        float4 t = slab4(nd, r, h.t);
        const float4 rf = __ldg(nd + 6);
        int c0 = __float_as_int(rf.x), c1 = __float_as_int(rf.y), c2 = __float_as_int(rf.z),
            c3 = __float_as_int(rf.w);
        if (STATS) {
            ++*node_visits;
            *box_tests += (c0 != kEmptyRef) + (c1 != kEmptyRef) + (c2 != kEmptyRef) + (c3 != kEmptyRef);
        }
#define VAFR_LEAF(T, C)                                                                   \
        if (T < INFINITY && C < 0) {                                                      \
            if (C != kEmptyRef) {                                                         \
                if ((unsigned)~C >= (unsigned)sc.n_tris) return kFaultBadNode;            \
                test_leaf<STATS, SKIP>(sc, r, ~C, h, tri_tests);                          \
            }                                                                             \
            T = INFINITY;                                                                 \
        }
        VAFR_LEAF(t.x, c0)
        VAFR_LEAF(t.y, c1)
        VAFR_LEAF(t.z, c2)
        VAFR_LEAF(t.w, c3)
#undef VAFR_LEAF
        if (ANY && h.leaf >= 0) return 0u;   // occlusion query: any hit ends it
        // children entering beyond an updated closest hit are dropped
        const float lim = h.t * kFarScale;
        if (t.x > lim) t.x = INFINITY;
        if (t.y > lim) t.y = INFINITY;
        if (t.z > lim) t.z = INFINITY;
        if (t.w > lim) t.w = INFINITY;
        if (ORDER == 0) {
            // ascending (t, ref): sorting network (0,1) (2,3) (0,2) (1,3) (1,2)
            sort2(t.x, c0, t.y, c1);
            sort2(t.z, c2, t.w, c3);
            sort2(t.x, c0, t.z, c2);
            sort2(t.y, c1, t.w, c3);
            sort2(t.y, c1, t.z, c2);
        } else {
            // nearest first, the rest in slot order: (0,1) (2,3) (0,2)
            sort2(t.x, c0, t.y, c1);
            sort2(t.z, c2, t.w, c3);
            sort2(t.x, c0, t.z, c2);
        }
        if (t.x < INFINITY) {
            if (t.w < INFINITY) {
                if (sp >= kStackSize) return kFaultStack;
                stack[sp] = c3; stack_t[sp] = t.w; ++sp;
            }
            if (t.z < INFINITY) {
                if (sp >= kStackSize) return kFaultStack;
                stack[sp] = c2; stack_t[sp] = t.z; ++sp;
            }
            if (t.y < INFINITY) {
                if (sp >= kStackSize) return kFaultStack;
                stack[sp] = c1; stack_t[sp] = t.y; ++sp;
            }
            node = c0;
        } else {
            while (true) {
                if (sp == 0) return 0u;
                --sp;
                if (stack_t[sp] <= h.t * kFarScale) break;
            }
            node = stack[sp];
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
    if (sc.n_plights > 0) {
        // unshadowed inverse-square point lights: rgb max(0, n . l) / |x - p|^2
        const float px = fmaf(h.t, r.dx, r.ox), py = fmaf(h.t, r.dy, r.oy), pz = fmaf(h.t, r.dz, r.oz);
        for (int q = 0; q < sc.n_plights; ++q) {
            const float4 lp = __ldg(sc.plights + 2 * q), lc = __ldg(sc.plights + 2 * q + 1);
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
    }
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
// texels in screen-space Morton order; texel t = (c, j) sits at distance
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

// ---- path tracing into the LP buffer (Sec. 8) ------------------------------------
// The estimator of the ray-casting pipeline's path-traced counterpart: 1 path
// per LP texel, next-event estimation towards the directional light, no Russian
// roulette, at most `depth` diffuse bounces; every surface Lambertian.  Per
// segment: closest hit (ignoring the surface the ray leaves); a miss adds
// beta * sky(d) and ends the path; at a hit (normal n facing the ray, albedo
// rho) the ray origin for what follows is p + 1e-5 max(1, |p|_inf) n; when
// cos = n . (-L) > 0 a shadow ray towards the light (any hit ends it) decides
// whether beta rho cos is added; then, below the depth limit, the next
// direction is cosine-distributed about n (orthonormal basis of Duff et al.
// 2017) and beta *= rho.  Random numbers: the top 24 bits of SplitMix64's
// output function (Steele, Lea, Flood 2014) applied to seed, texel index and
// 2 k + dim in turn.

__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float pt_uniform(unsigned long long seed_h, unsigned long long texel, int k, int dim) {
    const unsigned long long h = sm64_mix(sm64_mix(seed_h ^ texel) ^ (unsigned long long)(2 * k + dim));
    return (float)(h >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ float3 sky_rgb(float dx, float dy, float dz) {
    const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float s = 0.5f * fmaf(dy, inv, 1.0f);
    return make_float3(1.0f - 0.5f * s, 1.0f - 0.3f * s, 1.0f);
}

// Unit geometric normal of the hit leaf, turned to face the ray.
__device__ __forceinline__ float3 face_normal(const SceneDev& sc, const Ray& r, int leaf) {
    const float4 a = __ldg(sc.leaves + 3ll * leaf);
    const float4 b = __ldg(sc.leaves + 3ll * leaf + 1);
    const float4 c = __ldg(sc.leaves + 3ll * leaf + 2);
    const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    float nx = e1y * e2z - e1z * e2y;
    float ny = e1z * e2x - e1x * e2z;
    float nz = e1x * e2y - e1y * e2x;
    const float inv = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    nx *= inv; ny *= inv; nz *= inv;
    if (fmaf(nx, r.dx, fmaf(ny, r.dy, nz * r.dz)) > 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
    return make_float3(nx, ny, nz);
}

// One path from the primary ray r; returns the radiance, fills sig (depth + 2
// ints: hit id per segment, -1 miss, -2 not traced; then the shadow mask: bit k
// = segment k's shadow ray reached the light, bit 16 + k = it was cast).
template <int ORDER>
__device__ float3 trace_path(const SceneDev& sc, Ray r, unsigned long long seed_h, unsigned long long texel,
                             int depth, int* sig, unsigned* fault) {
    float3 beta = make_float3(1.0f, 1.0f, 1.0f), acc = make_float3(0.0f, 0.0f, 0.0f);
    const float tlx = -sc.light[0], tly = -sc.light[1], tlz = -sc.light[2];
    unsigned mask = 0u;
    int k = 0;
    for (; k <= depth; ++k) {
        ray_setup(r);
        Hit h;
        *fault |= traverse4<false, ORDER, false, true>(sc, r, h, nullptr, nullptr, nullptr);
        if (sig) sig[k] = h.leaf >= 0 ? h.id : -1;
        if (h.leaf < 0) {
            const float3 sky = sky_rgb(r.dx, r.dy, r.dz);
            acc.x = fmaf(beta.x, sky.x, acc.x);
            acc.y = fmaf(beta.y, sky.y, acc.y);
            acc.z = fmaf(beta.z, sky.z, acc.z);
            ++k;
            break;
        }
        const float3 n = face_normal(sc, r, h.leaf);
        float px = fmaf(h.t, r.dx, r.ox), py = fmaf(h.t, r.dy, r.oy), pz = fmaf(h.t, r.dz, r.oz);
        const float off = 1e-5f * fmaxf(1.0f, fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))));
        px = fmaf(off, n.x, px);
        py = fmaf(off, n.y, py);
        pz = fmaf(off, n.z, pz);
        const float4 rho = __ldg(sc.albedo + h.id);
        const float cosl = fmaf(n.x, tlx, fmaf(n.y, tly, n.z * tlz));
        if (cosl > 0.0f) {
            mask |= 1u << (16 + k);   // a shadow ray was cast
            Ray s;
            s.ox = px; s.oy = py; s.oz = pz;
            s.dx = tlx; s.dy = tly; s.dz = tlz;
            s.skip = h.id;
            ray_setup(s);
            Hit hs;
            *fault |= traverse4<false, ORDER, true, true>(sc, s, hs, nullptr, nullptr, nullptr);
            if (hs.leaf < 0) {
                mask |= 1u << k;
                acc.x = fmaf(beta.x * rho.x, cosl, acc.x);
                acc.y = fmaf(beta.y * rho.y, cosl, acc.y);
                acc.z = fmaf(beta.z * rho.z, cosl, acc.z);
            }
        }
        if (k == depth) { ++k; break; }
        const float u1 = pt_uniform(seed_h, texel, k, 0), u2 = pt_uniform(seed_h, texel, k, 1);
        float sp, cp;
        sincospif(2.0f * u2, &sp, &cp);
        const float rr = sqrtf(u1);
        const float lx = rr * cp, ly = rr * sp, lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
        const float sg = copysignf(1.0f, n.z);
        const float aa = -1.0f / (sg + n.z);
        const float bb = n.x * n.y * aa;
        const float t1x = 1.0f + sg * n.x * n.x * aa, t1y = sg * bb, t1z = -sg * n.x;
        const float t2x = bb, t2y = sg + n.y * n.y * aa, t2z = -n.y;
        r.dx = fmaf(lx, t1x, fmaf(ly, t2x, lz * n.x));
        r.dy = fmaf(lx, t1y, fmaf(ly, t2y, lz * n.y));
        r.dz = fmaf(lx, t1z, fmaf(ly, t2z, lz * n.z));
        r.ox = px; r.oy = py; r.oz = pz;
        r.skip = h.id;
        beta.x *= rho.x; beta.y *= rho.y; beta.z *= rho.z;
    }
    if (sig) {
        for (; k <= depth; ++k) sig[k] = -2;
        sig[depth + 1] = (int)mask;
    }
    return acc;
}

template <int TPB, int FETCH, int ORDER, class B>
__global__ void __launch_bounds__(TPB)
k_path_lp(const SceneDev sc, const __grid_constant__ B b, unsigned long long seed, int depth) {
    const int lane = threadIdx.x & 31;
    const unsigned long long seed_h = sm64_mix(seed);
    while (true) {
        unsigned long long base = 0ull;
        if (lane == 0) base = atomicAdd(b.work_counter, (unsigned long long)FETCH);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= b.total_work) break;
#pragma unroll 1
        for (int k = 0; k < FETCH; k += 32) {
            const long long w = (long long)base + k + lane;
            if (w >= b.total_work) break;
            const FrameDesc& f = b.d[find_frame(b, w, false)];
            Ray r;
            int glo, ghi;
            const int local = (int)(w - f.work_begin);
            const int t = lp_ray(f, local, r, glo, ghi);
            const int col = __ldg(f.work + local).y;
            const unsigned long long texel = (unsigned long long)(t - (2 * col + 1));  // oracle (compact) index
            int* sig = f.hit_ids ? f.hit_ids + (long long)t * (depth + 2) : nullptr;
            unsigned fault = 0u;
            const float3 c = trace_path<ORDER>(sc, r, seed_h, texel, depth, sig, &fault);
            if (fault) atomicOr(f.status, fault);
            const float4 v = make_float4(c.x, c.y, c.z, 1.0f);
            store_px(f.lp, t, f.lp_fmt, v);
            if (glo >= 0) store_px(f.lp, glo, f.lp_fmt, v);
            if (ghi >= 0) store_px(f.lp, ghi, f.lp_fmt, v);
        }
    }
}

// Full-resolution path-traced GT: one path per display pixel centre (random
// numbers keyed by the pixel index y W + x), written straight to the display.
template <int TPB, int FETCH, int ORDER, class B>
__global__ void __launch_bounds__(TPB)
k_path_gt(const SceneDev sc, const __grid_constant__ B b, unsigned long long seed, int depth) {
    const int lane = threadIdx.x & 31;
    const unsigned long long seed_h = sm64_mix(seed);
    while (true) {
        unsigned long long base = 0ull;
        if (lane == 0) base = atomicAdd(b.work_counter, (unsigned long long)FETCH);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= b.total_work) break;
#pragma unroll 1
        for (int k = 0; k < FETCH; k += 32) {
            const long long w = (long long)base + k + lane;
            if (w >= b.total_work) break;
            const FrameDesc& f = b.d[find_frame(b, w, false)];
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
            const long long p = (long long)y * f.W + x;
            unsigned fault = 0u;
            const float3 c = trace_path<ORDER>(sc, r, seed_h, (unsigned long long)p, depth, nullptr, &fault);
            if (fault) atomicOr(f.status, fault);
            store_px(f.disp, p, f.disp_fmt, make_float4(c.x, c.y, c.z, 1.0f));
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

// ---- deferred path (Sec. 3.4 / Sec. 5: G-buffer at native resolution, lighting
// in the LP buffer) ------------------------------------------------------------
// The G-buffer is a visibility buffer: per display pixel the 64-bit key
// (hit distance bits << 32) | triangle id of the closest triangle, written by
// a rasteriser whose coverage test is the watertight test of the pixel-centre
// ray (so the buffer equals the GT cast's closest hits exactly); the LP pass
// shades each texel from the pixel under its screen point, the GT pass every
// pixel.

constexpr float kClipZ = 1e-4f;       // camera-space near plane for bounding boxes

__device__ __forceinline__ void pixel_ray(const FrameDesc& f, int x, int y, Ray& r) {
    const float cx = f.cr * ((float)x + 0.5f - 0.5f * (float)f.W);
    const float cy = f.cr * (0.5f * (float)f.H - ((float)y + 0.5f));
    world_ray(f, cx, cy, r);
}

// Camera coordinates R^T (v - o) of a world point.
__device__ __forceinline__ float3 to_camera(const FrameDesc& f, float4 v) {
    const float x = v.x - f.org[0], y = v.y - f.org[1], z = v.z - f.org[2];
    return make_float3(fmaf(f.R[0], x, fmaf(f.R[3], y, f.R[6] * z)),
                       fmaf(f.R[1], x, fmaf(f.R[4], y, f.R[7] * z)),
                       fmaf(f.R[2], x, fmaf(f.R[5], y, f.R[8] * z)));
}

// Pixel bounding box of a triangle's part inside the view frustum: the
// triangle (camera coordinates) is clipped (Sutherland-Hodgman) by z >= kClipZ
// and by the four side planes |x| <= z hx, |y| <= z hy of the display widened
// by two pixels, then projected; the box is widened by one pixel.  False if
// nothing remains.
__device__ __forceinline__ int clip_poly(const float3* in, int n, float3* out, float px, float py, float pz, float pw) {
    // keeps the points with px x + py y + pz z + pw >= 0
    int m = 0;
    for (int e = 0; e < n; ++e) {
        const float3 a = in[e], b = in[e + 1 == n ? 0 : e + 1];
        const float da = fmaf(px, a.x, fmaf(py, a.y, fmaf(pz, a.z, pw)));
        const float db = fmaf(px, b.x, fmaf(py, b.y, fmaf(pz, b.z, pw)));
        if (da >= 0.0f) out[m++] = a;
        if ((da >= 0.0f) != (db >= 0.0f)) {
            const float s = da / (da - db);
            out[m++] = make_float3(fmaf(s, b.x - a.x, a.x), fmaf(s, b.y - a.y, a.y), fmaf(s, b.z - a.z, a.z));
        }
    }
    return m;
}

__device__ __forceinline__ bool tri_bbox(const FrameDesc& f, float3 p[3], int& x0, int& y0, int& x1, int& y1) {
    float3 A[8], Bv[8];
    A[0] = p[0]; A[1] = p[1]; A[2] = p[2];
    const float hx = f.cr * (0.5f * (float)f.W + 2.0f), hy = f.cr * (0.5f * (float)f.H + 2.0f);
    int m = clip_poly(A, 3, Bv, 0.0f, 0.0f, 1.0f, -kClipZ);
    if (m) m = clip_poly(Bv, m, A, -1.0f, 0.0f, hx, 0.0f);
    if (m) m = clip_poly(A, m, Bv, 1.0f, 0.0f, hx, 0.0f);
    if (m) m = clip_poly(Bv, m, A, 0.0f, -1.0f, hy, 0.0f);
    if (m) m = clip_poly(A, m, Bv, 0.0f, 1.0f, hy, 0.0f);
    if (m == 0) return false;
    float lx = INFINITY, ly = INFINITY, hxs = -INFINITY, hys = -INFINITY;
    const float ic = 1.0f / f.cr;
    for (int k = 0; k < m; ++k) {
        const float sx = fmaf(Bv[k].x / Bv[k].z, ic, 0.5f * (float)f.W);
        const float sy = fmaf(-Bv[k].y / Bv[k].z, ic, 0.5f * (float)f.H);
        lx = fminf(lx, sx); hxs = fmaxf(hxs, sx);
        ly = fminf(ly, sy); hys = fmaxf(hys, sy);
    }
    // pixel x covers [x, x + 1): centres in the box, plus a pixel of slack
    const float fx0 = fmaxf(floorf(lx - 0.5f) - 1.0f, 0.0f), fy0 = fmaxf(floorf(ly - 0.5f) - 1.0f, 0.0f);
    const float fx1 = fminf(ceilf(hxs - 0.5f) + 1.0f, (float)(f.W - 1));
    const float fy1 = fminf(ceilf(hys - 0.5f) + 1.0f, (float)(f.H - 1));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return false;
    x0 = (int)fx0; y0 = (int)fy0; x1 = (int)fx1; y1 = (int)fy1;
    return true;
}

// The shear set-up of ray_setup alone (the triangle test needs no box data).
__device__ __forceinline__ void ray_setup_tri(Ray& r) {
    const float ax = fabsf(r.dx), ay = fabsf(r.dy), az = fabsf(r.dz);
    const int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = kz == 0 ? r.dx : (kz == 1 ? r.dy : r.dz);
    if (dkz < 0.0f) { const int s = kx; kx = ky; ky = s; }
    const float dkx = kx == 0 ? r.dx : (kx == 1 ? r.dy : r.dz);
    const float dky = ky == 0 ? r.dx : (ky == 1 ? r.dy : r.dz);
    const float Sx = dkx / dkz, Sy = dky / dkz, Sz = 1.0f / dkz;
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

// Per-triangle raster set-up: world vertices, id, the camera-depth lower
// bound t_lo of any hit (rays are (cx, cy, 1) in camera space, so a hit's
// distance t is its camera depth), and the screen-space pre-filter.
//
// Pre-filter: the three edge functions of the triangle's projection, scaled
// so each is the signed pixel distance to its edge (positive inside).  A pixel
// whose centre is more than `slack` pixels outside an edge cannot be hit by
// its ray.  The slack bounds the gap between the FP32 projection and the FP32
// watertight test: both err by a few units in the last place of the
// coordinates they handle, which in pixel units is ~2^-24 (|s| + (|v| + |o| +
// |v - o|) / (z_min c_r)) for projected coordinates s, world vertices v, eye o
// and nearest depth z_min; the slack takes 2^-16 times that (256x margin)
// plus 1/64 pixel.  Triangles crossing the near plane, degenerate
// projections, or a slack above 2^16 pixels use no filter.
constexpr float kEdgeSlack = 1.0f / 64.0f;
struct TriSetup {
    float4 a, b, c;
    int id;
    float t_lo;               // every hit of the triangle has t >= t_lo
    float ea[3], eb[3], ec[3];  // e_i(x, y) = ea_i x + eb_i y + ec_i
    float slack;
    bool filt;
};

__device__ __forceinline__ float max_abs3(float x, float y, float z) {
    return fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
}

__device__ __forceinline__ void tri_setup(const FrameDesc& f, const float4& a, const float4& b, const float4& c,
                                          const float3 p[3], TriSetup& T) {
    T.a = a; T.b = b; T.c = c;
    T.id = __float_as_int(a.w);
    const float zmin = fminf(p[0].z, fminf(p[1].z, p[2].z));
    const float vmax = fmaxf(max_abs3(a.x, a.y, a.z), fmaxf(max_abs3(b.x, b.y, b.z), max_abs3(c.x, c.y, c.z)));
    const float omax = max_abs3(f.org[0], f.org[1], f.org[2]);
    float dmax = 0.0f;
    for (int k = 0; k < 3; ++k) dmax = fmaxf(dmax, max_abs3(p[k].x, p[k].y, p[k].z));
    // camera depth of a hit is >= zmin; FP32 rounding of depths and of t is
    // far below 2^-12 of the magnitudes involved
    T.t_lo = zmin - ldexpf(fabsf(zmin) + vmax + omax + dmax, -12);
    T.filt = false;
    T.slack = 0.0f;
    if (!(zmin > kClipZ)) return;
    float sx[3], sy[3];
    const float ic = 1.0f / f.cr;
    float M = 0.5f * (float)max(f.W, f.H);
    for (int k = 0; k < 3; ++k) {
        sx[k] = fmaf(p[k].x / p[k].z, ic, 0.5f * (float)f.W);
        sy[k] = fmaf(-p[k].y / p[k].z, ic, 0.5f * (float)f.H);
        M = fmaxf(M, fmaxf(fabsf(sx[k]), fabsf(sy[k])));
    }
    const float area = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0]);
    T.slack = kEdgeSlack + ldexpf(M + (vmax + omax + dmax) / (zmin * f.cr), -16);
    if (!(isfinite(area) && fabsf(area) > 1e-6f && T.slack < 65536.0f)) return;
    const float sg = area > 0.0f ? 1.0f : -1.0f;
    for (int k = 0; k < 3; ++k) {
        const int q = k == 2 ? 0 : k + 1;
        const float ex = sx[q] - sx[k], ey = sy[q] - sy[k];
        const float inv = sg * rsqrtf(fmaxf(fmaf(ex, ex, ey * ey), 1e-30f));
        // e = (ex (y - sy_k) - ey (x - sx_k)) / |edge|, positive inside
        T.ea[k] = -ey * inv;
        T.eb[k] = ex * inv;
        T.ec[k] = (ey * sx[k] - ex * sy[k]) * inv;
    }
    T.filt = true;
}

__device__ __forceinline__ bool maybe_inside(const TriSetup& T, int x, int y) {
    if (!T.filt) return true;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    return fmaf(T.ea[0], px, fmaf(T.eb[0], py, T.ec[0])) > -T.slack &&
           fmaf(T.ea[1], px, fmaf(T.eb[1], py, T.ec[1])) > -T.slack &&
           fmaf(T.ea[2], px, fmaf(T.eb[2], py, T.ec[2])) > -T.slack;
}

// Exact coverage of pixel (x, y): skipped when the pixel already holds a hit
// nearer than any of the triangle's (a stale read only costs a test), else
// the pixel ray's watertight test and an atomic minimum of the key.
__device__ __forceinline__ void raster_pixel(const FrameDesc& f, unsigned long long* vbuf, int x, int y,
                                             const TriSetup& T) {
    unsigned long long* px = vbuf + (long long)y * f.W + x;
    const unsigned long long cur = __ldcg(px);
    if (__uint_as_float((unsigned)(cur >> 32)) < T.t_lo) return;   // sky (~0) reads as NaN: never skipped
    Ray r;
    pixel_ray(f, x, y, r);
    ray_setup_tri(r);
    const float t = tri_test(r, T.a, T.b, T.c);
    if (t < INFINITY) {
        const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)T.id;
        if (key < cur) atomicMin(px, key);
    }
}

// Large triangles are split into kTileW x kTileH pixel tiles of their boxes.
// One 64-bit counter hands out (record slot << kTileBits) | first tile, so the
// records' first tiles increase with the slot: the tile pass finds a tile's
// record by binary search.  n_tris < 2^30 bounds the slots; a tile sum that
// would pass 2^kTileBits is reported as a fault.
constexpr int kSmallTriPixels = 64;   // larger boxes go to the tile pass
constexpr int kTileW = 16, kTileH = 8;
constexpr int kTileBits = 34;
constexpr unsigned long long kTileMask = (1ull << kTileBits) - 1;

// Pass 1: one thread per triangle; small boxes are rasterised here, large
// ones recorded for pass 2.
__global__ void __launch_bounds__(256)
k_vbuf_raster(const SceneDev sc, const __grid_constant__ SmallBatch b, unsigned long long* vbuf, int4* big,
              int* big_leaf, long long* big_first, unsigned long long* counter, unsigned big_cap) {
    const FrameDesc& f = b.d[0];
    for (int k = blockIdx.x * 256 + threadIdx.x; k < sc.n_tris; k += gridDim.x * 256) {
        const float4 a = __ldg(sc.leaves + 3ll * k), bb = __ldg(sc.leaves + 3ll * k + 1),
                     c = __ldg(sc.leaves + 3ll * k + 2);
        float3 p[3] = {to_camera(f, a), to_camera(f, bb), to_camera(f, c)};
        if (p[0].z <= 0.0f && p[1].z <= 0.0f && p[2].z <= 0.0f) continue;   // behind the eye
        int x0, y0, x1, y1;
        if (!tri_bbox(f, p, x0, y0, x1, y1)) continue;
        const int w = x1 - x0 + 1, h = y1 - y0 + 1;
        if (w * h <= kSmallTriPixels) {
            TriSetup T;
            tri_setup(f, a, bb, c, p, T);
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x)
                    if (maybe_inside(T, x, y)) raster_pixel(f, vbuf, x, y, T);
        } else {
            const unsigned long long nt =
                (unsigned long long)((w + kTileW - 1) / kTileW) * (unsigned long long)((h + kTileH - 1) / kTileH);
            const unsigned long long old = atomicAdd(counter, (1ull << kTileBits) | nt);
            const unsigned long long slot = old >> kTileBits, first = old & kTileMask;
            if (slot < big_cap && first + nt <= kTileMask) {
                big[slot] = make_int4(x0, y0, x1, y1);
                big_leaf[slot] = k;
                big_first[slot] = (long long)first;
            } else {
                atomicOr(f.status, kFaultBadNode);   // list overflow: reported, never silent
            }
        }
    }
}

// Pass 2: every warp takes an equal run of consecutive tiles; a tile's 128
// pixels are four rows of 16 x 2 lanes.  Records are checked against the
// display and the scene before use, so a list damaged by an overflow (already
// reported by pass 1) cannot lead out of bounds.
__global__ void __launch_bounds__(256)
k_vbuf_tiles(const SceneDev sc, const __grid_constant__ SmallBatch b, unsigned long long* vbuf, const int4* big,
             const int* big_leaf, const long long* big_first, const unsigned long long* counter, unsigned big_cap) {
    const FrameDesc& f = b.d[0];
    const unsigned long long cnt = *counter;
    const long long total = (long long)(cnt & kTileMask);
    const long long n_rec = min((long long)(cnt >> kTileBits), (long long)big_cap);
    if (n_rec <= 0 || total <= 0) return;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long g0 = total * warp / n_warps, g1 = total * (warp + 1) / n_warps;
    if (g0 >= g1) return;
    long long lo = 0, hi = n_rec - 1;   // last record whose first tile is <= g0
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (__ldg(big_first + mid) <= g0) lo = mid; else hi = mid - 1;
    }
    long long rec = -1, first = 0;
    int4 bx = make_int4(0, 0, -1, -1);
    int ntx = 1, nt = 0;
    TriSetup T;
    for (long long g = g0; g < g1; ++g) {
        while (lo + 1 < n_rec && __ldg(big_first + lo + 1) <= g) ++lo;
        if (lo != rec) {
            rec = lo;
            first = __ldg(big_first + rec);
            bx = __ldg(big + rec);
            const int k = __ldg(big_leaf + rec);
            nt = 0;
            if (k >= 0 && k < sc.n_tris && bx.x >= 0 && bx.y >= 0 && bx.x <= bx.z && bx.y <= bx.w &&
                bx.z < f.W && bx.w < f.H) {
                const float4 a = __ldg(sc.leaves + 3ll * k), bb = __ldg(sc.leaves + 3ll * k + 1),
                             c = __ldg(sc.leaves + 3ll * k + 2);
                const float3 p[3] = {to_camera(f, a), to_camera(f, bb), to_camera(f, c)};
                tri_setup(f, a, bb, c, p, T);
                ntx = (bx.z - bx.x + kTileW) / kTileW;
                nt = ntx * ((bx.w - bx.y + kTileH) / kTileH);
            }
        }
        const long long t = g - first;
        if (t < 0 || t >= nt) continue;
        const int tx = bx.x + (int)(t % ntx) * kTileW, ty = bx.y + (int)(t / ntx) * kTileH;
        const int x = tx + (lane & 15);
        if (T.filt) {
            // whole tile outside one edge (at the tile's pixel-centre corner
            // that maximises it, with twice the slack): skip
            const float cx0 = (float)tx + 0.5f, cx1 = (float)min(tx + kTileW - 1, bx.z) + 0.5f;
            const float cy0 = (float)ty + 0.5f, cy1 = (float)min(ty + kTileH - 1, bx.w) + 0.5f;
            bool out = false;
            for (int e = 0; e < 3; ++e)
                out |= fmaf(T.ea[e], T.ea[e] > 0.0f ? cx1 : cx0, fmaf(T.eb[e], T.eb[e] > 0.0f ? cy1 : cy0, T.ec[e])) <=
                       -2.0f * T.slack;
            if (out) continue;
        }
        if (x > bx.z) continue;
#pragma unroll
        for (int i = 0; i < kTileH / 2; ++i) {
            const int y = ty + (lane >> 4) + 2 * i;
            if (y <= bx.w && maybe_inside(T, x, y)) raster_pixel(f, vbuf, x, y, T);
        }
    }
}

// Shading of display pixel (x, y) from the visibility buffer (the GT cast's
// shading of that pixel: its ray, hit distance and triangle).
__device__ __forceinline__ float4 shade_vbuf(const SceneDev& sc, const FrameDesc& f, const unsigned long long* vbuf,
                                             const int* leaf_of, int x, int y) {
    Ray r;
    pixel_ray(f, x, y, r);
    const unsigned long long key = vbuf[(long long)y * f.W + x];
    Hit h;
    if (key == ~0ull) {
        h.leaf = -1;
        h.id = -1;
        h.t = INFINITY;
    } else {
        h.id = (int)(unsigned)(key & 0xffffffffu);
        h.t = __uint_as_float((unsigned)(key >> 32));
        h.leaf = __ldg(leaf_of + h.id);
    }
    return shade(sc, r, h);
}

// LP lighting: texel -> the pixel under its screen point (clamped to the
// display) -> that pixel's shading.
__global__ void __launch_bounds__(256)
k_shade_lp_vbuf(const SceneDev sc, const __grid_constant__ SmallBatch b, const unsigned long long* vbuf,
                const int* leaf_of) {
    const FrameDesc& f = b.d[0];
    for (int k = blockIdx.x * 256 + threadIdx.x; k < f.n_texels; k += gridDim.x * 256) {
        const int2 tc = __ldg(f.work + k);
        const int2 cc = __ldg(&f.col[tc.y]);
        const int j = tc.x - cc.x;
        const float te = __ldg(&f.tan_e[tc.y]);
        float sp, cp;
        sincospif(__fdiv_rn((float)(2 * j + 1), (float)cc.y), &sp, &cp);
        const float cx = fmaf(te, cp, f.gx), cy = fmaf(-te, sp, f.gy);
        const float sx = fmaf(cx, 1.0f / f.cr, 0.5f * (float)f.W), sy = fmaf(-cy, 1.0f / f.cr, 0.5f * (float)f.H);
        const int x = min(max((int)floorf(sx), 0), f.W - 1), y = min(max((int)floorf(sy), 0), f.H - 1);
        const float4 v = shade_vbuf(sc, f, vbuf, leaf_of, x, y);
        store_px(f.lp, tc.x, f.lp_fmt, v);
        if (j == 0) store_px(f.lp, tc.x + cc.y, f.lp_fmt, v);
        if (j == cc.y - 1) store_px(f.lp, tc.x - cc.y, f.lp_fmt, v);
    }
}

// Full-resolution lighting (the deferred GT).
__global__ void __launch_bounds__(256)
k_shade_gt_vbuf(const SceneDev sc, const __grid_constant__ SmallBatch b, const unsigned long long* vbuf,
                const int* leaf_of) {
    const FrameDesc& f = b.d[0];
    const long long n = (long long)f.W * f.H;
    for (long long p = blockIdx.x * 256ll + threadIdx.x; p < n; p += gridDim.x * 256ll) {
        const int y = (int)(p / f.W), x = (int)(p - (long long)y * f.W);
        store_px(f.disp, p, f.disp_fmt, shade_vbuf(sc, f, vbuf, leaf_of, x, y));
    }
}

__global__ void k_leaf_of(const float4* leaves, int n, int* leaf_of) {
    for (int k = blockIdx.x * 256 + threadIdx.x; k < n; k += gridDim.x * 256)
        leaf_of[__float_as_int(leaves[3ll * k].w)] = k;
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

template <bool GT, class B>
cudaError_t launch_path_one(const SceneDev& sc, const B& b, unsigned long long seed, int depth, cudaStream_t s,
                            int num_sms) {
    if (b.total_work <= 0) return cudaSuccess;
    constexpr int TPB = 128, FETCH = 32;
    auto kern = GT ? k_path_gt<TPB, FETCH, 1, B> : k_path_lp<TPB, FETCH, 1, B>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    e = cudaMemsetAsync(b.work_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const long long want_warps = (b.total_work + FETCH - 1) / FETCH;
    long long grid = (long long)per_sm * num_sms;
    const long long need = (want_warps * 32 + TPB - 1) / TPB;
    if (need < grid) grid = need < 1 ? 1 : need;
    kern<<<(unsigned)grid, TPB, 0, s>>>(sc, b, seed, depth);
    count_launch(1);
    return cudaGetLastError();
}

template <bool GT, class B>
cudaError_t launch_variant(const SceneDev& sc, const B& b, int variant, cudaStream_t s, int sms) {
    if (b.total_work <= 0) return cudaSuccess;
    // (threads per block, rays per warp fetch, tree width, child order, min blocks/SM)
    switch (variant) {
        case 0: return launch_one<128, 32, 4, 1, 1, GT>(sc, b, s, sms);
        case 1: return launch_one<256, 32, 4, 0, 1, GT>(sc, b, s, sms);
        case 2: return launch_one<128, 32, 4, 0, 1, GT>(sc, b, s, sms);
        case 3: return launch_one<128, 32, 2, 0, 1, GT>(sc, b, s, sms);
        case 4: return launch_one<128, 32, 4, 0, 10, GT>(sc, b, s, sms);
        default: return launch_one<128, 32, 4, 1, 10, GT>(sc, b, s, sms);
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

template <class B>
cudaError_t launch_path_lp(const SceneDev& scene, const B& batch, unsigned long long seed, int depth,
                           cudaStream_t s, int num_sms) {
    return launch_path_one<false>(scene, batch, seed, depth, s, num_sms);
}
template <class B>
cudaError_t launch_path_gt(const SceneDev& scene, const B& batch, unsigned long long seed, int depth,
                           cudaStream_t s, int num_sms) {
    return launch_path_one<true>(scene, batch, seed, depth, s, num_sms);
}
template cudaError_t launch_path_gt<SmallBatch>(const SceneDev&, const SmallBatch&, unsigned long long, int,
                                                cudaStream_t, int);
template cudaError_t launch_path_lp<SmallBatch>(const SceneDev&, const SmallBatch&, unsigned long long, int,
                                                cudaStream_t, int);
template cudaError_t launch_path_lp<BigBatch>(const SceneDev&, const BigBatch&, unsigned long long, int,
                                              cudaStream_t, int);

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

cudaError_t launch_vbuffer(const SceneDev& sc, const SmallBatch& b, const VbufScratch& v, cudaStream_t s,
                           int num_sms) {
    const FrameDesc& f = b.d[0];
    cudaError_t e = cudaMemsetAsync(v.vbuf, 0xff, sizeof(unsigned long long) * (size_t)f.W * f.H, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(v.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if (sc.n_tris <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)min((sc.n_tris + 255) / 256, num_sms * 16);
    k_vbuf_raster<<<grid, 256, 0, s>>>(sc, b, v.vbuf, v.big, v.big_leaf, v.big_first, v.counter, v.big_cap);
    k_vbuf_tiles<<<(unsigned)(num_sms * 8), 256, 0, s>>>(sc, b, v.vbuf, v.big, v.big_leaf, v.big_first, v.counter,
                                                          v.big_cap);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_leaf_of(const SceneDev& sc, int* leaf_of, cudaStream_t s, int num_sms) {
    if (sc.n_tris <= 0) return cudaSuccess;
    k_leaf_of<<<(unsigned)min((sc.n_tris + 255) / 256, num_sms * 16), 256, 0, s>>>(sc.leaves, sc.n_tris, leaf_of);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_shade_vbuf(const SceneDev& sc, const SmallBatch& b, const unsigned long long* vbuf,
                              const int* leaf_of, bool full_res, cudaStream_t s, int num_sms) {
    if (full_res) {
        const long long n = (long long)b.d[0].W * b.d[0].H;
        k_shade_gt_vbuf<<<(unsigned)min((n + 255) / 256, (long long)num_sms * 16), 256, 0, s>>>(sc, b, vbuf, leaf_of);
    } else {
        k_shade_lp_vbuf<<<(unsigned)min((b.d[0].n_texels + 255) / 256, num_sms * 16), 256, 0, s>>>(sc, b, vbuf, leaf_of);
    }
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
