// raster.cu -- the deferred pipeline (Sec. 3.4, Sec. 5): a visibility buffer
// rasterised at display resolution whose coverage test is the GT cast's, and
// lighting from it in the LP buffer or at every pixel.
#include "trace.cuh"

namespace vafr {
namespace {

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
    // the same five planes on the vertices: all outside one plane -> nothing
    // to draw; all inside every plane -> the vertices are the polygon
    unsigned in_all = 0x1fu, out_any = 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 v = p[k];
        const unsigned in = (v.z - kClipZ >= 0.0f ? 1u : 0u) | (fmaf(v.z, hx, -v.x) >= 0.0f ? 2u : 0u) |
                            (fmaf(v.z, hx, v.x) >= 0.0f ? 4u : 0u) | (fmaf(v.z, hy, -v.y) >= 0.0f ? 8u : 0u) |
                            (fmaf(v.z, hy, v.y) >= 0.0f ? 16u : 0u);
        in_all &= in;
        out_any |= in;
    }
    if (out_any != 0x1fu) return false;   // some plane has every vertex outside
    int m;
    if (in_all == 0x1fu) {
        Bv[0] = p[0]; Bv[1] = p[1]; Bv[2] = p[2];
        m = 3;
    } else {
        m = clip_poly(A, 3, Bv, 0.0f, 0.0f, 1.0f, -kClipZ);
        if (m) m = clip_poly(Bv, m, A, -1.0f, 0.0f, hx, 0.0f);
        if (m) m = clip_poly(A, m, Bv, 1.0f, 0.0f, hx, 0.0f);
        if (m) m = clip_poly(Bv, m, A, 0.0f, -1.0f, hy, 0.0f);
        if (m) m = clip_poly(A, m, Bv, 0.0f, 1.0f, hy, 0.0f);
        if (m == 0) return false;
    }
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

// The watertight test of trace.cuh's tri_test with the three vertex-minus-
// origin differences already formed (every pixel ray of a frame starts at the
// eye, so they are per triangle): the same FP32 operations in the same order,
// hence the same t bit for bit.
__device__ __forceinline__ float tri_test_rel(const Ray& r, float3 A, float3 B, float3 C) {
    const float Ax = fmaf(r.mx0, A.x, fmaf(r.mx1, A.y, __fmul_rn(r.mx2, A.z)));
    const float Ay = fmaf(r.my0, A.x, fmaf(r.my1, A.y, __fmul_rn(r.my2, A.z)));
    const float Bx = fmaf(r.mx0, B.x, fmaf(r.mx1, B.y, __fmul_rn(r.mx2, B.z)));
    const float By = fmaf(r.my0, B.x, fmaf(r.my1, B.y, __fmul_rn(r.my2, B.z)));
    const float Cx = fmaf(r.mx0, C.x, fmaf(r.mx1, C.y, __fmul_rn(r.mx2, C.z)));
    const float Cy = fmaf(r.my0, C.x, fmaf(r.my1, C.y, __fmul_rn(r.my2, C.z)));
    const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return INFINITY;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return INFINITY;
    const float Az = fmaf(r.mz0, A.x, fmaf(r.mz1, A.y, __fmul_rn(r.mz2, A.z)));
    const float Bz = fmaf(r.mz0, B.x, fmaf(r.mz1, B.y, __fmul_rn(r.mz2, B.z)));
    const float Cz = fmaf(r.mz0, C.x, fmaf(r.mz1, C.y, __fmul_rn(r.mz2, C.z)));
    const float T = fmaf(U, Az, fmaf(V, Bz, __fmul_rn(W, Cz)));
    const float t = __fdiv_rn(T, det);
    return t > 0.0f ? t : INFINITY;
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
    float3 A, B, C;           // vertices minus the eye, as the watertight test forms them
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
    T.A = make_float3(__fsub_rn(a.x, f.org[0]), __fsub_rn(a.y, f.org[1]), __fsub_rn(a.z, f.org[2]));
    T.B = make_float3(__fsub_rn(b.x, f.org[0]), __fsub_rn(b.y, f.org[1]), __fsub_rn(b.z, f.org[2]));
    T.C = make_float3(__fsub_rn(c.x, f.org[0]), __fsub_rn(c.y, f.org[1]), __fsub_rn(c.z, f.org[2]));
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
// Counters of the instrumented (STATS) rasteriser launch: pre-filter
// evaluations (box pixels outside culled tiles), pixels past the pre-filter,
// exact tests run (past the depth pre-test), atomic minima issued.
struct RasterCounts {
    unsigned long long box_px, filtered, tests, atomics;
};

template <bool STATS>
__device__ __forceinline__ void raster_pixel(const FrameDesc& f, unsigned long long* vbuf, int x, int y,
                                             const TriSetup& T, RasterCounts& n) {
    unsigned long long* px = vbuf + (long long)y * f.W + x;
    const unsigned long long cur = *px;   // may be stale in L1: values only decrease
    if (__uint_as_float((unsigned)(cur >> 32)) < T.t_lo) return;   // sky (~0) reads as NaN: never skipped
    if (STATS) ++n.tests;
    Ray r;
    pixel_ray(f, x, y, r);
    ray_setup_tri(r);
    const float t = tri_test_rel(r, T.A, T.B, T.C);
    if (t < INFINITY) {
        const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)T.id;
        if (key < cur) {
            atomicMin(px, key);
            if (STATS) ++n.atomics;
        }
    }
}

template <bool STATS>
__device__ __forceinline__ void raster_if(const FrameDesc& f, unsigned long long* vbuf, int x, int y,
                                          const TriSetup& T, RasterCounts& n) {
    if (STATS) ++n.box_px;
    if (!maybe_inside(T, x, y)) return;
    if (STATS) ++n.filtered;
    raster_pixel<STATS>(f, vbuf, x, y, T, n);
}

template <bool STATS>
__device__ __forceinline__ void flush_counts(const RasterCounts& n, unsigned long long* stats) {
    if (!STATS || stats == nullptr) return;
    atomicAdd(stats + 0, n.box_px);
    atomicAdd(stats + 1, n.filtered);
    atomicAdd(stats + 2, n.tests);
    atomicAdd(stats + 3, n.atomics);
}

// Large triangles are split into kTileW x kTileH pixel tiles of their boxes.
// One 64-bit counter hands out (record slot << kTileBits) | first tile, so the
// records' first tiles increase with the slot: the tile pass finds a tile's
// record by binary search.  n_tris < 2^30 bounds the slots; a tile sum that
// would pass 2^kTileBits is reported as a fault.
constexpr int kSmallTriPixels = 128;  // larger boxes go to the tile pass
constexpr int kTileW = 16, kTileH = 8;
constexpr int kTileRows = 32 / kTileW;   // tile rows a warp covers per pass
static_assert(32 % kTileW == 0 && kTileH % kTileRows == 0, "tile shape");
constexpr int kTileBits = 34;
constexpr unsigned long long kTileMask = (1ull << kTileBits) - 1;

// Pass 1: one thread per triangle; small boxes are rasterised here, large
// ones recorded for pass 2.
template <bool STATS>
__global__ void __launch_bounds__(256)
k_vbuf_raster(const SceneDev sc, const __grid_constant__ SmallBatch b, unsigned long long* vbuf, int4* big,
              int* big_leaf, long long* big_first, unsigned long long* counter, unsigned big_cap,
              unsigned long long* stats) {
    const FrameDesc& f = b.d[0];
    RasterCounts n{};
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
                for (int x = x0; x <= x1; ++x) raster_if<STATS>(f, vbuf, x, y, T, n);
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
    flush_counts<STATS>(n, stats);
}

// Pass 2: every warp takes an equal run of consecutive tiles; a tile's 128
// pixels are four rows of 16 x 2 lanes.  Records are checked against the
// display and the scene before use, so a list damaged by an overflow (already
// reported by pass 1) cannot lead out of bounds.
template <bool STATS>
__global__ void __launch_bounds__(256, 4)
k_vbuf_tiles(const SceneDev sc, const __grid_constant__ SmallBatch b, unsigned long long* vbuf, const int4* big,
             const int* big_leaf, const long long* big_first, const unsigned long long* counter, unsigned big_cap,
             unsigned long long* stats) {
    const FrameDesc& f = b.d[0];
    RasterCounts n{};
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
        const int ti = (int)t;   // < nt <= 2^23: 32-bit division
        const int tx = bx.x + (ti % ntx) * kTileW, ty = bx.y + (ti / ntx) * kTileH;
        const int x = tx + lane % kTileW;
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
        for (int i = 0; i < kTileH / kTileRows; ++i) {
            const int y = ty + lane / kTileW + kTileRows * i;
            if (y <= bx.w) raster_if<STATS>(f, vbuf, x, y, T, n);
        }
    }
    flush_counts<STATS>(n, stats);
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

}  // namespace

cudaError_t launch_vbuffer(const SceneDev& sc, const SmallBatch& b, const VbufScratch& v, cudaStream_t s,
                           int num_sms, unsigned long long* stats) {
    const FrameDesc& f = b.d[0];
    cudaError_t e = cudaMemsetAsync(v.vbuf, 0xff, sizeof(unsigned long long) * (size_t)f.W * f.H, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(v.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if (sc.n_tris <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)min((sc.n_tris + 255) / 256, num_sms * 16);
    const unsigned tgrid = (unsigned)(num_sms * 8);
    if (stats) {
        k_vbuf_raster<true><<<grid, 256, 0, s>>>(sc, b, v.vbuf, v.big, v.big_leaf, v.big_first, v.counter,
                                                  v.big_cap, stats);
        k_vbuf_tiles<true><<<tgrid, 256, 0, s>>>(sc, b, v.vbuf, v.big, v.big_leaf, v.big_first, v.counter,
                                                  v.big_cap, stats);
    } else {
        k_vbuf_raster<false><<<grid, 256, 0, s>>>(sc, b, v.vbuf, v.big, v.big_leaf, v.big_first, v.counter,
                                                   v.big_cap, nullptr);
        k_vbuf_tiles<false><<<tgrid, 256, 0, s>>>(sc, b, v.vbuf, v.big, v.big_leaf, v.big_first, v.counter,
                                                   v.big_cap, nullptr);
    }
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

}  // namespace vafr
