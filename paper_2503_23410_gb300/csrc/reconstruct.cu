// reconstruct.cu -- the inverse-mapping pass (Sec. 3.4): every display pixel is
// mapped forward to LP coordinates and filtered bilinearly from the LP buffer.
//
// Per pixel centre p = (x + 0.5, y + 0.5):
//   d = p - gaze, computed as (x - floor(x0)) + (0.5 - frac(x0)) so the FP32
//       offset is exact near the gaze even at 16K;
//   z = c_r |d| = tan(e) (Eq. 3; |d| by the hardware square-root
//       approximation), clamped to tan(e_max);
//   u(e(z)) - 1/2 (Eq. 12) from a per-acuity table of cubic Hermite pieces on
//       2,048 uniform intervals of z, built in FP64 on the host from the exact
//       u(e) and du/dz (interpolation error < 1e-5 texel, below FP32 rounding);
//   angle fraction = atan2(dy, dx) / 2pi in [0, 1), by octant reduction and an
//       odd degree-15 polynomial for atan(t)/2pi on [0, 1] (near-minimax fit by
//       Lawson's reweighted least squares, csrc/fit_atan.py; |err| < 3e-8);
//   columns c0 = floor(u - 0.5) and c0 + 1 (one 16-byte load of the
//       column-pair table, whose entries -1 and C - 1 pair a column with
//       itself, so u below the first or past the last column centre clamps
//       without arithmetic); in each column rows floor(frac n_c - 0.5) and +1
//       wrapped modulo n_c -- two adjacent slots thanks to the column's guard
//       slots; bilinear blend in FP32.
// Two kernel families compute exactly these operations: row tiles (a thread
// takes PX pixels of a row) and column runs (a thread takes R pixels of a
// column and reuses table entries and LP texels between them).  The LP buffer
// (8-17 MB per eye) and the tables stay cache-resident; display writes go to HBM.
#include "lp_map.cuh"
#include "vafr_internal.cuh"

#include <limits.h>

namespace vafr {
namespace {

// Texel as two channel pairs, so the filter runs on paired FP32 instructions.
struct px2 {
    float2 rg, ba;
};

__device__ __forceinline__ px2 load_lp(const void* lp, int fmt, int idx) {
    px2 r;
    if (fmt == VAFR_FMT_RGBA16F) {
        const uint2 p = __ldg(reinterpret_cast<const uint2*>(lp) + idx);
        r.rg = __half22float2(*reinterpret_cast<const __half2*>(&p.x));
        r.ba = __half22float2(*reinterpret_cast<const __half2*>(&p.y));
    } else {
        const float4 q = __ldg(reinterpret_cast<const float4*>(lp) + idx);
        r.rg = make_float2(q.x, q.y);
        r.ba = make_float2(q.z, q.w);
    }
    return r;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// b - a, one rounding (the FMA's product a * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 b, float2 a) { return __ffma2_rn(a, f2(-1.0f, -1.0f), b); }

// a + w (b - a): exact when a == b (a constant LP reconstructs exactly).
__device__ __forceinline__ px2 lerp2(px2 a, px2 b, float w) {
    const float2 w2 = f2(w, w);
    px2 r;
    r.rg = __ffma2_rn(w2, sub2(b.rg, a.rg), a.rg);
    r.ba = __ffma2_rn(w2, sub2(b.ba, a.ba), a.ba);
    return r;
}

// Row pair of column (off, n) that brackets the angle fraction: v = frac n_c
// - 1/2, rows floor(v) in [-1, n_c - 1] and floor(v) + 1.  The column's guard
// slots (off - 1 holds row n_c - 1, off + n_c holds row 0) make the pair the
// two adjacent slots i0, i0 + 1 for every v; w is the weight of i0 + 1.
__device__ __forceinline__ void column_index(int off, float n, float frac, int& i0, float& w) {
    const float v = fmaf(frac, n, -0.5f);
    const float j0f = floorf(v);
    w = v - j0f;
    i0 = off + (int)j0f;
}

__device__ __forceinline__ px2 column_sample(const void* lp, int fmt, int off, float n, float frac) {
    int i0;
    float w;
    column_index(off, n, frac, i0, w);
    return lerp2(load_lp(lp, fmt, i0), load_lp(lp, fmt, i0 + 1), w);
}

// Frame parameters, staged through shared memory by one thread and then held
// in registers: read-only parameter-space values may otherwise be reloaded
// at every use.
struct ReconRegs {
    float zs;        // c_r * u_n / tan(e_max): radius in pixels -> table coordinate
    float u_nf;      // u_n (the clamp entry)
    const float4* u_tab;
    const int4* col_pair;
    const void* lp;
    int lp_fmt;
};

struct ReconShared {
    ReconRegs r;
    int gxi, gyi;
    float gxf, gyf;
    int W, H, disp_fmt, tile_begin;
    int n_cols;
    void* disp;
};

// Thread 0 of a block finds the frame that owns display tile `tile` (binary
// search over the frames' first tiles) and stages its parameters.
template <class B>
__device__ __forceinline__ void stage_frame(const B& b, int tile, ReconShared& sh) {
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.d[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    const FrameDesc& fd = b.d[lo];
    sh.r.zs = fd.cr * fd.u_inv_h;
    sh.r.u_nf = (float)fd.u_n;
    sh.r.u_tab = fd.u_tab;
    sh.r.col_pair = fd.col_pair;
    sh.r.lp = fd.lp_aa ? fd.lp_aa : fd.lp;   // the FXAA output when the pass ran
    sh.r.lp_fmt = fd.lp_fmt;
    sh.gxi = fd.gxi;
    sh.gyi = fd.gyi;
    sh.gxf = fd.gxf;
    sh.gyf = fd.gyf;
    sh.W = fd.W;
    sh.H = fd.H;
    sh.disp_fmt = fd.disp_fmt;
    sh.tile_begin = (int)fd.tile_begin;
    sh.n_cols = fd.n_cols;
    sh.disp = fd.disp;
}

// Table coordinate of a pixel: s = z u_n / tan(e_max) in [0, u_n]; the piece
// is floor(s), t the position inside it.
__device__ __forceinline__ float table_coord(const ReconRegs& f, float dx, float dy2) {
    return fminf(f.zs * sqrt_approx(fmaf(dx, dx, dy2)), f.u_nf);
}

// One pixel of a row: dx is its gaze offset, dy2 the row's squared offset.
__device__ __forceinline__ px2 recon_pixel(const ReconRegs& f, float dx, float dy, float dy2) {
    const float s = table_coord(f, dx, dy2);
    const int i = (int)s;
    const float t = s - (float)i;
    const float uf = piece_eval(__ldg(f.u_tab + i), t);
    const int c0 = __float2int_rd(uf);
    const float wu = uf - (float)c0;
    const float frac = angle_fraction(dy, dx, fmaxf(fabsf(dx), 1e-30f));
    const int4 cp = __ldg(f.col_pair + c0);  // (slot, count) of c0 and of c0 + 1 (clamped)
    const px2 v0 = column_sample(f.lp, f.lp_fmt, cp.x, __int_as_float(cp.y), frac);
    const px2 v1 = column_sample(f.lp, f.lp_fmt, cp.z, __int_as_float(cp.w), frac);
    return lerp2(v0, v1, wu);
}

__device__ __forceinline__ unsigned pack_half2(float2 p) {
    const __half2 h = __floats2half2_rn(p.x, p.y);
    return *reinterpret_cast<const unsigned*>(&h);
}

// Tile of TW x TH pixels; TW / PX threads per row, each thread PX pixels of one
// row, so the per-thread set-up (frame lookup, row offset) is shared by PX
// pixels.  FP32 display: pixel q of a thread is x = x_tile + q TW/PX + tx, and
// each 16-byte store of a warp is contiguous.  FP16 display: the thread takes
// PX/2 pairs of adjacent pixels, pair q at x = x_tile + 2 (q TW/PX + tx), each
// pair one 16-byte store, again contiguous across the warp.
template <int TW, int TH, int PX, class B>
__global__ void __launch_bounds__((TW / PX) * TH)
k_reconstruct(const __grid_constant__ B b) {
    static_assert(PX % 2 == 0, "pixels per thread must be even");
    __shared__ ReconShared sh;
    const int tile = (int)blockIdx.x;
    if (threadIdx.x == 0) stage_frame(b, tile, sh);
    __syncthreads();
    const ReconRegs f = sh.r;
    const int W = sh.W, H = sh.H;
    void* const disp = sh.disp;
    const int local = tile - sh.tile_begin;
    const int tiles_x = (W + TW - 1) / TW;
    const int ty = local / tiles_x;
    const int tx_tile = local - ty * tiles_x;
    constexpr int TX = TW / PX;
    const int tx = (int)(threadIdx.x % TX);
    const int y = ty * TH + (int)(threadIdx.x / TX);
    if (y >= H) return;
    const float dy = (float)(y - sh.gyi) + sh.gyf;
    const float dy2 = dy * dy;
    const long long row = (long long)y * W;
    const int xt = tx_tile * TW;
    // every pixel's gaze offset is one rounding of (x - floor(x0)) + (0.5 - frac(x0)),
    // so results do not depend on the tile shape
    const int gxi = sh.gxi;
    const float gxf = sh.gxf;
    if (sh.disp_fmt == VAFR_FMT_RGBA16F) {
        const bool pair_ok = (W & 1) == 0;   // 16-byte alignment of pixel pairs
#pragma unroll
        for (int q = 0; q < PX / 2; ++q) {
            const int xo = 2 * (q * TX + tx);
            const int x = xt + xo;
            if (x >= W) break;
            const px2 a = recon_pixel(f, (float)(x - gxi) + gxf, dy, dy2);
            if (pair_ok && x + 1 < W) {
                const px2 c = recon_pixel(f, (float)(x + 1 - gxi) + gxf, dy, dy2);
                __stcs(reinterpret_cast<uint4*>(reinterpret_cast<uint2*>(disp) + row + x),
                       make_uint4(pack_half2(a.rg), pack_half2(a.ba), pack_half2(c.rg), pack_half2(c.ba)));
            } else {
                __stcs(reinterpret_cast<uint2*>(disp) + row + x, make_uint2(pack_half2(a.rg), pack_half2(a.ba)));
                if (x + 1 < W) {
                    const px2 c = recon_pixel(f, (float)(x + 1 - gxi) + gxf, dy, dy2);
                    __stcs(reinterpret_cast<uint2*>(disp) + row + x + 1,
                           make_uint2(pack_half2(c.rg), pack_half2(c.ba)));
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < PX; ++q) {
            const int xo = q * TX + tx;
            const int x = xt + xo;
            if (x >= W) break;
            const px2 a = recon_pixel(f, (float)(x - gxi) + gxf, dy, dy2);
            __stcs(reinterpret_cast<float4*>(disp) + row + x, make_float4(a.rg.x, a.rg.y, a.ba.x, a.ba.y));
        }
    }
}

// ---- LP texels staged in shared memory -----------------------------------------
// A staged tile first copies the LP texels its pixels can reach into shared
// memory (coalesced loads of each column's row span), then filters from there.
// The span comes from the tile's rectangle: the nearest and farthest pixel
// centres bound the table coordinate, hence the columns (the forward map is
// monotone in the radius); the corners bound the angle when the gaze lies
// outside the rectangle.  Spans carry one column and one or two rows of
// margin; a tile holding the gaze, spanning more than a quarter turn, more
// than kStageCols columns or more texels than the buffer holds stages nothing.
// Whatever the plan, each texel pair is read from shared memory only if its
// slots lie inside its column's staged span, else from global memory, so the
// texel values -- and the results -- are those of the other variants.
constexpr int kStageCols = 64;
constexpr int kStageBytes = 24576;    // 1,536 FP32 or 3,072 FP16 texel slots

struct StagePlan {
    int4 col[kStageCols];   // per staged column: (first slot, last slot, buffer index - slot, 0)
    int off[kStageCols];    // buffer index of each column's first slot
    int c_lo, n, total;     // first column, staged columns (0: none), staged slots
};

// Warp 0 plans the tile whose pixel centres span columns x0..x1, rows y0..y1.
__device__ void stage_plan(const ReconRegs& f, const ReconShared& sh, int x0, int y0, int x1, int y1,
                           int cap_slots, StagePlan& st) {
    const int lane = (int)(threadIdx.x & 31);
    // pixel-centre offsets from the gaze, computed as the pixels compute them
    const float dxa = (float)(x0 - sh.gxi) + sh.gxf, dxb = (float)(x1 - sh.gxi) + sh.gxf;
    const float dya = (float)(y0 - sh.gyi) + sh.gyf, dyb = (float)(y1 - sh.gyi) + sh.gyf;
    const bool holds_gaze = dxa <= 0.0f && dxb >= 0.0f && dya <= 0.0f && dyb >= 0.0f;
    const float nx = dxa > 0.0f ? dxa : (dxb < 0.0f ? dxb : 0.0f);
    const float ny = dya > 0.0f ? dya : (dyb < 0.0f ? dyb : 0.0f);
    const float fx = fmaxf(fabsf(dxa), fabsf(dxb)), fy = fmaxf(fabsf(dya), fabsf(dyb));
    const float s0 = table_coord(f, nx, ny * ny), s1 = table_coord(f, fx, fy * fy);
    const int p0 = (int)s0, p1 = (int)s1;
    const float u0 = piece_eval(__ldg(f.u_tab + p0), s0 - (float)p0);
    const float u1 = piece_eval(__ldg(f.u_tab + p1), s1 - (float)p1);
    const int c_lo = max(__float2int_rd(u0) - 1, 0);
    const int c_hi = min(__float2int_rd(u1) + 2, sh.n_cols - 1);
    // the angle fractions of the corners, relative to the first, give the arc
    const float cx[4] = {dxa, dxb, dxa, dxb}, cy[4] = {dya, dya, dyb, dyb};
    float fr0 = 0.0f, lo = 0.0f, hi = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float fq = angle_fraction(cy[q], cx[q], fmaxf(fabsf(cx[q]), 1e-30f));
        if (q == 0) {
            fr0 = fq;
        } else {
            float d = fq - fr0;
            d = d >= 0.5f ? d - 1.0f : (d < -0.5f ? d + 1.0f : d);
            lo = fminf(lo, d);
            hi = fmaxf(hi, d);
        }
    }
    const bool ok = !holds_gaze && hi - lo <= 0.25f && c_hi - c_lo + 1 <= kStageCols;
    const float flo = fr0 + lo, fhi = fr0 + hi;
    // each lane plans columns c_lo + lane and c_lo + lane + 32
    int cnt[2] = {0, 0};
    int4 info[2] = {make_int4(INT_MAX, INT_MIN, 0, 0), make_int4(INT_MAX, INT_MIN, 0, 0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = c_lo + lane + 32 * h;
        if (ok && c <= c_hi) {
            const int4 cp = __ldg(f.col_pair + c);       // (first slot, FP32 count) of column c
            const float nf = __int_as_float(cp.y);
            const int n = (int)nf;
            int jl = __float2int_rd(fmaf(flo, nf, -0.5f)) - 1;
            int jh = __float2int_rd(fmaf(fhi, nf, -0.5f)) + 2;
            if (jl < -1 || jh > n) {   // the arc wraps in this column: all of it, guards included
                jl = -1;
                jh = n;
            }
            info[h] = make_int4(cp.x + jl, cp.x + jh, 0, 0);
            cnt[h] = jh - jl + 1;
        }
    }
    // exclusive offsets of the counts, columns in order (lane, then lane + 32)
    int sa = cnt[0], sb = cnt[1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ya = __shfl_up_sync(0xffffffffu, sa, o), yb = __shfl_up_sync(0xffffffffu, sb, o);
        if (lane >= o) {
            sa += ya;
            sb += yb;
        }
    }
    const int ta = __shfl_sync(0xffffffffu, sa, 31), tb = __shfl_sync(0xffffffffu, sb, 31);
    const int total = ta + tb;
    const bool fits = ok && total <= cap_slots;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        const int off = h == 0 ? sa - cnt[0] : ta + sb - cnt[1];
        info[h].z = off - info[h].x;
        if (!fits) info[h] = make_int4(INT_MAX, INT_MIN, 0, 0);
        st.col[k] = info[h];
        st.off[k] = off;
    }
    if (lane == 0) {
        st.c_lo = c_lo;
        st.n = fits ? c_hi - c_lo + 1 : 0;
        st.total = fits ? total : 0;
    }
}

// The block copies the planned slots into the buffer: warp w takes columns
// w, w + TW/32, ..., its lanes consecutive slots of the column's span.
template <int TW>
__device__ __forceinline__ void stage_copy(const ReconRegs& f, const StagePlan& st, unsigned char* buf) {
    const bool h16 = f.lp_fmt == VAFR_FMT_RGBA16F;
    const int lane = (int)(threadIdx.x & 31);
    for (int k = (int)(threadIdx.x >> 5); k < st.n; k += TW / 32) {
        const int4 ci = st.col[k];
        const int n = ci.y - ci.x + 1, to = ci.x + ci.z;
        for (int q = lane; q < n; q += 32) {
            if (h16)
                reinterpret_cast<uint2*>(buf)[to + q] = __ldg(reinterpret_cast<const uint2*>(f.lp) + ci.x + q);
            else
                reinterpret_cast<float4*>(buf)[to + q] = __ldg(reinterpret_cast<const float4*>(f.lp) + ci.x + q);
        }
    }
}

// Staged span of the column holding slots i, i + 1 (as an int4 of the plan).
__device__ __forceinline__ int4 stage_info(const StagePlan* st, int c) {
    const int k = c - st->c_lo;
    return (unsigned)k < (unsigned)st->n ? st->col[k] : make_int4(INT_MAX, INT_MIN, 0, 0);
}

template <int LPF>
__device__ __forceinline__ px2 load_lp_shared(const unsigned char* buf, int idx) {
    px2 r;
    if (LPF == VAFR_FMT_RGBA16F) {
        const uint2 p = reinterpret_cast<const uint2*>(buf)[idx];
        r.rg = __half22float2(*reinterpret_cast<const __half2*>(&p.x));
        r.ba = __half22float2(*reinterpret_cast<const __half2*>(&p.y));
    } else {
        const float4 q = reinterpret_cast<const float4*>(buf)[idx];
        r.rg = make_float2(q.x, q.y);
        r.ba = make_float2(q.z, q.w);
    }
    return r;
}

// Texel pair (i, i + 1) of one column into (a, b) if p: from the buffer when
// both slots are staged, else from global memory.
template <int LPF>
__device__ __forceinline__ void pair_staged(bool p, const void* lp, const unsigned char* buf, int4 si, int i,
                                            px2& a, px2& b) {
    if (!p) return;
    if (i >= si.x && i + 1 <= si.y) {
        a = load_lp_shared<LPF>(buf, i + si.z);
        b = load_lp_shared<LPF>(buf, i + 1 + si.z);
    } else {
        a = load_lp(lp, LPF, i);
        b = load_lp(lp, LPF, i + 1);
    }
}

// ---- column runs ---------------------------------------------------------------
// A thread owns one display column x and R consecutive rows; the 32 lanes of a
// warp take 32 consecutive x, so every row store of a warp is contiguous.  Down
// the run the thread keeps the last u-table piece, column pair and the two LP
// row pairs in registers and reloads each only when its index changes: away
// from the gaze several display pixels fall into one LP cell (about 2.5 on
// average at 4K, 100 degrees), so most of the per-pixel loads of the row
// kernel disappear.  The arithmetic per pixel is the row kernel's, operation
// for operation, so both produce identical bits.
template <int LPF>
__device__ __forceinline__ px2 load_lp_t(const void* lp, int idx) {
    return load_lp(lp, LPF, idx);
}

template <int DF>
__device__ __forceinline__ void store_px(void* disp, long long idx, px2 v) {
    if (DF == VAFR_FMT_RGBA16F)
        __stcs(reinterpret_cast<uint2*>(disp) + idx, make_uint2(pack_half2(v.rg), pack_half2(v.ba)));
    else
        __stcs(reinterpret_cast<float4*>(disp) + idx, make_float4(v.rg.x, v.rg.y, v.ba.x, v.ba.y));
}

// Predicated loads: when `p` is false nothing is read and `v` keeps its value,
// without a branch (the index bookkeeping of a run is branch-free); FP16 LP
// texels, which need widening after the load, take a branch instead.
__device__ __forceinline__ void ld_if(bool p, const float4* ptr, float4& v) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
        "@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w)
        : "r"((int)p), "l"(ptr));
}

__device__ __forceinline__ void ld_if(bool p, const int4* ptr, int4& v) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
        "@q ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
        : "r"((int)p), "l"(ptr));
}

// LP texel `idx` into `v` if `p`: FP32 RGBA, or FP16 RGBA widened exactly.
template <int LPF>
__device__ __forceinline__ void ld_texel_if(bool p, const void* lp, int idx, px2& v) {
    if (LPF == VAFR_FMT_RGBA16F) {
        // a branch: predicated-off widening instructions would still issue
        if (p) v = load_lp(lp, LPF, idx);
    } else {
        asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
            "@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%5];\n\t}"
            : "+f"(v.rg.x), "+f"(v.rg.y), "+f"(v.ba.x), "+f"(v.ba.y)
            : "r"((int)p), "l"(reinterpret_cast<const float4*>(lp) + idx));
    }
}

// R rows (FULL) or the first `nrows` of them, of display column x.  The
// column's dx is fixed, so angle_fraction's dx < 0 reflection becomes the
// per-thread FMA a * sx + ox (0.5 - a rounded once, or a exactly).
template <int R, int LH, bool FULL, bool REUSE_U, int LPF, int DF, bool STAGED = false>
__device__ __forceinline__ void recon_run(const ReconRegs& f, void* disp, int W, int x, int y0, int nrows,
                                          float dx, int gyi, float gyf, const StagePlan* st = nullptr,
                                          const unsigned char* buf = nullptr, int n_cols = 0) {
    constexpr float c[8] = {VAFR_ATAN_COEFS};
    constexpr int BPP = DF == VAFR_FMT_RGBA16F ? 8 : 16;
    int piece = -1, c0_held = -2, k0 = -1, k1 = -1;
    float4 cf = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int4 cp = make_int4(0, 0x3f800000, 0, 0x3f800000);
    int4 si0 = make_int4(INT_MAX, INT_MIN, 0, 0), si1 = si0;   // staged spans of the column pair
    px2 a0{}, b0{}, a1{}, b1{};
    const float ax = fmaxf(fabsf(dx), 1e-30f);
    const float sx = dx < 0.0f ? -1.0f : 1.0f, ox = dx < 0.0f ? 0.5f : 0.0f;
    const float dy0 = (float)(y0 - gyi);
    char* out = static_cast<char*>(disp) + ((long long)y0 * W + x) * BPP;
    const long long row_bytes = (long long)W * BPP * LH;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        if (!FULL && k >= nrows) break;
        const float dy = (dy0 + (float)(LH * k)) + gyf;   // (float)(y - floor(y0)) exactly: |y - floor(y0)| < 2^24
        const float s = table_coord(f, dx, dy * dy);
        const int i = (int)s;
        const float t = s - (float)i;
        if (REUSE_U) {
            ld_if(i != piece, f.u_tab + i, cf);
            piece = i;
        } else {
            cf = __ldg(f.u_tab + i);
        }
        const float uf = piece_eval(cf, t);
        const int c0 = __float2int_rd(uf);
        const float wu = uf - (float)c0;
        if (STAGED && c0 != c0_held) {
            si0 = stage_info(st, max(c0, 0));
            si1 = stage_info(st, min(c0 + 1, n_cols - 1));
        }
        ld_if(c0 != c0_held, f.col_pair + c0, cp);
        c0_held = c0;
        // angle_fraction(dy, dx, ax) with the dx reflection as one FMA
        const float ay = fabsf(dy);
        const float tt = fminf(ax, ay) * rcp_approx(fmaxf(ax, ay));
        const float ss = tt * tt;
        float p = c[0];
#pragma unroll
        for (int q = 1; q < 8; ++q) p = fmaf(p, ss, c[q]);
        float a = p * tt;
        a = ay > ax ? 0.25f - a : a;
        a = fmaf(a, sx, ox);
        const float frac = dy < 0.0f ? 1.0f - a : a;
        int i0, i2;
        float w0, w1;
        column_index(cp.x, __int_as_float(cp.y), frac, i0, w0);
        column_index(cp.z, __int_as_float(cp.w), frac, i2, w1);
        const bool l0 = i0 != k0, l1 = i2 != k1;
        if (STAGED) {
            pair_staged<LPF>(l0, f.lp, buf, si0, i0, a0, b0);
            pair_staged<LPF>(l1, f.lp, buf, si1, i2, a1, b1);
        } else {
            ld_texel_if<LPF>(l0, f.lp, i0, a0);
            ld_texel_if<LPF>(l0, f.lp, i0 + 1, b0);
            ld_texel_if<LPF>(l1, f.lp, i2, a1);
            ld_texel_if<LPF>(l1, f.lp, i2 + 1, b1);
        }
        k0 = i0;
        k1 = i2;
        store_px<DF>(out, 0, lerp2(lerp2(a0, b0, w0), lerp2(a1, b1, w1), wu));
        out += row_bytes;
    }
}

template <int R, int LH, bool REUSE_U, int LPF, int DF>
__device__ __forceinline__ void recon_run_any(const ReconRegs& f, void* disp, int W, int x, int y0, int nrows,
                                              float dx, int gyi, float gyf) {
    if (nrows == R)
        recon_run<R, LH, true, REUSE_U, LPF, DF>(f, disp, W, x, y0, nrows, dx, gyi, gyf);
    else
        recon_run<R, LH, false, REUSE_U, LPF, DF>(f, disp, W, x, y0, nrows, dx, gyi, gyf);
}

// Block of TW threads (TW / 32 warps side by side).  A warp covers LW columns
// and LH = 32 / LW interleaved runs: lane (lx, ly) owns column lx and rows
// ly, ly + LH, ..., ly + (R - 1) LH of the warp's LW x (LH R) window, so at each
// step the warp touches an LW x LH block of pixels (its stores are LH
// contiguous row segments of LW pixels).  Tile: (TW / 32) LW x LH R pixels.
// The LP and display formats are uniform over a block, so the format branch
// is taken once per block.
template <int TW, int R, int LW, int MINB, bool REUSE_U, class B>
__global__ void __launch_bounds__(TW, MINB)
k_reconstruct_runs(const __grid_constant__ B b) {
    constexpr int LH = 32 / LW;
    constexpr int TX = (TW / 32) * LW, TY = LH * R;
    __shared__ ReconShared sh;
    const int tile = (int)blockIdx.x;
    if (threadIdx.x == 0) stage_frame(b, tile, sh);
    __syncthreads();
    const ReconRegs f = sh.r;
    const int W = sh.W, H = sh.H;
    const int local = tile - sh.tile_begin;
    const int tiles_x = (W + TX - 1) / TX;
    const int ty = local / tiles_x;
    const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5);
    const int x = (local - ty * tiles_x) * TX + warp * LW + lane % LW;
    const int y0 = ty * TY + lane / LW;
    if (x >= W || y0 >= H) return;
    const int nrows = min(R, (H - y0 + LH - 1) / LH);
    const float dx = (float)(x - sh.gxi) + sh.gxf;
    const int gyi = sh.gyi;
    const float gyf = sh.gyf;
    void* const disp = sh.disp;
    if (f.lp_fmt == VAFR_FMT_RGBA16F) {
        if (sh.disp_fmt == VAFR_FMT_RGBA16F)
            recon_run_any<R, LH, REUSE_U, VAFR_FMT_RGBA16F, VAFR_FMT_RGBA16F>(f, disp, W, x, y0, nrows, dx, gyi, gyf);
        else
            recon_run_any<R, LH, REUSE_U, VAFR_FMT_RGBA16F, VAFR_FMT_RGBA32F>(f, disp, W, x, y0, nrows, dx, gyi, gyf);
    } else {
        if (sh.disp_fmt == VAFR_FMT_RGBA16F)
            recon_run_any<R, LH, REUSE_U, VAFR_FMT_RGBA32F, VAFR_FMT_RGBA16F>(f, disp, W, x, y0, nrows, dx, gyi, gyf);
        else
            recon_run_any<R, LH, REUSE_U, VAFR_FMT_RGBA32F, VAFR_FMT_RGBA32F>(f, disp, W, x, y0, nrows, dx, gyi, gyf);
    }
}

template <int TW, int R, int LW, int MINB, bool REUSE_U, class B>
cudaError_t launch_runs(const B& b, cudaStream_t s) {
    if (b.total_tiles <= 0) return cudaSuccess;
    k_reconstruct_runs<TW, R, LW, MINB, REUSE_U, B><<<(unsigned)b.total_tiles, TW, 0, s>>>(b);
    count_launch(1);
    return cudaGetLastError();
}

// Column-run tile (TW threads, one display column each, R rows) whose LP
// footprint is first staged in shared memory (stage_plan / stage_copy).
template <int TW, int R, int MINB, class B>
__global__ void __launch_bounds__(TW, MINB)
k_reconstruct_staged(const __grid_constant__ B b) {
    constexpr int TX = TW, TY = R;
    __shared__ ReconShared sh;
    __shared__ StagePlan st;
    __shared__ __align__(16) unsigned char buf[kStageBytes];
    const int tile = (int)blockIdx.x;
    if (threadIdx.x == 0) stage_frame(b, tile, sh);
    __syncthreads();
    const ReconRegs f = sh.r;
    const int W = sh.W, H = sh.H;
    const int local = tile - sh.tile_begin;
    const int tiles_x = (W + TX - 1) / TX;
    const int ty = local / tiles_x;
    const int xt = (local - ty * tiles_x) * TX, yt = ty * TY;
    if (threadIdx.x < 32) {
        const int cap = kStageBytes / (f.lp_fmt == VAFR_FMT_RGBA16F ? 8 : 16);
        stage_plan(f, sh, xt, yt, min(xt + TX, W) - 1, min(yt + TY, H) - 1, cap, st);
    }
    __syncthreads();
    stage_copy<TW>(f, st, buf);
    __syncthreads();
    const int x = xt + (int)threadIdx.x;
    const int y0 = yt;
    if (x >= W || y0 >= H) return;
    const int nrows = min(R, H - y0);
    const float dx = (float)(x - sh.gxi) + sh.gxf;
    const int gyi = sh.gyi;
    const float gyf = sh.gyf;
    void* const disp = sh.disp;
    const int C = sh.n_cols;
#define VAFR_STAGED_RUN(LPF, DF)                                                                     \
    (nrows == R ? recon_run<R, 1, true, false, LPF, DF, true>(f, disp, W, x, y0, nrows, dx, gyi, gyf, &st, buf, C) \
                : recon_run<R, 1, false, false, LPF, DF, true>(f, disp, W, x, y0, nrows, dx, gyi, gyf, &st, buf, C))
    if (f.lp_fmt == VAFR_FMT_RGBA16F) {
        if (sh.disp_fmt == VAFR_FMT_RGBA16F) VAFR_STAGED_RUN(VAFR_FMT_RGBA16F, VAFR_FMT_RGBA16F);
        else VAFR_STAGED_RUN(VAFR_FMT_RGBA16F, VAFR_FMT_RGBA32F);
    } else {
        if (sh.disp_fmt == VAFR_FMT_RGBA16F) VAFR_STAGED_RUN(VAFR_FMT_RGBA32F, VAFR_FMT_RGBA16F);
        else VAFR_STAGED_RUN(VAFR_FMT_RGBA32F, VAFR_FMT_RGBA32F);
    }
#undef VAFR_STAGED_RUN
}

template <int TW, int R, int MINB, class B>
cudaError_t launch_staged(const B& b, cudaStream_t s) {
    if (b.total_tiles <= 0) return cudaSuccess;
    k_reconstruct_staged<TW, R, MINB, B><<<(unsigned)b.total_tiles, TW, 0, s>>>(b);
    count_launch(1);
    return cudaGetLastError();
}

template <int TW, int TH, int PX, class B>
cudaError_t launch_shape(const B& b, cudaStream_t s) {
    if (b.total_tiles <= 0) return cudaSuccess;
    k_reconstruct<TW, TH, PX, B><<<(unsigned)b.total_tiles, (TW / PX) * TH, 0, s>>>(b);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace

// Tile shapes the autotuner chooses between: column runs (0-3: rows per
// thread, lanes per warp row, minimum blocks per SM, u-table piece reuse), row
// tiles (4-7: pixels wide, rows, pixels per thread) and the column run with
// its LP footprint staged in shared memory (8).
ReconShape recon_shape(int variant) {
    switch (variant) {
        case 0: return {128, 8, 0};
        case 1: return {128, 8, 0};
        case 2: return {128, 16, 0};
        case 3: return {64, 16, 0};
        case 4: return {256, 4, 8};
        case 5: return {128, 8, 4};
        case 6: return {64, 8, 2};
        case 7: return {128, 4, 4};
        default: return {128, 16, 0};
    }
}

template <class B>
cudaError_t launch_reconstruct(const B& batch, int variant, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_runs<128, 8, 32, 10, false>(batch, s);
        case 1: return launch_runs<128, 8, 32, 8, true>(batch, s);
        case 2: return launch_runs<128, 16, 32, 10, false>(batch, s);
        case 3: return launch_runs<128, 8, 16, 10, false>(batch, s);
        case 4: return launch_shape<256, 4, 8>(batch, s);
        case 5: return launch_shape<128, 8, 4>(batch, s);
        case 6: return launch_shape<64, 8, 2>(batch, s);
        case 7: return launch_shape<128, 4, 4>(batch, s);
        default: return launch_staged<128, 16, 6>(batch, s);
    }
}

template cudaError_t launch_reconstruct<SmallBatch>(const SmallBatch&, int, cudaStream_t);
template cudaError_t launch_reconstruct<BigBatch>(const BigBatch&, int, cudaStream_t);

}  // namespace vafr
