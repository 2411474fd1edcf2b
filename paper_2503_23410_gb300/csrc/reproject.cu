// reproject.cu -- VaFR_Rep (Sec. 5.1): the right eye's LP buffer by forward
// grid warping of the left eye's LP buffer (the reprojection of Wissmann et
// al. 2020, done directly from the LP buffer), disocclusions re-rendered.
//
//   vertices  each left texel's hit point P = o + t d (a miss: the point at
//             infinity in direction d) seen from the right eye: camera
//             coordinates, then the right eye's forward map with its own gaze
//             (Eq. 3, e clamped to e_max through the u table, Eq. 12):
//             U = u - 1/2 (column c at U = c), F = angle fraction (row j of
//             column c at F = (j + 1/2)/n_c), depth = distance to the right
//             eye (1e30 at infinity).
//   mesh      the strip between LP columns c and c+1 is zipped by angle: a
//             step of ring c from a_j to a_j+1 makes (a_j, a_j+1, b_k) with
//             k = max{k : (2k+1) n_c < (2j+3) n_c+1}; a step of ring c+1 from
//             b_k to b_k+1 makes (b_k, b_k+1, a_j), j = max{j : (2j+1) n_c+1 <=
//             (2k+3) n_c} (modulo the ring sizes).  Left texel t (column
//             order, guard slots excluded) owns triangle 2t (towards c+1) and
//             2t + 1 (towards c-1).
//   reject    a vertex behind the right eye, hits mixed with misses, depths
//             spread over more than 1.1x, more than 64 columns or (after the
//             unwrap) a quarter turn spanned.
//   raster    in the (U, F) plane, a triangle over half a turn wide is
//             unwrapped and drawn at F and F - 1; column c takes [min, max] of
//             the edge crossings of U = c, rows with (j + 1/2)/n_c inside;
//             depth interpolates barycentrically; a 64-bit atomicMin on
//             (depth bits, triangle id) keeps the nearest (ties: lower id).
//   resolve   a covered right texel interpolates the three left colours;
//             uncovered ones are listed as holes and ray cast.
// All arithmetic FP32 (the oracle does the same steps in FP64).
#include "lp_map.cuh"
#include "vafr_internal.cuh"

namespace vafr {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr float kDepthRatio = 1.1f;
constexpr int kMaxSpan = 64;
constexpr float kMaxFSpan = 0.25f;

__device__ __forceinline__ float4 ld_rgba(const void* lp, int fmt, int slot) {
    if (fmt == VAFR_FMT_RGBA16F) {
        const uint2 p = __ldg(reinterpret_cast<const uint2*>(lp) + slot);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&p.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&p.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    return __ldg(reinterpret_cast<const float4*>(lp) + slot);
}

__device__ __forceinline__ void st_rgba(void* lp, int fmt, int slot, float4 v) {
    if (fmt == VAFR_FMT_RGBA16F) {
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        uint2 p;
        p.x = *reinterpret_cast<const unsigned*>(&lo);
        p.y = *reinterpret_cast<const unsigned*>(&hi);
        reinterpret_cast<uint2*>(lp)[slot] = p;
    } else {
        reinterpret_cast<float4*>(lp)[slot] = v;
    }
}

// camera direction of LP work item k of frame f (the render kernel's ray)
__device__ __forceinline__ void lp_dir(const FrameDesc& f, int k, int& slot, int& col, float3& o, float3& d) {
    const int2 tc = __ldg(f.work + k);
    const int2 cc = __ldg(&f.col[tc.y]);
    const int j = tc.x - cc.x;
    const float te = __ldg(&f.tan_e[tc.y]);
    float sp, cp;
    sincospif(__fdiv_rn((float)(2 * j + 1), (float)cc.y), &sp, &cp);
    const float cx = fmaf(te, cp, f.gx), cy = fmaf(-te, sp, f.gy);
    d.x = fmaf(f.R[0], cx, fmaf(f.R[1], cy, f.R[2]));
    d.y = fmaf(f.R[3], cx, fmaf(f.R[4], cy, f.R[5]));
    d.z = fmaf(f.R[6], cx, fmaf(f.R[7], cy, f.R[8]));
    o = make_float3(f.org[0], f.org[1], f.org[2]);
    slot = tc.x;
    col = tc.y;
}

// Pass 1: the right-eye (U, F, depth, flags) of every left texel.
__global__ void __launch_bounds__(256) k_rep_vertices(const __grid_constant__ SmallBatch b, float4* vert) {
    const FrameDesc& L = b.d[0];
    const FrameDesc& R = b.d[1];
    for (int k = blockIdx.x * 256 + threadIdx.x; k < L.n_texels; k += gridDim.x * 256) {
        int slot, col;
        float3 o, d;
        lp_dir(L, k, slot, col, o, d);
        const float t = __ldg(L.depth + slot);
        const bool inf = !(t < INFINITY);
        float3 P;
        if (inf) {
            P = d;
        } else {
            P.x = fmaf(t, d.x, o.x) - R.org[0];
            P.y = fmaf(t, d.y, o.y) - R.org[1];
            P.z = fmaf(t, d.z, o.z) - R.org[2];
        }
        // right camera coordinates R^T P
        const float px = fmaf(R.R[0], P.x, fmaf(R.R[3], P.y, R.R[6] * P.z));
        const float py = fmaf(R.R[1], P.x, fmaf(R.R[4], P.y, R.R[7] * P.z));
        const float pz = fmaf(R.R[2], P.x, fmaf(R.R[5], P.y, R.R[8] * P.z));
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (pz > 0.0f) {
            const float iz = 1.0f / pz;
            const float qx = fmaf(px, iz, -R.gx), qy = R.gy - py * iz;   // gaze-relative tangent offsets
            const float s = fminf(R.u_inv_h * sqrt_approx(fmaf(qx, qx, qy * qy)), (float)R.u_n);
            const int i = (int)s;
            v.x = piece_eval(__ldg(R.u_tab + i), s - (float)i);
            v.y = angle_fraction(qy, qx, fmaxf(fabsf(qx), 1e-30f));
            v.z = inf ? 1e30f : sqrtf(fmaf(P.x, P.x, fmaf(P.y, P.y, P.z * P.z)));
            v.w = __int_as_float(1 | (inf ? 2 : 0));
        }
        vert[slot] = v;
    }
}

// The three left slots of triangle s of left texel (c, j) (see the mesh rule).
__device__ __forceinline__ bool rep_triangle(const int2* colt, int C, int c, int j, int s, int tv[3]) {
    const int c2 = s == 0 ? c + 1 : c - 1;
    if (c2 < 0 || c2 >= C) return false;
    const int2 a = __ldg(colt + c), b = __ldg(colt + c2);
    const long long n = a.y, n2 = b.y;
    long long k;
    if (s == 0) {
        const long long w = ((2ll * j + 3) * n2 + n - 1) / n - 2;
        k = w >= 0 ? w / 2 : -1;
    } else {
        const long long q = ((2ll * j + 3) * n2) / n;
        k = q >= 1 ? (q - 1) / 2 : -1;
    }
    k = ((k % n2) + n2) % n2;
    tv[0] = a.x + j;
    tv[1] = a.x + (j + 1 == a.y ? 0 : j + 1);
    tv[2] = b.x + (int)k;
    return true;
}

__device__ __forceinline__ bool bary(const float U[3], const float F[3], float u, float f, float w[3]) {
    const float x1 = U[1] - U[0], y1 = F[1] - F[0];
    const float x2 = U[2] - U[0], y2 = F[2] - F[0];
    const float det = x1 * y2 - x2 * y1;
    if (det == 0.0f) return false;
    const float px = u - U[0], py = f - F[0];
    w[1] = (px * y2 - x2 * py) / det;
    w[2] = (x1 * py - px * y1) / det;
    w[0] = 1.0f - w[1] - w[2];
    return true;
}

// Loads the triangle's vertices, applies the rejection rules and the seam
// unwrap; false if the triangle is dropped.
__device__ __forceinline__ bool load_tri(const float4* vert, const int tv[3], float U[3], float F[3], float Z[3],
                                         int& copies) {
    int ninf = 0;
    for (int q = 0; q < 3; ++q) {
        const float4 v = vert[tv[q]];
        const int fl = __float_as_int(v.w);
        if (!(fl & 1)) return false;
        ninf += (fl >> 1) & 1;
        U[q] = v.x;
        F[q] = v.y;
        Z[q] = v.z;
    }
    if (ninf != 0 && ninf != 3) return false;
    const float zlo = fminf(Z[0], fminf(Z[1], Z[2])), zhi = fmaxf(Z[0], fmaxf(Z[1], Z[2]));
    if (ninf == 0 && zhi > kDepthRatio * zlo) return false;
    const float ulo = fminf(U[0], fminf(U[1], U[2])), uhi = fmaxf(U[0], fmaxf(U[1], U[2]));
    if (uhi - ulo > (float)kMaxSpan) return false;
    float flo = fminf(F[0], fminf(F[1], F[2])), fhi = fmaxf(F[0], fmaxf(F[1], F[2]));
    copies = 1;
    if (fhi - flo > 0.5f) {
        for (int q = 0; q < 3; ++q)
            if (F[q] < 0.5f) F[q] += 1.0f;
        copies = 2;
        flo = fminf(F[0], fminf(F[1], F[2]));
        fhi = fmaxf(F[0], fmaxf(F[1], F[2]));
    }
    return fhi - flo <= kMaxFSpan;
}

// Pass 2: rasterise the two triangles of every left texel into the z-buffer.
__global__ void __launch_bounds__(256)
k_rep_raster(const __grid_constant__ SmallBatch b, const float4* vert, unsigned long long* zbuf) {
    const FrameDesc& L = b.d[0];
    const FrameDesc& R = b.d[1];
    const int C = R.n_cols;
    for (int k = blockIdx.x * 256 + threadIdx.x; k < L.n_texels; k += gridDim.x * 256) {
        const int2 tc = __ldg(L.work + k);
        const int c = tc.y, j = tc.x - __ldg(L.col + c).x;
        const int compact = tc.x - (2 * c + 1);
        for (int s = 0; s < 2; ++s) {
            int tv[3];
            if (!rep_triangle(L.col, C, c, j, s, tv)) continue;
            float U[3], F[3], Z[3];
            int copies;
            if (!load_tri(vert, tv, U, F, Z, copies)) continue;
            const unsigned tid = (unsigned)(2 * compact + s);
            const float ulo = fminf(U[0], fminf(U[1], U[2])), uhi = fmaxf(U[0], fmaxf(U[1], U[2]));
            const int c0 = max((int)ceilf(ulo), 0), c1 = min((int)floorf(uhi), C - 1);
            for (int cr = c0; cr <= c1; ++cr) {
                float lo = INFINITY, hi = -INFINITY;
                for (int e = 0; e < 3; ++e) {
                    const int p = e, q = e == 2 ? 0 : e + 1;
                    const float up = U[p] - (float)cr, uq = U[q] - (float)cr;
                    if (up * uq > 0.0f) continue;
                    if (U[p] == U[q]) {
                        lo = fminf(lo, fminf(F[p], F[q]));
                        hi = fmaxf(hi, fmaxf(F[p], F[q]));
                        continue;
                    }
                    const float f = F[p] + ((float)cr - U[p]) / (U[q] - U[p]) * (F[q] - F[p]);
                    lo = fminf(lo, f);
                    hi = fmaxf(hi, f);
                }
                if (!(lo <= hi)) continue;
                const int2 rc = __ldg(R.col + cr);
                const float n = (float)rc.y;
                for (int cp = 0; cp < copies; ++cp) {
                    const float sh = cp ? -1.0f : 0.0f;
                    const int j0 = max((int)ceilf(fmaf(lo + sh, n, -0.5f)), 0);
                    const int j1 = min((int)floorf(fmaf(hi + sh, n, -0.5f)), rc.y - 1);
                    for (int jj = j0; jj <= j1; ++jj) {
                        float w[3];
                        const float f = ((float)jj + 0.5f) / n - sh;
                        if (!bary(U, F, (float)cr, f, w)) continue;
                        const float z = fmaf(w[0], Z[0], fmaf(w[1], Z[1], w[2] * Z[2]));
                        const unsigned long long key =
                            ((unsigned long long)__float_as_uint(fmaxf(z, 0.0f)) << 32) | tid;
                        atomicMin(zbuf + rc.x + jj, key);
                    }
                }
            }
        }
    }
}

// Pass 3: colours of covered right texels, the rest listed as holes.  A
// block takes 1,024 consecutive work items (4 per thread, in the LP work
// order) and appends its holes as one contiguous run in that order, so the
// warps of the hole cast get spatially coherent rays.
constexpr int kResolveItems = 4;

__global__ void __launch_bounds__(256)
k_rep_resolve(const __grid_constant__ SmallBatch b, const float4* vert, const unsigned long long* zbuf,
              int2* holes, unsigned* count, int* tri_out) {
    const FrameDesc& L = b.d[0];
    const FrameDesc& R = b.d[1];
    const int C = L.n_cols;
    __shared__ unsigned warp_off[8];
    __shared__ unsigned block_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long chunk = 256ll * kResolveItems;
    for (long long c0 = (long long)blockIdx.x * chunk; c0 < R.n_texels; c0 += (long long)gridDim.x * chunk) {
        int2 tcq[kResolveItems];
        unsigned hm = 0u;
#pragma unroll
        for (int q = 0; q < kResolveItems; ++q) {
            const long long k = c0 + (long long)threadIdx.x * kResolveItems + q;
            tcq[q] = make_int2(0, 0);
            if (k >= R.n_texels) continue;
            const int2 tc = __ldg(R.work + k);
            tcq[q] = tc;
            const int2 rc = __ldg(R.col + tc.y);
            const int jr = tc.x - rc.x;
            const unsigned long long key = zbuf[tc.x];
            if (key == kEmptyKey) {
                hm |= 1u << q;
                if (tri_out) tri_out[tc.x] = -1;
                continue;
            }
            const unsigned tid = (unsigned)(key & 0xffffffffu);
            const int compact = (int)(tid >> 1), sd = (int)(tid & 1u);
            int lo = 0, hi = C - 1;   // left column holding compact texel `compact`
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(L.col + mid).x - (2 * mid + 1) <= compact) lo = mid; else hi = mid - 1;
            }
            const int jl = compact - (__ldg(L.col + lo).x - (2 * lo + 1));
            int tv[3];
            rep_triangle(L.col, C, lo, jl, sd, tv);
            float U[3], F[3], Z[3];
            int copies;
            load_tri(vert, tv, U, F, Z, copies);
            float w[3];
            const float f = ((float)jr + 0.5f) / (float)rc.y;
            if (!bary(U, F, (float)tc.y, f, w) || fminf(w[0], fminf(w[1], w[2])) < -0.25f)
                bary(U, F, (float)tc.y, f + 1.0f, w);
            const float4 a = ld_rgba(L.lp, L.lp_fmt, tv[0]);
            const float4 bb = ld_rgba(L.lp, L.lp_fmt, tv[1]);
            const float4 cc = ld_rgba(L.lp, L.lp_fmt, tv[2]);
            const float4 v = make_float4(fmaf(w[0], a.x, fmaf(w[1], bb.x, w[2] * cc.x)),
                                         fmaf(w[0], a.y, fmaf(w[1], bb.y, w[2] * cc.y)),
                                         fmaf(w[0], a.z, fmaf(w[1], bb.z, w[2] * cc.z)),
                                         fmaf(w[0], a.w, fmaf(w[1], bb.w, w[2] * cc.w)));
            st_rgba(R.lp, R.lp_fmt, tc.x, v);
            if (jr == 0) st_rgba(R.lp, R.lp_fmt, tc.x + rc.y, v);
            if (jr == rc.y - 1) st_rgba(R.lp, R.lp_fmt, tc.x - rc.y, v);
            if (tri_out) tri_out[tc.x] = (int)tid;
        }
        // block-wide exclusive scan of the hole counts, one atomic per block
        const unsigned nh = (unsigned)__popc(hm);
        unsigned incl = nh;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_off[wid] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t = 0u;
            for (int q = 0; q < 8; ++q) {
                const unsigned u = warp_off[q];
                warp_off[q] = t;
                t += u;
            }
            block_base = t ? atomicAdd(count, t) : 0u;
        }
        __syncthreads();
        unsigned pos = block_base + warp_off[wid] + incl - nh;
#pragma unroll
        for (int q = 0; q < kResolveItems; ++q)
            if (hm & (1u << q)) holes[pos++] = tcq[q];
        __syncthreads();   // warp_off and block_base are rewritten by the next chunk
    }
}

}  // namespace

cudaError_t launch_reproject(const SmallBatch& b, const RepScratch& r, cudaStream_t s, int num_sms) {
    const FrameDesc& R = b.d[1];
    cudaError_t e = cudaMemsetAsync(r.zbuf, 0xff, sizeof(unsigned long long) * (size_t)(R.n_texels + 2 * R.n_cols), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(r.count, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)min((b.d[0].n_texels + 255) / 256, num_sms * 16);
    const unsigned rgrid =
        (unsigned)max(1, min((R.n_texels + 256 * kResolveItems - 1) / (256 * kResolveItems), num_sms * 8));
    k_rep_vertices<<<grid, 256, 0, s>>>(b, r.vert);
    k_rep_raster<<<grid, 256, 0, s>>>(b, r.vert, r.zbuf);
    k_rep_resolve<<<rgrid, 256, 0, s>>>(b, r.vert, r.zbuf, r.holes, r.count, r.tri_out);
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace vafr
