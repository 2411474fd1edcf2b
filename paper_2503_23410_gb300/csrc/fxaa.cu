// fxaa.cu -- anti-aliasing inside the LP buffer (Sec. 3.4: the LP buffer gets
// FXAA before the inverse mapping; Sec. 7 ablates it).  The paper names FXAA
// (Lottes 2009) without parameters; this is that method on the LP grid:
//
//   grid    texel (c, j); along the angle its neighbours are rows j -+ 1 of
//           column c (the guard slots hold the wrap); across the radius,
//           column c' = c -+ 1 (clamped to [0, C-1]) contributes its texel
//           whose angular interval holds the angle of (c, j):
//           j' = floor((2j + 1) n_c' / (2 n_c)).
//   luma    0.299 R + 0.587 G + 0.114 B.
//   1 skip    luma range of {M, N, S, E, W} below max(1/12, max/6): copy.
//   2 axis    second differences across the angle (kA) and across the radius
//             (kR) over the 3 x 3 neighbourhood; kR >= kA: the blend steps a
//             column and the edge is walked along the angle, else the reverse.
//   3 side    blend towards the neighbour with the larger luma step (the
//             positive one on a tie); mid-line luma = their mean, threshold
//             a quarter of the step.
//   4 search  up to 12 unit steps each way along the edge; a step averages
//             the luma of the walked texel and of its partner across the
//             edge; the end is where that leaves the mid-line by the threshold.
//   5 offset  1/2 - d/D from the nearer end (d) and both ends (D), when that
//             end's luma lies across the mid-line from the texel's.
//   6 subpix  a = |3x3 mean (edges 2, corners 1) - M| / range;
//             ((3 - 2a) a^2)^2 x 3/4.
//   7 blend   texel + max(offset, subpix) (neighbour - texel), every channel.
// Luma and every branch decision use FP32 in one fixed order (no contraction),
// offsets and the blend FP32.  Two passes, one thread per texel in the
// frame's screen-space Hilbert order: the luma of every slot into a scratch
// array, then the filter, which reads lumas (4 bytes) for its neighbourhood
// and search and colours only for the texel and its blend partner.  The
// output (a second LP buffer) gets the guard copies too.
#include "vafr_internal.cuh"

namespace vafr {
namespace {

constexpr int kFxaaSteps = 12;

__device__ __forceinline__ float4 ld_texel(const void* lp, int fmt, int slot) {
    if (fmt == VAFR_FMT_RGBA16F) {
        const uint2 p = __ldg(reinterpret_cast<const uint2*>(lp) + slot);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&p.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&p.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    return __ldg(reinterpret_cast<const float4*>(lp) + slot);
}

__device__ __forceinline__ void st_texel(void* lp, int fmt, int slot, float4 v) {
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

__device__ __forceinline__ float luma_of(float4 c) {
    float y = __fmul_rn(0.299f, c.x);
    y = __fadd_rn(y, __fmul_rn(0.587f, c.y));
    return __fadd_rn(y, __fmul_rn(0.114f, c.z));
}

// floor(num / D) for a divisor D = 2 n_c fixed per texel: with num < 2^24 the
// FP32 product num * (1/D) is within one of the quotient (relative error
// <= 2^-23 and quotients < 2^16), fixed by one step each way; larger
// numerators divide in integers.
struct RowDiv {
    unsigned D;
    float rD;
    __device__ __forceinline__ explicit RowDiv(int n) : D(2u * (unsigned)n), rD(1.0f / (float)(2 * n)) {}
    __device__ __forceinline__ int operator()(unsigned num) const {
        if (num >= (1u << 24)) return (int)(num / D);
        unsigned q = (unsigned)((float)num * rD);
        q += (q + 1u) * D <= num ? 1u : 0u;
        q -= q * D > num ? 1u : 0u;
        return (int)q;
    }
};

struct Grid {
    const int2* col;   // (slot of row 0, count)
    int C;
    const void* lp;
    int fmt;
    const float* lum;  // luma of every slot (guards included)

    // slot of the texel of column c2 (clamped) at the angle of row j of column
    // c, moved dj rows; |dj| <= 1 may land on a guard slot.  The row is
    // floor((2j + 1) n_c2 / (2 n_c)): the one whose angular interval holds the
    // centre of row j.
    __device__ __forceinline__ int at(int c, int j, const RowDiv& div, int c2, int dj) const {
        c2 = min(max(c2, 0), C - 1);
        const int2 cc = __ldg(col + c2);
        const unsigned long long num = (unsigned long long)(2 * j + 1) * (unsigned)cc.y;
        const int j2 = c2 == c ? j
                               : (num < (1ull << 32) ? div((unsigned)num) : (int)(num / div.D));
        return cc.x + j2 + dj;
    }
    __device__ __forceinline__ float luma(int slot) const { return __ldg(lum + slot); }
};

__device__ __forceinline__ float abs_second_diff(float a, float b, float m) {
    return fabsf(__fsub_rn(__fadd_rn(a, b), __fmul_rn(2.0f, m)));
}

// The filtered colour of texel (c, j) (slot t, count n).
__device__ float4 fxaa_texel(const Grid& g, int c, int j, int n, int t) {
    const RowDiv div(n);
    const float M = g.luma(t);
    // radial neighbours; their angular neighbours are the adjacent slots
    const int sE = g.at(c, j, div, c + 1, 0), sW = g.at(c, j, div, c - 1, 0);
    const float N = g.luma(t + 1), S = g.luma(t - 1);
    const float E = g.luma(sE), W = g.luma(sW);
    // 1 skip
    const float lo = fminf(M, fminf(fminf(N, S), fminf(E, W)));
    const float hi = fmaxf(M, fmaxf(fmaxf(N, S), fmaxf(E, W)));
    const float range = __fsub_rn(hi, lo);
    const float4 cM = ld_texel(g.lp, g.fmt, t);
    if (range < fmaxf(1.0f / 12.0f, __fmul_rn(hi, 1.0f / 6.0f))) return cM;
    const float NE = g.luma(sE + 1), SE = g.luma(sE - 1);
    const float NW = g.luma(sW + 1), SW = g.luma(sW - 1);
    // 2 axis
    const float kA = __fadd_rn(__fadd_rn(__fmul_rn(2.0f, abs_second_diff(N, S, M)), abs_second_diff(NE, SE, E)),
                               abs_second_diff(NW, SW, W));
    const float kR = __fadd_rn(__fadd_rn(__fmul_rn(2.0f, abs_second_diff(E, W, M)), abs_second_diff(NE, NW, N)),
                               abs_second_diff(SE, SW, S));
    const bool across_cols = kR >= kA;
    // 3 side
    const float Ln = across_cols ? W : S, Lp = across_cols ? E : N;
    const float gn = fabsf(__fsub_rn(Ln, M)), gp = fabsf(__fsub_rn(Lp, M));
    const bool pos = gp >= gn;
    const float avg = __fmul_rn(0.5f, __fadd_rn(M, pos ? Lp : Ln));
    const float thr = __fmul_rn(0.25f, fmaxf(gn, gp));
    const int side = pos ? 1 : -1;
    const int2 cc = __ldg(g.col + c);
    // 4 search
    int dist[2];
    float end[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const int sgn = d ? 1 : -1;
        dist[d] = kFxaaSteps;
        end[d] = 0.0f;
#pragma unroll 1
        for (int k = 1; k <= kFxaaSteps; ++k) {
            int ta, tb;
            if (across_cols) {   // walk the rows of column c
                int jk = j + sgn * k;
                if (n > kFxaaSteps) {            // at most one wrap
                    jk = jk < 0 ? jk + n : (jk >= n ? jk - n : jk);
                } else {
                    jk %= n;
                    jk = jk < 0 ? jk + n : jk;
                }
                ta = cc.x + jk;
                tb = g.at(c, jk, div, c + side, 0);
            } else {             // walk the columns at the angle of (c, j)
                ta = g.at(c, j, div, c + sgn * k, 0);
                tb = ta + side;
            }
            const float s = __fmul_rn(0.5f, __fadd_rn(g.luma(ta), g.luma(tb)));
            end[d] = s;
            if (fabsf(__fsub_rn(s, avg)) >= thr) {
                dist[d] = k;
                break;
            }
        }
    }
    // 5 offset
    const bool near_neg = dist[0] < dist[1];
    const int dn = near_neg ? dist[0] : dist[1];
    const float lend = near_neg ? end[0] : end[1];
    const bool good = (__fsub_rn(lend, avg) < 0.0f) != (__fsub_rn(M, avg) < 0.0f);
    const float off_edge = good ? 0.5f - (float)dn / (float)(dist[0] + dist[1]) : 0.0f;
    // 6 subpix
    const float l3 = (2.0f * (N + S + E + W) + (NE + NW + SE + SW)) * (1.0f / 12.0f);
    const float a = fminf(fabsf(l3 - M) / range, 1.0f);
    const float bsub = (3.0f - 2.0f * a) * a * a;
    const float w = fmaxf(off_edge, bsub * bsub * 0.75f);
    // 7 blend
    const float4 q = ld_texel(g.lp, g.fmt, across_cols ? (pos ? sE : sW) : t + side);
    return make_float4(fmaf(w, q.x - cM.x, cM.x), fmaf(w, q.y - cM.y, cM.y), fmaf(w, q.z - cM.z, cM.z),
                       fmaf(w, q.w - cM.w, cM.w));
}

template <class B>
__device__ __forceinline__ int find_aa_frame(const B& b, long long w) {
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.d[mid].aa_begin <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Pass 1: the luma of every texel into the frame's scratch, guard slots too.
template <class B>
__global__ void __launch_bounds__(256) k_lp_luma(const __grid_constant__ B b) {
    for (long long w = (long long)blockIdx.x * 256 + threadIdx.x; w < b.total_aa;
         w += (long long)gridDim.x * 256) {
        const FrameDesc& f = b.d[find_aa_frame(b, w)];
        const int2 tc = __ldg(f.work + (w - f.aa_begin));   // (slot, column)
        const int2 cc = __ldg(f.col + tc.y);
        const int j = tc.x - cc.x, n = cc.y;
        const float y = luma_of(ld_texel(f.lp, f.lp_fmt, tc.x));
        f.luma[tc.x] = y;
        if (j == 0) f.luma[tc.x + n] = y;
        if (j == n - 1) f.luma[tc.x - n] = y;
    }
}

// Pass 2: the filter.
template <class B>
__global__ void __launch_bounds__(256, 6) k_fxaa_lp(const __grid_constant__ B b) {
    for (long long w = (long long)blockIdx.x * 256 + threadIdx.x; w < b.total_aa;
         w += (long long)gridDim.x * 256) {
        const FrameDesc& f = b.d[find_aa_frame(b, w)];
        const int2 tc = __ldg(f.work + (w - f.aa_begin));   // (slot, column)
        const int2 cc = __ldg(f.col + tc.y);
        const int j = tc.x - cc.x, n = cc.y;
        const Grid g{f.col, f.n_cols, f.lp, f.lp_fmt, f.luma};
        const float4 v = fxaa_texel(g, tc.y, j, n, tc.x);
        st_texel(f.lp_aa, f.lp_fmt, tc.x, v);
        if (j == 0) st_texel(f.lp_aa, f.lp_fmt, tc.x + n, v);       // guard after the column
        if (j == n - 1) st_texel(f.lp_aa, f.lp_fmt, tc.x - n, v);   // guard before it
    }
}

}  // namespace

template <class B>
cudaError_t launch_fxaa(const B& b, cudaStream_t s, int num_sms) {
    if (b.total_aa <= 0) return cudaSuccess;
    const long long want = (b.total_aa + 255) / 256;   // one thread per texel
    const long long cap = (long long)num_sms * 64;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    k_lp_luma<B><<<grid, 256, 0, s>>>(b);
    k_fxaa_lp<B><<<grid, 256, 0, s>>>(b);
    count_launch(2);
    return cudaGetLastError();
}

template cudaError_t launch_fxaa<SmallBatch>(const SmallBatch&, cudaStream_t, int);
template cudaError_t launch_fxaa<BigBatch>(const BigBatch&, cudaStream_t, int);

}  // namespace vafr
