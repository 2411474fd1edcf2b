// pathtrace.cu -- path tracing into the LP buffer and the path-traced
// full-resolution GT (Sec. 8), on the traversal of trace.cuh.
#include "trace.cuh"

namespace vafr {
namespace {

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
}  // namespace

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

}  // namespace vafr
