// lp_map.cuh -- device pieces of the forward log-polar map shared by the
// reconstruction and the reprojection kernels: the FP32 angle fraction and the
// u-table evaluation, with the hardware reciprocal / square-root
// approximations they use.
#pragma once

#include <cuda_runtime.h>

namespace vafr {

// Hardware reciprocal approximation (PTX rcp.approx, flush-to-zero); the
// argument is kept >= 1e-30, so it is a normal number.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Odd polynomial for atan(t) / 2pi on [0, 1]: coefficients of t^15 ... t^1
// (near-minimax fit by Lawson's reweighted least squares, csrc/fit_atan.py).
#define VAFR_ATAN_COEFS                                                      \
    -0.0006453031091950834f, 0.0034795934334397316f, -0.008898717351257801f, \
        0.01534602977335453f, -0.022136269137263298f, 0.031745944172143936f, \
        -0.05304612219333649f, 0.15915483236312866f

// atan2(dy, dx) / 2pi wrapped to [0, 1); (0, 0) -> 0.  Octant reduction
// t = min(ax, |dy|) / max(ax, |dy|) with ax = max(|dx|, 1e-30) (a pixel offset
// is 0 or far above 1e-30, so this only keeps the quotient finite at d = 0),
// then the polynomial, then the octant is undone as 0.25 - a, 0.5 - a, 1 - a.
__device__ __forceinline__ float angle_fraction(float dy, float dx, float ax) {
    constexpr float c[8] = {VAFR_ATAN_COEFS};
    const float ay = fabsf(dy);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mn * rcp_approx(mx);
    const float s = t * t;
    float p = c[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) p = fmaf(p, s, c[k]);
    float a = p * t;                       // first-octant fraction in [0, 1/8]
    a = ay > ax ? 0.25f - a : a;           // first quadrant
    a = dx < 0.0f ? 0.5f - a : a;          // upper half plane
    a = dy < 0.0f ? 1.0f - a : a;          // full turn
    return a;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// u - 1/2 from the piece's cubic (Horner in FP32).
__device__ __forceinline__ float piece_eval(float4 c, float t) {
    return fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
}

}  // namespace vafr
