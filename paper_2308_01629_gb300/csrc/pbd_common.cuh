// pbd_common.cuh -- pair geometry of the LR constraints, shared by the
// forward passes and their reverse mode so both take the same decisions.
#pragma once

#include <cuda_runtime.h>

struct PairGeo {
    float ex, ey, ez;   // e = y_q - y_p
    float d2, d;
};

__device__ __forceinline__ PairGeo pair_geo(float4 yp, float4 yq)
{
    PairGeo g;
    g.ex = yq.x - yp.x;
    g.ey = yq.y - yp.y;
    g.ez = yq.z - yp.z;
    g.d2 = fmaf(g.ez, g.ez, fmaf(g.ey, g.ey, g.ex * g.ex));
    g.d = sqrtf(g.d2);
    return g;
}

// Eqs. 3-4 friction scale for a tangential displacement of length L.
__device__ __forceinline__ float friction_scale(float L, float thr_s, float thr_k)
{
    if (L < thr_s) return 1.0f;
    return (L > 0.0f && thr_k / L < 1.0f) ? thr_k / L : 1.0f;
}

// Tangential part of a relative displacement r with respect to a direction
// e (e.e = ee): t = r - (r.e / ee) e, and its length.
struct Tangent {
    float tx, ty, tz, L;
};

__device__ __forceinline__ Tangent tangent_part(float rx, float ry, float rz, float ex, float ey, float ez, float ee)
{
    Tangent t;
    const float al = fmaf(rz, ez, fmaf(ry, ey, rx * ex)) / ee;
    t.tx = fmaf(-al, ex, rx);
    t.ty = fmaf(-al, ey, ry);
    t.tz = fmaf(-al, ez, rz);
    t.L = sqrtf(fmaf(t.tz, t.tz, fmaf(t.ty, t.ty, t.tx * t.tx)));
    return t;
}
