// sdf.cuh -- analytic signed distance functions of the boundaries (device).
//
// The paper samples rigid bodies and domain boundaries with immovable
// particles (Sec. 3); here they are analytic SDFs, phi > 0 in free space and
// n = grad phi.  A box interior contributes six half-space walls (x-lo, x-hi,
// y-lo, y-hi, z-lo, z-hi); a cone shell and a solid box one component each.
#pragma once

#include <cuda_runtime.h>

#include "gs.h"

struct SdfHit {
    float phi;
    float nx, ny, nz;
};

__device__ __forceinline__ int sdf_components(int kind)
{
    return kind == GS_SDF_BOX_INTERIOR ? 6 : ((kind == GS_SDF_CONE_SHELL || kind == GS_SDF_SOLID_BOX) ? 1 : 0);
}

// True when the one-component SDF s (cone shell, solid box) is surely at
// least r away from x, so that its contact test phi < r fails.  Solid box:
// phi >= max_k (|x_k - c_k| - h_k) when outside, with the excesses computed
// by the same float operations as sdf_eval (and sqrt(a^2 + ...) >= a in
// float), plus a margin of 1e-4 r + 1e-6.  Cone shell: the distance to the
// bounding rectangle of its profile, a different rounding path, so the
// margin also grows with the magnitudes involved (1e-5 of them, far above
// the evaluation's rounding).  Skipping never changes a decision.  A box
// interior (six cheap walls) is never skipped.
__device__ __forceinline__ bool sdf_far(const gs_sdf& s, float x, float y, float z, float r)
{
    const float* p = s.p;
    const float m = r + 1.0e-4f * r + 1.0e-6f;
    if (s.kind == GS_SDF_SOLID_BOX) {
        const float q = fmaxf(fmaxf(fabsf(x - p[0]) - p[3], fabsf(y - p[1]) - p[4]), fabsf(z - p[2]) - p[5]);
        return q > m;
    }
    if (s.kind == GS_SDF_CONE_SHELL) {
        const float dx = x - p[0], dy = y - p[1];
        const float rho = sqrtf(dx * dx + dy * dy);
        const float rlo = fminf(p[3], p[5]), rhi = fmaxf(p[3], p[5]);
        const float zlo = fminf(p[2], p[4]), zhi = fmaxf(p[2], p[4]);
        const float q = fmaxf(fmaxf(rho - rhi, rlo - rho), fmaxf(z - zhi, zlo - z));
        const float scale = rho + rhi + fabsf(z) + fmaxf(fabsf(zlo), fabsf(zhi)) + fabsf(p[0]) + fabsf(p[1]);
        return q - p[6] > m + 1.0e-5f * scale;
    }
    return false;
}

// Component c of SDF s at x.
__device__ __forceinline__ SdfHit sdf_eval(const gs_sdf& s, int c, float x, float y, float z)
{
    SdfHit h;
    const float* p = s.p;
    if (s.kind == GS_SDF_BOX_INTERIOR) {
        int k = c >> 1;
        float xk = k == 0 ? x : (k == 1 ? y : z);
        float sgn = (c & 1) ? -1.0f : 1.0f;
        h.phi = (c & 1) ? (p[3 + k] - xk) : (xk - p[k]);
        h.nx = k == 0 ? sgn : 0.0f;
        h.ny = k == 1 ? sgn : 0.0f;
        h.nz = k == 2 ? sgn : 0.0f;
        return h;
    }
    if (s.kind == GS_SDF_CONE_SHELL) {
        // segment (R_out, z_out)-(R_top, z_top) in the (rho, z) half-plane,
        // revolved about the vertical axis through (cx, cy), half thickness p[6]
        float dx = x - p[0], dy = y - p[1];
        float rho = sqrtf(dx * dx + dy * dy);
        float rx = 1.0f, ry = 0.0f;
        if (rho > 0.0f) {
            rx = dx / rho;
            ry = dy / rho;
        }
        float er = p[5] - p[3], ez = p[4] - p[2];
        float qr = rho - p[3], qz = z - p[2];
        float ee = er * er + ez * ez;
        float t = (qr * er + qz * ez) / ee;
        float dist, n2r, n2z;
        if (t > 0.0f && t < 1.0f) {
            // closest point inside the segment: the normal is the segment's
            // fixed perpendicular (its sign picks the side), which avoids
            // the cancellation of q - t e close to the mid-surface
            float le = sqrtf(ee);
            float pr = -ez / le, pz = er / le;
            float sd = qr * pr + qz * pz;
            dist = fabsf(sd);
            float sg = sd < 0.0f ? -1.0f : 1.0f;
            n2r = sg * pr;
            n2z = sg * pz;
        } else {
            t = fminf(fmaxf(t, 0.0f), 1.0f);
            float dr = qr - t * er, dz = qz - t * ez;
            dist = sqrtf(dr * dr + dz * dz);
            if (dist > 0.0f) {
                n2r = dr / dist;
                n2z = dz / dist;
            } else {
                float le = sqrtf(ee);
                n2r = -ez / le;
                n2z = er / le;
            }
        }
        h.phi = dist - p[6];
        h.nx = n2r * rx;
        h.ny = n2r * ry;
        h.nz = n2z;
        return h;
    }
    if (s.kind == GS_SDF_SOLID_BOX) {
        float d[3] = {x - p[0], y - p[1], z - p[2]};
        float q[3], sg[3];
        bool outside = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sg[k] = d[k] < 0.0f ? -1.0f : 1.0f;
            q[k] = fabsf(d[k]) - p[3 + k];
            outside |= q[k] > 0.0f;
        }
        if (outside) {
            float a = fmaxf(q[0], 0.0f), b = fmaxf(q[1], 0.0f), cc = fmaxf(q[2], 0.0f);
            float l = sqrtf(a * a + b * b + cc * cc);
            h.phi = l;
            h.nx = sg[0] * a / l;
            h.ny = sg[1] * b / l;
            h.nz = sg[2] * cc / l;
        } else {
            int a = 0;
            if (q[1] > q[a]) a = 1;
            if (q[2] > q[a]) a = 2;
            h.phi = q[a];
            h.nx = a == 0 ? sg[0] : 0.0f;
            h.ny = a == 1 ? sg[1] : 0.0f;
            h.nz = a == 2 ? sg[2] : 0.0f;
        }
        return h;
    }
    h.phi = 3.0e38f;
    h.nx = h.ny = h.nz = 0.0f;
    return h;
}
