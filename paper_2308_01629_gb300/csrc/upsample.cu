// upsample.cu -- HR upsampling of Sec. 4 as one fused kernel.
//
// Each warp owns 32 consecutive HR particles of the cell-ordered HR array
// (one float4 position + one float4 velocity each, read once, written once).
// The warp bounds its particles with an axis-aligned box, walks the rows of
// LR grid cells that the box widened by the 3 r_LR support touches (each row
// of cells is one contiguous run of the cell-ordered LR array), keeps the LR
// particles within 3 r_LR of the box, and stages them in shared memory.
// Every lane then sums the kernel weights of Sec. 4 over the staged LR set:
//   w = max(0, 1 - |x_ij|^2 / (9 r_LR^2))^3,  S = sum w,  V = sum w v_j,
//   wmax = max w,  vtilde = V / S (0 when S = 0),
//   alpha = 1 - wmax if wmax <= c1 or wmax / S >= c2, else 0,
//   v = (1 - alpha) vtilde + alpha (v + dt g),  x = x + dt v,
// and applies the SDF rule (project to phi = r_HR, drop the inward normal
// velocity relative to the boundary), then writes the particle back.
#include <cuda_runtime.h>

#include "gs_internal.cuh"
#include "sdf.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kBuf = 64;   // staged LR per warp; flushed at >= 32

__device__ __forceinline__ int cell_coord(float x, float o, float inv_h, int dim)
{
    float a = __fmul_rn(__fsub_rn(x, o), inv_h);
    float f = floorf(a);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(dim - 1)) return dim - 1;
    return (int)f;
}

__device__ __forceinline__ void hr_boundary(float& x, float& y, float& z, float& vx, float& vy, float& vz,
                                            const gs_sdf* sdf, int n_sdf, float rh)
{
    for (int s = 0; s < n_sdf; ++s) {
        const gs_sdf& b = sdf[s];
        int nc = sdf_components(b.kind);
        for (int c = 0; c < nc; ++c) {
            SdfHit h = sdf_eval(b, c, x, y, z);
            if (h.phi < rh) {
                float push = rh - h.phi;
                x += push * h.nx;
                y += push * h.ny;
                z += push * h.nz;
                float vn = (vx - b.vel[0]) * h.nx + (vy - b.vel[1]) * h.ny + (vz - b.vel[2]) * h.nz;
                if (vn < 0.0f) {
                    vx -= vn * h.nx;
                    vy -= vn * h.ny;
                    vz -= vn * h.nz;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_upsample(const UpsampleArgs a)
{
    __shared__ float4 s_pos[kWarps][kBuf];
    __shared__ float4 s_vel[kWarps][kBuf];
    __shared__ gs_sdf s_sdf[GS_MAX_SDF];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < a.n_sdf; k += kThreads) s_sdf[k] = a.sdf[k];
    __syncthreads();

    const int64_t first = ((int64_t)blockIdx.x * kWarps + warp) * 32;
    if (first >= a.m) return;
    const int64_t i = first + lane;
    const bool valid = i < a.m;

    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        p = __ldcs(a.hr_pos + i);
        v = __ldcs(a.hr_vel + i);
    }

    // bounding box of the warp's particles
    float lx = valid ? p.x : 3.0e38f, ly = valid ? p.y : 3.0e38f, lz = valid ? p.z : 3.0e38f;
    float hx = valid ? p.x : -3.0e38f, hy = valid ? p.y : -3.0e38f, hz = valid ? p.z : -3.0e38f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
    }

    const float R = 3.0f * a.r_low * (1.0f + 1.0e-5f);    // support, padded against rounding
    const float R2 = R * R;
    const float inv9r2 = 1.0f / (9.0f * a.r_low * a.r_low);
    const GridDev& g = a.g;
    const int cx0 = cell_coord(lx - R, g.ox, g.inv_h, g.dx), cx1 = cell_coord(hx + R, g.ox, g.inv_h, g.dx);
    const int cy0 = cell_coord(ly - R, g.oy, g.inv_h, g.dy), cy1 = cell_coord(hy + R, g.oy, g.inv_h, g.dy);
    const int cz0 = cell_coord(lz - R, g.oz, g.inv_h, g.dz), cz1 = cell_coord(hz + R, g.oz, g.inv_h, g.dz);

    float S = 0.f, Vx = 0.f, Vy = 0.f, Vz = 0.f, wmax = 0.f;
    int cnt = 0;
    const unsigned lt = (1u << lane) - 1u;
    float4* bp = s_pos[warp];
    float4* bv = s_vel[warp];

    auto flush = [&](int count) {
        __syncwarp();
        for (int k = 0; k < count; ++k) {
            float4 q = bp[k];
            float4 qv = bv[k];
            float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            float d2 = dx * dx + dy * dy + dz * dz;
            float t = fmaxf(1.0f - d2 * inv9r2, 0.0f);
            float w = t * t * t;
            S += w;
            Vx = fmaf(w, qv.x, Vx);
            Vy = fmaf(w, qv.y, Vy);
            Vz = fmaf(w, qv.z, Vz);
            wmax = fmaxf(wmax, w);
        }
        __syncwarp();
    };

    for (int cz = cz0; cz <= cz1; ++cz) {
        for (int cy = cy0; cy <= cy1; ++cy) {
            const int64_t row = ((int64_t)cz * g.dy + cy) * g.dx;
            const uint32_t b = a.cell_start[row + cx0];
            const uint32_t e = a.cell_start[row + cx1 + 1];
            for (uint32_t base = b; base < e; base += 32) {
                const uint32_t j = base + lane;
                bool take = false;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < e) {
                    q = __ldg(a.lr_spos + j);
                    float ex = fmaxf(fmaxf(lx - q.x, q.x - hx), 0.0f);
                    float ey = fmaxf(fmaxf(ly - q.y, q.y - hy), 0.0f);
                    float ez = fmaxf(fmaxf(lz - q.z, q.z - hz), 0.0f);
                    take = ex * ex + ey * ey + ez * ez < R2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (take) {
                    int slot = cnt + __popc(bal & lt);
                    bp[slot] = q;
                    bv[slot] = __ldg(a.lr_svel + j);
                }
                cnt += __popc(bal);
                if (cnt >= 32) {
                    flush(cnt);
                    cnt = 0;
                }
            }
        }
    }
    if (cnt > 0) flush(cnt);

    if (!valid) return;
    float vtx = 0.f, vty = 0.f, vtz = 0.f;
    if (S > 0.0f) {
        vtx = Vx / S;
        vty = Vy / S;
        vtz = Vz / S;
    }
    const bool A = wmax <= a.c1;
    const bool B = S > 0.0f && wmax >= a.c2 * S;
    const float alpha = (A || B) ? 1.0f - wmax : 0.0f;
    float nvx = (1.0f - alpha) * vtx + alpha * (v.x + a.dt * a.gx);
    float nvy = (1.0f - alpha) * vty + alpha * (v.y + a.dt * a.gy);
    float nvz = (1.0f - alpha) * vtz + alpha * (v.z + a.dt * a.gz);
    float nx = p.x + a.dt * nvx, ny = p.y + a.dt * nvy, nz = p.z + a.dt * nvz;
    hr_boundary(nx, ny, nz, nvx, nvy, nvz, s_sdf, a.n_sdf, a.r_high);
    __stcs(a.out_pos + i, make_float4(nx, ny, nz, p.w));
    __stcs(a.out_vel + i, make_float4(nvx, nvy, nvz, 0.0f));
}

}  // namespace

cudaError_t gs_launch_upsample(cudaStream_t s, const UpsampleArgs& a, int64_t* launches)
{
    if (a.m <= 0) return cudaSuccess;
    int64_t warps = (a.m + 31) / 32;
    k_upsample<<<gs_blocks(warps, kWarps), kThreads, 0, s>>>(a);
    *launches += 1;
    return cudaGetLastError();
}
