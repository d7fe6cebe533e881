// upsample.cu -- HR upsampling of Sec. 4 as one fused kernel.
//
// Each warp owns 32 consecutive HR particles of the cell-ordered HR array
// (one float4 position + one float4 velocity each, read once, written once).
// The warp splits its lanes into spatially compact groups, bounds each group
// with an axis-aligned box, and walks the rows of LR grid cells that the box
// widened by the 3 r_LR support touches (each row of cells is one contiguous
// run of the cell-ordered LR array; all rows' ranges are fetched at once and
// the concatenated range is walked 32 candidates at a time).  LR particles
// within 3 r_LR of the box are staged in shared memory.
// Every lane then sums the kernel weights of Sec. 4 over the staged LR set:
//   w = max(0, 1 - |x_ij|^2 / (9 r_LR^2))^3,  S = sum w,  V = sum w v_j,
//   wmax = max w,  vtilde = V / S (0 when S = 0),
//   alpha = 1 - wmax if wmax <= c1 or wmax / S >= c2, else 0,
//   v = (1 - alpha) vtilde + alpha (v + dt g),  x = x + dt v,
// and applies the SDF rule (project to phi = r_HR, drop the inward normal
// velocity relative to the boundary), then writes the particle back.
// LR particles of infinite mass (w of the position 0: sampled boundaries and
// rigid bodies) are summed apart (per lane, in shared memory) and join the
// sums only where some grain has a positive weight, so an HR particle with
// no grain in reach moves ballistically instead of sticking to them
// (Sec. 4).  That handling lives in a second instantiation of the kernel;
// the LR binning before the gather raises a device flag when any LR particle
// has w = 0, and each instantiation returns at once unless the flag selects
// it, so scenes without such particles run the plain gather.
#include <cuda_runtime.h>

#include "gs_internal.cuh"
#include "sdf.cuh"

namespace {

constexpr int kBuf = 64;   // staged LR per warp; flushed at >= 32
// The staged LR set of a warp is eight arrays of kBuf floats (structure of
// arrays): 2 w_x, 2 w_y, 2 w_z, -|w|^2 (w the LR position relative to the
// group's centre in units of 3 r_LR), v_x, v_y, v_z, and the solid flag, so
// the evaluation reads four candidates of a component with one 16-byte load
// and evaluates them in packed pairs (f32x2 arithmetic).
enum { kAx = 0, kAy = kBuf, kAz = 2 * kBuf, kAw = 3 * kBuf, kVx = 4 * kBuf, kVy = 5 * kBuf, kVz = 6 * kBuf,
       kFl = 7 * kBuf, kStage = 8 * kBuf };

__device__ __forceinline__ int cell_coord(float x, float o, float inv_h, int dim)
{
    float a = __fmul_rn(__fsub_rn(x, o), inv_h);
    float f = floorf(a);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(dim - 1)) return dim - 1;
    return (int)f;
}

// One wall of a box interior along axis x_k: wall at `w`, inward normal sign
// sg (+1 for the lower wall, -1 for the upper), boundary velocity u.
__device__ __forceinline__ void wall_project(float& x, float& v, float w, float sg, float u, float rh)
{
    const float phi = sg * (x - w);
    if (phi < rh) {
        x += sg * (rh - phi);
        const float vn = sg * (v - u);
        if (vn < 0.0f) v -= sg * vn;
    }
}

__device__ __forceinline__ void hr_boundary(float& x, float& y, float& z, float& vx, float& vy, float& vz,
                                            const gs_sdf* sdf, int n_sdf, float rh)
{
    for (int s = 0; s < n_sdf; ++s) {
        const gs_sdf& b = sdf[s];
        if (b.kind == GS_SDF_BOX_INTERIOR) {
            // the six walls in the order x-lo, x-hi, y-lo, y-hi, z-lo, z-hi
            wall_project(x, vx, b.p[0], 1.0f, b.vel[0], rh);
            wall_project(x, vx, b.p[3], -1.0f, b.vel[0], rh);
            wall_project(y, vy, b.p[1], 1.0f, b.vel[1], rh);
            wall_project(y, vy, b.p[4], -1.0f, b.vel[1], rh);
            wall_project(z, vz, b.p[2], 1.0f, b.vel[2], rh);
            wall_project(z, vz, b.p[5], -1.0f, b.vel[2], rh);
            continue;
        }
        if (sdf_far(b, x, y, z, rh)) continue;
        SdfHit h = sdf_eval(b, 0, x, y, z);
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

// Order-preserving map of non-NaN floats onto unsigned integers (and back),
// so that a warp's minimum or maximum of a float is one integer reduction.
__device__ __forceinline__ unsigned f2ord(float f)
{
    const unsigned u = __float_as_uint(f);
    return u ^ ((u & 0x80000000u) ? 0xffffffffu : 0x80000000u);
}

__device__ __forceinline__ float ord2f(unsigned u)
{
    return __uint_as_float(u ^ ((u & 0x80000000u) ? 0x80000000u : 0xffffffffu));
}

// Lanes whose sub-cells (side h/2) are within one of the group leader's are
// gathered together; a warp that straddles a jump in the cell order (the end
// of a row or a slab, or particles that drifted since the last reorder)
// splits into several compact groups instead of one box across the domain.
__device__ __forceinline__ int sub_floor(float x, float o, float inv_h)
{
    float a = __fmul_rn(__fsub_rn(x, o), inv_h);
    float f = floorf(__fmul_rn(a, 2.0f));
    f = fminf(fmaxf(f, -1.0e6f), 1.0e6f);
    return (int)f;
}

// One warp item: the 32 HR slots [32 item, 32 item + 32) of one scene.
// st: this warp's staged LR set (kStage floats).  sol (kSolid): this warp's
// 5 x 32 sums of solid particles (S, V, max w per lane), zero on entry and on
// return.
template <bool kSolid>
__device__ __forceinline__ void upsample_item(const UpsampleArgs& a, int64_t item, float* st, float* sol, int lane)
{
    const int64_t first = item * 32;
    const uint32_t tag = __ldg(a.hr_tag + first);          // the first slot of an item is never padding
    const SceneDev& sc = a.scenes[tag & ~kPadBit];
    const int64_t i = first + lane;
    const bool valid = i < sc.hr_end;

    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        p = __ldcs(a.hr_pos + i);
        v = __ldcs(a.hr_vel + i);
    }
    const GridDev& g = sc.g;
    const int sx = sub_floor(p.x, g.ox, g.inv_h), sy = sub_floor(p.y, g.oy, g.inv_h), sz = sub_floor(p.z, g.oz, g.inv_h);

    const float R = 3.0f * sc.r_low * (1.0f + 1.0e-5f);    // support, padded against rounding
    const float R2 = R * R;
    const unsigned lt = (1u << lane) - 1u;
    const float inv3r = 1.0f / (3.0f * sc.r_low);
    const int64_t coff = sc.cell_off;

    // grains: sums over even and odd staged slots (packed pairs), and the
    // largest clamped t (max w = tmax^3, the cube being monotone)
    float2 S2 = make_float2(0.f, 0.f), Vx2 = S2, Vy2 = S2, Vz2 = S2;
    float tmax = 0.f;
    bool any_solid = false;                                    // warp-uniform
    unsigned pending = __ballot_sync(0xffffffffu, valid);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int gx0 = __shfl_sync(0xffffffffu, sx, leader);
        const int gy0 = __shfl_sync(0xffffffffu, sy, leader);
        const int gz0 = __shfl_sync(0xffffffffu, sz, leader);
        const bool member = ((pending >> lane) & 1u) && abs(sx - gx0) <= 1 && abs(sy - gy0) <= 1 && abs(sz - gz0) <= 1;
        pending &= ~__ballot_sync(0xffffffffu, member);

        // the group's bounding box (non-members sit at +-3e38)
        const float lx = ord2f(__reduce_min_sync(0xffffffffu, f2ord(member ? p.x : 3.0e38f)));
        const float ly = ord2f(__reduce_min_sync(0xffffffffu, f2ord(member ? p.y : 3.0e38f)));
        const float lz = ord2f(__reduce_min_sync(0xffffffffu, f2ord(member ? p.z : 3.0e38f)));
        const float hx = ord2f(__reduce_max_sync(0xffffffffu, f2ord(member ? p.x : -3.0e38f)));
        const float hy = ord2f(__reduce_max_sync(0xffffffffu, f2ord(member ? p.y : -3.0e38f)));
        const float hz = ord2f(__reduce_max_sync(0xffffffffu, f2ord(member ? p.z : -3.0e38f)));
        const int cx0 = cell_coord(lx - R, g.ox, g.inv_h, g.dx), cx1 = cell_coord(hx + R, g.ox, g.inv_h, g.dx);
        const int cy0 = cell_coord(ly - R, g.oy, g.inv_h, g.dy), cy1 = cell_coord(hy + R, g.oy, g.inv_h, g.dy);
        const int cz0 = cell_coord(lz - R, g.oz, g.inv_h, g.dz), cz1 = cell_coord(hz + R, g.oz, g.inv_h, g.dz);
        const int ny = cy1 - cy0 + 1;
        const int nrows = ny * (cz1 - cz0 + 1);
        const float inv_ny = 1.0f / (float)ny;

        // Sec. 4 weight in the expanded form: with u = (x - c0) / (3 r_LR),
        //   1 - |x_i - x_j|^2 / (9 r_LR^2) = (1 - |u_i|^2) + 2 u_i . u_j - |u_j|^2.
        // Non-members sit far away (t hugely negative, weight exactly 0).
        const float c0x = 0.5f * (lx + hx), c0y = 0.5f * (ly + hy), c0z = 0.5f * (lz + hz);
        float ux = 1.0e4f, uy = 1.0e4f, uz = 1.0e4f, ci = -1.0e9f;
        if (member) {
            ux = (p.x - c0x) * inv3r;
            uy = (p.y - c0y) * inv3r;
            uz = (p.z - c0z) * inv3r;
            ci = 1.0f - (ux * ux + uy * uy + uz * uz);
        }

        int cnt = 0;
        bool batch_solid = false;
        const float2 u2x = make_float2(ux, ux), u2y = make_float2(uy, uy), u2z = make_float2(uz, uz);
        const float2 ci2 = make_float2(ci, ci);
        auto stage = [&](int slot, float4 c, float4 cv) {
            const float wx = (c.x - c0x) * inv3r, wy = (c.y - c0y) * inv3r, wz = (c.z - c0z) * inv3r;
            st[kAx + slot] = 2.0f * wx;
            st[kAy + slot] = 2.0f * wy;
            st[kAz + slot] = 2.0f * wz;
            st[kAw + slot] = -(wx * wx + wy * wy + wz * wz);
            st[kVx + slot] = cv.x;
            st[kVy + slot] = cv.y;
            st[kVz + slot] = cv.z;
            if constexpr (kSolid) st[kFl + slot] = c.w == 0.0f ? 1.0f : 0.0f;
        };
        auto flush = [&](int count, bool with_solid) {
            __syncwarp();
            if (kSolid && with_solid) {
                // the batch holds solid particles (rb.w = 1): their sums apart
                float s = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, sm = 0.f;
#pragma unroll 1
                for (int k = 0; k < count; ++k) {
                    float t = fmaf(st[kAx + k], ux, fmaf(st[kAy + k], uy, fmaf(st[kAz + k], uz, st[kAw + k] + ci)));
                    t = fmaxf(t, 0.0f);
                    const float w = t * t * t;
                    const float vx = st[kVx + k], vy = st[kVy + k], vz = st[kVz + k];
                    if (st[kFl + k] != 0.0f) {   // the same k on every lane: uniform
                        s += w;
                        sx = fmaf(w, vx, sx);
                        sy = fmaf(w, vy, sy);
                        sz = fmaf(w, vz, sz);
                        sm = fmaxf(sm, w);
                    } else {
                        S2.x += w;
                        Vx2.x = fmaf(w, vx, Vx2.x);
                        Vy2.x = fmaf(w, vy, Vy2.x);
                        Vz2.x = fmaf(w, vz, Vz2.x);
                        tmax = fmaxf(tmax, t);
                    }
                }
                sol[lane] += s;
                sol[32 + lane] += sx;
                sol[64 + lane] += sy;
                sol[96 + lane] += sz;
                sol[128 + lane] = fmaxf(sol[128 + lane], sm);
                any_solid = true;
                __syncwarp();
                return;
            }
            // pad to a multiple of 4 with weightless entries (finite values)
            const int L = (count + 3) & ~3;
            if (lane < L - count) {
                const int k = count + lane;
                st[kAx + k] = 0.0f;
                st[kAy + k] = 0.0f;
                st[kAz + k] = 0.0f;
                st[kAw + k] = -1.0e30f;
                st[kVx + k] = 0.0f;
                st[kVy + k] = 0.0f;
                st[kVz + k] = 0.0f;
            }
            __syncwarp();
#pragma unroll 1
            for (int k = 0; k < L; k += 4) {
                const float4 X = *reinterpret_cast<const float4*>(st + kAx + k);
                const float4 Y = *reinterpret_cast<const float4*>(st + kAy + k);
                const float4 Z = *reinterpret_cast<const float4*>(st + kAz + k);
                const float4 B = *reinterpret_cast<const float4*>(st + kAw + k);
                // t = (1 - |u|^2) + 2 u . w - |w|^2 for candidates (k, k+1) and (k+2, k+3)
                float2 t0 = __fadd2_rn(make_float2(B.x, B.y), ci2);
                float2 t1 = __fadd2_rn(make_float2(B.z, B.w), ci2);
                t0 = __ffma2_rn(make_float2(Z.x, Z.y), u2z, t0);
                t1 = __ffma2_rn(make_float2(Z.z, Z.w), u2z, t1);
                t0 = __ffma2_rn(make_float2(Y.x, Y.y), u2y, t0);
                t1 = __ffma2_rn(make_float2(Y.z, Y.w), u2y, t1);
                t0 = __ffma2_rn(make_float2(X.x, X.y), u2x, t0);
                t1 = __ffma2_rn(make_float2(X.z, X.w), u2x, t1);
                t0.x = fmaxf(t0.x, 0.0f);
                t0.y = fmaxf(t0.y, 0.0f);
                t1.x = fmaxf(t1.x, 0.0f);
                t1.y = fmaxf(t1.y, 0.0f);
                tmax = fmaxf(fmaxf(tmax, fmaxf(t0.x, t0.y)), fmaxf(t1.x, t1.y));
                const float2 w0 = __fmul2_rn(__fmul2_rn(t0, t0), t0);
                const float2 w1 = __fmul2_rn(__fmul2_rn(t1, t1), t1);
                const float4 VX = *reinterpret_cast<const float4*>(st + kVx + k);
                const float4 VY = *reinterpret_cast<const float4*>(st + kVy + k);
                const float4 VZ = *reinterpret_cast<const float4*>(st + kVz + k);
                S2 = __fadd2_rn(S2, w0);
                Vx2 = __ffma2_rn(w0, make_float2(VX.x, VX.y), Vx2);
                Vy2 = __ffma2_rn(w0, make_float2(VY.x, VY.y), Vy2);
                Vz2 = __ffma2_rn(w0, make_float2(VZ.x, VZ.y), Vz2);
                S2 = __fadd2_rn(S2, w1);
                Vx2 = __ffma2_rn(w1, make_float2(VX.z, VX.w), Vx2);
                Vy2 = __ffma2_rn(w1, make_float2(VY.z, VY.w), Vy2);
                Vz2 = __ffma2_rn(w1, make_float2(VZ.z, VZ.w), Vz2);
            }
            __syncwarp();
        };

        // rows of cells (cz, cy) in chunks of 32: lane j fetches row j's range
        for (int r0 = 0; r0 < nrows; r0 += 32) {
            const int j = r0 + lane;
            uint32_t rb = 0, len = 0;
            if (j < nrows) {
                const int jz = (int)(((float)j + 0.5f) * inv_ny);   // j / ny, exact for small j
                const int cz = cz0 + jz, cy = cy0 + (j - jz * ny);
                const int64_t row = ((int64_t)cz * g.dy + cy) * g.dx;
                rb = __ldg(a.cell_start + coff + row + cx0);
                len = __ldg(a.cell_start + coff + row + cx1 + 1) - rb;
            }
            uint32_t incl = len;   // inclusive prefix over rows
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - len;
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t f = base + lane;
                bool take = false;
                float4 c = make_float4(0.f, 0.f, 0.f, 0.f), cv = c;
                // row of flat index f: last row whose exclusive prefix is <= f
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t e = __shfl_sync(0xffffffffu, excl, lo + step);
                    if (lo + step < 32 && e <= f) lo += step;
                }
                const uint32_t rbase = __shfl_sync(0xffffffffu, rb, lo);
                const uint32_t rex = __shfl_sync(0xffffffffu, excl, lo);
                if (f < total) {
                    const uint32_t jj = rbase + (f - rex);
                    c = __ldg(a.lr_spos + jj);
                    cv = __ldg(a.lr_svel + jj);
                    const float ex = fmaxf(fmaxf(lx - c.x, c.x - hx), 0.0f);
                    const float ey = fmaxf(fmaxf(ly - c.y, c.y - hy), 0.0f);
                    const float ez = fmaxf(fmaxf(lz - c.z, c.z - hz), 0.0f);
                    take = ex * ex + ey * ey + ez * ez < R2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (take) stage(cnt + __popc(bal & lt), c, cv);
                cnt += __popc(bal);
                if constexpr (kSolid) batch_solid |= __any_sync(0xffffffffu, take && c.w == 0.0f);
                if (cnt >= 32) {
                    flush(cnt, batch_solid);
                    cnt = 0;
                    batch_solid = false;
                }
            }
        }
        if (cnt > 0) flush(cnt, batch_solid);
    }
    float S = S2.x + S2.y, Vx = Vx2.x + Vx2.y, Vy = Vy2.x + Vy2.y, Vz = Vz2.x + Vz2.y;
    float wmax = tmax * tmax * tmax;
    if (kSolid && any_solid) {
        // the solid particles count only where a grain has a positive weight
        if (S > 0.0f) {
            S += sol[lane];
            Vx += sol[32 + lane];
            Vy += sol[64 + lane];
            Vz += sol[96 + lane];
            wmax = fmaxf(wmax, sol[128 + lane]);
        }
        for (int m = 0; m < 5; ++m) sol[32 * m + lane] = 0.0f;
        __syncwarp();
    }

    if (!valid) return;
    float vtx = 0.f, vty = 0.f, vtz = 0.f;
    if (S > 0.0f) {
        const float inv = 1.0f / S;
        vtx = Vx * inv;
        vty = Vy * inv;
        vtz = Vz * inv;
    }
    const bool A = wmax <= sc.c1;
    const bool B = S > 0.0f && wmax >= sc.c2 * S;
    const float alpha = (A || B) ? 1.0f - wmax : 0.0f;
    float nvx = (1.0f - alpha) * vtx + alpha * (v.x + a.dt * sc.gx);
    float nvy = (1.0f - alpha) * vty + alpha * (v.y + a.dt * sc.gy);
    float nvz = (1.0f - alpha) * vtz + alpha * (v.z + a.dt * sc.gz);
    float nx = p.x + a.dt * nvx, ny = p.y + a.dt * nvy, nz = p.z + a.dt * nvz;
    hr_boundary(nx, ny, nz, nvx, nvy, nvz, a.sdf + sc.sdf_begin, sc.n_sdf, sc.r_high);
    __stcs(a.out_pos + i, make_float4(nx, ny, nz, p.w));
    __stcs(a.out_vel + i, make_float4(nvx, nvy, nvz, 0.0f));
}

template <int WARPS, bool kSolid>
__global__ void __launch_bounds__(WARPS * 32, 24 / WARPS) k_upsample(const UpsampleArgs a, int persistent)
{
    if ((*a.solid_flag != 0u) != kSolid) return;   // the other instantiation does the frame
    __shared__ __align__(16) float s_st[WARPS][kStage];
    __shared__ float s_sol[kSolid ? WARPS : 1][5 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (kSolid) {
        for (int m = 0; m < 5; ++m) s_sol[warp][32 * m + lane] = 0.0f;
        __syncwarp();
    }
    // One call site for both launch modes, so both run the same code.  In
    // the persistent mode warps pull items until the counter passes
    // n_warps; every warp leaves after at most n_warps + 1 iterations.
    // Items are counted from a.item_begin (a slab of the HR slots).
    for (int64_t guard = 0; guard <= a.n_warps; ++guard) {
        int64_t item;
        if (persistent) {
            unsigned it = 0;
            if (lane == 0) it = atomicAdd(a.work, 1u);
            item = (int64_t)__shfl_sync(0xffffffffu, it, 0);
        } else {
            item = guard == 0 ? (int64_t)blockIdx.x * WARPS + warp : a.n_warps;
        }
        if (item >= a.n_warps) break;
        if (persistent) {
            // Pull the HR lines of the item one wave ahead into L2 (one lane
            // per 128-byte line); whichever warp takes that item then finds
            // its first loads there.  ahead < n_warps keeps the address
            // inside the launch's items, which lie inside the slot arrays.
            const int64_t ahead = item + (int64_t)gridDim.x * WARPS;
            if (ahead < a.n_warps && (lane & 7) == 0) {
                const int64_t line = (a.item_begin + ahead) * 32 + lane;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.hr_pos + line));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.hr_vel + line));
            }
        }
        upsample_item<kSolid>(a, a.item_begin + item, s_st[warp], s_sol[kSolid ? warp : 0], lane);
    }
}

}  // namespace

template <int WARPS>
static cudaError_t launch_w(cudaStream_t s, const UpsampleArgs& a, int blocks_per_sm, int sm_count)
{
    // both instantiations; the one the device flag does not select returns
    if (blocks_per_sm <= 0) {
        k_upsample<WARPS, false><<<gs_blocks(a.n_warps, WARPS), WARPS * 32, 0, s>>>(a, 0);
        k_upsample<WARPS, true><<<gs_blocks(a.n_warps, WARPS), WARPS * 32, 0, s>>>(a, 0);
    } else {
        int64_t nb = (int64_t)blocks_per_sm * sm_count;
        const int64_t need = (a.n_warps + WARPS - 1) / WARPS;
        if (nb > need) nb = need;
        k_upsample<WARPS, false><<<(unsigned)nb, WARPS * 32, 0, s>>>(a, 1);
        k_upsample<WARPS, true><<<(unsigned)nb, WARPS * 32, 0, s>>>(a, 1);
    }
    return cudaGetLastError();
}

cudaError_t gs_launch_upsample(cudaStream_t s, const UpsampleArgs& a, int warps_per_block, int blocks_per_sm,
                               int sm_count, int64_t* launches)
{
    if (a.n_warps <= 0) return cudaSuccess;
    if (blocks_per_sm > 0) {
        cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e;
    switch (warps_per_block) {
    case 4: e = launch_w<4>(s, a, blocks_per_sm, sm_count); break;
    case 16: e = launch_w<16>(s, a, blocks_per_sm, sm_count); break;
    default: e = launch_w<8>(s, a, blocks_per_sm, sm_count); break;
    }
    *launches += 2;   // the two instantiations
    return e;
}
