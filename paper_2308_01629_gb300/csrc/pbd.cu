// pbd.cu -- one LR time step of Algorithm 1 (Sec. 3) on the GPU.
//
// The step runs in cell order: after prediction the LR set is binned on its
// predicted positions, every particle collects its candidate partners within
// the neighbour radius from the 27 surrounding cells once, and each Jacobi
// pass is one launch in which a thread gathers the corrections of all its
// active constraints (a per-particle gather instead of a scatter, so no
// atomics and a fixed summation order):
//   contact (Eqs. 1-2):   dx_i = -mhat_ij (2 r - |x_ij|) x_ij / |x_ij|,
//                         mhat_ij = w_i / (w_i + w_j), w = 1 / m*
//   friction (Eqs. 3-4):  relative displacement over the step so far
//                         (xt_i - x_i) - (xt_j - x_j), tangential part,
//                         static below 2 r mu_s, else scaled by
//                         min(2 r mu_k / |dx_perp|, 1)
//   averaging:            dx_i = (1 / n_i) sum_k dx_ik
// SDF contacts act as partners of infinite mass (mass ratio 1).  The
// stabilization passes evaluate their contacts on x and move x and xt; the
// solver passes evaluate and move xt.
#include <cuda_runtime.h>

#include "gs_internal.cuh"
#include "pbd_common.cuh"
#include "sdf.cuh"

namespace {

__global__ void k_predict(const PbdArgs a, const float4* __restrict__ pos, const float4* __restrict__ vel,
                          float4* __restrict__ xt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const SceneDev& sc = a.scenes[a.lr_scene[i]];
    float4 x = pos[i], v = vel[i];
    float vx = v.x + a.dt * sc.gx, vy = v.y + a.dt * sc.gy, vz = v.z + a.dt * sc.gz;
    // 1/m* = (1/m) e^{h(x)}, h = k (z - ground), at the start-of-step position
    float ws = x.w * expf(sc.mass_k * (x.z - sc.ground_z));
    xt[i] = make_float4(x.x + a.dt * vx, x.y + a.dt * vy, x.z + a.dt * vz, ws);
}

__global__ void k_step_gather(int64_t n, const uint32_t* __restrict__ idx, const float4* __restrict__ xt,
                              const float4* __restrict__ pos, float4* __restrict__ s_xt, float4* __restrict__ s_x)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t i = idx[p];
    s_xt[p] = xt[i];
    s_x[p] = pos[i];   // w carries the inverse mass
}

// Candidate partners of every particle within the neighbour radius, in
// ascending sorted index row by row of the 27 surrounding cells.  Four lanes
// share one particle and take every fourth candidate of a row; a ballot over
// the four keeps the list in ascending order.
constexpr int kNbrLanes = 4;

__global__ void __launch_bounds__(128) k_neighbors(const PbdArgs a, const float4* __restrict__ s_xt,
                                                   const uint32_t* __restrict__ skeys,
                                                   const uint32_t* __restrict__ cell_start, uint32_t* __restrict__ nbr,
                                                   uint32_t* __restrict__ cnt, int cap, int* err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = t / kNbrLanes;
    const int sub = (int)(t % kNbrLanes);
    const int gbase = (int)(threadIdx.x & 31u) & ~(kNbrLanes - 1);
    const unsigned gmask = ((1u << kNbrLanes) - 1u) << gbase;
    if (p >= a.n) return;   // the four lanes of a particle leave together
    const SceneDev& sc = a.scenes[a.lr_scene[p]];
    const GridDev& g = sc.g;
    const float4 xp = s_xt[p];
    const uint32_t c = skeys[p] - sc.cell_off;
    const int cx = (int)(c % (uint32_t)g.dx);
    const int cy = (int)((c / (uint32_t)g.dx) % (uint32_t)g.dy);
    const int cz = (int)(c / ((uint32_t)g.dx * (uint32_t)g.dy));
    const float rc2 = sc.rc * sc.rc;
    const int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < g.dx ? cx + 1 : g.dx - 1;
    const unsigned below = (1u << sub) - 1u;
    int k = 0;
    for (int z = cz - 1; z <= cz + 1; ++z) {
        if (z < 0 || z >= g.dz) continue;
        for (int y = cy - 1; y <= cy + 1; ++y) {
            if (y < 0 || y >= g.dy) continue;
            const int64_t row = (int64_t)sc.cell_off + ((int64_t)z * g.dy + y) * g.dx;
            const uint32_t b = cell_start[row + x0], e = cell_start[row + x1 + 1];
            for (uint32_t q0 = b; q0 < e; q0 += kNbrLanes) {
                const uint32_t q = q0 + (uint32_t)sub;
                bool take = false;
                if (q < e && (int64_t)q != p) {
                    const float4 xq = s_xt[q];
                    const float dx = xq.x - xp.x, dy = xq.y - xp.y, dz = xq.z - xp.z;
                    take = dx * dx + dy * dy + dz * dz < rc2;
                }
                const unsigned bal = __ballot_sync(gmask, take) >> gbase;
                if (take) {
                    const int pos = k + __popc(bal & below);
                    if (pos < cap) nbr[(int64_t)pos * a.n + p] = q;
                }
                k += __popc(bal);
            }
        }
    }
    if (sub != 0) return;
    if (k > cap) {
        atomicOr(err, GS_DEVERR_NEIGHBOR_CAP);
        k = cap;
    }
    cnt[p] = (uint32_t)k;
}

// kLanes lanes share one particle: lane `sub` takes candidates sub, sub +
// kLanes, ... two at a time (so the loads of both are in flight together)
// and the SDF components whose running index is sub modulo kLanes; the
// partial sums are added with shuffles in a fixed order and lane 0 writes
// the particle.
constexpr int kLanes = 4;

struct PassAcc {
    float Dx, Dy, Dz;
    int n;
};

__device__ __forceinline__ void pair_term(PassAcc& acc, const SceneDev& sc, int stab, float4 yp, float wp, float dpx,
                                          float dpy, float dpz, float4 xtq, float4 xq, float d0)
{
    const float4 yq = stab ? xq : xtq;
    const PairGeo pg = pair_geo(yp, yq);
    if (!(pg.d < d0) || pg.d2 == 0.0f) return;
    const float wsum = wp + xtq.w;
    if (!(wsum > 0.0f)) return;
    const float m = wp / wsum;
    const float pen = d0 - pg.d;
    const float s = m * pen / pg.d;
    acc.Dx -= s * pg.ex;
    acc.Dy -= s * pg.ey;
    acc.Dz -= s * pg.ez;
    if (!stab) {
        const float rx = dpx - (xtq.x - xq.x), ry = dpy - (xtq.y - xq.y), rz = dpz - (xtq.z - xq.z);
        const Tangent tg = tangent_part(rx, ry, rz, pg.ex, pg.ey, pg.ez, pg.d2);
        const float base = sc.friction_mode == 1 ? pen : d0;
        const float f = m * friction_scale(tg.L, base * sc.mu_s, base * sc.mu_k);
        acc.Dx -= f * tg.tx;
        acc.Dy -= f * tg.ty;
        acc.Dz -= f * tg.tz;
    }
    ++acc.n;
}

__global__ void __launch_bounds__(128) k_pass(const PbdArgs a, int stab, const float4* __restrict__ x_in,
                                              const float4* __restrict__ xt_in, float4* __restrict__ x_out,
                                              float4* __restrict__ xt_out, const uint32_t* __restrict__ nbr,
                                              const uint32_t* __restrict__ cnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = t / kLanes;
    const int sub = (int)(t % kLanes);
    const bool valid = p < a.n;
    const SceneDev& sc = a.scenes[valid ? a.lr_scene[p] : 0];
    const float d0 = 2.0f * sc.r_low;
    float4 xtp = make_float4(0.f, 0.f, 0.f, 0.f), xp = xtp;
    int nc = 0;
    if (valid) {
        xtp = xt_in[p];
        xp = x_in[p];
        nc = (int)cnt[p];
    }
    const float4 yp = stab ? xp : xtp;          // positions the constraints are evaluated on
    const float wp = xtp.w;                      // inverse height-scaled mass
    const float dpx = xtp.x - xp.x, dpy = xtp.y - xp.y, dpz = xtp.z - xp.z;
    PassAcc acc = {0.f, 0.f, 0.f, 0};
    for (int k = sub; k < nc; k += 2 * kLanes) {
        const int k2 = k + kLanes;
        const bool two = k2 < nc;
        const uint32_t q1 = nbr[(int64_t)k * a.n + p];
        const uint32_t q2 = two ? nbr[(int64_t)k2 * a.n + p] : q1;
        const float4 xtq1 = xt_in[q1], xq1 = x_in[q1];
        const float4 xtq2 = xt_in[q2], xq2 = x_in[q2];
        pair_term(acc, sc, stab, yp, wp, dpx, dpy, dpz, xtq1, xq1, d0);
        if (two) pair_term(acc, sc, stab, yp, wp, dpx, dpy, dpz, xtq2, xq2, d0);
    }
    if (valid && wp > 0.0f) {
        int gc = 0;
        for (int sI = 0; sI < sc.n_sdf; ++sI) {
            const gs_sdf& b = a.sdf[sc.sdf_begin + sI];
            const int ncomp = sdf_components(b.kind);
            for (int c = 0; c < ncomp; ++c, ++gc) {
                if ((gc & (kLanes - 1)) != sub) continue;
                const SdfHit h = sdf_eval(b, c, yp.x, yp.y, yp.z);
                if (!(h.phi < sc.r_low)) continue;
                const float pen = sc.r_low - h.phi;
                acc.Dx += pen * h.nx;
                acc.Dy += pen * h.ny;
                acc.Dz += pen * h.nz;
                if (!stab) {
                    const float bmu_s = sqrtf(sc.mu_s * b.mu_s), bmu_k = sqrtf(sc.mu_k * b.mu_k);
                    const float rx = dpx - b.vel[0] * a.dt, ry = dpy - b.vel[1] * a.dt, rz = dpz - b.vel[2] * a.dt;
                    const Tangent tg = tangent_part(rx, ry, rz, h.nx, h.ny, h.nz, 1.0f);
                    const float base = sc.friction_mode == 1 ? pen : d0;
                    const float f = friction_scale(tg.L, base * bmu_s, base * bmu_k);
                    acc.Dx -= f * tg.tx;
                    acc.Dy -= f * tg.ty;
                    acc.Dz -= f * tg.tz;
                }
                ++acc.n;
            }
        }
    }
#pragma unroll
    for (int o = 1; o < kLanes; o <<= 1) {
        acc.Dx += __shfl_xor_sync(0xffffffffu, acc.Dx, o);
        acc.Dy += __shfl_xor_sync(0xffffffffu, acc.Dy, o);
        acc.Dz += __shfl_xor_sync(0xffffffffu, acc.Dz, o);
        acc.n += __shfl_xor_sync(0xffffffffu, acc.n, o);
    }
    if (!valid || sub != 0) return;
    float4 nt = xtp;
    float4 nx = xp;
    if (acc.n > 0) {
        const float inv = 1.0f / (float)acc.n;
        const float ux = acc.Dx * inv, uy = acc.Dy * inv, uz = acc.Dz * inv;
        nt.x += ux;
        nt.y += uy;
        nt.z += uz;
        if (stab) {
            nx.x += ux;
            nx.y += uy;
            nx.z += uz;
        }
    }
    xt_out[p] = nt;
    if (stab) x_out[p] = nx;
}

__global__ void k_finalize(const PbdArgs a, const uint32_t* __restrict__ idx, const float4* __restrict__ s_x,
                           const float4* __restrict__ s_xt, float4* __restrict__ pos, float4* __restrict__ vel)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    const uint32_t i = idx[p];
    const float4 x = s_x[p], xt = s_xt[p];
    vel[i] = make_float4((xt.x - x.x) / a.dt, (xt.y - x.y) / a.dt, (xt.z - x.z) / a.dt, 0.0f);
    pos[i] = make_float4(xt.x, xt.y, xt.z, x.w);
}

}  // namespace

cudaError_t gs_launch_predict(cudaStream_t s, const PbdArgs& a, const float4* pos, const float4* vel, float4* xt,
                              int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_predict<<<gs_blocks(a.n, 256), 256, 0, s>>>(a, pos, vel, xt);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_step_gather(cudaStream_t s, int64_t n, const uint32_t* idx, const float4* xt,
                                  const float4* pos, float4* s_xt, float4* s_x, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    k_step_gather<<<gs_blocks(n, 256), 256, 0, s>>>(n, idx, xt, pos, s_xt, s_x);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_neighbors(cudaStream_t s, const PbdArgs& a, const float4* s_xt, const uint32_t* skeys,
                                const uint32_t* cell_start, uint32_t* nbr, uint32_t* cnt, int cap, int* err,
                                int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_neighbors<<<gs_blocks(a.n * kNbrLanes, 128), 128, 0, s>>>(a, s_xt, skeys, cell_start, nbr, cnt, cap, err);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_pass(cudaStream_t s, const PbdArgs& a, int stab, const float4* x_in, const float4* xt_in,
                           float4* x_out, float4* xt_out, const uint32_t* nbr, const uint32_t* cnt,
                           int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_pass<<<gs_blocks(a.n * kLanes, 128), 128, 0, s>>>(a, stab, x_in, xt_in, x_out, xt_out, nbr, cnt);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_finalize(cudaStream_t s, const PbdArgs& a, const uint32_t* idx, const float4* s_x,
                               const float4* s_xt, float4* pos, float4* vel, int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_finalize<<<gs_blocks(a.n, 256), 256, 0, s>>>(a, idx, s_x, s_xt, pos, vel);
    *launches += 1;
    return cudaGetLastError();
}
