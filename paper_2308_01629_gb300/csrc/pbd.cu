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
//                         min(2 r mu_k / |dx_perp|, 1); with grain
//                         materials mu = sqrt(mu_i mu_j) per pair (Sec. 3)
//   averaging:            dx_i = (1 / n_i) sum_k dx_ik
// SDF contacts act as partners of infinite mass (mass ratio 1), as do LR
// particles of inverse mass 0 (sampled boundaries and rigid bodies, which
// move with their prescribed velocity and feel no gravity).  The
// stabilization passes evaluate their contacts on x and move x and xt; the
// solver passes evaluate and move xt.
#include <cuda_runtime.h>

#include <algorithm>

#include "grid.cuh"
#include "gs_internal.cuh"
#include "pbd_common.cuh"
#include "sdf.cuh"

namespace {

// The step length: a kernel parameter, or (adaptive frames) the value the
// substep picker left in device memory.
__device__ __forceinline__ float step_dt(const PbdArgs& a) { return a.dt_dev ? *a.dt_dev : a.dt; }

// |v| / (2 r_LR) in float32 with correctly rounded operations and no fused
// multiply-add (the CFL rate of gs_frame_adaptive), as float bits: the
// value is >= 0, so the bits order like the values.
__device__ __forceinline__ unsigned cfl_rate_bits(float vx, float vy, float vz, float r_low)
{
    const float s = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    return __float_as_uint(__fdiv_rn(__fsqrt_rn(s), __fmul_rn(2.0f, r_low)));
}

__global__ void k_predict(const PbdArgs a, const float4* __restrict__ pos, const float4* __restrict__ vel,
                          float4* __restrict__ xt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const SceneDev& sc = a.scenes[a.lr_scene[i]];
    const float dt = step_dt(a);
    float4 x = pos[i], v = vel[i];
    // particles of infinite mass (1/m = 0: sampled boundaries, rigid bodies)
    // keep their prescribed velocity
    const float gdt = x.w > 0.0f ? dt : 0.0f;
    float vx = v.x + gdt * sc.gx, vy = v.y + gdt * sc.gy, vz = v.z + gdt * sc.gz;
    // 1/m* = (1/m) e^{h(x)}, h = k (z - ground), at the start-of-step position
    float ws = x.w * expf(sc.mass_k * (x.z - sc.ground_z));
    xt[i] = make_float4(x.x + dt * vx, x.y + dt * vy, x.z + dt * vz, ws);
}

// Prediction fused with the first stage of the binning: x~ as above, then
// the cell of x~ under the grid contract and its arrival rank in the cell.
__global__ void k_predict_keys(const PbdArgs a, const float4* __restrict__ pos, const float4* __restrict__ vel,
                               float4* __restrict__ xt, uint32_t* __restrict__ keys, uint32_t* __restrict__ rank,
                               uint32_t* __restrict__ cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const SceneDev& sc = a.scenes[a.lr_scene[i]];
    const float dt = step_dt(a);
    float4 x = pos[i], v = vel[i];
    const float gdt = x.w > 0.0f ? dt : 0.0f;   // no gravity for 1/m = 0
    float vx = v.x + gdt * sc.gx, vy = v.y + gdt * sc.gy, vz = v.z + gdt * sc.gz;
    float ws = x.w * expf(sc.mass_k * (x.z - sc.ground_z));
    const float4 p = make_float4(x.x + dt * vx, x.y + dt * vy, x.z + dt * vz, ws);
    xt[i] = p;
    const uint32_t cell = grid_cell_of(sc, p.x, p.y, p.z);
    keys[i] = cell;
    rank[i] = atomicAdd(cnt + cell, 1u);
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
// ascending sorted index row by row of the 27 surrounding cells.  The
// particles of a cell share their 27-cell candidate set, so one warp walks
// it once, 32 candidates at a time (lane j takes flat candidate j of the
// concatenated row ranges), and for each particle of the cell a ballot keeps
// its accepted candidates in ascending order.  Two ways to hand out cells,
// with the same lists: on a dense grid one warp per cell (empty cells leave
// at once); on a sparse grid (many small scenes) warp w takes the cells whose
// first sorted particle lies in [kNbrGroup w, kNbrGroup (w + 1)), so empty
// cells cost nothing.
constexpr int kNbrGroup = 8;

__device__ __forceinline__ void neighbors_of_cell(const PbdArgs& a, const float4* __restrict__ s_xt,
                                                  const uint32_t* __restrict__ cell_start, int64_t cell,
                                                  uint32_t* __restrict__ nbr, uint32_t* __restrict__ cnt, int cap,
                                                  int* err, int lane)
{
    const uint32_t pb = __ldg(cell_start + cell), pe = __ldg(cell_start + cell + 1);
    const SceneDev& sc = a.scenes[a.lr_scene[pb]];
    const GridDev& g = sc.g;
    const uint32_t c = (uint32_t)(cell - sc.cell_off);
    const int cx = (int)(c % (uint32_t)g.dx);
    const int cy = (int)((c / (uint32_t)g.dx) % (uint32_t)g.dy);
    const int cz = (int)(c / ((uint32_t)g.dx * (uint32_t)g.dy));
    const float rc2 = sc.rc * sc.rc;
    const int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < g.dx ? cx + 1 : g.dx - 1;
    // lane r < 9 fetches row r = (z, y) of the 3 x 3 rows around the cell
    uint32_t rb = 0, len = 0;
    if (lane < 9) {
        const int z = cz - 1 + lane / 3, y = cy - 1 + lane % 3;
        if (z >= 0 && z < g.dz && y >= 0 && y < g.dy) {
            const int64_t row = (int64_t)sc.cell_off + ((int64_t)z * g.dy + y) * g.dx;
            rb = __ldg(cell_start + row + x0);
            len = __ldg(cell_start + row + x1 + 1) - rb;
        }
    }
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - len;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 8);
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t i0 = pb; i0 < pe; i0 += 32) {       // the cell's particles, 32 at a time
        const uint32_t mine = i0 + (uint32_t)lane;
        const bool own = mine < pe;
        const float4 xo = own ? s_xt[mine] : make_float4(0.f, 0.f, 0.f, 0.f);
        int k = 0;                                      // lane j: count of particle i0 + j
        const int np = (int)min(pe - i0, 32u);
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t f = base + (uint32_t)lane;
            // row of flat index f: last row whose exclusive prefix is <= f
            int r = 0;
#pragma unroll
            for (int step = 8; step > 0; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, excl, (r + step) & 31);
                if (r + step < 9 && e <= f) r += step;
            }
            const uint32_t q = __shfl_sync(0xffffffffu, rb, r) + (f - __shfl_sync(0xffffffffu, excl, r));
            const bool in = f < total;
            const float4 xq = in ? s_xt[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int j = 0; j < np; ++j) {
                const float px = __shfl_sync(0xffffffffu, xo.x, j);
                const float py = __shfl_sync(0xffffffffu, xo.y, j);
                const float pz = __shfl_sync(0xffffffffu, xo.z, j);
                const float dx = xq.x - px, dy = xq.y - py, dz = xq.z - pz;
                const bool take = in && q != i0 + (uint32_t)j && dx * dx + dy * dy + dz * dz < rc2;
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                const int kj = __shfl_sync(0xffffffffu, k, j);
                if (take) {
                    const int pos = kj + __popc(bal & lt);
                    if (pos < cap) nbr[(int64_t)pos * a.n + i0 + j] = q;
                }
                if (lane == j) k += __popc(bal);
            }
        }
        if (own) {
            if (k > cap) {
                atomicOr(err, GS_DEVERR_NEIGHBOR_CAP);
                k = cap;
            }
            cnt[mine] = (uint32_t)k;
        }
    }
}

__global__ void __launch_bounds__(128) k_neighbors_cells(const PbdArgs a, const float4* __restrict__ s_xt,
                                                         const uint32_t* __restrict__ cell_start, int64_t n_cell,
                                                         uint32_t* __restrict__ nbr, uint32_t* __restrict__ cnt,
                                                         int cap, int* err)
{
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= n_cell) return;   // whole warps leave together
    if (__ldg(cell_start + cell) == __ldg(cell_start + cell + 1)) return;
    neighbors_of_cell(a, s_xt, cell_start, cell, nbr, cnt, cap, err, lane);
}

__global__ void __launch_bounds__(128) k_neighbors(const PbdArgs a, const float4* __restrict__ s_xt,
                                                   const uint32_t* __restrict__ skeys,
                                                   const uint32_t* __restrict__ cell_start,
                                                   uint32_t* __restrict__ nbr, uint32_t* __restrict__ cnt, int cap,
                                                   int* err)
{
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t p = w * kNbrGroup + lane;
    bool head = false;
    uint32_t key = 0;
    if (lane < kNbrGroup && p < a.n) {
        key = __ldg(skeys + p);
        head = p == 0 || __ldg(skeys + p - 1) != key;   // the first particle of its cell
    }
    unsigned heads = __ballot_sync(0xffffffffu, head);
    while (heads) {                                    // warp-uniform
        const int j = __ffs(heads) - 1;
        heads &= heads - 1u;
        const int64_t cell = (int64_t)__shfl_sync(0xffffffffu, key, j);
        neighbors_of_cell(a, s_xt, cell_start, cell, nbr, cnt, cap, err, lane);
    }
}

// kLanes lanes share one particle: lane `sub` takes candidates sub, sub +
// kLanes, ... (their distances kDistGroup at a time, the contact terms of
// those that may touch kContactGroup at a time, loads in flight together)
// and the SDF components whose running index is sub modulo kLanes; the
// partial sums are added with shuffles in a fixed order and lane 0 writes
// the particle.
constexpr int kLanes = 2;
constexpr int kDistGroup = 4;      // candidate distances whose loads are in flight together
constexpr int kContactGroup = 2;   // contact terms whose loads are in flight together

struct PassAcc {
    float Dx, Dy, Dz;
    int n;
};

// mu_s, mu_k: the pair's friction coefficients (the scene's, or the cross
// coefficients of the two grains' materials)
__device__ __forceinline__ void pair_term(PassAcc& acc, const SceneDev& sc, int stab, float4 yp, float wp, float dpx,
                                          float dpy, float dpz, float4 xtq, float4 xq, float d0, float mu_s,
                                          float mu_k)
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
        const float f = m * friction_scale(tg.L, base * mu_s, base * mu_k);
        acc.Dx -= f * tg.tx;
        acc.Dy -= f * tg.ty;
        acc.Dz -= f * tg.tz;
    }
    ++acc.n;
}

// Loads and stores of the position buffers.  The per-pass kernel reads
// buffers that no thread of the launch writes.  The persistent solver reads
// buffers other blocks wrote before the last grid barrier: plain (weak,
// L1-cacheable) loads, which the barrier's fences order after those writes,
// but never the non-coherent read-only path a const __restrict__ pointer
// may select, hence the explicit instruction.
template <bool kL2>
__device__ __forceinline__ float4 ld_pos(const float4* p)
{
    if constexpr (kL2) {
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(p));
        return v;
    } else {
        return *p;
    }
}
template <bool kL2>
__device__ __forceinline__ void st_pos(float4* p, float4 v)
{
    if constexpr (kL2) __stcg(p, v);
    else *p = v;
}

// One Jacobi pass of particle p (valid == p < n) by its kLanes lanes; every
// lane of the warp takes part (the partial sums meet in full-warp shuffles).
// Finalize of the step (last loop of Algorithm 1) folded into its last pass:
// v = (x~ - x) / dt and x = x~, written to original order through idx.
struct FinalOut {
    const uint32_t* idx;   // null: write the pass's outputs instead
    float4* pos;
    float4* vel;
    unsigned* rate;        // not null: atomic max of the CFL rate of the new velocities
};

// kMat: grains carry materials (their ids in the w of x); a pair's
// coefficients are the cross coefficients of the two materials, an SDF
// contact's sqrt(mu_i mu_b).
// kBody: rigid bodies; in solver passes a body particle also receives its
// shape-matching delta (R xo + c) - x~ (Sec. 3), counted once in n_i.
template <bool kL2, bool kMat, bool kBody = false>
__device__ __forceinline__ void pass_particle(const PbdArgs& a, int stab, int64_t p, bool valid, int sub,
                                              const float4* __restrict__ x_in, const float4* __restrict__ xt_in,
                                              float4* __restrict__ x_out, float4* __restrict__ xt_out,
                                              const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ cnt,
                                              const FinalOut fin = FinalOut{nullptr, nullptr, nullptr, nullptr})
{
    const SceneDev& sc = a.scenes[valid ? a.lr_scene[p] : 0];
    const float d0 = 2.0f * sc.r_low;
    float4 xtp = make_float4(0.f, 0.f, 0.f, 0.f), xp = xtp;
    int nc = 0;
    if (valid) {
        xtp = ld_pos<kL2>(xt_in + p);
        xp = ld_pos<kL2>(x_in + p);
        nc = (int)__ldg(cnt + p);
    }
    const uint32_t matp = kMat ? __float_as_uint(xp.w) : 0u;
    const float2* cross_p = kMat ? a.mu_cross + matp * GS_MAX_MATERIALS : nullptr;
    const float4 yp = stab ? xp : xtp;          // positions the constraints are evaluated on
    const float wp = xtp.w;                      // inverse height-scaled mass
    const float dpx = xtp.x - xp.x, dpy = xtp.y - xp.y, dpz = xtp.z - xp.z;
    PassAcc acc = {0.f, 0.f, 0.f, 0};
    // The lane's candidates k = sub, sub + kLanes, ... in windows of 32.
    // First their distances alone: kDistGroup at a time, the loads of the
    // evaluated positions in flight together, a bit per candidate that may
    // be in contact (a slightly wider test than pair_term's, which decides).
    // Then the contact terms for the marked candidates only, in candidate
    // order (the summation order of the lane).  A warp thus runs the contact
    // code as often as its busiest lane has contacts, not once per candidate
    // slot that any lane fills.
    const float4* yq_in = stab ? x_in : xt_in;
    const float d2_mark = d0 * d0 * 1.0001f;
    for (int w0 = sub; w0 < nc; w0 += 32 * kLanes) {
        const int wend = min(nc, w0 + 32 * kLanes);
        uint32_t marked = 0u;
        for (int k = w0; k < wend; k += kDistGroup * kLanes) {
            uint32_t q[kDistGroup];
            bool in[kDistGroup];
#pragma unroll
            for (int j = 0; j < kDistGroup; ++j) {
                in[j] = k + j * kLanes < wend;
                q[j] = in[j] ? __ldg(nbr + (int64_t)(k + j * kLanes) * a.n + p) : (uint32_t)p;
            }
            float4 yq[kDistGroup];
#pragma unroll
            for (int j = 0; j < kDistGroup; ++j) yq[j] = ld_pos<kL2>(yq_in + q[j]);
#pragma unroll
            for (int j = 0; j < kDistGroup; ++j) {
                const float ex = yq[j].x - yp.x, ey = yq[j].y - yp.y, ez = yq[j].z - yp.z;
                const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));   // as pair_geo
                if (in[j] && d2 < d2_mark) marked |= 1u << ((k - w0) / kLanes + j);
            }
        }
        // the marked candidates kContactGroup at a time, their loads in flight
        // together, then their terms in candidate order
        while (marked) {
            uint32_t q[kContactGroup];
            bool ok[kContactGroup];
#pragma unroll
            for (int j = 0; j < kContactGroup; ++j) {
                ok[j] = marked != 0u;
                const int li = ok[j] ? __ffs(marked) - 1 : 0;
                marked &= marked - 1u;
                q[j] = ok[j] ? __ldg(nbr + (int64_t)(w0 + li * kLanes) * a.n + p) : (uint32_t)p;
            }
            float4 xtq[kContactGroup], xq[kContactGroup];
#pragma unroll
            for (int j = 0; j < kContactGroup; ++j) {
                xtq[j] = ld_pos<kL2>(xt_in + q[j]);
                xq[j] = ld_pos<kL2>(x_in + q[j]);
            }
#pragma unroll
            for (int j = 0; j < kContactGroup; ++j) {
                if (!ok[j]) continue;
                if constexpr (kMat) {
                    const float2 mu = __ldg(cross_p + __float_as_uint(xq[j].w));
                    pair_term(acc, sc, stab, yp, wp, dpx, dpy, dpz, xtq[j], xq[j], d0, mu.x, mu.y);
                } else {
                    pair_term(acc, sc, stab, yp, wp, dpx, dpy, dpz, xtq[j], xq[j], d0, sc.mu_s, sc.mu_k);
                }
            }
        }
    }
    if (valid && wp > 0.0f) {
        float gmu_s = sc.mu_s, gmu_k = sc.mu_k;   // the grain's own coefficients
        if constexpr (kMat) {
            const float2 mu = __ldg(a.mu_mat + matp);
            gmu_s = mu.x;
            gmu_k = mu.y;
        }
        const float sdt = step_dt(a);
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
                    const float bmu_s = sqrtf(gmu_s * b.mu_s), bmu_k = sqrtf(gmu_k * b.mu_k);
                    const float rx = dpx - b.vel[0] * sdt, ry = dpy - b.vel[1] * sdt, rz = dpz - b.vel[2] * sdt;
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
    if constexpr (kBody) {
        if (!stab && valid && sub == 0) {
            const uint32_t i = __ldg(a.sorted_idx + p);
            const uint32_t bid = __ldg(a.body + i);
            if (bid != 0u) {
                const float4* T = a.body_xf + 4 * (bid - 1);
                const float4 r0 = T[0], r1 = T[1], r2 = T[2], o = __ldg(a.xo + i);
                acc.Dx += fmaf(r0.x, o.x, fmaf(r0.y, o.y, fmaf(r0.z, o.z, r0.w))) - xtp.x;
                acc.Dy += fmaf(r1.x, o.x, fmaf(r1.y, o.y, fmaf(r1.z, o.z, r1.w))) - xtp.y;
                acc.Dz += fmaf(r2.x, o.x, fmaf(r2.y, o.y, fmaf(r2.z, o.z, r2.w))) - xtp.z;
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
    const bool writer = valid && sub == 0;
    const bool reduce = fin.idx && fin.rate;   // the whole warp meets in the rate reduction below
    if (!writer && !reduce) return;
    float4 nt = xtp;
    float4 nx = xp;
    if (writer && acc.n > 0) {
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
    if (fin.idx) {
        unsigned q = 0u;
        if (writer) {
            const float dt = step_dt(a);
            const uint32_t i = fin.idx[p];
            const float4 nv = make_float4((nt.x - nx.x) / dt, (nt.y - nx.y) / dt, (nt.z - nx.z) / dt, 0.0f);
            fin.vel[i] = nv;
            // with materials x.w holds the material id: the inverse mass comes
            // from the step-start position, which only this thread touches
            const float w = kMat ? fin.pos[i].w : nx.w;
            fin.pos[i] = make_float4(nt.x, nt.y, nt.z, w);
            if (reduce) q = cfl_rate_bits(nv.x, nv.y, nv.z, sc.r_low);
        }
        if (reduce) {
            q = __reduce_max_sync(0xffffffffu, q);
            if ((threadIdx.x & 31) == 0 && q != 0u) atomicMax(fin.rate, q);
        }
        return;
    }
    st_pos<kL2>(xt_out + p, nt);
    if (stab) st_pos<kL2>(x_out + p, nx);
}

template <bool kMat, bool kBody>
__global__ void __launch_bounds__(128, 6) k_pass(const PbdArgs a, int stab, const float4* __restrict__ x_in,
                                              const float4* __restrict__ xt_in, float4* __restrict__ x_out,
                                              float4* __restrict__ xt_out, const uint32_t* __restrict__ nbr,
                                              const uint32_t* __restrict__ cnt, const FinalOut fin)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = t / kLanes;
    pass_particle<false, kMat, kBody>(a, stab, p, p < a.n, (int)(t % kLanes), x_in, xt_in, x_out, xt_out, nbr, cnt,
                                      fin);
}

// ---- all passes of one step in one launch --------------------------------
// Every block is resident at once (cooperative launch); the passes are
// separated by a grid barrier.  Its wait is bounded: a block that waits
// longer than kBarrierTimeoutNs (GPU global timer) or kBarrierSpins polls
// sets GS_DEVERR_BARRIER_TIMEOUT and leaves, and every other block then
// gives up at the same barrier as soon as it sees the flag, so the launch
// always ends.  The passes, lanes and summation order are those of k_pass,
// so the two paths give the same bits.  extra_arrivals > 0 is a self-test:
// the barrier then waits for blocks that do not exist and must time out.
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;   // one second
constexpr unsigned kBarrierSpins = 1u << 26;                       // backstop to the timer

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct SolveArgs {
    PbdArgs a;
    int n_stab, iters;
    float4 *x0, *x1, *xt0, *xt1;   // separate fields: an indexed parameter array would go to local memory
    const uint32_t* nbr;
    const uint32_t* cnt;
    unsigned* bar;   // {arrived, generation}, zero at launch
    int* err;
    unsigned extra_arrivals;   // 0; > 0 only in the timeout self-test
};

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned gen, int* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicExch(bar + 1, gen);
        } else {
            unsigned spins = 0;
            const unsigned long long t0 = global_ns();
            while (atomicAdd(bar + 1, 0u) != gen) {
                if (++spins > kBarrierSpins || global_ns() - t0 > kBarrierTimeoutNs ||
                    (atomicAdd(err, 0) & GS_DEVERR_BARRIER_TIMEOUT)) {
                    atomicOr(err, GS_DEVERR_BARRIER_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <bool kMat>
__global__ void __launch_bounds__(128, 6) k_solve(const SolveArgs s)
{
    const int sub = (int)(threadIdx.x % kLanes);
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kLanes);
    const int64_t group = (int64_t)blockIdx.x * (blockDim.x / kLanes) + threadIdx.x / kLanes;
    // the warp's first group decides the trip count, so whole warps iterate
    const int64_t warp_first = group & ~(int64_t)(32 / kLanes - 1);
    int bx = 0, bt = 0;
    const int total = s.n_stab + s.iters;
    for (int it = 0; it < total; ++it) {
        const int stab = it < s.n_stab;
        for (int64_t base = warp_first; base < s.a.n; base += groups) {
            const int64_t p = base + (group - warp_first);
            float4* xi = bx ? s.x1 : s.x0;
            float4* xo = bx ? s.x0 : s.x1;
            float4* ti = bt ? s.xt1 : s.xt0;
            float4* to = bt ? s.xt0 : s.xt1;
            pass_particle<true, kMat>(s.a, stab, p, p < s.a.n, sub, xi, ti, xo, to, s.nbr, s.cnt);
        }
        bt ^= 1;
        if (stab) bx ^= 1;
        if (it + 1 < total && !grid_barrier(s.bar, gridDim.x + s.extra_arrivals, (unsigned)it + 1u, s.err)) return;
    }
}

__global__ void k_finalize(const PbdArgs a, const uint32_t* __restrict__ idx, const float4* __restrict__ s_x,
                           const float4* __restrict__ s_xt, float4* __restrict__ pos, float4* __restrict__ vel,
                           unsigned* rate)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned q = 0u;
    if (p < a.n) {
        const float dt = step_dt(a);
        const uint32_t i = idx[p];
        const float4 x = s_x[p], xt = s_xt[p];
        const float4 nv = make_float4((xt.x - x.x) / dt, (xt.y - x.y) / dt, (xt.z - x.z) / dt, 0.0f);
        vel[i] = nv;
        const float w = a.mu_cross ? pos[i].w : x.w;   // x.w is the material id with materials
        pos[i] = make_float4(xt.x, xt.y, xt.z, w);
        if (rate) q = cfl_rate_bits(nv.x, nv.y, nv.z, a.scenes[a.lr_scene[i]].r_low);
    }
    if (rate) {   // whole warps: the launch covers multiples of 32 threads
        q = __reduce_max_sync(0xffffffffu, q);
        if ((threadIdx.x & 31) == 0 && q != 0u) atomicMax(rate, q);
    }
}

// ---- shape matching of rigid bodies (Sec. 3) -------------------------------
// Rotation of the polar decomposition of C by the iteration of Mueller et
// al., "A Robust Method to Extract the Rotational Part of Deformations"
// (2016): with r_k and c_k the columns of R(q) and C,
//   omega = sum_k r_k x c_k / (|sum_k r_k . c_k| + eps),  q <- exp(omega) q,
// started from the body's previous rotation.  q = (x, y, z, w).
__device__ void quat_to_rows(const float4 q, float R[9])
{
    const float x = q.x, y = q.y, z = q.z, w = q.w;
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - z * w);
    R[2] = 2.f * (x * z + y * w);
    R[3] = 2.f * (x * y + z * w);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - x * w);
    R[6] = 2.f * (x * z - y * w);
    R[7] = 2.f * (y * z + x * w);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ float4 extract_rotation(const float C[9], float4 q)
{
    float n2 = 0.f;
    for (int k = 0; k < 9; ++k) n2 += C[k] * C[k];
    const float eps = 1e-9f * sqrtf(n2) + 1e-30f;
    for (int it = 0; it < 24; ++it) {
        float R[9];
        quat_to_rows(q, R);
        float ox = 0.f, oy = 0.f, oz = 0.f, d = 0.f;
        for (int k = 0; k < 3; ++k) {   // column k of R and of C
            const float rx = R[k], ry = R[3 + k], rz = R[6 + k];
            const float cx = C[k], cy = C[3 + k], cz = C[6 + k];
            ox += ry * cz - rz * cy;
            oy += rz * cx - rx * cz;
            oz += rx * cy - ry * cx;
            d += rx * cx + ry * cy + rz * cz;
        }
        const float inv = 1.0f / (fabsf(d) + eps);
        ox *= inv;
        oy *= inv;
        oz *= inv;
        const float ang = sqrtf(ox * ox + oy * oy + oz * oz);
        if (!(ang > 1e-7f)) break;
        const float s = sinf(0.5f * ang) / ang, cw = cosf(0.5f * ang);
        const float4 e = make_float4(ox * s, oy * s, oz * s, cw);   // exp(omega)
        float4 nq = make_float4(e.w * q.x + e.x * q.w + e.y * q.z - e.z * q.y,
                                e.w * q.y - e.x * q.z + e.y * q.w + e.z * q.x,
                                e.w * q.z + e.x * q.y - e.y * q.x + e.z * q.w,
                                e.w * q.w - e.x * q.x - e.y * q.y - e.z * q.z);
        const float nn = rsqrtf(nq.x * nq.x + nq.y * nq.y + nq.z * nq.z + nq.w * nq.w);
        q = make_float4(nq.x * nn, nq.y * nn, nq.z * nn, nq.w * nn);
    }
    return q;
}

// One block per body.  Sums relative to the body's first particle keep the
// float32 products small: with p' = x~ - p0, c = p0 + sum m p' / M and
// C = sum m p' xo^T - (c - p0) (sum m xo)^T.
__global__ void __launch_bounds__(256) k_body_xform(const uint32_t* __restrict__ start,
                                                    const uint32_t* __restrict__ members,
                                                    const uint32_t* __restrict__ slot_of,
                                                    const float4* __restrict__ xt, const float4* __restrict__ xo,
                                                    float4* __restrict__ xf)
{
    const int b = blockIdx.x;
    const uint32_t k0 = start[b], k1 = start[b + 1];
    if (k0 == k1) return;
    const float4 p0 = xt[slot_of[members[k0]]];
    float acc[16];   // M, sum m p' (3), sum m xo (3), sum m p' xo^T (9)
    for (int k = 0; k < 16; ++k) acc[k] = 0.f;
    for (uint32_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const uint32_t i = members[k];
        const float4 x = xt[slot_of[i]], o = xo[i];
        const float m = o.w, px = x.x - p0.x, py = x.y - p0.y, pz = x.z - p0.z;
        acc[0] += m;
        acc[1] += m * px;
        acc[2] += m * py;
        acc[3] += m * pz;
        acc[4] += m * o.x;
        acc[5] += m * o.y;
        acc[6] += m * o.z;
        const float mp[3] = {m * px, m * py, m * pz}, oo[3] = {o.x, o.y, o.z};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) acc[7 + 3 * r + s] += mp[r] * oo[s];
    }
    __shared__ float red[8][16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 0; k < 16; ++k) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][k];
        acc[k] = v;
    }
    const float M = acc[0];
    const float dx = acc[1] / M, dy = acc[2] / M, dz = acc[3] / M;   // c - p0
    const float d[3] = {dx, dy, dz};
    float C[9];
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) C[3 * r + s] = acc[7 + 3 * r + s] - d[r] * acc[4 + s];
    float4 q = xf[4 * b + 3];
    if (!(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w > 0.5f)) q = make_float4(0.f, 0.f, 0.f, 1.f);
    q = extract_rotation(C, q);
    float R[9];
    quat_to_rows(q, R);
    const float c[3] = {p0.x + dx, p0.y + dy, p0.z + dz};
    for (int r = 0; r < 3; ++r) xf[4 * b + r] = make_float4(R[3 * r], R[3 * r + 1], R[3 * r + 2], c[r]);
    xf[4 * b + 3] = q;
}

// ---- CFL-limited LR substeps of a frame (gs_frame_adaptive) ----------------
__global__ void k_cfl_begin(CflState* st, float t)
{
    st->t_rem = t;
    st->dt = 0.0f;
    st->rate = 0u;
    st->taken = 0;
    st->more = 1;
}

__global__ void k_cfl_rate(const PbdArgs a, const float4* __restrict__ vel, unsigned* rate)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned q = 0u;
    if (i < a.n) {
        const float4 v = vel[i];
        q = cfl_rate_bits(v.x, v.y, v.z, a.scenes[a.lr_scene[i]].r_low);
    }
    q = __reduce_max_sync(0xffffffffu, q);
    if ((threadIdx.x & 31) == 0 && q != 0u) atomicMax(rate, q);
}

// One thread.  limit = min(dt_max, cfl / rate) (dt_max for rate 0, 0 for a
// rate that is not finite); n = ceil(t_rem / limit) within the steps still
// allowed; this step = t_rem / n; the frame ends with the step of n = 1.
// n <= max_sub - taken, and taken grows by one per call, so a frame takes
// at most max_sub steps whatever the velocities.
__global__ void k_cfl_pick(CflState* st, float dt_max, float cfl, int max_sub, cudaGraphConditionalHandle h,
                           int in_graph, unsigned body_kernels)
{
    const float rate = __uint_as_float(st->rate);
    st->rate = 0u;   // the step's finalize accumulates the next rate
    float lim = dt_max;
    if (!(rate <= 3.40282347e38f)) lim = 0.0f;
    else if (rate > 0.0f) lim = fminf(dt_max, __fdiv_rn(cfl, rate));
    const int left = max_sub - st->taken;
    int n = left;
    if (left > 1) {
        const float q = lim > 0.0f ? __fdiv_rn(st->t_rem, lim) : __int_as_float(0x7f800000);
        if (q < (float)left) n = max(1, (int)ceilf(q));
    } else {
        n = 1;
    }
    const float dt = __fdiv_rn(st->t_rem, (float)n);
    st->dt = dt;
    if (st->taken >= 0 && st->taken < GS_MAX_SUBSTEPS) st->log[st->taken] = dt;
    st->taken += 1;
    st->t_rem = n > 1 ? __fsub_rn(st->t_rem, dt) : 0.0f;
    st->more = n > 1 ? 1 : 0;
    if (in_graph) {
        st->kernels += body_kernels;
        cudaGraphSetConditional(h, n > 1 ? 1u : 0u);
    }
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

cudaError_t gs_launch_predict_keys(cudaStream_t s, const PbdArgs& a, const float4* pos, const float4* vel,
                                   float4* xt, uint32_t* keys, uint32_t* rank, uint32_t* cnt, int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_predict_keys<<<gs_blocks(a.n, 256), 256, 0, s>>>(a, pos, vel, xt, keys, rank, cnt);
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
                                const uint32_t* cell_start, int64_t n_cell, uint32_t* nbr, uint32_t* cnt, int cap,
                                int* err, int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    if (n_cell <= 2 * a.n) {
        k_neighbors_cells<<<gs_blocks(n_cell * 32, 128), 128, 0, s>>>(a, s_xt, cell_start, n_cell, nbr, cnt, cap,
                                                                      err);
    } else {
        const int64_t warps = (a.n + kNbrGroup - 1) / kNbrGroup;
        k_neighbors<<<gs_blocks(warps * 32, 128), 128, 0, s>>>(a, s_xt, skeys, cell_start, nbr, cnt, cap, err);
    }
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_pass(cudaStream_t s, const PbdArgs& a, int stab, const float4* x_in, const float4* xt_in,
                           float4* x_out, float4* xt_out, const uint32_t* nbr, const uint32_t* cnt,
                           int64_t* launches, const uint32_t* fin_idx, float4* fin_pos, float4* fin_vel,
                           unsigned* fin_rate)
{
    if (a.n <= 0) return cudaSuccess;
    const FinalOut fin{fin_idx, fin_pos, fin_vel, fin_idx ? fin_rate : nullptr};
    const unsigned nb = gs_blocks(a.n * kLanes, 128);
    if (a.body) {
        if (a.mu_cross)
            k_pass<true, true><<<nb, 128, 0, s>>>(a, stab, x_in, xt_in, x_out, xt_out, nbr, cnt, fin);
        else
            k_pass<false, true><<<nb, 128, 0, s>>>(a, stab, x_in, xt_in, x_out, xt_out, nbr, cnt, fin);
    } else if (a.mu_cross) {
        k_pass<true, false><<<nb, 128, 0, s>>>(a, stab, x_in, xt_in, x_out, xt_out, nbr, cnt, fin);
    } else {
        k_pass<false, false><<<nb, 128, 0, s>>>(a, stab, x_in, xt_in, x_out, xt_out, nbr, cnt, fin);
    }
    *launches += 1;
    return cudaGetLastError();
}

int gs_solve_blocks(int sm_count)
{
    // both variants must fit: the grid is sized once per context
    int per_sm = 0, per_sm_mat = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<false>, 128, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_mat, k_solve<true>, 128, 0) != cudaSuccess)
        return 0;
    per_sm = std::min(per_sm, per_sm_mat);
    if (per_sm <= 0) return 0;
    return per_sm * sm_count;
}

cudaError_t gs_launch_solve(cudaStream_t s, const PbdArgs& a, int n_stab, int iters, float4* x[2], float4* xt[2],
                            const uint32_t* nbr, const uint32_t* cnt, unsigned* bar, int* err, int max_blocks,
                            int64_t* launches, unsigned extra_arrivals)
{
    if (a.n <= 0 || n_stab + iters <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    SolveArgs sa;
    sa.a = a;
    sa.n_stab = n_stab;
    sa.iters = iters;
    sa.x0 = x[0];
    sa.x1 = x[1];
    sa.xt0 = xt[0];
    sa.xt1 = xt[1];
    sa.nbr = nbr;
    sa.cnt = cnt;
    sa.bar = bar;
    sa.err = err;
    sa.extra_arrivals = extra_arrivals;
    int64_t need = (a.n * kLanes + 127) / 128;
    const int grid = (int)std::min<int64_t>(need, max_blocks);
    void* args[] = {&sa};
    const void* fn = a.mu_cross ? (const void*)k_solve<true> : (const void*)k_solve<false>;
    e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(128), args, 0, s);
    *launches += 1;
    return e;
}

cudaError_t gs_launch_finalize(cudaStream_t s, const PbdArgs& a, const uint32_t* idx, const float4* s_x,
                               const float4* s_xt, float4* pos, float4* vel, int64_t* launches, unsigned* rate)
{
    if (a.n <= 0) return cudaSuccess;
    k_finalize<<<gs_blocks(a.n, 256), 256, 0, s>>>(a, idx, s_x, s_xt, pos, vel, rate);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_cfl_begin(cudaStream_t s, CflState* st, float t, int64_t* launches)
{
    k_cfl_begin<<<1, 1, 0, s>>>(st, t);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_cfl_rate(cudaStream_t s, const PbdArgs& a, const float4* vel, unsigned* rate, int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_cfl_rate<<<gs_blocks(a.n, 256), 256, 0, s>>>(a, vel, rate);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_cfl_pick(cudaStream_t s, CflState* st, float dt_max, float cfl, int max_sub,
                               cudaGraphConditionalHandle h, int in_graph, unsigned body_kernels, int64_t* launches)
{
    k_cfl_pick<<<1, 1, 0, s>>>(st, dt_max, cfl, max_sub, h, in_graph, body_kernels);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_body_xform(cudaStream_t s, int n_bodies, const uint32_t* start, const uint32_t* members,
                                 const uint32_t* slot_of, const float4* xt, const float4* xo, float4* xf,
                                 int64_t* launches)
{
    if (n_bodies <= 0) return cudaSuccess;
    k_body_xform<<<(unsigned)n_bodies, 256, 0, s>>>(start, members, slot_of, xt, xo, xf);
    *launches += 1;
    return cudaGetLastError();
}
