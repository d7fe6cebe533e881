// adjoint.cu -- reverse mode of the HR frame (Sec. 4) for the
// differentiable pattern: gradients of a loss on the HR particles after one
// frame with respect to the LR positions and velocities and the HR state
// before the frame.
//
// One thread per HR particle recomputes the forward pass of its particle
// (weights, blend case, the LR particle of largest weight, SDF contacts) and
// then applies the chain rule backwards for those branch decisions:
//   SDF steps (last first), normal held fixed:  g <- g - n (n . g)
//   x' = x + dt v'        :  g_v' = g_v'' + dt g_x'',  g_x += g_x''
//   v' = (1-a) vt + a (v + dt g):  g_vt = (1-a) g_v',  g_v = a g_v',
//                                  g_a = g_v' . (v + dt g - vt)
//   a = 1 - wmax (blend case)   :  g_wmax = -g_a
//   vt = V / S                  :  g_V = g_vt / S,  g_S = -(g_vt . vt) / S
//   w_j = (1 - |x - X_j|^2 / 9r^2)^3:
//        g_w_j = g_S + g_V . V_j + [j = argmax] g_wmax
//        g_X_j += g_w_j 6 t^2 (x - X_j) / 9r^2,  g_x -= the same,
//        g_V_j += w_j g_V
// LR gradients are summed in cell order with atomics and then scattered back
// to the original LR order.
#include <cuda_runtime.h>

#include "gs_internal.cuh"
#include "pbd_common.cuh"
#include "sdf.cuh"

namespace {

__device__ __forceinline__ int cell_of(float x, float o, float inv_h, int dim)
{
    float a = __fmul_rn(__fsub_rn(x, o), inv_h);
    float f = floorf(a);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(dim - 1)) return dim - 1;
    return (int)f;
}

constexpr int kMaxSteps = 32;
constexpr int kBwdLanes = 4;

// rec (optional): the decisions this reverse mode differentiates, four words
// per HR particle: the LR particle of largest weight (original index through
// lr_idx, or all ones), the blend case (1: alpha = 1 - max w), bit c = SDF
// component c in contact, bit c = normal velocity removed at component c.
__global__ void k_upsample_bwd(const SceneDev* __restrict__ scenes, const gs_sdf* __restrict__ sdf,
                               const float4* __restrict__ lr_spos, const float4* __restrict__ lr_svel,
                               const uint32_t* __restrict__ cell_start, const float4* __restrict__ hx,
                               const float4* __restrict__ hv, const float4* __restrict__ gxo,
                               const float4* __restrict__ gvo, float4* __restrict__ ghx, float4* __restrict__ ghv,
                               float4* __restrict__ gXs, float4* __restrict__ gVs, int64_t m, float dt,
                               uint32_t* __restrict__ rec, const uint32_t* __restrict__ lr_idx,
                               float4* __restrict__ coef, const uint32_t* __restrict__ order,
                               float4* __restrict__ pos_sorted)
{
    // kBwdLanes lanes per HR particle: lane `sub` takes the LR candidates
    // sub, sub + kBwdLanes, ... of every row of cells; the lanes' partial
    // sums meet in shuffles, and each lane pushes its own candidates'
    // gradients.  Every lane stays until the last shuffle.  With coef: the
    // particles are taken in the order `order` (slot -> particle), and the
    // coefficients and the position go to the slot (coef[2 slot ..],
    // pos_sorted[slot]) instead of any atomic.
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t slot = t / kBwdLanes;
    const int sub = (int)(t % kBwdLanes);
    const bool live = slot < m;
    const int64_t i = (order && live) ? (int64_t)order[slot] : slot;
    const SceneDev& sc = scenes[0];
    const GridDev& g = sc.g;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 p = live ? hx[i] : zero4, v = live ? hv[i] : zero4;
    const float R = 3.0f * sc.r_low;
    const float R2 = R * R;
    const float inv9r2 = 1.0f / R2;
    const int cx0 = cell_of(p.x - R, g.ox, g.inv_h, g.dx), cx1 = cell_of(p.x + R, g.ox, g.inv_h, g.dx);
    const int cy0 = cell_of(p.y - R, g.oy, g.inv_h, g.dy), cy1 = cell_of(p.y + R, g.oy, g.inv_h, g.dy);
    const int cz0 = cell_of(p.z - R, g.oz, g.inv_h, g.dz), cz1 = cell_of(p.z + R, g.oz, g.inv_h, g.dz);
    // forward
    float S = 0.f, Vx = 0.f, Vy = 0.f, Vz = 0.f, wmax = 0.f;
    uint32_t jstar = 0xffffffffu;
    for (int cz = cz0; live && cz <= cz1; ++cz)
        for (int cy = cy0; cy <= cy1; ++cy) {
            const int64_t row = (int64_t)sc.cell_off + ((int64_t)cz * g.dy + cy) * g.dx;
            const uint32_t b = cell_start[row + cx0], e = cell_start[row + cx1 + 1];
            for (uint32_t j = b + sub; j < e; j += kBwdLanes) {
                const float4 q = lr_spos[j];
                const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
                const float d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < R2)) continue;
                const float t = 1.0f - d2 * inv9r2;
                const float w = t * t * t;
                const float4 qv = lr_svel[j];
                S += w;
                Vx += w * qv.x;
                Vy += w * qv.y;
                Vz += w * qv.z;
                if (w > wmax) {
                    wmax = w;
                    jstar = j;
                }
            }
        }
    // the lanes' sums; the largest weight with the lowest slot among equals
    // (the first one met in slot order)
#pragma unroll
    for (int o = 1; o < kBwdLanes; o <<= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, o);
        Vx += __shfl_xor_sync(0xffffffffu, Vx, o);
        Vy += __shfl_xor_sync(0xffffffffu, Vy, o);
        Vz += __shfl_xor_sync(0xffffffffu, Vz, o);
        const float w2 = __shfl_xor_sync(0xffffffffu, wmax, o);
        const uint32_t j2 = __shfl_xor_sync(0xffffffffu, jstar, o);
        if (w2 > wmax || (w2 == wmax && j2 < jstar)) {
            wmax = w2;
            jstar = j2;
        }
    }
    float vtx = 0.f, vty = 0.f, vtz = 0.f;
    if (S > 0.0f) {
        vtx = Vx / S;
        vty = Vy / S;
        vtz = Vz / S;
    }
    const bool branch = (wmax <= sc.c1) || (S > 0.0f && wmax >= sc.c2 * S);
    const float alpha = branch ? 1.0f - wmax : 0.0f;
    const float bx = v.x + dt * sc.gx, by = v.y + dt * sc.gy, bz = v.z + dt * sc.gz;
    float vpx = (1.0f - alpha) * vtx + alpha * bx, vpy = (1.0f - alpha) * vty + alpha * by,
          vpz = (1.0f - alpha) * vtz + alpha * bz;
    float xpx = p.x + dt * vpx, xpy = p.y + dt * vpy, xpz = p.z + dt * vpz;
    float nx_[kMaxSteps], ny_[kMaxSteps], nz_[kMaxSteps];
    bool vrem[kMaxSteps];
    int n_steps = 0, dec = 0;
    uint32_t act_bits = 0u, rem_bits = 0u;
    for (int s = 0; s < sc.n_sdf; ++s) {
        const gs_sdf& bsdf = sdf[sc.sdf_begin + s];
        const int nc = sdf_components(bsdf.kind);
        for (int c = 0; c < nc; ++c, ++dec) {
            const SdfHit h = sdf_eval(bsdf, c, xpx, xpy, xpz);
            if (!(h.phi < sc.r_high)) continue;
            if (dec < 32) act_bits |= 1u << dec;
            const float push = sc.r_high - h.phi;
            xpx += push * h.nx;
            xpy += push * h.ny;
            xpz += push * h.nz;
            const float vn = (vpx - bsdf.vel[0]) * h.nx + (vpy - bsdf.vel[1]) * h.ny + (vpz - bsdf.vel[2]) * h.nz;
            if (vn < 0.0f) {
                vpx -= vn * h.nx;
                vpy -= vn * h.ny;
                vpz -= vn * h.nz;
                if (dec < 32) rem_bits |= 1u << dec;
            }
            if (n_steps < kMaxSteps) {
                nx_[n_steps] = h.nx;
                ny_[n_steps] = h.ny;
                nz_[n_steps] = h.nz;
                vrem[n_steps] = vn < 0.0f;
                ++n_steps;
            }
        }
    }
    if (rec && live && sub == 0) {
        rec[4 * i + 0] = jstar != 0xffffffffu ? lr_idx[jstar] : 0xffffffffu;
        rec[4 * i + 1] = branch ? 1u : 0u;
        rec[4 * i + 2] = act_bits;
        rec[4 * i + 3] = rem_bits;
    }
    // reverse
    const float4 go = live ? gxo[i] : zero4, gw = live ? gvo[i] : zero4;
    float ax = go.x, ay = go.y, az = go.z, avx = gw.x, avy = gw.y, avz = gw.z;
    for (int k = n_steps - 1; k >= 0; --k) {
        if (vrem[k]) {
            const float d = avx * nx_[k] + avy * ny_[k] + avz * nz_[k];
            avx -= d * nx_[k];
            avy -= d * ny_[k];
            avz -= d * nz_[k];
        }
        const float d = ax * nx_[k] + ay * ny_[k] + az * nz_[k];
        ax -= d * nx_[k];
        ay -= d * ny_[k];
        az -= d * nz_[k];
    }
    // dL/dx (HR input): the direct term on lane 0, each lane's candidates' terms
    float gpx = sub == 0 ? ax : 0.f, gpy = sub == 0 ? ay : 0.f, gpz = sub == 0 ? az : 0.f;
    const float gvpx = avx + dt * ax, gvpy = avy + dt * ay, gvpz = avz + dt * az;
    const float gvtx = (1.0f - alpha) * gvpx, gvty = (1.0f - alpha) * gvpy, gvtz = (1.0f - alpha) * gvpz;
    const float galpha = gvpx * (bx - vtx) + gvpy * (by - vty) + gvpz * (bz - vtz);
    const float gwmax = branch ? -galpha : 0.0f;
    if (live && sub == 0) ghv[i] = make_float4(alpha * gvpx, alpha * gvpy, alpha * gvpz, 0.0f);
    if (live && S > 0.0f) {
        const float gVx = gvtx / S, gVy = gvty / S, gVz = gvtz / S;
        const float gS = -(gvtx * vtx + gvty * vty + gvtz * vtz) / S;
        for (int cz = cz0; cz <= cz1; ++cz)
            for (int cy = cy0; cy <= cy1; ++cy) {
                const int64_t row = (int64_t)sc.cell_off + ((int64_t)cz * g.dy + cy) * g.dx;
                const uint32_t b = cell_start[row + cx0], e = cell_start[row + cx1 + 1];
                for (uint32_t j = b + sub; j < e; j += kBwdLanes) {
                    const float4 q = lr_spos[j];
                    const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    if (!(d2 < R2)) continue;
                    const float t = 1.0f - d2 * inv9r2;
                    const float w = t * t * t;
                    const float4 qv = lr_svel[j];
                    const float gwj = gS + gVx * qv.x + gVy * qv.y + gVz * qv.z + (j == jstar ? gwmax : 0.0f);
                    const float k6 = gwj * 6.0f * t * t * inv9r2;
                    if (!coef) {   // one vector reduction per gradient (global float4 atomics, sm_90 and later)
                        atomicAdd(gXs + j, make_float4(k6 * dx, k6 * dy, k6 * dz, 0.0f));
                        atomicAdd(gVs + j, make_float4(w * gVx, w * gVy, w * gVz, 0.0f));
                    }
                    gpx -= k6 * dx;
                    gpy -= k6 * dy;
                    gpz -= k6 * dz;
                }
            }
    }
#pragma unroll
    for (int o = 1; o < kBwdLanes; o <<= 1) {
        gpx += __shfl_xor_sync(0xffffffffu, gpx, o);
        gpy += __shfl_xor_sync(0xffffffffu, gpy, o);
        gpz += __shfl_xor_sync(0xffffffffu, gpz, o);
    }
    if (live && sub == 0) ghx[i] = make_float4(gpx, gpy, gpz, 0.0f);
    if (coef && live && sub == 0) {
        // the particle's coefficients for the LR side's gather (k_upsample_bwd_lr)
        float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = make_float4(0.f, __uint_as_float(0xffffffffu), 0.f, 0.f);
        if (S > 0.0f) {
            c0 = make_float4(-(gvtx * vtx + gvty * vty + gvtz * vtz) / S, gvtx / S, gvty / S, gvtz / S);
            c1 = make_float4(gwmax, __uint_as_float(jstar), 0.f, 0.f);
        }
        coef[2 * slot] = c0;
        coef[2 * slot + 1] = c1;
        pos_sorted[slot] = p;
    }
}

// The LR side of the HR frame's reverse mode without atomics: one warp per
// cell-ordered LR slot j gathers over the HR particles of the 27 cells around
// its own (HR binned by the same cells: hr_cell_start, positions and
// coefficients in that order: hx_sorted, coef) the terms
// k_upsample_bwd would add to slot j, from every HR particle's coefficients
// (gS, gV, max-w gradient, largest-weight slot), lanes over the HR
// candidates and a fixed shuffle tree for the sums: the same result on every
// run.
__global__ void __launch_bounds__(128) k_upsample_bwd_lr(const SceneDev* __restrict__ scenes,
                                                         const float4* __restrict__ lr_spos,
                                                         const float4* __restrict__ lr_svel,
                                                         const uint32_t* __restrict__ lr_skeys,
                                                         const float4* __restrict__ hx_sorted,
                                                         const uint32_t* __restrict__ hr_cell_start,
                                                         const float4* __restrict__ coef, float4* __restrict__ gXs,
                                                         float4* __restrict__ gVs, int64_t n_low)
{
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= n_low) return;   // whole warps
    const SceneDev& sc = scenes[0];
    const GridDev& g = sc.g;
    const uint32_t c = lr_skeys[j] - sc.cell_off;
    const int cx = (int)(c % (uint32_t)g.dx);
    const int cy = (int)((c / (uint32_t)g.dx) % (uint32_t)g.dy);
    const int cz = (int)(c / ((uint32_t)g.dx * (uint32_t)g.dy));
    const int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < g.dx ? cx + 1 : g.dx - 1;
    const float R = 3.0f * sc.r_low;
    const float R2 = R * R;
    const float inv9r2 = 1.0f / R2;
    const float4 q = lr_spos[j], qv = lr_svel[j];
    // lane r < 9: row r = (z, y) of the 3 x 3 rows around the cell
    uint32_t rb = 0, len = 0;
    if (lane < 9) {
        const int z = cz - 1 + lane / 3, y = cy - 1 + lane % 3;
        if (z >= 0 && z < g.dz && y >= 0 && y < g.dy) {
            const int64_t row = (int64_t)sc.cell_off + ((int64_t)z * g.dy + y) * g.dx;
            rb = hr_cell_start[row + x0];
            len = hr_cell_start[row + x1 + 1] - rb;
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
    float ax = 0.f, ay = 0.f, az = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t f = base + (uint32_t)lane;
        int r = 0;   // the row of flat index f
#pragma unroll
        for (int step = 8; step > 0; step >>= 1) {
            const uint32_t e = __shfl_sync(0xffffffffu, excl, (r + step) & 31);
            if (r + step < 9 && e <= f) r += step;
        }
        const uint32_t slot = __shfl_sync(0xffffffffu, rb, r) + (f - __shfl_sync(0xffffffffu, excl, r));
        if (f >= total) continue;
        const float4 p = hx_sorted[slot];
        const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
        const float d2 = dx * dx + dy * dy + dz * dz;
        if (!(d2 < R2)) continue;
        const float4 c0 = coef[2 * (int64_t)slot], c1 = coef[2 * (int64_t)slot + 1];
        const float t = 1.0f - d2 * inv9r2;
        const float w = t * t * t;
        const float gwj = c0.x + c0.y * qv.x + c0.z * qv.y + c0.w * qv.z +
                          (__float_as_uint(c1.y) == (uint32_t)j ? c1.x : 0.0f);
        const float k6 = gwj * 6.0f * t * t * inv9r2;
        ax += k6 * dx;
        ay += k6 * dy;
        az += k6 * dz;
        bx += w * c0.y;
        by += w * c0.z;
        bz += w * c0.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
        bz += __shfl_xor_sync(0xffffffffu, bz, o);
    }
    if (lane == 0) {
        gXs[j] = make_float4(ax, ay, az, 0.0f);
        gVs[j] = make_float4(bx, by, bz, 0.0f);
    }
}

// out[idx[p]] = in[p] for both arrays
__global__ void k_scatter2(const uint32_t* __restrict__ idx, const float4* __restrict__ a, const float4* __restrict__ b,
                           float4* __restrict__ ao, float4* __restrict__ bo, int64_t n)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t i = idx[p];
    ao[i] = a[p];
    bo[i] = b[p];
}


// ---------------------------------------------------------------------------
// Reverse mode of one LR step (Algorithm 1) for the forward pass's branch
// decisions.  Pair (p, q) evaluated on y (x in stabilization, xt in the
// solver), e = y_q - y_p, L = |e|, u = e / L, pen = 2r - L, W = w_p + w_q:
//   contact   c_p = -m_p pen u,  c_q = +m_q pen u,
//             d(pen u)/de = (2r/L - 1) I - (2r/L) u u^T =: K
//   friction  rel = (xt_p - x_p) - (xt_q - x_q),  c_p -= m_p F,  c_q += m_q F,
//             F = s P rel (P = I - e e^T / e.e; s = 1 or thr_k / |P rel|)
// A pass moves p by (sum c)/n_p; the reverse pass pushes h = g / n back
// through every contribution that involves p (its own and its partners').
struct M3 {
    float a[9];
};

__device__ __forceinline__ void m3_eye(M3& A, float s)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) A.a[k] = 0.0f;
    A.a[0] = A.a[4] = A.a[8] = s;
}

__device__ __forceinline__ void m3_outer_add(M3& A, float s, const float* u, const float* v)
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) A.a[3 * r + c] += s * u[r] * v[c];
}

// out += s A^T h
__device__ __forceinline__ void m3_tmul_add(float* out, float s, const M3& A, const float* h)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] += s * (A.a[c] * h[0] + A.a[3 + c] * h[1] + A.a[6 + c] * h[2]);
}

__device__ __forceinline__ M3 m3_mul(const M3& A, const M3& B)
{
    M3 R;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            R.a[3 * r + c] = A.a[3 * r] * B.a[c] + A.a[3 * r + 1] * B.a[3 + c] + A.a[3 * r + 2] * B.a[6 + c];
    return R;
}

// F and its Jacobians with respect to rel and e (e_is_normal: SDF, e = n).
__device__ void fric_jac(const float* rel, const float* e, float ee, bool e_is_normal, float thr_s, float thr_k,
                         bool mode1, float mu_k, const float* u, float* F, M3& Fr, M3& Fe, bool* kinetic = nullptr)
{
    const Tangent tg = tangent_part(rel[0], rel[1], rel[2], e[0], e[1], e[2], ee);
    const float perp[3] = {tg.tx, tg.ty, tg.tz};
    M3 P, G;
    m3_eye(P, 1.0f);
    m3_outer_add(P, -1.0f / ee, e, e);
#pragma unroll
    for (int k = 0; k < 9; ++k) G.a[k] = 0.0f;
    if (!e_is_normal) {
        const float re = rel[0] * e[0] + rel[1] * e[1] + rel[2] * e[2];
        m3_outer_add(G, -1.0f / ee, e, rel);
        G.a[0] -= re / ee;
        G.a[4] -= re / ee;
        G.a[8] -= re / ee;
        m3_outer_add(G, 2.0f * re / (ee * ee), e, e);
    }
    const float Lp = tg.L;
    const bool clipped = !(Lp < thr_s) && Lp > 0.0f && thr_k / Lp < 1.0f;
    if (kinetic) *kinetic = clipped;
    if (clipped) {
        const float pu[3] = {perp[0] / Lp, perp[1] / Lp, perp[2] / Lp};
        M3 Q;
        m3_eye(Q, thr_k / Lp);
        m3_outer_add(Q, -thr_k / Lp, pu, pu);
        F[0] = thr_k * pu[0];
        F[1] = thr_k * pu[1];
        F[2] = thr_k * pu[2];
        Fr = m3_mul(Q, P);
        Fe = m3_mul(Q, G);
        if (mode1) m3_outer_add(Fe, -mu_k, pu, u);
    } else {
        F[0] = perp[0];
        F[1] = perp[1];
        F[2] = perp[2];
        Fr = P;
        Fe = G;
    }
}

__global__ void k_adj_init(int64_t n, const uint32_t* __restrict__ idx, const float4* __restrict__ gxo,
                           const float4* __restrict__ gvo, float dt, float4* __restrict__ gx, float4* __restrict__ gxt,
                           float* __restrict__ gws)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t i = idx[p];
    const float4 a = gxo[i], b = gvo[i];
    gxt[p] = make_float4(a.x + b.x / dt, a.y + b.y / dt, a.z + b.z / dt, 0.0f);
    gx[p] = make_float4(-b.x / dt, -b.y / dt, -b.z / dt, 0.0f);
    gws[p] = 0.0f;
}

// The reverse pass gives each LR particle kAdjLanes lanes of a warp: lane l
// takes candidates l, l + kAdjLanes, ... and SDF components likewise, and
// the lanes' sums are added up by shuffles (a small LR set, such as the 4k
// particles of a differentiable rollout, then still fills the GPU).
constexpr int kAdjLanes = 16;

__device__ __forceinline__ float lanes_sum(float v)
{
#pragma unroll
    for (int o = kAdjLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int lanes_sum(int v)
{
#pragma unroll
    for (int o = kAdjLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The active constraints of particle p's pass on y (its pair contacts and
// SDF contacts), counted by the lanes of p (lane takes candidates lane,
// lane + kAdjLanes, ...; components likewise); the lanes' partial counts.
__device__ __forceinline__ int lane_active_count(const PbdArgs& a, const SceneDev& sc, const float4* __restrict__ Y,
                                                 const float4* __restrict__ WS, const uint32_t* __restrict__ nbr,
                                                 int64_t p, int nc, float4 yp, float wp, int lane)
{
    const float d0 = 2.0f * sc.r_low;
    int n_act = 0;
    for (int k = lane; k < nc; k += kAdjLanes) {
        const uint32_t q = nbr[(int64_t)k * a.n + p];
        const PairGeo g = pair_geo(yp, Y[q]);
        if (!(g.d < d0) || g.d2 == 0.0f) continue;
        if (!(wp + WS[q].w > 0.0f)) continue;
        ++n_act;
    }
    if (wp > 0.0f) {
        int gc = 0;   // component index over all the scene's SDFs
        for (int s = 0; s < sc.n_sdf; ++s) {
            const gs_sdf& b = a.sdf[sc.sdf_begin + s];
            const int ncomp = sdf_components(b.kind);
            for (int c = 0; c < ncomp; ++c, ++gc)
                if (gc % kAdjLanes == lane && sdf_eval(b, c, yp.x, yp.y, yp.z).phi < sc.r_low) ++n_act;
        }
    }
    return n_act;
}

// h_p = upstream_p / n_p for one pass (n_p = active pair and SDF contacts)
__global__ void k_adj_h(const PbdArgs a, int stab, const float4* __restrict__ Y, const float4* __restrict__ WS,
                        const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ cnt,
                        const float4* __restrict__ gx, const float4* __restrict__ gxt, float4* __restrict__ H)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = t / kAdjLanes;
    const int lane = (int)(t % kAdjLanes);
    const bool live = p < a.n;   // every lane stays for the shuffles
    int n_act = 0;
    if (live) {
        const SceneDev& sc = a.scenes[a.lr_scene[p]];
        n_act = lane_active_count(a, sc, Y, WS, nbr, p, (int)cnt[p], Y[p], WS[p].w, lane);
    }
    n_act = lanes_sum(n_act);
    if (!live || lane != 0) return;
    float4 up = gxt[p];
    if (stab) {
        const float4 u2 = gx[p];
        up.x += u2.x;
        up.y += u2.y;
        up.z += u2.z;
    }
    const float inv = n_act > 0 ? 1.0f / (float)n_act : 0.0f;
    H[p] = make_float4(up.x * inv, up.y * inv, up.z * inv, 0.0f);
}

// rec (optional): the decisions of this pass that the reverse mode
// differentiates, in original particle order (rec.idx: slot -> particle):
// for candidate k of particle i, cand[k n + i] = the partner's index and
// pair[k n + i] = bit 0 contact (|x_ij| < 2 r_LR), bit 1 kinetic friction
// scale; for SDF component c, sdf[i n_comp + c] = bit 0 contact, bit 1
// kinetic friction scale.  Entries of absent candidates: index -1, bits 0.
// Y_next (not null): the evaluation positions of the pass before this one
// (the next to reverse), whose h = upstream / n_p the particle's lanes
// compute at the end from its updated gradients (stab_next: that pass is a
// stabilization pass) into H_next, bitwise as k_adj_h would.
__global__ void k_adj_pass(const PbdArgs a, int stab, const float4* __restrict__ Y, const float4* __restrict__ XT,
                           const float4* __restrict__ XF, const float4* __restrict__ WS,
                           const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ cnt,
                           const float4* __restrict__ H, float4* __restrict__ gx, float4* __restrict__ gxt,
                           float* __restrict__ gws, const AdjRecord rec, const float4* __restrict__ Y_next,
                           int stab_next, float4* __restrict__ H_next)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = t / kAdjLanes;
    const int lane = (int)(t % kAdjLanes);
    const bool live = p < a.n;   // every lane stays for the shuffles
    float acc[3] = {0.f, 0.f, 0.f}, accx[3] = {0.f, 0.f, 0.f}, gw = 0.0f;
    int n_next = 0;
    if (live && Y_next) {
        const SceneDev& sc = a.scenes[a.lr_scene[p]];
        n_next = lane_active_count(a, sc, Y_next, WS, nbr, p, (int)cnt[p], Y_next[p], WS[p].w, lane);
    }
    if (live) {
        const SceneDev& sc = a.scenes[a.lr_scene[p]];
        const float d0 = 2.0f * sc.r_low;
        const float4 yp = Y[p];
        const float wp = WS[p].w;
        const float4 hp4 = H[p];
        const float hp[3] = {hp4.x, hp4.y, hp4.z};
        const float4 xtp = XT[p], xfp = XF[p];
        const int nc = (int)cnt[p];
        const int64_t ri = rec.pair ? (int64_t)rec.idx[p] : 0;
        if (rec.pair)
            for (int k = nc + lane; k < rec.cap; k += kAdjLanes) {
                rec.cand[(int64_t)k * a.n + ri] = -1;
                rec.pair[(int64_t)k * a.n + ri] = 0;
            }
        for (int k = lane; k < nc; k += kAdjLanes) {
            const uint32_t q = nbr[(int64_t)k * a.n + p];
            const float4 yq = Y[q];
            const PairGeo g = pair_geo(yp, yq);
            uint8_t* rb = nullptr;
            if (rec.pair) {
                rec.cand[(int64_t)k * a.n + ri] = (int32_t)rec.idx[q];
                rb = rec.pair + (int64_t)k * a.n + ri;
                *rb = g.d < d0 ? 1 : 0;
            }
            if (!(g.d < d0) || g.d2 == 0.0f) continue;
            const float wq = WS[q].w;
            const float W = wp + wq;
            if (!(W > 0.0f)) continue;
            const float mp = wp / W, mq = wq / W, pen = d0 - g.d;
            const float e[3] = {g.ex, g.ey, g.ez};
            const float u[3] = {g.ex / g.d, g.ey / g.d, g.ez / g.d};
            const float4 hq4 = H[q];
            const float hq[3] = {hq4.x, hq4.y, hq4.z};
            M3 K;
            m3_eye(K, d0 / g.d - 1.0f);
            m3_outer_add(K, -d0 / g.d, u, u);
            float tv[3] = {0.f, 0.f, 0.f};
            m3_tmul_add(tv, -mp, K, hp);
            m3_tmul_add(tv, mq, K, hq);
            acc[0] -= tv[0];
            acc[1] -= tv[1];
            acc[2] -= tv[2];
            const float uh = u[0] * (hp[0] + hq[0]) + u[1] * (hp[1] + hq[1]) + u[2] * (hp[2] + hq[2]);
            gw += -pen * (wq / (W * W)) * uh;
            if (!stab) {
                const float4 xtq = XT[q], xfq = XF[q];
                const float rel[3] = {(xtp.x - xfp.x) - (xtq.x - xfq.x), (xtp.y - xfp.y) - (xtq.y - xfq.y),
                                      (xtp.z - xfp.z) - (xtq.z - xfq.z)};
                const float base = sc.friction_mode == 1 ? pen : d0;
                float F[3];
                M3 Fr, Fe;
                bool kin = false;
                fric_jac(rel, e, g.d2, false, base * sc.mu_s, base * sc.mu_k, sc.friction_mode == 1, sc.mu_k, u, F, Fr,
                         Fe, &kin);
                if (rb && kin) *rb |= 2;
                const float hF[3] = {-mp * hp[0] + mq * hq[0], -mp * hp[1] + mq * hq[1], -mp * hp[2] + mq * hq[2]};
                float grel[3] = {0.f, 0.f, 0.f}, ge[3] = {0.f, 0.f, 0.f};
                m3_tmul_add(grel, 1.0f, Fr, hF);
                m3_tmul_add(ge, 1.0f, Fe, hF);
    #pragma unroll
                for (int k2 = 0; k2 < 3; ++k2) {
                    acc[k2] += grel[k2] - ge[k2];
                    accx[k2] -= grel[k2];
                }
                const float Fh = F[0] * (hp[0] + hq[0]) + F[1] * (hp[1] + hq[1]) + F[2] * (hp[2] + hq[2]);
                gw += -(wq / (W * W)) * Fh;
            }
        }
        if (rec.sdf)
            for (int c = lane; c < rec.n_comp; c += kAdjLanes) rec.sdf[ri * rec.n_comp + c] = 0;
        if (wp > 0.0f) {
            int gc = 0;   // component index over all the scene's SDFs; lane gc % kAdjLanes takes it
            for (int s = 0; s < sc.n_sdf; ++s) {
                const gs_sdf& b = a.sdf[sc.sdf_begin + s];
                const int ncomp = sdf_components(b.kind);
                const float bmu_s = sqrtf(sc.mu_s * b.mu_s), bmu_k = sqrtf(sc.mu_k * b.mu_k);
                for (int c = 0; c < ncomp; ++c, ++gc) {
                    if (gc % kAdjLanes != lane) continue;
                    const SdfHit h = sdf_eval(b, c, yp.x, yp.y, yp.z);
                    if (!(h.phi < sc.r_low)) continue;
                    uint8_t* sb = (rec.sdf && gc < rec.n_comp) ? rec.sdf + ri * rec.n_comp + gc : nullptr;
                    if (sb) *sb = 1;
                    const float n[3] = {h.nx, h.ny, h.nz};
                    const float an = n[0] * hp[0] + n[1] * hp[1] + n[2] * hp[2];
                    acc[0] -= an * n[0];
                    acc[1] -= an * n[1];
                    acc[2] -= an * n[2];
                    if (!stab) {
                        const float pen = sc.r_low - h.phi;
                        const float dv[3] = {(xtp.x - xfp.x) - b.vel[0] * a.dt, (xtp.y - xfp.y) - b.vel[1] * a.dt,
                                             (xtp.z - xfp.z) - b.vel[2] * a.dt};
                        const float base = sc.friction_mode == 1 ? pen : d0;
                        float F[3];
                        M3 Fr, Fe;
                        bool kin = false;
                        fric_jac(dv, n, 1.0f, true, base * bmu_s, base * bmu_k, false, bmu_k, n, F, Fr, Fe, &kin);
                        if (sb && kin) *sb |= 2;
                        float gd[3] = {0.f, 0.f, 0.f};
                        m3_tmul_add(gd, -1.0f, Fr, hp);
    #pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2) {
                            acc[k2] += gd[k2];
                            accx[k2] -= gd[k2];
                        }
                        if (sc.friction_mode == 1) {
                            const Tangent tg = tangent_part(dv[0], dv[1], dv[2], n[0], n[1], n[2], 1.0f);
                            const float thr_s = base * bmu_s, thr_k = base * bmu_k;
                            if (!(tg.L < thr_s) && tg.L > 0.0f && thr_k / tg.L < 1.0f) {
                                const float q = (tg.tx * hp[0] + tg.ty * hp[1] + tg.tz * hp[2]) / tg.L;
                                acc[0] += q * bmu_k * n[0];
                                acc[1] += q * bmu_k * n[1];
                                acc[2] += q * bmu_k * n[2];
                            }
                        }
                    }
                }
            }
        }
    }   // live
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc[k] = lanes_sum(acc[k]);
        accx[k] = lanes_sum(accx[k]);
    }
    gw = lanes_sum(gw);
    if (Y_next) n_next = lanes_sum(n_next);
    if (!live || lane != 0) return;
    float4 ngx = gx[p], ngxt = gxt[p];
    if (stab) {
        ngx = make_float4(ngx.x + acc[0], ngx.y + acc[1], ngx.z + acc[2], 0.0f);
        gx[p] = ngx;
    } else {
        ngxt = make_float4(ngxt.x + acc[0], ngxt.y + acc[1], ngxt.z + acc[2], 0.0f);
        gxt[p] = ngxt;
        ngx = make_float4(ngx.x + accx[0], ngx.y + accx[1], ngx.z + accx[2], 0.0f);
        gx[p] = ngx;
    }
    gws[p] += gw;
    if (Y_next) {   // h of the next pass to reverse, as k_adj_h
        float4 up = ngxt;
        if (stab_next) {
            up.x += ngx.x;
            up.y += ngx.y;
            up.z += ngx.z;
        }
        const float inv = n_next > 0 ? 1.0f / (float)n_next : 0.0f;
        H_next[p] = make_float4(up.x * inv, up.y * inv, up.z * inv, 0.0f);
    }
}

// predict: xt = x + dt (v + dt g), w = (1/m) e^{k (z - ground)}
__global__ void k_adj_final(const PbdArgs a, const uint32_t* __restrict__ idx, const float4* __restrict__ WS,
                            const float4* __restrict__ gx, const float4* __restrict__ gxt,
                            const float* __restrict__ gws, float4* __restrict__ gx0, float4* __restrict__ gv0)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    const SceneDev& sc = a.scenes[a.lr_scene[p]];
    const uint32_t i = idx[p];
    const float4 u = gx[p], t = gxt[p];
    gx0[i] = make_float4(u.x + t.x, u.y + t.y, u.z + t.z + gws[p] * WS[p].w * sc.mass_k, 0.0f);
    gv0[i] = make_float4(a.dt * t.x, a.dt * t.y, a.dt * t.z, 0.0f);
}

}  // namespace

cudaError_t gs_launch_upsample_bwd(cudaStream_t s, const SceneDev* scenes, const gs_sdf* sdf, const float4* lr_spos,
                                   const float4* lr_svel, const uint32_t* cell_start, const float4* hx,
                                   const float4* hv, const float4* gxo, const float4* gvo, float4* ghx, float4* ghv,
                                   float4* gXs, float4* gVs, int64_t m, float dt, int64_t* launches, uint32_t* rec,
                                   const uint32_t* lr_idx, float4* coef, const uint32_t* order, float4* pos_sorted)
{
    if (m <= 0) return cudaSuccess;
    k_upsample_bwd<<<gs_blocks(m * kBwdLanes, 128), 128, 0, s>>>(scenes, sdf, lr_spos, lr_svel, cell_start, hx, hv, gxo, gvo, ghx,
                                                      ghv, gXs, gVs, m, dt, rec, lr_idx, coef, order, pos_sorted);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_upsample_bwd_lr(cudaStream_t s, const SceneDev* scenes, const float4* lr_spos,
                                      const float4* lr_svel, const uint32_t* lr_skeys, const float4* hx_sorted,
                                      const uint32_t* hr_cell_start, const float4* coef, float4* gXs, float4* gVs,
                                      int64_t n_low, int64_t* launches)
{
    if (n_low <= 0) return cudaSuccess;
    k_upsample_bwd_lr<<<gs_blocks(n_low * 32, 128), 128, 0, s>>>(scenes, lr_spos, lr_svel, lr_skeys, hx_sorted,
                                                                  hr_cell_start, coef, gXs, gVs, n_low);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_scatter2(cudaStream_t s, const uint32_t* idx, const float4* a, const float4* b, float4* ao,
                               float4* bo, int64_t n, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    k_scatter2<<<gs_blocks(n, 256), 256, 0, s>>>(idx, a, b, ao, bo, n);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_adj_init(cudaStream_t s, int64_t n, const uint32_t* idx, const float4* gxo, const float4* gvo,
                               float dt, float4* gx, float4* gxt, float* gws, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    k_adj_init<<<gs_blocks(n, 256), 256, 0, s>>>(n, idx, gxo, gvo, dt, gx, gxt, gws);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_adj_h(cudaStream_t s, const PbdArgs& a, int stab, const float4* Y, const float4* WS,
                            const uint32_t* nbr, const uint32_t* cnt, const float4* gx, const float4* gxt, float4* H,
                            int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_adj_h<<<gs_blocks(a.n * kAdjLanes, 128), 128, 0, s>>>(a, stab, Y, WS, nbr, cnt, gx, gxt, H);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_adj_pass(cudaStream_t s, const PbdArgs& a, int stab, const float4* Y, const float4* XT,
                               const float4* XF, const float4* WS, const uint32_t* nbr, const uint32_t* cnt,
                               const float4* H, float4* gx, float4* gxt, float* gws, int64_t* launches,
                               const AdjRecord& rec, const float4* Y_next, int stab_next, float4* H_next)
{
    if (a.n <= 0) return cudaSuccess;
    k_adj_pass<<<gs_blocks(a.n * kAdjLanes, 128), 128, 0, s>>>(a, stab, Y, XT, XF, WS, nbr, cnt, H, gx, gxt, gws, rec,
                                                                Y_next, stab_next, H_next);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_adj_final(cudaStream_t s, const PbdArgs& a, const uint32_t* idx, const float4* WS,
                                const float4* gx, const float4* gxt, const float* gws, float4* gx0, float4* gv0,
                                int64_t* launches)
{
    if (a.n <= 0) return cudaSuccess;
    k_adj_final<<<gs_blocks(a.n, 256), 256, 0, s>>>(a, idx, WS, gx, gxt, gws, gx0, gv0);
    *launches += 1;
    return cudaGetLastError();
}
