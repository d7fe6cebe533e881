// Initial sampling of a closed triangle mesh's volume (Sec. 4): cells of side
// 2 r / sqrt(3) over the mesh's bounding box, random candidates (given),
// those inside the mesh (generalized winding number > 1/2) assigned to their
// cells in input order, then per cell the first candidate at least 2 r from
// every sample taken so far.  The cells are taken in 27 phases
// (cx mod 3, cy mod 3, cz mod 3; phase index (cx mod 3) + 3 (cy mod 3) +
// 9 (cz mod 3) ascending): two cells of a phase are three cells apart along
// some axis, more than 2 r, so one launch takes a whole phase, one thread per
// cell, with the result of taking its cells one by one.  The decisions are
// taken in double precision with the multiplications and additions rounded
// one by one, so that they are those of a plain sequential evaluation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "gs.h"
#include "gs_internal.cuh"

namespace {

__device__ __forceinline__ double dot3_rn(const double* a, const double* b)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

// Solid angle of the triangle seen from p over 4 pi (Van Oosterom and
// Strackee 1983: tan(Omega / 2) = det[a b c] / (|a||b||c| + (a.b)|c| +
// (b.c)|a| + (c.a)|b|), a, b, c the corners relative to p).
__device__ double tri_winding(const double* A, const double* B, const double* C, const double* p)
{
    double a[3], b[3], c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = __dsub_rn(A[k], p[k]);
        b[k] = __dsub_rn(B[k], p[k]);
        c[k] = __dsub_rn(C[k], p[k]);
    }
    const double la = sqrt(dot3_rn(a, a)), lb = sqrt(dot3_rn(b, b)), lc = sqrt(dot3_rn(c, c));
    const double m0 = __dsub_rn(__dmul_rn(b[1], c[2]), __dmul_rn(b[2], c[1]));
    const double m1 = __dsub_rn(__dmul_rn(b[0], c[2]), __dmul_rn(b[2], c[0]));
    const double m2 = __dsub_rn(__dmul_rn(b[0], c[1]), __dmul_rn(b[1], c[0]));
    const double det = __dadd_rn(__dsub_rn(__dmul_rn(a[0], m0), __dmul_rn(a[1], m1)), __dmul_rn(a[2], m2));
    const double den = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(la, lb), lc), __dmul_rn(dot3_rn(a, b), lc)),
                                           __dmul_rn(dot3_rn(b, c), la)),
                                 __dmul_rn(dot3_rn(c, a), lb));
    return atan2(det, den) / (2.0 * 3.14159265358979323846);
}

struct SampleGrid {
    double lo[3];
    double h;
    int64_t dims[3];
    int64_t n_cell;
};

// Inside flag and cell of every candidate; the cell's counter gives the
// candidate its arrival rank (the counting sort puts each cell in index
// order afterwards).
// surface: every candidate counts (points on the surface), no winding number.
__global__ void k_sample_classify(const double* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                                  const double* __restrict__ cand, int64_t nc, const SampleGrid g,
                                  uint8_t* __restrict__ inside, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ rank, uint32_t* __restrict__ cell_count, int surface)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double p[3] = {cand[3 * i], cand[3 * i + 1], cand[3 * i + 2]};
    if (surface) {
        inside[i] = 1;
    } else {
        double w = 0.0;
        for (int64_t t = 0; t < nt; ++t)
            w = __dadd_rn(w, tri_winding(V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2], p));
        inside[i] = w > 0.5 ? 1 : 0;
    }
    int64_t c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double f = floor(__ddiv_rn(__dsub_rn(p[k], g.lo[k]), g.h));
        c[k] = f < 0.0 ? 0 : (f >= (double)(g.dims[k] - 1) ? g.dims[k] - 1 : (int64_t)f);
    }
    const uint32_t key = (uint32_t)(c[0] + g.dims[0] * (c[1] + g.dims[1] * c[2]));
    keys[i] = key;
    rank[i] = atomicAdd(cell_count + key, 1u);
}

// One phase: a thread per cell (cx, cy, cz) = (px + 3 i, py + 3 j, pz + 3 k).
__global__ void k_sample_phase(const double* __restrict__ cand, const uint8_t* __restrict__ inside,
                               const uint32_t* __restrict__ order, const uint32_t* __restrict__ cell_start,
                               int32_t* __restrict__ pick, const SampleGrid g, int px, int py, int pz, int64_t nx,
                               int64_t ny, int64_t n_phase, double d2min)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_phase) return;
    const int64_t cx = px + 3 * (t % nx), cy = py + 3 * ((t / nx) % ny), cz = pz + 3 * (t / (nx * ny));
    const int64_t c = cx + g.dims[0] * (cy + g.dims[1] * cz);
    for (uint32_t q = cell_start[c]; q < cell_start[c + 1]; ++q) {
        const uint32_t i = order[q];
        if (!inside[i]) continue;
        const double p[3] = {cand[3 * i], cand[3 * i + 1], cand[3 * i + 2]};
        bool free_ = true;
        for (int64_t z = cz - 2; z <= cz + 2 && free_; ++z)
            for (int64_t y = cy - 2; y <= cy + 2 && free_; ++y)
                for (int64_t x = cx - 2; x <= cx + 2 && free_; ++x) {
                    if (x < 0 || y < 0 || z < 0 || x >= g.dims[0] || y >= g.dims[1] || z >= g.dims[2]) continue;
                    const int32_t s = pick[x + g.dims[0] * (y + g.dims[1] * z)];
                    if (s < 0) continue;
                    const double d[3] = {__dsub_rn(p[0], cand[3 * (int64_t)s]), __dsub_rn(p[1], cand[3 * (int64_t)s + 1]),
                                         __dsub_rn(p[2], cand[3 * (int64_t)s + 2])};
                    if (dot3_rn(d, d) < d2min) free_ = false;
                }
        if (free_) {
            pick[c] = (int32_t)i;
            return;
        }
    }
}

struct DevBufs {
    std::vector<void*> p;
    ~DevBufs()
    {
        for (void* q : p) cudaFree(q);
    }
    template <class T>
    bool get(T** out, size_t count)
    {
        void* q = nullptr;
        if (gs_dalloc_bytes(&q, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        p.push_back(q);
        *out = (T*)q;
        return true;
    }
};

struct StreamGuard {
    cudaStream_t s = nullptr;
    ~StreamGuard()
    {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

}  // namespace

static int sample_impl(const double* vertices, int64_t n_vertices, const int32_t* triangles, int64_t n_triangles,
                       const double* candidates, int64_t n_candidates, double r, int64_t* selected, int64_t capacity,
                       int64_t* n_selected, uint8_t* inside, int surface)
{
    if (!n_selected || n_vertices < 0 || n_triangles < 0 || n_candidates < 0 || capacity < 0) return GS_ERR_ARG;
    *n_selected = 0;
    if (!(r > 0.0) || !std::isfinite(r) || (n_vertices > 0 && !vertices) || (n_triangles > 0 && !triangles) ||
        (n_candidates > 0 && !candidates) || (capacity > 0 && !selected) || n_candidates > 0x7fffffffLL ||
        (n_triangles > 0 && n_vertices == 0))
        return GS_ERR_ARG;
    for (int64_t k = 0; k < 3 * n_triangles; ++k)
        if (triangles[k] < 0 || triangles[k] >= n_vertices) return GS_ERR_ARG;
    for (int64_t k = 0; k < 3 * n_vertices; ++k)
        if (!std::isfinite(vertices[k])) return GS_ERR_DOMAIN;
    for (int64_t k = 0; k < 3 * n_candidates; ++k)
        if (!std::isfinite(candidates[k])) return GS_ERR_DOMAIN;
    // the grid, on the host in double precision
    SampleGrid g;
    double hi[3];
    for (int k = 0; k < 3; ++k) g.lo[k] = hi[k] = n_vertices ? vertices[k] : 0.0;
    for (int64_t i = 0; i < n_vertices; ++i)
        for (int k = 0; k < 3; ++k) {
            g.lo[k] = std::fmin(g.lo[k], vertices[3 * i + k]);
            hi[k] = std::fmax(hi[k], vertices[3 * i + k]);
        }
    g.h = 2.0 * r / std::sqrt(3.0);
    // Surface candidates lie on the triangles, so inside the box up to
    // rounding.  One farther out would be clamped into an edge cell, and the
    // phases keep two picks at least 2 r apart only while every candidate is
    // within (2 h - 2 r) / 2 = 0.154 r of its cell: refuse those beyond 0.15 r.
    if (surface) {
        const double m = 0.15 * r;
        for (int64_t i = 0; i < n_candidates; ++i)
            for (int k = 0; k < 3; ++k)
                if (candidates[3 * i + k] < g.lo[k] - m || candidates[3 * i + k] > hi[k] + m) return GS_ERR_ARG;
    }
    double cells = 1.0;
    for (int k = 0; k < 3; ++k) {
        g.dims[k] = (int64_t)std::floor((hi[k] - g.lo[k]) / g.h) + 1;
        cells *= (double)g.dims[k];
    }
    if (cells > 2147483646.0) return GS_ERR_ARG;   // cell ids and picks are 32-bit
    g.n_cell = g.dims[0] * g.dims[1] * g.dims[2];
    const double d2min = 4.0 * r * r;
    const int64_t nc = n_candidates, ncell = g.n_cell;

    StreamGuard sg;
    if (cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking) != cudaSuccess) return GS_ERR_CUDA;
    cudaStream_t s = sg.s;
    DevBufs B;
    double *dV = nullptr, *dC = nullptr;
    int32_t *dT = nullptr, *dpick = nullptr;
    uint8_t* din = nullptr;
    uint32_t *keys = nullptr, *rank = nullptr, *okeys = nullptr, *oidx = nullptr, *start = nullptr, *aux = nullptr;
    if (!B.get(&dV, 3 * (size_t)n_vertices) || !B.get(&dT, 3 * (size_t)n_triangles) || !B.get(&dC, 3 * (size_t)nc) ||
        !B.get(&din, (size_t)nc) || !B.get(&keys, (size_t)nc) || !B.get(&rank, (size_t)nc) ||
        !B.get(&okeys, (size_t)nc) || !B.get(&oidx, (size_t)nc) || !B.get(&start, (size_t)ncell + 1) ||
        !B.get(&aux, gs_scan_aux_words(ncell + 1)) || !B.get(&dpick, (size_t)ncell))
        return GS_ERR_OOM;
#define SK(call)                                  \
    do {                                          \
        if ((call) != cudaSuccess) {              \
            cudaGetLastError();                   \
            return GS_ERR_CUDA;                   \
        }                                         \
    } while (0)
    int64_t launches = 0;
    if (n_vertices) SK(cudaMemcpyAsync(dV, vertices, 24 * (size_t)n_vertices, cudaMemcpyHostToDevice, s));
    if (n_triangles) SK(cudaMemcpyAsync(dT, triangles, 12 * (size_t)n_triangles, cudaMemcpyHostToDevice, s));
    if (nc) SK(cudaMemcpyAsync(dC, candidates, 24 * (size_t)nc, cudaMemcpyHostToDevice, s));
    SK(gs_cs_clear(s, start, ncell));
    SK(cudaMemsetAsync(dpick, 0xff, sizeof(int32_t) * (size_t)ncell, s));
    if (nc) {
        k_sample_classify<<<gs_blocks(nc, 128), 128, 0, s>>>(dV, dT, n_triangles, dC, nc, g, din, keys, rank, start,
                                                             surface);
        SK(cudaGetLastError());
        // stable counting sort by cell: each cell's candidates in input order
        SK(gs_cs_finish(s, nc, ncell, keys, rank, okeys, oidx, start, aux, nullptr, nullptr, nullptr, nullptr,
                        &launches));
        for (int phase = 0; phase < 27; ++phase) {
            const int px = phase % 3, py = (phase / 3) % 3, pz = phase / 9;
            const int64_t nx = (g.dims[0] - px + 2) / 3, ny = (g.dims[1] - py + 2) / 3, nz = (g.dims[2] - pz + 2) / 3;
            const int64_t n_phase = nx * ny * nz;
            if (n_phase <= 0) continue;
            k_sample_phase<<<gs_blocks(n_phase, 128), 128, 0, s>>>(dC, din, oidx, start, dpick, g, px, py, pz, nx, ny,
                                                                   n_phase, d2min);
            SK(cudaGetLastError());
        }
    }
    // the picks, in ascending cell order, compacted on the host
    std::vector<int32_t> pick((size_t)ncell);
    SK(cudaMemcpyAsync(pick.data(), dpick, sizeof(int32_t) * (size_t)ncell, cudaMemcpyDeviceToHost, s));
    if (inside && nc) SK(cudaMemcpyAsync(inside, din, (size_t)nc, cudaMemcpyDeviceToHost, s));
    SK(cudaStreamSynchronize(s));
#undef SK
    int64_t n = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        if (pick[(size_t)c] < 0) continue;
        if (n < capacity) selected[n] = pick[(size_t)c];
        ++n;
    }
    *n_selected = n;
    return n > capacity ? GS_ERR_CAPACITY : GS_OK;
}

extern "C" int gs_sample_volume(const double* vertices, int64_t n_vertices, const int32_t* triangles,
                                int64_t n_triangles, const double* candidates, int64_t n_candidates, double r,
                                int64_t* selected, int64_t capacity, int64_t* n_selected, uint8_t* inside)
{
    return sample_impl(vertices, n_vertices, triangles, n_triangles, candidates, n_candidates, r, selected, capacity,
                       n_selected, inside, 0);
}

extern "C" int gs_sample_surface(const double* vertices, int64_t n_vertices, const double* candidates,
                                 int64_t n_candidates, double r, int64_t* selected, int64_t capacity,
                                 int64_t* n_selected)
{
    return sample_impl(vertices, n_vertices, nullptr, 0, candidates, n_candidates, r, selected, capacity, n_selected,
                       nullptr, 1);
}
