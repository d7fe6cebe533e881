// gs_api.cu -- host side of the C ABI declared in gs.h: argument checks,
// buffer ownership, the order in which the kernels of one LR step and one HR
// frame are enqueued on the context's stream, CUDA graphs of whole frames,
// and the launch-shape autotuner of the upsampling kernel.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "gs_internal.cuh"

namespace {

int fail(gs_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return code;
}

int cuda_fail(gs_ctx* c, cudaError_t e, const char* what)
{
    if (c) c->poisoned = true;
    return fail(c, GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// Host-side allocation failure injection (gs_set_alloc_failure): the
// countdown of device allocations left before every further one fails;
// negative: off.  Process-wide, like the allocator it stands in for.
std::atomic<long long> g_alloc_countdown{-1};

template <class T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) <= 0) {
        g_alloc_countdown.store(0);
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void**)p, count * sizeof(T));
}

}  // namespace

int gs_ctx_fail(gs_ctx* c, int code, const char* msg)
{
    return fail(c, code, "%s", msg);
}


cudaError_t gs_dalloc_bytes(void** p, size_t bytes)
{
    return dalloc((unsigned char**)p, bytes);
}

namespace {

struct Timed {
    gs_ctx* c;
    int id;
    cudaEvent_t stop = nullptr;
    Timed(gs_ctx* c_, int id_) : c(c_), id(id_)
    {
        if (!c->timing) return;
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return;
        }
        cudaEventRecord(a, c->stream);
        c->ev[id].push_back({a, b});
        stop = b;
    }
    ~Timed()
    {
        if (stop) cudaEventRecord(stop, c->stream);
    }
};

int check_state(gs_ctx* c)
{
    if (!c) return GS_ERR_ARG;
    if (c->poisoned) return fail(c, GS_ERR_STATE, "context is poisoned by an earlier CUDA error");
    return GS_OK;
}

int report_device_errors(gs_ctx* c)
{
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error word");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    int e = *c->h_err;
    if (e) {
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear error word");
        if (e & GS_DEVERR_NEIGHBOR_CAP)
            return fail(c, GS_ERR_CAPACITY, "an LR particle had more than %d candidate partners (max_neighbors)",
                        c->nbr_cap);
        if (e & GS_DEVERR_BAD_ID) return fail(c, GS_ERR_STATE, "HR id outside [0, n_high) met while unpermuting");
        if (e & GS_DEVERR_NONFINITE_ASYNC)
            return fail(c, GS_ERR_DOMAIN, "an asynchronously written field held a non-finite value; the state is invalid");
        if (e & GS_DEVERR_SOLID_REVERSE)
            return fail(c, GS_ERR_STATE, "a reverse mode was given LR particles of infinite mass; its gradients are "
                                         "invalid");
        if (e & GS_DEVERR_BARRIER_TIMEOUT)
            return fail(c, GS_ERR_TIMEOUT, "a grid barrier of the persistent LR solver timed out; results are invalid");
    }
    return GS_OK;
}

size_t field_bytes(const gs_ctx* c, int field)
{
    switch (field) {
    case GS_FIELD_LR_POS:
    case GS_FIELD_LR_VEL: return (size_t)c->n_low * sizeof(float4);
    case GS_FIELD_HR_POS:
    case GS_FIELD_HR_VEL: return (size_t)c->n_high * sizeof(float4);
    case GS_FIELD_HR_POS_INTERNAL:
    case GS_FIELD_HR_VEL_INTERNAL: return (size_t)c->hr_slots * sizeof(float4);
    case GS_FIELD_LR_CELL_START: return (size_t)(c->n_cell_total + 1) * sizeof(uint32_t);
    case GS_FIELD_LR_SORTED_INDEX: return (size_t)c->n_low * sizeof(uint32_t);
    case GS_FIELD_HR_SORTED_KEY: return (size_t)c->hr_slots * sizeof(uint32_t);
    case GS_FIELD_LR_MATERIAL:
    case GS_FIELD_LR_BODY: return (size_t)c->n_low * sizeof(uint32_t);
    default: return (size_t)-1;
    }
}

// ---- HR slots <-> original order (kernels local to this file) ---------------
// Slot p of scene s that is not padding holds the particle with original id
// hr_real_begin + (p - hr_begin) in the identity order.
__global__ void k_hr_load(const float4* __restrict__ src, float4* __restrict__ dst, const uint32_t* __restrict__ tag,
                          const SceneDev* __restrict__ scenes, int64_t n_slots, int set_ids)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_slots) return;
    const uint32_t t = tag[p];
    if (t & kPadBit) {
        dst[p] = make_float4(0.f, 0.f, 0.f, set_ids ? __uint_as_float(0xffffffffu) : 0.f);
        return;
    }
    const SceneDev& sc = scenes[t];
    const int64_t id = sc.hr_real_begin + (p - sc.hr_begin);
    float4 v = src[id];
    if (set_ids) v.w = __uint_as_float((uint32_t)id);
    dst[p] = v;
}

// Largest of n material ids (into *out, zero beforehand).
__global__ void k_max_id(const uint32_t* __restrict__ ids, int64_t n, unsigned* out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned m = i < n ? ids[i] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

// Sets `bit` in *err when some of the n positions has w = 0 (an LR particle
// of infinite mass).
__global__ void k_flag_solid(const float4* __restrict__ pos, int64_t n, int* err, int bit)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pos[i].w == 0.0f) atomicOr(err, bit);
}

// Asynchronous writes of both fields of a kind, checked on the way: a copy
// of LR position and velocity, and the load of HR position and velocity into
// the identity slot order (ids into the w of the position); a non-finite
// x, y, z sets `bit` in *err.
__global__ void k_copy2_checked(const float4* __restrict__ a, const float4* __restrict__ b, float4* __restrict__ oa,
                                float4* __restrict__ ob, int64_t n, int* err, int bit)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 u = a[i], v = b[i];
    if (!(isfinite(u.x) && isfinite(u.y) && isfinite(u.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z)))
        atomicOr(err, bit);
    oa[i] = u;
    ob[i] = v;
}

// The check of an assembled HR state (gs_hr_slab_assemble): bit 1 of *err
// when some x, y, z is not finite, bit 2 when the id bits in the w of a
// slot's position differ from the context's.
__global__ void k_slab_check(const float4* __restrict__ pos, const float4* __restrict__ vel,
                             const float4* __restrict__ cur, int64_t n, int* err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float4 u = pos[p], v = vel[p];
    if (!(isfinite(u.x) && isfinite(u.y) && isfinite(u.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z)))
        atomicOr(err, 1);
    if (__float_as_uint(u.w) != __float_as_uint(cur[p].w)) atomicOr(err, 2);
}

__global__ void k_hr_load2_checked(const float4* __restrict__ sp, const float4* __restrict__ sv,
                                   float4* __restrict__ dp, float4* __restrict__ dv, const uint32_t* __restrict__ tag,
                                   const SceneDev* __restrict__ scenes, int64_t n_slots, int* err, int bit)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_slots) return;
    const uint32_t t = tag[p];
    if (t & kPadBit) {
        dp[p] = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
        dv[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const SceneDev& sc = scenes[t];
    const int64_t id = sc.hr_real_begin + (p - sc.hr_begin);
    float4 u = sp[id];
    const float4 v = sv[id];
    if (!(isfinite(u.x) && isfinite(u.y) && isfinite(u.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z)))
        atomicOr(err, bit);
    u.w = __uint_as_float((uint32_t)id);
    dp[p] = u;
    dv[p] = v;
}

cudaError_t launch_hr_load(gs_ctx* c, const float4* src, float4* dst, int set_ids)
{
    if (c->hr_slots <= 0) return cudaSuccess;
    k_hr_load<<<gs_blocks(c->hr_slots, 256), 256, 0, c->stream>>>(src, dst, c->hr_scene, c->d_scenes, c->hr_slots,
                                                                   set_ids);
    c->launches += 1;
    return cudaGetLastError();
}

int bin_low_at(gs_ctx* c, const float4* positions)
{
    const int64_t n = c->n_low;
    CK(gs_count_sort_cells(c->stream, positions, n, c->d_scenes, c->lr_scene, c->n_cell_total, c->lr_keys[0],
                           c->lr_vals[0], c->lr_keys[1], c->lr_vals[1], c->lr_cell_start, c->scan_aux, &c->launches),
       "bin by cell");
    c->lr_sorted_keys = c->lr_keys[1];
    c->lr_sorted_idx = c->lr_vals[1];
    return GS_OK;
}

PbdArgs pbd_args(const gs_ctx* c, float dt)
{
    PbdArgs a;
    a.n = c->n_low;
    a.dt = dt;
    a.dt_dev = nullptr;
    a.scenes = c->d_scenes;
    a.lr_scene = c->lr_scene;
    a.sdf = c->d_sdf;
    const bool mat = c->n_materials > 0;
    a.mu_mat = mat ? c->d_mu : nullptr;
    a.mu_cross = mat ? c->d_mu + GS_MAX_MATERIALS : nullptr;
    const bool bodies = c->n_bodies > 0;
    a.body = bodies ? c->lr_body : nullptr;
    a.xo = bodies ? c->lr_xo : nullptr;
    a.body_xf = bodies ? c->body_xf : nullptr;
    a.sorted_idx = c->lr_vals[1];   // the step's binning leaves the particle of each slot here
    return a;
}

// The LR step's cell-order copy: material ids ride in the w of x; with rigid
// bodies the slot of every particle is recorded for the body reductions.
CsExtras step_extras(const gs_ctx* c, const PbdArgs& a)
{
    CsExtras ex;
    ex.gb_w = a.mu_cross ? c->lr_mat : nullptr;
    ex.slot_of = c->n_bodies > 0 ? c->lr_slot : nullptr;
    return ex;
}

int create_impl(int S, const gs_scene* scenes, const float* r_low, const float* r_high, const int* ratio,
                void* cuda_stream, gs_ctx** out)
{
    if (!out) return GS_ERR_ARG;
    *out = nullptr;
    if (S < 1 || S > 65536 || !scenes || !r_low || !ratio) return GS_ERR_ARG;
    gs_ctx* c = new (std::nothrow) gs_ctx();
    if (!c) return GS_ERR_OOM;
    c->n_scenes = S;
    c->scenes.resize(S);
    c->prm.resize(S);
    int64_t lr = 0, hr_real = 0, hr_slot = 0, cells = 0;
    for (int s = 0; s < S; ++s) {
        const gs_scene& in = scenes[s];
        const float rl = r_low[s];
        const float rh_in = r_high ? r_high[s] : 0.0f;
        const int ra = ratio[s];
        bool bad = !(rl > 0.0f) || !std::isfinite(rl) || ra < 1 || in.n_low < 0 || in.n_high < 0 ||
                   in.n_high > 0x7fffffffLL || in.n_sdf < 0 ||
                   in.n_sdf > GS_MAX_SDF || (in.n_sdf > 0 && !in.sdf);
        for (int k = 0; k < 3 && !bad; ++k)
            bad = !(in.box_hi[k] > in.box_lo[k]) || !std::isfinite(in.box_lo[k]) || !std::isfinite(in.box_hi[k]);
        gs_params p = in.params;
        if (std::isnan(p.ground_z)) p.ground_z = in.box_lo[2];
        if (p.neighbor_radius <= 0.0f) p.neighbor_radius = 3.0f * rl;
        if (p.max_neighbors <= 0) p.max_neighbors = 64;
        bad = bad || !(p.neighbor_radius > 2.0f * rl) || p.neighbor_radius > 3.0f * rl || p.n_stab < 0 ||
              p.n_stab > 100 || p.resort_every < 0 || p.max_neighbors > 4096 ||
              (p.friction_mode != 0 && p.friction_mode != 1);
        if (s > 0)   // one solver configuration per context
            bad = bad || p.n_stab != c->prm[0].n_stab || p.resort_every != c->prm[0].resort_every ||
                  p.max_neighbors != c->prm[0].max_neighbors;
        if (bad) {
            delete c;
            return GS_ERR_ARG;
        }
        c->prm[s] = p;
        SceneDev& d = c->scenes[s];
        std::memset(&d, 0, sizeof d);
        // grid contract
        const double hd = 3.0 * (double)rl * (1.0 + 1.0 / 1024.0);
        const float hf = (float)hd;
        d.g.h = hf;
        d.g.inv_h = (float)(1.0 / (double)hf);
        d.g.ox = in.box_lo[0];
        d.g.oy = in.box_lo[1];
        d.g.oz = in.box_lo[2];
        int dims[3];
        for (int k = 0; k < 3; ++k) {
            double n = std::ceil(((double)in.box_hi[k] - (double)in.box_lo[k]) / (double)hf);
            if (n > (double)(1 << 20)) {
                delete c;
                return GS_ERR_ARG;
            }
            dims[k] = n < 1 ? 1 : (int)n;
        }
        d.g.dx = dims[0];
        d.g.dy = dims[1];
        d.g.dz = dims[2];
        const int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
        d.cell_off = (uint32_t)cells;
        d.n_cell = (uint32_t)ncell;
        cells += ncell + 1;
        if (cells * 8 > 0xffffffffLL) {
            delete c;
            return GS_ERR_ARG;
        }
        const int64_t m = in.n_high > 0 ? in.n_high : (int64_t)in.n_low * ra;
        d.lr_begin = lr;
        d.lr_end = lr + in.n_low;
        d.hr_begin = hr_slot;
        d.hr_end = hr_slot + m;
        d.hr_real_begin = hr_real;
        d.warp_begin = hr_slot / 32;
        lr += in.n_low;
        hr_real += m;
        hr_slot += (m + 31) / 32 * 32;
        d.r_low = rl;
        d.r_high = rh_in > 0.0f ? rh_in : (float)((double)rl * std::pow((double)ra, -1.0 / 3.0));
        d.gx = p.gravity[0];
        d.gy = p.gravity[1];
        d.gz = p.gravity[2];
        d.mu_s = p.mu_s;
        d.mu_k = p.mu_k;
        d.c1 = p.c1;
        d.c2 = p.c2;
        d.mass_k = p.mass_scale_k;
        d.ground_z = p.ground_z;
        d.rc = p.neighbor_radius;
        d.friction_mode = p.friction_mode;
        d.sdf_begin = (int)c->sdf_host.size();
        d.n_sdf = in.n_sdf;
        for (int k = 0; k < in.n_sdf; ++k) c->sdf_host.push_back(in.sdf[k]);
    }
    if (hr_real > 0x7fffffffLL || hr_slot > 0x7fffffffLL || lr > 0x7fffffffLL) {
        delete c;
        return GS_ERR_ARG;   // ids and slots are stored as uint32
    }
    c->n_low = lr;
    c->n_high = hr_real;
    c->hr_slots = hr_slot;
    c->n_warps = hr_slot / 32;
    c->n_cell_total = cells;
    c->lr_key_bits = gs_key_bits(cells);
    c->hr_key_bits = gs_key_bits(cells * 8);
    c->resort_every = c->prm[0].resort_every;
    c->nbr_cap = c->prm[0].max_neighbors;
    c->n_stab = c->prm[0].n_stab;

    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    if (e == cudaSuccess && coop) c->solve_blocks = gs_solve_blocks(c->sm_count);
    if (e != cudaSuccess) {
        delete c;
        return GS_ERR_CUDA;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return GS_ERR_CUDA;
        }
        c->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&c->stream_hr, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream_d2h, cudaStreamNonBlocking);
    for (int f = 0; f < 4 && e == cudaSuccess; ++f) {
        e = cudaEventCreateWithFlags(&c->ev_in_ready[f], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in_free[f], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out_ready[f], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out_free[f], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        gs_destroy(c);
        return GS_ERR_CUDA;
    }
    const int64_t N = c->n_low, MS = c->hr_slots, MR = c->n_high;
    const int64_t NM = std::max(N, MS);
    bool ok = true;
    auto A = [&](cudaError_t r) { ok = ok && r == cudaSuccess; };
    A(dalloc(&c->d_scenes, (size_t)S));
    A(dalloc(&c->d_sdf, std::max<size_t>(c->sdf_host.size(), 1)));
    A(dalloc(&c->lr_scene, N));
    A(dalloc(&c->hr_scene, MS));
    A(dalloc(&c->lr_pos, N));
    A(dalloc(&c->lr_vel, N));
    A(dalloc(&c->lr_keys[0], N));
    A(dalloc(&c->lr_keys[1], N));
    A(dalloc(&c->lr_vals[0], N));
    A(dalloc(&c->lr_vals[1], N));
    A(dalloc(&c->lr_cell_start, cells + 2));   // + the flag of particles of infinite mass
    A(dalloc(&c->step_cell_start, cells + 1));
    A(dalloc(&c->d_sdf_pend, std::max<size_t>(c->sdf_host.size(), 1)));
    A(dalloc(&c->scan_aux, gs_scan_aux_words(cells + 1)));
    A(dalloc(&c->lr_spos, N));
    A(dalloc(&c->lr_svel, N));
    A(dalloc(&c->lr_xt, N));
    A(dalloc(&c->lr_mat, N));
    A(dalloc(&c->lr_body, N));
    A(dalloc(&c->lr_xo, N));
    A(dalloc(&c->body_members, N));
    A(dalloc(&c->body_start, GS_MAX_BODIES + 1));
    A(dalloc(&c->body_xf, 4 * GS_MAX_BODIES));
    A(dalloc(&c->lr_slot, N));
    A(dalloc(&c->d_mu, (size_t)GS_MAX_MATERIALS * (GS_MAX_MATERIALS + 1)));
    for (int k = 0; k < 2; ++k) {
        A(dalloc(&c->s_xt[k], N));
        A(dalloc(&c->s_x[k], N));
        A(dalloc(&c->hr_pos[k], MS));
        A(dalloc(&c->hr_vel[k], MS));
        A(dalloc(&c->hr_keys[k], MS));
        A(dalloc(&c->hr_vals[k], MS));
    }
    A(dalloc(&c->nbr, (size_t)N * c->nbr_cap));
    A(dalloc(&c->gXs, N));
    A(dalloc(&c->gVs, N));
    A(dalloc(&c->nbr_cnt, N));
    A(dalloc(&c->tmp4, std::max(NM, MR)));
    A(dalloc(&c->stage_in, std::max(N, MR)));
    c->sort_hist_cap = std::max(gs_sort_hist_words(N), gs_sort_hist_words(MS));
    A(dalloc(&c->sort_hist, c->sort_hist_cap));
    c->hr_bins = cells * 8;
    c->hr_counting = MS > 0 && c->hr_bins <= std::max<int64_t>(8 * MS, (int64_t)1 << 20);
    if (c->hr_counting) {
        A(dalloc(&c->hr_bin_start, c->hr_bins + 2));
        A(dalloc(&c->hr_big, MS / 33 + 1));
        A(dalloc(&c->hr_scan_aux, gs_scan_aux_words(c->hr_bins + 1)));
    }
    A(dalloc(&c->d_work, 1));
    A(dalloc(&c->d_err, 2));   // [0] device error bits, [1] scratch word of the host checks
    A(dalloc(&c->d_bar, 2));
    A(dalloc(&c->d_cfl, 1));
    if (ok) ok = cudaMallocHost((void**)&c->h_err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        gs_destroy(c);
        return GS_ERR_OOM;
    }
    *c->h_err = 0;
    // scene tags of every LR and HR slot
    std::vector<uint32_t> lt((size_t)N), ht((size_t)MS);
    for (int s = 0; s < S; ++s) {
        const SceneDev& d = c->scenes[s];
        for (int64_t i = d.lr_begin; i < d.lr_end; ++i) lt[(size_t)i] = (uint32_t)s;
        const int64_t slot_end = (s + 1 < S) ? c->scenes[s + 1].hr_begin : MS;
        for (int64_t i = d.hr_begin; i < slot_end; ++i) ht[(size_t)i] = (uint32_t)s | (i >= d.hr_end ? kPadBit : 0u);
    }
    bool z = true;
    auto Z = [&](cudaError_t r) { z = z && r == cudaSuccess; };
    Z(cudaMemcpy(c->d_scenes, c->scenes.data(), S * sizeof(SceneDev), cudaMemcpyHostToDevice));
    if (!c->sdf_host.empty())
        Z(cudaMemcpy(c->d_sdf, c->sdf_host.data(), c->sdf_host.size() * sizeof(gs_sdf), cudaMemcpyHostToDevice));
    if (N) Z(cudaMemcpy(c->lr_scene, lt.data(), N * sizeof(uint32_t), cudaMemcpyHostToDevice));
    if (MS) Z(cudaMemcpy(c->hr_scene, ht.data(), MS * sizeof(uint32_t), cudaMemcpyHostToDevice));
    Z(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    Z(cudaMemsetAsync(c->lr_pos, 0, std::max<int64_t>(N, 1) * sizeof(float4), c->stream));
    Z(cudaMemsetAsync(c->lr_vel, 0, std::max<int64_t>(N, 1) * sizeof(float4), c->stream));
    Z(cudaMemsetAsync(c->lr_mat, 0, std::max<int64_t>(N, 1) * sizeof(uint32_t), c->stream));
    Z(cudaMemsetAsync(c->lr_body, 0, std::max<int64_t>(N, 1) * sizeof(uint32_t), c->stream));
    Z(cudaMemsetAsync(c->d_cfl, 0, sizeof(CflState), c->stream));
    Z(cudaMemsetAsync(c->tmp4, 0, std::max<int64_t>(std::max(NM, MR), 1) * sizeof(float4), c->stream));
    Z(cudaMemsetAsync(c->lr_cell_start, 0, (cells + 2) * sizeof(uint32_t), c->stream));
    if (z) Z(launch_hr_load(c, c->tmp4, c->hr_pos[0], 1));
    if (z) Z(launch_hr_load(c, c->tmp4, c->hr_vel[0], 0));
    if (z) Z(cudaStreamSynchronize(c->stream));
    if (!z) {
        gs_destroy(c);
        return GS_ERR_CUDA;
    }
    *out = c;
    return GS_OK;
}

// The key buffer that holds the sorted HR keys after a reorder.
uint32_t* hr_sorted_after_resort(const gs_ctx* c)
{
    return c->hr_counting ? c->hr_keys[1] : c->hr_keys[((c->hr_key_bits + 7) / 8) & 1];   // where the radix passes end
}

int resort_high_impl(gs_ctx* c)
{
    const int64_t MS = c->hr_slots;
    if (MS == 0) return GS_OK;
    Timed t(c, GS_TIMER_RESORT);
    const int cur = c->hr_cur;
    int which = 0;
    if (c->hr_counting) {
        CK(gs_cs_clear(c->stream, c->hr_bin_start, c->hr_bins, 1), "clear counts");
        CK(gs_launch_scene_keys(c->stream, c->hr_pos[cur], MS, c->d_scenes, c->hr_scene, 1, c->hr_keys[0],
                                c->hr_vals[0], &c->launches, c->hr_bin_start),
           "keys");
        CsExtras ex;
        ex.big_list = c->hr_big;
        ex.big_count = c->hr_bin_start + c->hr_bins + 1;
        ex.big_scratch = c->hr_vals[0];   // the ranks are dead once scattered
        ex.big_bits = gs_key_bits(MS);
        ex.big_blocks = std::max(c->sm_count, 1);
        CK(gs_cs_finish(c->stream, MS, c->hr_bins, c->hr_keys[0], c->hr_vals[0], c->hr_keys[1], c->hr_vals[1],
                        c->hr_bin_start, c->hr_scan_aux, nullptr, nullptr, nullptr, nullptr, &c->launches, ex),
           "counting sort");
        which = 1;
    } else {
        CK(gs_launch_scene_keys(c->stream, c->hr_pos[cur], MS, c->d_scenes, c->hr_scene, 1, c->hr_keys[0],
                                c->hr_vals[0], &c->launches),
           "keys");
        CK(gs_radix_sort(c->stream, c->hr_keys, c->hr_vals, &which, c->sort_hist, MS, c->hr_key_bits, &c->launches),
           "radix sort");
    }
    CK(gs_launch_gather2(c->stream, c->hr_vals[which], c->hr_pos[cur], c->hr_vel[cur], c->hr_pos[cur ^ 1],
                         c->hr_vel[cur ^ 1], MS, &c->launches),
       "permute");
    c->hr_sorted_keys = c->hr_keys[which];
    c->hr_keys_valid = true;
    c->hr_cur = cur ^ 1;
    c->hr_identity = false;
    return GS_OK;
}

int bin_low_impl(gs_ctx* c)
{
    Timed t(c, GS_TIMER_BIN_LOW);
    // counting sort by cell; its last stage copies pos and vel into cell order
    // the word after the cell starts flags LR particles of infinite mass or
    // of rigid bodies for the gather (the binning reads every position
    // anyway); body particles enter the gather's view with w = 0
    const uint32_t* body = c->n_bodies > 0 ? c->lr_body : nullptr;
    CK(gs_cs_clear(c->stream, c->lr_cell_start, c->n_cell_total, 1), "clear counts");
    CK(gs_cs_keys(c->stream, c->lr_pos, c->n_low, c->d_scenes, c->lr_scene, c->lr_keys[0], c->lr_vals[0],
                  c->lr_cell_start, &c->launches, c->lr_cell_start + c->n_cell_total + 1, body),
       "cell keys");
    CsExtras ex;
    ex.ga_solid = body;
    CK(gs_cs_finish(c->stream, c->n_low, c->n_cell_total, c->lr_keys[0], c->lr_vals[0], c->lr_keys[1], c->lr_vals[1],
                    c->lr_cell_start, c->scan_aux, c->lr_pos, c->lr_vel, c->lr_spos, c->lr_svel, &c->launches, ex),
       "bin by cell");
    c->lr_sorted_keys = c->lr_keys[1];
    c->lr_sorted_idx = c->lr_vals[1];
    c->lr_binned = true;
    return GS_OK;
}

UpsampleArgs upsample_args(const gs_ctx* c, float dt, const float4* in_pos, const float4* in_vel, float4* out_pos,
                           float4* out_vel)
{
    UpsampleArgs u;
    u.hr_pos = in_pos;
    u.hr_vel = in_vel;
    u.out_pos = out_pos;
    u.out_vel = out_vel;
    u.lr_spos = c->lr_spos;
    u.lr_svel = c->lr_svel;
    u.cell_start = c->lr_cell_start;
    u.scenes = c->d_scenes;
    u.hr_tag = c->hr_scene;
    u.sdf = c->d_sdf;
    u.n_scenes = c->n_scenes;
    u.n_warps = c->n_warps;
    u.item_begin = 0;
    u.work = c->d_work;
    u.solid_flag = c->lr_cell_start + c->n_cell_total + 1;
    u.dt = dt;
    return u;
}

// Records gather timer event k on the main stream: inside a stream capture
// as an event record node of the graph, so that every replay records it.
cudaError_t record_gather_event(gs_ctx* c, int k)
{
    if (!c->ev_gather[k]) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags(c->ev_gather[k], c->stream,
                                    cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u);
}

// The HR frame: reorder when due, bin LR, gather in place.
int upsample_impl(gs_ctx* c, float dt)
{
    int st;
    if (c->n_high == 0) {
        c->frame++;
        return GS_OK;
    }
    if (c->resort_every > 0 && c->frame % c->resort_every == 0) {
        st = resort_high_impl(c);
        if (st) return st;
    }
    st = bin_low_impl(c);
    if (st) return st;
    const int cur = c->hr_cur;
    UpsampleArgs u = upsample_args(c, dt, c->hr_pos[cur], c->hr_vel[cur], c->hr_pos[cur], c->hr_vel[cur]);
    if (c->slab_parts > 1) {   // this context's slab of the HR slots only
        u.item_begin = c->slab_item_begin;
        u.n_warps = c->slab_item_end - c->slab_item_begin;
    }
    {
        Timed t(c, GS_TIMER_GATHER);
        CK(record_gather_event(c, 0), "gather timer");
        CK(gs_launch_upsample(c->stream, u, c->tune_warps, c->tune_blocks_per_sm, c->sm_count, &c->launches),
           "upsample");
        CK(record_gather_event(c, 1), "gather timer");
    }
    c->frame++;
    return GS_OK;
}

// dt_dev (adaptive frames): the step length is read from device memory
// instead of dt; rate: the finalize's atomic max of |v| / (2 r_LR).
int step_low_impl(gs_ctx* c, float dt, int iters, const float* dt_dev = nullptr, unsigned* rate = nullptr)
{
    const int64_t N = c->n_low;
    if (N == 0) return GS_OK;
    Timed t(c, GS_TIMER_STEP_LOW);
    PbdArgs a = pbd_args(c, dt);
    a.dt_dev = dt_dev;
    // prediction fused with the counting stage of the binning of x~; the
    // binning's last stage copies x~ and x into cell order
    CK(gs_cs_clear(c->stream, c->step_cell_start, c->n_cell_total), "clear counts");
    CK(gs_launch_predict_keys(c->stream, a, c->lr_pos, c->lr_vel, c->lr_xt, c->lr_keys[0], c->lr_vals[0],
                              c->step_cell_start, &c->launches),
       "predict");
    CK(gs_cs_finish(c->stream, N, c->n_cell_total, c->lr_keys[0], c->lr_vals[0], c->lr_keys[1], c->lr_vals[1],
                    c->step_cell_start, c->scan_aux, c->lr_xt, c->lr_pos, c->s_xt[0], c->s_x[0], &c->launches,
                    step_extras(c, a)),
       "bin by cell");
    c->lr_sorted_keys = c->lr_keys[1];
    c->lr_sorted_idx = c->lr_vals[1];
    CK(gs_launch_neighbors(c->stream, a, c->s_xt[0], c->lr_sorted_keys, c->step_cell_start, c->n_cell_total, c->nbr, c->nbr_cnt,
                           c->nbr_cap, c->d_err, &c->launches),
       "neighbours");
    int bx = 0, bt = 0;   // buffers holding the current x and xt
    if (c->use_solver && c->solve_blocks > 0 && c->n_bodies == 0) {
        // all passes in one cooperative launch; the buffers alternate as in
        // the loop below
        CK(gs_launch_solve(c->stream, a, c->n_stab, iters, c->s_x, c->s_xt, c->nbr, c->nbr_cnt, c->d_bar, c->d_err,
                           c->solve_blocks, &c->launches, c->solver_selftest ? 1u : 0u),
           "solver");
        bt = (c->n_stab + iters) & 1;
        bx = c->n_stab & 1;
    } else {
        // the last pass also finalizes (v = (x~ - x) / dt, x = x~, original order)
        const int total = c->n_stab + iters;
        for (int it = 0; it < total; ++it) {
            const int stab = it < c->n_stab;
            const bool last = it + 1 == total;
            if (c->n_bodies > 0 && !stab)   // the bodies' transforms from this pass's x~
                CK(gs_launch_body_xform(c->stream, c->n_bodies, c->body_start, c->body_members, c->lr_slot,
                                        c->s_xt[bt], c->lr_xo, c->body_xf, &c->launches),
                   "body transforms");
            CK(gs_launch_pass(c->stream, a, stab, c->s_x[bx], c->s_xt[bt], c->s_x[bx ^ 1], c->s_xt[bt ^ 1], c->nbr,
                              c->nbr_cnt, &c->launches, last ? c->lr_sorted_idx : nullptr,
                              last ? c->lr_pos : nullptr, last ? c->lr_vel : nullptr, last ? rate : nullptr),
               "pass");
            bt ^= 1;
            if (stab) bx ^= 1;
        }
        if (total > 0) {
            c->lr_binned = false;   // the binning above is of the predicted positions
            return GS_OK;
        }
    }
    CK(gs_launch_finalize(c->stream, a, c->lr_sorted_idx, c->s_x[bx], c->s_xt[bt], c->lr_pos, c->lr_vel,
                          &c->launches, rate),
       "finalize");
    c->lr_binned = false;   // the binning above is of the predicted positions
    return GS_OK;
}

// HR frames of a context restricted to a slab: a reorder reads the whole
// HR state, so it must not come while slots outside the slab are stale.
int slab_frame_begin(gs_ctx* c)
{
    if (c->hr_partial && c->n_high > 0 && c->resort_every > 0 && c->frame % c->resort_every == 0)
        return fail(c, GS_ERR_STATE, "an HR reorder is due and the slots outside this context's slab are stale: "
                                     "assemble the HR state (gs_hr_slab_assemble) first");
    return GS_OK;
}

void slab_frame_end(gs_ctx* c)
{
    if (c->slab_parts > 1 && c->n_high > 0) c->hr_partial = true;
}

int slab_refuse_hr_field(gs_ctx* c, int field)
{
    if (c->hr_partial && (field == GS_FIELD_HR_POS || field == GS_FIELD_HR_VEL))
        return fail(c, GS_ERR_STATE, "field %d needs the whole HR state, and the slots outside this context's slab "
                                     "are stale (gs_hr_slab_assemble)", field);
    return GS_OK;
}

void drop_graphs(gs_ctx* c)
{
    for (auto& g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    c->graphs.clear();
    for (auto& g : c->fgraphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    c->fgraphs.clear();
}

// The functional LR step entry points copy the caller's buffers in and out
// around a fixed sequence on the context's own buffers; with graphs enabled
// (and a stream that can be captured: not the legacy or per-thread default
// stream) that sequence is captured once per key and replayed.
bool capturable(const gs_ctx* c)
{
    return c->use_graphs && !c->timing && !c->capturing && c->stream != nullptr && c->stream != cudaStreamLegacy &&
           c->stream != cudaStreamPerThread;
}

HostAfter host_after(const gs_ctx* c)
{
    HostAfter h;
    h.hr_cur = c->hr_cur;
    h.hr_identity = c->hr_identity;
    h.hr_keys_valid = c->hr_keys_valid;
    h.lr_binned = c->lr_binned;
    h.hr_sorted_keys = c->hr_sorted_keys;
    h.lr_sorted_keys = c->lr_sorted_keys;
    h.lr_sorted_idx = c->lr_sorted_idx;
    return h;
}

void apply_after(gs_ctx* c, const HostAfter& h)
{
    c->hr_cur = h.hr_cur;
    c->hr_identity = h.hr_identity;
    c->hr_keys_valid = h.hr_keys_valid;
    c->lr_binned = h.lr_binned;
    c->hr_sorted_keys = h.hr_sorted_keys;
    c->lr_sorted_keys = h.lr_sorted_keys;
    c->lr_sorted_idx = h.lr_sorted_idx;
}

// The key must hold every host-side input the sequence depends on; the
// host-side state it leaves is recorded at capture and applied on replay.
template <class F>
int replay_or_run(gs_ctx* c, uint64_t key, F&& body)
{
    if (!capturable(c)) return body();
    GraphEntry* ge = nullptr;
    for (auto& g : c->fgraphs)
        if (g.key == key) ge = &g;
    if (!ge) {
        const int64_t l0 = c->launches;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        c->capturing = true;   // sequences called by the body are captured into this graph
        const int st = body();
        c->capturing = false;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (st != GS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        GraphEntry g;
        g.key = key;
        g.kernels = c->launches - l0;
        g.after = host_after(c);
        c->launches = l0;
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_fail(c, ei, "instantiate graph");
        c->fgraphs.push_back(g);
        ge = &c->fgraphs.back();
    }
    CK(cudaGraphLaunch(ge->exec, c->stream), "graph launch");
    c->launches += ge->kernels;
    apply_after(c, ge->after);
    return GS_OK;
}

uint64_t step_key(const gs_ctx* c, char kind, float dt, int iters)
{
    uint32_t db;
    std::memcpy(&db, &dt, 4);
    uint64_t k = 0xcbf29ce484222325ull;
    for (uint64_t v : {(uint64_t)kind, (uint64_t)db, (uint64_t)iters, (uint64_t)c->use_solver,
                       (uint64_t)c->solver_selftest, (uint64_t)(c->n_materials > 0), (uint64_t)(c->n_bodies > 0),
                       (uint64_t)c->hr_cur, (uint64_t)c->tune_warps, (uint64_t)c->tune_blocks_per_sm})
        k = (k ^ v) * 0x100000001b3ull;
    return k;
}

// ---- pipelined frames ------------------------------------------------------
// The HR frame of frame f depends only on the LR state at the end of frame f,
// and the LR steps of frame f + 1 only on that state too, so the HR frame is
// deferred: the next gs_frame runs it on stream_hr while its own LR steps run
// on the main stream (their binning uses step_cell_start, the gather reads
// the binned view lr_spos / lr_svel / lr_cell_start and the SDF table as of
// frame f).  Every call that reads or changes the HR state or the binned
// view completes a deferred frame first, in stream order, so results equal
// those of sequential frames bit for bit.

// Enqueues the deferred HR frame on stream s.
int run_pending_on(gs_ctx* c, cudaStream_t s, int warps, int blocks)
{
    cudaStream_t main_stream = c->stream;
    c->stream = s;
    c->pending = false;
    int st = GS_OK;
    if (c->pend_resort) st = resort_high_impl(c);
    if (st == GS_OK) {
        const int cur = c->hr_cur;
        UpsampleArgs u = upsample_args(c, c->pend_dt, c->hr_pos[cur], c->hr_vel[cur], c->hr_pos[cur], c->hr_vel[cur]);
        u.sdf = c->d_sdf_pend;
        cudaError_t e = gs_launch_upsample(c->stream, u, warps, blocks, c->sm_count, &c->launches);
        if (e != cudaSuccess) st = cuda_fail(c, e, "upsample (deferred frame)");
    }
    c->stream = main_stream;
    return st;
}

int flush_pending(gs_ctx* c)
{
    if (!c->pending) return GS_OK;
    return run_pending_on(c, c->stream, c->tune_warps, c->tune_blocks_per_sm);
}

// One pipelined frame: [deferred HR frame on stream_hr] || [n_sub LR steps],
// join, then bin the new LR state and defer this frame's HR part.
int frame_pipelined(gs_ctx* c, float dt, int n_sub, int iters)
{
    const float dts = n_sub > 0 ? dt / (float)n_sub : dt;
    const bool had = c->pending;
    int st;
    if (had) {
        CK(cudaEventRecord(c->ev_fork, c->stream), "fork");
        CK(cudaStreamWaitEvent(c->stream_hr, c->ev_fork, 0), "fork");
        st = run_pending_on(c, c->stream_hr, c->pipe_warps, c->pipe_blocks_per_sm);
        if (st) return st;
    }
    for (int k = 0; k < n_sub; ++k) {
        st = step_low_impl(c, dts, iters);
        if (st) return st;
    }
    if (had) {
        CK(cudaEventRecord(c->ev_join, c->stream_hr), "join");
        CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join");
    }
    if (c->n_high > 0) {
        st = bin_low_impl(c);
        if (st) return st;
        if (!c->sdf_host.empty())
            CK(cudaMemcpyAsync(c->d_sdf_pend, c->d_sdf, c->sdf_host.size() * sizeof(gs_sdf), cudaMemcpyDeviceToDevice,
                               c->stream),
               "SDF snapshot");
        c->pending = true;
        c->pend_dt = dt;
        c->pend_resort = c->resort_every > 0 && c->frame % c->resort_every == 0;
    }
    c->frame++;
    return GS_OK;
}

int frame_pipelined_graph(gs_ctx* c, float dt, int n_sub, int iters)
{
    // what the captured work depends on
    uint32_t dbits, pbits;
    std::memcpy(&dbits, &dt, 4);
    std::memcpy(&pbits, &c->pend_dt, 4);
    const bool had = c->pending;
    uint64_t key = 0x9e3779b97f4a7c15ull;
    auto mix = [&](uint64_t v) { key = (key ^ v) * 0x100000001b3ull; };
    mix(1);   // pipelined
    mix(dbits);
    mix((uint64_t)(n_sub & 0x3ff) | ((uint64_t)(iters & 0x3ff) << 10));
    mix((uint64_t)had | ((uint64_t)(had && c->pend_resort) << 1) | ((uint64_t)c->hr_cur << 2));
    mix(had ? pbits : 0u);
    mix((uint64_t)c->pipe_warps | ((uint64_t)c->pipe_blocks_per_sm << 8) | ((uint64_t)c->n_stab << 16));
    GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
        if (g.key == key && !g.graph) ge = &g;
    const int64_t frame0 = c->frame;
    const int cur0 = c->hr_cur;
    const bool ident0 = c->hr_identity, keys0 = c->hr_keys_valid, binned0 = c->lr_binned;
    const bool pend0 = c->pending, pres0 = c->pend_resort;
    const float pdt0 = c->pend_dt;
    uint32_t* skeys0 = c->hr_sorted_keys;
    if (!ge) {
        cudaGraph_t graph = nullptr;
        const int64_t launches0 = c->launches;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int st2 = frame_pipelined(c, dt, n_sub, iters);
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (st2 != GS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st2;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        GraphEntry g;
        g.key = key;
        g.kernels = c->launches - launches0;
        c->launches = launches0;
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(c, e, "instantiate graph");
        c->graphs.push_back(g);
        ge = &c->graphs.back();
        // the capture only recorded the frame: restore the host state, run it below
        c->frame = frame0;
        c->hr_cur = cur0;
        c->hr_identity = ident0;
        c->hr_keys_valid = keys0;
        c->lr_binned = binned0;
        c->pending = pend0;
        c->pend_resort = pres0;
        c->pend_dt = pdt0;
        c->hr_sorted_keys = skeys0;
    }
    CK(cudaGraphLaunch(ge->exec, c->stream), "graph launch");
    c->launches += ge->kernels;
    // host-side state as if the frame had been enqueued directly
    if (had && c->pend_resort) {
        c->hr_sorted_keys = hr_sorted_after_resort(c);
        c->hr_cur ^= 1;
        c->hr_identity = false;
        c->hr_keys_valid = true;
    }
    if (c->n_high > 0) {
        c->lr_binned = true;
        c->pending = true;
        c->pend_dt = dt;
        c->pend_resort = c->resort_every > 0 && c->frame % c->resort_every == 0;
    }
    c->frame = frame0 + 1;
    return GS_OK;
}

}  // namespace

int gs_replay_or_run(gs_ctx* c, uint64_t key, int (*body)(gs_ctx*, void*), void* arg)
{
    return replay_or_run(c, key, [&] { return body(c, arg); });
}

uint64_t gs_sequence_key(const gs_ctx* c, char kind, float dt, int iters)
{
    return step_key(c, kind, dt, iters);
}

// Writes a checked device copy of a state field (original order) into the
// context's state, on the main stream.
int apply_field(gs_ctx* c, int field, const float4* dsrc, size_t bytes)
{
    const cudaMemcpyKind kind = cudaMemcpyDeviceToDevice;
    const int cur = c->hr_cur;
    switch (field) {
    case GS_FIELD_LR_POS:
        CK(cudaMemcpyAsync(c->lr_pos, dsrc, bytes, kind, c->stream), "copy");
        c->lr_binned = false;
        break;
    case GS_FIELD_LR_VEL: CK(cudaMemcpyAsync(c->lr_vel, dsrc, bytes, kind, c->stream), "copy"); break;
    case GS_FIELD_HR_POS:
        if (!c->hr_identity) {
            // bring the velocities back to the identity slot order first
            CK(gs_launch_unpermute(c->stream, c->hr_pos[cur], c->hr_vel[cur], c->hr_scene, c->tmp4, c->hr_slots,
                                   c->n_high, c->d_err, &c->launches),
               "unpermute");
            CK(launch_hr_load(c, c->tmp4, c->hr_vel[cur], 0), "load");
        }
        CK(launch_hr_load(c, dsrc, c->hr_pos[cur], 1), "load");
        c->hr_identity = true;
        c->hr_keys_valid = false;
        break;
    case GS_FIELD_HR_VEL:
        if (c->hr_identity)
            CK(launch_hr_load(c, dsrc, c->hr_vel[cur], 0), "load");
        else
            CK(gs_launch_permute_in(c->stream, c->hr_pos[cur], dsrc, c->hr_scene, c->hr_vel[cur], c->hr_slots,
                                    c->n_high, c->d_err, &c->launches),
               "permute");
        break;
    }
    return GS_OK;
}

// Commits asynchronously written fields, in field order, on the main stream
// once their host -> device copies are done.  Each is checked for finite
// values on the device (an offending field sets GS_DEVERR_NONFINITE_ASYNC,
// reported by the next gs_sync or gs_read) and then applied.
int commit_async_writes(gs_ctx* c)
{
    // both fields of a kind staged (the usual round trip): one checked copy
    // or load for the pair
    for (int f = 0; f < 4; f += 2) {
        if (!(c->in_pending[f] && c->in_pending[f + 1])) continue;
        c->in_pending[f] = c->in_pending[f + 1] = false;
        CK(cudaStreamWaitEvent(c->stream, c->ev_in_ready[f], 0), "wait for a staged field");
        CK(cudaStreamWaitEvent(c->stream, c->ev_in_ready[f + 1], 0), "wait for a staged field");
        if (f == 0 && c->n_low > 0) {
            k_copy2_checked<<<gs_blocks(c->n_low, 256), 256, 0, c->stream>>>(
                c->async_in[0], c->async_in[1], c->lr_pos, c->lr_vel, c->n_low, c->d_err, GS_DEVERR_NONFINITE_ASYNC);
            c->launches += 1;
            CK(cudaGetLastError(), "apply");
            c->lr_binned = false;
        } else if (f == 2 && c->hr_slots > 0) {
            const int cur = c->hr_cur;
            k_hr_load2_checked<<<gs_blocks(c->hr_slots, 256), 256, 0, c->stream>>>(
                c->async_in[2], c->async_in[3], c->hr_pos[cur], c->hr_vel[cur], c->hr_scene, c->d_scenes, c->hr_slots,
                c->d_err, GS_DEVERR_NONFINITE_ASYNC);
            c->launches += 1;
            CK(cudaGetLastError(), "apply");
            c->hr_identity = true;
            c->hr_keys_valid = false;
        }
        CK(cudaEventRecord(c->ev_in_free[f], c->stream), "record");
        CK(cudaEventRecord(c->ev_in_free[f + 1], c->stream), "record");
    }
    for (int f = 0; f < 4; ++f) {
        if (!c->in_pending[f]) continue;
        c->in_pending[f] = false;
        CK(cudaStreamWaitEvent(c->stream, c->ev_in_ready[f], 0), "wait for a staged field");
        const int64_t n = f < 2 ? c->n_low : c->n_high;
        CK(gs_launch_check_finite(c->stream, c->async_in[f], n, c->d_err, &c->launches, GS_DEVERR_NONFINITE_ASYNC),
           "finite check");
        int st = apply_field(c, f, c->async_in[f], field_bytes(c, f));
        if (st) return st;
        CK(cudaEventRecord(c->ev_in_free[f], c->stream), "record");
    }
    return GS_OK;
}

// Everything a call that reads or changes the state must see first: the
// deferred HR frame of a pipelined frame (it reads the state as of its
// frame), then the asynchronously written fields.
int settle(gs_ctx* c)
{
    int st = flush_pending(c);
    if (st) return st;
    return commit_async_writes(c);
}

int async_buffer(gs_ctx* c, float4** buf, int field)
{
    if (*buf) return GS_OK;
    const int64_t n = field < 2 ? c->n_low : c->n_high;
    if (dalloc(buf, (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GS_ERR_OOM, "no memory for an asynchronous transfer buffer");
    }
    return GS_OK;
}

extern "C" {

void gs_default_params(gs_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->gravity[0] = 0.0f;
    p->gravity[1] = 0.0f;
    p->gravity[2] = -9.81f;
    p->mu_s = 0.35f;
    p->mu_k = 0.30f;
    p->c1 = 512.0f / 729.0f;
    p->c2 = 0.6f;
    p->n_stab = 2;
    p->mass_scale_k = 1.0f;
    p->ground_z = NAN;          // resolved to box_lo z at create
    p->neighbor_radius = 0.0f;  // resolved to 3 r_low
    p->friction_mode = 0;
    p->resort_every = 8;
    p->max_neighbors = 0;       // resolved to 64
}

int gs_create(const gs_scene* scene, float r_low, float r_high, int ratio, void* cuda_stream, gs_ctx** out)
{
    if (!scene) {
        if (out) *out = nullptr;
        return GS_ERR_ARG;
    }
    return create_impl(1, scene, &r_low, &r_high, &ratio, cuda_stream, out);
}

int gs_batch_create(int n_scenes, const gs_scene* scenes, const float* r_low, const float* r_high, const int* ratio,
                    void* cuda_stream, gs_ctx** out)
{
    return create_impl(n_scenes, scenes, r_low, r_high, ratio, cuda_stream, out);
}

static void free_tapes(gs_ctx* c);

void gs_destroy(gs_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->stream_hr) cudaStreamSynchronize(c->stream_hr);
    if (c->stream_h2d) cudaStreamSynchronize(c->stream_h2d);
    if (c->stream_d2h) cudaStreamSynchronize(c->stream_d2h);
    drop_graphs(c);
    for (int t = 0; t < GS_TIMER_COUNT; ++t)
        for (auto& pr : c->ev[t]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    void* bufs[] = {c->d_scenes,   c->d_sdf,      c->lr_scene,   c->hr_scene,   c->lr_pos,    c->lr_vel,
                    c->lr_keys[0], c->lr_keys[1], c->lr_vals[0], c->lr_vals[1], c->lr_cell_start, c->lr_spos,
                    c->lr_svel,    c->lr_xt,      c->s_xt[0],    c->s_xt[1],    c->s_x[0],    c->s_x[1],
                    c->hr_pos[0],  c->hr_pos[1],  c->hr_vel[0],  c->hr_vel[1],  c->hr_keys[0], c->hr_keys[1],
                    c->hr_vals[0], c->hr_vals[1], c->nbr,        c->nbr_cnt,    c->tmp4,      c->sort_hist,
                    c->d_work,     c->d_err,      c->gXs,        c->gVs,       c->snap,      c->snap_xt,
                    c->adj_io,     c->fscratch,   c->adj_gx,     c->adj_gxt,    c->adj_h,      c->adj_h2,     c->adj_gws,   c->scan_aux,   c->d_bar,
                    c->step_cell_start, c->d_sdf_pend, c->stage_in, c->lr_mat, c->d_mu, c->d_cfl, c->lr_body, c->lr_xo, c->body_members,
                    c->body_start, c->body_xf, c->lr_slot, c->hr_bin_start, c->hr_big, c->hr_scan_aux,
                    c->async_in[0], c->async_in[1], c->async_in[2], c->async_in[3],
                    c->async_out[0], c->async_out[1], c->async_out[2], c->async_out[3], c->slab_stage};
    for (void* b : bufs)
        if (b) cudaFree(b);
    free_tapes(c);
    if (c->ro_ckpt) cudaFree(c->ro_ckpt);
    if (c->ro_work) cudaFree(c->ro_work);
    if (c->ro_io) cudaFree(c->ro_io);
    if (c->det_coef) cudaFree(c->det_coef);
    if (c->det_big) cudaFree(c->det_big);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->stream_hr) cudaStreamDestroy(c->stream_hr);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (cudaEvent_t e : c->ev_gather)
        if (e) cudaEventDestroy(e);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->stream_h2d) cudaStreamDestroy(c->stream_h2d);
    if (c->stream_d2h) cudaStreamDestroy(c->stream_d2h);
    for (int f = 0; f < 4; ++f)
        for (cudaEvent_t ev : {c->ev_in_ready[f], c->ev_in_free[f], c->ev_out_ready[f], c->ev_out_free[f]})
            if (ev) cudaEventDestroy(ev);
    delete c;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

int gs_info(const gs_ctx* c, int64_t* n_low, int64_t* n_high, gs_grid_info* grid)
{
    if (!c) return GS_ERR_ARG;
    if (n_low) *n_low = c->n_low;
    if (n_high) *n_high = c->n_high;
    if (grid) {
        const SceneDev& d = c->scenes[0];
        grid->origin[0] = d.g.ox;
        grid->origin[1] = d.g.oy;
        grid->origin[2] = d.g.oz;
        grid->h = d.g.h;
        grid->inv_h = d.g.inv_h;
        grid->dims[0] = d.g.dx;
        grid->dims[1] = d.g.dy;
        grid->dims[2] = d.g.dz;
        grid->n_cell = (int64_t)d.n_cell;
    }
    return GS_OK;
}

int gs_scene_info(const gs_ctx* c, int scene, gs_scene_layout* out)
{
    if (!c || !out || scene < 0 || scene >= c->n_scenes) return GS_ERR_ARG;
    const SceneDev& d = c->scenes[scene];
    out->lr_offset = d.lr_begin;
    out->n_low = d.lr_end - d.lr_begin;
    out->hr_offset = d.hr_real_begin;
    out->n_high = d.hr_end - d.hr_begin;
    out->hr_slot_offset = d.hr_begin;
    out->hr_slot_end = (scene + 1 < c->n_scenes) ? c->scenes[scene + 1].hr_begin : c->hr_slots;
    out->cell_offset = d.cell_off;
    out->grid.origin[0] = d.g.ox;
    out->grid.origin[1] = d.g.oy;
    out->grid.origin[2] = d.g.oz;
    out->grid.h = d.g.h;
    out->grid.inv_h = d.g.inv_h;
    out->grid.dims[0] = d.g.dx;
    out->grid.dims[1] = d.g.dy;
    out->grid.dims[2] = d.g.dz;
    out->grid.n_cell = (int64_t)d.n_cell;
    out->r_low = d.r_low;
    out->r_high = d.r_high;
    return GS_OK;
}

// The material field: ids checked against the table before anything of the
// state changes.
static int write_materials(gs_ctx* c, const void* src, size_t bytes, int src_is_device)
{
    if (bytes != field_bytes(c, GS_FIELD_LR_MATERIAL))
        return fail(c, GS_ERR_ARG, "size %zu does not match the material field", bytes);
    if (c->n_materials == 0) return fail(c, GS_ERR_STATE, "no material table (gs_set_materials)");
    const int64_t n = c->n_low;
    if (n == 0) return GS_OK;
    if (!src) return fail(c, GS_ERR_ARG, "null source");
    const uint32_t* dsrc = (const uint32_t*)src;
    if (!src_is_device) {
        CK(cudaMemcpyAsync(c->stage_in, src, bytes, cudaMemcpyHostToDevice, c->stream), "copy in");
        dsrc = (const uint32_t*)c->stage_in;
    }
    unsigned* word = (unsigned*)(c->d_err + 1);
    CK(cudaMemsetAsync(word, 0, sizeof(unsigned), c->stream), "clear word");
    k_max_id<<<gs_blocks(n, 256), 256, 0, c->stream>>>(dsrc, n, word);
    c->launches += 1;
    CK(cudaGetLastError(), "max id");
    CK(cudaMemcpyAsync(c->h_err, word, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "read word");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    const uint32_t max_id = (uint32_t)*c->h_err;
    if (max_id >= (uint32_t)c->n_materials)
        return fail(c, GS_ERR_ARG, "material id %u >= %d materials", max_id, c->n_materials);
    CK(cudaMemcpyAsync(c->lr_mat, dsrc, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy");
    c->mat_max_id = max_id;
    return GS_OK;
}

// The body field: ids, then every body's rest shape from the current LR
// positions (offsets from its centre of mass, masses 1 / w), in double on
// the host; the transforms start at R = I, c = the centre of mass.
static int write_bodies(gs_ctx* c, const void* src, size_t bytes, int src_is_device)
{
    if (bytes != field_bytes(c, GS_FIELD_LR_BODY))
        return fail(c, GS_ERR_ARG, "size %zu does not match the body field", bytes);
    const int64_t n = c->n_low;
    if (n == 0) return GS_OK;
    if (!src) return fail(c, GS_ERR_ARG, "null source");
    std::vector<uint32_t> ids((size_t)n);
    std::vector<float4> pos((size_t)n);
    CK(cudaMemcpyAsync(ids.data(), src, bytes, src_is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                       c->stream),
       "copy ids");
    CK(cudaMemcpyAsync(pos.data(), c->lr_pos, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream), "copy pos");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    int nb = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (ids[(size_t)i] > (uint32_t)GS_MAX_BODIES)
            return fail(c, GS_ERR_ARG, "body id %u above %d", ids[(size_t)i], GS_MAX_BODIES);
        if (ids[(size_t)i] != 0u && !(pos[(size_t)i].w > 0.0f))
            return fail(c, GS_ERR_ARG, "particle %lld of body %u has no finite mass", (long long)i, ids[(size_t)i]);
        nb = std::max(nb, (int)ids[(size_t)i]);
    }
    std::vector<double> M((size_t)nb + 1, 0.0), cx((size_t)nb + 1, 0.0), cy(cx), cz(cx);
    std::vector<uint32_t> count((size_t)nb + 1, 0u);
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = ids[(size_t)i];
        if (!b) continue;
        const double m = 1.0 / (double)pos[(size_t)i].w;
        M[b] += m;
        cx[b] += m * pos[(size_t)i].x;
        cy[b] += m * pos[(size_t)i].y;
        cz[b] += m * pos[(size_t)i].z;
        count[b] += 1u;
    }
    // start[b - 1] = first member of body b, start[b] one past its last
    std::vector<uint32_t> start((size_t)GS_MAX_BODIES + 1, 0u);
    for (int b = 1; b <= GS_MAX_BODIES; ++b) start[(size_t)b] = start[(size_t)b - 1] + (b <= nb ? count[(size_t)b] : 0u);
    const uint32_t run = start[(size_t)nb];
    std::vector<uint32_t> members(std::max<size_t>(run, 1)), fill(start.begin(), start.end());
    std::vector<float4> xo((size_t)n, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = ids[(size_t)i];
        if (!b) continue;
        members[fill[b - 1]++] = (uint32_t)i;
        const double m = 1.0 / (double)pos[(size_t)i].w;
        xo[(size_t)i] = make_float4((float)(pos[(size_t)i].x - cx[b] / M[b]), (float)(pos[(size_t)i].y - cy[b] / M[b]),
                                    (float)(pos[(size_t)i].z - cz[b] / M[b]), (float)m);
    }
    std::vector<float4> xf((size_t)4 * GS_MAX_BODIES, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int b = 1; b <= nb; ++b) {
        const double cc[3] = {M[b] > 0 ? cx[b] / M[b] : 0.0, M[b] > 0 ? cy[b] / M[b] : 0.0, M[b] > 0 ? cz[b] / M[b] : 0.0};
        for (int r = 0; r < 3; ++r)
            xf[(size_t)4 * (b - 1) + r] = make_float4(r == 0 ? 1.f : 0.f, r == 1 ? 1.f : 0.f, r == 2 ? 1.f : 0.f,
                                                      (float)cc[r]);
        xf[(size_t)4 * (b - 1) + 3] = make_float4(0.f, 0.f, 0.f, 1.f);
    }
    CK(cudaMemcpyAsync(c->lr_body, ids.data(), bytes, cudaMemcpyHostToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->lr_xo, xo.data(), n * sizeof(float4), cudaMemcpyHostToDevice, c->stream), "copy");
    if (run) CK(cudaMemcpyAsync(c->body_members, members.data(), run * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                c->stream),
                "copy");
    CK(cudaMemcpyAsync(c->body_start, start.data(), start.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                       c->stream),
       "copy");
    CK(cudaMemcpyAsync(c->body_xf, xf.data(), xf.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream),
       "copy");
    CK(cudaStreamSynchronize(c->stream), "synchronize");   // the host vectors go out of scope
    if ((nb > 0) != (c->n_bodies > 0)) drop_graphs(c);
    c->n_bodies = nb;
    return GS_OK;
}

int gs_set_materials(gs_ctx* c, int n_materials, const float* mu)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (n_materials < 0 || n_materials > GS_MAX_MATERIALS)
        return fail(c, GS_ERR_ARG, "material count %d outside 0..%d", n_materials, GS_MAX_MATERIALS);
    if (n_materials == 0) {
        if (c->n_low > 0) CK(cudaMemsetAsync(c->lr_mat, 0, c->n_low * sizeof(uint32_t), c->stream), "reset ids");
        c->mat_max_id = 0;
        if (c->n_materials != 0) drop_graphs(c);
        c->n_materials = 0;
        return GS_OK;
    }
    if (!mu) return fail(c, GS_ERR_ARG, "null coefficient table");
    for (int m = 0; m < 2 * n_materials; ++m)
        if (!(std::isfinite(mu[m]) && mu[m] >= 0.0f)) return fail(c, GS_ERR_ARG, "invalid coefficient %g", (double)mu[m]);
    if (c->mat_max_id >= (uint32_t)n_materials)
        return fail(c, GS_ERR_ARG, "material id %u in use, table of %d", c->mat_max_id, n_materials);
    // Sec. 3 cross coefficients mu_ij = sqrt(mu_i mu_j), static and kinetic,
    // rounded once from double; unused entries stay zero
    float2* h = c->h_mu;
    for (int k = 0; k < GS_MAX_MATERIALS * (GS_MAX_MATERIALS + 1); ++k) h[k] = make_float2(0.0f, 0.0f);
    for (int i = 0; i < n_materials; ++i) {
        h[i] = make_float2(mu[2 * i], mu[2 * i + 1]);
        for (int j = 0; j < n_materials; ++j)
            h[GS_MAX_MATERIALS + i * GS_MAX_MATERIALS + j] =
                make_float2((float)std::sqrt((double)mu[2 * i] * (double)mu[2 * j]),
                            (float)std::sqrt((double)mu[2 * i + 1] * (double)mu[2 * j + 1]));
    }
    CK(cudaMemcpyAsync(c->d_mu, h, sizeof(c->h_mu), cudaMemcpyHostToDevice, c->stream), "copy table");
    CK(cudaStreamSynchronize(c->stream), "synchronize");   // the host table is reused by the next call
    if (c->n_materials == 0) drop_graphs(c);   // the captured steps gather no materials
    c->n_materials = n_materials;
    return GS_OK;
}

int gs_write(gs_ctx* c, int field, const void* src, size_t bytes, int src_is_device)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (field == GS_FIELD_LR_MATERIAL) return write_materials(c, src, bytes, src_is_device);
    if (field == GS_FIELD_LR_BODY) return write_bodies(c, src, bytes, src_is_device);
    if (field != GS_FIELD_LR_POS && field != GS_FIELD_LR_VEL && field != GS_FIELD_HR_POS && field != GS_FIELD_HR_VEL)
        return fail(c, GS_ERR_ARG, "field %d is not writable", field);
    if (bytes != field_bytes(c, field)) return fail(c, GS_ERR_ARG, "size %zu does not match field %d", bytes, field);
    st = slab_refuse_hr_field(c, field);
    if (st) return st;
    if (bytes == 0) return GS_OK;
    if (!src) return fail(c, GS_ERR_ARG, "null source");
    // errors of earlier work first: the check below reuses the error word
    st = report_device_errors(c);
    if (st) return st;
    const int64_t n = (field == GS_FIELD_LR_POS || field == GS_FIELD_LR_VEL) ? c->n_low : c->n_high;
    // host data is staged on the device first; the finiteness check runs
    // there, before anything of the context's state changes
    const float4* dsrc = (const float4*)src;
    if (!src_is_device) {
        CK(cudaMemcpyAsync(c->stage_in, src, bytes, cudaMemcpyHostToDevice, c->stream), "copy in");
        dsrc = c->stage_in;
    }
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear flag");
    CK(gs_launch_check_finite(c->stream, dsrc, n, c->d_err, &c->launches), "finite check");
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
    CK(cudaStreamSynchronize(c->stream), "synchronize");   // the host source is consumed from here on
    if (*c->h_err) {
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear flag");
        return fail(c, GS_ERR_DOMAIN, "non-finite value in field %d", field);
    }
    return apply_field(c, field, dsrc, bytes);
}


int gs_read(gs_ctx* c, int field, void* dst, size_t bytes, int dst_is_device)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    size_t fb = field_bytes(c, field);
    if (fb == (size_t)-1) return fail(c, GS_ERR_ARG, "unknown field %d", field);
    if (bytes != fb) return fail(c, GS_ERR_ARG, "size %zu does not match field %d", bytes, field);
    if (bytes > 0 && !dst) return fail(c, GS_ERR_ARG, "null destination");
    st = slab_refuse_hr_field(c, field);
    if (st) return st;
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const int cur = c->hr_cur;
    const void* srcp = nullptr;
    switch (field) {
    case GS_FIELD_LR_POS: srcp = c->lr_pos; break;
    case GS_FIELD_LR_VEL: srcp = c->lr_vel; break;
    case GS_FIELD_LR_MATERIAL: srcp = c->lr_mat; break;
    case GS_FIELD_LR_BODY: srcp = c->lr_body; break;
    case GS_FIELD_HR_POS_INTERNAL: srcp = c->hr_pos[cur]; break;
    case GS_FIELD_HR_VEL_INTERNAL: srcp = c->hr_vel[cur]; break;
    case GS_FIELD_LR_CELL_START:
        if (!c->lr_binned) return fail(c, GS_ERR_STATE, "LR particles have not been binned");
        srcp = c->lr_cell_start;
        break;
    case GS_FIELD_LR_SORTED_INDEX:
        if (!c->lr_binned) return fail(c, GS_ERR_STATE, "LR particles have not been binned");
        srcp = c->lr_sorted_idx;
        break;
    case GS_FIELD_HR_SORTED_KEY:
        if (!c->hr_keys_valid) return fail(c, GS_ERR_STATE, "HR particles have not been reordered");
        srcp = c->hr_sorted_keys;
        break;
    case GS_FIELD_HR_POS:
    case GS_FIELD_HR_VEL: {
        const float4* f = field == GS_FIELD_HR_POS ? c->hr_pos[cur] : c->hr_vel[cur];
        float4* target = dst_is_device ? (float4*)dst : c->tmp4;
        CK(gs_launch_unpermute(c->stream, c->hr_pos[cur], f, c->hr_scene, target, c->hr_slots, c->n_high, c->d_err,
                               &c->launches),
           "unpermute");
        if (dst_is_device) return GS_OK;
        srcp = c->tmp4;
        break;
    }
    }
    if (bytes > 0) CK(cudaMemcpyAsync(dst, srcp, bytes, kind, c->stream), "copy");
    if (!dst_is_device) return report_device_errors(c);
    return GS_OK;
}

int gs_set_sdf(gs_ctx* c, int index, const gs_sdf* sdf)
{
    int st = check_state(c);
    if (st) return st;
    if (!sdf || index < 0 || index >= (int)c->sdf_host.size()) return fail(c, GS_ERR_ARG, "bad SDF index %d", index);
    c->sdf_host[index] = *sdf;
    CK(cudaMemcpyAsync(c->d_sdf + index, &c->sdf_host[index], sizeof(gs_sdf), cudaMemcpyHostToDevice, c->stream),
       "copy SDF");
    return GS_OK;
}

int gs_bin_low(gs_ctx* c)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    return bin_low_impl(c);
}

int gs_resort_high(gs_ctx* c)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (c->hr_partial)
        return fail(c, GS_ERR_STATE, "the slots outside this context's HR slab are stale (gs_hr_slab_assemble)");
    return resort_high_impl(c);
}

int gs_step_low(gs_ctx* c, float dt, int iters)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid dt %g or iters %d", (double)dt, iters);
    return step_low_impl(c, dt, iters);
}

int gs_upsample(gs_ctx* c, float dt)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(c, GS_ERR_ARG, "invalid dt %g", (double)dt);
    st = slab_frame_begin(c);
    if (st) return st;
    st = upsample_impl(c, dt);
    if (st == GS_OK) slab_frame_end(c);
    return st;
}

int gs_set_pipeline(gs_ctx* c, int enable, int warps_per_block, int blocks_per_sm)
{
    int st = check_state(c);
    if (st) return st;
    if ((warps_per_block != 4 && warps_per_block != 8 && warps_per_block != 16) || blocks_per_sm < 0 ||
        blocks_per_sm > 32)
        return fail(c, GS_ERR_ARG, "unsupported launch shape %d x %d", warps_per_block, blocks_per_sm);
    st = settle(c);
    if (st) return st;
    if (enable && c->slab_parts > 1)
        return fail(c, GS_ERR_STATE, "pipelined frames do not combine with an HR slab");
    c->pipeline = enable != 0;
    c->pipe_warps = warps_per_block;
    c->pipe_blocks_per_sm = blocks_per_sm;
    drop_graphs(c);
    return GS_OK;
}

// ---- CFL-limited LR substeps (gs_frame_adaptive) -------------------------
namespace {

// Frame prologue: reset the control block, then the rate of the current
// velocities.
int adaptive_begin(gs_ctx* c, float dt)
{
    CK(gs_launch_cfl_begin(c->stream, c->d_cfl, dt, &c->launches), "begin frame");
    const PbdArgs a = pbd_args(c, dt);
    CK(gs_launch_cfl_rate(c->stream, a, c->lr_vel, &c->d_cfl->rate, &c->launches), "rate");
    return GS_OK;
}

// One LR step: pick its length, then the step reading it, whose finalize
// accumulates the rate for the next pick.
int adaptive_step(gs_ctx* c, float dt_max, float cfl, int max_sub, int iters, cudaGraphConditionalHandle h,
                  int in_graph, unsigned body_kernels)
{
    CK(gs_launch_cfl_pick(c->stream, c->d_cfl, dt_max, cfl, max_sub, h, in_graph, body_kernels, &c->launches),
       "pick step");
    return step_low_impl(c, dt_max, iters, &c->d_cfl->dt, &c->d_cfl->rate);
}

// Captures one loop body into `body` (or, with body null, into a throwaway
// graph to count its launches); *kernels receives the count.
int capture_body(gs_ctx* c, cudaGraph_t body, float dt_max, float cfl, int max_sub, int iters,
                 cudaGraphConditionalHandle h, unsigned body_kernels, int64_t* kernels)
{
    const int64_t l0 = c->launches;
    cudaError_t e = body ? cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                                         cudaStreamCaptureModeThreadLocal)
                         : cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
    int st = adaptive_step(c, dt_max, cfl, max_sub, iters, h, 1, body_kernels);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    if (!body && g) cudaGraphDestroy(g);
    *kernels = c->launches - l0;
    c->launches = l0;
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    return GS_OK;
}

// The frame as one graph: prologue -> while (more) { pick; LR step } -> HR
// frame.  The while node's condition starts at 1 on every launch.
int build_adaptive_graph(gs_ctx* c, float dt, float dt_max, float cfl, int max_sub, int iters, GraphEntry* out)
{
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0), "create graph");
    const int64_t l0 = c->launches;
    int st = GS_OK;
    cudaError_t e = cudaSuccess;
    std::vector<cudaGraphNode_t> deps;
    cudaGraphNode_t wnode = nullptr;
    do {
        // 1. prologue, and the nodes the loop depends on
        e = cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        st = adaptive_begin(c, dt);
        if (st == GS_OK) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t* d = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, nullptr, &d, nullptr, &nd);
            if (e == cudaSuccess) deps.assign(d, d + nd);
        }
        cudaGraph_t gg = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c->stream, &gg);
        if (st != GS_OK || e != cudaSuccess) break;
        if ((e = e2) != cudaSuccess) break;
        // 2. the loop
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) break;
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // the rest zero
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, g, deps.data(), nullptr, deps.size(), &np);
        if (e != cudaSuccess) break;
        int64_t body_kernels = 0;
        st = capture_body(c, nullptr, dt_max, cfl, max_sub, iters, h, 0u, &body_kernels);
        if (st) break;
        st = capture_body(c, np.conditional.phGraph_out[0], dt_max, cfl, max_sub, iters, h, (unsigned)body_kernels,
                          &body_kernels);
        if (st) break;
        // 3. the HR frame after the loop
        e = cudaStreamBeginCaptureToGraph(c->stream, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        st = upsample_impl(c, dt);
        e = cudaStreamEndCapture(c->stream, &gg);
        if (st != GS_OK || e != cudaSuccess) break;
        e = cudaGraphInstantiate(&out->exec, g, 0);
    } while (false);
    out->kernels = c->launches - l0;   // prologue and HR frame; the loop's steps are credited on the device
    c->launches = l0;
    if (st != GS_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        out->exec = nullptr;
        return st != GS_OK ? st : cuda_fail(c, e, "adaptive frame graph");
    }
    out->graph = g;   // a graph with a conditional node stays with its single instantiation
    return GS_OK;
}

}  // namespace

// Adds the kernel launches of device-looped LR steps (counted by the step
// picker) to the context's launch count.  Blocks.
static int fold_cfl_launches(gs_ctx* c)
{
    if (!c->cfl_used) return GS_OK;
    unsigned long long k = 0;
    CK(cudaMemcpyAsync(&k, &c->d_cfl->kernels, sizeof(k), cudaMemcpyDeviceToHost, c->stream), "read count");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    c->launches += (int64_t)(k - c->cfl_kernels_seen);
    c->cfl_kernels_seen = k;
    return GS_OK;
}

static int frame_body(gs_ctx* c, float dt, int n_sub, int iters)
{
    int st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || n_sub < 0 || n_sub > 1000 || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid frame arguments");
    if (c->pipeline && !c->timing) {
        if (c->in_pending[0] || c->in_pending[1] || c->in_pending[2] || c->in_pending[3]) {
            st = settle(c);   // staged fields must see the deferred frame first
            if (st) return st;
        }
        if (c->use_graphs) return frame_pipelined_graph(c, dt, n_sub, iters);
        return frame_pipelined(c, dt, n_sub, iters);
    }
    st = settle(c);
    if (st) return st;
    const float dts = n_sub > 0 ? dt / (float)n_sub : dt;
    const bool resort = c->n_high > 0 && c->resort_every > 0 && c->frame % c->resort_every == 0;
    if (!c->use_graphs || c->timing) {
        for (int k = 0; k < n_sub; ++k) {
            st = step_low_impl(c, dts, iters);
            if (st) return st;
        }
        return upsample_impl(c, dt);
    }
    // one graph per (time step, substeps, iterations, reorder, buffer parity)
    uint32_t dbits;
    std::memcpy(&dbits, &dt, 4);
    const uint64_t key = ((uint64_t)dbits << 32) ^ ((uint64_t)(n_sub & 0x3ff) << 20) ^ ((uint64_t)(iters & 0x3ff) << 8) ^
                         ((uint64_t)resort << 1) ^ (uint64_t)c->hr_cur ^ ((uint64_t)c->tune_warps << 2) ^
                         ((uint64_t)c->tune_blocks_per_sm << 5);
    GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
        if (g.key == key && !g.graph) ge = &g;
    const int64_t frame0 = c->frame;
    const int cur0 = c->hr_cur;
    if (!ge) {
        cudaGraph_t graph = nullptr;
        const int64_t launches0 = c->launches;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int st2 = GS_OK;
        for (int k = 0; k < n_sub && st2 == GS_OK; ++k) st2 = step_low_impl(c, dts, iters);
        if (st2 == GS_OK) st2 = upsample_impl(c, dt);
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (st2 != GS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st2;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        GraphEntry g;
        g.key = key;
        g.kernels = c->launches - launches0;
        c->launches = launches0;
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(c, e, "instantiate graph");
        c->graphs.push_back(g);
        ge = &c->graphs.back();
        // the capture only recorded the frame; run it below
        c->frame = frame0;
        c->hr_cur = cur0;
    }
    CK(cudaGraphLaunch(ge->exec, c->stream), "graph launch");
    c->launches += ge->kernels;
    // host-side state as if the frame had been enqueued directly
    if (resort) {
        c->hr_cur ^= 1;
        c->hr_identity = false;
        c->hr_keys_valid = true;
    }
    c->lr_binned = c->n_high > 0;
    c->frame = frame0 + 1;
    return GS_OK;
}

static int frame_adaptive_body(gs_ctx* c, float dt, float dt_max, float cfl, int max_sub, int iters)
{
    int st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || !(dt_max > 0.0f) || !std::isfinite(dt_max) || !(cfl > 0.0f) ||
        !std::isfinite(cfl) || max_sub < 1 || max_sub > GS_MAX_SUBSTEPS || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid adaptive frame arguments");
    st = settle(c);   // a deferred pipelined HR frame and staged writes come first
    if (st) return st;
    c->cfl_used = true;
    if (!c->use_graphs || c->timing) {
        // host-driven: the same kernels, the host reads after every step
        // whether another follows
        st = adaptive_begin(c, dt);
        if (st) return st;
        for (int k = 0; k < max_sub; ++k) {
            st = adaptive_step(c, dt_max, cfl, max_sub, iters, cudaGraphConditionalHandle{}, 0, 0u);
            if (st) return st;
            CK(cudaMemcpyAsync(c->h_err, &c->d_cfl->more, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read");
            CK(cudaStreamSynchronize(c->stream), "synchronize");
            if (!*c->h_err) break;
        }
        return upsample_impl(c, dt);
    }
    const bool resort = c->n_high > 0 && c->resort_every > 0 && c->frame % c->resort_every == 0;
    uint32_t b[3];
    std::memcpy(&b[0], &dt, 4);
    std::memcpy(&b[1], &dt_max, 4);
    std::memcpy(&b[2], &cfl, 4);
    uint64_t key = 0xadadadad00000000ull;
    for (uint64_t v : {(uint64_t)b[0], (uint64_t)b[1], (uint64_t)b[2], (uint64_t)max_sub, (uint64_t)iters,
                       (uint64_t)resort, (uint64_t)c->hr_cur, (uint64_t)c->tune_warps,
                       (uint64_t)c->tune_blocks_per_sm})
        key = (key ^ v) * 0x100000001b3ull;
    GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
        if (g.key == key && g.graph) ge = &g;
    const int64_t frame0 = c->frame;
    const int cur0 = c->hr_cur;
    if (!ge) {
        GraphEntry g;
        g.key = key;
        st = build_adaptive_graph(c, dt, dt_max, cfl, max_sub, iters, &g);
        c->frame = frame0;   // the capture only recorded the frame
        c->hr_cur = cur0;
        if (st) return st;
        c->graphs.push_back(g);
        ge = &c->graphs.back();
    }
    CK(cudaGraphLaunch(ge->exec, c->stream), "graph launch");
    c->launches += ge->kernels;
    if (resort) {
        c->hr_cur ^= 1;
        c->hr_identity = false;
        c->hr_keys_valid = true;
    }
    c->lr_binned = c->n_high > 0;
    c->frame = frame0 + 1;
    return GS_OK;
}

int gs_frame(gs_ctx* c, float dt, int n_sub, int iters)
{
    int st = check_state(c);
    if (st) return st;
    st = slab_frame_begin(c);
    if (st) return st;
    st = frame_body(c, dt, n_sub, iters);
    if (st == GS_OK) slab_frame_end(c);
    return st;
}

int gs_frame_adaptive(gs_ctx* c, float dt, float dt_max, float cfl, int max_sub, int iters)
{
    int st = check_state(c);
    if (st) return st;
    st = slab_frame_begin(c);
    if (st) return st;
    st = frame_adaptive_body(c, dt, dt_max, cfl, max_sub, iters);
    if (st == GS_OK) slab_frame_end(c);
    return st;
}

int gs_hr_slab_range(int64_t n_slots, int part, int n_parts, int64_t* begin, int64_t* end)
{
    if (!begin || !end || n_parts < 1 || n_parts > 4096 || part < 0 || part >= n_parts || n_slots < 0 ||
        n_slots % 32 != 0)
        return GS_ERR_ARG;
    // whole 32-slot items, as even as possible (item counts differ by one at most)
    const int64_t items = n_slots / 32;
    *begin = items * part / n_parts * 32;
    *end = items * (part + 1) / n_parts * 32;
    return GS_OK;
}

int gs_set_hr_slab(gs_ctx* c, int part, int n_parts)
{
    int st = check_state(c);
    if (st) return st;
    int64_t b = 0, e = 0;
    if (gs_hr_slab_range(c->hr_slots, part, n_parts, &b, &e) != GS_OK)
        return fail(c, GS_ERR_ARG, "bad HR slab %d of %d", part, n_parts);
    st = settle(c);
    if (st) return st;
    if (c->pipeline) return fail(c, GS_ERR_STATE, "an HR slab does not combine with pipelined frames");
    if (c->hr_partial)
        return fail(c, GS_ERR_STATE, "the slots outside the current HR slab are stale; assemble them first");
    c->slab_parts = n_parts;
    c->slab_item_begin = b / 32;
    c->slab_item_end = e / 32;
    drop_graphs(c);   // the captured gathers cover the old range
    return GS_OK;
}

int gs_hr_slab_assemble(gs_ctx* c, const void* pos, const void* vel, size_t bytes, int src_is_device)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (bytes != (size_t)c->hr_slots * sizeof(float4))
        return fail(c, GS_ERR_ARG, "size %zu does not match the HR slots (%lld x 16 bytes)", bytes,
                    (long long)c->hr_slots);
    if (bytes == 0) {
        c->hr_partial = false;
        return GS_OK;
    }
    if (!pos || !vel) return fail(c, GS_ERR_ARG, "null source");
    st = report_device_errors(c);   // the check below reuses the error word
    if (st) return st;
    const float4* dp = (const float4*)pos;
    const float4* dv = (const float4*)vel;
    if (!src_is_device) {
        if (!c->slab_stage && dalloc(&c->slab_stage, (size_t)2 * c->hr_slots) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, GS_ERR_OOM, "no memory to stage the assembled HR state");
        }
        CK(cudaMemcpyAsync(c->slab_stage, pos, bytes, cudaMemcpyHostToDevice, c->stream), "copy in");
        CK(cudaMemcpyAsync(c->slab_stage + c->hr_slots, vel, bytes, cudaMemcpyHostToDevice, c->stream), "copy in");
        dp = c->slab_stage;
        dv = c->slab_stage + c->hr_slots;
    }
    const int cur = c->hr_cur;
    k_slab_check<<<gs_blocks(c->hr_slots, 256), 256, 0, c->stream>>>(dp, dv, c->hr_pos[cur], c->hr_slots, c->d_err);
    c->launches += 1;
    CK(cudaGetLastError(), "check");
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
    CK(cudaStreamSynchronize(c->stream), "synchronize");   // the sources are consumed from here on
    const int bad = *c->h_err;
    if (bad) {
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear flag");
        return fail(c, GS_ERR_ARG, (bad & 2) ? "the assembled HR positions' ids differ from this context's slot order"
                                             : "non-finite value in the assembled HR state");
    }
    CK(cudaMemcpyAsync(c->hr_pos[cur], dp, bytes, cudaMemcpyDeviceToDevice, c->stream), "apply");
    CK(cudaMemcpyAsync(c->hr_vel[cur], dv, bytes, cudaMemcpyDeviceToDevice, c->stream), "apply");
    CK(cudaStreamSynchronize(c->stream), "synchronize");   // device sources too are consumed on return
    c->hr_partial = false;
    c->hr_pair_field = -1;
    return GS_OK;
}

int gs_substeps(gs_ctx* c, float* dts, int cap, int* n_out)
{
    int st = check_state(c);
    if (st) return st;
    if (!n_out || cap < 0 || (cap > 0 && !dts)) return fail(c, GS_ERR_ARG, "invalid substep buffer");
    st = settle(c);
    if (st) return st;
    CflState h;
    CK(cudaMemcpyAsync(&h, c->d_cfl, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "read substeps");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    st = fold_cfl_launches(c);
    if (st) return st;
    const int n = std::min(std::max(h.taken, 0), GS_MAX_SUBSTEPS);
    *n_out = n;
    for (int k = 0; k < std::min(n, cap); ++k) dts[k] = h.log[k];
    return GS_OK;
}

int gs_set_graphs(gs_ctx* c, int enable)
{
    int st = check_state(c);
    if (st) return st;
    c->use_graphs = enable != 0;
    if (!c->use_graphs) drop_graphs(c);
    return GS_OK;
}

int gs_set_lr_solver(gs_ctx* c, int persistent)
{
    int st = check_state(c);
    if (st) return st;
    if (persistent < 0 || persistent > 2) return fail(c, GS_ERR_ARG, "unknown solver mode %d", persistent);
    if (persistent && c->solve_blocks <= 0)
        return fail(c, GS_ERR_STATE, "the device does not support cooperative launches");
    c->use_solver = persistent != 0;
    c->solver_selftest = persistent == 2;
    drop_graphs(c);
    return GS_OK;
}

int gs_set_deterministic_backward(gs_ctx* c, int enable)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    c->det_bwd = enable != 0;
    drop_graphs(c);
    return GS_OK;
}

int gs_set_gather_timer(gs_ctx* c, int enable)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    drop_graphs(c);   // captured frames hold the event nodes (or lack them)
    for (auto& e : c->ev_gather)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (enable)
        for (auto& e : c->ev_gather) CK(cudaEventCreate(&e), "create timer event");
    return GS_OK;
}

int gs_gather_timer_ms(gs_ctx* c, float* ms)
{
    int st = check_state(c);
    if (st) return st;
    if (!ms) return fail(c, GS_ERR_ARG, "null output");
    if (!c->ev_gather[0]) return fail(c, GS_ERR_STATE, "the gather timer is off");
    st = settle(c);
    if (st) return st;
    CK(cudaEventSynchronize(c->ev_gather[1]), "synchronize");
    CK(cudaEventElapsedTime(ms, c->ev_gather[0], c->ev_gather[1]), "elapsed time");
    return GS_OK;
}

int gs_set_tuning(gs_ctx* c, int warps_per_block, int blocks_per_sm)
{
    int st = check_state(c);
    if (st) return st;
    if ((warps_per_block != 4 && warps_per_block != 8 && warps_per_block != 16) || blocks_per_sm < 0 ||
        blocks_per_sm > 32)
        return fail(c, GS_ERR_ARG, "unsupported launch shape %d x %d", warps_per_block, blocks_per_sm);
    c->tune_warps = warps_per_block;
    c->tune_blocks_per_sm = blocks_per_sm;
    drop_graphs(c);
    return GS_OK;
}

int gs_autotune(gs_ctx* c, float dt, int reps, int* warps_per_block, int* blocks_per_sm, float* best_us)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || reps < 1 || reps > 1000) return fail(c, GS_ERR_ARG, "invalid autotune arguments");
    if (c->n_high == 0) return fail(c, GS_ERR_STATE, "no HR particles");
    st = bin_low_impl(c);
    if (st) return st;
    // candidate shapes, timed on the current state written out of place
    // (the state is left unchanged)
    const int shapes[][2] = {{8, 0}, {4, 0}, {16, 0}, {8, 1}, {8, 2}, {8, 3}, {8, 4}, {4, 4},
                             {4, 8}, {16, 1}, {16, 2}};
    const int cur = c->hr_cur;
    UpsampleArgs u = upsample_args(c, dt, c->hr_pos[cur], c->hr_vel[cur], c->hr_pos[cur ^ 1], c->hr_vel[cur ^ 1]);
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a), "event");
    CK(cudaEventCreate(&b), "event");
    float best = 3.0e38f;
    int bw = c->tune_warps, bb = c->tune_blocks_per_sm;
    for (const auto& sh : shapes) {
        CK(gs_launch_upsample(c->stream, u, sh[0], sh[1], c->sm_count, &c->launches), "warm-up");
        CK(cudaEventRecord(a, c->stream), "event");
        for (int r = 0; r < reps; ++r) CK(gs_launch_upsample(c->stream, u, sh[0], sh[1], c->sm_count, &c->launches), "tune");
        CK(cudaEventRecord(b, c->stream), "event");
        CK(cudaEventSynchronize(b), "event");
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, a, b), "event");
        const float us = 1000.0f * ms / (float)reps;
        if (us < best) {
            best = us;
            bw = sh[0];
            bb = sh[1];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->tune_warps = bw;
    c->tune_blocks_per_sm = bb;
    drop_graphs(c);
    if (warps_per_block) *warps_per_block = bw;
    if (blocks_per_sm) *blocks_per_sm = bb;
    if (best_us) *best_us = best;
    return GS_OK;
}

// The functional upsampling entries' copies of the caller's HR buffers
// (6 x n_high) and LR gradients (2 x n_low), allocated on first use.
static int ensure_fscratch(gs_ctx* c)
{
    if (c->fscratch) return GS_OK;
    if (dalloc(&c->fscratch, (size_t)(6 * c->n_high + 2 * c->n_low)) != cudaSuccess ||
        dalloc(&c->det_coef, (size_t)(3 * c->n_high)) != cudaSuccess ||
        dalloc(&c->det_big, (size_t)(c->n_high / 33 + 2)) != cudaSuccess) {
        cudaGetLastError();
        if (c->fscratch) cudaFree(c->fscratch);
        c->fscratch = nullptr;
        return fail(c, GS_ERR_OOM, "no memory for the functional frame's buffers");
    }
    return GS_OK;
}

// The HR frame on copies: HR state in from fscratch[0..2), out to
// fscratch[2..4) (original order); the internal order is reset and sorted.
static int upsample_fwd_seq(gs_ctx* c, float dt)
{
    const int64_t M = c->n_high;
    float4* F = c->fscratch;
    int cur = c->hr_cur;
    CK(launch_hr_load(c, F, c->hr_pos[cur], 1), "load");
    CK(launch_hr_load(c, F + M, c->hr_vel[cur], 0), "load");
    c->hr_identity = true;
    int st = resort_high_impl(c);
    if (st) return st;
    st = bin_low_impl(c);
    if (st) return st;
    cur = c->hr_cur;
    UpsampleArgs u = upsample_args(c, dt, c->hr_pos[cur], c->hr_vel[cur], c->hr_pos[cur], c->hr_vel[cur]);
    CK(gs_launch_upsample(c->stream, u, c->tune_warps, c->tune_blocks_per_sm, c->sm_count, &c->launches), "upsample");
    CK(gs_launch_unpermute2(c->stream, c->hr_pos[cur], c->hr_vel[cur], c->hr_scene, F + 2 * M, F + 3 * M,
                            c->hr_slots, M, c->d_err, &c->launches),
       "unpermute");
    return GS_OK;
}

int gs_upsample_forward(gs_ctx* c, const float* lr_pos, const float* lr_vel, const float* hr_pos_in,
                        const float* hr_vel_in, float* hr_pos_out, float* hr_vel_out, float dt)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (c->n_scenes != 1) return fail(c, GS_ERR_STATE, "the functional frame needs a single-scene context");
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(c, GS_ERR_ARG, "invalid dt %g", (double)dt);
    const int64_t N = c->n_low, M = c->n_high;
    if ((N > 0 && (!lr_pos || !lr_vel)) || (M > 0 && (!hr_pos_in || !hr_vel_in || !hr_pos_out || !hr_vel_out)))
        return fail(c, GS_ERR_ARG, "null buffer");
    if (N) {
        CK(cudaMemcpyAsync(c->lr_pos, lr_pos, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
        CK(cudaMemcpyAsync(c->lr_vel, lr_vel, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    }
    c->lr_binned = false;
    if (M == 0) return GS_OK;
    st = ensure_fscratch(c);
    if (st) return st;
    float4* F = c->fscratch;
    CK(cudaMemcpyAsync(F, hr_pos_in, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(F + M, hr_vel_in, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    st = replay_or_run(c, step_key(c, 'u', dt, 0), [&] { return upsample_fwd_seq(c, dt); });
    if (st) return st;
    CK(cudaMemcpyAsync(hr_pos_out, F + 2 * M, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(hr_vel_out, F + 3 * M, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    return GS_OK;
}

// The reverse modes differentiate grains only: LR positions (device memory,
// n of them) holding particles of infinite mass raise a device error bit,
// reported as GS_ERR_STATE by the next blocking call (no wait here).
static int flag_solid(gs_ctx* c, const float* pos, int64_t n)
{
    if (n <= 0) return GS_OK;
    k_flag_solid<<<gs_blocks(n, 256), 256, 0, c->stream>>>((const float4*)pos, n, c->d_err,
                                                            GS_DEVERR_SOLID_REVERSE);
    c->launches += 1;
    CK(cudaGetLastError(), "flag");
    return GS_OK;
}

// The reverse HR frame on copies: HR state and dL/d outputs in from
// fscratch[0..4), dL/d HR inputs out to fscratch[4..6), dL/d LR inputs out
// to the two n_low blocks after them (original order).
static int upsample_bwd_seq(gs_ctx* c, float dt)
{
    const int64_t N = c->n_low, M = c->n_high;
    float4* F = c->fscratch;
    float4* G = F + 6 * M;
    int st = flag_solid(c, (const float*)c->lr_pos, N);
    if (st) return st;
    if (N && !c->det_bwd) {
        CK(cudaMemsetAsync(c->gXs, 0, N * sizeof(float4), c->stream), "clear");
        CK(cudaMemsetAsync(c->gVs, 0, N * sizeof(float4), c->stream), "clear");
    }
    st = bin_low_impl(c);
    if (st) return st;
    if (c->det_bwd) {   // HR binned by the LR cells, for the LR side's gather
        // (its cells hold dozens of HR particles: ordered over the whole grid
        // from a list, as the HR reorder's fine cells of more than 32)
        uint32_t* big_count = c->det_big + M / 33 + 1;
        CK(gs_cs_clear(c->stream, c->step_cell_start, c->n_cell_total), "clear counts");
        CK(cudaMemsetAsync(big_count, 0, sizeof(uint32_t), c->stream), "clear list");
        CK(gs_cs_keys(c->stream, F, M, c->d_scenes, c->hr_scene, c->hr_keys[0], c->hr_vals[0], c->step_cell_start,
                      &c->launches),
           "HR cell keys");
        CsExtras ex;
        ex.big_list = c->det_big;
        ex.big_count = big_count;
        ex.big_scratch = c->hr_vals[0];   // the ranks are dead once scattered
        ex.big_bits = gs_key_bits(M);
        ex.big_blocks = std::max(c->sm_count, 1);
        CK(gs_cs_finish(c->stream, M, c->n_cell_total, c->hr_keys[0], c->hr_vals[0], c->hr_keys[1], c->hr_vals[1],
                        c->step_cell_start, c->scan_aux, nullptr, nullptr, nullptr, nullptr, &c->launches, ex),
           "bin HR by LR cell");
    }
    CK(gs_launch_upsample_bwd(c->stream, c->d_scenes, c->d_sdf, c->lr_spos, c->lr_svel, c->lr_cell_start, F, F + M,
                              F + 2 * M, F + 3 * M, F + 4 * M, F + 5 * M, c->gXs, c->gVs, M, dt, &c->launches,
                              c->rec_hr, c->lr_sorted_idx, c->det_bwd ? c->det_coef : nullptr,
                              c->det_bwd ? c->hr_vals[1] : nullptr, c->det_bwd ? c->det_coef + 2 * M : nullptr),
       "upsample backward");
    if (c->det_bwd)
        CK(gs_launch_upsample_bwd_lr(c->stream, c->d_scenes, c->lr_spos, c->lr_svel, c->lr_sorted_keys,
                                     c->det_coef + 2 * M, c->step_cell_start, c->det_coef, c->gXs, c->gVs, N,
                                     &c->launches),
           "upsample backward, LR side");
    CK(gs_launch_scatter2(c->stream, c->lr_sorted_idx, c->gXs, c->gVs, G, G + N, N, &c->launches), "scatter");
    return GS_OK;
}

int gs_upsample_backward(gs_ctx* c, const float* lr_pos, const float* lr_vel, const float* hr_pos_in,
                         const float* hr_vel_in, const float* g_hr_pos_out, const float* g_hr_vel_out, float* g_lr_pos,
                         float* g_lr_vel, float* g_hr_pos_in, float* g_hr_vel_in, float dt)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (c->n_scenes != 1) return fail(c, GS_ERR_STATE, "the functional frame needs a single-scene context");
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(c, GS_ERR_ARG, "invalid dt %g", (double)dt);
    const int64_t N = c->n_low, M = c->n_high;
    if ((N > 0 && (!lr_pos || !lr_vel || !g_lr_pos || !g_lr_vel)) ||
        (M > 0 && (!hr_pos_in || !hr_vel_in || !g_hr_pos_out || !g_hr_vel_out || !g_hr_pos_in || !g_hr_vel_in)))
        return fail(c, GS_ERR_ARG, "null buffer");
    if (c->n_bodies > 0) return fail(c, GS_ERR_STATE, "the reverse modes do not support rigid bodies");
    st = ensure_fscratch(c);
    if (st) return st;
    float4* F = c->fscratch;
    float4* G = F + 6 * M;
    if (N) {
        CK(cudaMemcpyAsync(c->lr_pos, lr_pos, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
        CK(cudaMemcpyAsync(c->lr_vel, lr_vel, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    }
    if (M) {
        const void* in[4] = {hr_pos_in, hr_vel_in, g_hr_pos_out, g_hr_vel_out};
        for (int k = 0; k < 4; ++k)
            CK(cudaMemcpyAsync(F + k * M, in[k], M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    }
    st = replay_or_run(c, step_key(c, 'v', dt, 0), [&] { return upsample_bwd_seq(c, dt); });
    if (st) return st;
    if (M) {
        CK(cudaMemcpyAsync(g_hr_pos_in, F + 4 * M, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
        CK(cudaMemcpyAsync(g_hr_vel_in, F + 5 * M, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    }
    if (N) {
        CK(cudaMemcpyAsync(g_lr_pos, G, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
        CK(cudaMemcpyAsync(g_lr_vel, G + N, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    }
    return GS_OK;
}

int gs_step_low_forward(gs_ctx* c, const float* x_in, const float* v_in, float* x_out, float* v_out, float dt,
                        int iters)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid dt %g or iters %d", (double)dt, iters);
    const int64_t N = c->n_low;
    if (N == 0) return GS_OK;
    if (!x_in || !v_in || !x_out || !v_out) return fail(c, GS_ERR_ARG, "null buffer");
    CK(cudaMemcpyAsync(c->lr_pos, x_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->lr_vel, v_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    st = replay_or_run(c, step_key(c, 'f', dt, iters), [&] { return step_low_impl(c, dt, iters); });
    if (st) return st;
    c->lr_sorted_keys = c->lr_keys[1];   // the host state the step leaves, replayed or not
    c->lr_sorted_idx = c->lr_vals[1];
    c->lr_binned = false;
    CK(cudaMemcpyAsync(x_out, c->lr_pos, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(v_out, c->lr_vel, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    return GS_OK;
}

void gs_set_alloc_failure(long long after)
{
    g_alloc_countdown.store(after < 0 ? -1 : after);
}

// SDF components of the context's SDFs (a box interior counts its six walls).
static int sdf_component_count(const gs_ctx* c)
{
    int n = 0;
    for (const gs_sdf& b : c->sdf_host)
        n += b.kind == GS_SDF_BOX_INTERIOR ? 6 : ((b.kind == GS_SDF_CONE_SHELL || b.kind == GS_SDF_SOLID_BOX) ? 1 : 0);
    return n;
}

int gs_set_decision_record(gs_ctx* c, uint32_t* hr_record, int32_t* lr_candidates, uint8_t* lr_pair_bits,
                           uint8_t* lr_sdf_bits, int max_passes)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (c->n_scenes != 1) return fail(c, GS_ERR_STATE, "the decision record serves single-scene contexts");
    const bool lr_any = lr_candidates || lr_pair_bits || lr_sdf_bits;
    if (lr_any && (!lr_candidates || !lr_pair_bits || max_passes < 1 ||
                   (sdf_component_count(c) > 0 && !lr_sdf_bits)))
        return fail(c, GS_ERR_ARG, "the LR record needs candidates, pair bits, SDF bits and max_passes >= 1");
    if (hr_record && sdf_component_count(c) > 32) return fail(c, GS_ERR_ARG, "more than 32 SDF components");
    c->rec_hr = hr_record;
    c->rec_lr_cand = lr_any ? lr_candidates : nullptr;
    c->rec_lr_pair = lr_any ? lr_pair_bits : nullptr;
    c->rec_lr_sdf = lr_any ? lr_sdf_bits : nullptr;
    c->rec_max_passes = lr_any ? max_passes : 0;
    drop_graphs(c);   // captured reverse sequences hold the previous record pointers
    return GS_OK;
}

// Per-pass snapshot buffers of the LR step ((total + 1) x n_low each),
// allocated on first use and grown when a step has more passes.
static int ensure_snapshots(gs_ctx* c, int total)
{
    const int64_t N = c->n_low;
    if (total <= c->snap_cap && c->snap) return GS_OK;
    if (c->snap) cudaFree(c->snap);
    if (c->snap_xt) cudaFree(c->snap_xt);
    c->snap = c->snap_xt = nullptr;
    c->snap_cap = 0;
    if (dalloc(&c->snap, (size_t)(total + 1) * N) != cudaSuccess ||
        dalloc(&c->snap_xt, (size_t)(total + 1) * N) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GS_ERR_OOM, "no memory for the per-pass snapshots");
    }
    c->snap_cap = total;
    drop_graphs(c);   // captured sequences hold the old snapshot buffers
    return GS_OK;
}

static int step_low_reverse(gs_ctx* c, float dt, int iters);
static int step_low_record(gs_ctx* c, float dt, int iters);
static int step_low_record_into(gs_ctx* c, float dt, int iters, float4* X, float4* XT, uint32_t* nbr, uint32_t* cnt);
static int step_low_reverse_from(gs_ctx* c, float dt, int iters, const float4* X, const float4* XT,
                                 const uint32_t* nbr, const uint32_t* cnt, const uint32_t* idx);

int gs_step_low_trace(gs_ctx* c, const float* x_in, const float* v_in, float dt, int iters, float* x_trace,
                      float* xt_trace, int n_records)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid dt %g or iters %d", (double)dt, iters);
    if (c->n_materials > 0 || c->n_bodies > 0)
        return fail(c, GS_ERR_STATE, "the pass record covers grains of the scenes' coefficients only");
    const int total = c->n_stab + iters;
    if (n_records != total + 1) return fail(c, GS_ERR_ARG, "n_records must be n_stab + iters + 1 = %d", total + 1);
    const int64_t N = c->n_low;
    if (N == 0) return GS_OK;
    if (!x_in || !v_in || !x_trace || !xt_trace) return fail(c, GS_ERR_ARG, "null buffer");
    st = ensure_snapshots(c, total);
    if (st) return st;
    CK(cudaMemcpyAsync(c->lr_pos, x_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->lr_vel, v_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    st = step_low_record(c, dt, iters);
    if (st) return st;
    float4* xo = reinterpret_cast<float4*>(x_trace);
    float4* xto = reinterpret_cast<float4*>(xt_trace);
    for (int k = 0; k <= total; ++k)
        CK(gs_launch_scatter2(c->stream, c->lr_sorted_idx, c->snap + (size_t)std::min(k, c->n_stab) * N,
                              c->snap_xt + (size_t)k * N, xo + (size_t)k * N, xto + (size_t)k * N, N, &c->launches),
           "scatter");
    c->lr_binned = false;
    return GS_OK;
}


static int ensure_adjoint_buffers(gs_ctx* c)
{
    const int64_t N = c->n_low;
    if (c->adj_gx) return GS_OK;
    bool ok = dalloc(&c->adj_gx, N) == cudaSuccess && dalloc(&c->adj_gxt, N) == cudaSuccess &&
              dalloc(&c->adj_h, N) == cudaSuccess && dalloc(&c->adj_h2, N) == cudaSuccess &&
              dalloc(&c->adj_gws, N) == cudaSuccess &&
              dalloc(&c->adj_io, (size_t)4 * N) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(c, GS_ERR_OOM, "no memory for the reverse-mode buffers");
    }
    return GS_OK;
}

static void free_tapes(gs_ctx* c)
{
    for (auto& t : c->tapes)
        for (void* b : {(void*)t.X, (void*)t.XT, (void*)t.nbr, (void*)t.cnt, (void*)t.idx})
            if (b) cudaFree(b);
    c->tapes.clear();
    c->tape_passes = 0;
    c->tape_next = 0;
}

int gs_set_step_tapes(gs_ctx* c, int n_slots)
{
    int st = check_state(c);
    if (st) return st;
    if (n_slots < 0 || n_slots > 1024) return fail(c, GS_ERR_ARG, "bad tape count %d", n_slots);
    st = settle(c);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream), "synchronize");   // no graph still reads the old tapes
    drop_graphs(c);
    free_tapes(c);
    c->tapes.resize((size_t)n_slots);
    return GS_OK;
}

// (Re)allocates every tape slot for steps of `total` passes (growing only).
static int ensure_tapes(gs_ctx* c, int total)
{
    if (total <= c->tape_passes && !c->tapes.empty() && c->tapes[0].X) return GS_OK;
    const size_t n_slots = c->tapes.size();
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    drop_graphs(c);   // captured sequences hold the old tape buffers
    free_tapes(c);
    c->tapes.resize(n_slots);
    const int64_t N = c->n_low;
    for (auto& t : c->tapes) {
        bool ok = dalloc(&t.X, (size_t)(total + 1) * N) == cudaSuccess &&
                  dalloc(&t.XT, (size_t)(total + 1) * N) == cudaSuccess &&
                  dalloc(&t.nbr, (size_t)c->nbr_cap * N) == cudaSuccess && dalloc(&t.cnt, (size_t)N) == cudaSuccess &&
                  dalloc(&t.idx, (size_t)N) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_tapes(c);
            c->tapes.resize(n_slots);
            return fail(c, GS_ERR_OOM, "no memory for the LR step tapes");
        }
    }
    c->tape_passes = total;
    return GS_OK;
}

static uint64_t tape_key(const gs_ctx* c, char kind, float dt, int iters, int slot)
{
    return (step_key(c, kind, dt, iters) ^ (0x9e3779b97f4a7c15ull * (uint64_t)(slot + 1))) * 0x100000001b3ull;
}

// The recorded forward into tape slot t, then the step's finalize from the
// last snapshots (v = (x~ - x) / dt, x = x~, original order).
static int step_low_tape_forward(gs_ctx* c, gs_ctx::StepTape& t, float dt, int iters)
{
    const int64_t N = c->n_low;
    const int total = c->n_stab + iters;
    int st = step_low_record_into(c, dt, iters, t.X, t.XT, t.nbr, t.cnt);
    if (st) return st;
    CK(cudaMemcpyAsync(t.idx, c->lr_sorted_idx, N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream),
       "keep the cell order");
    const PbdArgs a = pbd_args(c, dt);
    CK(gs_launch_finalize(c->stream, a, t.idx, t.X + (size_t)std::min(total, c->n_stab) * N, t.XT + (size_t)total * N,
                          c->lr_pos, c->lr_vel, &c->launches, nullptr),
       "finalize");
    c->lr_binned = false;
    return GS_OK;
}

int gs_step_low_forward_taped(gs_ctx* c, const float* x_in, const float* v_in, float* x_out, float* v_out, float dt,
                              int iters, int64_t tag)
{
    int st = check_state(c);
    if (st) return st;
    if (tag < 0) return fail(c, GS_ERR_ARG, "negative tape tag");
    if (c->tapes.empty()) return gs_step_low_forward(c, x_in, v_in, x_out, v_out, dt, iters);
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid dt %g or iters %d", (double)dt, iters);
    if (c->n_materials > 0 || c->n_bodies > 0)
        return fail(c, GS_ERR_STATE, "taped LR steps cover grains of the scenes' coefficients only");
    const int64_t N = c->n_low;
    if (N == 0) return GS_OK;
    if (!x_in || !v_in || !x_out || !v_out) return fail(c, GS_ERR_ARG, "null buffer");
    st = ensure_tapes(c, c->n_stab + iters);
    if (st) return st;
    const int slot = c->tape_next;
    gs_ctx::StepTape& t = c->tapes[(size_t)slot];
    t.tag = -1;   // until the step below is enqueued
    CK(cudaMemcpyAsync(c->lr_pos, x_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->lr_vel, v_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    st = replay_or_run(c, tape_key(c, 'F', dt, iters, slot), [&] { return step_low_tape_forward(c, t, dt, iters); });
    if (st) return st;
    CK(cudaMemcpyAsync(x_out, c->lr_pos, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(v_out, c->lr_vel, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    t.tag = tag;
    t.serial = c->tape_serial++;
    t.dt = dt;
    t.iters = iters;
    c->tape_next = (slot + 1) % (int)c->tapes.size();
    return GS_OK;
}

int gs_step_low_backward_taped(gs_ctx* c, int64_t tag, const float* g_x_out, const float* g_v_out, float* g_x_in,
                               float* g_v_in)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    const int64_t N = c->n_low;
    int slot = -1;
    for (size_t k = 0; k < c->tapes.size(); ++k)
        if (tag >= 0 && c->tapes[k].tag == tag && (slot < 0 || c->tapes[k].serial > c->tapes[(size_t)slot].serial))
            slot = (int)k;
    if (slot < 0) return fail(c, GS_ERR_STATE, "no kept tape has tag %lld", (long long)tag);
    if (N == 0) return GS_OK;
    if (!g_x_out || !g_v_out || !g_x_in || !g_v_in) return fail(c, GS_ERR_ARG, "null buffer");
    const gs_ctx::StepTape& t = c->tapes[(size_t)slot];
    if (c->rec_lr_pair && c->n_stab + t.iters > c->rec_max_passes)
        return fail(c, GS_ERR_ARG, "%d passes exceed the decision record's %d", c->n_stab + t.iters,
                    c->rec_max_passes);
    st = ensure_adjoint_buffers(c);
    if (st) return st;
    CK(cudaMemcpyAsync(c->adj_io, g_x_out, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->adj_io + N, g_v_out, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    st = replay_or_run(c, tape_key(c, 'B', t.dt, t.iters, slot), [&] {
        return step_low_reverse_from(c, t.dt, t.iters, t.X, t.XT, t.nbr, t.cnt, t.idx);
    });
    if (st) return st;
    CK(cudaMemcpyAsync(g_x_in, c->adj_io + 2 * N, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(g_v_in, c->adj_io + 3 * N, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    return GS_OK;
}

int gs_step_low_backward(gs_ctx* c, const float* x_in, const float* v_in, const float* g_x_out, const float* g_v_out,
                         float* g_x_in, float* g_v_in, float dt, int iters)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid dt %g or iters %d", (double)dt, iters);
    if (c->n_materials > 0)
        return fail(c, GS_ERR_STATE, "the reverse mode of the LR step does not support grain materials");
    if (c->n_bodies > 0) return fail(c, GS_ERR_STATE, "the reverse modes do not support rigid bodies");
    const int64_t N = c->n_low;
    if (N == 0) return GS_OK;
    if (!x_in || !v_in || !g_x_out || !g_v_out || !g_x_in || !g_v_in) return fail(c, GS_ERR_ARG, "null buffer");
    if (c->rec_lr_pair && c->n_stab + iters > c->rec_max_passes)
        return fail(c, GS_ERR_ARG, "%d passes exceed the decision record's %d", c->n_stab + iters, c->rec_max_passes);
    st = ensure_snapshots(c, c->n_stab + iters);
    if (st) return st;
    st = ensure_adjoint_buffers(c);
    if (st) return st;
    // the caller's buffers in; the rest runs on the context's own buffers
    // (replayed as a graph when graphs are enabled)
    CK(cudaMemcpyAsync(c->lr_pos, x_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->lr_vel, v_in, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->adj_io, g_x_out, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(c->adj_io + N, g_v_out, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    st = replay_or_run(c, step_key(c, 'b', dt, iters), [&] { return step_low_reverse(c, dt, iters); });
    if (st) return st;
    CK(cudaMemcpyAsync(g_x_in, c->adj_io + 2 * N, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    CK(cudaMemcpyAsync(g_v_in, c->adj_io + 3 * N, N * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream), "copy");
    c->lr_sorted_keys = c->lr_keys[1];   // the host state the reverse step leaves
    c->lr_sorted_idx = c->lr_vals[1];
    c->lr_binned = false;
    return GS_OK;
}

// The LR step on the context's buffers (from lr_pos, lr_vel) keeping what
// every pass evaluates on, in cell order: x~ before pass it is
// snap_xt[it], x before stabilization pass it is snap[it] (after the
// stabilization passes snap[n_stab] throughout); snap_xt[total] holds the
// step's final x~.  The passes read and write the snapshot buffers
// themselves.
// The recording into given buffers (the snapshots X, XT and the candidate
// lists nbr / cnt; the cell order is left in lr_sorted_idx).
static int step_low_record_into(gs_ctx* c, float dt, int iters, float4* X, float4* XT, uint32_t* nbr, uint32_t* cnt)
{
    const int64_t N = c->n_low;
    const int total = c->n_stab + iters;
    int st = flag_solid(c, (const float*)c->lr_pos, N);
    if (st) return st;
    PbdArgs a = pbd_args(c, dt);
    CK(gs_launch_predict(c->stream, a, c->lr_pos, c->lr_vel, c->lr_xt, &c->launches), "predict");
    st = bin_low_at(c, c->lr_xt);
    if (st) return st;
    CK(gs_launch_step_gather(c->stream, N, c->lr_sorted_idx, c->lr_xt, c->lr_pos, XT, X, &c->launches), "gather");
    CK(gs_launch_neighbors(c->stream, a, XT, c->lr_sorted_keys, c->lr_cell_start, c->n_cell_total, nbr, cnt,
                           c->nbr_cap, c->d_err, &c->launches),
       "neighbours");
    for (int it = 0; it < total; ++it) {
        const int stab = it < c->n_stab;
        CK(gs_launch_pass(c->stream, a, stab, X + (size_t)std::min(it, c->n_stab) * N, XT + (size_t)it * N,
                          X + (size_t)(it + 1) * N, XT + (size_t)(it + 1) * N, nbr, cnt, &c->launches),
           "pass");
    }
    return GS_OK;
}

static int step_low_record(gs_ctx* c, float dt, int iters)
{
    return step_low_record_into(c, dt, iters, c->snap, c->snap_xt, c->nbr, c->nbr_cnt);
}

// The passes of a recorded LR step in reverse: dL/d outputs from
// adj_io[0..1], dL/d inputs into adj_io[2..3]; X, XT, nbr, cnt as recorded,
// idx the recording's cell order.
static int step_low_reverse_from(gs_ctx* c, float dt, int iters, const float4* X, const float4* XT,
                                 const uint32_t* nbr, const uint32_t* cnt, const uint32_t* idx);

// The reverse LR step on the context's buffers: the step again from
// (lr_pos, lr_vel) keeping what every pass evaluates on, then the passes in
// reverse.
static int step_low_reverse(gs_ctx* c, float dt, int iters)
{
    int st = step_low_record(c, dt, iters);
    if (st) return st;
    return step_low_reverse_from(c, dt, iters, c->snap, c->snap_xt, c->nbr, c->nbr_cnt, c->lr_sorted_idx);
}

static int step_low_reverse_from(gs_ctx* c, float dt, int iters, const float4* X, const float4* XT,
                                 const uint32_t* nbr, const uint32_t* cnt, const uint32_t* idx)
{
    const int64_t N = c->n_low;
    const int total = c->n_stab + iters;
    PbdArgs a = pbd_args(c, dt);
    auto x_before = [&](int it) { return X + (size_t)std::min(it, c->n_stab) * N; };
    const float4* xfix = x_before(total);     // x after stabilization
    const float4* ws = XT;                    // w of xt carries the inverse scaled mass (every pass keeps it)
    CK(gs_launch_adj_init(c->stream, N, idx, c->adj_io, c->adj_io + N, dt, c->adj_gx, c->adj_gxt, c->adj_gws,
                          &c->launches),
       "reverse init");
    float4* Hb[2] = {c->adj_h, c->adj_h2};
    int hc = 0;
    auto y_of = [&](int it) { return it < c->n_stab ? x_before(it) : XT + (size_t)it * N; };
    if (total > 0)
        CK(gs_launch_adj_h(c->stream, a, (total - 1) < c->n_stab, y_of(total - 1), ws, nbr, cnt, c->adj_gx, c->adj_gxt,
                           Hb[0], &c->launches),
           "reverse h");
    for (int it = total - 1; it >= 0; --it) {
        const int stab = it < c->n_stab;
        AdjRecord rec;
        if (c->rec_lr_pair) {
            const int n_comp = sdf_component_count(c);
            rec.idx = idx;
            rec.cand = c->rec_lr_cand;
            rec.pair = c->rec_lr_pair + (size_t)it * c->nbr_cap * N;
            rec.sdf = n_comp > 0 ? c->rec_lr_sdf + (size_t)it * N * n_comp : nullptr;
            rec.cap = c->nbr_cap;
            rec.n_comp = n_comp;
        }
        CK(gs_launch_adj_pass(c->stream, a, stab, y_of(it), XT + (size_t)it * N, xfix, ws, nbr, cnt, Hb[hc],
                              c->adj_gx, c->adj_gxt, c->adj_gws, &c->launches, rec, it > 0 ? y_of(it - 1) : nullptr,
                              (it - 1) < c->n_stab, Hb[hc ^ 1]),
           "reverse pass");
        hc ^= 1;
    }
    CK(gs_launch_adj_final(c->stream, a, idx, ws, c->adj_gx, c->adj_gxt, c->adj_gws, c->adj_io + 2 * N,
                           c->adj_io + 3 * N, &c->launches),
       "reverse predict");
    c->lr_binned = false;
    return GS_OK;
}

int gs_sync(gs_ctx* c)
{
    int st = check_state(c);
    if (st) return st;
    st = settle(c);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream_h2d), "synchronize host-to-device copies");
    CK(cudaStreamSynchronize(c->stream_d2h), "synchronize device-to-host copies");
    st = fold_cfl_launches(c);
    if (st) return st;
    return report_device_errors(c);
}

int gs_write_async(gs_ctx* c, int field, const void* src, size_t bytes, int src_is_device)
{
    int st = check_state(c);
    if (st) return st;
    if (field < GS_FIELD_LR_POS || field > GS_FIELD_HR_VEL)
        return fail(c, GS_ERR_ARG, "field %d is not writable", field);
    if (bytes != field_bytes(c, field)) return fail(c, GS_ERR_ARG, "size %zu does not match field %d", bytes, field);
    st = slab_refuse_hr_field(c, field);
    if (st) return st;
    if (bytes == 0) return GS_OK;
    if (!src) return fail(c, GS_ERR_ARG, "null source");
    st = async_buffer(c, &c->async_in[field], field);
    if (st) return st;
    // the staging buffer is reused once the previous commit has read it
    CK(cudaStreamWaitEvent(c->stream_h2d, c->ev_in_free[field], 0), "wait for the staging buffer");
    CK(cudaMemcpyAsync(c->async_in[field], src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream_h2d),
       "copy in");
    CK(cudaEventRecord(c->ev_in_ready[field], c->stream_h2d), "record");
    c->in_pending[field] = true;
    return GS_OK;
}

int gs_read_async(gs_ctx* c, int field, void* dst, size_t bytes, int dst_is_device)
{
    int st = check_state(c);
    if (st) return st;
    if (field < GS_FIELD_LR_POS || field > GS_FIELD_HR_VEL)
        return fail(c, GS_ERR_ARG, "field %d has no asynchronous read", field);
    if (bytes != field_bytes(c, field)) return fail(c, GS_ERR_ARG, "size %zu does not match field %d", bytes, field);
    if (bytes > 0 && !dst) return fail(c, GS_ERR_ARG, "null destination");
    st = slab_refuse_hr_field(c, field);
    if (st) return st;
    if (dst_is_device) return gs_read(c, field, dst, bytes, 1);   // already asynchronous
    st = settle(c);
    if (st) return st;
    if (bytes == 0) return GS_OK;
    st = async_buffer(c, &c->async_out[field], field);
    if (st) return st;
    float4* out = c->async_out[field];
    // an HR field whose snapshot the read of the other one took, with no
    // kernel launched since: only the copy out is left
    const bool paired = c->hr_pair_field == field && c->hr_pair_launches == c->launches;
    c->hr_pair_field = -1;
    if (!paired) {
        // snapshot in stream order, then copy it out on its own stream
        CK(cudaStreamWaitEvent(c->stream, c->ev_out_free[field], 0), "wait for the snapshot buffer");
        const int cur = c->hr_cur;
        switch (field) {
        case GS_FIELD_LR_POS:
            CK(cudaMemcpyAsync(out, c->lr_pos, bytes, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
            break;
        case GS_FIELD_LR_VEL:
            CK(cudaMemcpyAsync(out, c->lr_vel, bytes, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
            break;
        default: {
            // both HR fields in one pass (the ids are read once); the other
            // snapshot serves the usual next call, the read of that field
            const int other = field == GS_FIELD_HR_POS ? GS_FIELD_HR_VEL : GS_FIELD_HR_POS;
            st = async_buffer(c, &c->async_out[other], other);
            if (st) return st;
            CK(cudaStreamWaitEvent(c->stream, c->ev_out_free[other], 0), "wait for the snapshot buffer");
            CK(gs_launch_unpermute2(c->stream, c->hr_pos[cur], c->hr_vel[cur], c->hr_scene,
                                    c->async_out[GS_FIELD_HR_POS], c->async_out[GS_FIELD_HR_VEL], c->hr_slots,
                                    c->n_high, c->d_err, &c->launches),
               "unpermute");
            CK(cudaEventRecord(c->ev_out_ready[other], c->stream), "record");
            c->hr_pair_field = other;
            c->hr_pair_launches = c->launches;
        }
        }
        CK(cudaEventRecord(c->ev_out_ready[field], c->stream), "record");
    }
    CK(cudaStreamWaitEvent(c->stream_d2h, c->ev_out_ready[field], 0), "wait for the snapshot");
    CK(cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, c->stream_d2h), "copy out");
    CK(cudaEventRecord(c->ev_out_free[field], c->stream_d2h), "record");
    return GS_OK;
}

int gs_set_timing(gs_ctx* c, int enable)
{
    int st = check_state(c);
    if (st) return st;
    c->timing = enable != 0;
    return GS_OK;
}

int gs_timing_read(gs_ctx* c, int timer, double* total_ms, int64_t* launches)
{
    int st = check_state(c);
    if (st) return st;
    if (timer < 0 || timer >= GS_TIMER_COUNT) return fail(c, GS_ERR_ARG, "bad timer %d", timer);
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    double tot = 0.0;
    for (auto& pr : c->ev[timer]) {
        float ms = 0.0f;
        cudaError_t e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e == cudaSuccess) tot += ms;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (launches) *launches = (int64_t)c->ev[timer].size();
    if (total_ms) *total_ms = tot;
    c->ev[timer].clear();
    return GS_OK;
}

int64_t gs_launch_count(const gs_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
