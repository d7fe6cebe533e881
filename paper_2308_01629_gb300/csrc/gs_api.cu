// gs_api.cu -- host side of the C ABI declared in gs.h: argument checks,
// buffer ownership, and the order in which the kernels of one LR step and
// one HR frame are enqueued on the context's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
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

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

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
    }
    return GS_OK;
}

size_t field_bytes(const gs_ctx* c, int field)
{
    switch (field) {
    case GS_FIELD_LR_POS:
    case GS_FIELD_LR_VEL: return (size_t)c->n_low * sizeof(float4);
    case GS_FIELD_HR_POS:
    case GS_FIELD_HR_VEL:
    case GS_FIELD_HR_POS_INTERNAL:
    case GS_FIELD_HR_VEL_INTERNAL: return (size_t)c->n_high * sizeof(float4);
    case GS_FIELD_LR_CELL_START: return (size_t)(c->n_cell + 1) * sizeof(uint32_t);
    case GS_FIELD_LR_SORTED_INDEX: return (size_t)c->n_low * sizeof(uint32_t);
    case GS_FIELD_HR_SORTED_KEY: return (size_t)c->n_high * sizeof(uint32_t);
    default: return (size_t)-1;
    }
}

bool finite3_host(const float4* a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!(std::isfinite(a[i].x) && std::isfinite(a[i].y) && std::isfinite(a[i].z))) return false;
    return true;
}

int bin_low_at(gs_ctx* c, const float4* positions)
{
    const int64_t n = c->n_low;
    CK(gs_launch_cell_keys(c->stream, positions, n, c->grid, 0, c->lr_keys[0], c->lr_vals[0], &c->launches),
       "cell keys");
    int which = 0;
    CK(gs_radix_sort(c->stream, c->lr_keys, c->lr_vals, &which, c->sort_hist, n, c->lr_key_bits, &c->launches),
       "radix sort");
    c->lr_sorted_keys = c->lr_keys[which];
    c->lr_sorted_idx = c->lr_vals[which];
    CK(gs_launch_cell_start(c->stream, c->lr_sorted_keys, n, c->n_cell, c->lr_cell_start, &c->launches),
       "cell start");
    return GS_OK;
}

PbdArgs pbd_args(const gs_ctx* c, float dt)
{
    PbdArgs a;
    a.n = c->n_low;
    a.r = c->r_low;
    a.dt = dt;
    a.gx = c->prm.gravity[0];
    a.gy = c->prm.gravity[1];
    a.gz = c->prm.gravity[2];
    a.mu_s = c->prm.mu_s;
    a.mu_k = c->prm.mu_k;
    a.mass_k = c->prm.mass_scale_k;
    a.ground_z = c->prm.ground_z;
    a.rc = c->prm.neighbor_radius;
    a.friction_mode = c->prm.friction_mode;
    a.sdf = c->d_sdf;
    a.n_sdf = c->n_sdf;
    return a;
}

}  // namespace

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
    if (!out) return GS_ERR_ARG;
    *out = nullptr;
    if (!scene || !(r_low > 0.0f) || !std::isfinite(r_low) || ratio < 1 || scene->n_low < 0) return GS_ERR_ARG;
    if (scene->n_sdf < 0 || scene->n_sdf > GS_MAX_SDF || (scene->n_sdf > 0 && !scene->sdf)) return GS_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (!(scene->box_hi[k] > scene->box_lo[k]) || !std::isfinite(scene->box_lo[k]) ||
            !std::isfinite(scene->box_hi[k]))
            return GS_ERR_ARG;
    const int64_t n_high = (int64_t)scene->n_low * ratio;
    if (n_high > 0x7fffffffLL) return GS_ERR_ARG;   // ids are stored as uint32, indices as int32 slots

    gs_ctx* c = new (std::nothrow) gs_ctx();
    if (!c) return GS_ERR_OOM;
    c->n_low = scene->n_low;
    c->n_high = n_high;
    c->ratio = ratio;
    c->r_low = r_low;
    c->r_high = r_high > 0.0f ? r_high : (float)((double)r_low * std::pow((double)ratio, -1.0 / 3.0));
    c->prm = scene->params;
    if (std::isnan(c->prm.ground_z)) c->prm.ground_z = scene->box_lo[2];
    if (c->prm.neighbor_radius <= 0.0f) c->prm.neighbor_radius = 3.0f * r_low;
    if (c->prm.max_neighbors <= 0) c->prm.max_neighbors = 64;
    c->nbr_cap = c->prm.max_neighbors;
    if (!(c->prm.neighbor_radius > 2.0f * r_low) || c->prm.neighbor_radius > 3.0f * r_low || c->prm.n_stab < 0 ||
        c->prm.n_stab > 100 || c->prm.resort_every < 0 || c->nbr_cap > 4096 ||
        (c->prm.friction_mode != 0 && c->prm.friction_mode != 1)) {
        delete c;
        return GS_ERR_ARG;
    }
    c->n_sdf = scene->n_sdf;
    for (int k = 0; k < c->n_sdf; ++k) c->sdf_host[k] = scene->sdf[k];

    // grid contract
    {
        double hd = 3.0 * (double)r_low * (1.0 + 1.0 / 1024.0);
        float hf = (float)hd;
        c->grid.h = hf;
        c->grid.inv_h = (float)(1.0 / (double)hf);
        c->grid.ox = scene->box_lo[0];
        c->grid.oy = scene->box_lo[1];
        c->grid.oz = scene->box_lo[2];
        int dims[3];
        for (int k = 0; k < 3; ++k) {
            double n = std::ceil(((double)scene->box_hi[k] - (double)scene->box_lo[k]) / (double)hf);
            if (n > (double)(1 << 20)) {
                delete c;
                return GS_ERR_ARG;
            }
            dims[k] = n < 1 ? 1 : (int)n;
        }
        c->grid.dx = dims[0];
        c->grid.dy = dims[1];
        c->grid.dz = dims[2];
        c->n_cell = (int64_t)dims[0] * dims[1] * dims[2];
        if (c->n_cell * 8 > 0xffffffffLL) {
            delete c;
            return GS_ERR_ARG;
        }
        c->lr_key_bits = gs_key_bits(c->n_cell);
        c->hr_key_bits = gs_key_bits(c->n_cell * 8);
    }

    cudaError_t e = cudaGetDevice(&c->device);
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
    const int64_t N = c->n_low, M = c->n_high;
    const int64_t NM = N > M ? N : M;
    bool ok = true;
    auto A = [&](cudaError_t r) { ok = ok && r == cudaSuccess; };
    A(dalloc(&c->d_sdf, GS_MAX_SDF));
    A(dalloc(&c->lr_pos, N));
    A(dalloc(&c->lr_vel, N));
    A(dalloc(&c->lr_keys[0], N));
    A(dalloc(&c->lr_keys[1], N));
    A(dalloc(&c->lr_vals[0], N));
    A(dalloc(&c->lr_vals[1], N));
    A(dalloc(&c->lr_cell_start, c->n_cell + 1));
    A(dalloc(&c->lr_spos, N));
    A(dalloc(&c->lr_svel, N));
    A(dalloc(&c->lr_xt, N));
    for (int k = 0; k < 2; ++k) {
        A(dalloc(&c->s_xt[k], N));
        A(dalloc(&c->s_x[k], N));
        A(dalloc(&c->hr_pos[k], M));
        A(dalloc(&c->hr_vel[k], M));
        A(dalloc(&c->hr_keys[k], M));
        A(dalloc(&c->hr_vals[k], M));
    }
    A(dalloc(&c->nbr, (size_t)N * c->nbr_cap));
    A(dalloc(&c->nbr_cnt, N));
    A(dalloc(&c->tmp4, NM));
    c->sort_hist_cap = std::max(gs_sort_hist_words(N), gs_sort_hist_words(M));
    A(dalloc(&c->sort_hist, c->sort_hist_cap));
    A(dalloc(&c->d_err, 1));
    if (ok) ok = cudaMallocHost((void**)&c->h_err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        gs_destroy(c);
        return GS_ERR_OOM;
    }
    *c->h_err = 0;
    bool z = true;
    auto Z = [&](void* p, size_t b) { z = z && cudaMemsetAsync(p, 0, b, c->stream) == cudaSuccess; };
    Z(c->d_err, sizeof(int));
    Z(c->lr_pos, N * sizeof(float4));
    Z(c->lr_vel, N * sizeof(float4));
    Z(c->hr_pos[0], M * sizeof(float4));
    Z(c->hr_vel[0], M * sizeof(float4));
    Z(c->lr_cell_start, (c->n_cell + 1) * sizeof(uint32_t));
    if (c->n_sdf > 0)
        z = z && cudaMemcpyAsync(c->d_sdf, c->sdf_host, c->n_sdf * sizeof(gs_sdf), cudaMemcpyHostToDevice,
                                 c->stream) == cudaSuccess;
    if (z) z = gs_launch_set_ids(c->stream, c->hr_pos[0], M, &c->launches) == cudaSuccess;
    if (z) z = cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (!z) {
        gs_destroy(c);
        return GS_ERR_CUDA;
    }
    *out = c;
    return GS_OK;
}

void gs_destroy(gs_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int t = 0; t < GS_TIMER_COUNT; ++t)
        for (auto& pr : c->ev[t]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    void* bufs[] = {c->d_sdf,      c->lr_pos,    c->lr_vel,     c->lr_keys[0], c->lr_keys[1], c->lr_vals[0],
                    c->lr_vals[1], c->lr_cell_start, c->lr_spos, c->lr_svel,   c->lr_xt,      c->s_xt[0],
                    c->s_xt[1],    c->s_x[0],    c->s_x[1],     c->hr_pos[0],  c->hr_pos[1],  c->hr_vel[0],
                    c->hr_vel[1],  c->hr_keys[0], c->hr_keys[1], c->hr_vals[0], c->hr_vals[1], c->nbr,
                    c->nbr_cnt,    c->tmp4,      c->sort_hist,  c->d_err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

int gs_info(const gs_ctx* c, int64_t* n_low, int64_t* n_high, gs_grid_info* grid)
{
    if (!c) return GS_ERR_ARG;
    if (n_low) *n_low = c->n_low;
    if (n_high) *n_high = c->n_high;
    if (grid) {
        grid->origin[0] = c->grid.ox;
        grid->origin[1] = c->grid.oy;
        grid->origin[2] = c->grid.oz;
        grid->h = c->grid.h;
        grid->inv_h = c->grid.inv_h;
        grid->dims[0] = c->grid.dx;
        grid->dims[1] = c->grid.dy;
        grid->dims[2] = c->grid.dz;
        grid->n_cell = c->n_cell;
    }
    return GS_OK;
}

int gs_write(gs_ctx* c, int field, const void* src, size_t bytes, int src_is_device)
{
    int st = check_state(c);
    if (st) return st;
    if (field != GS_FIELD_LR_POS && field != GS_FIELD_LR_VEL && field != GS_FIELD_HR_POS && field != GS_FIELD_HR_VEL)
        return fail(c, GS_ERR_ARG, "field %d is not writable", field);
    if (bytes != field_bytes(c, field)) return fail(c, GS_ERR_ARG, "size %zu does not match field %d", bytes, field);
    if (bytes == 0) return GS_OK;
    if (!src) return fail(c, GS_ERR_ARG, "null source");
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int64_t n = (field == GS_FIELD_LR_POS || field == GS_FIELD_LR_VEL) ? c->n_low : c->n_high;
    if (!src_is_device) {
        if (!finite3_host((const float4*)src, n))
            return fail(c, GS_ERR_DOMAIN, "non-finite value in field %d", field);
    } else {
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear flag");
        CK(gs_launch_check_finite(c->stream, (const float4*)src, n, c->d_err, &c->launches), "finite check");
        CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        if (*c->h_err) {
            CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear flag");
            return fail(c, GS_ERR_DOMAIN, "non-finite value in field %d", field);
        }
    }
    switch (field) {
    case GS_FIELD_LR_POS:
        CK(cudaMemcpyAsync(c->lr_pos, src, bytes, kind, c->stream), "copy");
        c->lr_binned = false;
        break;
    case GS_FIELD_LR_VEL: CK(cudaMemcpyAsync(c->lr_vel, src, bytes, kind, c->stream), "copy"); break;
    case GS_FIELD_HR_POS: {
        const int cur = c->hr_cur;
        if (!c->hr_identity) {
            // bring the velocities back to original-id order first
            CK(gs_launch_unpermute(c->stream, c->hr_pos[cur], c->hr_vel[cur], c->hr_vel[cur ^ 1], c->n_high,
                                   c->d_err, &c->launches),
               "unpermute");
            CK(cudaMemcpyAsync(c->hr_vel[cur], c->hr_vel[cur ^ 1], bytes, cudaMemcpyDeviceToDevice, c->stream),
               "copy");
        }
        CK(cudaMemcpyAsync(c->hr_pos[cur], src, bytes, kind, c->stream), "copy");
        CK(gs_launch_set_ids(c->stream, c->hr_pos[cur], c->n_high, &c->launches), "ids");
        c->hr_identity = true;
        c->hr_keys_valid = false;
        break;
    }
    case GS_FIELD_HR_VEL: {
        const int cur = c->hr_cur;
        if (c->hr_identity) {
            CK(cudaMemcpyAsync(c->hr_vel[cur], src, bytes, kind, c->stream), "copy");
        } else {
            CK(cudaMemcpyAsync(c->tmp4, src, bytes, kind, c->stream), "copy");
            CK(gs_launch_permute_in(c->stream, c->hr_pos[cur], c->tmp4, c->hr_vel[cur], c->n_high, c->d_err,
                                    &c->launches),
               "permute");
        }
        break;
    }
    }
    if (!src_is_device) CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GS_OK;
}

int gs_read(gs_ctx* c, int field, void* dst, size_t bytes, int dst_is_device)
{
    int st = check_state(c);
    if (st) return st;
    size_t fb = field_bytes(c, field);
    if (fb == (size_t)-1) return fail(c, GS_ERR_ARG, "unknown field %d", field);
    if (bytes != fb) return fail(c, GS_ERR_ARG, "size %zu does not match field %d", bytes, field);
    if (bytes > 0 && !dst) return fail(c, GS_ERR_ARG, "null destination");
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const int cur = c->hr_cur;
    const void* srcp = nullptr;
    switch (field) {
    case GS_FIELD_LR_POS: srcp = c->lr_pos; break;
    case GS_FIELD_LR_VEL: srcp = c->lr_vel; break;
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
        if (c->hr_identity) {
            srcp = f;
        } else {
            float4* target = dst_is_device ? (float4*)dst : c->tmp4;
            CK(gs_launch_unpermute(c->stream, c->hr_pos[cur], f, target, c->n_high, c->d_err, &c->launches),
               "unpermute");
            if (dst_is_device) return GS_OK;
            srcp = c->tmp4;
        }
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
    if (!sdf || index < 0 || index >= c->n_sdf) return fail(c, GS_ERR_ARG, "bad SDF index %d", index);
    c->sdf_host[index] = *sdf;
    CK(cudaMemcpyAsync(c->d_sdf + index, &c->sdf_host[index], sizeof(gs_sdf), cudaMemcpyHostToDevice, c->stream),
       "copy SDF");
    return GS_OK;
}

int gs_bin_low(gs_ctx* c)
{
    int st = check_state(c);
    if (st) return st;
    Timed t(c, GS_TIMER_BIN_LOW);
    st = bin_low_at(c, c->lr_pos);
    if (st) return st;
    CK(gs_launch_gather2(c->stream, c->lr_sorted_idx, c->lr_pos, c->lr_vel, c->lr_spos, c->lr_svel, c->n_low,
                         &c->launches),
       "gather");
    c->lr_binned = true;
    return GS_OK;
}

int gs_resort_high(gs_ctx* c)
{
    int st = check_state(c);
    if (st) return st;
    const int64_t M = c->n_high;
    if (M == 0) return GS_OK;
    Timed t(c, GS_TIMER_RESORT);
    const int cur = c->hr_cur;
    CK(gs_launch_cell_keys(c->stream, c->hr_pos[cur], M, c->grid, 1, c->hr_keys[0], c->hr_vals[0], &c->launches),
       "keys");
    int which = 0;
    CK(gs_radix_sort(c->stream, c->hr_keys, c->hr_vals, &which, c->sort_hist, M, c->hr_key_bits, &c->launches),
       "radix sort");
    CK(gs_launch_gather2(c->stream, c->hr_vals[which], c->hr_pos[cur], c->hr_vel[cur], c->hr_pos[cur ^ 1],
                         c->hr_vel[cur ^ 1], M, &c->launches),
       "permute");
    c->hr_sorted_keys = c->hr_keys[which];
    c->hr_keys_valid = true;
    c->hr_cur = cur ^ 1;
    c->hr_identity = false;
    return GS_OK;
}

int gs_step_low(gs_ctx* c, float dt, int iters)
{
    int st = check_state(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt) || iters < 0 || iters > 1000)
        return fail(c, GS_ERR_ARG, "invalid dt %g or iters %d", (double)dt, iters);
    const int64_t N = c->n_low;
    if (N == 0) return GS_OK;
    Timed t(c, GS_TIMER_STEP_LOW);
    PbdArgs a = pbd_args(c, dt);
    CK(gs_launch_predict(c->stream, a, c->lr_pos, c->lr_vel, c->lr_xt, &c->launches), "predict");
    st = bin_low_at(c, c->lr_xt);
    if (st) return st;
    CK(gs_launch_step_gather(c->stream, N, c->lr_sorted_idx, c->lr_xt, c->lr_pos, c->s_xt[0], c->s_x[0],
                             &c->launches),
       "gather");
    CK(gs_launch_neighbors(c->stream, a, c->s_xt[0], c->lr_sorted_keys, c->lr_cell_start, c->grid, c->nbr, c->nbr_cnt,
                           c->nbr_cap, c->d_err, &c->launches),
       "neighbours");
    int bx = 0, bt = 0;   // buffers holding the current x and xt
    for (int it = 0; it < c->prm.n_stab + iters; ++it) {
        const int stab = it < c->prm.n_stab;
        CK(gs_launch_pass(c->stream, a, stab, c->s_x[bx], c->s_xt[bt], c->s_x[bx ^ 1], c->s_xt[bt ^ 1], c->nbr,
                          c->nbr_cnt, c->nbr_cap, &c->launches),
           "pass");
        bt ^= 1;
        if (stab) bx ^= 1;
    }
    CK(gs_launch_finalize(c->stream, a, c->lr_sorted_idx, c->s_x[bx], c->s_xt[bt], c->lr_pos, c->lr_vel,
                          &c->launches),
       "finalize");
    c->lr_binned = false;   // the binning above is of the predicted positions
    return GS_OK;
}

int gs_upsample(gs_ctx* c, float dt)
{
    int st = check_state(c);
    if (st) return st;
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(c, GS_ERR_ARG, "invalid dt %g", (double)dt);
    if (c->n_high == 0) {
        c->frame++;
        return GS_OK;
    }
    if (c->prm.resort_every > 0 && c->frame % c->prm.resort_every == 0) {
        st = gs_resort_high(c);
        if (st) return st;
    }
    st = gs_bin_low(c);
    if (st) return st;
    UpsampleArgs u;
    const int cur = c->hr_cur;
    u.hr_pos = c->hr_pos[cur];
    u.hr_vel = c->hr_vel[cur];
    u.out_pos = c->hr_pos[cur ^ 1];
    u.out_vel = c->hr_vel[cur ^ 1];
    u.m = c->n_high;
    u.lr_spos = c->lr_spos;
    u.lr_svel = c->lr_svel;
    u.cell_start = c->lr_cell_start;
    u.g = c->grid;
    u.r_low = c->r_low;
    u.r_high = c->r_high;
    u.dt = dt;
    u.gx = c->prm.gravity[0];
    u.gy = c->prm.gravity[1];
    u.gz = c->prm.gravity[2];
    u.c1 = c->prm.c1;
    u.c2 = c->prm.c2;
    u.sdf = c->d_sdf;
    u.n_sdf = c->n_sdf;
    {
        Timed t(c, GS_TIMER_GATHER);
        CK(gs_launch_upsample(c->stream, u, &c->launches), "upsample");
    }
    c->hr_cur = cur ^ 1;
    c->frame++;
    return GS_OK;
}

int gs_sync(gs_ctx* c)
{
    int st = check_state(c);
    if (st) return st;
    return report_device_errors(c);
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
