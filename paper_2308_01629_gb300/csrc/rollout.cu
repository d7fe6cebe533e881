// Differentiable rollout run by the library itself: frames of n_sub LR steps
// (Algorithm 1) and one HR frame (Sec. 4) from an initial state, keeping the
// state at every checkpoint_every-th frame; its backward recomputes each
// segment from its checkpoint with taped LR steps (the recorded passes kept
// for their reverse) and runs the reverse modes frame by frame, last to
// first.  The same functional entry points as a rollout driven from the
// caller, without a host round trip per operation in the caller's language:
// with graphs enabled the whole forward, and the whole backward, of one
// configuration are captured (on their second call; the first allocates
// what they need) and replayed as one CUDA graph each, on the context's
// own copies of the caller's buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gs.h"
#include "gs_internal.cuh"

namespace {

// a += b over n float4 records (the w components are left as they are)
__global__ void k_add4(float4* __restrict__ a, const float4* __restrict__ b, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 x = a[i], y = b[i];
    a[i] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w);
}

int grow(gs_ctx* c, float4** buf, int64_t* cap, int64_t need, const char* what)
{
    if (need <= *cap && *buf) return GS_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (gs_dalloc_bytes((void**)buf, (size_t)std::max<int64_t>(need, 1) * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return gs_ctx_fail(c, GS_ERR_OOM, what);
    }
    *cap = need;
    return GS_OK;
}

int copy(gs_ctx* c, float4* dst, const float4* src, int64_t n)
{
    if (n <= 0) return GS_OK;
    if (cudaMemcpyAsync(dst, src, (size_t)n * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return gs_ctx_fail(c, GS_ERR_CUDA, "rollout copy failed");
    }
    return GS_OK;
}

#define RO(call)                     \
    do {                             \
        const int st_ = (call);      \
        if (st_ != GS_OK) return st_; \
    } while (0)

struct RolloutCfg {
    float dt;
    int frames, n_sub, iters, every;
};

// The context's copies of the caller's buffers: ro_io holds eight fields,
// [0..3] the forward's initial state / the backward's final cotangents,
// [4..7] the forward's final state / the backward's initial gradients, each
// LR x, LR v, HR x, HR v.
float4* io(gs_ctx* c, int field)
{
    const int64_t N = c->n_low, M = c->n_high;
    const int64_t off[8] = {0, N, 2 * N, 2 * N + M, 2 * N + 2 * M, 3 * N + 2 * M, 4 * N + 2 * M, 4 * N + 3 * M};
    return c->ro_io + off[field];
}

int rollout_forward_body(gs_ctx* c, void* arg)
{
    const RolloutCfg& g = *(const RolloutCfg*)arg;
    const int64_t N = c->n_low, M = c->n_high, rec = 2 * N + 2 * M;
    float *lx = (float*)io(c, 4), *lv = (float*)io(c, 5), *hx = (float*)io(c, 6), *hv = (float*)io(c, 7);
    RO(copy(c, io(c, 4), io(c, 0), rec));   // the four fields are contiguous
    const float dts = g.dt / (float)g.n_sub;
    for (int f = 0; f < g.frames; ++f) {
        if (f % g.every == 0) RO(copy(c, c->ro_ckpt + (int64_t)(f / g.every) * rec, io(c, 4), rec));
        for (int s = 0; s < g.n_sub; ++s) RO(gs_step_low_forward(c, lx, lv, lx, lv, dts, g.iters));
        RO(gs_upsample_forward(c, lx, lv, hx, hv, hx, hv, g.dt));
    }
    return GS_OK;
}

int rollout_backward_body(gs_ctx* c, void* arg)
{
    const RolloutCfg& g = *(const RolloutCfg*)arg;
    const int64_t N = c->n_low, M = c->n_high, rec = 2 * N + 2 * M;
    const int frames = g.frames, n_sub = g.n_sub, iters = g.iters, every = g.every;
    const float dt = g.dt, dts = dt / (float)n_sub;
    const int k_max = std::min(every, std::max(frames, 1));
    const int64_t L0 = 0, H0 = L0 + (int64_t)(k_max * n_sub + 1) * 2 * N;
    const int64_t G0 = H0 + (int64_t)k_max * 2 * M;
    float4* W = c->ro_work;
    auto Lx = [&](int i) { return W + L0 + (int64_t)i * 2 * N; };
    auto Hx = [&](int j) { return W + H0 + (int64_t)j * 2 * M; };
    float4* gl = W + G0;            // cotangent of the LR state (x | v)
    float4* gl2 = gl + 2 * N;       // the LR step's input cotangent
    float4* gu = gl2 + 2 * N;       // the upsampling's LR gradient
    float4* gh = gu + 2 * N;        // cotangent of the HR state (x | v)
    float4* gh2 = gh + 2 * M;       // the upsampling's HR-input gradient
    RO(copy(c, gl, io(c, 0), 2 * N));
    RO(copy(c, gh, io(c, 2), 2 * M));
    // tags of the taped steps: the step's index in the rollout, above the
    // range a caller's own tags use
    const int64_t base = (int64_t)1 << 56;
    const int n_seg = (frames + every - 1) / every;
    for (int seg = n_seg - 1; seg >= 0; --seg) {
        const int f0 = seg * every, k = std::min(every, frames - f0);
        const float4* ck = c->ro_ckpt + (int64_t)seg * rec;
        RO(copy(c, Lx(0), ck, 2 * N));
        RO(copy(c, Hx(0), ck + 2 * N, 2 * M));
        // recompute the segment, LR steps taped
        for (int j = 0; j < k; ++j) {
            for (int s = 0; s < n_sub; ++s) {
                float4* in = Lx(j * n_sub + s);
                float4* out = Lx(j * n_sub + s + 1);
                RO(gs_step_low_forward_taped(c, (const float*)in, (const float*)(in + N), (float*)out,
                                             (float*)(out + N), dts, iters, base + (int64_t)(f0 + j) * n_sub + s));
            }
            if (j + 1 < k) {
                const float4* lr = Lx((j + 1) * n_sub);
                RO(gs_upsample_forward(c, (const float*)lr, (const float*)(lr + N), (const float*)Hx(j),
                                       (const float*)(Hx(j) + M), (float*)Hx(j + 1), (float*)(Hx(j + 1) + M), dt));
            }
        }
        // the frames in reverse
        for (int j = k - 1; j >= 0; --j) {
            const float4* lr = Lx((j + 1) * n_sub);
            RO(gs_upsample_backward(c, (const float*)lr, (const float*)(lr + N), (const float*)Hx(j),
                                    (const float*)(Hx(j) + M), (const float*)gh, (const float*)(gh + M), (float*)gu,
                                    (float*)(gu + N), (float*)gh2, (float*)(gh2 + M), dt));
            k_add4<<<gs_blocks(2 * N, 256), 256, 0, c->stream>>>(gl, gu, 2 * N);
            if (cudaGetLastError() != cudaSuccess) return gs_ctx_fail(c, GS_ERR_CUDA, "rollout add failed");
            c->launches += 1;
            std::swap(gh, gh2);
            for (int s = n_sub - 1; s >= 0; --s) {
                const int64_t tag = base + (int64_t)(f0 + j) * n_sub + s;
                int st = gs_step_low_backward_taped(c, tag, (const float*)gl, (const float*)(gl + N), (float*)gl2,
                                                    (float*)(gl2 + N));
                if (st == GS_ERR_STATE) {   // the record is gone: record the step again
                    const float4* in = Lx(j * n_sub + s);
                    st = gs_step_low_backward(c, (const float*)in, (const float*)(in + N), (const float*)gl,
                                              (const float*)(gl + N), (float*)gl2, (float*)(gl2 + N), dts, iters);
                }
                if (st != GS_OK) return st;
                std::swap(gl, gl2);
            }
        }
    }
    RO(copy(c, io(c, 4), gl, 2 * N));
    RO(copy(c, io(c, 6), gh, 2 * M));
    return GS_OK;
}

uint64_t rollout_key(const gs_ctx* c, char kind, const RolloutCfg& g)
{
    uint64_t k = gs_sequence_key(c, kind, g.dt, g.iters);
    for (uint64_t v : {(uint64_t)g.frames, (uint64_t)g.n_sub, (uint64_t)g.every}) k = (k ^ v) * 0x100000001b3ull;
    return k;
}

// The first call of a configuration runs directly (it allocates what the
// sequence needs); later calls are captured once and replayed.
int run_sequence(gs_ctx* c, uint64_t key, int (*body)(gs_ctx*, void*), void* arg)
{
    if (std::find(c->ro_seen.begin(), c->ro_seen.end(), key) == c->ro_seen.end()) {
        c->ro_seen.push_back(key);
        return body(c, arg);
    }
    return gs_replay_or_run(c, key, body, arg);
}

}  // namespace

extern "C" int gs_rollout_forward(gs_ctx* c, const float* lr_x0, const float* lr_v0, const float* hr_x0,
                                  const float* hr_v0, float dt, int frames, int n_sub, int iters, int checkpoint_every,
                                  float* lr_x, float* lr_v, float* hr_x, float* hr_v)
{
    if (!c) return GS_ERR_ARG;
    if (!(dt > 0.0f) || frames < 0 || frames > 100000 || n_sub < 1 || n_sub > 1000 || iters < 0 || iters > 1000 ||
        checkpoint_every < 1)
        return gs_ctx_fail(c, GS_ERR_ARG, "invalid rollout arguments");
    if (c->n_scenes != 1) return gs_ctx_fail(c, GS_ERR_STATE, "the rollout needs a single-scene context");
    const int64_t N = c->n_low, M = c->n_high;
    if (!lr_x0 || !lr_v0 || !hr_x0 || !hr_v0 || !lr_x || !lr_v || !hr_x || !hr_v)
        return gs_ctx_fail(c, GS_ERR_ARG, "null buffer");
    c->ro_valid = false;
    const int64_t rec = 2 * N + 2 * M;                                    // one state
    const int n_ckpt = (frames + checkpoint_every - 1) / checkpoint_every;  // segment starts
    int64_t cap_io = 0;
    if (c->ro_io) cap_io = 4 * rec;
    RO(grow(c, &c->ro_io, &cap_io, 4 * rec, "no memory for the rollout's buffers"));
    if (c->ro_ckpt_cap < (int64_t)std::max(n_ckpt, 1) * rec) c->ro_seen.clear();   // buffers move: capture anew
    RO(grow(c, &c->ro_ckpt, &c->ro_ckpt_cap, (int64_t)std::max(n_ckpt, 1) * rec, "no memory for the checkpoints"));
    RO(copy(c, io(c, 0), (const float4*)lr_x0, N));
    RO(copy(c, io(c, 1), (const float4*)lr_v0, N));
    RO(copy(c, io(c, 2), (const float4*)hr_x0, M));
    RO(copy(c, io(c, 3), (const float4*)hr_v0, M));
    RolloutCfg g{dt, frames, n_sub, iters, checkpoint_every};
    RO(run_sequence(c, rollout_key(c, 'R', g), rollout_forward_body, &g));
    RO(copy(c, (float4*)lr_x, io(c, 4), N));
    RO(copy(c, (float4*)lr_v, io(c, 5), N));
    RO(copy(c, (float4*)hr_x, io(c, 6), M));
    RO(copy(c, (float4*)hr_v, io(c, 7), M));
    c->ro_valid = true;
    c->ro_dt = dt;
    c->ro_frames = frames;
    c->ro_n_sub = n_sub;
    c->ro_iters = iters;
    c->ro_every = checkpoint_every;
    return GS_OK;
}

extern "C" int gs_rollout_backward(gs_ctx* c, const float* g_lr_x, const float* g_lr_v, const float* g_hr_x,
                                   const float* g_hr_v, float* g_lr_x0, float* g_lr_v0, float* g_hr_x0,
                                   float* g_hr_v0)
{
    if (!c) return GS_ERR_ARG;
    if (!c->ro_valid) return gs_ctx_fail(c, GS_ERR_STATE, "no rollout forward to differentiate");
    if (!g_lr_x || !g_lr_v || !g_hr_x || !g_hr_v || !g_lr_x0 || !g_lr_v0 || !g_hr_x0 || !g_hr_v0)
        return gs_ctx_fail(c, GS_ERR_ARG, "null buffer");
    const int64_t N = c->n_low, M = c->n_high;
    RolloutCfg g{c->ro_dt, c->ro_frames, c->ro_n_sub, c->ro_iters, c->ro_every};
    const int k_max = std::min(g.every, std::max(g.frames, 1));
    const int64_t need = (int64_t)(k_max * g.n_sub + 1) * 2 * N + (int64_t)k_max * 2 * M + 3 * 2 * N + 2 * 2 * M;
    if (c->ro_work_cap < need) c->ro_seen.clear();   // buffers move: capture anew
    RO(grow(c, &c->ro_work, &c->ro_work_cap, need, "no memory for the rollout's backward"));
    if ((int)c->tapes.size() < k_max * g.n_sub) {
        c->ro_seen.clear();
        RO(gs_set_step_tapes(c, k_max * g.n_sub));
    }
    RO(copy(c, io(c, 0), (const float4*)g_lr_x, N));
    RO(copy(c, io(c, 1), (const float4*)g_lr_v, N));
    RO(copy(c, io(c, 2), (const float4*)g_hr_x, M));
    RO(copy(c, io(c, 3), (const float4*)g_hr_v, M));
    const int st = run_sequence(c, rollout_key(c, 'Q', g), rollout_backward_body, &g);
    // the sequence used the tape slots (a replay does so without the host's
    // bookkeeping): no kept record is valid for a caller afterwards
    for (auto& t : c->tapes) t.tag = -1;
    if (st != GS_OK) return st;
    RO(copy(c, (float4*)g_lr_x0, io(c, 4), N));
    RO(copy(c, (float4*)g_lr_v0, io(c, 5), N));
    RO(copy(c, (float4*)g_hr_x0, io(c, 6), M));
    RO(copy(c, (float4*)g_hr_v0, io(c, 7), M));
    return GS_OK;
}
