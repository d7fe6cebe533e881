// gs_internal.cuh -- context layout and launch helpers shared by the CUDA
// translation units of the library (not part of the public ABI).
//
// A context holds S >= 1 independent scenes.  Their particles are stored
// back to back (LR scene-major; HR scene-major with every scene's slots
// starting on a multiple of 32 so a warp never spans two scenes), and their
// grids share one concatenated cell index space: scene s owns the global
// cells [cell_off, cell_off + n_cell] where the last one is a padding cell
// that only HR padding slots use.  Sorting by global key therefore keeps
// every scene's particles inside its own slot range.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "gs.h"

// Dense-grid contract (see gs.h): origin, cell side, inverse, dimensions.
struct GridDev {
    float ox, oy, oz;
    float h, inv_h;
    int dx, dy, dz;
};

// Per-scene descriptor, read by every kernel.
struct SceneDev {
    GridDev g;
    uint32_t cell_off;       // first global cell id of the scene
    uint32_t n_cell;         // real cells (a padding cell follows)
    int64_t lr_begin, lr_end;
    int64_t hr_begin, hr_end;    // real HR slots; [hr_end, next hr_begin) is padding
    int64_t hr_real_begin;       // original id of the scene's first HR particle
    int64_t warp_begin;          // first global warp item of the scene
    float r_low, r_high;
    float gx, gy, gz;
    float mu_s, mu_k, c1, c2;
    float mass_k, ground_z, rc;
    int friction_mode;
    int sdf_begin, n_sdf;        // into the context's SDF table
};

// Device-side error bits, reported by the next blocking call.
enum : int {
    GS_DEVERR_NEIGHBOR_CAP = 1,   // an LR particle had more candidates than max_neighbors
    GS_DEVERR_BAD_ID = 2,         // an HR id outside [0, n_high) was met while unpermuting
    GS_DEVERR_BARRIER_TIMEOUT = 4,   // a grid barrier of the persistent LR solver gave up waiting
    GS_DEVERR_NONFINITE_ASYNC = 8,   // an asynchronously written field held a non-finite value
    GS_DEVERR_SOLID_REVERSE = 16,    // a reverse mode met LR particles of infinite mass
};

// HR slot tag: scene index, with this bit set on padding slots.
constexpr uint32_t kPadBit = 0x80000000u;

// Host-side bookkeeping a captured sequence leaves behind (applied again on
// every replay of the functional entry points' graphs).
struct HostAfter {
    int hr_cur = 0;
    bool hr_identity = true, hr_keys_valid = false, lr_binned = false;
    uint32_t* hr_sorted_keys = nullptr;
    uint32_t* lr_sorted_keys = nullptr;
    uint32_t* lr_sorted_idx = nullptr;
};

struct GraphEntry {
    uint64_t key = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;    // kernel launches the graph replays
    cudaGraph_t graph = nullptr;   // kept with the exec when it holds a conditional node
    HostAfter after;        // functional entry points: the state after the sequence
};

// Device state of an adaptive frame's LR substeps (gs_frame_adaptive).
struct CflState {
    float t_rem;                     // frame time left
    float dt;                        // the current LR step, read by the step's kernels
    unsigned rate;                   // max |v| / (2 r_LR) as float bits, accumulated by the step's finalize
    int taken;                       // LR steps taken in this frame
    int more;                        // 1 while another step follows (read by the host-driven loop)
    int pad;
    unsigned long long kernels;      // kernel launches of device-looped steps, for the launch count
    float log[GS_MAX_SUBSTEPS];      // the frame's step lengths
};

struct gs_ctx {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // pipelined frames: the HR frame of frame f runs on stream_hr while the
    // LR steps of frame f + 1 run on stream (fork / join by events)
    cudaStream_t stream_hr = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // gs_set_gather_timer: events around the gather launches, recorded by
    // direct frames and by every replay of captured frames
    cudaEvent_t ev_gather[2] = {nullptr, nullptr};
    bool pipeline = false;
    int pipe_warps = 8, pipe_blocks_per_sm = 1;   // gather launch shape while it overlaps the LR steps
    bool pending = false;        // an HR frame is deferred
    float pend_dt = 0.0f;
    bool pend_resort = false;
    gs_sdf* d_sdf_pend = nullptr;   // the SDF table as of the deferred frame
    int device = 0;

    int n_scenes = 1;
    std::vector<SceneDev> scenes;       // host copy of the descriptor table
    std::vector<gs_params> prm;         // per scene, resolved defaults
    std::vector<gs_sdf> sdf_host;       // all scenes' SDFs back to back
    SceneDev* d_scenes = nullptr;
    gs_sdf* d_sdf = nullptr;

    int64_t n_low = 0;                  // LR particles, all scenes
    int64_t n_high = 0;                 // real HR particles, all scenes
    int64_t hr_slots = 0;               // HR slots including padding
    int64_t n_warps = 0;                // HR warp items (32 slots each)
    int64_t n_cell_total = 0;           // global cells incl. one padding cell per scene
    int lr_key_bits = 0, hr_key_bits = 0;
    int resort_every = 8;
    int nbr_cap = 64;
    int n_stab = 2;

    uint32_t* lr_scene = nullptr;       // scene of each LR slot (same in original and cell order)
    uint32_t* hr_scene = nullptr;       // scene of each HR slot | kPadBit on padding

    // LR state (original order) and the binning view
    float4* lr_pos = nullptr;
    float4* lr_vel = nullptr;
    uint32_t* lr_keys[2] = {nullptr, nullptr};   // counting sort: [0] cell keys, [1] keys in cell order
    uint32_t* lr_vals[2] = {nullptr, nullptr};   // [0] arrival ranks, [1] particle indices in cell order
    uint32_t* lr_sorted_keys = nullptr;           // lr_keys[1] after a binning
    uint32_t* lr_sorted_idx = nullptr;            // lr_vals[1] after a binning
    uint32_t* lr_cell_start = nullptr;            // n_cell_total + 1 (upsampling view)
    uint32_t* step_cell_start = nullptr;          // n_cell_total + 1 (binning of x~ in the LR step)
    uint32_t* scan_aux = nullptr;                 // tile sums of the cell-start scan
    float4* lr_spos = nullptr;                    // cell-ordered LR position (upsampling view)
    float4* lr_svel = nullptr;                    // cell-ordered LR velocity
    bool lr_binned = false;

    // LR step buffers (cell order)
    float4* s_xt[2] = {nullptr, nullptr};
    float4* s_x[2] = {nullptr, nullptr};
    float4* lr_xt = nullptr;                      // predicted positions, original order
    uint32_t* nbr = nullptr;                      // [cap][n_low] candidate slots

    // grain materials (per-particle friction); off while n_materials == 0
    int n_materials = 0;
    uint32_t mat_max_id = 0;                      // largest material id stored in lr_mat
    uint32_t* lr_mat = nullptr;                   // n_low material ids, original order (in the LR
                                                  // step they ride in the w of the cell-ordered x)
    float2* d_mu = nullptr;                       // [GS_MAX_MATERIALS] (mu_s, mu_k), then the
                                                  // [GS_MAX_MATERIALS^2] cross coefficients
    float2 h_mu[GS_MAX_MATERIALS * (GS_MAX_MATERIALS + 1)];   // host copy of d_mu

    // rigid bodies (shape matching); off while n_bodies == 0
    int n_bodies = 0;
    uint32_t* lr_body = nullptr;        // n_low body ids (0: a grain), original order
    float4* lr_xo = nullptr;            // n_low rest offsets from the body's centre of mass, w = mass
    uint32_t* body_members = nullptr;   // the particles of body 1, body 2, ... (original indices)
    uint32_t* body_start = nullptr;     // GS_MAX_BODIES + 1 offsets into body_members
    float4* body_xf = nullptr;          // 4 per body: (R_r0, R_r1, R_r2, c_r) for r = 0..2, quaternion
    uint32_t* lr_slot = nullptr;        // n_low: slot of each particle in the LR step's cell order
    uint32_t* nbr_cnt = nullptr;

    // HR state (internal order), ping-pong
    float4* hr_pos[2] = {nullptr, nullptr};
    float4* hr_vel[2] = {nullptr, nullptr};
    int hr_cur = 0;
    // HR slab (gs_set_hr_slab): the HR frames update warp items
    // [slab_item_begin, slab_item_end) only; hr_partial: the slots outside
    // were not updated by the latest frames (until gs_hr_slab_assemble)
    int slab_parts = 1;
    int64_t slab_item_begin = 0, slab_item_end = 0;
    bool hr_partial = false;
    float4* slab_stage = nullptr;       // 2 x hr_slots, for host sources of gs_hr_slab_assemble
    bool hr_identity = true;
    uint32_t* hr_keys[2] = {nullptr, nullptr};
    uint32_t* hr_vals[2] = {nullptr, nullptr};
    uint32_t* hr_sorted_keys = nullptr;
    bool hr_keys_valid = false;
    // HR reorder by counting sort over the fine cells (hr_bins = 8 x cells
    // keys), chosen when that key space is not much larger than the HR set;
    // otherwise the radix sort.  hr_bin_start: counts, then cell starts
    // (hr_bins + 1 words) and the count of listed big cells; hr_big: the list.
    bool hr_counting = false;
    int64_t hr_bins = 0;
    uint32_t* hr_bin_start = nullptr;
    uint32_t* hr_big = nullptr;
    uint32_t* hr_scan_aux = nullptr;
    float4* tmp4 = nullptr;                       // staging for reads / writes
    float4* stage_in = nullptr;                   // host data written in, checked on the device
    // asynchronous field I/O (LR_POS, LR_VEL, HR_POS, HR_VEL): host -> device
    // copies on stream_h2d into async_in, committed in stream order before
    // the next call that reads the state; device -> host copies of a
    // snapshot (async_out) on stream_d2h
    cudaStream_t stream_h2d = nullptr, stream_d2h = nullptr;
    float4* async_in[4] = {nullptr, nullptr, nullptr, nullptr};
    float4* async_out[4] = {nullptr, nullptr, nullptr, nullptr};
    // An asynchronous read of one HR field snapshots both; the other's
    // snapshot (field hr_pair_field) serves its own read if no kernel was
    // launched in between (launch count hr_pair_launches).
    int hr_pair_field = -1;
    int64_t hr_pair_launches = -1;
    cudaEvent_t ev_in_ready[4] = {}, ev_in_free[4] = {}, ev_out_ready[4] = {}, ev_out_free[4] = {};
    bool in_pending[4] = {false, false, false, false};
    bool in_used[4] = {false, false, false, false}, out_used[4] = {false, false, false, false};

    // reverse-mode scratch: LR gradients in cell order
    float4* gXs = nullptr;
    float4* gVs = nullptr;
    // LR-step reverse mode: per-pass snapshots (allocated on first use)
    float4* snap = nullptr;        // [n_pass_cap][n_low] positions each pass evaluates on
    float4* snap_xt = nullptr;     // [n_pass_cap][n_low] xt at each pass input
    int snap_cap = 0;
    // taped LR steps (gs_set_step_tapes): each slot keeps what a recorded
    // forward step evaluated on -- the pass snapshots, the candidate lists
    // and the cell order -- for the step's backward without recomputation
    struct StepTape {
        int64_t tag = -1;          // the caller's tag; -1: empty
        int64_t serial = -1;       // order of recording (the latest of equal tags wins)
        float dt = 0.0f;
        int iters = 0;
        float4* X = nullptr;       // [tape_passes + 1][n_low], as snap
        float4* XT = nullptr;      // [tape_passes + 1][n_low], as snap_xt
        uint32_t* nbr = nullptr;   // [nbr_cap][n_low]
        uint32_t* cnt = nullptr;   // [n_low]
        uint32_t* idx = nullptr;   // [n_low] particle of each cell-ordered slot
    };
    std::vector<StepTape> tapes;
    // native differentiable rollout (gs_rollout_forward / _backward): the
    // checkpoints of the latest forward and the backward's scratch
    float4* ro_ckpt = nullptr;       // [n_ckpt][2 n_low + 2 n_high]
    int64_t ro_ckpt_cap = 0;         // float4 records
    float4* ro_work = nullptr;       // a segment's states and the gradients
    int64_t ro_work_cap = 0;
    float4* ro_io = nullptr;         // the rollout's own copies of the caller's buffers (8 fields)
    bool ro_valid = false;
    bool capturing = false;          // a sequence is being captured: inner sequences run directly
    std::vector<uint64_t> ro_seen;   // rollout sequences run once directly (captured on the next call)
    float ro_dt = 0.0f;
    int ro_frames = 0, ro_n_sub = 0, ro_iters = 0, ro_every = 0;
    int64_t ro_serial = 0;
    int tape_passes = 0;
    int64_t tape_serial = 0;
    int tape_next = 0;
    float4* adj_gx = nullptr;
    float4* adj_gxt = nullptr;
    float4* adj_h = nullptr;
    float4* adj_h2 = nullptr;      // the next pass's h (the reverse passes alternate the two)
    bool det_bwd = false;          // gs_set_deterministic_backward
    float4* det_coef = nullptr;    // [3 n_high] the HR particles' coefficients and positions in cell order
                                   // (deterministic backward)
    uint32_t* det_big = nullptr;   // its HR binning's list of cells of more than 32, then their count
    float* adj_gws = nullptr;
    float4* adj_io = nullptr;      // [4][n_low]: dL/dx_out, dL/dv_out in; dL/dx_in, dL/dv_in out (original order)
    float4* fscratch = nullptr;    // [6][n_high] + [2][n_low]: the functional upsampling entries' in/out copies
    // decision record of the reverse modes (gs_set_decision_record); null: off
    uint32_t* rec_hr = nullptr;
    int32_t* rec_lr_cand = nullptr;
    uint8_t* rec_lr_pair = nullptr;
    uint8_t* rec_lr_sdf = nullptr;
    int rec_max_passes = 0;
    std::vector<GraphEntry> fgraphs;   // graphs of the functional LR step entry points

    // radix sort histogram scratch (HR reorder, static-scratch binning)
    uint32_t* sort_hist = nullptr;
    size_t sort_hist_cap = 0;

    // persistent upsampling: work counter and launch shape (autotuned)
    unsigned* d_work = nullptr;
    int tune_warps = 8;          // warps per block
    int tune_blocks_per_sm = 0;  // 0: one warp item per warp (grid launch); else persistent
    int sm_count = 152;

    // CUDA graphs of whole frames
    bool use_graphs = false;
    std::vector<GraphEntry> graphs;
    // adaptive frames: device control block, kernel credit folded so far
    CflState* d_cfl = nullptr;
    unsigned long long cfl_kernels_seen = 0;
    bool cfl_used = false;

    // errors
    int* d_err = nullptr;
    unsigned* d_bar = nullptr;   // grid-barrier words of the persistent LR solver
    int solve_blocks = 0;        // resident blocks of the solver; 0 = per-pass launches
    bool use_solver = false;    // per-pass launches by default: faster under graph replay
    bool solver_selftest = false;   // the barrier waits for one block that does not exist
    int* h_err = nullptr;                         // pinned
    std::string last_error;
    bool poisoned = false;

    int64_t frame = 0;
    int64_t launches = 0;

    // timing
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[GS_TIMER_COUNT];
};

// ---- launchers implemented in the .cu files --------------------------------
// sort.cu
size_t gs_sort_hist_words(int64_t n);
int gs_key_bits(int64_t n_keys);
// Stable LSD radix sort of (keys, vals) by the low key_bits bits; the result
// lands in keys[*which] / vals[*which] (which is flipped once per pass).
cudaError_t gs_radix_sort(cudaStream_t s, uint32_t* keys[2], uint32_t* vals[2], int* which, uint32_t* hist,
                          int64_t n, int key_bits, int64_t* launches);
// Cell keys of one grid (single-grid form, used by gs_bin_points_static).
cudaError_t gs_launch_cell_keys(cudaStream_t s, const float4* pos, int64_t n, GridDev g, int fine, uint32_t* keys,
                                uint32_t* vals, int64_t* launches);
// Cell keys of slots that belong to several scenes: scene of slot i is
// tag[i] & ~kPadBit; padding slots get the scene's padding cell.
// Stable counting sort of n items by the cell of their position (coarse
// keys): out_keys / out_idx in ascending (cell, item) order and cell_start
// (n_cell + 1 entries) the start of every cell.  aux holds
// gs_scan_aux_words(n_cell + 1) words.
size_t gs_scan_aux_words(int64_t total);
// The same sort in stages, so that the keys can come from a fused kernel:
// clear the counts, count (keys + arrival ranks; gs_cs_keys or a kernel
// that does the same with grid_cell_of), then scan + scatter + per-cell
// order; finish also copies ga / gb (when not null) into cell order.
// Zeroes the n_cell + 1 cell starts and `extra` words after them.
cudaError_t gs_cs_clear(cudaStream_t s, uint32_t* cell_start, int64_t n_cell, int extra = 0);
// solid_flag (optional): set to 1 when some position has w = 0 or, with
// body not null, some particle belongs to a rigid body.
cudaError_t gs_cs_keys(cudaStream_t s, const float4* pos, int64_t n, const SceneDev* scenes, const uint32_t* tag,
                       uint32_t* keys, uint32_t* rank, uint32_t* cell_start, int64_t* launches,
                       unsigned* solid_flag = nullptr, const uint32_t* body = nullptr);
// Optional work of the cell-order copy (all null: none).
struct CsExtras {
    const uint32_t* gb_w = nullptr;       // the w of gb's copies is gb_w[particle] (as bits)
    const uint32_t* ga_solid = nullptr;   // nonzero: the w of ga's copy is 0
    uint32_t* slot_of = nullptr;          // slot_of[particle] = its slot
    // Cells of more than 32 entries (big_list not null; only without copies):
    // listed in big_list (capacity n / 33 + 1, count in *big_count, zero on
    // entry) and ordered afterwards by big_blocks cooperating blocks, each
    // cell by LSD passes over its item indices (< 2^big_bits) through
    // big_scratch (n words; its cells' ranges are overwritten).  Without a
    // list the warp that meets such a cell orders it (through the ranks).
    uint32_t* big_list = nullptr;
    uint32_t* big_count = nullptr;
    uint32_t* big_scratch = nullptr;
    int big_bits = 32;
    int big_blocks = 0;
};
// ga and gb are copied into cell order: x_out[slot] = x[particle of the
// slot], with the extras above.  rank is overwritten where cells of more
// than 256 entries are ordered (it is dead once scattered).
cudaError_t gs_cs_finish(cudaStream_t s, int64_t n, int64_t n_cell, const uint32_t* keys, uint32_t* rank,
                         uint32_t* out_keys, uint32_t* out_idx, uint32_t* cell_start, uint32_t* aux, const float4* ga,
                         const float4* gb, float4* ga_out, float4* gb_out, int64_t* launches,
                         const CsExtras& ex = CsExtras{});
cudaError_t gs_count_sort_cells(cudaStream_t s, const float4* pos, int64_t n, const SceneDev* scenes,
                                const uint32_t* tag, int64_t n_cell, uint32_t* keys, uint32_t* rank,
                                uint32_t* out_keys, uint32_t* out_idx, uint32_t* cell_start, uint32_t* aux,
                                int64_t* launches);
// vals[i] = i, or with count not null the arrival rank of slot i in its
// key's counter (count[key] += 1), for a counting sort by key.
cudaError_t gs_launch_scene_keys(cudaStream_t s, const float4* pos, int64_t n, const SceneDev* scenes,
                                 const uint32_t* tag, int fine, uint32_t* keys, uint32_t* vals, int64_t* launches,
                                 uint32_t* count = nullptr);
cudaError_t gs_launch_cell_start(cudaStream_t s, const uint32_t* sorted_keys, int64_t n, int64_t n_cell,
                                 uint32_t* start, int64_t* launches);
cudaError_t gs_launch_gather2(cudaStream_t s, const uint32_t* idx, const float4* a, const float4* b, float4* a_out,
                              float4* b_out, int64_t n, int64_t* launches);
cudaError_t gs_launch_unpermute(cudaStream_t s, const float4* pos_internal, const float4* field_internal,
                                const uint32_t* hr_tag, float4* out, int64_t n_slots, int64_t n_real, int* err,
                                int64_t* launches);
// Both HR fields to original-id order in one pass (out_pos[id] = pos[p],
// out_vel[id] = vel[p]).
cudaError_t gs_launch_unpermute2(cudaStream_t s, const float4* pos_internal, const float4* vel_internal,
                                 const uint32_t* hr_tag, float4* out_pos, float4* out_vel, int64_t n_slots,
                                 int64_t n_real, int* err, int64_t* launches);
cudaError_t gs_launch_permute_in(cudaStream_t s, const float4* pos_internal, const float4* field_original,
                                 const uint32_t* hr_tag, float4* out, int64_t n_slots, int64_t n_real, int* err,
                                 int64_t* launches);
cudaError_t gs_launch_check_finite(cudaStream_t s, const float4* a, int64_t n, int* flag, int64_t* launches,
                                   int bit = 1);

// upsample.cu
struct UpsampleArgs {
    const float4* hr_pos;
    const float4* hr_vel;
    float4* out_pos;
    float4* out_vel;
    const float4* lr_spos;
    const float4* lr_svel;
    const uint32_t* cell_start;
    const SceneDev* scenes;
    const uint32_t* hr_tag;
    const gs_sdf* sdf;
    int n_scenes;
    int64_t n_warps;           // warp items
    int64_t item_begin;        // first item: the launch covers items [item_begin, item_begin + n_warps)
    unsigned* work;            // persistent mode: next warp item (zeroed before the launch)
    const unsigned* solid_flag;   // nonzero: some LR particle has w = 0 (set by the LR binning)
    float dt;
};
// blocks_per_sm == 0: one warp per item; else a persistent grid of
// blocks_per_sm blocks per SM pulling items from *work (bounded loop).
cudaError_t gs_launch_upsample(cudaStream_t s, const UpsampleArgs& a, int warps_per_block, int blocks_per_sm,
                               int sm_count, int64_t* launches);

// pbd.cu
struct PbdArgs {
    int64_t n;
    float dt;
    const float* dt_dev;   // not null: the step length is *dt_dev (adaptive frames), not dt
    const SceneDev* scenes;
    const uint32_t* lr_scene;
    const gs_sdf* sdf;
    // grain materials: null for the scenes' coefficients; else the table
    // (mu_s, mu_k) per material and the cross coefficients
    // [m_i * GS_MAX_MATERIALS + m_j].  With materials the w of the
    // cell-ordered x holds the particle's material id (as bits) instead of
    // its inverse mass, which the step's finalize reads from the
    // original-order positions.
    const float2* mu_mat;
    const float2* mu_cross;
    // rigid bodies: null without; else the body of each particle (original
    // order), rest offsets (w = mass), per-body transforms of the current
    // pass (k_body_xform) and the particle of each slot of the step's order
    const uint32_t* body;
    const float4* xo;
    const float4* body_xf;
    const uint32_t* sorted_idx;
};
cudaError_t gs_launch_predict(cudaStream_t s, const PbdArgs& a, const float4* pos, const float4* vel, float4* xt,
                              int64_t* launches);
cudaError_t gs_launch_step_gather(cudaStream_t s, int64_t n, const uint32_t* idx, const float4* xt,
                                  const float4* pos, float4* s_xt, float4* s_x, int64_t* launches);
cudaError_t gs_launch_neighbors(cudaStream_t s, const PbdArgs& a, const float4* s_xt, const uint32_t* skeys,
                                const uint32_t* cell_start, int64_t n_cell, uint32_t* nbr, uint32_t* cnt, int cap,
                                int* err, int64_t* launches);
// One Jacobi pass.  With fin_idx not null the pass is the step's last: it
// writes the finalized position and velocity to original order (fin_pos,
// fin_vel through fin_idx) instead of x_out / xt_out.
// fin_rate (not null, last pass only): atomic max of |v| / (2 r_LR) of the
// finalized velocities, as float bits.
cudaError_t gs_launch_pass(cudaStream_t s, const PbdArgs& a, int stab, const float4* x_in, const float4* xt_in,
                           float4* x_out, float4* xt_out, const uint32_t* nbr, const uint32_t* cnt,
                           int64_t* launches, const uint32_t* fin_idx = nullptr, float4* fin_pos = nullptr,
                           float4* fin_vel = nullptr, unsigned* fin_rate = nullptr);
// Prediction + cell keys + arrival ranks (the counting stage of the binning).
cudaError_t gs_launch_predict_keys(cudaStream_t s, const PbdArgs& a, const float4* pos, const float4* vel,
                                   float4* xt, uint32_t* keys, uint32_t* rank, uint32_t* cnt, int64_t* launches);
// All n_stab + iters passes of one step in one cooperative launch of at most
// max_blocks blocks (gs_solve_blocks: the blocks that fit on the GPU at
// once), with grid barriers between passes.  bar: two words of scratch.
// The result lands where the per-pass loop would leave it.
int gs_solve_blocks(int sm_count);
cudaError_t gs_launch_solve(cudaStream_t s, const PbdArgs& a, int n_stab, int iters, float4* x[2], float4* xt[2],
                            const uint32_t* nbr, const uint32_t* cnt, unsigned* bar, int* err, int max_blocks,
                            int64_t* launches, unsigned extra_arrivals = 0);
cudaError_t gs_launch_finalize(cudaStream_t s, const PbdArgs& a, const uint32_t* idx, const float4* s_x,
                               const float4* s_xt, float4* pos, float4* vel, int64_t* launches,
                               unsigned* rate = nullptr);
// CFL-limited substeps (gs_frame_adaptive): reset the control block for a
// frame of t seconds; the largest |v| / (2 r_LR) of vel into st->rate; pick
// the next step (and, in a graph, set the while node's condition).
cudaError_t gs_launch_cfl_begin(cudaStream_t s, CflState* st, float t, int64_t* launches);
// Shape matching (Sec. 3): for each of n_bodies bodies, c and the rotation
// R of C = sum m (x~ - c) xo^T from the pass's cell-ordered positions xt
// (slot_of maps particles to slots), into xf (4 float4 per body; the
// quaternion entry is also the start of the next extraction).
cudaError_t gs_launch_body_xform(cudaStream_t s, int n_bodies, const uint32_t* start, const uint32_t* members,
                                 const uint32_t* slot_of, const float4* xt, const float4* xo, float4* xf,
                                 int64_t* launches);
cudaError_t gs_launch_cfl_rate(cudaStream_t s, const PbdArgs& a, const float4* vel, unsigned* rate,
                               int64_t* launches);
cudaError_t gs_launch_cfl_pick(cudaStream_t s, CflState* st, float dt_max, float cfl, int max_sub,
                               cudaGraphConditionalHandle h, int in_graph, unsigned body_kernels, int64_t* launches);

// adjoint.cu
// rec (optional): uint32[m][4] decisions of the HR frame's reverse mode in
// original LR indices (lr_idx: cell-ordered slot -> LR particle).
cudaError_t gs_launch_upsample_bwd(cudaStream_t s, const SceneDev* scenes, const gs_sdf* sdf, const float4* lr_spos,
                                   const float4* lr_svel, const uint32_t* cell_start, const float4* hx,
                                   const float4* hv, const float4* gxo, const float4* gvo, float4* ghx, float4* ghv,
                                   float4* gXs, float4* gVs, int64_t m, float dt, int64_t* launches,
                                   uint32_t* rec = nullptr, const uint32_t* lr_idx = nullptr,
                                   float4* coef = nullptr, const uint32_t* order = nullptr,
                                   float4* pos_sorted = nullptr);
// coef (not null): instead of adding into gXs / gVs, the HR particles are
// taken in the order `order` (slot -> particle: HR binned by the LR cells)
// and every one's coefficients go to coef[2 slot ..] and its position to
// pos_sorted[slot]; k_upsample_bwd_lr then gathers them per LR slot
// (hr_cell_start: the HR binning's cell starts; lr_skeys: the LR slots'
// cells).
cudaError_t gs_launch_upsample_bwd_lr(cudaStream_t s, const SceneDev* scenes, const float4* lr_spos,
                                      const float4* lr_svel, const uint32_t* lr_skeys, const float4* hx_sorted,
                                      const uint32_t* hr_cell_start, const float4* coef, float4* gXs, float4* gVs,
                                      int64_t n_low, int64_t* launches);
// Decisions of one pass of the LR step's reverse mode, in original particle
// order (idx: slot -> particle): cand / pair [cap][n], sdf [n][n_comp]
// (gs_set_decision_record).  All null: nothing is recorded.
struct AdjRecord {
    const uint32_t* idx = nullptr;
    int32_t* cand = nullptr;
    uint8_t* pair = nullptr;
    uint8_t* sdf = nullptr;
    int cap = 0;
    int n_comp = 0;
};
cudaError_t gs_launch_scatter2(cudaStream_t s, const uint32_t* idx, const float4* a, const float4* b, float4* ao,
                               float4* bo, int64_t n, int64_t* launches);
cudaError_t gs_launch_adj_init(cudaStream_t s, int64_t n, const uint32_t* idx, const float4* gxo, const float4* gvo,
                               float dt, float4* gx, float4* gxt, float* gws, int64_t* launches);
// h = upstream / n per particle for one pass (the first pass to reverse).
cudaError_t gs_launch_adj_h(cudaStream_t s, const PbdArgs& a, int stab, const float4* Y, const float4* WS,
                            const uint32_t* nbr, const uint32_t* cnt, const float4* gx, const float4* gxt, float4* H,
                            int64_t* launches);
// The reverse of one pass from its h (H); with Y_next the h of the pass
// before it (evaluated on Y_next, a stabilization pass when stab_next) into
// H_next, from the gradients this pass leaves.
cudaError_t gs_launch_adj_pass(cudaStream_t s, const PbdArgs& a, int stab, const float4* Y, const float4* XT,
                               const float4* XF, const float4* WS, const uint32_t* nbr, const uint32_t* cnt,
                               const float4* H, float4* gx, float4* gxt, float* gws, int64_t* launches,
                               const AdjRecord& rec = AdjRecord{}, const float4* Y_next = nullptr,
                               int stab_next = 0, float4* H_next = nullptr);
cudaError_t gs_launch_adj_final(cudaStream_t s, const PbdArgs& a, const uint32_t* idx, const float4* WS,
                                const float4* gx, const float4* gxt, const float* gws, float4* gx0, float4* gv0,
                                int64_t* launches);

// Records an error on the context (gs_last_error) and returns code.
int gs_ctx_fail(gs_ctx* c, int code, const char* msg);
// Runs body(c, arg) directly, or (graphs enabled, a capturable stream, not
// inside another capture) as a CUDA graph captured once per key and
// replayed; the host-side state the body leaves is recorded at capture and
// applied on every replay.
int gs_replay_or_run(gs_ctx* c, uint64_t key, int (*body)(gs_ctx*, void*), void* arg);
// A key of the functional sequences: kind, step length, passes and the
// context's launch configuration.
uint64_t gs_sequence_key(const gs_ctx* c, char kind, float dt, int iters);

// Device allocation through the library's allocation-failure hook
// (gs_set_alloc_failure), for code outside a context.
cudaError_t gs_dalloc_bytes(void** p, size_t bytes);

// Grid-stride helper: blocks for n threads of `threads` each, capped.
inline unsigned gs_blocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 2147483647LL) b = 2147483647LL;
    return (unsigned)b;
}
