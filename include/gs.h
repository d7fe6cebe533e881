/*
 * gs.h -- C ABI of the GB300 library for the two-level granular method of
 * "Interactive High-Resolution Simulation of Granular Material" (arXiv
 * 2308.01629): a low-resolution (LR) position-based-dynamics simulation
 * (Sec. 3, Algorithm 1) and the per-frame upsampling of a large
 * high-resolution (HR) particle set from it (Sec. 4).
 *
 * Every step runs in hand-written CUDA kernels for sm_103a on one GPU; the
 * host side only validates arguments, owns buffers and enqueues work.
 *
 * Conventions
 *   - Units are metres and seconds; z is up; gravity is a parameter.
 *   - Particle arrays are float4 records, array-of-structures, 16-byte
 *     aligned:  LR position (x, y, z, inverse mass), LR velocity
 *     (vx, vy, vz, 0), HR position (x, y, z, id) where id is the particle's
 *     original index stored as the bits of a uint32, HR velocity
 *     (vx, vy, vz, 0).
 *   - All buffers that hold simulation state belong to the context and live
 *     in device memory allocated at gs_create.  Caller buffers passed to
 *     gs_read / gs_write stay owned by the caller.
 *   - Calls are asynchronous on the context's stream unless stated
 *     otherwise.  gs_read into host memory, gs_sync and gs_timing_read block
 *     until the stream is idle.
 *   - Every call returns a gs_status.  After GS_ERR_ARG / GS_ERR_DOMAIN /
 *     GS_ERR_CAPACITY the context stays usable; after GS_ERR_CUDA it is
 *     poisoned and every later call returns GS_ERR_STATE.
 *     gs_last_error gives the message of the most recent failure.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_ctx gs_ctx;

typedef enum {
    GS_OK = 0,
    GS_ERR_ARG = -1,       /* invalid argument (null pointer, size, range) */
    GS_ERR_OOM = -2,       /* device or host allocation failed */
    GS_ERR_CUDA = -3,      /* a CUDA call failed; the context is poisoned */
    GS_ERR_DOMAIN = -4,    /* non-finite input positions or velocities */
    GS_ERR_TIMEOUT = -5,   /* a bounded device loop reached its limit */
    GS_ERR_STATE = -6,     /* call not valid in the context's state */
    GS_ERR_CAPACITY = -7   /* a per-particle capacity was exceeded */
} gs_status;

/* Analytic boundaries.  The paper samples boundaries with immovable particles
 * (Sec. 3, particle-sampled rigid bodies and domain boundaries); this library
 * uses signed distance functions (phi > 0 in free space) instead.
 *   GS_SDF_BOX_INTERIOR: p = lo[3], hi[3]; particles stay inside; evaluated
 *                        as six half-space walls in the order x-lo, x-hi,
 *                        y-lo, y-hi, z-lo, z-hi.
 *   GS_SDF_CONE_SHELL:   p = cx, cy, z_out, R_out, z_top, R_top, half
 *                        thickness: the segment (R_out, z_out)-(R_top, z_top)
 *                        in the (radius, z) half-plane revolved about the
 *                        vertical axis through (cx, cy), thickened.
 *   GS_SDF_SOLID_BOX:    p = centre[3], half extents[3]; particles stay out.
 * vel is the boundary's velocity (kinematic boundaries); mu_s / mu_k are its
 * friction coefficients, combined with the grains' as sqrt(mu_i mu_b)
 * (Sec. 3, cross friction coefficients). */
enum { GS_SDF_BOX_INTERIOR = 1, GS_SDF_CONE_SHELL = 2, GS_SDF_SOLID_BOX = 3 };
#define GS_MAX_SDF 16

typedef struct {
    int32_t kind;
    float p[12];
    float vel[3];
    float mu_s, mu_k;
} gs_sdf;

/* Method parameters.  gs_default_params fills the paper's values. */
typedef struct {
    float gravity[3];        /* Algorithm 1: |g| = 9.81 m/s^2; default (0,0,-9.81) */
    float mu_s, mu_k;        /* Sec. 3 / 5.2: grain friction, default 0.35 / 0.30 */
    float c1, c2;            /* Sec. 4 blend constants, default 512/729 and 0.6 */
    int32_t n_stab;          /* Algorithm 1 stabilization iterations, default 2 */
    float mass_scale_k;      /* Sec. 3 height-scaled mass m* = m exp(-k (z - ground_z)), default 1 (1/m) */
    float ground_z;          /* height of the ground plane for m*, default box_lo z */
    float neighbor_radius;   /* LR candidate radius; 0 = 3 r_low */
    int32_t friction_mode;   /* 0: thresholds 2 r mu (Eqs. 3-4); 1: penetration depth times mu */
    int32_t resort_every;    /* reorder HR by cell every this many frames; 0 = never; default 8 */
    int32_t max_neighbors;   /* LR candidate capacity per particle; 0 = 64 */
} gs_params;

typedef struct {
    float box_lo[3], box_hi[3];  /* domain of the neighbour grid (metres) */
    int32_t n_low;               /* number of LR particles */
    int32_t n_sdf;               /* 0 .. GS_MAX_SDF */
    const gs_sdf* sdf;           /* copied at gs_create */
    gs_params params;
    int64_t n_high;              /* number of HR particles; 0 selects n_low * ratio (e.g. a volume
                                    sampling of a mesh gives its own count, Sec. 4) */
} gs_scene;

/* Readable / writable state.  LR and HR fields hold all scenes of the
 * context back to back (scene order, see gs_scene_info).  HR fields are always
 * exchanged in original-id order (index = id), whatever the internal cell
 * order.  Internally every scene's HR particles occupy a range of slots that
 * starts on a multiple of 32, followed by up to 31 padding slots (w = all
 * ones); the *_INTERNAL fields and GS_FIELD_HR_SORTED_KEY expose those slots.
 * Grid cells of scene s are numbered from its cell offset, and every scene
 * owns one extra padding cell after its real cells. */
enum {
    GS_FIELD_LR_POS = 0,         /* float4[n_low], read / write; w = inverse mass 1/m.  w = 0 marks a
                                    particle of a sampled boundary or rigid body (Sec. 3): it feels no
                                    gravity, moves with its velocity (GS_FIELD_LR_VEL, set by the
                                    caller), is an infinite mass in contacts, and counts in the
                                    upsampling weights only where a grain reaches the HR particle */
    GS_FIELD_LR_VEL = 1,         /* float4[n_low], read / write */
    GS_FIELD_HR_POS = 2,         /* float4[n_high], read / write (w is set to the id on write) */
    GS_FIELD_HR_VEL = 3,         /* float4[n_high], read / write */
    GS_FIELD_HR_POS_INTERNAL = 4,/* float4[HR slots], read: internal (cell) order, see gs_scene_info */
    GS_FIELD_HR_VEL_INTERNAL = 5,/* float4[HR slots], read: internal (cell) order */
    GS_FIELD_LR_CELL_START = 6,  /* uint32[total cells + 1], read: first sorted slot of each cell */
    GS_FIELD_LR_SORTED_INDEX = 7,/* uint32[n_low], read: particle index of each sorted slot */
    GS_FIELD_HR_SORTED_KEY = 8,  /* uint32[HR slots], read: fine cell key of each internal slot
                                    after the latest reorder */
    GS_FIELD_LR_MATERIAL = 9,    /* uint32[n_low], read / write: material of each LR particle
                                    (gs_set_materials); all 0 at gs_create */
    GS_FIELD_LR_BODY = 10        /* uint32[n_low], read / write: rigid body of each LR particle
                                    (0: a grain; 1 .. GS_MAX_BODIES); writing it takes every body's
                                    rest shape from the current LR positions (see below) */
};

/* Rigid bodies (Sec. 3, shape matching): the particles of a movable rigid
 * body are LR particles of finite mass that collide like grains; in every
 * solver pass each body b is matched to its rest shape:
 *   c = sum m x~ / sum m over the body (m = 1 / w, unscaled masses),
 *   C = sum m (x~ - c) xo^T,  R = the rotation of the polar decomposition
 *   of C,  and each body particle receives the constraint
 *   delta = (R xo + c) - x~, counted once in the Jacobi average;
 * xo are the particles' offsets from the body's centre of mass when
 * GS_FIELD_LR_BODY was written.  The paper's rule against HR particles
 * sticking to rigid bodies covers body particles too (see gs_upsample).
 * Writing the field synchronizes; GS_ERR_ARG for an id above
 * GS_MAX_BODIES or a body particle with w = 0.  With bodies the LR step
 * runs one launch per pass (not the persistent solver), and the reverse
 * modes refuse to run (GS_ERR_STATE). */
#define GS_MAX_BODIES 256

/* Neighbour-grid contract (Sec. 5.1 uses a compact-hashing grid; this
 * library fixes a dense uniform grid so cell ids are reproducible):
 *   h = float(3 r_low (1 + 2^-10)), inv_h = float(1 / h), o = box_lo,
 *   dims[k] = ceil((box_hi[k] - box_lo[k]) / h);
 *   a = (x - o) * inv_h in float32, round-to-nearest, no fused multiply-add;
 *   sub = clamp(floor(2 a), 0, 2 dims - 1); cell = sub >> 1;
 *   cell id = (cz dims[1] + cy) dims[0] + cx;
 *   fine key (HR order) = 8 cell id + 4 (sub_z & 1) + 2 (sub_y & 1) + (sub_x & 1).
 * Binning sorts stably by (cell id, particle index). */
typedef struct {
    float origin[3];
    float h, inv_h;
    int32_t dims[3];
    int64_t n_cell;
} gs_grid_info;

/* Layout of one scene inside a context. */
typedef struct {
    int64_t lr_offset, n_low;         /* LR particles [lr_offset, lr_offset + n_low) of the LR fields */
    int64_t hr_offset, n_high;        /* HR particles (original ids) of the HR fields */
    int64_t hr_slot_offset, hr_slot_end; /* internal HR slots of the scene, padding included */
    int64_t cell_offset;              /* first global cell id of the scene */
    gs_grid_info grid;                /* the scene's grid contract */
    float r_low, r_high;
} gs_scene_layout;

/* Fill p with the paper's default parameters (see gs_params). */
void gs_default_params(gs_params* p);

/* Create a context: allocate LR state for scene->n_low particles and HR
 * state for scene->n_high particles (n_low * ratio when n_high is 0; total
 * below 2^31), the neighbour grid over the scene box,
 * and all scratch buffers.  r_low: LR radius (Sec. 3, constant for all LR
 * particles); r_high: HR radius (<= 0 selects r_low * ratio^(-1/3)); ratio:
 * HR per LR (>= 1).  cuda_stream: a cudaStream_t the context enqueues on, or
 * NULL for a stream owned by the context.  The particle state starts at zero
 * and is loaded with gs_write.  Errors: GS_ERR_ARG, GS_ERR_OOM, GS_ERR_CUDA. */
int gs_create(const gs_scene* scene, float r_low, float r_high, int ratio, void* cuda_stream, gs_ctx** out);

/* Create one context for n_scenes independent scenes (the batched pattern
 * of serving many small simulations at once; not in the paper).  scenes,
 * r_low, ratio: arrays of n_scenes entries with the meaning of gs_create's
 * arguments; r_high may be NULL (defaults).  All scenes step together: the
 * kernels of a frame cover every scene, the upsampling runs as one launch
 * over all scenes' warp items, and gs_frame can replay a whole frame as one
 * CUDA graph.  n_stab, resort_every and max_neighbors must agree across
 * scenes.  Errors as gs_create. */
int gs_batch_create(int n_scenes, const gs_scene* scenes, const float* r_low, const float* r_high, const int* ratio,
                    void* cuda_stream, gs_ctx** out);

/* Layout of scene number `scene` of the context. */
int gs_scene_info(const gs_ctx* ctx, int scene, gs_scene_layout* out);

/* Release every buffer of the context (waits for its stream). */
void gs_destroy(gs_ctx* ctx);

/* Message of the most recent failure of this context ("" if none). */
const char* gs_last_error(const gs_ctx* ctx);

/* Counts and the grid contract of the context. */
int gs_info(const gs_ctx* ctx, int64_t* n_low, int64_t* n_high, gs_grid_info* grid);

/* Copy bytes from src (host memory when src_is_device == 0, else device
 * memory) into a state field.  bytes must equal the field's size.  Writing
 * GS_FIELD_HR_POS resets the internal order to the identity and sets w to
 * each particle's index.  Non-finite x, y, z (or velocities) give
 * GS_ERR_DOMAIN and leave the previous state in place.  Blocks when src is
 * host memory. */
int gs_write(gs_ctx* ctx, int field, const void* src, size_t bytes, int src_is_device);

/* Copy a field into dst (host memory when dst_is_device == 0, else device
 * memory).  bytes must equal the field's size.  HR fields come back in
 * original-id order.  Blocks when dst is host memory; it also reports
 * device-side errors raised since the previous check (GS_ERR_CAPACITY,
 * GS_ERR_TIMEOUT). */
int gs_read(gs_ctx* ctx, int field, void* dst, size_t bytes, int dst_is_device);

/* Replace SDF number index (0 <= index < n_sdf) -- e.g. a kinematic bucket's
 * pose for the next frame.  Stream-ordered. */
int gs_set_sdf(gs_ctx* ctx, int index, const gs_sdf* sdf);

/* Bin the LR particles at their current positions: stable counting sort by
 * grid cell (fields GS_FIELD_LR_CELL_START / GS_FIELD_LR_SORTED_INDEX) and
 * cell-ordered copies of LR position and velocity for the upsampling gather.
 * gs_step_low and gs_upsample call this themselves. */
int gs_bin_low(gs_ctx* ctx);

/* Reorder the HR particles stably by fine cell key (grid contract above) so
 * the upsampling gather reads them coalesced.  gs_upsample calls this every
 * params.resort_every frames. */
int gs_resort_high(gs_ctx* ctx);

/* One LR time step of Algorithm 1 (Sec. 3): predict v += dt g, xt = x + dt v
 * and the height-scaled inverse mass; build candidate pairs within
 * neighbor_radius of xt; n_stab contact-only Jacobi passes (Eqs. 1-2)
 * evaluated on x and applied to x and xt; iters contact + friction passes
 * (Eqs. 1-4) on xt with constraint averaging; v = (xt - x)/dt, x = xt.
 * Analytic SDF contacts act as partners of infinite mass.  dt > 0,
 * 0 <= iters <= 1000.  Candidate overflow is reported as GS_ERR_CAPACITY by
 * the next blocking call. */
int gs_step_low(gs_ctx* ctx, float dt, int iters);

/* One HR frame of Sec. 4 from the current LR state (x^{t+1}, v^{t+1}).
 * LR particles of infinite mass (w = 0) count in the sums below, except for
 * an HR particle that no grain reaches with a positive weight: there they
 * are ignored (sum w = 0, so alpha = 1), the paper's rule against HR
 * particles sticking to rigid bodies that are moved externally.  In order:
 * (re)bin the LR particles, reorder HR when due, then for every HR particle
 * w_ij = max(0, (1 - |x_ij|^2 / (9 r_low^2))^3) over LR within 3 r_low,
 * vtilde = sum w v / sum w (0 when the sum is 0),
 * alpha = 1 - max w if max w <= c1 or max w / sum w >= c2, else 0,
 * v = (1 - alpha) vtilde + alpha (v + dt g), x = x + dt v,
 * followed by the SDF rule: for each SDF component in order, when
 * phi(x) < r_high the particle moves to phi = r_high along the normal and
 * the normal velocity into the boundary (relative to the boundary velocity)
 * is removed.  dt > 0. */
int gs_upsample(gs_ctx* ctx, float dt);

/* One whole frame: n_sub LR steps of dt / n_sub (Algorithm 1) followed by
 * one HR frame of dt (gs_upsample), for every scene of the context.  With
 * graphs enabled (gs_set_graphs) the first frame of each configuration is
 * captured into a CUDA graph and later frames replay it (kernel timing with
 * gs_set_timing switches the replay off).  Asynchronous. */
int gs_frame(gs_ctx* ctx, float dt, int n_sub, int iters);

/* One frame with CFL-limited LR substeps (Sec. 5.2: a default LR time step
 * dt_max, shortened by the CFL condition when grains move fast; one HR frame
 * of dt).  Before every LR step the library takes
 *   rate = max over LR particles of |v| / (2 r_LR)   (float32),
 *   limit = min(dt_max, cfl / rate)   (dt_max when rate = 0; 0 when rate is
 *           not finite),
 * and splits the frame time left into the fewest equal steps no longer than
 * limit: n = ceil(t_left / limit), capped by the steps still allowed
 * (max_sub per frame), step = t_left / n.  The last step of the frame is
 * the one with n = 1, so the steps add up to dt.  All in float32, correctly
 * rounded.  Then one HR frame of dt (gs_upsample).  With graphs enabled the
 * frame is one CUDA graph whose LR steps run in a device-side loop (a
 * conditional while node), so the host neither waits nor learns the step
 * count; otherwise (graphs off, or kernel timing on) the host waits after
 * every step.  Adaptive frames are not pipelined (gs_set_pipeline).  dt,
 * dt_max, cfl > 0 and finite, 1 <= max_sub <= GS_MAX_SUBSTEPS, 0 <= iters
 * <= 1000.  The LR steps of adaptive frames enter gs_launch_count at the
 * next gs_sync or gs_substeps. */
#define GS_MAX_SUBSTEPS 256
int gs_frame_adaptive(gs_ctx* ctx, float dt, float dt_max, float cfl, int max_sub, int iters);

/* One scene's HR set split across GPUs (Sec. 4: given the LR state, every
 * HR particle's update depends on the LR particles alone, never on another
 * HR particle).  Every rank runs the whole LR computation (the same
 * deterministic kernels on the same input, so the same bits everywhere) and
 * updates only its slab of the HR slots in internal (cell) order, the
 * slots of GS_FIELD_HR_POS_INTERNAL; the ranks exchange their slabs (the
 * caller's all-gather) before each HR reorder and before reading the HR
 * state in original order.
 *
 * gs_hr_slab_range: slab `part` of `n_parts` of n_slots HR slots is
 * [*begin, *end): whole 32-slot items split as evenly as possible (item
 * counts differ by one at most; a slab may be empty).  Host arithmetic, no
 * context, no GPU.  GS_ERR_ARG unless 1 <= n_parts <= 4096,
 * 0 <= part < n_parts, n_slots >= 0 and a multiple of 32 (the size of
 * GS_FIELD_HR_POS_INTERNAL in float4 is), begin and end not null. */
int gs_hr_slab_range(int64_t n_slots, int part, int n_parts, int64_t* begin, int64_t* end);

/* Restricts the HR frames of the context (gs_upsample, gs_frame,
 * gs_frame_adaptive) to slab `part` of `n_parts` of its HR slots; slots
 * outside keep their values, and every slot inside gets bitwise the value
 * the unrestricted context computes (the gather's work items are the same
 * 32 slots with the same arithmetic).  n_parts = 1 restores the whole set.
 * After a restricted frame the context's HR state is "partial": until
 * gs_hr_slab_assemble, a frame on which an HR reorder is due
 * (params.resort_every), gs_resort_high, reads and writes of GS_FIELD_HR_POS
 * / GS_FIELD_HR_VEL (synchronous or asynchronous) and another
 * gs_set_hr_slab return GS_ERR_STATE; the internal fields stay readable.
 * Not with pipelined frames (GS_ERR_STATE both ways).  Bad part / n_parts:
 * GS_ERR_ARG. */
int gs_set_hr_slab(gs_ctx* ctx, int part, int n_parts);

/* The gather-back: writes the whole HR state in internal slot order, pos
 * and vel each float4[HR slots] (bytes = 16 x HR slots) as read from
 * GS_FIELD_HR_POS_INTERNAL / GS_FIELD_HR_VEL_INTERNAL, each slab taken from
 * the context that updated it, and ends the partial state.  The w of every
 * slot's position (the particle id, padding included) must equal the
 * context's bit for bit, and every x, y, z must be finite; otherwise
 * GS_ERR_ARG and nothing changes.  Pending device errors of earlier calls
 * are reported first.  Host or device sources (src_is_device); blocks until
 * the state is applied, so the sources may change on return.  A context
 * without a slab may call it too (a state written back unchanged). */
int gs_hr_slab_assemble(gs_ctx* ctx, const void* pos, const void* vel, size_t bytes, int src_is_device);

/* Initial sampling of a closed triangle mesh's volume (Sec. 4), for seeding
 * LR and HR particles.  The bounding box of the vertices is divided into
 * cells of side h = 2 r / sqrt(3) (origin: the box's low corner; dims =
 * floor(extent / h) + 1 per axis); the candidates (uniform random positions
 * in the box, drawn by the caller) that lie inside the mesh -- generalized
 * winding number above 1/2, so overlapping closed parts count as their
 * union -- are assigned to their cells in input order; then, cell by cell,
 * the first candidate that is at least 2 r away from every sample taken so
 * far becomes the cell's sample.  Cells are taken in 27 phases: phase
 * (cx mod 3) + 3 (cy mod 3) + 9 (cz mod 3) ascending (cells of one phase
 * never compete, so their order within the phase does not matter).  All
 * decisions in double precision.
 *   vertices   double[n_vertices][3];  triangles int32[n_triangles][3],
 *              counter-clockwise seen from outside, indices < n_vertices;
 *   candidates double[n_candidates][3], n_candidates < 2^31;
 *   r          the particle radius (samples are >= 2 r apart);
 *   selected   receives the indices of the chosen candidates in ascending
 *              cell order (at most capacity); *n_selected their number;
 *   inside     (optional) uint8[n_candidates]: 1 for candidates inside.
 * Host arrays; synchronous; uses the current device with device memory of
 * its own, freed on return.  GS_ERR_ARG (null pointers, r <= 0, a triangle
 * index out of range, more than 2^31 - 2 cells), GS_ERR_DOMAIN (a
 * non-finite coordinate), both before any device work; GS_ERR_CAPACITY when
 * more than capacity samples were chosen (*n_selected is their number);
 * GS_ERR_OOM, GS_ERR_CUDA. */
int gs_sample_volume(const double* vertices, int64_t n_vertices, const int32_t* triangles, int64_t n_triangles,
                     const double* candidates, int64_t n_candidates, double r, int64_t* selected, int64_t capacity,
                     int64_t* n_selected, uint8_t* inside);

/* Surface sampling for particle-sampled boundaries (Sec. 3: a stationary
 * body's particles of infinite mass need only cover its surface): the same
 * grid over the vertices' bounding box and the same cell-by-cell pick as
 * gs_sample_volume, with every candidate valid; the candidates are points
 * on the mesh's triangles (uniform by area, drawn by the caller).  Arguments,
 * outputs and errors as gs_sample_volume; in addition GS_ERR_ARG when a
 * candidate lies more than 0.15 r outside the vertices' bounding box (one
 * that far out could be picked closer than 2 r to another). */
int gs_sample_surface(const double* vertices, int64_t n_vertices, const double* candidates, int64_t n_candidates,
                      double r, int64_t* selected, int64_t capacity, int64_t* n_selected);

/* The LR steps of the latest adaptive frame: *n_out receives their number
 * and dts[0 .. min(n, cap)) their lengths.  Blocks. */
int gs_substeps(gs_ctx* ctx, float* dts, int cap, int* n_out);

/* Asynchronous forms of gs_write / gs_read for the four state fields
 * (GS_FIELD_LR_POS, _LR_VEL, _HR_POS, _HR_VEL; same layouts and sizes), so
 * that a caller can overlap host <-> device traffic with the simulation.
 * gs_write_async copies src into a device staging buffer on a copy stream of
 * the context and returns at once; the field is checked for finite values on
 * the device and applied, in order, before the next call that reads or
 * changes the state (gs_frame, gs_step_low, gs_upsample, gs_read, ...).  src
 * must stay valid and unchanged until the next gs_sync.  A non-finite value
 * cannot be refused synchronously: the field is applied and the next gs_sync
 * or gs_read returns GS_ERR_DOMAIN (the state is then invalid).
 * gs_read_async takes the field's value as of this point in the context's
 * work (everything enqueued before it) into a device snapshot and copies it
 * to dst on a second copy stream; dst holds it after the next gs_sync.  A
 * device dst is written as by gs_read.  GS_ERR_ARG for another field or a
 * size mismatch, GS_ERR_OOM if a transfer buffer cannot be allocated (on
 * first use of a field). */
int gs_write_async(gs_ctx* ctx, int field, const void* src, size_t bytes, int src_is_device);
int gs_read_async(gs_ctx* ctx, int field, void* dst, size_t bytes, int dst_is_device);

/* Grain materials: per-particle friction coefficients (Sec. 3).  mu holds
 * n_materials pairs (mu_s, mu_k) in host memory, each finite and >= 0;
 * 1 <= n_materials <= GS_MAX_MATERIALS.  From the next LR step on, LR
 * particle i has the coefficients of its material m_i (field
 * GS_FIELD_LR_MATERIAL, 0 unless written) instead of its scene's
 * params.mu_s / mu_k, and a contact uses the cross coefficients of the two
 * partners, static and kinetic alike: mu_ij = sqrt(mu_i mu_j) between
 * grains, sqrt(mu_i mu_b) with an SDF boundary.  One table serves all scenes
 * of a context.  n_materials = 0 returns to the scenes' coefficients and
 * resets every particle's material to 0.  Errors: GS_ERR_ARG for an invalid
 * count or coefficient, or when a particle's material id is >= n_materials
 * (the table is then unchanged).  gs_step_low_backward refuses to run
 * (GS_ERR_STATE) while a material table is set: the LR step's reverse mode
 * knows the scenes' coefficients only.  Writing
 * GS_FIELD_LR_MATERIAL needs a table; ids >= n_materials give GS_ERR_ARG
 * and leave the field unchanged. */
#define GS_MAX_MATERIALS 16
int gs_set_materials(gs_ctx* ctx, int n_materials, const float* mu);

/* Enable (1) or disable (0) CUDA-graph replay of gs_frame, and of the fixed
 * launch sequence inside gs_step_low_forward / gs_step_low_backward (between
 * the copies of the caller's buffers; not on the legacy or per-thread
 * default stream, which cannot be captured).  Results are the same bits
 * (gradients up to the order of atomic accumulations, which varies from run
 * to run either way). */
int gs_set_graphs(gs_ctx* ctx, int enable);

/* Pipelined frames (enable = 1): the HR frame of frame f is deferred and
 * runs, on a second stream of the context, while gs_frame of frame f + 1
 * runs its LR steps (Sec. 4's HR frame reads only the LR state at the end
 * of frame f, which the LR steps of frame f + 1 start from; the deferred
 * frame keeps a copy of the SDF table as of frame f).  warps_per_block /
 * blocks_per_sm: the upsampling launch shape while it overlaps the LR steps
 * (blocks_per_sm 0 = one warp item per warp).  Every other call that reads
 * or changes the HR state or the binned LR view (gs_read, gs_write, gs_sync,
 * gs_upsample, gs_step_low, gs_bin_low, gs_resort_high, gs_autotune, the
 * functional forms) first completes the deferred frame in stream order, so
 * results equal those of sequential frames bit for bit; gs_frame with
 * timing enabled runs sequentially.  Disabling completes a deferred frame.
 * Returns GS_ERR_ARG for an unsupported launch shape. */
int gs_set_pipeline(gs_ctx* ctx, int enable, int warps_per_block, int blocks_per_sm);

/* How gs_step_low runs the n_stab + iters Jacobi passes of a step: 1 = one
 * persistent cooperative launch whose blocks are all resident and meet at a
 * grid barrier between passes; 0 (the default) = one launch per pass, which
 * measured faster when frames are replayed as CUDA graphs.  Both give the
 * same bits.  A barrier that waits longer than one second (GPU global timer)
 * gives up, every block leaves, and the next gs_sync or gs_read returns
 * GS_ERR_TIMEOUT; the context stays usable but the LR state of that step is
 * invalid.  2 = self-test of that path: the barrier waits for one block more
 * than the launch has, so every step times out after about a second.
 * GS_ERR_ARG for another mode, GS_ERR_STATE where the device has no
 * cooperative launches.  Does not apply to the functional forms
 * (gs_step_low_forward / _backward), which keep every pass's input. */
int gs_set_lr_solver(gs_ctx* ctx, int persistent);

/* The HR frame's reverse mode (gs_upsample_backward and the rollouts) adds
 * the LR gradients either by float atomics from every HR particle (the
 * default; their order, and so the last bits of the sums, vary from run to
 * run) or (1) deterministically: every HR particle's coefficients first, the
 * HR particles binned by the LR cells, then one warp per LR particle
 * gathering the terms of the HR particles in the 27 cells around it in a
 * fixed order, so gradients are the same bits on every run (about 50 us
 * more per call for 4k LR / 64k HR). */
int gs_set_deterministic_backward(gs_ctx* ctx, int enable);

/* A timer around the upsampling gather inside whole frames: with it on,
 * two CUDA events of the context bracket the gather's launches of every HR
 * frame (in captured frames as event nodes of the graph, so every replay
 * records them), and gs_gather_timer_ms returns the time between them for
 * the latest frame (it waits for that frame).  Turning it on or off drops
 * the captured frames.  GS_ERR_STATE when it is off. */
int gs_set_gather_timer(gs_ctx* ctx, int enable);
int gs_gather_timer_ms(gs_ctx* ctx, float* ms);

/* Launch shape of the upsampling kernel: warps per block (4, 8 or 16) and
 * blocks per SM of a persistent grid that pulls 32-particle work items from
 * an atomic counter (0: one warp per item, no persistent loop). */
int gs_set_tuning(gs_ctx* ctx, int warps_per_block, int blocks_per_sm);

/* Time the upsampling kernel on the current state (written out of place,
 * the state is not changed) for a fixed list of launch shapes, reps
 * launches each, and keep the fastest.  Returns the shape and its time per
 * launch in microseconds.  Blocks. */
int gs_autotune(gs_ctx* ctx, float dt, int reps, int* warps_per_block, int* blocks_per_sm, float* best_us);

/* Differentiable pattern (not in the paper): one HR frame as a function of
 * caller-owned device buffers, and its reverse mode.  Single-scene contexts
 * only; the context is used as workspace and its LR and HR state are
 * overwritten.  All arrays are float4 records in original order (w of
 * positions is ignored on input, gradients have w = 0):
 *   gs_upsample_forward:  (lr_pos, lr_vel [n_low], hr_pos_in, hr_vel_in
 *                          [n_high]) -> hr_pos_out, hr_vel_out [n_high],
 *                          the same map as gs_upsample (Sec. 4).
 *   gs_upsample_backward: given dL/d hr_pos_out and dL/d hr_vel_out, writes
 *                          dL/d lr_pos, dL/d lr_vel, dL/d hr_pos_in and
 *                          dL/d hr_vel_in for the forward pass's branch
 *                          decisions (blend case, LR particle of largest
 *                          weight, SDF contacts); each SDF contact is
 *                          differentiated with its normal held fixed, which
 *                          is exact for planar walls.
 * Outputs are overwritten, not accumulated.  Asynchronous. */
int gs_upsample_forward(gs_ctx* ctx, const float* lr_pos, const float* lr_vel, const float* hr_pos_in,
                        const float* hr_vel_in, float* hr_pos_out, float* hr_vel_out, float dt);
int gs_upsample_backward(gs_ctx* ctx, const float* lr_pos, const float* lr_vel, const float* hr_pos_in,
                         const float* hr_vel_in, const float* g_hr_pos_out, const float* g_hr_vel_out, float* g_lr_pos,
                         float* g_lr_vel, float* g_hr_pos_in, float* g_hr_vel_in, float dt);

/* One LR step (Algorithm 1, as gs_step_low) as a function of caller-owned
 * device buffers, and its reverse mode (differentiable pattern; not in the
 * paper).  x, v: float4[n_low] in original order (w of x is the inverse
 * mass).  The context is used as workspace; its LR state is overwritten.
 * gs_step_low_backward recomputes the step from (x_in, v_in) and, given
 * dL/dx_out and dL/dv_out, writes dL/dx_in and dL/dv_in for the forward
 * pass's branch decisions (contact sets, static / kinetic / clipped
 * friction, SDF contacts with fixed normals), including the dependence of the
 * height-scaled mass ratios on the start-of-step heights.  Outputs are
 * overwritten.  Asynchronous.  Both backward entry points differentiate
 * grains only: LR positions holding particles of inverse mass 0 make the
 * next blocking call (gs_sync, gs_read) return GS_ERR_STATE, and the
 * gradients of that call are invalid. */
int gs_step_low_forward(gs_ctx* ctx, const float* x_in, const float* v_in, float* x_out, float* v_out, float dt,
                        int iters);
int gs_step_low_backward(gs_ctx* ctx, const float* x_in, const float* v_in, const float* g_x_out, const float* g_v_out,
                         float* g_x_in, float* g_v_in, float dt, int iters);

/* Decision record of the reverse modes (not in the paper): where the method
 * branches (blend case and largest weight, contact activation, static or
 * kinetic friction, SDF contacts), gs_upsample_backward and
 * gs_step_low_backward differentiate the branch each decision takes; with a
 * record set they also write those decisions, so that a reference can be
 * evaluated on exactly the same smooth piece of the method.  Device
 * buffers, caller-owned, original particle order; every later backward call
 * overwrites them.  Single-scene contexts only (GS_ERR_STATE otherwise).
 *   hr_record      uint32[n_high][4] (NULL: off), per HR particle: the LR
 *                  particle of largest weight (index, or 0xffffffff), the
 *                  blend case (1: alpha = 1 - max w, 0: alpha = 0), bit c
 *                  set when SDF component c is in contact, bit c set when
 *                  the normal velocity was removed at component c (at most
 *                  32 components; a box interior counts its six walls).
 *   lr_candidates  int32[cap][n_low]: the candidate partners of each LR
 *                  particle (-1 beyond its count); cap = params.max_neighbors
 *                  (0 there means 64).
 *   lr_pair_bits   uint8[max_passes][cap][n_low]: per pass (stabilization
 *                  passes first) and candidate, bit 0 = contact
 *                  (|x_ij| < 2 r_LR), bit 1 = kinetic friction scale.
 *   lr_sdf_bits    uint8[max_passes][n_low][n_comp] (n_comp = the SDF
 *                  components): bit 0 = contact, bit 1 = kinetic friction.
 *   max_passes     capacity in passes; a backward call with more passes
 *                  (n_stab + iters) returns GS_ERR_ARG.
 * The LR pointers are all NULL (off) or all set (lr_sdf_bits may be NULL
 * without SDFs); GS_ERR_ARG otherwise. */
int gs_set_decision_record(gs_ctx* ctx, uint32_t* hr_record, int32_t* lr_candidates, uint8_t* lr_pair_bits,
                           uint8_t* lr_sdf_bits, int max_passes);

/* Taped LR steps for checkpointed rollouts.  A differentiable rollout runs
 * each LR step forward (again, when its segment is recomputed from a
 * checkpoint) and then backward; gs_step_low_backward records the step once
 * more to know what every pass evaluated on.  With n_slots > 0,
 * gs_step_low_forward_taped keeps that record (per-pass snapshots, candidate
 * lists, cell order) of the latest n_slots steps in slots of the context
 * (about 2 (n_stab + iters + 1) x 16 + (max_neighbors + 2) x 4 bytes per LR
 * particle each) under the caller's tag (>= 0; a recomputation of the same
 * step gives the same tag), and gs_step_low_backward_taped runs only the
 * reverse passes from the latest kept record with that tag.  Outputs and
 * gradients equal those of gs_step_low_forward / gs_step_low_backward bit
 * for bit.  gs_set_step_tapes(ctx, 0) frees the slots (the default); a new
 * count drops the kept records.  Without slots gs_step_low_forward_taped is
 * gs_step_low_forward.  gs_step_low_backward_taped returns GS_ERR_STATE when
 * no kept record has the tag (never taken or overwritten by later steps):
 * the caller then uses gs_step_low_backward.  Device buffers as for the
 * functional forms; grains of the scenes' coefficients only (GS_ERR_STATE
 * with materials or bodies). */
int gs_set_step_tapes(gs_ctx* ctx, int n_slots);
int gs_step_low_forward_taped(gs_ctx* ctx, const float* x_in, const float* v_in, float* x_out, float* v_out, float dt,
                              int iters, int64_t tag);
int gs_step_low_backward_taped(gs_ctx* ctx, int64_t tag, const float* g_x_out, const float* g_v_out, float* g_x_in,
                               float* g_v_in);

/* A differentiable rollout run by the library: `frames` frames of n_sub LR
 * steps of dt / n_sub (Algorithm 1) and one HR frame of dt (Sec. 4) from
 * the initial state (lr_x0, lr_v0, hr_x0, hr_v0; original order, float4
 * records as the functional forms) into (lr_x, lr_v, hr_x, hr_v), keeping
 * the state at every checkpoint_every-th frame inside the context
 * (2 (n_low + n_high) x 16 bytes each).  gs_rollout_backward then maps the
 * cotangents of the final state to those of the initial state: each segment
 * is recomputed from its checkpoint with taped LR steps (gs_set_step_tapes
 * grows to checkpoint_every x n_sub slots) and reversed frame by frame
 * (gs_upsample_backward, gs_step_low_backward_taped), the LR cotangent of a
 * frame's end summing the next step's and the HR frame's.  The same
 * operations, in the same order, as a checkpointed rollout driven through
 * the functional entry points.  Single-scene contexts; the context's state
 * is used as workspace.  Device buffers; the w components carry no
 * gradient.  GS_ERR_STATE for a backward without a forward. */
int gs_rollout_forward(gs_ctx* ctx, const float* lr_x0, const float* lr_v0, const float* hr_x0, const float* hr_v0,
                       float dt, int frames, int n_sub, int iters, int checkpoint_every, float* lr_x, float* lr_v,
                       float* hr_x, float* hr_v);
int gs_rollout_backward(gs_ctx* ctx, const float* g_lr_x, const float* g_lr_v, const float* g_hr_x, const float* g_hr_v,
                        float* g_lr_x0, float* g_lr_v0, float* g_hr_x0, float* g_hr_v0);

/* Pass-by-pass record of one LR step (Algorithm 1, Sec. 3), for checking the
 * step against a reference one Jacobi pass at a time: each pass is a
 * function of the state before it, so a pass can be compared on its own
 * from the record of its input, without the branch decisions of the earlier
 * passes compounding.  Same step as gs_step_low_forward from (x_in, v_in)
 * (float4[n_low] device buffers in original order; w of x = inverse mass):
 * record k = 0 .. n_stab + iters holds, in original particle order, the
 * positions x (the start-of-step positions as corrected by the
 * stabilization passes so far) and the predictions x~ (as corrected by all
 * passes so far) before pass k; record n_stab + iters is the state after
 * the last pass, from which the step's finalize takes v = (x~ - x) / dt,
 * x = x~.  The w of an x record is the inverse mass; the w of an x~ record
 * is the inverse height-scaled mass 1/m* the passes use.
 *   x_trace, xt_trace  device float4[(n_stab + iters + 1) * n_low], caller-owned
 *   n_records          must equal n_stab + iters + 1 (GS_ERR_ARG otherwise)
 * The context is used as workspace; its LR state is overwritten.
 * GS_ERR_STATE while grain materials or rigid bodies are set; LR positions
 * with inverse mass 0 make the next blocking call return GS_ERR_STATE (as
 * for the reverse modes).  GS_ERR_OOM if the per-pass buffers cannot be
 * allocated (first use).  Asynchronous. */
int gs_step_low_trace(gs_ctx* ctx, const float* x_in, const float* v_in, float dt, int iters, float* x_trace,
                      float* xt_trace, int n_records);

/* Block until the context's stream is idle and report device-side errors. */
int gs_sync(gs_ctx* ctx);

/* Kernel timing with CUDA events on the context's stream.  When enabled,
 * every launch group below is bracketed by an event pair.  gs_timing_read
 * blocks, returns the summed milliseconds and the number of launches of one
 * group since the previous read, and resets that group. */
enum {
    GS_TIMER_BIN_LOW = 0,    /* LR binning (keys, sort, cell starts, copies) */
    GS_TIMER_RESORT = 1,     /* HR reorder */
    GS_TIMER_GATHER = 2,     /* upsampling gather + advection + SDF (one kernel) */
    GS_TIMER_STEP_LOW = 3,   /* one whole LR step */
    GS_TIMER_COUNT = 4
};
int gs_set_timing(gs_ctx* ctx, int enable);
int gs_timing_read(gs_ctx* ctx, int timer, double* total_ms, int64_t* launches);

/* Binning without allocation.  No counterpart in the paper: this is a service
 * for callers that cannot call cudaMalloc -- for example code that records
 * its work into a CUDA graph under the global capture mode (where an
 * allocation is an error), a real-time render loop that cannot afford the
 * implicit device synchronization cudaMalloc may cause, or a host that hands
 * out all device memory from a pool it does not let the library touch.
 *
 * Bins n points exactly like gs_bin_low bins the LR set: cell ids from the
 * grid contract above, a stable sort by (cell id, index), cell starts.
 *   pos4          device, float4[n] (x, y, z, unused), 16-byte aligned
 *   grid          the grid contract (e.g. from gs_info); n_cell must equal
 *                 dims[0] dims[1] dims[2]
 *   sorted_index  device, uint32[n]: point index of each sorted slot
 *   cell_start    device, uint32[n_cell + 1]: first sorted slot of each cell
 *   cuda_stream   stream to enqueue on (NULL: the legacy default stream)
 * Inputs and outputs stay owned by the caller.  The scratch the sort needs is
 * a fixed static array of GS_STATIC_BIN_SCRATCH_BYTES in device memory that
 * every GPU loading this library holds until the process exits; no call
 * allocates or frees anything.  The first call on a device looks the
 * array's device address up (with that device current); make that first
 * call before any stream capture.  All calls on a device share the array, so
 * calls whose work overlaps on the GPU race: order them on one stream or
 * synchronize between them.
 * Returns GS_ERR_CAPACITY when n > GS_STATIC_BIN_MAX_POINTS (nothing is
 * enqueued), GS_ERR_ARG for null or misaligned pointers (pos4 to 16 bytes,
 * sorted_index and cell_start to 4) or an inconsistent grid (a dimension
 * below 1 or above 2^20, as gs_create allows), GS_ERR_CUDA when a CUDA call
 * fails.  Asynchronous on cuda_stream. */
#define GS_STATIC_BIN_MAX_POINTS 262144
#define GS_STATIC_BIN_SCRATCH_BYTES 4358144
int gs_bin_points_static(const float* pos4, int64_t n, const gs_grid_info* grid, uint32_t* sorted_index,
                         uint32_t* cell_start, void* cuda_stream);

/* Failure detection test hook (not in the paper): after `after` more device
 * allocations by the library, every further one fails as if the device
 * were out of memory, until the hook is switched off (after < 0).  The
 * failure is injected on the host, in the library's allocation helper; no
 * device work is involved.  Calls then return GS_ERR_OOM and release what
 * they had allocated (gs_create leaves nothing behind).  Process-wide. */
void gs_set_alloc_failure(long long after);

/* Number of kernels this context has launched since creation. */
int64_t gs_launch_count(const gs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
