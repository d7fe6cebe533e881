/*
 * gs_oracle.c -- plain, slow FP64 CPU oracle for the two-level granular
 * method of "Interactive High-Resolution Simulation of Granular Material"
 * (arXiv 2308.01629): the low-resolution (LR) position-based-dynamics step of
 * Sec. 3 / Algorithm 1, the high-resolution (HR) upsampling of Sec. 4 and the
 * initial volume sampling of a closed triangle mesh (Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; both sides are written from
 * the paper independently and meet only through seeded input arrays.
 *
 * Conventions (all arrays row-major, caller-owned):
 *   positions / velocities: double[n][3]; z is up, gravity is a parameter.
 *   SDF records: double[20] = {kind, p[12], u_b[3], mu_s, mu_k, 0, 0}
 *     kind 1 = box interior   p = lo[3], hi[3]          (6 half-space walls)
 *     kind 2 = cone shell     p = cx, cy, z_out, R_out, z_top, R_top, half
 *                             thickness (a segment in (rho, z) revolved
 *                             about the vertical axis through (cx, cy))
 *     kind 3 = solid box      p = centre[3], half extents[3]
 *   u_b is the velocity of the boundary (kinematic SDFs).
 *
 * Readings of silent or garbled passages are listed next to the code that
 * implements them.  Every decision taken on a floating-point comparison is
 * checked against a margin; decisions inside the margin are reported so that
 * a lower-precision implementation can be compared against both branches.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_SDF_STRIDE 20
#define OR_MAX_COMP 6

enum { SDF_BOX_INTERIOR = 1, SDF_CONE_SHELL = 2, SDF_SOLID_BOX = 3 };

/* upsampling parameters, prm[] indices */
enum { UP_R_LOW = 0, UP_R_HIGH, UP_DT, UP_GX, UP_GY, UP_GZ, UP_C1, UP_C2,
       UP_EPS_W, UP_EPS_X, UP_NPRM };
/* LR step parameters, prm[] indices */
enum { PB_R = 0, PB_DT, PB_GX, PB_GY, PB_GZ, PB_MU_S, PB_MU_K, PB_N_STAB,
       PB_ITERS, PB_MASS_K, PB_GROUND_Z, PB_RC, PB_FRIC_MODE, PB_EPS_X,
       PB_EPS_IMPACT, PB_NPRM };

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ */
/* Uniform-grid cell contract (neighbour search, Sec. 5.1 uses a        */
/* compact-hashing grid; this library fixes a dense grid instead).      */
/*   cell side  h = 3 r_LR (1 + 2^-10), rounded once to float           */
/*   inv_h = float(1/h), origin o = float(box_lo), dims = ceil(L/h)     */
/*   a = (x - o) * inv_h evaluated in float, no contraction            */
/*   sub = clamp(floor(2a), 0, 2 dim - 1); cell = sub >> 1              */
/*   cell id = (cz*dy + cy)*dx + cx; fine key = 8*cell + octant bits     */
/* The factor (1 + 2^-10) keeps every pair closer than 3 r_LR within    */
/* one cell of each other after float rounding of a.                    */
/* ------------------------------------------------------------------ */
int or_grid(double r_low, const double* lo, const double* hi, float* o, float* h, float* inv_h, int* dims)
{
    if (!(r_low > 0)) return -1;
    double hd = 3.0 * r_low * (1.0 + 1.0 / 1024.0);
    float hf = (float)hd;
    *h = hf;
    *inv_h = (float)(1.0 / (double)hf);
    for (int k = 0; k < 3; ++k) {
        if (!(hi[k] > lo[k])) return -1;
        o[k] = (float)lo[k];
        double n = ceil((hi[k] - lo[k]) / (double)hf);
        dims[k] = n < 1 ? 1 : (int)n;
    }
    return 0;
}


void or_cell_keys(const float* pos4, long n, const float* o, float inv_h, const int* dims, int fine, uint32_t* keys)
{
    for (long i = 0; i < n; ++i) {
        int s[3];
        for (int k = 0; k < 3; ++k) {
            float a = (pos4[4 * i + k] - o[k]) * inv_h;   /* float, no FMA (-ffp-contract=off) */
            float f = floorf(a * 2.0f);
            int si;
            if (!(f >= 0.0f)) si = 0;                       /* negative (or NaN) -> 0 */
            else if (f >= (float)(2 * dims[k] - 1)) si = 2 * dims[k] - 1;
            else si = (int)f;
            s[k] = si;
        }
        uint32_t cell = ((uint32_t)(s[2] >> 1) * (uint32_t)dims[1] + (uint32_t)(s[1] >> 1)) * (uint32_t)dims[0]
                        + (uint32_t)(s[0] >> 1);
        if (fine)
            keys[i] = cell * 8u + (uint32_t)((s[2] & 1) * 4 + (s[1] & 1) * 2 + (s[0] & 1));
        else
            keys[i] = cell;
    }
}

/* Stable counting sort of keys in [0, nkeys): start[c] = first slot of key c,
 * sorted_idx lists element indices by (key, index).  Sequential scatter in
 * index order is what makes it stable. */
int or_counting_sort(const uint32_t* keys, long n, long nkeys, uint32_t* sorted_idx, uint32_t* start)
{
    uint32_t* cursor = (uint32_t*)calloc((size_t)nkeys + 1, sizeof(uint32_t));
    if (!cursor) return -1;
    for (long i = 0; i < n; ++i) {
        if ((long)keys[i] >= nkeys) { free(cursor); return -2; }
        cursor[keys[i] + 1]++;
    }
    for (long c = 0; c < nkeys; ++c) cursor[c + 1] += cursor[c];
    memcpy(start, cursor, ((size_t)nkeys + 1) * sizeof(uint32_t));
    for (long i = 0; i < n; ++i) sorted_idx[cursor[keys[i]]++] = (uint32_t)i;
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Oracle-private neighbour search: a plain grid with cell side R over  */
/* the bounding box of the points.  It returns, for one query point,    */
/* every point index with |x_q - x_j|^2 < R^2 in ascending order, so    */
/* sums taken over it equal the brute-force sums bit for bit.           */
/* ------------------------------------------------------------------ */
typedef struct {
    double R, lo[3];
    long dim[3];
    long* start;   /* ncell + 1 */
    long* idx;     /* n */
    const double* x;
    long n;
} or_grid_t;

static int grid_build(or_grid_t* g, const double* x, long n, double R)
{
    memset(g, 0, sizeof(*g));
    g->R = R;
    g->x = x;
    g->n = n;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) { lo[k] = n ? x[k] : 0; hi[k] = lo[k]; }
    for (long i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            if (x[3 * i + k] < lo[k]) lo[k] = x[3 * i + k];
            if (x[3 * i + k] > hi[k]) hi[k] = x[3 * i + k];
        }
    long ncell = 1;
    for (int k = 0; k < 3; ++k) {
        g->lo[k] = lo[k];
        long d = (long)floor((hi[k] - lo[k]) / R) + 1;
        if (d > 1024) d = 1024;
        g->dim[k] = d;
        ncell *= d;
    }
    g->start = (long*)calloc((size_t)ncell + 1, sizeof(long));
    g->idx = (long*)malloc((size_t)(n ? n : 1) * sizeof(long));
    long* cell = (long*)malloc((size_t)(n ? n : 1) * sizeof(long));
    if (!g->start || !g->idx || !cell) { free(cell); return -1; }
    for (long i = 0; i < n; ++i) {
        long c[3];
        for (int k = 0; k < 3; ++k) {
            long v = (long)floor((x[3 * i + k] - g->lo[k]) / R);
            c[k] = v < 0 ? 0 : (v >= g->dim[k] ? g->dim[k] - 1 : v);
        }
        cell[i] = (c[2] * g->dim[1] + c[1]) * g->dim[0] + c[0];
        g->start[cell[i] + 1]++;
    }
    for (long c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
    long* cur = (long*)malloc((size_t)ncell * sizeof(long));
    if (!cur) { free(cell); return -1; }
    memcpy(cur, g->start, (size_t)ncell * sizeof(long));
    for (long i = 0; i < n; ++i) g->idx[cur[cell[i]]++] = i;
    free(cur);
    free(cell);
    return 0;
}

static void grid_free(or_grid_t* g) { free(g->start); free(g->idx); }

static int cmp_long(const void* a, const void* b)
{
    long x = *(const long*)a, y = *(const long*)b;
    return (x > y) - (x < y);
}

/* Collect points within R of q (strict), ascending.  Returns the count;
 * out must hold n entries.  Points were binned with clamped cell
 * coordinates; clamping is monotone, so clamping the query's cell range
 * (widened by one cell against rounding) still covers every point in
 * reach, and each cell is visited once. */
static long grid_query(const or_grid_t* g, const double* q, long* out)
{
    long c0[3], c1[3], m = 0;
    for (int k = 0; k < 3; ++k) {
        double a = floor((q[k] - g->R - g->lo[k]) / g->R) - 1;
        double b = floor((q[k] + g->R - g->lo[k]) / g->R) + 1;
        double top = (double)(g->dim[k] - 1);
        c0[k] = (long)(a < 0 ? 0 : (a > top ? top : a));
        c1[k] = (long)(b < 0 ? 0 : (b > top ? top : b));
    }
    double R2 = g->R * g->R;
    for (long cz = c0[2]; cz <= c1[2]; ++cz)
        for (long cy = c0[1]; cy <= c1[1]; ++cy)
            for (long cx = c0[0]; cx <= c1[0]; ++cx) {
                long cid = (cz * g->dim[1] + cy) * g->dim[0] + cx;
                for (long p = g->start[cid]; p < g->start[cid + 1]; ++p) {
                    long j = g->idx[p];
                    double d[3] = {g->x[3 * j] - q[0], g->x[3 * j + 1] - q[1], g->x[3 * j + 2] - q[2]};
                    if (dot3(d, d) < R2) out[m++] = j;
                }
            }
    qsort(out, (size_t)m, sizeof(long), cmp_long);
    return m;
}

/* ------------------------------------------------------------------ */
/* Analytic SDF boundaries.  The paper samples boundaries with          */
/* infinite-mass particles (Sec. 3, rigid bodies and domain             */
/* boundaries); this library uses analytic signed distance functions    */
/* instead and treats each active SDF contact as a pair whose partner   */
/* has inverse mass 0.  Returns the number of contact components (6 for */
/* the box interior, else 1).  phi > 0 is free space, n = grad phi.     */
/* *tie is set when the normal is not unique within eps (solid box).    */
/* ------------------------------------------------------------------ */
int or_sdf_eval(const double* s, const double* x, double* phi, double* n, int* tie, double eps)
{
    int kind = (int)s[0];
    const double* p = s + 1;
    *tie = 0;
    if (kind == SDF_BOX_INTERIOR) {
        for (int k = 0; k < 3; ++k) {
            phi[2 * k] = x[k] - p[k];
            phi[2 * k + 1] = p[3 + k] - x[k];
            for (int m = 0; m < 3; ++m) {
                n[3 * (2 * k) + m] = (m == k) ? 1.0 : 0.0;
                n[3 * (2 * k + 1) + m] = (m == k) ? -1.0 : 0.0;
            }
        }
        return 6;
    }
    if (kind == SDF_CONE_SHELL) {
        double dx = x[0] - p[0], dy = x[1] - p[1];
        double rho = sqrt(dx * dx + dy * dy);
        double rx = 1.0, ry = 0.0;
        if (rho > 0) { rx = dx / rho; ry = dy / rho; }
        double e[2] = {p[5] - p[3], p[4] - p[2]};          /* (rho, z) segment direction */
        double q[2] = {rho - p[3], x[2] - p[2]};
        double ee = e[0] * e[0] + e[1] * e[1];
        double t = (q[0] * e[0] + q[1] * e[1]) / ee;
        if (t < 0) t = 0;
        if (t > 1) t = 1;
        double dq[2] = {q[0] - t * e[0], q[1] - t * e[1]};
        double dist = sqrt(dq[0] * dq[0] + dq[1] * dq[1]);
        double n2[2];
        if (dist > 0) { n2[0] = dq[0] / dist; n2[1] = dq[1] / dist; }
        else { double le = sqrt(ee); n2[0] = -e[1] / le; n2[1] = e[0] / le; }
        /* on the mid-surface the side the particle is pushed to is not
         * unique */
        if (dist <= eps) *tie = 1;
        phi[0] = dist - p[6];
        n[0] = n2[0] * rx;
        n[1] = n2[0] * ry;
        n[2] = n2[1];
        return 1;
    }
    if (kind == SDF_SOLID_BOX) {
        double d[3], q[3], sg[3];
        int outside = 0;
        for (int k = 0; k < 3; ++k) {
            d[k] = x[k] - p[k];
            sg[k] = d[k] < 0 ? -1.0 : 1.0;
            q[k] = fabs(d[k]) - p[3 + k];
            if (q[k] > 0) outside = 1;
        }
        if (outside) {
            double qp[3], l2 = 0;
            for (int k = 0; k < 3; ++k) { qp[k] = q[k] > 0 ? q[k] : 0; l2 += qp[k] * qp[k]; }
            double l = sqrt(l2);
            phi[0] = l;
            for (int k = 0; k < 3; ++k) n[k] = sg[k] * qp[k] / l;
        } else {
            int a = 0;
            for (int k = 1; k < 3; ++k)
                if (q[k] > q[a]) a = k;
            for (int k = 0; k < 3; ++k)
                if (k != a && q[a] - q[k] <= eps) *tie = 1;
            phi[0] = q[a];
            n[0] = n[1] = n[2] = 0;
            n[a] = sg[a];
        }
        return 1;
    }
    return 0;
}

static int sdf_ncomp(const double* rec)
{
    int kind = (int)rec[0];
    return kind == SDF_BOX_INTERIOR ? 6 : ((kind == SDF_CONE_SHELL || kind == SDF_SOLID_BOX) ? 1 : 0);
}

/* ------------------------------------------------------------------ */
/* HR upsampling, Sec. 4.                                               */
/* ------------------------------------------------------------------ */

/* Distance weight between a HR and a LR particle (Sec. 4):
 *   w = max(0, (1 - |x_ij|^2 / (9 r_LR^2))^3)                          */
double or_weight(double d2, double r_low)
{
    double t = 1.0 - d2 / (9.0 * r_low * r_low);
    double w = t * t * t;
    return w > 0 ? w : 0.0;
}

/* Decision tapes.  The method is piecewise smooth: the blend branch, the
 * largest weight, contact activation, static or kinetic friction and the
 * SDF active set switch discontinuously.  A tape records these decisions in
 * one evaluation (tape mode 1) and imposes them in another (mode 2), which
 * then evaluates the formula of each recorded branch even where the
 * comparison would now go the other way.  The replayed map is the smooth
 * piece that contains the recording point; its derivative is the one the
 * reverse modes compute, so finite differences of replays check them. */
enum { TAPE_OFF = 0, TAPE_RECORD = 1, TAPE_REPLAY = 2 };

/* Advection and boundary handling of one HR particle after the blend
 * parameter alpha is known (Sec. 4):
 *   v^{t+1} = (1 - alpha) vtilde + alpha (v^t + dt g),
 *   x^{t+1} = x^t + dt v^{t+1}.
 * The paper states only that advection was modified for the domain
 * boundaries (Sec. 2, last paragraph) and gives no formula.  Reading used
 * here: each SDF contact component, in list order, projects the particle to
 * phi = r_HR along n and removes the normal velocity component that points
 * into the boundary relative to the boundary velocity u_b; the tangential
 * part is kept.
 * flip_k >= 0 inverts the k-th contact decision (used for the alternative
 * branch).  Ambiguous contact decisions are appended to amb[]. */
static void hr_finish(const double* x0, const double* v0, const double* vt, double alpha,
                      const double* sdf, int n_sdf, const double* prm, int flip_k,
                      double* xo, double* vo, int* amb, int* n_amb, int* hard, int* n_act,
                      int tmode, uint32_t* tp)
{
    double dt = prm[UP_DT], rh = prm[UP_R_HIGH], eps_x = prm[UP_EPS_X];
    const double g[3] = {prm[UP_GX], prm[UP_GY], prm[UP_GZ]};
    for (int k = 0; k < 3; ++k) {
        vo[k] = (1.0 - alpha) * vt[k] + alpha * (v0[k] + dt * g[k]);
        xo[k] = x0[k] + dt * vo[k];
    }
    int dec = 0;
    for (int s = 0; s < n_sdf; ++s) {
        const double* rec = sdf + OR_SDF_STRIDE * s;
        const double* ub = rec + 13;
        int nc = sdf_ncomp(rec);
        for (int c = 0; c < nc; ++c, ++dec) {
            /* re-evaluated after every applied component: sequential */
            double phi[OR_MAX_COMP], nn[3 * OR_MAX_COMP];
            int tie;
            or_sdf_eval(rec, xo, phi, nn, &tie, eps_x);
            int active = phi[c] < rh;
            if (fabs(phi[c] - rh) <= eps_x) amb[(*n_amb)++] = dec;
            if (dec == flip_k) active = !active;
            /* tape words: tp[0] bit dec = component active, tp[1] bit dec =
             * normal velocity removed */
            if (tmode == TAPE_REPLAY) active = (tp[0] >> dec) & 1u;
            else if (tmode == TAPE_RECORD && active) tp[0] |= 1u << dec;
            if (!active) continue;
            if (tie) *hard = 1;
            if (n_act) ++*n_act;
            const double* n = nn + 3 * c;
            double push = rh - phi[c];
            for (int k = 0; k < 3; ++k) xo[k] += push * n[k];
            double vr[3] = {vo[0] - ub[0], vo[1] - ub[1], vo[2] - ub[2]};
            double vn = dot3(vr, n);
            int rem = vn < 0;
            if (tmode == TAPE_REPLAY) rem = (tp[1] >> dec) & 1u;
            else if (tmode == TAPE_RECORD && rem) tp[1] |= 1u << dec;
            if (rem)
                for (int k = 0; k < 3; ++k) vo[k] -= vn * n[k];
        }
    }
}

/* One HR frame.  lr_x, lr_v: LR state after the latest LR step (x^{t+1},
 * v^{t+1}); hr_x, hr_v: HR state at t.  sub (optional) selects which HR
 * particles to compute; outputs are indexed by position in sub.
 * mode 0 sums over every LR particle (the definition); mode 1 restricts the
 * sum to the LR particles a plain grid returns within 3 r_LR, in ascending
 * index order, which gives the same sums bit for bit.
 * flag: 0 = every decision clear of its margin; 1 = exactly one decision
 * inside its margin, alt_x/alt_v hold the other branch; 2 = more than one
 * (or a non-unique SDF normal), alt = primary.
 * diag (optional, 6 per output): sum w, max w, alpha, #LR with w > 0, and
 * the sensitivities |d x_out / d x_in| - 1 and |d v_out / d x_in| of the SDF
 * rule (0 without an active contact). */
/* solid (optional, N): 1 for LR particles of infinite mass (particle-sampled
 * boundaries and rigid bodies, Sec. 3), 0 for grains.  Sec. 4 counts both
 * in the weights, except that an HR particle with no grain of positive
 * weight in its support ignores the solid ones (the paper's rule against HR
 * particles sticking to rigid bodies moved externally): sum w = 0, alpha =
 * 1, ballistic motion.  A grain whose t = 1 - |x_ij|^2 / (9 r_LR^2) lies
 * within kRuleEps of 0 makes that decision ambiguous (flag 2). */
#define kRuleEps 4e-6
static int upsample_impl(const double* lr_x, const double* lr_v, long N,
                         const double* hr_x, const double* hr_v, long M,
                         const long* sub, long n_sub,
                         const double* sdf, int n_sdf, const double* prm, int mode,
                         double* out_x, double* out_v, int* flag, double* alt_x, double* alt_v, double* diag,
                         int tmode, uint32_t* tape, const unsigned char* solid)
{
    double r = prm[UP_R_LOW], c1 = prm[UP_C1], c2 = prm[UP_C2], eps_w = prm[UP_EPS_W];
    double R2 = 9.0 * r * r;
    long n_out = sub ? n_sub : M;
    or_grid_t grid;
    if (mode == 1 && grid_build(&grid, lr_x, N, 3.0 * r) != 0) return -1;
    int nth = g_threads;
    int err = 0;
#pragma omp parallel num_threads(nth) if (nth > 1)
    {
    long* cand = NULL;
    if (mode == 1) cand = (long*)malloc((size_t)(N ? N : 1) * sizeof(long));
#pragma omp for schedule(dynamic, 64)
    for (long k = 0; k < n_out; ++k) {
        long i = sub ? sub[k] : k;
        if (i < 0 || i >= M) { err = -2; continue; }
        const double* xi = hr_x + 3 * i;
        const double* vi = hr_v + 3 * i;
        double S = 0, V[3] = {0, 0, 0}, wmax = 0;
        long cnt = 0, jstar = -1;
        long nc = N;
        int grain_hit = 0, grain_edge = 0;
        if (mode == 1) nc = grid_query(&grid, xi, cand);
        for (long q = 0; q < nc; ++q) {
            long j = cand ? cand[q] : q;
            double d[3] = {xi[0] - lr_x[3 * j], xi[1] - lr_x[3 * j + 1], xi[2] - lr_x[3 * j + 2]};
            double d2 = dot3(d, d);
            if (solid && !solid[j] && fabs(1.0 - d2 / R2) <= kRuleEps) grain_edge = 1;
            if (!(d2 < R2)) continue;
            double w = or_weight(d2, r);
            if (solid && !solid[j] && w > 0 && 1.0 - d2 / R2 > kRuleEps) grain_hit = 1;
            S += w;
            for (int m = 0; m < 3; ++m) V[m] += w * lr_v[3 * j + m];
            if (w > wmax) { wmax = w; jstar = j; }
            ++cnt;
        }
        int rule_amb = 0;
        if (solid && !grain_hit) {
            /* no grain in reach (or only at the edge of the support): the
             * solid particles are ignored */
            rule_amb = grain_edge && S > 0;
            int any_grain = 0;
            for (long q = 0; q < nc && !any_grain; ++q) {
                long j = cand ? cand[q] : q;
                if (solid[j]) continue;
                double d[3] = {xi[0] - lr_x[3 * j], xi[1] - lr_x[3 * j + 1], xi[2] - lr_x[3 * j + 2]};
                if (dot3(d, d) < R2 && or_weight(dot3(d, d), r) > 0) any_grain = 1;
            }
            if (!any_grain) {
                S = 0;
                V[0] = V[1] = V[2] = 0;
                wmax = 0;
                jstar = -1;
                cnt = 0;
            }
        }
        /* tape record of one HR particle: {argmax LR index, blend branch,
         * SDF active bits, velocity removal bits} */
        uint32_t* tp = tape ? tape + 4 * k : NULL;
        if (tmode == TAPE_REPLAY) {
            jstar = (long)(int32_t)tp[0];
            wmax = 0.0;
            if (jstar >= 0 && jstar < N) {
                double d[3] = {xi[0] - lr_x[3 * jstar], xi[1] - lr_x[3 * jstar + 1], xi[2] - lr_x[3 * jstar + 2]};
                wmax = or_weight(dot3(d, d), r);
            }
        }
        /* interpolated LR velocity; with no LR particle in reach it is
         * undefined in the paper and alpha = 1 makes it irrelevant: use 0 */
        double vt[3] = {0, 0, 0};
        if (S > 0)
            for (int m = 0; m < 3; ++m) vt[m] = V[m] / S;
        /* blend parameter (Sec. 4): alpha = 1 - max w if max w <= c1 or
         * max w / sum w >= c2, else 0 */
        int A = wmax <= c1;
        int B = S > 0 && wmax >= c2 * S;
        int Aamb = fabs(wmax - c1) <= eps_w;
        int Bamb = S > 0 && fabs(wmax - c2 * S) <= eps_w * S;
        int prim = A || B;
        if (tmode == TAPE_REPLAY) prim = (int)tp[1];
        else if (tmode == TAPE_RECORD) {
            tp[0] = (uint32_t)(int32_t)jstar;
            tp[1] = (uint32_t)prim;
            tp[2] = tp[3] = 0;
        }
        int alt_out = prim;
        if (Aamb && ((!A) || B) != prim) alt_out = !prim;
        if (Bamb && (A || (!B)) != prim) alt_out = !prim;
        if (Aamb && Bamb && ((!A) || (!B)) != prim) alt_out = !prim;
        double alpha = prim ? 1.0 - wmax : 0.0;
        int amb[64], n_amb = 0, hard = rule_amb, n_act = 0;
        double xo[3], vo[3];
        hr_finish(xi, vi, vt, alpha, sdf, n_sdf, prm, -1, xo, vo, amb, &n_amb, &hard, &n_act, tmode,
                  tp ? tp + 2 : NULL);
        if (tmode != TAPE_OFF) {
            /* taped evaluation: no branch diagnostics */
            for (int m = 0; m < 3; ++m) { out_x[3 * k + m] = xo[m]; out_v[3 * k + m] = vo[m]; }
            continue;
        }
        int n_total = n_amb + (alt_out != prim);
        double ax[3] = {xo[0], xo[1], xo[2]}, av[3] = {vo[0], vo[1], vo[2]};
        int fl = 0;
        if (hard || n_total > 1) fl = 2;
        else if (n_total == 1) {
            fl = 1;
            int tmp[64], nt = 0, h2 = 0;
            if (alt_out != prim)
                hr_finish(xi, vi, vt, prim ? 0.0 : 1.0 - wmax, sdf, n_sdf, prm, -1, ax, av, tmp, &nt, &h2, NULL,
                          TAPE_OFF, NULL);
            else
                hr_finish(xi, vi, vt, alpha, sdf, n_sdf, prm, amb[0], ax, av, tmp, &nt, &h2, NULL, TAPE_OFF,
                          NULL);
        }
        /* Conditioning of the SDF rule: near an edge or corner of a boundary
         * the contact normal turns quickly with position, so a rounding of
         * the advected position changes the result by more than the
         * rounding itself.  Estimated by moving the particle by +-eps_x
         * along each axis (decisions kept as they fall). */
        double sens_x = 0.0, sens_v = 0.0;
        if (n_act > 0 && !hard) {
            double dlt = prm[UP_EPS_X];
            for (int a = 0; a < 3; ++a)
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    double xp[3] = {xi[0], xi[1], xi[2]}, px[3], pv[3];
                    int tmp[64], nt = 0, h2 = 0;
                    xp[a] += sgn * dlt;
                    hr_finish(xp, vi, vt, alpha, sdf, n_sdf, prm, -1, px, pv, tmp, &nt, &h2, NULL, TAPE_OFF,
                              NULL);
                    if (nt != n_amb) continue;   /* a decision flipped: covered by the flags */
                    double ex[3] = {px[0] - xo[0], px[1] - xo[1], px[2] - xo[2]};
                    ex[a] -= sgn * dlt;
                    double ev[3] = {pv[0] - vo[0], pv[1] - vo[1], pv[2] - vo[2]};
                    double sx = sqrt(dot3(ex, ex)) / dlt, sv = sqrt(dot3(ev, ev)) / dlt;
                    if (sx > sens_x) sens_x = sx;
                    if (sv > sens_v) sens_v = sv;
                }
        }
        for (int m = 0; m < 3; ++m) {
            out_x[3 * k + m] = xo[m];
            out_v[3 * k + m] = vo[m];
            if (alt_x) alt_x[3 * k + m] = ax[m];
            if (alt_v) alt_v[3 * k + m] = av[m];
        }
        if (flag) flag[k] = fl;
        if (diag) {
            diag[6 * k] = S;
            diag[6 * k + 1] = wmax;
            diag[6 * k + 2] = alpha;
            diag[6 * k + 3] = (double)cnt;
            diag[6 * k + 4] = sens_x;
            diag[6 * k + 5] = sens_v;
        }
    }
    free(cand);
    }
    if (mode == 1) grid_free(&grid);
    return err;
}

int or_upsample(const double* lr_x, const double* lr_v, long N,
                const double* hr_x, const double* hr_v, long M,
                const long* sub, long n_sub,
                const double* sdf, int n_sdf, const double* prm, int mode,
                double* out_x, double* out_v, int* flag, double* alt_x, double* alt_v, double* diag)
{
    return upsample_impl(lr_x, lr_v, N, hr_x, hr_v, M, sub, n_sub, sdf, n_sdf, prm, mode, out_x, out_v, flag,
                         alt_x, alt_v, diag, TAPE_OFF, NULL, NULL);
}

/* or_upsample with particle-sampled boundaries and rigid bodies: solid[j]
 * = 1 marks LR particle j as one of infinite mass (see upsample_impl). */
int or_upsample_solid(const double* lr_x, const double* lr_v, const unsigned char* solid, long N,
                      const double* hr_x, const double* hr_v, long M,
                      const long* sub, long n_sub,
                      const double* sdf, int n_sdf, const double* prm, int mode,
                      double* out_x, double* out_v, int* flag, double* alt_x, double* alt_v, double* diag)
{
    if (!solid && N > 0) return -1;
    return upsample_impl(lr_x, lr_v, N, hr_x, hr_v, M, sub, n_sub, sdf, n_sdf, prm, mode, out_x, out_v, flag,
                         alt_x, alt_v, diag, TAPE_OFF, NULL, solid);
}

static int total_components(const double* sdf, int n_sdf)
{
    int t = 0;
    for (int s = 0; s < n_sdf; ++s) t += sdf_ncomp(sdf + OR_SDF_STRIDE * s);
    return t;
}

/* One HR frame (grid neighbour search) that records its decisions into, or
 * replays them from, tape = uint32[M][4].  At most 32 SDF components. */
int or_upsample_tape(const double* lr_x, const double* lr_v, long N, const double* hr_x, const double* hr_v, long M,
                     const double* sdf, int n_sdf, const double* prm, int tmode, uint32_t* tape,
                     double* out_x, double* out_v)
{
    if ((tmode != TAPE_RECORD && tmode != TAPE_REPLAY) || !tape || total_components(sdf, n_sdf) > 32) return -1;
    return upsample_impl(lr_x, lr_v, N, hr_x, hr_v, M, NULL, 0, sdf, n_sdf, prm, 1, out_x, out_v, NULL, NULL, NULL,
                         NULL, tmode, tape, NULL);
}

/* ------------------------------------------------------------------ */
/* LR step, Sec. 3 and Algorithm 1.                                     */
/* ------------------------------------------------------------------ */

typedef struct { long i, j; } or_pair;

/* Candidate pairs i < j with |xt_i - xt_j| < Rc, ordered by (i, j).  Pairs
 * whose distance is within eps_x of Rc are marked in border[] (kept pairs)
 * or listed in *out_excl (dropped pairs): a float32 implementation may
 * decide them the other way. */
static long make_pairs(const double* xt, long N, double Rc, int mode, or_pair** out, unsigned char** border,
                       or_pair** out_excl, long* n_excl, double eps_x)
{
    long cap = 1024, n = 0, cap_e = 64, ne = 0;
    or_pair* P = (or_pair*)malloc((size_t)cap * sizeof(or_pair));
    unsigned char* B = (unsigned char*)malloc((size_t)cap);
    or_pair* E = (or_pair*)malloc((size_t)cap_e * sizeof(or_pair));
    if (!P || !B || !E) return -1;
    double R2 = Rc * Rc;
    or_grid_t g;
    long* cand = NULL;
    if (mode == 1) {
        if (grid_build(&g, xt, N, Rc + eps_x) != 0) return -1;
        cand = (long*)malloc((size_t)(N ? N : 1) * sizeof(long));
    }
    for (long i = 0; i < N; ++i) {
        long nc = N, q0 = i + 1;
        if (mode == 1) { nc = grid_query(&g, xt + 3 * i, cand); q0 = 0; }
        for (long q = q0; q < nc; ++q) {
            long j = cand ? cand[q] : q;
            if (j <= i) continue;
            double d[3] = {xt[3 * j] - xt[3 * i], xt[3 * j + 1] - xt[3 * i + 1], xt[3 * j + 2] - xt[3 * i + 2]};
            double d2 = dot3(d, d);
            int bord = fabs(sqrt(d2) - Rc) <= eps_x;
            if (!(d2 < R2)) {
                if (bord) {
                    if (ne == cap_e) { cap_e *= 2; E = (or_pair*)realloc(E, (size_t)cap_e * sizeof(or_pair)); }
                    E[ne].i = i; E[ne].j = j; ++ne;
                }
                continue;
            }
            if (n == cap) {
                cap *= 2;
                P = (or_pair*)realloc(P, (size_t)cap * sizeof(or_pair));
                B = (unsigned char*)realloc(B, (size_t)cap);
                if (!P || !B) return -1;
            }
            P[n].i = i;
            P[n].j = j;
            B[n] = (unsigned char)bord;
            ++n;
        }
    }
    if (mode == 1) { free(cand); grid_free(&g); }
    *out = P;
    *border = B;
    *out_excl = E;
    *n_excl = ne;
    return n;
}

/* One decision taken within its margin: had it gone the other way, the
 * particle's summed correction would change by dD and its constraint count
 * by dn. */
typedef struct { long i; double dD[3]; int dn; } or_alt;

typedef struct { or_alt* a; long n, cap; } or_alts;

static void alt_push(or_alts* L, long i, const double* dD, int dn)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->a = (or_alt*)realloc(L->a, (size_t)L->cap * sizeof(or_alt));
    }
    or_alt* e = &L->a[L->n++];
    e->i = i;
    e->dn = dn;
    for (int k = 0; k < 3; ++k) e->dD[k] = dD[k];
}

/* Friction delta of Eqs. 3-4 for a relative tangential displacement perp
 * (the caller multiplies by the mass ratio and the sign).  thr_s / thr_k
 * are the static / kinetic thresholds.  When the static test is within eps
 * of its threshold and the branches differ, *amb is set and f_alt holds the
 * other branch. */
static void friction_delta(const double* perp, double thr_s, double thr_k, double eps_x, double* f, double* f_alt,
                           int* amb, int tmode, unsigned char* bits)
{
    double L = sqrt(dot3(perp, perp));
    double kin = (L > 0 && thr_k / L < 1.0) ? thr_k / L : 1.0;
    double scale = L < thr_s ? 1.0 : kin;
    double other = L < thr_s ? kin : 1.0;
    *amb = fabs(L - thr_s) <= eps_x && scale != other;
    /* tape bit 1: the kinetic scale thr_k / |perp| applies (otherwise the
     * whole tangential displacement is removed) */
    if (tmode == TAPE_RECORD && !(L < thr_s) && L > 0 && thr_k / L < 1.0) *bits |= 2;
    if (tmode == TAPE_REPLAY) {
        scale = ((*bits & 2) && L > 0) ? thr_k / L : 1.0;
        other = scale;
        *amb = 0;
    }
    for (int k = 0; k < 3; ++k) {
        f[k] = perp[k] * scale;
        f_alt[k] = perp[k] * other;
    }
}

/* One LR time step (Algorithm 1) on N particles.
 *
 * x, v: double[N][3], updated in place.  inv_m: inverse masses m^-1 (0 =
 * immovable).  Readings of the passages that are silent or garbled:
 *  - Height-scaled mass m* = m e^{-h(x)} (Sec. 3, stable piling) with
 *    h = k (z - ground_z) in metres; k = prm[PB_MASS_K]; it is evaluated at
 *    the positions at the start of the step.
 *  - Stabilization (Sec. 3, Algorithm 1) repairs positions that are invalid
 *    at the start of the step, so its contact-only constraints are
 *    evaluated on x (as updated by earlier stabilization passes) and the
 *    resulting delta is applied to both x and xt.  Evaluating them on xt
 *    would cancel the gravity-induced penetration without touching the
 *    velocity, and a resting particle would fall ever faster.
 *  - Candidate constraints are generated once per step after the
 *    prediction, from every pair with |xt_i - xt_j| < Rc; a candidate is an
 *    active contact in a pass when |x_ij| < 2 r_LR (Eqs. 1-2).  A pair at
 *    exactly zero distance has no direction and is skipped.
 *  - Friction (Eqs. 3-4): read literally, the displacement is the contact
 *    correction itself, which is parallel to x_ij and has no tangential
 *    part.  Reading used: the relative displacement over the step so far,
 *    (xt_i - x_i) - (xt_j - x_j), as in the unified-particle friction model
 *    the paper builds on.  Static branch below 2 r_LR mu_s, kinetic branch
 *    scaled by min(2 r_LR mu_k / |dx_perp|, 1).  friction mode 1 uses the
 *    penetration depth (2 r_LR - |x_ij|) in place of 2 r_LR, following the
 *    prose that follows Eqs. 3-4.
 *  - Cross coefficients mu_ij = sqrt(mu_i mu_j) (Sec. 3), the static and
 *    the kinetic one each from the two partners' own: between two grains
 *    when per-particle coefficients mu (N x 2: mu_s, mu_k) are given, and
 *    between a grain and an SDF boundary.  Without mu every grain has the
 *    step's mu_s, mu_k.
 *  - A contact pair (penetration + friction) counts once towards n_i;
 *    each active SDF contact component counts once; particles with n_i = 0
 *    are not moved.  No over-relaxation.
 *  - SDF contacts: a pair with an immovable partner (mass ratio 1), active
 *    when phi(xt_i) < r_LR, penetration (r_LR - phi) along n; friction uses
 *    the displacement relative to the boundary's displacement u_b dt.
 * Decisions taken within eps_x of their threshold (contact active, static or
 * kinetic friction, SDF contact active, candidate membership) are evaluated
 * both ways; when the other branch would move the particle's averaged
 * correction by more than eps_impact the particle is suspect, and so is
 * every candidate partner of a suspect in later passes.
 * suspect (optional, N): 1 for suspect particles.
 * stats (optional): [0] #candidate pairs, [1] #significant ambiguous
 * decisions, [2] max candidates of one particle, [3] #active pair contacts
 * in the last pass, [4] #ambiguous decisions (significant or not). */
/* Tape of one LR step (bytes): int64 header {#pairs, N, #SDF components,
 * #passes}, the candidate pairs as int64 (i, j), then per pass one byte per
 * pair and one per (particle, SDF component): bit 0 = contact active,
 * bit 1 = kinetic friction scale applies. */
static long pbd_tape_bytes(long np, long N, int nct, int passes)
{
    return 32 + 16 * np + (long)passes * (np + N * (long)nct);
}

/* Rotation of the polar decomposition C = R S (S symmetric positive
 * definite): R = C (C^T C)^(-1/2), with (C^T C)^(-1/2) from the eigen-
 * decomposition of C^T C by cyclic Jacobi rotations (the textbook method).
 * When det C < 0 the closest rotation flips the direction of the smallest
 * singular value: R = C S^-1 - 2 u3 v3^T with v3 its eigenvector and u3 =
 * C v3 / sigma3.  Returns -1 for a degenerate C (smallest eigenvalue below
 * 1e-24 of the largest: a body whose rest shape is flat or a line). */
static int polar_rotation(const double C[9], double R[9])
{
    double S[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += C[3 * k + a] * C[3 * k + b];
            S[3 * a + b] = s;
        }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = fabs(S[1]) + fabs(S[2]) + fabs(S[5]);
        double norm = fabs(S[0]) + fabs(S[4]) + fabs(S[8]);
        if (off <= 1e-18 * norm) break;
        for (int pp = 0; pp < 2; ++pp)
            for (int q = pp + 1; q < 3; ++q) {
                double apq = S[3 * pp + q];
                if (apq == 0.0) continue;
                double theta = (S[3 * q + q] - S[3 * pp + pp]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {   /* S <- J^T S J, columns then rows */
                    double skp = S[3 * k + pp], skq = S[3 * k + q];
                    S[3 * k + pp] = c * skp - s * skq;
                    S[3 * k + q] = s * skp + c * skq;
                }
                for (int k = 0; k < 3; ++k) {
                    double spk = S[3 * pp + k], sqk = S[3 * q + k];
                    S[3 * pp + k] = c * spk - s * sqk;
                    S[3 * q + k] = s * spk + c * sqk;
                }
                for (int k = 0; k < 3; ++k) {   /* V <- V J */
                    double vkp = V[3 * k + pp], vkq = V[3 * k + q];
                    V[3 * k + pp] = c * vkp - s * vkq;
                    V[3 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    double lam[3] = {S[0], S[4], S[8]};
    double lmax = fmax(lam[0], fmax(lam[1], lam[2]));
    int kmin = 0;
    for (int k = 1; k < 3; ++k)
        if (lam[k] < lam[kmin]) kmin = k;
    if (!(lmax > 0) || !(lam[kmin] > 1e-24 * lmax)) return -1;
    double Sinv[9];   /* V diag(lam^-1/2) V^T */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += V[3 * a + k] * V[3 * b + k] / sqrt(lam[k]);
            Sinv[3 * a + b] = s;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += C[3 * a + k] * Sinv[3 * k + b];
            R[3 * a + b] = s;
        }
    double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                 R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (det < 0) {
        double v3[3] = {V[kmin], V[3 + kmin], V[6 + kmin]}, u3[3];
        double sig = sqrt(lam[kmin]);
        for (int a = 0; a < 3; ++a) u3[a] = (C[3 * a] * v3[0] + C[3 * a + 1] * v3[1] + C[3 * a + 2] * v3[2]) / sig;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) R[3 * a + b] -= 2.0 * u3[a] * v3[b];
    }
    return 0;
}

int or_polar_rotation(const double* C, double* R) { return polar_rotation(C, R); }

/* Shape matching of rigid bodies (Sec. 3): body[i] = b >= 1 puts particle i
 * in body b (0: a grain); xo[i] is its offset from the body's centre of mass
 * at rest.  In every solver pass each body, from the pass's positions xt:
 *   c = sum m xt / sum m (m = 1 / inv_m, the unscaled masses),
 *   C = sum m (xt - c) xo^T,  R = rotation of the polar decomposition of C,
 * and each of its particles receives the constraint delta (R xo + c) - xt,
 * counted once in n_i. */
typedef struct {
    const int* body;
    const double* xo;
    int n_bodies;
} or_bodies;

/* Everything one Jacobi pass of the LR step reads and writes. */
typedef struct {
    long N;
    double *x, *xt;                /* [N][3]: start-of-step positions (as stabilized so far), predictions */
    const double* ws;              /* [N] inverse height-scaled masses 1/m* */
    const double* inv_m;           /* [N] inverse masses (rigid bodies use the unscaled masses) */
    const double* sdf;
    int n_sdf, nct;
    const double* mu;              /* [N][2] per-particle (mu_s, mu_k), or NULL */
    const or_bodies* bodies;
    double r, dt, mu_s, mu_k, d0, eps_x, eps_imp;
    int fmode;
    const or_pair* P;              /* candidate pairs and their border flags */
    const unsigned char* border;
    long np;
    const or_pair* E;              /* pairs dropped within eps_x of the candidate radius */
    long n_excl;
    int tmode;
    /* scratch and outputs */
    double* D;                     /* [N][3] summed corrections */
    long* cnt;                     /* [N] constraint counts n_i */
    unsigned char* mark;           /* [N] suspect particles */
    or_alts alts;
    long n_sig, n_amb, active_last;
} pbd_work;

/* One Jacobi pass (Algorithm 1; Eqs. 1-2, plus Eqs. 3-4 in a solver pass):
 * every constraint is evaluated on the pass's input, the corrections are
 * summed per particle and averaged, delta_i = (1/n_i) sum_k delta_ik, and
 * applied to xt (and to x in a stabilization pass).  tpair (tape modes): the
 * pass's decision bytes, one per pair then one per (particle, SDF
 * component).  Returns 0, or -1 / -4 on allocation / degenerate-body
 * failures. */
static int pbd_pass(pbd_work* w, int stab, unsigned char* tpair)
{
    const long N = w->N;
    double *x = w->x, *xt = w->xt, *D = w->D;
    const double* ws = w->ws;
    long* cnt = w->cnt;
    unsigned char* mark = w->mark;
    const double r = w->r, dt = w->dt, d0 = w->d0, eps_x = w->eps_x;
    const int tmode = w->tmode;
    unsigned char* tsdf = tpair ? tpair + w->np : NULL;
    memset(D, 0, (size_t)N * 3 * sizeof(double));
    memset(cnt, 0, (size_t)N * sizeof(long));
    w->alts.n = 0;
    w->active_last = 0;
    /* Stabilization repairs invalid positions at the start of the step
     * (Sec. 3): its contacts are evaluated on x, the solver's on xt. */
    const double* y = stab ? x : xt;
    /* a candidate pair decided the other way by a float32 neighbour
     * search matters only if it comes into contact */
    for (long p = 0; p < w->n_excl; ++p) {
        long i = w->E[p].i, j = w->E[p].j;
        double e[3] = {y[3 * j] - y[3 * i], y[3 * j + 1] - y[3 * i + 1], y[3 * j + 2] - y[3 * i + 2]};
        if (sqrt(dot3(e, e)) < d0 + eps_x) { mark[i] = mark[j] = 1; ++w->n_sig; }
    }
    /* particle-particle contacts: Eqs. 1-2 (+ Eqs. 3-4 when solving) */
    for (long p = 0; p < w->np; ++p) {
        long i = w->P[p].i, j = w->P[p].j;
        double xij[3] = {y[3 * j] - y[3 * i], y[3 * j + 1] - y[3 * i + 1], y[3 * j + 2] - y[3 * i + 2]};
        double d2 = dot3(xij, xij);
        double d = sqrt(d2);
        if (w->border[p] && d < d0 + eps_x) { mark[i] = mark[j] = 1; ++w->n_sig; }
        int active = d < d0;
        int amb_act = fabs(d - d0) <= eps_x;
        if (tmode == TAPE_REPLAY) { active = tpair[p] & 1; amb_act = 0; }
        else if (tmode == TAPE_RECORD && active) tpair[p] |= 1;
        if ((!active && !amb_act) || d2 == 0.0) continue;
        double wsum = ws[i] + ws[j];
        if (!(wsum > 0)) continue;
        double mi = ws[i] / wsum, mj = ws[j] / wsum;
        double pen = d0 - d;
        double u[3] = {xij[0] / d, xij[1] / d, xij[2] / d};
        double ci[3], cj[3], ci_alt[3], cj_alt[3];
        int amb_f = 0;
        for (int k = 0; k < 3; ++k) {
            ci[k] = -mi * pen * u[k];
            cj[k] = mj * pen * u[k];
        }
        memcpy(ci_alt, ci, sizeof ci);
        memcpy(cj_alt, cj, sizeof cj);
        if (!stab) {
            double dx[3], perp[3], f[3], fa[3];
            for (int k = 0; k < 3; ++k)
                dx[k] = (xt[3 * i + k] - x[3 * i + k]) - (xt[3 * j + k] - x[3 * j + k]);
            double a = dot3(dx, xij) / d2;
            for (int k = 0; k < 3; ++k) perp[k] = dx[k] - a * xij[k];
            double base = (w->fmode == 1) ? pen : d0;
            double pmu_s = w->mu_s, pmu_k = w->mu_k;
            if (w->mu) {   /* cross coefficients of the pair (Sec. 3) */
                pmu_s = sqrt(w->mu[2 * i] * w->mu[2 * j]);
                pmu_k = sqrt(w->mu[2 * i + 1] * w->mu[2 * j + 1]);
            }
            friction_delta(perp, base * pmu_s, base * pmu_k, eps_x, f, fa, &amb_f, tmode, tpair ? tpair + p : NULL);
            for (int k = 0; k < 3; ++k) {
                ci_alt[k] = ci[k] - mi * fa[k];
                cj_alt[k] = cj[k] + mj * fa[k];
                ci[k] -= mi * f[k];
                cj[k] += mj * f[k];
            }
        }
        if (active) {
            for (int k = 0; k < 3; ++k) {
                D[3 * i + k] += ci[k];
                D[3 * j + k] += cj[k];
            }
            cnt[i]++;
            cnt[j]++;
            ++w->active_last;
        }
        if (amb_act) {
            double si = active ? -1.0 : 1.0;
            double a1[3] = {si * ci[0], si * ci[1], si * ci[2]}, a2[3] = {si * cj[0], si * cj[1], si * cj[2]};
            alt_push(&w->alts, i, a1, active ? -1 : 1);
            alt_push(&w->alts, j, a2, active ? -1 : 1);
        }
        if (amb_f && active) {
            double a1[3] = {ci_alt[0] - ci[0], ci_alt[1] - ci[1], ci_alt[2] - ci[2]};
            double a2[3] = {cj_alt[0] - cj[0], cj_alt[1] - cj[1], cj_alt[2] - cj[2]};
            alt_push(&w->alts, i, a1, 0);
            alt_push(&w->alts, j, a2, 0);
        }
    }
    /* SDF contacts */
    for (long i = 0; i < N; ++i) {
        if (!(ws[i] > 0)) continue;
        int comp0 = 0;
        for (int s = 0; s < w->n_sdf; comp0 += sdf_ncomp(w->sdf + OR_SDF_STRIDE * s), ++s) {
            const double* rec = w->sdf + OR_SDF_STRIDE * s;
            double phi[OR_MAX_COMP], nn[3 * OR_MAX_COMP];
            int tie;
            int nc = or_sdf_eval(rec, y + 3 * i, phi, nn, &tie, eps_x);
            const double* ub = rec + 13;
            double gmu_s = w->mu ? w->mu[2 * i] : w->mu_s, gmu_k = w->mu ? w->mu[2 * i + 1] : w->mu_k;
            double bmu_s = sqrt(gmu_s * rec[16]), bmu_k = sqrt(gmu_k * rec[17]);
            for (int c = 0; c < nc; ++c) {
                int active = phi[c] < r;
                int amb_act = fabs(phi[c] - r) <= eps_x;
                unsigned char* tb = tsdf ? tsdf + i * (long)w->nct + comp0 + c : NULL;
                if (tmode == TAPE_REPLAY) { active = *tb & 1; amb_act = 0; }
                else if (tmode == TAPE_RECORD && active) *tb |= 1;
                if (!active && !amb_act) continue;
                if (tie) { mark[i] = 1; ++w->n_sig; }
                const double* n = nn + 3 * c;
                double pen = r - phi[c];
                double ci[3], ci_alt[3];
                int amb_f = 0;
                for (int k = 0; k < 3; ++k) ci[k] = pen * n[k];
                memcpy(ci_alt, ci, sizeof ci);
                if (!stab) {
                    double dx[3], perp[3], f[3], fa[3];
                    for (int k = 0; k < 3; ++k) dx[k] = (xt[3 * i + k] - x[3 * i + k]) - ub[k] * dt;
                    double a = dot3(dx, n);
                    for (int k = 0; k < 3; ++k) perp[k] = dx[k] - a * n[k];
                    double base = (w->fmode == 1) ? pen : d0;
                    friction_delta(perp, base * bmu_s, base * bmu_k, eps_x, f, fa, &amb_f, tmode, tb);
                    for (int k = 0; k < 3; ++k) {
                        ci_alt[k] = ci[k] - fa[k];
                        ci[k] -= f[k];
                    }
                }
                if (active) {
                    for (int k = 0; k < 3; ++k) D[3 * i + k] += ci[k];
                    cnt[i]++;
                }
                if (amb_act) {
                    double si = active ? -1.0 : 1.0;
                    double a1[3] = {si * ci[0], si * ci[1], si * ci[2]};
                    alt_push(&w->alts, i, a1, active ? -1 : 1);
                }
                if (amb_f && active) {
                    double a1[3] = {ci_alt[0] - ci[0], ci_alt[1] - ci[1], ci_alt[2] - ci[2]};
                    alt_push(&w->alts, i, a1, 0);
                }
            }
        }
    }
    /* shape matching of the rigid bodies (solver passes) */
    if (!stab && w->bodies && w->bodies->n_bodies > 0) {
        const or_bodies* bd = w->bodies;
        int nb = bd->n_bodies;
        double* acc = (double*)calloc((size_t)nb * 13, sizeof(double));   /* M, sum m xt, sum m xt xo^T */
        double* tf = (double*)malloc((size_t)nb * 12 * sizeof(double));   /* R, c */
        if (!acc || !tf) return -1;
        for (long i = 0; i < N; ++i) {
            int b = bd->body[i];
            if (b < 1 || b > nb) continue;
            double m = 1.0 / w->inv_m[i], *a = acc + 13 * (b - 1);
            a[0] += m;
            for (int k = 0; k < 3; ++k) a[1 + k] += m * xt[3 * i + k];
            for (int rr = 0; rr < 3; ++rr)
                for (int ss = 0; ss < 3; ++ss) a[4 + 3 * rr + ss] += m * xt[3 * i + rr] * bd->xo[3 * i + ss];
        }
        for (int b = 0; b < nb; ++b) {
            double *a = acc + 13 * b, *t = tf + 12 * b, C[9];
            if (!(a[0] > 0)) continue;
            for (int k = 0; k < 3; ++k) t[9 + k] = a[1 + k] / a[0];
            /* C = sum m xt xo^T - c sum m xo^T, and sum m xo = 0 at rest */
            for (int k = 0; k < 9; ++k) C[k] = a[4 + k];
            if (polar_rotation(C, t) != 0) { free(acc); free(tf); return -4; }
        }
        for (long i = 0; i < N; ++i) {
            int b = bd->body[i];
            if (b < 1 || b > nb) continue;
            const double *t = tf + 12 * (b - 1), *o = bd->xo + 3 * i;
            for (int rr = 0; rr < 3; ++rr)
                D[3 * i + rr] += t[3 * rr] * o[0] + t[3 * rr + 1] * o[1] + t[3 * rr + 2] * o[2] + t[9 + rr] - xt[3 * i + rr];
            cnt[i]++;
        }
        free(acc);
        free(tf);
    }
    /* would the other branch of an ambiguous decision move the particle
     * by more than eps_impact? */
    for (long q = 0; q < w->alts.n; ++q) {
        const or_alt* e = &w->alts.a[q];
        long i = e->i;
        double u0[3] = {0, 0, 0}, u1[3] = {0, 0, 0};
        long n0 = cnt[i], n1a = cnt[i] + e->dn;
        for (int k = 0; k < 3; ++k) {
            if (n0 > 0) u0[k] = D[3 * i + k] / (double)n0;
            if (n1a > 0) u1[k] = (D[3 * i + k] + e->dD[k]) / (double)n1a;
        }
        double dd[3] = {u1[0] - u0[0], u1[1] - u0[1], u1[2] - u0[2]};
        ++w->n_amb;
        if (sqrt(dot3(dd, dd)) > w->eps_imp) { mark[i] = 1; ++w->n_sig; }
    }
    /* Jacobi averaging: delta_i = (1/n_i) sum_k delta_ik.  Stabilization
     * applies it to xt and x, solver iterations to xt only. */
    for (long i = 0; i < N; ++i) {
        if (cnt[i] == 0) continue;
        for (int k = 0; k < 3; ++k) {
            double dd = D[3 * i + k] / (double)cnt[i];
            xt[3 * i + k] += dd;
            if (stab) x[3 * i + k] += dd;
        }
    }
    return 0;
}

/* The work record of a pass over N particles with its scratch allocated;
 * pbd_work_free releases the scratch. */
static int pbd_work_init(pbd_work* w, long N, double* x, double* xt, const double* ws, const double* inv_m,
                         const double* sdf, int n_sdf, const double* prm, const double* mu, const or_bodies* bodies,
                         int tmode)
{
    memset(w, 0, sizeof *w);
    size_t n1 = (size_t)(N ? N : 1);
    w->N = N;
    w->x = x;
    w->xt = xt;
    w->ws = ws;
    w->inv_m = inv_m;
    w->sdf = sdf;
    w->n_sdf = n_sdf;
    w->nct = total_components(sdf, n_sdf);
    w->mu = mu;
    w->bodies = bodies;
    w->r = prm[PB_R];
    w->dt = prm[PB_DT];
    w->mu_s = prm[PB_MU_S];
    w->mu_k = prm[PB_MU_K];
    w->d0 = 2.0 * w->r;
    w->eps_x = prm[PB_EPS_X];
    w->eps_imp = prm[PB_EPS_IMPACT];
    w->fmode = (int)prm[PB_FRIC_MODE];
    w->tmode = tmode;
    w->D = (double*)malloc(n1 * 3 * sizeof(double));
    w->cnt = (long*)malloc(n1 * sizeof(long));
    w->mark = (unsigned char*)calloc(n1, 1);
    return (w->D && w->cnt && w->mark) ? 0 : -1;
}

static void pbd_work_free(pbd_work* w)
{
    free(w->D);
    free(w->cnt);
    free(w->mark);
    free(w->alts.a);
}

/* Algorithm 1, first loop: v += dt g; xt = x + dt v; m* = m e^{-h(x)}
 * (Sec. 3, height-scaled mass with h = k (z - ground_z)), stored as the
 * inverse scaled mass 1/m* = m^-1 e^{h}.  Particles of infinite mass
 * (m^-1 = 0: sampled boundaries and rigid bodies, Sec. 3) keep their
 * prescribed velocity: no gravity.  v is updated in place. */
static void pbd_predict(const double* x, double* v, const double* inv_m, long N, const double* prm, double* xt,
                        double* ws)
{
    const double dt = prm[PB_DT], mass_k = prm[PB_MASS_K], ground = prm[PB_GROUND_Z];
    const double g[3] = {prm[PB_GX], prm[PB_GY], prm[PB_GZ]};
    for (long i = 0; i < N; ++i) {
        for (int k = 0; k < 3; ++k) {
            if (inv_m[i] > 0) v[3 * i + k] += dt * g[k];
            xt[3 * i + k] = x[3 * i + k] + dt * v[3 * i + k];
        }
        ws[i] = inv_m[i] * exp(mass_k * (x[3 * i + 2] - ground));
    }
}

static int pbd_impl(double* x, double* v, const double* inv_m, long N,
                    const double* sdf, int n_sdf, const double* prm, const double* mu, int mode,
                    int* suspect, long* stats, int tmode, unsigned char* tape, long tape_cap, long* tape_len,
                    const or_bodies* bodies)
{
    int n_stab = (int)prm[PB_N_STAB], iters = (int)prm[PB_ITERS];
    double dt = prm[PB_DT], Rc = prm[PB_RC], eps_x = prm[PB_EPS_X];
    size_t n1 = (size_t)(N ? N : 1);

    double* xt = (double*)malloc(n1 * 3 * sizeof(double));
    double* ws = (double*)malloc(n1 * sizeof(double));
    unsigned char* mark2 = (unsigned char*)calloc(n1, 1);
    if (!xt || !ws || !mark2) return -1;
    pbd_predict(x, v, inv_m, N, prm, xt, ws);

    /* neighbour search and constraint generation */
    or_pair *P = NULL, *E = NULL;
    unsigned char* border = NULL;
    long n_excl = 0;
    long np;
    int nct = total_components(sdf, n_sdf);
    int total = n_stab + iters;
    int64_t* th = (int64_t*)tape;
    if (tmode == TAPE_REPLAY) {
        /* the candidate pairs are part of the recorded decisions */
        if (tape_cap < 32 || th[1] != N || th[2] != nct || th[3] != total) return -3;
        np = (long)th[0];
        if (tape_cap < pbd_tape_bytes(np, N, nct, total)) return -3;
        P = (or_pair*)malloc((size_t)(np ? np : 1) * sizeof(or_pair));
        border = (unsigned char*)calloc((size_t)(np ? np : 1), 1);
        E = (or_pair*)malloc(sizeof(or_pair));
        if (!P || !border || !E) return -1;
        for (long q = 0; q < np; ++q) { P[q].i = (long)th[4 + 2 * q]; P[q].j = (long)th[5 + 2 * q]; }
    } else {
        np = make_pairs(xt, N, Rc, mode, &P, &border, &E, &n_excl, eps_x);
        if (np < 0) return -1;
    }
    unsigned char* tpass = NULL;
    if (tmode != TAPE_OFF) {
        long need = pbd_tape_bytes(np, N, nct, total);
        if (tape_len) *tape_len = need;
        if (tape_cap < need) { free(P); free(E); free(border); return -3; }
        if (tmode == TAPE_RECORD) {
            th[0] = np; th[1] = N; th[2] = nct; th[3] = total;
            for (long q = 0; q < np; ++q) { th[4 + 2 * q] = P[q].i; th[5 + 2 * q] = P[q].j; }
            memset(tape + 32 + 16 * np, 0, (size_t)(need - 32 - 16 * np));
        }
        tpass = tape + 32 + 16 * np;
    }
    long maxc = 0;
    if (stats) {
        long* c = (long*)calloc(n1, sizeof(long));
        for (long p = 0; p < np; ++p) { c[P[p].i]++; c[P[p].j]++; }
        for (long i = 0; i < N; ++i)
            if (c[i] > maxc) maxc = c[i];
        free(c);
    }

    pbd_work w;
    if (pbd_work_init(&w, N, x, xt, ws, inv_m, sdf, n_sdf, prm, mu, bodies, tmode) != 0) return -1;
    w.P = P;
    w.border = border;
    w.np = np;
    w.E = E;
    w.n_excl = n_excl;
    int rc = 0;
    for (int it = 0; it < total && rc == 0; ++it) {
        /* a particle that read a suspect candidate partner in an earlier
         * pass is itself suspect from now on */
        if (it > 0) {
            memcpy(mark2, w.mark, (size_t)N);
            for (long p = 0; p < np; ++p) {
                if (mark2[P[p].i]) w.mark[P[p].j] = 1;
                if (mark2[P[p].j]) w.mark[P[p].i] = 1;
            }
        }
        unsigned char* tpair = tpass ? tpass + (long)it * (np + N * (long)nct) : NULL;
        rc = pbd_pass(&w, it < n_stab, tpair);
    }
    if (rc == 0) {
        /* last loop of Algorithm 1: v = (xt - x) / dt, x = xt */
        for (long i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] = (xt[3 * i + k] - x[3 * i + k]) / dt;
                x[3 * i + k] = xt[3 * i + k];
            }
        if (suspect)
            for (long i = 0; i < N; ++i) suspect[i] = w.mark[i];
        if (stats) {
            stats[0] = np;
            stats[1] = w.n_sig;
            stats[2] = maxc;
            stats[3] = w.active_last;
            stats[4] = w.n_amb;
        }
    }
    pbd_work_free(&w);
    free(P);
    free(E);
    free(border);
    free(xt);
    free(ws);
    free(mark2);
    return rc;
}

/* One Jacobi pass of the LR step from a given state, the oracle a pass-by-
 * pass comparison needs (Algorithm 1, Sec. 3):
 *   x0        [N][3] positions at the start of the step (they fix the
 *             height-scaled masses, as in the step's first loop);
 *   xt0       [N][3] predicted positions (the candidate pairs of the step
 *             are generated from them, |xt0_i - xt0_j| < Rc);
 *   x, xt     [N][3] the pass's input, updated in place: x as stabilized so
 *             far, xt as corrected so far;
 *   stab      1 for a stabilization pass (contacts only, evaluated on x and
 *             applied to x and xt), 0 for a solver pass (Eqs. 1-4 on xt).
 * suspect (optional, N) marks the particles whose result in this pass hangs
 * on a decision within the margins prm[PB_EPS_X] / prm[PB_EPS_IMPACT]
 * (candidate membership, contact, static / kinetic friction, SDF contact);
 * marks are not carried over from earlier passes.  mode as or_pbd_step;
 * stats as or_pbd_step ([3]: active pair contacts of this pass). */
int or_pbd_pass(double* x, double* xt, const double* x0, const double* xt0, const double* inv_m, long N,
                const double* sdf, int n_sdf, const double* prm, int stab, int mode, int* suspect, long* stats)
{
    size_t n1 = (size_t)(N ? N : 1);
    double* ws = (double*)malloc(n1 * sizeof(double));
    double* vt = (double*)calloc(n1 * 3, sizeof(double));
    double* xp = (double*)malloc(n1 * 3 * sizeof(double));
    if (!ws || !vt || !xp) return -1;
    pbd_predict(x0, vt, inv_m, N, prm, xp, ws);   /* only the masses are used */
    or_pair *P = NULL, *E = NULL;
    unsigned char* border = NULL;
    long n_excl = 0;
    long np = make_pairs(xt0, N, prm[PB_RC], mode, &P, &border, &E, &n_excl, prm[PB_EPS_X]);
    if (np < 0) return -1;
    pbd_work w;
    int rc = pbd_work_init(&w, N, x, xt, ws, inv_m, sdf, n_sdf, prm, NULL, NULL, TAPE_OFF);
    if (rc == 0) {
        w.P = P;
        w.border = border;
        w.np = np;
        w.E = E;
        w.n_excl = n_excl;
        rc = pbd_pass(&w, stab, NULL);
    }
    if (rc == 0) {
        if (suspect)
            for (long i = 0; i < N; ++i) suspect[i] = w.mark[i];
        if (stats) {
            stats[0] = np;
            stats[1] = w.n_sig;
            stats[2] = 0;
            stats[3] = w.active_last;
            stats[4] = w.n_amb;
        }
    }
    pbd_work_free(&w);
    free(P);
    free(E);
    free(border);
    free(ws);
    free(vt);
    free(xp);
    return rc;
}

int or_pbd_step(double* x, double* v, const double* inv_m, long N,
                const double* sdf, int n_sdf, const double* prm, int mode,
                int* suspect, long* stats)
{
    return pbd_impl(x, v, inv_m, N, sdf, n_sdf, prm, NULL, mode, suspect, stats, TAPE_OFF, NULL, 0, NULL, NULL);
}

/* or_pbd_step with per-particle friction coefficients mu (N x 2: mu_s,
 * mu_k); pairs and boundary contacts use the cross coefficients of Sec. 3. */
int or_pbd_step_mu(double* x, double* v, const double* inv_m, long N,
                   const double* sdf, int n_sdf, const double* prm, int mode, const double* mu,
                   int* suspect, long* stats)
{
    if (!mu && N > 0) return -1;
    return pbd_impl(x, v, inv_m, N, sdf, n_sdf, prm, mu, mode, suspect, stats, TAPE_OFF, NULL, 0, NULL, NULL);
}

/* or_pbd_step with optional per-particle friction coefficients (mu, may be
 * NULL) and rigid bodies matched to their rest shapes (body, xo; n_bodies
 * bodies numbered from 1; see pbd_impl).  -4 for a body whose shape is
 * degenerate. */
int or_pbd_step_bodies(double* x, double* v, const double* inv_m, long N,
                       const double* sdf, int n_sdf, const double* prm, int mode, const double* mu,
                       const int* body, const double* xo, int n_bodies, int* suspect, long* stats)
{
    if (n_bodies > 0 && (!body || !xo)) return -1;
    for (long i = 0; i < N && n_bodies > 0; ++i)
        if (body[i] > 0 && !(inv_m[i] > 0)) return -1;   /* body particles have finite mass */
    or_bodies bd = {body, xo, n_bodies};
    return pbd_impl(x, v, inv_m, N, sdf, n_sdf, prm, mu, mode, suspect, stats, TAPE_OFF, NULL, 0, NULL, &bd);
}

/* One LR step (grid neighbour search) that records its decisions into, or
 * replays them from, a byte tape of tape_cap bytes.  *tape_len receives the
 * size the tape needs; -3 when tape_cap is too small (x and v are then
 * partly updated and must be restored by the caller) or a replayed tape does
 * not match N, the SDF list or the pass count. */
int or_pbd_step_tape(double* x, double* v, const double* inv_m, long N, const double* sdf, int n_sdf,
                     const double* prm, int tmode, unsigned char* tape, long tape_cap, long* tape_len)
{
    if ((tmode != TAPE_RECORD && tmode != TAPE_REPLAY) || !tape) return -1;
    return pbd_impl(x, v, inv_m, N, sdf, n_sdf, prm, NULL, 1, NULL, NULL, tmode, tape, tape_cap, tape_len, NULL);
}

/* Brute-force pair listing for tests of the neighbour search: every (i, j)
 * with |a_i - b_j|^2 < R^2, i ascending then j ascending.  Returns the
 * number found (at most cap are written). */
long or_pairs_within(const double* a, long na, const double* b, long nb, double R, long* out_i, long* out_j, long cap)
{
    long n = 0;
    double R2 = R * R;
    for (long i = 0; i < na; ++i)
        for (long j = 0; j < nb; ++j) {
            double d[3] = {a[3 * i] - b[3 * j], a[3 * i + 1] - b[3 * j + 1], a[3 * i + 2] - b[3 * j + 2]};
            if (dot3(d, d) < R2) {
                if (n < cap) { out_i[n] = i; out_j[n] = j; }
                ++n;
            }
        }
    return n;
}

/* Grid version of or_pairs_within (same order, same set). */
long or_pairs_within_grid(const double* a, long na, const double* b, long nb, double R, long* out_i, long* out_j,
                          long cap)
{
    or_grid_t g;
    if (grid_build(&g, b, nb, R) != 0) return -1;
    long* cand = (long*)malloc((size_t)(nb ? nb : 1) * sizeof(long));
    long n = 0;
    for (long i = 0; i < na; ++i) {
        long nc = grid_query(&g, a + 3 * i, cand);
        for (long q = 0; q < nc; ++q) {
            if (n < cap) { out_i[n] = i; out_j[n] = cand[q]; }
            ++n;
        }
    }
    free(cand);
    grid_free(&g);
    return n;
}

/* ------------------------------------------------------------------ */
/* Reverse mode of the HR frame (for the differentiable pattern).       */
/* ------------------------------------------------------------------ */

/* Vector-Jacobian product of or_upsample's map
 *   (X_j, V_j [LR], x_i, v_i [HR]) -> (x_i^{t+1}, v_i^{t+1})
 * for the branch decisions of the forward pass (blend case, which LR
 * particle has the largest weight, SDF contacts).  Each active SDF
 * contact component is differentiated with its normal held fixed (exact for
 * planar walls): the projection x + (r_HR - phi) n has Jacobian I - n n^T,
 * and the removal of an inward normal velocity has Jacobian I - n n^T.
 * gx, gv: dL/dx^{t+1}, dL/dv^{t+1} (HR, n x 3).  Outputs (accumulated, the
 * caller zeroes them): gX, gV (LR, N x 3), ghx, ghv (HR, M x 3). */
/* tape (optional, uint32[M][4] of or_upsample_tape): the LR particle of
 * largest weight, the blend case and the SDF decisions of every HR particle
 * are taken from it, which gives the derivative of the replayed frame. */
static int upsample_vjp_impl(const double* lr_x, const double* lr_v, long N, const double* hr_x, const double* hr_v,
                             long M, const double* sdf, int n_sdf, const double* prm, const uint32_t* tape,
                             const double* gx_out, const double* gv_out, double* gX, double* gV, double* ghx,
                             double* ghv)
{
    double r = prm[UP_R_LOW], c1 = prm[UP_C1], c2 = prm[UP_C2], dt = prm[UP_DT], rh = prm[UP_R_HIGH];
    double eps_x = prm[UP_EPS_X];
    const double g[3] = {prm[UP_GX], prm[UP_GY], prm[UP_GZ]};
    double R2 = 9.0 * r * r;
    for (long i = 0; i < M; ++i) {
        const double* xi = hr_x + 3 * i;
        const double* vi = hr_v + 3 * i;
        /* forward, as in or_upsample */
        double S = 0, V[3] = {0, 0, 0}, wmax = 0;
        long jstar = -1;
        for (long j = 0; j < N; ++j) {
            double d[3] = {xi[0] - lr_x[3 * j], xi[1] - lr_x[3 * j + 1], xi[2] - lr_x[3 * j + 2]};
            double d2 = dot3(d, d);
            if (!(d2 < R2)) continue;
            double w = or_weight(d2, r);
            S += w;
            for (int m = 0; m < 3; ++m) V[m] += w * lr_v[3 * j + m];
            if (w > wmax) { wmax = w; jstar = j; }
        }
        const uint32_t* tp = tape ? tape + 4 * i : NULL;
        if (tp) {
            jstar = (long)(int32_t)tp[0];
            wmax = 0.0;
            if (jstar >= 0 && jstar < N) {
                double d[3] = {xi[0] - lr_x[3 * jstar], xi[1] - lr_x[3 * jstar + 1], xi[2] - lr_x[3 * jstar + 2]};
                wmax = or_weight(dot3(d, d), r);
            } else {
                jstar = -1;
            }
        }
        double vt[3] = {0, 0, 0};
        if (S > 0)
            for (int m = 0; m < 3; ++m) vt[m] = V[m] / S;
        int branch = tp ? (int)tp[1] : (wmax <= c1) || (S > 0 && wmax >= c2 * S);
        double alpha = branch ? 1.0 - wmax : 0.0;
        double vp[3], xp[3];
        for (int m = 0; m < 3; ++m) {
            vp[m] = (1.0 - alpha) * vt[m] + alpha * (vi[m] + dt * g[m]);
            xp[m] = xi[m] + dt * vp[m];
        }
        /* SDF rule forward, recording the normals of the active steps */
        double nrm[64][3];
        int kind_v[64], n_steps = 0, dec = 0;
        for (int s = 0; s < n_sdf; ++s) {
            const double* rec = sdf + OR_SDF_STRIDE * s;
            const double* ub = rec + 13;
            int nc = sdf_ncomp(rec);
            for (int c = 0; c < nc; ++c, ++dec) {
                double phi[OR_MAX_COMP], nn[3 * OR_MAX_COMP];
                int tie;
                or_sdf_eval(rec, xp, phi, nn, &tie, eps_x);
                const int active = tp ? (tp[2] >> dec) & 1u : phi[c] < rh;
                if (!active) continue;
                const double* n = nn + 3 * c;
                double push = rh - phi[c];
                for (int m = 0; m < 3; ++m) xp[m] += push * n[m];
                double vr[3] = {vp[0] - ub[0], vp[1] - ub[1], vp[2] - ub[2]};
                double vn = dot3(vr, n);
                const int rem = tp ? (tp[3] >> dec) & 1u : vn < 0;
                if (rem)
                    for (int m = 0; m < 3; ++m) vp[m] -= vn * n[m];
                if (n_steps < 64) {
                    for (int m = 0; m < 3; ++m) nrm[n_steps][m] = n[m];
                    kind_v[n_steps] = rem;
                    ++n_steps;
                }
            }
        }
        /* reverse: SDF steps, last first */
        double ax[3], av[3];
        for (int m = 0; m < 3; ++m) { ax[m] = gx_out[3 * i + m]; av[m] = gv_out[3 * i + m]; }
        for (int k = n_steps - 1; k >= 0; --k) {
            const double* n = nrm[k];
            if (kind_v[k]) {
                double a = dot3(av, n);
                for (int m = 0; m < 3; ++m) av[m] -= a * n[m];
            }
            double a = dot3(ax, n);
            for (int m = 0; m < 3; ++m) ax[m] -= a * n[m];
        }
        /* x' = x + dt v' */
        double gvp[3], gvt[3], galpha = 0;
        for (int m = 0; m < 3; ++m) {
            ghx[3 * i + m] += ax[m];
            gvp[m] = av[m] + dt * ax[m];
        }
        /* v' = (1 - alpha) vtilde + alpha (v + dt g) */
        for (int m = 0; m < 3; ++m) {
            gvt[m] = (1.0 - alpha) * gvp[m];
            ghv[3 * i + m] += alpha * gvp[m];
            galpha += gvp[m] * (vi[m] + dt * g[m] - vt[m]);
        }
        double gwmax = branch ? -galpha : 0.0;
        if (!(S > 0)) continue;           /* no LR particle in reach: nothing else depends on LR */
        /* vtilde = V / S */
        double gV_[3] = {gvt[0] / S, gvt[1] / S, gvt[2] / S};
        double gS = -dot3(gvt, vt) / S;
        for (long j = 0; j < N; ++j) {
            double d[3] = {xi[0] - lr_x[3 * j], xi[1] - lr_x[3 * j + 1], xi[2] - lr_x[3 * j + 2]};
            double d2 = dot3(d, d);
            if (!(d2 < R2)) continue;
            double t = 1.0 - d2 / R2;
            double w = t * t * t;
            double gw = gS + dot3(gV_, lr_v + 3 * j) + (j == jstar ? gwmax : 0.0);
            /* dw/dx_i = -6 t^2 d / (9 r^2) = -dw/dX_j */
            double k6 = 6.0 * t * t / R2;
            for (int m = 0; m < 3; ++m) {
                gX[3 * j + m] += gw * k6 * d[m];
                ghx[3 * i + m] -= gw * k6 * d[m];
                gV[3 * j + m] += w * gV_[m];
            }
        }
    }
    return 0;
}

int or_upsample_vjp(const double* lr_x, const double* lr_v, long N, const double* hr_x, const double* hr_v, long M,
                    const double* sdf, int n_sdf, const double* prm, const double* gx_out, const double* gv_out,
                    double* gX, double* gV, double* ghx, double* ghv)
{
    return upsample_vjp_impl(lr_x, lr_v, N, hr_x, hr_v, M, sdf, n_sdf, prm, NULL, gx_out, gv_out, gX, gV, ghx, ghv);
}

/* Reverse mode of the HR frame replayed from a tape (uint32[M][4] of
 * or_upsample_tape's layout). */
int or_upsample_vjp_tape(const double* lr_x, const double* lr_v, long N, const double* hr_x, const double* hr_v,
                         long M, const double* sdf, int n_sdf, const double* prm, const uint32_t* tape,
                         const double* gx_out, const double* gv_out, double* gX, double* gV, double* ghx, double* ghv)
{
    if (!tape || total_components(sdf, n_sdf) > 32) return -1;
    return upsample_vjp_impl(lr_x, lr_v, N, hr_x, hr_v, M, sdf, n_sdf, prm, tape, gx_out, gv_out, gX, gV, ghx, ghv);
}

/* Reverse mode of one LR step (Algorithm 1) for the branch decisions of the
 * forward pass: which candidate pairs and SDF components are in contact in
 * each pass, static or kinetic friction, and whether the kinetic scale is
 * clipped.  SDF normals are held fixed (exact for planar walls).
 *
 * Pair (i, j) evaluated on positions y (x in stabilization, xt in the solver),
 * e = y_j - y_i, L = |e|, u = e / L, pen = 2r - L, W = w_i + w_j (inverse
 * scaled masses), m_i = w_i / W, m_j = w_j / W:
 *   contact     c_i = -m_i pen u,  c_j = +m_j pen u,
 *               d(pen u)/de = (2r/L - 1) I - (2r/L) u u^T =: K
 *   friction    rel = (xt_i - x_i) - (xt_j - x_j),  perp = P rel,
 *               P = I - e e^T / (e.e),  F = s perp  (s = 1, or
 *               thr_k / |perp| when clipped),  c_i -= m_i F,  c_j += m_j F
 *               dF/d rel = Q P,  dF/de = Q dperp/de,  Q = I or
 *               (thr_k / |perp|)(I - p p^T) (+ threshold terms in mode 1)
 *   SDF         c = (r - phi) n - F(d),  d = (xt - x) - u_b dt
 * A pass moves particle i by (sum_k c_ik) / n_i; the adjoint pushes
 * h_i = g_i / n_i back through every contribution. */

typedef struct { double v[9]; } m33;

static void m33_outer_add(m33* A, double s, const double* a, const double* b)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) A->v[3 * r + c] += s * a[r] * b[c];
}

static void m33_eye(m33* A, double s)
{
    memset(A, 0, sizeof *A);
    A->v[0] = A->v[4] = A->v[8] = s;
}

/* out += s * A^T h */
static void m33_tmul_add(double* out, double s, const m33* A, const double* h)
{
    for (int c = 0; c < 3; ++c)
        out[c] += s * (A->v[c] * h[0] + A->v[3 + c] * h[1] + A->v[6 + c] * h[2]);
}

static void m33_mul(m33* C, const m33* A, const m33* B)
{
    m33 R;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R.v[3 * r + c] = A->v[3 * r] * B->v[c] + A->v[3 * r + 1] * B->v[3 + c] + A->v[3 * r + 2] * B->v[6 + c];
    *C = R;
}

/* Friction F(rel) with tangent plane normal to e (pair) or n (SDF): value
 * and Jacobians dF/drel and dF/de (zero for SDF, where e_is_normal). */
static void friction_jac(const double* rel, const double* e, int e_is_normal, double thr_s, double thr_k,
                         int mode1, double mu_k, const double* u_for_thr, double* F, m33* Frel, m33* Fe, int force)
{
    double ee = dot3(e, e);
    double a = dot3(rel, e) / ee;
    double perp[3] = {rel[0] - a * e[0], rel[1] - a * e[1], rel[2] - a * e[2]};
    m33 P, G;
    m33_eye(&P, 1.0);
    m33_outer_add(&P, -1.0 / ee, e, e);
    memset(&G, 0, sizeof G);
    if (!e_is_normal) {
        /* dperp_a/de_b = -(e_a rel_b + (rel.e) delta_ab)/(e.e) + 2 (rel.e) e_a e_b/(e.e)^2 */
        double re = dot3(rel, e);
        m33_outer_add(&G, -1.0 / ee, e, rel);
        for (int k = 0; k < 3; ++k) G.v[4 * k] -= re / ee;
        m33_outer_add(&G, 2.0 * re / (ee * ee), e, e);
    }
    double Lp = sqrt(dot3(perp, perp));
    int clipped = !(Lp < thr_s) && Lp > 0 && thr_k / Lp < 1.0;
    if (force >= 0) clipped = force && Lp > 0;   /* a decision replayed from a tape */
    m33 Q;
    if (clipped) {
        double p[3] = {perp[0] / Lp, perp[1] / Lp, perp[2] / Lp};
        m33_eye(&Q, thr_k / Lp);
        m33_outer_add(&Q, -thr_k / Lp, p, p);
        for (int k = 0; k < 3; ++k) F[k] = thr_k * p[k];
        m33_mul(Frel, &Q, &P);
        m33_mul(Fe, &Q, &G);
        if (mode1) {   /* thr_k = pen mu_k, dpen/de = -u^T */
            m33_outer_add(Fe, -mu_k, p, u_for_thr);
        }
    } else {
        for (int k = 0; k < 3; ++k) F[k] = perp[k];
        *Frel = P;
        *Fe = G;
    }
}

/* tape (optional, the layout of or_pbd_step_tape): the candidate pairs and
 * every pass's decisions are taken from it instead of from the comparisons,
 * which gives the derivative of the replayed step (the smooth piece the tape
 * was recorded on). */
static int pbd_vjp_impl(const double* x0, const double* v0, const double* inv_m, long N, const double* sdf, int n_sdf,
                        const double* prm, const unsigned char* tape, long tape_len, const double* gx_out,
                        const double* gv_out, double* gx0, double* gv0)
{
    double r = prm[PB_R], dt = prm[PB_DT];
    const double g[3] = {prm[PB_GX], prm[PB_GY], prm[PB_GZ]};
    double mu_s = prm[PB_MU_S], mu_k = prm[PB_MU_K];
    int n_stab = (int)prm[PB_N_STAB], iters = (int)prm[PB_ITERS];
    double mass_k = prm[PB_MASS_K], ground = prm[PB_GROUND_Z], Rc = prm[PB_RC];
    int fmode = (int)prm[PB_FRIC_MODE];
    double d0 = 2.0 * r;
    int total = n_stab + iters;
    size_t n1 = (size_t)(N ? N : 1);
    /* forward with snapshots: Y[p] = positions the pass p evaluates on */
    double* x = (double*)malloc(n1 * 3 * sizeof(double));
    double* xt = (double*)malloc(n1 * 3 * sizeof(double));
    double* ws = (double*)malloc(n1 * sizeof(double));
    double* Y = (double*)malloc((size_t)(total + 1) * n1 * 3 * sizeof(double));
    double* XT = (double*)malloc((size_t)(total + 1) * n1 * 3 * sizeof(double));
    double* D = (double*)malloc(n1 * 3 * sizeof(double));
    long* cnt = (long*)malloc(n1 * sizeof(long));
    long* CNT = (long*)malloc((size_t)(total + 1) * n1 * sizeof(long));
    if (!x || !xt || !ws || !Y || !XT || !D || !cnt || !CNT) return -1;
    for (long i = 0; i < N; ++i) {
        for (int k = 0; k < 3; ++k) {
            x[3 * i + k] = x0[3 * i + k];
            xt[3 * i + k] = x0[3 * i + k] + dt * (v0[3 * i + k] + dt * g[k]);
        }
        ws[i] = inv_m[i] * exp(mass_k * (x0[3 * i + 2] - ground));
    }
    or_pair *Pp = NULL, *E = NULL;
    unsigned char* border = NULL;
    long n_excl = 0;
    long np;
    const int nct = total_components(sdf, n_sdf);
    if (tape) {
        const int64_t* th = (const int64_t*)tape;
        if (tape_len < 32 || th[1] != N || th[2] != nct || th[3] != total) return -3;
        np = (long)th[0];
        if (tape_len < pbd_tape_bytes(np, N, nct, total)) return -3;
        Pp = (or_pair*)malloc((size_t)(np ? np : 1) * sizeof(or_pair));
        border = (unsigned char*)calloc((size_t)(np ? np : 1), 1);
        E = (or_pair*)malloc(sizeof(or_pair));
        if (!Pp || !border || !E) return -1;
        for (long q = 0; q < np; ++q) { Pp[q].i = (long)th[4 + 2 * q]; Pp[q].j = (long)th[5 + 2 * q]; }
    } else {
        np = make_pairs(xt, N, Rc, 0, &Pp, &border, &E, &n_excl, 0.0);
        if (np < 0) return -1;
    }
    /* the decision bytes of pass it: one per pair, then one per (particle,
     * SDF component); bit 0 = active, bit 1 = kinetic friction scale */
    const unsigned char* tpass = tape ? tape + 32 + 16 * np : NULL;
#define PASS_TAPE(it) (tpass ? tpass + (long)(it) * (np + N * (long)nct) : NULL)
    double* Xfix = NULL;
    for (int it = 0; it < total; ++it) {
        int stab = it < n_stab;
        const double* y = stab ? x : xt;
        memcpy(Y + (size_t)it * n1 * 3, y, (size_t)N * 3 * sizeof(double));
        memcpy(XT + (size_t)it * n1 * 3, xt, (size_t)N * 3 * sizeof(double));
        memset(D, 0, (size_t)N * 3 * sizeof(double));
        memset(cnt, 0, (size_t)N * sizeof(long));
        const unsigned char* tp = PASS_TAPE(it);
        for (long p = 0; p < np; ++p) {
            long i = Pp[p].i, j = Pp[p].j;
            double e[3] = {y[3 * j] - y[3 * i], y[3 * j + 1] - y[3 * i + 1], y[3 * j + 2] - y[3 * i + 2]};
            double L = sqrt(dot3(e, e));
            const int active = tp ? (tp[p] & 1) : L < d0;
            const int FORCE_PAIR = tp ? (tp[p] >> 1) & 1 : -1;
            if (!active || L == 0.0 || !(ws[i] + ws[j] > 0)) continue;
            double W = ws[i] + ws[j], mi = ws[i] / W, mj = ws[j] / W, pen = d0 - L;
            double u[3] = {e[0] / L, e[1] / L, e[2] / L};
            for (int k = 0; k < 3; ++k) {
                D[3 * i + k] -= mi * pen * u[k];
                D[3 * j + k] += mj * pen * u[k];
            }
            if (!stab) {
                double rel[3], F[3];
                m33 Fr, Fe;
                for (int k = 0; k < 3; ++k) rel[k] = (xt[3 * i + k] - x[3 * i + k]) - (xt[3 * j + k] - x[3 * j + k]);
                double base = fmode == 1 ? pen : d0;
                friction_jac(rel, e, 0, base * mu_s, base * mu_k, fmode == 1, mu_k, u, F, &Fr, &Fe, FORCE_PAIR);
                for (int k = 0; k < 3; ++k) {
                    D[3 * i + k] -= mi * F[k];
                    D[3 * j + k] += mj * F[k];
                }
            }
            cnt[i]++;
            cnt[j]++;
        }
        for (long i = 0; i < N; ++i) {
            if (!(ws[i] > 0)) continue;
            int comp0 = 0;
            for (int s = 0; s < n_sdf; comp0 += sdf_ncomp(sdf + OR_SDF_STRIDE * s), ++s) {
                const double* rec = sdf + OR_SDF_STRIDE * s;
                double phi[OR_MAX_COMP], nn[3 * OR_MAX_COMP];
                int tie;
                int nc = or_sdf_eval(rec, y + 3 * i, phi, nn, &tie, 0.0);
                double bmu_s = sqrt(mu_s * rec[16]), bmu_k = sqrt(mu_k * rec[17]);
                for (int c = 0; c < nc; ++c) {
                    const unsigned char* tb = tp ? tp + np + i * (long)nct + comp0 + c : NULL;
                    const int active = tb ? (*tb & 1) : phi[c] < r;
                    const int FORCE_SDF = tb ? (*tb >> 1) & 1 : -1;
                    if (!active) continue;
                    const double* n = nn + 3 * c;
                    double pen = r - phi[c];
                    for (int k = 0; k < 3; ++k) D[3 * i + k] += pen * n[k];
                    if (!stab) {
                        double d[3], F[3];
                        m33 Fr, Fe;
                        for (int k = 0; k < 3; ++k) d[k] = (xt[3 * i + k] - x[3 * i + k]) - rec[13 + k] * dt;
                        double base = fmode == 1 ? pen : d0;
                        friction_jac(d, n, 1, base * bmu_s, base * bmu_k, fmode == 1, bmu_k, n, F, &Fr, &Fe, FORCE_SDF);
                        for (int k = 0; k < 3; ++k) D[3 * i + k] -= F[k];
                    }
                    cnt[i]++;
                }
            }
        }
        memcpy(CNT + (size_t)it * n1, cnt, (size_t)N * sizeof(long));
        for (long i = 0; i < N; ++i) {
            if (cnt[i] == 0) continue;
            for (int k = 0; k < 3; ++k) {
                double dd = D[3 * i + k] / (double)cnt[i];
                xt[3 * i + k] += dd;
                if (stab) x[3 * i + k] += dd;
            }
        }
        if (it == n_stab - 1 || (n_stab == 0 && it == 0)) {
            if (!Xfix) Xfix = (double*)malloc(n1 * 3 * sizeof(double));
        }
    }
    if (!Xfix) Xfix = (double*)malloc(n1 * 3 * sizeof(double));
    memcpy(Xfix, x, (size_t)N * 3 * sizeof(double));   /* x after stabilization (fixed in the solver) */

    /* reverse: outputs x_out = xt, v_out = (xt - x) / dt */
    double* gxt = (double*)calloc(n1 * 3, sizeof(double));
    double* gx = (double*)calloc(n1 * 3, sizeof(double));
    double* gws = (double*)calloc(n1, sizeof(double));
    double* H = (double*)malloc(n1 * 3 * sizeof(double));
    double* acc = (double*)malloc(n1 * 3 * sizeof(double));
    for (long i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) {
            gxt[3 * i + k] = gx_out[3 * i + k] + gv_out[3 * i + k] / dt;
            gx[3 * i + k] = -gv_out[3 * i + k] / dt;
        }
    for (int it = total - 1; it >= 0; --it) {
        int stab = it < n_stab;
        const double* y = Y + (size_t)it * n1 * 3;
        const double* xtp = XT + (size_t)it * n1 * 3;
        const long* cn = CNT + (size_t)it * n1;
        /* upstream of the averaged delta */
        for (long i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) {
                double up = stab ? gx[3 * i + k] + gxt[3 * i + k] : gxt[3 * i + k];
                H[3 * i + k] = cn[i] > 0 ? up / (double)cn[i] : 0.0;
            }
        /* gradient w.r.t. the positions the pass evaluates on (y) and, in
         * the solver, w.r.t. x through the friction */
        memset(acc, 0, (size_t)N * 3 * sizeof(double));
        double* accx = stab ? NULL : (double*)calloc(n1 * 3, sizeof(double));
        const unsigned char* tp = PASS_TAPE(it);
        for (long p = 0; p < np; ++p) {
            long i = Pp[p].i, j = Pp[p].j;
            double e[3] = {y[3 * j] - y[3 * i], y[3 * j + 1] - y[3 * i + 1], y[3 * j + 2] - y[3 * i + 2]};
            double L = sqrt(dot3(e, e));
            const int active = tp ? (tp[p] & 1) : L < d0;
            const int FORCE_PAIR = tp ? (tp[p] >> 1) & 1 : -1;
            if (!active || L == 0.0 || !(ws[i] + ws[j] > 0)) continue;
            double W = ws[i] + ws[j], mi = ws[i] / W, mj = ws[j] / W, pen = d0 - L;
            double u[3] = {e[0] / L, e[1] / L, e[2] / L};
            const double* hi = H + 3 * i;
            const double* hj = H + 3 * j;
            m33 K;
            m33_eye(&K, d0 / L - 1.0);
            m33_outer_add(&K, -d0 / L, u, u);
            /* c_i = -m_i pen u(e), c_j = m_j pen u(e), e = y_j - y_i */
            double tvec[3] = {0, 0, 0};
            m33_tmul_add(tvec, -mi, &K, hi);   /* (dc_i/de)^T h_i */
            m33_tmul_add(tvec, mj, &K, hj);    /* (dc_j/de)^T h_j */
            for (int k = 0; k < 3; ++k) {
                acc[3 * j + k] += tvec[k];
                acc[3 * i + k] -= tvec[k];
            }
            /* mass ratios: dc_i/dm_i = -pen u, dc_j/dm_j = pen u */
            double pu_hi = pen * dot3(u, hi), pu_hj = pen * dot3(u, hj);
            double dmi_dwi = ws[j] / (W * W), dmi_dwj = -ws[i] / (W * W);
            gws[i] += -pu_hi * dmi_dwi + pu_hj * (-dmi_dwi);
            gws[j] += -pu_hi * dmi_dwj + pu_hj * (-dmi_dwj);
            if (!stab) {
                double rel[3], F[3];
                m33 Fr, Fe;
                for (int k = 0; k < 3; ++k)
                    rel[k] = (xtp[3 * i + k] - Xfix[3 * i + k]) - (xtp[3 * j + k] - Xfix[3 * j + k]);
                double base = fmode == 1 ? pen : d0;
                friction_jac(rel, e, 0, base * mu_s, base * mu_k, fmode == 1, mu_k, u, F, &Fr, &Fe, FORCE_PAIR);
                /* c_i -= m_i F, c_j += m_j F; rel = (xt_i - x_i) - (xt_j - x_j) */
                double hF[3] = {-mi * hi[0] + mj * hj[0], -mi * hi[1] + mj * hj[1], -mi * hi[2] + mj * hj[2]};
                double grel[3] = {0, 0, 0}, ge[3] = {0, 0, 0};
                m33_tmul_add(grel, 1.0, &Fr, hF);
                m33_tmul_add(ge, 1.0, &Fe, hF);
                for (int k = 0; k < 3; ++k) {
                    acc[3 * i + k] += grel[k] - ge[k];
                    acc[3 * j + k] += -grel[k] + ge[k];
                    accx[3 * i + k] -= grel[k];
                    accx[3 * j + k] += grel[k];
                }
                double Fh_i = dot3(F, hi), Fh_j = dot3(F, hj);
                gws[i] += -Fh_i * dmi_dwi + Fh_j * (-dmi_dwi);
                gws[j] += -Fh_i * dmi_dwj + Fh_j * (-dmi_dwj);
            }
        }
        for (long i = 0; i < N; ++i) {
            if (!(ws[i] > 0)) continue;
            const double* hi = H + 3 * i;
            int comp0 = 0;
            for (int s = 0; s < n_sdf; comp0 += sdf_ncomp(sdf + OR_SDF_STRIDE * s), ++s) {
                const double* rec = sdf + OR_SDF_STRIDE * s;
                double phi[OR_MAX_COMP], nn[3 * OR_MAX_COMP];
                int tie;
                int nc = or_sdf_eval(rec, y + 3 * i, phi, nn, &tie, 0.0);
                double bmu_s = sqrt(mu_s * rec[16]), bmu_k = sqrt(mu_k * rec[17]);
                for (int c = 0; c < nc; ++c) {
                    const unsigned char* tb = tp ? tp + np + i * (long)nct + comp0 + c : NULL;
                    const int active = tb ? (*tb & 1) : phi[c] < r;
                    const int FORCE_SDF = tb ? (*tb >> 1) & 1 : -1;
                    if (!active) continue;
                    const double* n = nn + 3 * c;
                    double a = dot3(n, hi);       /* d((r - phi) n)/dy = -n n^T */
                    for (int k = 0; k < 3; ++k) acc[3 * i + k] -= a * n[k];
                    if (!stab) {
                        double d[3], F[3];
                        m33 Fr, Fe;
                        double pen = r - phi[c];
                        for (int k = 0; k < 3; ++k) d[k] = (xtp[3 * i + k] - Xfix[3 * i + k]) - rec[13 + k] * dt;
                        double base = fmode == 1 ? pen : d0;
                        friction_jac(d, n, 1, base * bmu_s, base * bmu_k, fmode == 1, bmu_k, n, F, &Fr, &Fe, FORCE_SDF);
                        double gd[3] = {0, 0, 0};
                        m33_tmul_add(gd, -1.0, &Fr, hi);   /* c -= F(d) */
                        for (int k = 0; k < 3; ++k) {
                            acc[3 * i + k] += gd[k];
                            accx[3 * i + k] -= gd[k];
                        }
                        if (fmode == 1) {          /* clipped F depends on y through pen */
                            double Lp = sqrt(dot3(F, F));
                            (void)Lp;
                            m33 Fy;
                            memset(&Fy, 0, sizeof Fy);
                            double dd[3], perp[3];
                            for (int k = 0; k < 3; ++k) dd[k] = d[k];
                            double an = dot3(dd, n);
                            for (int k = 0; k < 3; ++k) perp[k] = dd[k] - an * n[k];
                            double Lq = sqrt(dot3(perp, perp));
                            const int clip = FORCE_SDF >= 0 ? FORCE_SDF && Lq > 0
                                                            : (!(Lq < base * bmu_s) && Lq > 0 && base * bmu_k / Lq < 1.0);
                            if (clip) {
                                /* F = pen mu_k perp/|perp|, dpen/dy = -n^T */
                                double q = dot3(perp, hi) / Lq;
                                for (int k = 0; k < 3; ++k) acc[3 * i + k] += q * bmu_k * n[k];
                            }
                        }
                    }
                }
            }
        }
        if (stab) {
            for (long i = 0; i < N * 3; ++i) gx[i] += acc[i];
        } else {
            for (long i = 0; i < N * 3; ++i) {
                gxt[i] += acc[i];
                gx[i] += accx[i];
            }
            free(accx);
        }
    }
    /* predict: xt = x + dt (v + dt g), w_i = inv_m e^{k (z - ground)} */
    for (long i = 0; i < N; ++i) {
        for (int k = 0; k < 3; ++k) {
            gx0[3 * i + k] += gx[3 * i + k] + gxt[3 * i + k];
            gv0[3 * i + k] += dt * gxt[3 * i + k];
        }
        gx0[3 * i + 2] += gws[i] * ws[i] * mass_k;
    }
    free(x); free(xt); free(ws); free(Y); free(XT); free(D); free(cnt); free(CNT); free(Pp); free(E); free(border);
    free(Xfix); free(gxt); free(gx); free(gws); free(H); free(acc);
#undef PASS_TAPE
    return 0;
}

int or_pbd_step_vjp(const double* x0, const double* v0, const double* inv_m, long N, const double* sdf, int n_sdf,
                    const double* prm, const double* gx_out, const double* gv_out, double* gx0, double* gv0)
{
    return pbd_vjp_impl(x0, v0, inv_m, N, sdf, n_sdf, prm, NULL, 0, gx_out, gv_out, gx0, gv0);
}

/* Reverse mode of the step replayed from a tape of or_pbd_step_tape's
 * layout (candidate pairs and every pass's decisions from the tape). */
int or_pbd_step_vjp_tape(const double* x0, const double* v0, const double* inv_m, long N, const double* sdf,
                         int n_sdf, const double* prm, const unsigned char* tape, long tape_len, const double* gx_out,
                         const double* gv_out, double* gx0, double* gv0)
{
    if (!tape) return -1;
    return pbd_vjp_impl(x0, v0, inv_m, N, sdf, n_sdf, prm, tape, tape_len, gx_out, gv_out, gx0, gv0);
}

/* ------------------------------------------------------------------ */
/* Plain definitions.                                                   */
/*                                                                      */
/* The LR step and the HR frame once more, as the paper states them and */
/* nothing else: no decision margins, tapes or branch bookkeeping, each */
/* particle's sums gathered by the particle itself (so the loops over   */
/* particles run in parallel without changing a bit).  They read like   */
/* Algorithm 1 and Sec. 4 and are checked bit for bit against the       */
/* instrumented functions above (same partners in the same ascending    */
/* order, same expressions), which carry the pins.  Scene coefficients */
/* only (no materials, bodies or solid particles).                      */
/* ------------------------------------------------------------------ */

/* One HR frame of Sec. 4 for every HR particle:
 *   w_ij = max(0, 1 - |x_i - x_j|^2 / (3 r_LR)^2)^3 over LR particles j,
 *   vtilde = sum w v_j / sum w (0 when the sum is 0),
 *   alpha = 1 - max w if max w <= c1 or max w >= c2 sum w, else 0,
 *   v = (1 - alpha) vtilde + alpha (v + dt g),  x = x + dt v,
 * then the SDF rule per component in order (phi < r_HR: move to
 * phi = r_HR along the normal, remove the normal velocity into the
 * boundary relative to its velocity).  LR partners in ascending index. */
int or_upsample_plain(const double* lr_x, const double* lr_v, long N, const double* hr_x, const double* hr_v,
                      long M, const double* sdf, int n_sdf, const double* prm, double* out_x, double* out_v)
{
    const double r = prm[UP_R_LOW], c1 = prm[UP_C1], c2 = prm[UP_C2], dt = prm[UP_DT], rh = prm[UP_R_HIGH];
    const double eps_x = prm[UP_EPS_X], R2 = 9.0 * r * r;
    const double g[3] = {prm[UP_GX], prm[UP_GY], prm[UP_GZ]};
    or_grid_t grid;
    if (grid_build(&grid, lr_x, N, 3.0 * r) != 0) return -1;
    int err = 0;
    const int nth = g_threads;
#pragma omp parallel num_threads(nth) if (nth > 1)
    {
        long* near = (long*)malloc((size_t)(N ? N : 1) * sizeof(long));
        if (!near) err = -1;
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < M; ++i) {
            if (!near) continue;
            const double *xi = hr_x + 3 * i, *vi = hr_v + 3 * i;
            double S = 0, V[3] = {0, 0, 0}, wmax = 0;
            const long nn = grid_query(&grid, xi, near);   /* within 3 r_LR, ascending */
            for (long q = 0; q < nn; ++q) {
                const long j = near[q];
                double d[3] = {xi[0] - lr_x[3 * j], xi[1] - lr_x[3 * j + 1], xi[2] - lr_x[3 * j + 2]};
                double d2 = dot3(d, d);
                if (!(d2 < R2)) continue;
                double w = or_weight(d2, r);
                S += w;
                for (int m = 0; m < 3; ++m) V[m] += w * lr_v[3 * j + m];
                if (w > wmax) wmax = w;
            }
            double vt[3] = {0, 0, 0};
            if (S > 0)
                for (int m = 0; m < 3; ++m) vt[m] = V[m] / S;
            const double alpha = (wmax <= c1 || (S > 0 && wmax >= c2 * S)) ? 1.0 - wmax : 0.0;
            double *xo = out_x + 3 * i, *vo = out_v + 3 * i;
            for (int m = 0; m < 3; ++m) {
                vo[m] = (1.0 - alpha) * vt[m] + alpha * (vi[m] + dt * g[m]);
                xo[m] = xi[m] + dt * vo[m];
            }
            for (int s = 0; s < n_sdf; ++s) {
                const double *rec = sdf + OR_SDF_STRIDE * s, *ub = rec + 13;
                for (int c = 0; c < sdf_ncomp(rec); ++c) {
                    double phi[OR_MAX_COMP], nrm[3 * OR_MAX_COMP];
                    int tie;
                    or_sdf_eval(rec, xo, phi, nrm, &tie, eps_x);   /* after the previous component moved it */
                    if (!(phi[c] < rh)) continue;
                    const double* n = nrm + 3 * c;
                    const double push = rh - phi[c];
                    for (int m = 0; m < 3; ++m) xo[m] += push * n[m];
                    double vr[3] = {vo[0] - ub[0], vo[1] - ub[1], vo[2] - ub[2]};
                    const double vn = dot3(vr, n);
                    if (vn < 0)
                        for (int m = 0; m < 3; ++m) vo[m] -= vn * n[m];
                }
            }
        }
        free(near);
    }
    grid_free(&grid);
    return err;
}

/* Friction of Eqs. 3-4 on a tangential displacement perp: all of it below
 * the static threshold, else the kinetic fraction thr_k / |perp| (capped at
 * the whole displacement). */
static void plain_friction(const double* perp, double thr_s, double thr_k, double* f)
{
    const double L = sqrt(dot3(perp, perp));
    const double kin = (L > 0 && thr_k / L < 1.0) ? thr_k / L : 1.0;
    const double scale = L < thr_s ? 1.0 : kin;
    for (int k = 0; k < 3; ++k) f[k] = perp[k] * scale;
}

/* One LR step, Algorithm 1 (Sec. 3), with the readings of the instrumented
 * or_pbd_step: predict (v += dt g for movable particles, xt = x + dt v,
 * inverse mass scaled by e^{k (z - ground)}); candidate partners
 * |xt_i - xt_j| < Rc; n_stab contact-only passes evaluated on x and applied
 * to x and xt; iters passes of contacts (Eqs. 1-2) and friction (Eqs. 3-4)
 * on xt, with the relative displacement over the step as the friction
 * displacement; every analytic SDF component is a partner of infinite mass;
 * Jacobi averaging x += (1/n_i) sum of the particle's corrections; then
 * v = (xt - x) / dt, x = xt.  x, v: double[N][3], updated in place. */
int or_pbd_step_plain(double* x, double* v, const double* inv_m, long N, const double* sdf, int n_sdf,
                      const double* prm)
{
    const int n_stab = (int)prm[PB_N_STAB], iters = (int)prm[PB_ITERS], fmode = (int)prm[PB_FRIC_MODE];
    const double r = prm[PB_R], dt = prm[PB_DT], Rc = prm[PB_RC], eps_x = prm[PB_EPS_X];
    const double mu_s = prm[PB_MU_S], mu_k = prm[PB_MU_K], d0 = 2.0 * r;
    const size_t n1 = (size_t)(N ? N : 1);
    double* xt = (double*)malloc(n1 * 3 * sizeof(double));
    double* ws = (double*)malloc(n1 * sizeof(double));
    double* D = (double*)malloc(n1 * 3 * sizeof(double));
    long* n_i = (long*)malloc(n1 * sizeof(long));
    long* first = (long*)calloc(n1 + 1, sizeof(long));   /* partners of i: partner[first[i] .. first[i+1]) */
    long* partner = NULL;
    int rc = (xt && ws && D && n_i && first) ? 0 : -1;
    or_grid_t grid;
    int have_grid = 0;
    if (rc == 0) {
        pbd_predict(x, v, inv_m, N, prm, xt, ws);
        rc = grid_build(&grid, xt, N, Rc);
        have_grid = rc == 0;
    }
    /* candidate partners from the predicted positions, ascending: counted,
     * then listed */
    const int nth = g_threads;
    for (int round = 0; round < 2 && rc == 0; ++round) {
#pragma omp parallel num_threads(nth) if (nth > 1)
        {
            long* near = (long*)malloc(n1 * sizeof(long));
            if (!near) rc = -1;
#pragma omp for schedule(dynamic, 256)
            for (long i = 0; i < N; ++i) {
                if (!near) continue;
                const long nn = grid_query(&grid, xt + 3 * i, near);
                long c = 0;
                for (long q = 0; q < nn; ++q) {
                    if (near[q] == i) continue;
                    if (round) partner[first[i] + c] = near[q];
                    ++c;
                }
                if (!round) first[i + 1] = c;
            }
            free(near);
        }
        if (round || rc) continue;
        for (long i = 0; i < N; ++i) first[i + 1] += first[i];
        if (!(partner = (long*)malloc((size_t)(first[N] ? first[N] : 1) * sizeof(long)))) rc = -1;
    }
    for (int it = 0; it < n_stab + iters && rc == 0; ++it) {
        const int stab = it < n_stab;
        const double* y = stab ? x : xt;   /* where the constraints are evaluated */
#pragma omp parallel for num_threads(nth) if (nth > 1) schedule(dynamic, 256)
        for (long i = 0; i < N; ++i) {
            double Di[3] = {0, 0, 0};
            long cnt = 0;
            /* Eqs. 1-2 (and 3-4) of each pair, evaluated from its lower index */
            for (long q = first[i]; q < first[i + 1]; ++q) {
                const long j = partner[q], a = i < j ? i : j, b = i < j ? j : i;
                double xab[3] = {y[3 * b] - y[3 * a], y[3 * b + 1] - y[3 * a + 1], y[3 * b + 2] - y[3 * a + 2]};
                const double d2 = dot3(xab, xab), d = sqrt(d2);
                if (!(d < d0) || d2 == 0.0) continue;
                const double wsum = ws[a] + ws[b];
                if (!(wsum > 0)) continue;
                const double ma = ws[a] / wsum, mb = ws[b] / wsum, pen = d0 - d;
                double ca[3], cb[3];
                for (int k = 0; k < 3; ++k) {
                    const double u = xab[k] / d;
                    ca[k] = -ma * pen * u;
                    cb[k] = mb * pen * u;
                }
                if (!stab) {
                    double dx[3], perp[3], f[3];
                    for (int k = 0; k < 3; ++k) dx[k] = (xt[3 * a + k] - x[3 * a + k]) - (xt[3 * b + k] - x[3 * b + k]);
                    const double s = dot3(dx, xab) / d2;
                    for (int k = 0; k < 3; ++k) perp[k] = dx[k] - s * xab[k];
                    const double base = fmode == 1 ? pen : d0;
                    plain_friction(perp, base * mu_s, base * mu_k, f);
                    for (int k = 0; k < 3; ++k) {
                        ca[k] -= ma * f[k];
                        cb[k] += mb * f[k];
                    }
                }
                for (int k = 0; k < 3; ++k) Di[k] += i == a ? ca[k] : cb[k];
                ++cnt;
            }
            /* boundary contacts: partners of infinite mass */
            for (int s = 0; s < n_sdf && ws[i] > 0; ++s) {
                const double *rec = sdf + OR_SDF_STRIDE * s, *ub = rec + 13;
                const double bmu_s = sqrt(mu_s * rec[16]), bmu_k = sqrt(mu_k * rec[17]);
                double phi[OR_MAX_COMP], nrm[3 * OR_MAX_COMP];
                int tie;
                const int nc = or_sdf_eval(rec, y + 3 * i, phi, nrm, &tie, eps_x);
                for (int c = 0; c < nc; ++c) {
                    if (!(phi[c] < r)) continue;
                    const double *n = nrm + 3 * c, pen = r - phi[c];
                    double ci[3];
                    for (int k = 0; k < 3; ++k) ci[k] = pen * n[k];
                    if (!stab) {
                        double dx[3], perp[3], f[3];
                        for (int k = 0; k < 3; ++k) dx[k] = (xt[3 * i + k] - x[3 * i + k]) - ub[k] * dt;
                        const double s2 = dot3(dx, n);
                        for (int k = 0; k < 3; ++k) perp[k] = dx[k] - s2 * n[k];
                        const double base = fmode == 1 ? pen : d0;
                        plain_friction(perp, base * bmu_s, base * bmu_k, f);
                        for (int k = 0; k < 3; ++k) ci[k] -= f[k];
                    }
                    for (int k = 0; k < 3; ++k) Di[k] += ci[k];
                    ++cnt;
                }
            }
            for (int k = 0; k < 3; ++k) D[3 * i + k] = Di[k];
            n_i[i] = cnt;
        }
        /* Jacobi averaging */
        for (long i = 0; i < N; ++i) {
            if (n_i[i] == 0) continue;
            for (int k = 0; k < 3; ++k) {
                const double dd = D[3 * i + k] / (double)n_i[i];
                xt[3 * i + k] += dd;
                if (stab) x[3 * i + k] += dd;
            }
        }
    }
    if (rc == 0)
        for (long i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] = (xt[3 * i + k] - x[3 * i + k]) / dt;
                x[3 * i + k] = xt[3 * i + k];
            }
    if (have_grid) grid_free(&grid);
    free(partner);
    free(first);
    free(n_i);
    free(D);
    free(ws);
    free(xt);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Initial sampling of a closed triangle mesh's volume (Sec. 4).        */
/*                                                                      */
/* The bounding box of the mesh is divided into cells of side           */
/* 2 r / sqrt(3); candidate positions (uniform random, given as input)  */
/* that lie inside the mesh are assigned to their cells; then, cell by  */
/* cell, the first candidate of the cell (in input order) that keeps a  */
/* distance of at least 2 r from every sample taken so far becomes the  */
/* cell's sample.  Readings:                                            */
/*  - inside = generalized winding number > 1/2 (a union of overlapping */
/*    closed meshes counts where any of them covers the point);        */
/*  - the cell order, which the paper leaves open: 27 phases            */
/*    (cx mod 3, cy mod 3, cz mod 3) with the phase index               */
/*    (cx mod 3) + 3 (cy mod 3) + 9 (cz mod 3) ascending, cells of a    */
/*    phase by linear index.  Two cells of one phase are at least three */
/*    cells apart along some axis, more than 2 r, so the cells of a     */
/*    phase never compete and the result does not depend on their      */
/*    order (which lets a parallel implementation take a phase at once);*/
/*  - two points of one cell are closer than 2 r (the cell's diagonal  */
/*    is 2 r), so a cell holds one sample at most, and a candidate can  */
/*    only conflict with samples of the 5 x 5 x 5 cells around it.      */
/* ------------------------------------------------------------------ */

/* Solid angle of triangle (a, b, c) seen from p over 4 pi (Van Oosterom and
 * Strackee, 1983: tan(Omega / 2) = det[a b c] / (|a||b||c| + (a.b)|c| +
 * (b.c)|a| + (c.a)|b|) with a, b, c relative to p). */
static double tri_winding(const double* A, const double* B, const double* C, const double* p)
{
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = A[k] - p[k];
        b[k] = B[k] - p[k];
        c[k] = C[k] - p[k];
    }
    const double la = sqrt(dot3(a, a)), lb = sqrt(dot3(b, b)), lc = sqrt(dot3(c, c));
    const double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                       a[2] * (b[0] * c[1] - b[1] * c[0]);
    const double den = la * lb * lc + dot3(a, b) * lc + dot3(b, c) * la + dot3(c, a) * lb;
    return atan2(det, den) / (2.0 * 3.14159265358979323846);   /* 2 atan2 / (4 pi) */
}

/* Generalized winding number of the mesh (V: double[nv][3], T: int[nt][3],
 * counter-clockwise seen from outside) at p: 1 inside a closed mesh, 0
 * outside. */
double or_winding_number(const double* V, const int32_t* T, long nt, const double* p)
{
    double w = 0.0;
    for (long t = 0; t < nt; ++t) w += tri_winding(V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2], p);
    return w;
}

/* The sampling grid over the bounding box of the nv vertices: origin lo[3],
 * cell side h = 2 r / sqrt(3), dims[3] = floor(extent / h) + 1. */
void or_sample_grid(const double* V, long nv, double r, double* lo, double* h, long* dims)
{
    double hi[3];
    for (int k = 0; k < 3; ++k) lo[k] = hi[k] = nv ? V[k] : 0.0;
    for (long i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k) {
            if (V[3 * i + k] < lo[k]) lo[k] = V[3 * i + k];
            if (V[3 * i + k] > hi[k]) hi[k] = V[3 * i + k];
        }
    *h = 2.0 * r / sqrt(3.0);
    for (int k = 0; k < 3; ++k) dims[k] = (long)floor((hi[k] - lo[k]) / *h) + 1;
}

/* The cell of p in the sampling grid (clamped to the grid). */
static long sample_cell(const double* p, const double* lo, double h, const long* dims, long* c)
{
    for (int k = 0; k < 3; ++k) {
        double f = floor((p[k] - lo[k]) / h);
        c[k] = f < 0 ? 0 : (f >= (double)(dims[k] - 1) ? dims[k] - 1 : (long)f);
    }
    return c[0] + dims[0] * (c[1] + dims[1] * c[2]);
}

/* The sampler.  cand: double[nc][3] candidate positions (uniform random in
 * the bounding box, drawn by the caller); r: particle radius.  selected
 * receives the indices of the chosen candidates in ascending cell order (at
 * most cap); returns their number, or -1 (allocation), -2 (cap too small),
 * -3 (grid of more than 2^31 cells).  inside (optional, nc) receives the
 * inside flag of every candidate. */
/* The cell-by-cell pick among the candidates flagged in in[] (see
 * or_sample_volume). */
static long sample_pick(const double* V, long nv, const double* cand, long nc, double r, const unsigned char* in,
                        long* selected, long cap)
{
    double lo[3], h;
    long dims[3];
    or_sample_grid(V, nv, r, lo, &h, dims);
    const double ncell_d = (double)dims[0] * (double)dims[1] * (double)dims[2];
    if (ncell_d > 2147483647.0) return -3;
    const long ncell = dims[0] * dims[1] * dims[2];
    long* first = (long*)calloc((size_t)ncell + 1, sizeof(long));   /* inside candidates of cell c: order[first[c] ..) */
    long* order = (long*)malloc((size_t)(nc ? nc : 1) * sizeof(long));
    long* pick = (long*)malloc((size_t)ncell * sizeof(long));        /* the cell's sample (candidate index) or -1 */
    long* cellof = (long*)malloc((size_t)(nc ? nc : 1) * sizeof(long));
    if (!first || !order || !pick || !cellof) {
        free(first); free(order); free(pick); free(cellof);
        return -1;
    }
    /* inside candidates by cell, in input order */
    for (long i = 0; i < nc; ++i) {
        long c3[3];
        cellof[i] = sample_cell(cand + 3 * i, lo, h, dims, c3);
        if (in[i]) first[cellof[i] + 1]++;
    }
    for (long c = 0; c < ncell; ++c) first[c + 1] += first[c];
    {
        long* fill = (long*)malloc((size_t)ncell * sizeof(long));
        if (!fill) { free(first); free(order); free(pick); free(cellof); return -1; }
        memcpy(fill, first, (size_t)ncell * sizeof(long));
        for (long i = 0; i < nc; ++i)
            if (in[i]) order[fill[cellof[i]]++] = i;
        free(fill);
    }
    for (long c = 0; c < ncell; ++c) pick[c] = -1;
    const double d2min = 4.0 * r * r;
    for (int phase = 0; phase < 27; ++phase) {
        const long px = phase % 3, py = (phase / 3) % 3, pz = phase / 9;
        for (long cz = pz; cz < dims[2]; cz += 3)
            for (long cy = py; cy < dims[1]; cy += 3)
                for (long cx = px; cx < dims[0]; cx += 3) {
                    const long c = cx + dims[0] * (cy + dims[1] * cz);
                    for (long q = first[c]; q < first[c + 1] && pick[c] < 0; ++q) {
                        const double* p = cand + 3 * order[q];
                        int free_ = 1;
                        for (long z = cz - 2; z <= cz + 2 && free_; ++z)
                            for (long y = cy - 2; y <= cy + 2 && free_; ++y)
                                for (long x = cx - 2; x <= cx + 2 && free_; ++x) {
                                    if (x < 0 || y < 0 || z < 0 || x >= dims[0] || y >= dims[1] || z >= dims[2]) continue;
                                    const long s = pick[x + dims[0] * (y + dims[1] * z)];
                                    if (s < 0) continue;
                                    const double* o = cand + 3 * s;
                                    double d[3] = {p[0] - o[0], p[1] - o[1], p[2] - o[2]};
                                    if (dot3(d, d) < d2min) free_ = 0;
                                }
                        if (free_) pick[c] = order[q];
                    }
                }
    }
    long n = 0;
    int full = 0;
    for (long c = 0; c < ncell; ++c) {
        if (pick[c] < 0) continue;
        if (n < cap) selected[n] = pick[c];
        else full = 1;
        ++n;
    }
    free(first); free(order); free(pick); free(cellof);
    return full ? -2 : n;
}

long or_sample_volume(const double* V, long nv, const int32_t* T, long nt, const double* cand, long nc, double r,
                      long* selected, long cap, unsigned char* inside)
{
    unsigned char* in = (unsigned char*)malloc((size_t)(nc ? nc : 1));
    if (!in) return -1;
    const int nth = g_threads;
#pragma omp parallel for num_threads(nth) if (nth > 1) schedule(dynamic, 64)
    for (long i = 0; i < nc; ++i) in[i] = or_winding_number(V, T, nt, cand + 3 * i) > 0.5;
    const long n = sample_pick(V, nv, cand, nc, r, in, selected, cap);
    if (inside)
        for (long i = 0; i < nc; ++i) inside[i] = in[i];
    free(in);
    return n;
}

/* Surface sampling (Sec. 3: a stationary body needs only its surface
 * sampled with particles of infinite mass): the same cell-by-cell pick,
 * every candidate valid.  The candidates are points on the mesh's triangles
 * (uniform by area, drawn by the caller); the grid is that of the vertices'
 * bounding box. */
long or_sample_surface(const double* V, long nv, const double* cand, long nc, double r, long* selected, long cap)
{
    unsigned char* in = (unsigned char*)malloc((size_t)(nc ? nc : 1));
    if (!in) return -1;
    memset(in, 1, (size_t)(nc ? nc : 1));
    const long n = sample_pick(V, nv, cand, nc, r, in, selected, cap);
    free(in);
    return n;
}
