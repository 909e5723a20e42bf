/*
 * rp.h -- C ABI of the GB300-native RadioPropa ray-propagation library.
 *
 * The library implements the ray-propagation method of Winchen, "RadioPropa -- A Modular
 * Raytracer for In-Matter Radio Propagation" (ARENA 2018): adaptive Cash-Karp integration
 * of the ray equation in a refractivity field (Sec. 2, Eqs. 1-2), the separate boundary
 * module (reflection, refraction by Snell's law, Fresnel amplitudes, a secondary ray cast
 * from the intersection point; Sec. 2), receivers, break conditions (Sec. 2, Fig. 1 text)
 * and source-receiver path finding (Sec. 2, accuracy study).  All computation runs in
 * CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions.  SI units.  z is depth, positive downward.  Angles are measured from +z.
 * Ray arrays are structure-of-arrays: a (3, n) array stores x[0..n), y[0..n), z[0..n).
 * Every array argument is a DEVICE pointer owned by the caller unless stated otherwise.
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls enqueue
 * their kernels on `stream` and return after synchronising it, so the device status can be
 * returned.
 *
 * Errors.  Every function returns RP_OK (0) or a negative RP_ERR_* code; rp_last_error()
 * gives a message for the last failure on the calling thread.  No C++ exception crosses the
 * ABI.  The library never traps, asserts or spins on the GPU: overflows are counted and
 * reported, every per-ray loop is bounded by max_steps.
 *
 * Concurrency.  Calls may come from several host threads; calls on the same device are
 * serialised internally because they share one grow-only device workspace.
 */
#ifndef RP_H
#define RP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RP_OK 0
#define RP_ERR_INVALID_ARG (-1)  /* bad argument (null pointer, size, parameter range) */
#define RP_ERR_CUDA (-2)         /* a CUDA runtime call failed (message has the detail) */
#define RP_ERR_OOM (-3)          /* device allocation failed */
#define RP_ERR_OVERFLOW (-4)     /* an output buffer was too small; rp_stats has the sizes */
#define RP_ERR_UNSUPPORTED (-5)  /* valid request this build does not provide */
#define RP_ERR_TIMEOUT (-6)      /* a bounded device-side wait gave up (the work it waited for
                                    did not complete in time); the context stays usable */

#define RP_MAX_LAYERS 8
#define RP_MAX_SPHERES 4
#define RP_MAX_WAVES 16 /* max_generation + 1 launches at most */

enum { RP_MEDIUM_LAYERED = 0, RP_MEDIUM_GRID = 1 };
enum { RP_FP64 = 0, RP_FP32_MIXED = 1 };
enum { RP_POL_S = 0, RP_POL_P = 1, RP_POL_UNPOL = 2 };
enum { RP_RHS_PROJECTED = 0, RP_RHS_PARAXIAL = 1, RP_RHS_MOMENTUM = 2 };

/* Per-ray end status. */
enum {
    RP_ST_ALIVE = 0,         /* never written for a finished ray */
    RP_ST_MAX_PATH = 1,      /* reached max_path (the last step is truncated to it) */
    RP_ST_MAX_TIME = 2,      /* travel time reached max_time (Fig. 1 text: 5 us) */
    RP_ST_MIN_AMP = 3,       /* |A| < min_amp |A0| (Fig. 1 text: A/A0 < 0.05) */
    RP_ST_LEFT_DOMAIN = 4,   /* left the refractivity grid */
    RP_ST_TRANSMITTED = 5,   /* refracted into an absorbing layer (e.g. air); not traced */
    RP_ST_REACHED_STOP = 6,  /* landed on the stop plane (path finding) */
    RP_ST_MAX_STEPS = 7,     /* attempted-step cap reached */
    RP_ST_BAD_INPUT = 8,     /* zero or non-finite direction */
    RP_ST_QUEUE_FULL = 9     /* secondary dropped: work queue full (also RP_ERR_OVERFLOW) */
};

/* ------------------------------------------------------------------------------------
 * Media (Sec. 2, Fig. 1 text and the paragraph after it)
 * ---------------------------------------------------------------------------------- */

/* Horizontal layer k spans z_top <= z < z_top of layer k+1 (layer 0's z_top is ignored and
 * read as -inf).  Inside it n(z) = n0 - dn * exp(-z / z0) + offset; dn = 0 gives a constant
 * index.  absorb != 0: a ray refracted into this layer is recorded with status
 * RP_ST_TRANSMITTED and not traced (the ice-air surface). */
typedef struct {
    double z_top, n0, dn, z0, offset;
    int32_t absorb, pad;
} rp_layer;

/* Spherical boundary inside a layered medium (curved boundaries, the paragraph after Fig. 1):
 * centre and radius [m]; inside it n(z) = n0 - dn * exp(-z / z0) + offset (dn = 0: constant);
 * absorb as for layers.  A ray inside sphere j is reported in region RP_MAX_LAYERS + j (the
 * `layer` output); outside every sphere its region is its layer.  The boundary split at the
 * sphere uses the local normal (r - centre) / radius. */
typedef struct {
    double center[3], radius, n0, dn, z0, offset;
    int32_t absorb, pad;
} rp_sphere;

/* Non-horizontal layer boundary (boundary shapes beyond the horizontal plane, the paragraph
 * after Fig. 1).  It replaces the plane z = z_top between layers `layer` - 1 and `layer`
 * (1 <= layer < n_layers) by the surface
 *   z = zb(x, y) = z_top + sx x + sy y + H(x, y),   (sx, sy) = -(normal[0], normal[1]) / normal[2]
 * -- the plane through (0, 0, z_top) with the given normal (normal[2] > 0; any length) -- plus,
 * if `height` is not NULL, the height field H: the bilinear interpolant of nx x ny (>= 2 each)
 * node heights [m], x fastest, node (i, j) at (origin[0] + i spacing[0], origin[1] +
 * j spacing[1]), held at its edge values beyond the nodes.  `height` may be a host or a device
 * pointer and is copied.  Layer k then spans zb_k(x, y) <= z < zb_{k+1}(x, y); the surfaces
 * must not cross where rays travel (not checked).  A ray lands on the surface by the Illinois
 * search on its vertical offset z - zb(x, y) (within eps_b), is put on it vertically, and the
 * boundary split uses the local normal (-dzb/dx, -dzb/dy, 1) / |...| and the indices of the two
 * layers at the point. */
typedef struct {
    int32_t layer, nx, ny, pad;
    double normal[3];
    double origin[2], spacing[2];
    const double *height;
} rp_surface;

/* kind = RP_MEDIUM_LAYERED: n_layers (1..8) layers, ordered top to bottom, z_top increasing,
 *   n_spheres (0..4) spheres, each strictly inside one layer, none overlapping another, and
 *   n_surfaces (0..n_layers-1) non-horizontal boundaries, each on a different layer boundary
 *   (media with spheres take no surfaces; rp_find_paths takes neither).
 * kind = RP_MEDIUM_GRID: node values of n on an nx * ny * nz grid (x fastest), node (i,j,k)
 *   at origin + spacing * (i,j,k); `grid_n` may be a host or a device pointer and is copied.
 *   The library derives grad n by central differences (one-sided on the faces) and stores
 *   (n, dn/dx, dn/dy, dn/dz) as FP32 node samples; n and grad n at a point are trilinear
 *   interpolations of those samples.  A ray whose committed position leaves the box ends
 *   with RP_ST_LEFT_DOMAIN.  Grid media have no boundaries. */
typedef struct {
    int32_t kind, n_layers;
    rp_layer layers[RP_MAX_LAYERS];
    int32_t nx, ny, nz, pad;
    double origin[3];
    double spacing;
    const float *grid_n;
    int32_t n_spheres, pad2;
    rp_sphere spheres[RP_MAX_SPHERES];
    int32_t n_surfaces, pad3;
    rp_surface surfaces[RP_MAX_LAYERS];
} rp_medium_desc;

typedef struct rp_medium_s *rp_medium_t;

/* Validates `desc`, copies it (and the grid, with its gradient precomputed by a kernel) to
 * the current device and returns an opaque handle in *out.  The handle owns its device
 * memory until rp_medium_destroy.  Errors: RP_ERR_INVALID_ARG (null pointer, bad layer count,
 * z_top not increasing, z0 <= 0 with dn != 0, grid smaller than 2 nodes per axis,
 * spacing <= 0, a sphere of radius <= 0, crossing a layer plane or overlapping another, a
 * surface on no inner boundary or on one taken, normal[2] <= 0, a height field of fewer than
 * 2 x 2 nodes, non-positive spacing or non-finite heights), RP_ERR_UNSUPPORTED (spheres and
 * surfaces in one medium), RP_ERR_OOM, RP_ERR_CUDA. */
int rp_medium_create(const rp_medium_desc *desc, void *stream, rp_medium_t *out);

/* Releases the handle and its device memory.  NULL is accepted. */
int rp_medium_destroy(rp_medium_t m);

/* ------------------------------------------------------------------------------------
 * Tracing (Sec. 2: Eqs. 1-2, Cash-Karp step control, boundary module, receivers, breaks)
 * ---------------------------------------------------------------------------------- */

/* n primaries: pos (3, n), dir (3, n; normalised by the library, a zero or non-finite
 * direction gives status RP_ST_BAD_INPUT), amp (n; NULL means 1).  Device pointers. */
typedef struct {
    int64_t n;
    const double *pos, *dir, *amp;
} rp_rays;

/* Receiver spheres: center (n, 3) row-major, radius (n).  Host or device pointers (when both
 * are host arrays they are read during the call; otherwise they are read back with a
 * synchronisation of the stream); n = 0 or a NULL rp_receivers pointer means none.  A hit is recorded when a committed step chord enters a
 * sphere (chord starts outside, entry point on the chord); receivers do not absorb. */
typedef struct {
    int32_t n, pad;
    const double *center, *radius;
} rp_receivers;

/* Integration parameters.
 *   tol          Cash-Karp tolerance on the error per unit step (dimensionless, > 0)
 *   h_min, h_max step bounds [m] (0 < h_min <= h_max); a step at h_min is always accepted
 *   h0           first step of a primary [m] (secondaries inherit their parent's step)
 *   max_path     arc-length limit [m]
 *   max_time     travel-time limit [s], <= 0: none
 *   min_amp      terminate when |A| < min_amp |A0|, <= 0: none (A0 of the root primary);
 *                a secondary whose amplitude would start below the threshold is not cast
 *   eps_b        boundary landing tolerance [m] (FP32_MIXED uses at least 2e-6 m)
 *   stop_n, stop_d, use_stop   optional stop plane stop_n . r = stop_d; stop_n must be +1 or -1
 *                along one coordinate axis and 0 along the others (RP_ERR_INVALID_ARG else)
 *   max_generation  secondaries are spawned while the parent's generation is below it
 *   precision    RP_FP64: every step in FP64 except the step-size factor of the step control
 *                (0.9 e^(-1/5), 0.9 e^(-1/4) on rejection: a heuristic, formed in FP32);
 *                RP_FP32_MIXED: Runge-Kutta stages, medium evaluation and step control in
 *                FP32; position, direction, travel time and path length accumulated in
 *                float-float (a pair of FP32 numbers, about 48 significant bits) on the FP32
 *                pipe; boundary splits in FP32 except the direction of a traced secondary
 *                (FP64); every output in FP64
 *   polarization RP_POL_S / RP_POL_P (signed field amplitudes) or RP_POL_UNPOL (square roots
 *                of the s/p-averaged reflectance and transmittance)
 *   rhs_form     RP_RHS_PROJECTED: t' = (grad n - (grad n . t) t)/n, Eq. 1 for unit t;
 *                RP_RHS_PARAXIAL: t' = grad n / n, Eq. 2, t renormalised after each step
 *                RP_RHS_MOMENTUM: Eq. 1 as written on p = n t (r' = p/|p|, p' = grad n), a
 *                cross-check of the projected form; RP_FP64 only (RP_ERR_INVALID_ARG else)
 *   max_steps    cap on attempted Cash-Karp steps per ray (> 0)
 * Scheduling knobs: they change which thread traces a ray and when, never a ray's record;
 * 0 selects the default.  rp_find_paths reads service_idle only.
 *   service_idle   idle lane-iterations after which a warp serves its parked lanes (boundary
 *                  splits, finished rays); default 256 in FP32_MIXED, 8 in FP64; >= 0
 *   flush_min      once a launch's input has run out, a thread hands the rest of its stack of
 *                  secondaries to the next launch when at least this many records remain
 *                  (default 2); >= 0
 *   block          threads per block of the tracing launches: 0 (128) or a multiple of 32 up
 *                  to 256
 *   blocks_per_sm  resident blocks per SM of the persistent launches: 0 or more than fit
 *                  means as many as fit
 *   ray_order      RP_ORDER_COHERENT (0, the default): rp_trace takes the primaries up in the
 *                  order of a counting sort on (launch direction's z component in 256 bins,
 *                  then start depth in 256 bins over the batch's range; 65,536 direction bins
 *                  if all rays start at one depth), so that the lanes of a warp trace rays that
 *                  follow similar paths and stay in step; each primary is still written at its
 *                  own index.  RP_ORDER_GIVEN (1): in the
 *                  order given.  rp_trace_static and rp_find_paths take the order given. */
typedef struct {
    double tol, h_min, h_max, h0, max_path, max_time, min_amp, eps_b;
    double stop_n[3], stop_d;
    int32_t use_stop, max_generation, precision, polarization, rhs_form, ray_order;
    int64_t max_steps;
    int32_t service_idle, flush_min, block, blocks_per_sm;
} rp_trace_params;

enum { RP_ORDER_COHERENT = 0, RP_ORDER_GIVEN = 1 };

/* Finished rays.  Primary i is written at index i; secondaries take the following indices as
 * they are cast, in no fixed order (each record's content does not depend on it).  Arrays of
 * length `capacity` (pos/dir: (3, capacity)); every pointer except end_pos may be NULL to skip
 * that field.  A secondary is identified by (parent, seq): seq is the index of the split on the
 * parent that cast it. */
typedef struct {
    int64_t capacity;
    double *end_pos, *end_dir, *path, *time, *amp;
    int32_t *status, *generation, *seq, *layer;
    int64_t *parent;
    int32_t *n_acc, *n_rej, *n_root, *n_refl, *n_turn;
} rp_ray_out;

/* Receiver hits, arrays of length `capacity` (pos/dir: (3, capacity)); order not
 * deterministic.  NULL rp_hits pointer: hits are only counted. */
typedef struct {
    int64_t capacity;
    int64_t *ray;
    int32_t *receiver;
    double *time, *path, *amp, *pos, *dir;
} rp_hits;

/* Host-side statistics of one call. */
typedef struct {
    int64_t rays;            /* rays finished (primaries + secondaries); output size needed */
    int64_t hits;            /* receiver hits; hit capacity needed */
    int64_t secondaries;     /* secondaries cast (queued or recorded as transmitted) */
    int64_t steps_accepted, steps_rejected, steps_root;
    int64_t queue_needed;    /* secondary records that had to be queued */
    int32_t waves, flags;    /* flags: 1 bad input, 2 output, 4 queue, 8 hit overflow,
                                16 a boundary search hit its iteration cap */
    double kernel_ms;        /* device time of the tracing kernels */
    double wave_ms[16];      /* device time of each generation's launch */
    double warp_end_ms[3];   /* first launch: earliest, median and last warp end [ms] */
    int64_t queue_capacity;  /* queue records the call had room for (queue_needed above it:
                                RP_ERR_OVERFLOW) */
    int32_t threads;         /* threads of each persistent launch (SMs x blocks x block) */
    int32_t stack_depth;     /* secondaries each thread keeps on its own stack */
} rp_stats;

/* Traces in->n primaries and every secondary they spawn, in max_generation + 1 persistent
 * launches: a thread traces the secondaries it casts itself until the launch's input runs out;
 * after that they go to a device queue that the next launch drains.  `rx` and `hits` may be
 * NULL, `stats` may be NULL.  Returns RP_OK, RP_ERR_INVALID_ARG (parameters, null arrays,
 * capacity < n), RP_ERR_OVERFLOW (out, queue or hit capacity exceeded: rp_stats holds the
 * sizes needed; everything that fitted was written), RP_ERR_OOM, RP_ERR_CUDA.  The
 * scheduling knobs of `p` (service_idle, flush_min, block, blocks_per_sm) change speed, not
 * any ray's record. */
int rp_trace(rp_medium_t m, const rp_rays *in, const rp_receivers *rx, const rp_trace_params *p,
             rp_ray_out *out, rp_hits *hits, rp_stats *stats, void *stream);

/* Size of the fixed device scratch array used by rp_trace_static, and the largest inputs
 * it accepts. */
#define RP_STATIC_SCRATCH_BYTES (32u << 20) /* 32 MiB, held by every device that loads the library */
#define RP_STATIC_MAX_RAYS (1 << 20)
#define RP_STATIC_MAX_RECEIVERS 1024

/* rp_trace without any device allocation (the paper has no counterpart: this is a deployment
 * variant).  For callers that cannot allocate device memory while they trace -- a process
 * whose device memory is owned by another allocator's pool, a service that forbids
 * cudaMalloc / cudaFree after start-up because they can synchronise the device, a tool with a
 * fixed memory budget.  Same arguments, semantics and results as rp_trace; its scratch space
 * (control block, receiver grid, per-thread secondary stacks, overflow queue) comes from one
 * static device array of RP_STATIC_SCRATCH_BYTES that every device using the library holds
 * until the process exits.  The call allocates no device or pinned host memory.
 *   - The first call on a device resolves the array's device address (cudaGetSymbolAddress,
 *     with that device current); make that first call before any stream capture.
 *   - All calls on a device share the array; they are serialised by a host lock, and calls
 *     that overlap on the GPU (e.g. from several processes' views of it) would race.  The
 *     control block is cleared at the start of every call; the rest is overwritten.
 *   - Limits: in->n <= RP_STATIC_MAX_RAYS and rx->n <= RP_STATIC_MAX_RECEIVERS
 *     (RP_ERR_INVALID_ARG beyond).  The secondary-ray queue is smaller than rp_trace's; if it
 *     fills, the call returns RP_ERR_OVERFLOW with rp_stats as for rp_trace
 *     (rp_stats.queue_needed against rp_stats.queue_capacity).  What fits depends on the
 *     workload and the launch: the per-thread stacks take at most half of the array (one
 *     120-byte record per thread and level), the queue the rest.  On a GB300 the FP32-mixed
 *     layered kernel runs 77,824 threads (152 SMs x 4 blocks x 128): one stacked secondary per
 *     thread and a queue of about 199,000 records, which holds the 2^20-primary two-layer-ice
 *     workload (0.75 secondaries per primary; it queues about 194,000).  Fewer blocks_per_sm
 *     give deeper stacks; the call also fails with RP_ERR_INVALID_ARG when not even one record
 *     per thread fits beside the receivers' tables.
 *   - Like rp_trace, it synchronises `stream` before it returns.
 *   - rp_stats.warp_end_ms is not filled (its read-back would need pinned host memory). */
int rp_trace_static(rp_medium_t m, const rp_rays *in, const rp_receivers *rx,
                    const rp_trace_params *p, rp_ray_out *out, rp_hits *hits, rp_stats *stats,
                    void *stream);

/* ------------------------------------------------------------------------------------
 * Source-receiver path finding (Sec. 2, accuracy study)
 * ---------------------------------------------------------------------------------- */

/* trace: integration parameters (max_path, use_stop, stop_* and max_generation are set per
 *   pair by the library: path budget 2 (D + z_s + z_r) + 100 m, stop plane x = D, no
 *   secondaries).  hit_tol: accept when the vertical miss at x = D is below it [m].
 *   max_iter: bisection cap per bracket.  max_sol: solution slots per pair (1..8). */
typedef struct {
    rp_trace_params trace;
    double hit_tol;
    int32_t max_iter, max_sol;
} rp_path_params;

enum { RP_SOL_DIRECT = 0, RP_SOL_REFRACTED = 1, RP_SOL_REFLECTED = 2 };

/* Solutions, device arrays: count (n_pairs); the rest (n_pairs, max_sol) row-major, slots
 * beyond count[i] zeroed, slots sorted by travel time.  type: RP_SOL_*; launch / receive:
 * launch and arrival angles from +z [rad]; time [s], path [m], amp (Fresnel factors);
 * miss: vertical miss at the receiver [m]; n_iter: bisection steps. */
typedef struct {
    int32_t *count, *type, *n_iter;
    double *launch, *receive, *time, *path, *amp, *miss;
} rp_solutions;

/* For each pair (z_s[i], z_r[i], D[i]) with n_angles[i] >= 2 scan angles: rays from
 * (0, 0, z_s) at angles pi j / (n_angles - 1) in the x-z plane are traced to the plane x = D;
 * adjacent angles whose vertical misses change sign are refined by FP64 bisection on the
 * launch angle until |miss| < hit_tol.  A ray that exhausts its path budget before x = D
 * scores +inf (it is far below).  D < hit_tol: the vertical ray to the receiver depth.
 * Layered media with horizontal boundaries and without spheres only.  Solution type: REFLECTED if the ray reflected off a
 * boundary, REFRACTED if it turned (t_z changed sign), else DIRECT.  Returns RP_OK, RP_ERR_INVALID_ARG, RP_ERR_OOM,
 * RP_ERR_CUDA. */
int rp_find_paths(rp_medium_t m, int64_t n_pairs, const double *z_s, const double *z_r,
                  const double *dist, const int32_t *n_angles, const rp_path_params *p,
                  rp_solutions *sol, rp_stats *stats, void *stream);

/* ------------------------------------------------------------------------------------
 * Learned surrogate of the path finder (not in the paper: a model that maps a
 * source-receiver geometry to the path finder's solutions)
 * ---------------------------------------------------------------------------------- */

/* Network 3 -> 256 -> 256 -> 256 -> 256 -> 12, GELU (0.5 x (1 + erf(x / sqrt 2))) after each
 * hidden layer.  Parameters are one flat float32 vector W0, b0, W1, b1, ..., W4, b4 with W_l
 * stored (in, out) row-major.  FP32 master weights; every product runs on the tensor cores
 * with BF16 operands (weights and activations rounded to BF16) and FP32 accumulation.
 * Inputs x: (n, 3) float32 rows; outputs: (n, 12) float32 rows = for slot k = 0, 1:
 * existence logit, then five regression outputs (see rp_surrogate_encode). */
typedef struct rp_surrogate_s *rp_surrogate_t;

/* Number of parameters (201,484). */
int rp_surrogate_n_params(void);

/* Creates a network on the current device from `params` (host or device, copied); Adam
 * state zeroed. */
int rp_surrogate_create(const float *params, rp_surrogate_t *out);
int rp_surrogate_destroy(rp_surrogate_t s);

/* Bound on every wait of the surrogate's tensor-core kernels for their own bulk copies and
 * matrix products (mbarrier waits), in SM clock cycles; 0 (the default) means 4e9, about two
 * seconds.  The paper has no counterpart: this is the library's hang protection.  A CTA whose
 * wait gives up records it, waits (with the default bound) for the work it has already issued,
 * releases its tensor memory and returns; the call then returns RP_ERR_TIMEOUT and the device
 * context stays usable.  Returns RP_ERR_INVALID_ARG for a null handle or a negative limit. */
int rp_surrogate_set_wait_limit(rp_surrogate_t s, int64_t cycles);

/* Replaces the parameters (host or device pointer; Adam state reset) / copies them out. */
int rp_surrogate_set_params(rp_surrogate_t s, const float *params);
int rp_surrogate_get_params(rp_surrogate_t s, float *params);

/* out (n, 12) = network(x (n, 3)).  Device pointers.  RP_ERR_TIMEOUT: see
 * rp_surrogate_set_wait_limit. */
int rp_surrogate_forward(rp_surrogate_t s, int64_t n, const float *x, float *out, void *stream);

/* Mean loss over n rows and its gradient (flat, like the parameters; device or host pointer,
 * may be NULL) without updating.  y: (n, 2) existence targets in [0, 1]; t: (n, 10) regression
 * targets (slot-major).  Loss per row: for each slot, softplus(logit) - y logit
 * + y * 0.5 * |regression outputs - t|^2. */
int rp_surrogate_loss_grad(rp_surrogate_t s, int64_t n, const float *x, const float *y,
                           const float *t, double *loss, float *grad, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the mean loss of the n
 * rows; *loss (may be NULL) receives that loss before the update. */
int rp_surrogate_train_step(rp_surrogate_t s, int64_t n, const float *x, const float *y,
                            const float *t, float lr, double *loss, void *stream);

/* Checkpoint: writes the parameters, the Adam moments and the step count to a host file /
 * creates a network on the current device from such a file.  Binary little-endian layout:
 * 8-byte magic "RPSUR001", int64 parameter count, int64 Adam step, then the float32 vectors
 * params, m, v.  RP_ERR_INVALID_ARG for a missing, short or foreign file. */
int rp_surrogate_save(rp_surrogate_t s, const char *path);
int rp_surrogate_load(const char *path, rp_surrogate_t *out);

/* Training schedule for rp_surrogate_train.  The n rows are split into floor(n / batch)
 * contiguous batches (a trailing partial batch is not used); each epoch visits them in an
 * order drawn from `seed`, one Adam step per batch, with the learning rate decayed from lr to
 * lr_final along a half cosine over all steps.  Rows must already be in random order (the
 * batches are contiguous). */
typedef struct {
    int32_t epochs, batch;
    float lr, lr_final;
    uint64_t seed;
} rp_train_params;

/* Runs the whole schedule on the device (device pointers x (n, 3), y (n, 2), t (n, 10)).
 * *loss (may be NULL): mean of the batch losses of the last epoch, each taken before its
 * update.  The Adam state carries over between calls. */
int rp_surrogate_train(rp_surrogate_t s, int64_t n, const float *x, const float *y,
                       const float *t, const rp_train_params *p, double *loss, void *stream);

/* Normalisation shared by training data and inference.
 *   x = (2 z_s / RP_SUR_ZS_MAX - 1, 2 z_r / RP_SUR_ZR_MAX - 1, 2 D / RP_SUR_D_MAX - 1);
 *   slot k holds the k-th earliest solution; y_k = 1 if it exists, 0 if not, and 0.5 for both
 *   slots of a pair with more than two solutions (the network cannot hold them, so it is
 *   taught to be unsure there and such pairs go to the path finder);
 *   t_k = (2 launch / pi - 1, 2 receive / pi - 1, (c T / RP_SUR_N_REF - L) / RP_SUR_LEN_SCALE,
 *          (path - L) / RP_SUR_LEN_SCALE, amp), L the straight source-receiver distance,
 *   zero for an empty slot. */
#define RP_SUR_ZS_MAX 2000.0
#define RP_SUR_ZR_MAX 200.0
#define RP_SUR_D_MAX 4000.0
#define RP_SUR_N_REF 1.78
#define RP_SUR_LEN_SCALE 100.0

/* Encodes n pairs (device arrays) into network inputs x (n, 3); with y and t non-NULL also the
 * targets y (n, 2) and t (n, 10) from the path finder's solutions `sol` (max_sol >= 2 slots
 * per pair). */
int rp_surrogate_encode(int64_t n, const double *z_s, const double *z_r, const double *dist,
                        const rp_solutions *sol, int32_t max_sol, float *x, float *y, float *t,
                        void *stream);

/* Inference with the tracer as judge and fallback.
 *   conf: a slot whose existence probability sigmoid(logit) is <= 1 - conf is taken to be
 *     absent (0.5 < conf < 1); every other slot is refined, and exists only if its
 *     refinement converges.  A pair whose slot 0 is taken to be absent but slot 1 not goes to
 *     the path finder.
 *   refine_tol: a refined solution is accepted when its vertical miss |z - z_r| < refine_tol
 *     [m]; travel time, path, angles, amplitude and type then come from that trace.
 *   refine_step: the second secant point is launch + refine_step [rad].
 *   max_step: secant steps (before a sign change brackets the root) are clamped to this
 *     length [rad]; a ray that exhausts its path budget sends the search halfway back.
 *   refine_iters: traces per slot at most. */
typedef struct {
    double conf, refine_tol, refine_step, max_step;
    int32_t refine_iters;
    int32_t deflate;  /* 1: slot 1's search runs on the miss with slot 0's root deflated away
                         (miss / (launch - root)); 0: on the miss itself */
} rp_surrogate_params;

typedef struct {
    int64_t queries;       /* pairs */
    int64_t tasks;         /* queries refined from the network's launch angles */
    int64_t tasks_failed;  /* of them: a slot did not converge (the pair fell back) */
    int64_t fail_end;      /*   ... a trace ended before the receiver plane */
    int64_t fail_iters;    /*   ... refine_iters traces without convergence */
    int64_t fail_step;     /*   ... a step longer than max_step or leaving (0, pi) */
    int64_t duplicates;    /* pairs whose two slots converged to the same ray (fell back) */
    int64_t deflated;      /* slot-1 searches run on the deflated miss */
    int64_t fallback;      /* pairs solved by the path finder */
    int64_t refine_rays, refine_steps;      /* traces (and accepted steps) of the refinement */
    int64_t fallback_rays, fallback_steps;  /* traces (and accepted steps) of the fallback */
    float ms_forward, ms_refine, ms_fallback, ms_total;  /* device time per phase */
    float ms_fallback_scan;  /* of ms_fallback: the path finder's angle scan */
} rp_surrogate_stats;

/* Solves n pairs like rp_find_paths: the network predicts, per pair, which of the two
 * earliest solutions exist and their launch angles; each solution not ruled out is refined
 * from its predicted launch angle (secant steps, then Illinois false position once a sign
 * change brackets the root; one full trace per step) until its miss is below refine_tol, slot
 * 0 first and slot 1 on the miss with slot 0's root deflated away.  Pairs with a slot that does
 * not converge, two slots on the same ray, or D < p->hit_tol are solved by rp_find_paths with
 * `p` instead (up to p->max_sol solutions;
 * network-served pairs have at most two).  Output as for
 * rp_find_paths (n_iter = traces of the refinement).  p->max_sol >= 2.  Returns RP_OK,
 * RP_ERR_INVALID_ARG, RP_ERR_OOM, RP_ERR_CUDA, or RP_ERR_OVERFLOW from the fallback. */
int rp_surrogate_find_paths(rp_surrogate_t s, rp_medium_t m, int64_t n, const double *z_s,
                            const double *z_r, const double *dist, const int32_t *n_angles,
                            const rp_path_params *p, const rp_surrogate_params *sp,
                            rp_solutions *sol, rp_surrogate_stats *stats, void *stream);

/* ------------------------------------------------------------------------------------
 * Misc
 * ---------------------------------------------------------------------------------- */

/* Roofline denominators of the current device, measured (the paper has no counterpart: this
 * is the measurement side of the library).  Three microkernels on `stream`, each the best of
 * three timed launches after an untimed one (about 10 ms each):
 *   fp32_tflops, fp64_tflops  fused multiply-adds on the CUDA cores, 8 independent chains per
 *                             thread, 1,024 threads per SM (FMA = 2 flops);
 *   l2_gbs                    16-byte loads that bypass L1, streamed by every SM over a
 *                             RP_PEAKS_L2_BUFFER-byte buffer (far smaller than L2, read once
 *                             before the timed launches, so every load hits L2).
 * The *_ms fields are the timed launches' durations; report the SM clock sampled while they
 * run beside the rates.  Allocates and frees the buffer.  Returns RP_OK, RP_ERR_INVALID_ARG
 * (null out), RP_ERR_OOM, RP_ERR_CUDA. */
#define RP_PEAKS_L2_BUFFER (32u << 20)
typedef struct {
    double fp32_tflops, fp64_tflops, l2_gbs;
    double fp32_ms, fp64_ms, l2_ms, l2_buffer_bytes;
} rp_peaks;
int rp_measure_peaks(rp_peaks *out, void *stream);

/* Copies the last error message of the calling thread into buf (NUL-terminated, truncated
 * to len).  Returns the full message length. */
int rp_last_error(char *buf, size_t len);

/* Library version string (static storage). */
const char *rp_version(void);

#ifdef __cplusplus
}
#endif
#endif
