/*
 * rp_oracle.h -- plain FP64 CPU oracle of the RadioPropa ray-propagation method
 * (Winchen, "RadioPropa -- A Modular Raytracer for In-Matter Radio Propagation", ARENA 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load this library.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only through the seeded input arrays.
 *
 * Conventions (all SI): z is depth, positive downward; launch angles are measured from +z;
 * c0 = 299 792 458 m/s; a ray state is y = (r, t, T) with r the position, t the unit tangent
 * dr/ds, T the travel time, s the arc length (Sec. 2, Eq. 1).
 *
 * Parity status of every function is stated beside it: each is pinned by the CPU tests
 * (closed forms, invariants, brute force, exact geometry); none is unpinned.
 */
#ifndef RP_ORACLE_H
#define RP_ORACLE_H
#include <stdint.h>

#define OR_MAX_LAYERS 8
#define OR_MAX_SPHERES 4

enum { OR_MEDIUM_LAYERED = 0, OR_MEDIUM_GRID = 1 };
enum { OR_RHS_PROJECTED = 0, OR_RHS_PARAXIAL = 1, OR_RHS_MOMENTUM = 2 };
enum { OR_POL_S = 0, OR_POL_P = 1, OR_POL_UNPOL = 2 };
enum {
    OR_ST_ALIVE = 0, OR_ST_MAX_PATH = 1, OR_ST_MAX_TIME = 2, OR_ST_MIN_AMP = 3,
    OR_ST_LEFT_DOMAIN = 4, OR_ST_TRANSMITTED = 5, OR_ST_REACHED_STOP = 6, OR_ST_MAX_STEPS = 7
};
enum { OR_SOL_DIRECT = 0, OR_SOL_REFRACTED = 1, OR_SOL_REFLECTED = 2 };

/* Refractivity model.  LAYERED: horizontal slabs in depth, layer k spans
 * z_top[k] <= z < z_top[k+1] (z_top[0] is ignored: -inf; the last layer extends to +inf);
 * inside layer k,  n(z) = n0[k] - dn[k] * exp(-z / z0[k]) + off[k]   (Sec. 2, Fig. 1 text);
 * dn[k] == 0 gives a constant layer.  absorb[k] != 0: rays refracted into layer k are recorded
 * as terminated (status TRANSMITTED) and not traced further.
 * Curved boundaries (the paragraph after Fig. 1): up to OR_MAX_SPHERES spheres in a layered
 * medium, sphere j of centre sph_c[j] and radius sph_R[j], with its own index formula inside,
 * n = sph_n0 - sph_dn exp(-z / sph_z0) + sph_off, and sph_absorb as for layers.  A sphere lies
 * inside one layer and spheres do not overlap.  Regions: a ray in layer k outside every sphere
 * is in region k, a ray inside sphere j in region OR_MAX_LAYERS + j.
 * GRID: node samples (n, dn/dx, dn/dy, dn/dz) as float4, x fastest, node (i,j,k) at
 * origin + spacing*(i,j,k); trilinear interpolation of all four channels.  No boundaries. */
typedef struct {
    int32_t kind, n_layers;
    double z_top[OR_MAX_LAYERS], n0[OR_MAX_LAYERS], dn[OR_MAX_LAYERS], z0[OR_MAX_LAYERS],
           off[OR_MAX_LAYERS];
    int32_t absorb[OR_MAX_LAYERS];
    int32_t nx, ny, nz, pad;
    double origin[3], spacing;
    const float *grid4;
    int32_t n_spheres, pad2;
    double sph_c[OR_MAX_SPHERES][3], sph_R[OR_MAX_SPHERES], sph_n0[OR_MAX_SPHERES],
           sph_dn[OR_MAX_SPHERES], sph_z0[OR_MAX_SPHERES], sph_off[OR_MAX_SPHERES];
    int32_t sph_absorb[OR_MAX_SPHERES];
    /* Non-horizontal boundaries (boundary shapes beyond the plane, the paragraph after Fig. 1):
     * with srf_on[k] != 0 the boundary between layers k-1 and k (k >= 1) is the surface
     *   z = zb_k(x, y) = z_top[k] + srf_sx[k] x + srf_sy[k] y + H_k(x, y)
     * instead of the plane z = z_top[k]: a tilted plane of slopes (srf_sx, srf_sy) through
     * (0, 0, z_top[k]) plus, if hf[k] != NULL, the height field H_k, the bilinear interpolant
     * of hf_nx[k] x hf_ny[k] node heights hf[k] (x fastest; node (i, j) at
     * (hf_ox[k] + i hf_dx[k], hf_oy[k] + j hf_dy[k])), held at its edge values outside the
     * nodes.  Layer k is zb_k(x, y) <= z < zb_{k+1}(x, y); the caller keeps the surfaces
     * from crossing where rays travel.  Not combined with spheres. */
    int32_t srf_on[OR_MAX_LAYERS];
    double srf_sx[OR_MAX_LAYERS], srf_sy[OR_MAX_LAYERS];
    int32_t hf_nx[OR_MAX_LAYERS], hf_ny[OR_MAX_LAYERS];
    double hf_ox[OR_MAX_LAYERS], hf_oy[OR_MAX_LAYERS], hf_dx[OR_MAX_LAYERS], hf_dy[OR_MAX_LAYERS];
    const double *hf[OR_MAX_LAYERS];
} or_medium;

/* Integration and termination parameters. */
typedef struct {
    double tol;        /* Cash-Karp error tolerance (dimensionless, per unit step) */
    double h_min, h_max, h0;   /* step bounds and initial step [m] */
    double max_path;   /* arc-length limit [m] */
    double max_time;   /* travel-time limit [s] (<= 0: none) */
    double min_amp;    /* discard when |A| < min_amp * |A0| (<= 0: none) */
    double eps_b;      /* boundary landing tolerance [m] */
    double stop_n[3], stop_d;  /* optional stop plane  stop_n . r = stop_d */
    int32_t use_stop, max_generation, polarization, rhs_form;
    int64_t max_steps; /* cap on attempted Cash-Karp steps per ray */
} or_params;

/* One finished ray (primary or secondary); `layer` is the ray's region (see or_medium). */
typedef struct {
    int64_t parent, root;      /* parent ray index (-1 for primaries), root primary index */
    int32_t seq, gen, status, layer;  /* seq: index of the split on the parent that made it */
    double pos[3], dir[3], path, time, amp, amp0;
    int64_t n_acc, n_rej, n_root;     /* committed steps, rejected steps, root-search steps */
    int32_t n_refl, n_turn;           /* boundary reflections, turning points (t_z sign flips) */
    int32_t root_fail, pad;
} or_ray;

/* One receiver hit: the ray entered receiver sphere `receiver`. */
typedef struct {
    int64_t ray;
    int32_t receiver, pad;
    double time, path, amp, pos[3], dir[3];
} or_hit;

/* One source-receiver solution. */
typedef struct {
    int32_t type, n_iter, converged, pad;
    double launch, receive, time, path, amp, miss;
} or_solution;

#ifdef __cplusplus
extern "C" {
#endif

/* Cash-Karp tableau as used by the stepper (exported for the order-condition tests).
 * Pinned: the 17 order conditions to order 5 (b5) and the 8 to order 4 (b4). */
extern const double or_ck_c[6];
extern const double or_ck_a[6][5];
extern const double or_ck_b5[6];
extern const double or_ck_b4[6];

/* One Cash-Karp step of the scalar quadrature y' = sum_k coef[k] x^k from (x0, y0) with
 * step h, returning the 5th- and 4th-order results (tableau exactness tests).
 * Pinned: exact for polynomials up to the order of each weight set. */
void or_ck_poly_step(const double *coef, int32_t n_coef, double x0, double y0, double h,
                     double *y5, double *y4);

/* n and grad n of the medium at r for a ray in region `layer` (layered: that region's
 * formula, continued smoothly beyond its boundaries; grid: trilinear, clamped to the box).
 * Pinned: the profile and its derivative at a point; exact on linear grid fields; offsets. */
void or_medium_eval(const or_medium *m, int32_t layer, const double *r, double *n, double *g);

/* Layer index containing depth z (a boundary depth belongs to the layer below).
 * Pinned: start layer of rays just above, at and just below a boundary. */
int32_t or_layer_of(const or_medium *m, double z);

/* Depth zb_k(x, y) of boundary k (1 <= k < n_layers) and its slopes dzb/dx, dzb/dy (the
 * plane z_top[k], or the tilted plane plus height field of or_medium).
 * Pinned: a height field sampled from a plane reproduces that plane; slopes of a bump. */
double or_boundary_depth(const or_medium *m, int32_t k, double x, double y, double *dzdx,
                         double *dzdy);

/* Layer containing the point r: the last k with r[2] >= zb_k(r[0], r[1]) (0 if none).
 * Pinned: start layer above, on and below a tilted boundary and a height field. */
int32_t or_layer_at(const or_medium *m, const double *r);

/* Region containing r: OR_MAX_LAYERS + j inside sphere j, else the layer of r[2].
 * Pinned: rays started at the centre and just inside the surface of a sphere. */
int32_t or_region_of(const or_medium *m, const double *r);

/* FP32 node samples (n, grad n) from FP32 node values of n: central differences inside,
 * one-sided differences on the faces, evaluated in double and rounded to float.
 * Pinned: exact gradients of linear fields on every node, faces included. */
void or_grid_prepare(const float *n, int32_t nx, int32_t ny, int32_t nz, double spacing,
                     float *out4);

/* Right-hand side of the ray equations (PROJECTED = Eq. 1 for unit t; PARAXIAL = Eq. 2;
 * MOMENTUM = Eq. 1 as written, on the state (r, p = n t, T): r' = p / |p|, p' = grad n).
 * Pinned: values at a point; t' orthogonal to t; Snell invariant and closed forms along
 * whole rays for PROJECTED and MOMENTUM; PARAXIAL shown less accurate. */
void or_rhs(const or_medium *m, int32_t layer, int32_t form, const double *y, double *k);

/* One Cash-Karp step of the ray system (pinned: local error ~ h^6; the error measure
 * ~ h^4, its position part per unit step); returns the unscaled error measure
 * max(|sum (b5-b4) k_r|, h |sum (b5-b4) k_t|); y5 is the 5th-order state (t not normalised).
 * MOMENTUM: the stages run on p = n(r0) t0; y5 holds p5 in place of t (its direction is t) and
 * the direction error is h |sum (b5-b4) k_p| / n(r0). */
double or_ck_step(const or_medium *m, int32_t layer, int32_t form, const double *y0, double h,
                  double *y5);

/* Boundary split (Snell + Fresnel) at a plane with unit normal nrm pointing toward the
 * incident side.  Outputs reflected and refracted unit directions, amplitude factors r, tau
 * and tir (1 = total internal reflection).
 * Pinned: vector Snell law, plane of incidence, total internal reflection past the critical
 * angle, matched media, exact geometry of splits at constant layers and spheres. */
void or_split_dirs(const double *t, const double *nrm, double n1, double n2, int32_t pol,
                   double *t_refl, double *t_refr, double *r, double *tau, int32_t *tir);

/* Fresnel coefficients: amplitude reflection r and transmission tau for incidence cosine
 * cos_i and refraction cosine cos_t (Sec. 2, last paragraph of the boundary module).
 * Pinned: R + T = 1 (s, p, unpolarised), normal incidence, Brewster angle, matched media. */
void or_fresnel(double n1, double n2, double cos_i, double cos_t, int32_t pol, double *r,
                double *tau);

/* Trace n primaries (SoA: pos[3][n], dir[3][n], amp[n]) with every secondary they spawn.
 * Pinned: straight lines at constant n; closed-form range, path and time in the exponential
 * profile; Fermat's principle in the random grid; splits, receivers, break conditions, step
 * law and landing against exact geometry (the CPU pin tests list each one).
 * Receivers: n_rx spheres, centre AoS rx_c[n_rx][3], radius rx_r[n_rx].
 * Writes up to out_cap rays and hit_cap hits; returns the total number of rays (may exceed
 * out_cap), *n_hits the total number of hits (may exceed hit_cap). */
int64_t or_trace(const or_medium *m, const or_params *p, int64_t n, const double *pos,
                 const double *dir, const double *amp, int32_t n_rx, const double *rx_c,
                 const double *rx_r, or_ray *out, int64_t out_cap, or_hit *hits,
                 int64_t hit_cap, int64_t *n_hits);

/* Source-receiver path finding (pinned: the paper's accuracy study and closed-form roots in
 * the Snell invariant, launch and receive angles; vertical pairs): for each pair
 * (z_s, z_r, D) scan n_angles launch angles in [0, pi], bracket sign changes of the vertical
 * miss at x = D and bisect in the launch angle until |miss| < hit_tol.  Solutions sorted by travel time, at most max_sol per pair;
 * count[i] receives their number.  Returns 0. */
int32_t or_find_paths(const or_medium *m, const or_params *p, int64_t n_pairs,
                      const double *zs, const double *zr, const double *dist,
                      const int32_t *n_angles, double hit_tol, int32_t max_iter,
                      int32_t max_sol, int32_t *count, or_solution *sol);

#ifdef __cplusplus
}
#endif
#endif
