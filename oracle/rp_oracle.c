/*
 * rp_oracle.c -- plain FP64 CPU oracle of the RadioPropa ray-propagation method.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark).  Written
 * from the paper's method description, straight-line and slow on purpose: no blocking, no
 * fusion, one ray at a time.  Shares nothing with the CUDA library.
 *
 * What it follows:
 *   ray equation            Sec. 2, Eq. (1) (eikonal) and Eq. (2) (locally paraxial form)
 *   integrator              Sec. 2: the Cash-Karp embedded Runge-Kutta pair (Cash & Karp 1990),
 *                           adaptive step with a minimum step and a tolerance (Sec. 2, accuracy
 *                           paragraph)
 *   boundaries              Sec. 2: boundaries are a separate module; on passing one the ray is
 *                           reflected and a secondary (refracted) ray is cast from the
 *                           intersection point, amplitudes from Fresnel's equations
 *   media                   Sec. 2, Fig. 1 text: n(z) = n0 - dn exp(-z/z0), layered; gridded
 *                           refractivity (Sec. 2, last paragraph before the accuracy study)
 *   break conditions        Sec. 2, Fig. 1 text: maximum propagation time, A/A0 threshold
 *   receivers               Sec. 2: receiver locations (spheres)
 *   path finding            Sec. 2, accuracy study: launch angles reaching a given observer
 * Readings where the paper is silent are listed in the design notes and restated where used.
 */
#include "rp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define C0 299792458.0
#define ROOT_MAX_ITER 40

/* ---------------------------------------------------------------------------------------
 * Cash-Karp 1990 tableau: nodes c, stage matrix a (lower triangle), fifth-order weights b5
 * and embedded fourth-order weights b4.  The fifth-order solution is propagated.
 * ------------------------------------------------------------------------------------- */
const double or_ck_c[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
const double or_ck_a[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
const double or_ck_b5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
const double or_ck_b4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                            277.0 / 14336.0, 1.0 / 4.0};

void or_ck_poly_step(const double *coef, int32_t n_coef, double x0, double y0, double h,
                     double *y5, double *y4)
{
    double k[6];
    for (int i = 0; i < 6; ++i) {
        double x = x0 + or_ck_c[i] * h, f = 0.0, xp = 1.0;
        for (int j = 0; j < n_coef; ++j) { f += coef[j] * xp; xp *= x; }
        k[i] = f;
    }
    double s5 = 0.0, s4 = 0.0;
    for (int i = 0; i < 6; ++i) { s5 += or_ck_b5[i] * k[i]; s4 += or_ck_b4[i] * k[i]; }
    *y5 = y0 + h * s5;
    *y4 = y0 + h * s4;
}

/* ---------------------------------------------------------------------------------------
 * Media
 * ------------------------------------------------------------------------------------- */
int32_t or_layer_of(const or_medium *m, double z)
{
    int32_t k = 0;
    for (int32_t j = 1; j < m->n_layers; ++j)
        if (z >= m->z_top[j]) k = j;
    return k;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Bilinear height field H_k at (x, y) and its partial derivatives (zero where the point lies
 * beyond the nodes along that axis: the field is held at its edge values there). */
static double height_field(const or_medium *m, int32_t k, double x, double y, double *hx,
                           double *hy)
{
    const int32_t nx = m->hf_nx[k], ny = m->hf_ny[k];
    const double u_raw = (x - m->hf_ox[k]) / m->hf_dx[k];
    const double v_raw = (y - m->hf_oy[k]) / m->hf_dy[k];
    const double u = clampd(u_raw, 0.0, (double)(nx - 1));
    const double v = clampd(v_raw, 0.0, (double)(ny - 1));
    int32_t i = (int32_t)floor(u), j = (int32_t)floor(v);
    if (i > nx - 2) i = nx - 2;
    if (j > ny - 2) j = ny - 2;
    const double fu = u - i, fv = v - j;
    const double *h = m->hf[k];
    const double h00 = h[(int64_t)j * nx + i], h10 = h[(int64_t)j * nx + i + 1];
    const double h01 = h[(int64_t)(j + 1) * nx + i], h11 = h[(int64_t)(j + 1) * nx + i + 1];
    *hx = (u_raw >= 0.0 && u_raw <= nx - 1)
              ? ((1.0 - fv) * (h10 - h00) + fv * (h11 - h01)) / m->hf_dx[k] : 0.0;
    *hy = (v_raw >= 0.0 && v_raw <= ny - 1)
              ? ((1.0 - fu) * (h01 - h00) + fu * (h11 - h10)) / m->hf_dy[k] : 0.0;
    return (1.0 - fu) * (1.0 - fv) * h00 + fu * (1.0 - fv) * h10 + (1.0 - fu) * fv * h01 +
           fu * fv * h11;
}

/* Depth of boundary k at (x, y): the plane z_top[k], or the tilted plane plus the height
 * field of a non-horizontal boundary; its slopes in *dzdx, *dzdy (may be NULL). */
double or_boundary_depth(const or_medium *m, int32_t k, double x, double y, double *dzdx,
                         double *dzdy)
{
    double z = m->z_top[k], gx = 0.0, gy = 0.0;
    if (m->srf_on[k]) {
        z += m->srf_sx[k] * x + m->srf_sy[k] * y;
        gx = m->srf_sx[k];
        gy = m->srf_sy[k];
        if (m->hf[k]) {
            double hx, hy;
            z += height_field(m, k, x, y, &hx, &hy);
            gx += hx;
            gy += hy;
        }
    }
    if (dzdx) *dzdx = gx;
    if (dzdy) *dzdy = gy;
    return z;
}

/* Layer containing the point r: the last boundary at or above it, at its (x, y). */
int32_t or_layer_at(const or_medium *m, const double *r)
{
    int32_t k = 0;
    for (int32_t j = 1; j < m->n_layers; ++j)
        if (r[2] >= or_boundary_depth(m, j, r[0], r[1], NULL, NULL)) k = j;
    return k;
}

/* Region containing r: inside sphere j -> OR_MAX_LAYERS + j, else the layer of the point. */
int32_t or_region_of(const or_medium *m, const double *r)
{
    for (int32_t j = 0; j < m->n_spheres; ++j) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) d2 += (r[a] - m->sph_c[j][a]) * (r[a] - m->sph_c[j][a]);
        if (d2 < m->sph_R[j] * m->sph_R[j]) return OR_MAX_LAYERS + j;
    }
    return or_layer_at(m, r);
}

/* n(z) = n0 - dn exp(-z/z0) + off and dn/dz = (dn/z0) exp(-z/z0) of region k (a layer, or
 * the inside of a sphere)  (Sec. 2, Fig. 1 text). */
static void layer_eval(const or_medium *m, int32_t k, double z, double *n, double *dndz)
{
    double n0, dn, z0, off;
    if (k >= OR_MAX_LAYERS) {
        const int32_t j = k - OR_MAX_LAYERS;
        n0 = m->sph_n0[j];
        dn = m->sph_dn[j];
        z0 = m->sph_z0[j];
        off = m->sph_off[j];
    } else {
        n0 = m->n0[k];
        dn = m->dn[k];
        z0 = m->z0[k];
        off = m->off[k];
    }
    if (dn == 0.0) {
        *n = n0 + off;
        *dndz = 0.0;
        return;
    }
    double e = exp(-z / z0);
    *n = n0 - dn * e + off;
    *dndz = dn / z0 * e;
}

static int32_t region_absorbs(const or_medium *m, int32_t k)
{
    return k >= OR_MAX_LAYERS ? m->sph_absorb[k - OR_MAX_LAYERS] : m->absorb[k];
}

static void grid_eval(const or_medium *m, const double *r, double *n, double *g)
{
    const int32_t dims[3] = {m->nx, m->ny, m->nz};
    int32_t idx[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        double f = clampd((r[a] - m->origin[a]) / m->spacing, 0.0, (double)(dims[a] - 1));
        int32_t i = (int32_t)floor(f);
        if (i > dims[a] - 2) i = dims[a] - 2;
        idx[a] = i;
        w[a] = f - (double)i;
    }
    double v[4];
    for (int c = 0; c < 4; ++c) {
        double e[2][2];
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy) {
                size_t base = ((size_t)(idx[2] + dz) * m->ny + (size_t)(idx[1] + dy)) * m->nx +
                              (size_t)idx[0];
                double a0 = (double)m->grid4[4 * base + c];
                double a1 = (double)m->grid4[4 * (base + 1) + c];
                e[dz][dy] = a0 + w[0] * (a1 - a0);
            }
        double f0 = e[0][0] + w[1] * (e[0][1] - e[0][0]);
        double f1 = e[1][0] + w[1] * (e[1][1] - e[1][0]);
        v[c] = f0 + w[2] * (f1 - f0);
    }
    *n = v[0];
    g[0] = v[1];
    g[1] = v[2];
    g[2] = v[3];
}

void or_medium_eval(const or_medium *m, int32_t layer, const double *r, double *n, double *g)
{
    if (m->kind == OR_MEDIUM_GRID) {
        grid_eval(m, r, n, g);
        return;
    }
    double dndz;
    layer_eval(m, layer, r[2], n, &dndz);
    g[0] = 0.0;
    g[1] = 0.0;
    g[2] = dndz;
}

void or_grid_prepare(const float *n, int32_t nx, int32_t ny, int32_t nz, double spacing,
                     float *out4)
{
    for (int32_t k = 0; k < nz; ++k)
        for (int32_t j = 0; j < ny; ++j)
            for (int32_t i = 0; i < nx; ++i) {
                size_t c = ((size_t)k * ny + j) * nx + i;
                const int32_t ijk[3] = {i, j, k}, dims[3] = {nx, ny, nz};
                const size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
                out4[4 * c] = n[c];
                for (int a = 0; a < 3; ++a) {
                    double d;
                    if (ijk[a] == 0)
                        d = ((double)n[c + stride[a]] - (double)n[c]) / spacing;
                    else if (ijk[a] == dims[a] - 1)
                        d = ((double)n[c] - (double)n[c - stride[a]]) / spacing;
                    else
                        d = ((double)n[c + stride[a]] - (double)n[c - stride[a]]) / (2.0 * spacing);
                    out4[4 * c + 1 + a] = (float)d;
                }
            }
}

static int grid_inside(const or_medium *m, const double *r)
{
    const int32_t dims[3] = {m->nx, m->ny, m->nz};
    for (int a = 0; a < 3; ++a) {
        double hi = m->origin[a] + m->spacing * (double)(dims[a] - 1);
        if (r[a] < m->origin[a] || r[a] > hi) return 0;
    }
    return 1;
}

/* ---------------------------------------------------------------------------------------
 * Ray equations.  State y = (x, y, z, tx, ty, tz, T), derivative with respect to s.
 *   PROJECTED: d/ds (n t) = grad n (Eq. 1) with |t| = 1 gives
 *              t' = (grad n - (grad n . t) t) / n
 *   PARAXIAL:  n d2r/ds2 = grad n (Eq. 2), i.e. t' = grad n / n
 *   r' = t, T' = n / c0 (phase index).
 * ------------------------------------------------------------------------------------- */
void or_rhs(const or_medium *m, int32_t layer, int32_t form, const double *y, double *k)
{
    double n, g[3];
    or_medium_eval(m, layer, y, &n, g);
    if (form == OR_RHS_MOMENTUM) {
        /* d/ds (n t) = grad n with p = n t:  r' = p / |p|,  p' = grad n */
        const double q = sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
        for (int i = 0; i < 3; ++i) {
            k[i] = y[3 + i] / q;
            k[3 + i] = g[i];
        }
        k[6] = n / C0;
        return;
    }
    k[0] = y[3];
    k[1] = y[4];
    k[2] = y[5];
    if (form == OR_RHS_PROJECTED) {
        double gt = g[0] * y[3] + g[1] * y[4] + g[2] * y[5];
        for (int i = 0; i < 3; ++i) k[3 + i] = (g[i] - gt * y[3 + i]) / n;
    } else {
        for (int i = 0; i < 3; ++i) k[3 + i] = g[i] / n;
    }
    k[6] = n / C0;
}

double or_ck_step(const or_medium *m, int32_t layer, int32_t form, const double *y0_in,
                  double h, double *y5)
{
    double k[6][7], ys[7], y0[7], n0 = 1.0;
    for (int c = 0; c < 7; ++c) y0[c] = y0_in[c];
    if (form == OR_RHS_MOMENTUM) { /* the stages run on p = n(r0) t0 */
        double g[3];
        or_medium_eval(m, layer, y0_in, &n0, g);
        for (int c = 3; c < 6; ++c) y0[c] = n0 * y0_in[c];
    }
    for (int i = 0; i < 6; ++i) {
        for (int c = 0; c < 7; ++c) {
            double acc = 0.0;
            for (int j = 0; j < i; ++j) acc += or_ck_a[i][j] * k[j][c];
            ys[c] = y0[c] + h * acc;
        }
        or_rhs(m, layer, form, ys, k[i]);
    }
    double er2 = 0.0, et2 = 0.0;
    for (int c = 0; c < 7; ++c) {
        double s5 = 0.0, d = 0.0;
        for (int i = 0; i < 6; ++i) {
            s5 += or_ck_b5[i] * k[i][c];
            d += (or_ck_b5[i] - or_ck_b4[i]) * k[i][c];
        }
        y5[c] = y0[c] + h * s5;
        if (c < 3)
            er2 += d * d;
        else if (c < 6)
            et2 += (h * d) * (h * d);
    }
    return fmax(sqrt(er2), sqrt(et2) / n0);
}

static void normalise3(double *v)
{
    double q = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= q;
    v[1] /= q;
    v[2] /= q;
}

/* ---------------------------------------------------------------------------------------
 * Boundary module: Snell reflection/refraction and Fresnel amplitudes (Sec. 2).
 * ------------------------------------------------------------------------------------- */
void or_fresnel(double n1, double n2, double cos_i, double cos_t, int32_t pol, double *r,
                double *tau)
{
    double rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
    double ts = 2.0 * n1 * cos_i / (n1 * cos_i + n2 * cos_t);
    double rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);
    double tp = 2.0 * n1 * cos_i / (n2 * cos_i + n1 * cos_t);
    if (pol == OR_POL_S) {
        *r = rs;
        *tau = ts;
    } else if (pol == OR_POL_P) {
        *r = rp;
        *tau = tp;
    } else {
        /* unpolarised: energy reflectance/transmittance averaged over s and p, amplitudes
         * returned as their square roots */
        double R = 0.5 * (rs * rs + rp * rp);
        *r = sqrt(R);
        *tau = sqrt(1.0 - R);
    }
}

void or_split_dirs(const double *t, const double *nrm, double n1, double n2, int32_t pol,
                   double *t_refl, double *t_refr, double *r, double *tau, int32_t *tir)
{
    double cos_i = -(t[0] * nrm[0] + t[1] * nrm[1] + t[2] * nrm[2]);
    if (cos_i < 0.0) cos_i = 0.0;
    for (int a = 0; a < 3; ++a) t_refl[a] = t[a] + 2.0 * cos_i * nrm[a];
    normalise3(t_refl);
    double eta = n1 / n2;
    double sin2_t = eta * eta * (1.0 - cos_i * cos_i);
    if (sin2_t > 1.0) {
        *tir = 1;
        *r = 1.0; /* |r| = 1; the phase of total internal reflection is not tracked */
        *tau = 0.0;
        for (int a = 0; a < 3; ++a) t_refr[a] = 0.0;
        return;
    }
    *tir = 0;
    double cos_t = sqrt(1.0 - sin2_t);
    for (int a = 0; a < 3; ++a) t_refr[a] = eta * t[a] + (eta * cos_i - cos_t) * nrm[a];
    normalise3(t_refr);
    or_fresnel(n1, n2, cos_i, cos_t, pol, r, tau);
}

/* ---------------------------------------------------------------------------------------
 * Tracer
 * ------------------------------------------------------------------------------------- */
typedef struct {
    double r[3], t[3], T, s, A, A0, h;
    int32_t layer, gen, seq;
    int64_t id, parent, root;
} start_state;

typedef struct {
    const or_medium *m;
    const or_params *p;
    int32_t n_rx;
    const double *rx_c, *rx_r;
    or_ray *out;
    int64_t out_cap, n_out;
    or_hit *hits;
    int64_t hit_cap, n_hits;
    start_state *queue;
    int64_t q_cap, q_len, q_head;
} trace_ctx;

/* Event kinds: the planes above and below the ray's layer, the stop plane, and sphere j's
 * surface (EV_SPHERE + j). */
enum { EV_NONE = 0, EV_TOP = 1, EV_BOTTOM = 2, EV_STOP = 3, EV_SPHERE = 4 };

/* distance of r from sphere j's centre */
static double sphere_dist(const or_medium *m, int32_t j, const double *y)
{
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) d2 += (y[a] - m->sph_c[j][a]) * (y[a] - m->sph_c[j][a]);
    return sqrt(d2);
}

/* Signed distance to an event surface, positive on the ray's own side. */
static double event_g(const trace_ctx *c, int32_t layer, int kind, double stop_sign,
                      const double *y)
{
    const or_medium *m = c->m;
    const or_params *p = c->p;
    if (kind == EV_TOP) return y[2] - or_boundary_depth(m, layer, y[0], y[1], NULL, NULL);
    if (kind == EV_BOTTOM) return or_boundary_depth(m, layer + 1, y[0], y[1], NULL, NULL) - y[2];
    if (kind >= EV_SPHERE) {
        const int32_t j = kind - EV_SPHERE;
        const double g = sphere_dist(m, j, y) - m->sph_R[j];
        return layer == OR_MAX_LAYERS + j ? -g : g;
    }
    double f = p->stop_n[0] * y[0] + p->stop_n[1] * y[1] + p->stop_n[2] * y[2] - p->stop_d;
    return stop_sign * f;
}

/* Puts the landing point exactly on the surface: a layer boundary at the point's (x, y)
 * depth, the stop plane by its normal, the sphere radially. */
static void snap_to_plane(const trace_ctx *c, int32_t layer, int kind, double *y)
{
    const or_params *p = c->p;
    if (kind == EV_TOP) {
        y[2] = or_boundary_depth(c->m, layer, y[0], y[1], NULL, NULL);
    } else if (kind == EV_BOTTOM) {
        y[2] = or_boundary_depth(c->m, layer + 1, y[0], y[1], NULL, NULL);
    } else if (kind >= EV_SPHERE) {
        const int32_t j = kind - EV_SPHERE;
        const double q = c->m->sph_R[j] / sphere_dist(c->m, j, y);
        for (int a = 0; a < 3; ++a) y[a] = c->m->sph_c[j][a] + q * (y[a] - c->m->sph_c[j][a]);
    } else {
        double f = p->stop_n[0] * y[0] + p->stop_n[1] * y[1] + p->stop_n[2] * y[2] - p->stop_d;
        for (int a = 0; a < 3; ++a) y[a] -= f * p->stop_n[a];
    }
}

static void emit_ray(trace_ctx *c, const start_state *st, const double *y, double s, double A,
                     int32_t layer, int32_t status, int64_t n_acc, int64_t n_rej,
                     int64_t n_root, int32_t n_refl, int32_t n_turn, int32_t root_fail)
{
    int64_t idx = st->id;
    if (idx < c->out_cap) {
        or_ray *o = &c->out[idx];
        o->parent = st->parent;
        o->root = st->root;
        o->seq = st->seq;
        o->gen = st->gen;
        o->status = status;
        o->layer = layer;
        for (int a = 0; a < 3; ++a) {
            o->pos[a] = y[a];
            o->dir[a] = y[3 + a];
        }
        o->path = s;
        o->time = y[6];
        o->amp = A;
        o->amp0 = st->A0;
        o->n_acc = n_acc;
        o->n_rej = n_rej;
        o->n_root = n_root;
        o->n_refl = n_refl;
        o->n_turn = n_turn;
        o->root_fail = root_fail;
        o->pad = 0;
    }
}

static void push_secondary(trace_ctx *c, const start_state *st)
{
    if (c->q_len == c->q_cap) {
        c->q_cap = c->q_cap ? 2 * c->q_cap : 1024;
        c->queue = (start_state *)realloc(c->queue, (size_t)c->q_cap * sizeof(start_state));
    }
    c->queue[c->q_len++] = *st;
}

/* Receiver test on the committed chord r0 -> r1: a hit is recorded when the chord enters
 * the sphere (start outside, entry point within the chord); quantities at the entry point
 * are interpolated linearly along the chord. */
static void receivers_on_chord(trace_ctx *c, const start_state *st, const double *y0,
                               double s0, const double *y1, double s1, double A)
{
    for (int32_t j = 0; j < c->n_rx; ++j) {
        const double *ctr = &c->rx_c[3 * j];
        double R = c->rx_r[j];
        double d[3], w[3];
        for (int a = 0; a < 3; ++a) {
            d[a] = y1[a] - y0[a];
            w[a] = y0[a] - ctr[a];
        }
        double qa = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double qb = 2.0 * (d[0] * w[0] + d[1] * w[1] + d[2] * w[2]);
        double qc = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] - R * R;
        if (qc <= 0.0 || qa == 0.0) continue; /* chord starts inside (or on) the sphere */
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc < 0.0) continue;
        double lam = (-qb - sqrt(disc)) / (2.0 * qa);
        if (lam < 0.0 || lam > 1.0) continue;
        int64_t k = c->n_hits++;
        if (k < c->hit_cap) {
            or_hit *hp = &c->hits[k];
            hp->ray = st->id;
            hp->receiver = j;
            hp->pad = 0;
            hp->time = y0[6] + lam * (y1[6] - y0[6]);
            hp->path = s0 + lam * (s1 - s0);
            hp->amp = A;
            double dir[3];
            for (int a = 0; a < 3; ++a) {
                hp->pos[a] = y0[a] + lam * d[a];
                dir[a] = y0[3 + a] + lam * (y1[3 + a] - y0[3 + a]);
            }
            normalise3(dir);
            for (int a = 0; a < 3; ++a) hp->dir[a] = dir[a];
        }
    }
}

/* Illinois (modified regula falsi) search for the step h* in (0, h] at which the step from
 * y0 lands on the event plane; writes the landing state (on the plane) to y_land. */
static double land_on_plane(trace_ctx *c, int32_t layer, int kind, double stop_sign,
                            const double *y0, double h, const double *y1, double g0, double g1,
                            double *y_land, int64_t *n_root, int32_t *fail)
{
    const or_params *p = c->p;
    double a = 0.0, ga = g0, b = h, gb = g1, cpt = h, yc[7];
    memcpy(yc, y1, sizeof yc);
    int done = 0;
    if (fabs(gb) <= p->eps_b) {
        done = 1; /* the trial step itself ends on the plane */
    } else if (ga <= p->eps_b) {
        /* the step starts on the plane: search beyond the minimum step */
        if (h <= p->h_min) {
            done = 1; /* the whole (minimum) step is the event step */
        } else {
            cpt = p->h_min;
            or_ck_step(c->m, layer, p->rhs_form, y0, cpt, yc);
            normalise3(yc + 3);
            ++*n_root;
            double gc = event_g(c, layer, kind, stop_sign, yc);
            if (gc <= p->eps_b) {
                done = 1;
            } else {
                a = cpt;
                ga = gc;
            }
        }
    }
    int side = 0, it = 0;
    while (!done) {
        if (it == ROOT_MAX_ITER) {
            *fail = 1;
            break;
        }
        ++it;
        cpt = b - gb * (b - a) / (gb - ga);
        if (!(cpt > a && cpt < b)) cpt = 0.5 * (a + b);
        or_ck_step(c->m, layer, p->rhs_form, y0, cpt, yc);
        normalise3(yc + 3);
        ++*n_root;
        double gc = event_g(c, layer, kind, stop_sign, yc);
        if (fabs(gc) <= p->eps_b) break;
        if (gc > 0.0) {
            a = cpt;
            ga = gc;
            if (side == 1) gb *= 0.5;
            side = 1;
        } else {
            b = cpt;
            gb = gc;
            if (side == -1) ga *= 0.5;
            side = -1;
        }
    }
    memcpy(y_land, yc, sizeof yc);
    snap_to_plane(c, layer, kind, y_land);
    return cpt;
}

static void trace_one(trace_ctx *c, const start_state *st)
{
    const or_medium *m = c->m;
    const or_params *p = c->p;
    double y[7] = {st->r[0], st->r[1], st->r[2], st->t[0], st->t[1], st->t[2], st->T};
    double s = st->s, A = st->A, h = st->h;
    int32_t layer = st->layer, status = OR_ST_ALIVE, n_refl = 0, n_turn = 0, n_split = 0,
            root_fail = 0;
    int64_t n_acc = 0, n_rej = 0, n_root = 0;
    int layered = (m->kind == OR_MEDIUM_LAYERED);
    double stop_sign = 0.0;
    if (p->use_stop) {
        double f = p->stop_n[0] * y[0] + p->stop_n[1] * y[1] + p->stop_n[2] * y[2] - p->stop_d;
        stop_sign = (f <= 0.0) ? -1.0 : 1.0;
    }

    while (status == OR_ST_ALIVE) {
        if (n_acc + n_rej + n_root >= p->max_steps) {
            status = OR_ST_MAX_STEPS;
            break;
        }
        /* never step beyond the path limit */
        double h_try = h;
        int last = 0;
        if (s + h_try >= p->max_path) {
            h_try = p->max_path - s;
            last = 1;
        }
        double y1[7];
        double e = or_ck_step(m, layer, p->rhs_form, y, h_try, y1) / p->tol;
        if (!(e <= 1.0) && h_try > p->h_min) {
            ++n_rej;
            double fac = 0.9 * pow(e, -0.25);
            if (!(fac >= 0.1)) fac = 0.1;
            h = h_try * fac;
            if (h < p->h_min) h = p->h_min;
            continue;
        }
        double grow = (e == 0.0) ? 5.0 : 0.9 * pow(e, -0.2);
        if (grow > 5.0) grow = 5.0;
        double h_next = h_try * grow;
        if (h_next < p->h_min) h_next = p->h_min;
        if (h_next > p->h_max) h_next = p->h_max;
        normalise3(y1 + 3);

        /* event detection: earliest crossed plane, by linear fraction along the step */
        int ev = EV_NONE;
        double ev_frac = 2.0, ev_g0 = 0.0, ev_g1 = 0.0;
        const int in_sphere = layer >= OR_MAX_LAYERS;
        for (int kind = EV_TOP; kind < EV_SPHERE + m->n_spheres; ++kind) {
            if (kind == EV_TOP && !(layered && !in_sphere && layer > 0)) continue;
            if (kind == EV_BOTTOM && !(layered && !in_sphere && layer < m->n_layers - 1)) continue;
            if (kind == EV_STOP && !p->use_stop) continue;
            /* a ray inside a sphere meets only that sphere's surface */
            if (kind >= EV_SPHERE && in_sphere && layer != OR_MAX_LAYERS + kind - EV_SPHERE)
                continue;
            double g0 = event_g(c, layer, kind, stop_sign, y);
            double g1 = event_g(c, layer, kind, stop_sign, y1);
            /* crossed, or arrived within eps_b of the plane from the ray's own side */
            if (g1 < 0.0 || (g1 <= p->eps_b && g0 > p->eps_b)) {
                double fr = (g0 > 0.0) ? g0 / (g0 - g1) : 0.0;
                if (fr < ev_frac) {
                    ev = kind;
                    ev_frac = fr;
                    ev_g0 = g0;
                    ev_g1 = g1;
                }
            }
        }
        double h_used = h_try;
        if (ev != EV_NONE) {
            double yl[7];
            h_used = land_on_plane(c, layer, ev, stop_sign, y, h_try, y1, ev_g0, ev_g1, yl,
                                   &n_root, &root_fail);
            memcpy(y1, yl, sizeof yl);
        }

        /* commit the chord y -> y1 */
        double s1 = (last && ev == EV_NONE) ? p->max_path : s + h_used;
        receivers_on_chord(c, st, y, s, y1, s1, A);
        if ((y[5] > 0.0) != (y1[5] > 0.0)) ++n_turn;
        memcpy(y, y1, sizeof y);
        s = s1;
        ++n_acc;
        h = h_next;

        if (ev == EV_TOP || ev == EV_BOTTOM || ev >= EV_SPHERE) {
            /* split at the plane between `layer` and its neighbour, or at a sphere's surface;
             * nrm: the unit normal pointing toward the incident side */
            int32_t other;
            double nrm[3] = {0.0, 0.0, (ev == EV_TOP) ? 1.0 : -1.0};
            if (ev >= EV_SPHERE) {
                const int32_t j = ev - EV_SPHERE;
                const int inside = layer == OR_MAX_LAYERS + j;
                const double d = sphere_dist(m, j, y);
                for (int a = 0; a < 3; ++a)
                    nrm[a] = (inside ? -1.0 : 1.0) * (y[a] - m->sph_c[j][a]) / d;
                other = inside ? or_layer_at(m, y) : OR_MAX_LAYERS + j;
            } else {
                other = (ev == EV_TOP) ? layer - 1 : layer + 1;
                const int32_t kb = (ev == EV_TOP) ? layer : layer + 1;
                if (m->srf_on[kb]) {
                    /* the surface z - zb(x, y) = 0: normal (-dzb/dx, -dzb/dy, 1) / |...|,
                     * pointing into the layer below; toward the incident side */
                    double bx, by;
                    or_boundary_depth(m, kb, y[0], y[1], &bx, &by);
                    const double q = sqrt(bx * bx + by * by + 1.0);
                    const double sg = (ev == EV_TOP) ? 1.0 : -1.0;
                    nrm[0] = -sg * bx / q;
                    nrm[1] = -sg * by / q;
                    nrm[2] = sg / q;
                }
            }
            double zb = y[2], n1, n2, dd;
            layer_eval(m, layer, zb, &n1, &dd);
            layer_eval(m, other, zb, &n2, &dd);
            double t_refl[3], t_refr[3], rr, tau;
            int32_t tir;
            or_split_dirs(y + 3, nrm, n1, n2, p->polarization, t_refl, t_refr, &rr, &tau, &tir);
            int weak = p->min_amp > 0.0 && fabs(A * tau) < p->min_amp * fabs(st->A0);
            if (!tir && st->gen < p->max_generation && !weak) {
                start_state sec;
                memcpy(sec.r, y, 3 * sizeof(double));
                memcpy(sec.t, t_refr, 3 * sizeof(double));
                sec.T = y[6];
                sec.s = s;
                sec.A = A * tau;
                sec.A0 = st->A0;
                sec.h = h;
                sec.layer = other;
                sec.gen = st->gen + 1;
                sec.seq = n_split;
                sec.id = c->n_out++;
                sec.parent = st->id;
                sec.root = st->root;
                if (region_absorbs(m, other)) {
                    /* refracted into an absorbing region: recorded, not traced */
                    double ys[7] = {y[0], y[1], y[2], t_refr[0], t_refr[1], t_refr[2], y[6]};
                    emit_ray(c, &sec, ys, s, sec.A, other, OR_ST_TRANSMITTED, 0, 0, 0, 0, 0, 0);
                } else {
                    push_secondary(c, &sec);
                }
            }
            ++n_split;
            ++n_refl;
            memcpy(y + 3, t_refl, 3 * sizeof(double));
            A *= rr;
        } else if (ev == EV_STOP) {
            status = OR_ST_REACHED_STOP;
            break;
        }

        if (last && ev == EV_NONE) {
            status = OR_ST_MAX_PATH;
        } else if (p->max_time > 0.0 && y[6] >= p->max_time) {
            status = OR_ST_MAX_TIME;
        } else if (p->min_amp > 0.0 && fabs(A) < p->min_amp * fabs(st->A0)) {
            status = OR_ST_MIN_AMP;
        } else if (!layered && !grid_inside(m, y)) {
            status = OR_ST_LEFT_DOMAIN;
        }
    }
    emit_ray(c, st, y, s, A, layer, status, n_acc, n_rej, n_root, n_refl, n_turn, root_fail);
}

int64_t or_trace(const or_medium *m, const or_params *p, int64_t n, const double *pos,
                 const double *dir, const double *amp, int32_t n_rx, const double *rx_c,
                 const double *rx_r, or_ray *out, int64_t out_cap, or_hit *hits,
                 int64_t hit_cap, int64_t *n_hits)
{
    trace_ctx c;
    memset(&c, 0, sizeof c);
    c.m = m;
    c.p = p;
    c.n_rx = n_rx;
    c.rx_c = rx_c;
    c.rx_r = rx_r;
    c.out = out;
    c.out_cap = out_cap;
    c.hits = hits;
    c.hit_cap = hit_cap;
    c.n_out = n;
    for (int64_t i = 0; i < n; ++i) {
        start_state st;
        st.r[0] = pos[i];
        st.r[1] = pos[n + i];
        st.r[2] = pos[2 * n + i];
        st.t[0] = dir[i];
        st.t[1] = dir[n + i];
        st.t[2] = dir[2 * n + i];
        normalise3(st.t);
        st.T = 0.0;
        st.s = 0.0;
        st.A = amp[i];
        st.A0 = amp[i];
        st.h = p->h0;
        st.layer = (m->kind == OR_MEDIUM_LAYERED) ? or_region_of(m, st.r) : 0;
        st.gen = 0;
        st.seq = 0;
        st.id = i;
        st.parent = -1;
        st.root = i;
        trace_one(&c, &st);
        /* secondaries of this primary, breadth first */
        while (c.q_head < c.q_len) {
            start_state sec = c.queue[c.q_head++];
            trace_one(&c, &sec);
        }
        c.q_head = c.q_len = 0;
    }
    free(c.queue);
    *n_hits = c.n_hits;
    return c.n_out;
}

/* ---------------------------------------------------------------------------------------
 * Source-receiver path finding (Sec. 2, accuracy study: launch angles that reach an
 * observation point).  Rays run in the x-z plane from (0, 0, z_s) with direction
 * (sin th, 0, cos th) and stop on the plane x = D; the vertical miss there is
 * z - z_r.  A ray that exhausts its path budget without reaching x = D is far below the
 * receiver (rays bend toward higher n, i.e. downward) and scores a miss of +inf.
 * Path budget per pair: 2 (D + z_s + z_r) + 100 m.  No secondaries are traced.
 * ------------------------------------------------------------------------------------- */
static void pf_trace(const or_medium *m, const or_params *pp, double zs, double th, or_ray *rec)
{
    double pos[3] = {0.0, 0.0, zs}, dir[3] = {sin(th), 0.0, cos(th)}, amp = 1.0;
    int64_t nh = 0;
    or_trace(m, pp, 1, pos, dir, &amp, 0, NULL, NULL, rec, 1, NULL, 0, &nh);
}

static double pf_miss(const or_ray *r, double zr)
{
    if (r->status == OR_ST_REACHED_STOP) return r->pos[2] - zr;
    if (r->status == OR_ST_MAX_PATH) return INFINITY;
    return NAN;
}

static int32_t pf_type(const or_ray *r)
{
    if (r->n_refl > 0) return OR_SOL_REFLECTED;
    if (r->n_turn > 0) return OR_SOL_REFRACTED;
    return OR_SOL_DIRECT;
}

static void pf_fill(or_solution *s, const or_ray *r, double th, int32_t it, double miss)
{
    s->type = pf_type(r);
    s->n_iter = it;
    s->converged = 1;
    s->pad = 0;
    s->launch = th;
    s->receive = acos(fmax(-1.0, fmin(1.0, r->dir[2])));
    s->time = r->time;
    s->path = r->path;
    s->amp = r->amp;
    s->miss = miss;
}

int32_t or_find_paths(const or_medium *m, const or_params *p, int64_t n_pairs,
                      const double *zs, const double *zr, const double *dist,
                      const int32_t *n_angles, double hit_tol, int32_t max_iter,
                      int32_t max_sol, int32_t *count, or_solution *sol)
{
    const double pi = 3.14159265358979323846;
    for (int64_t i = 0; i < n_pairs; ++i) {
        or_params pp = *p;
        pp.max_generation = 0;
        pp.use_stop = 1;
        pp.max_path = 2.0 * (dist[i] + zs[i] + zr[i]) + 100.0;
        or_solution found[64];
        int32_t nf = 0;
        or_ray rec;
        if (dist[i] < hit_tol) {
            /* receiver straight above or below the source: the vertical direct ray */
            double th = (zr[i] >= zs[i]) ? 0.0 : pi;
            pp.stop_n[0] = 0.0;
            pp.stop_n[1] = 0.0;
            pp.stop_n[2] = 1.0;
            pp.stop_d = zr[i];
            pf_trace(m, &pp, zs[i], th, &rec);
            if (rec.status == OR_ST_REACHED_STOP) pf_fill(&found[nf++], &rec, th, 0, 0.0);
        } else {
            pp.stop_n[0] = 1.0;
            pp.stop_n[1] = 0.0;
            pp.stop_n[2] = 0.0;
            pp.stop_d = dist[i];
            int32_t na = n_angles[i] < 2 ? 2 : n_angles[i];
            double *miss = (double *)malloc((size_t)na * sizeof(double));
            for (int32_t j = 0; j < na; ++j) {
                double th = pi * (double)j / (double)(na - 1);
                pf_trace(m, &pp, zs[i], th, &rec);
                miss[j] = pf_miss(&rec, zr[i]);
            }
            for (int32_t j = 0; j + 1 < na && nf < 64; ++j) {
                double ma = miss[j], mb = miss[j + 1];
                if (isnan(ma) || isnan(mb)) continue;
                if (!((ma > 0.0 && mb < 0.0) || (ma < 0.0 && mb > 0.0))) continue;
                double tha = pi * (double)j / (double)(na - 1);
                double thb = pi * (double)(j + 1) / (double)(na - 1);
                for (int32_t it = 1; it <= max_iter; ++it) {
                    double thm = 0.5 * (tha + thb);
                    if (!(thm > tha && thm < thb)) break; /* bracket exhausted */
                    pf_trace(m, &pp, zs[i], thm, &rec);
                    double mm = pf_miss(&rec, zr[i]);
                    if (isnan(mm)) break;
                    if (fabs(mm) < hit_tol) {
                        pf_fill(&found[nf++], &rec, thm, it, mm);
                        break;
                    }
                    if ((mm > 0.0) == (ma > 0.0)) {
                        tha = thm;
                        ma = mm;
                    } else {
                        thb = thm;
                        mb = mm;
                    }
                }
            }
            free(miss);
        }
        /* sort by travel time (insertion sort) */
        for (int32_t a = 1; a < nf; ++a) {
            or_solution key = found[a];
            int32_t b = a - 1;
            while (b >= 0 && found[b].time > key.time) {
                found[b + 1] = found[b];
                --b;
            }
            found[b + 1] = key;
        }
        int32_t keep = nf < max_sol ? nf : max_sol;
        count[i] = keep;
        for (int32_t a = 0; a < max_sol; ++a) {
            or_solution *o = &sol[i * max_sol + a];
            if (a < keep) {
                *o = found[a];
            } else {
                memset(o, 0, sizeof *o);
            }
        }
    }
    return 0;
}
