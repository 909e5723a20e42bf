// trace_core.cuh -- device-side core of the ray tracer (sm_103a).
//
// One GPU thread owns one ray at a time.  Each loop iteration performs exactly one
// Cash-Karp step evaluation (the expensive, warp-uniform part) and then a short, divergent
// state-machine update:
//   NORMAL  : error control (accept / reject), event detection on the planes of the ray's
//             layer and on the stop plane, commit of the step
//   PROBE   : the step started on a plane; first evaluation at h_min
//   ILLINOIS: modified regula falsi on the step length until the step lands on the plane
// so that every lane keeps executing the same Runge-Kutta code whatever phase it is in.
//
// Method (Sec. 2 of the paper): ray equation Eq. 1 (projected form, default) or Eq. 2
// (paraxial form), Cash-Karp embedded RK4(5) with step control, the boundary module
// (reflection, Snell refraction, Fresnel amplitudes, secondary ray from the intersection
// point), receivers, break conditions (Fig. 1 text).
//
// Precision policies:
//   PrecF64 : everything in FP64.
//   PrecF32 : Runge-Kutta stages, medium evaluation and error control in FP32; position and
//             direction accumulated in float-float (hi + lo, ~48-bit significand) on the FP32
//             pipe; travel time and arc length accumulated in FP64.  Boundary splits are
//             rare and done in FP64 in both policies.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "rp.h"

namespace rpk {

constexpr double kC0 = 299792458.0;
constexpr double kInvC0 = 1.0 / 299792458.0;
constexpr int kRootMaxIter = 40;

// ---------------------------------------------------------------------------------------
// Cash-Karp (1990) embedded RK4(5) coefficients: nodes c_i, stage matrix a_ij, fifth-order
// weights b5_i (propagated) and fourth-order weights b4_i (error estimate only).
// Written as constexpr functions so that fully unrolled loops fold them into immediates.
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr double ck_a(int i, int j)
{
    return i == 1   ? (j == 0 ? 1.0 / 5.0 : 0.0)
           : i == 2 ? (j == 0 ? 3.0 / 40.0 : j == 1 ? 9.0 / 40.0 : 0.0)
           : i == 3 ? (j == 0 ? 3.0 / 10.0 : j == 1 ? -9.0 / 10.0 : j == 2 ? 6.0 / 5.0 : 0.0)
           : i == 4 ? (j == 0   ? -11.0 / 54.0
                       : j == 1 ? 5.0 / 2.0
                       : j == 2 ? -70.0 / 27.0
                       : j == 3 ? 35.0 / 27.0
                                : 0.0)
           : i == 5 ? (j == 0   ? 1631.0 / 55296.0
                       : j == 1 ? 175.0 / 512.0
                       : j == 2 ? 575.0 / 13824.0
                       : j == 3 ? 44275.0 / 110592.0
                       : j == 4 ? 253.0 / 4096.0
                                : 0.0)
                    : 0.0;
}
__host__ __device__ constexpr double ck_b5(int i)
{
    return i == 0 ? 37.0 / 378.0 : i == 2 ? 250.0 / 621.0 : i == 3 ? 125.0 / 594.0
           : i == 5 ? 512.0 / 1771.0 : 0.0;
}
__host__ __device__ constexpr double ck_b4(int i)
{
    return i == 0   ? 2825.0 / 27648.0
           : i == 2 ? 18575.0 / 48384.0
           : i == 3 ? 13525.0 / 55296.0
           : i == 4 ? 277.0 / 14336.0
           : i == 5 ? 1.0 / 4.0
                    : 0.0;
}
__host__ __device__ constexpr double ck_db(int i) { return ck_b5(i) - ck_b4(i); }

// ---------------------------------------------------------------------------------------
// float-float helpers (error-free transformations: Knuth TwoSum, FMA TwoProduct)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_add(float &hi, float &lo, float d)
{
    float s, e;
    two_sum(hi, d, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// Splits a double into a float-float pair (hi = x truncated to 24 significant bits, lo = the
// rest rounded to float; |x - hi - lo| <= 2^-47 |x|) with integer operations only: on GB300 a
// conversion on the FP64 pipe costs as much issue time as a whole Runge-Kutta stage.
__device__ __forceinline__ void split_d2ff(double x, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int e = (unsigned int)(b >> 52) & 0x7FFu;
    if ((b << 1) == 0ull) {  // +-0
        hi = __int_as_float((int)((unsigned int)(b >> 32) & 0x80000000u));
        lo = 0.0f;
        return;
    }
    if (e < 949u || e > 1100u) {  // |x| outside [2^-74, 2^78): rare, use the FP64 pipe
        hi = __double2float_rn(x);
        lo = __double2float_rn(x - (double)hi);
        return;
    }
    const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
    hi = __uint_as_float(sgn | ((e - 896u) << 23) | (unsigned int)((b >> 29) & 0x7FFFFFull));
    const unsigned int low29 = (unsigned int)(b & 0x1FFFFFFFull);
    const float scale = __uint_as_float((e - 948u) << 23);  // 2^(e - 1075)
    lo = __uint_as_float(__float_as_uint(__uint2float_rn(low29) * scale) | sgn);
}

// A plane offset (or any coordinate constant) in both precisions.
struct PlaneC {
    double d;
    float hi, lo;
};

__host__ __device__ __forceinline__ PlaneC plane_of(double d)
{
    PlaneC c;
    c.d = d;
    c.hi = (float)d;
    c.lo = (float)(d - (double)c.hi);
    return c;
}

// ---------------------------------------------------------------------------------------
// Precision policies
// ---------------------------------------------------------------------------------------
struct PrecF64 {
    typedef double R;
    struct V {
        double v[3];
    };
    static constexpr bool kFF = false;
    static constexpr int kMinBlocks = 2;  // blocks of 128 per SM the register budget targets
    __device__ static __forceinline__ R base(const V &a, int i) { return a.v[i]; }
    __device__ static __forceinline__ void add(V &a, int i, R d) { a.v[i] += d; }
    __device__ static __forceinline__ double get(const V &a, int i) { return a.v[i]; }
    __device__ static __forceinline__ void set(V &a, int i, double x) { a.v[i] = x; }
    // (a_i + delta) - c, evaluated in the order the FP64 reference uses
    __device__ static __forceinline__ R rel(const V &a, int i, R delta, const PlaneC &c)
    {
        return (a.v[i] + delta) - c.d;
    }
    __device__ static __forceinline__ void snap(V &a, int i, const PlaneC &c) { a.v[i] = c.d; }
    __device__ static __forceinline__ R from_d(double x) { return x; }
    __device__ static __forceinline__ R rcp(R x) { return 1.0 / x; }
    __device__ static __forceinline__ R exp_(R x) { return exp(x); }
    __device__ static __forceinline__ R sqrt_(R x) { return sqrt(x); }
    // the step-size factor of the step control (a heuristic: its last bits do not matter) in
    // single precision on the FP32 pipe and the special-function unit: a double pow costs
    // about as many FP64 instructions as a third of a Runge-Kutta step
    __device__ static __forceinline__ R pow_(R x, R y)
    {
        return (double)exp2f((float)y * __log2f((float)x));
    }
    __device__ static __forceinline__ R c(double x) { return x; }
    // scalar accumulators (travel time, arc length)
    typedef double S;
    __device__ static __forceinline__ double sget(const S &a) { return a; }
    __device__ static __forceinline__ void sset(S &a, double x) { a = x; }
    __device__ static __forceinline__ void sadd(S &a, R d) { a += d; }
    __device__ static __forceinline__ R sdiff(const S &a, const PlaneC &c) { return a - c.d; }
};

struct PrecF32 {
    typedef float R;
    struct V {
        float hi[3], lo[3];
    };
    static constexpr bool kFF = true;
    static constexpr int kMinBlocks = 4;
    __device__ static __forceinline__ R base(const V &a, int i) { return a.hi[i]; }
    __device__ static __forceinline__ void add(V &a, int i, R d) { ff_add(a.hi[i], a.lo[i], d); }
    __device__ static __forceinline__ double get(const V &a, int i)
    {
        return (double)a.hi[i] + (double)a.lo[i];
    }
    __device__ static __forceinline__ void set(V &a, int i, double x)
    {
        split_d2ff(x, a.hi[i], a.lo[i]);
    }
    __device__ static __forceinline__ R rel(const V &a, int i, R delta, const PlaneC &c)
    {
        // hi - c.hi is exact near the plane (Sterbenz); the small terms follow
        return __fadd_rn(__fadd_rn(__fsub_rn(a.hi[i], c.hi), delta), __fsub_rn(a.lo[i], c.lo));
    }
    __device__ static __forceinline__ void snap(V &a, int i, const PlaneC &c)
    {
        a.hi[i] = c.hi;
        a.lo[i] = c.lo;
    }
    __device__ static __forceinline__ R from_d(double x) { return __double2float_rn(x); }
    // 1/n of a stage (n in [1, 2]): the approximate reciprocal (within 2 ulp) instead of the
    // correctly rounded one saves several instructions per stage on the issue-bound step; the
    // FP32-mixed results against FP64 are unchanged at the 1 mm / 0.01 ns bar
    __device__ static __forceinline__ R rcp(R x) { return __fdividef(1.0f, x); }
    __device__ static __forceinline__ R exp_(R x) { return expf(x); }
    __device__ static __forceinline__ R sqrt_(R x) { return sqrtf(x); }
    __device__ static __forceinline__ R pow_(R x, R y) { return exp2f(y * __log2f(x)); }
    __device__ static __forceinline__ R c(double x) { return (float)x; }
    // scalar accumulators in float-float: GB300 issues FP64 at 1/64 of the FP32 rate, so the
    // per-step accumulation of travel time and arc length stays on the FP32 pipe
    struct S {
        float hi, lo;
    };
    __device__ static __forceinline__ double sget(const S &a) { return (double)a.hi + (double)a.lo; }
    __device__ static __forceinline__ void sset(S &a, double x) { split_d2ff(x, a.hi, a.lo); }
    __device__ static __forceinline__ void sadd(S &a, R d) { ff_add(a.hi, a.lo, d); }
    __device__ static __forceinline__ R sdiff(const S &a, const PlaneC &c)
    {
        return __fadd_rn(__fsub_rn(a.hi, c.hi), __fsub_rn(a.lo, c.lo));
    }
};

// ---------------------------------------------------------------------------------------
// Media
// ---------------------------------------------------------------------------------------
struct LayerC {
    double n0, dn, off, inv_z0, gcoef;  // n = n0 - dn e + off, dn/dz = gcoef e, e = exp(-z/z0)
    float n0f, dnf, offf, inv_z0f, gcoeff;
    int32_t absorb, has_exp;
};

// Regions of a layered medium: layer k (k < RP_MAX_LAYERS) outside every sphere, or the inside
// of sphere j, region RP_MAX_LAYERS + j; L[region] holds the region's index formula.
constexpr int kRegions = RP_MAX_LAYERS + RP_MAX_SPHERES;

struct MediumLayered {
    int32_t n_layers, pad;
    LayerC L[kRegions];
    PlaneC top[RP_MAX_LAYERS];  // top[k]: plane z = z_top of layer k (k >= 1)
    // index just above / below plane k (layer k-1 / layer k evaluated at z_top[k])
    double n_above[RP_MAX_LAYERS], n_below[RP_MAX_LAYERS];
    float n_above_f[RP_MAX_LAYERS], n_below_f[RP_MAX_LAYERS];
    // index ratios n1 / n2 for a ray crossing plane k downward and upward
    double eta_down[RP_MAX_LAYERS], eta_up[RP_MAX_LAYERS];
    // (dn/dz) / n just above / below plane k: the ray equation's curvature scale there
    float kap_above_f[RP_MAX_LAYERS], kap_below_f[RP_MAX_LAYERS];
};

struct MediumGrid {
    const float4 *__restrict__ g;  // (n, dn/dx, dn/dy, dn/dz) node samples, x fastest
    int32_t nx, ny, nz, pad;
    double org[3], inv_sp, hi[3];
    float orgf[3], inv_spf;
    PlaneC lo_c[3], hi_c[3];  // box faces
};

// Spherical boundary (curved boundaries, the paragraph after Fig. 1): centre, radius, and the
// same as float-float constants for the FP32 path.
struct SphereB {
    double c[3], R;
    PlaneC cc[3];
    float R2h, R2l, Rf, pad;
};

// A layered medium with spherical inclusions, each inside one layer, none overlapping.
struct MediumSpheres : MediumLayered {
    int32_t n_sph, pad2;
    SphereB S[RP_MAX_SPHERES];
};

// Non-horizontal layer boundary k (boundary shapes beyond the plane, the paragraph after
// Fig. 1): zb(x, y) = z_top + sx x + sy y + H(x, y), H the bilinear interpolant of nx x ny node
// heights h (x fastest; node (i, j) at (ox + i dx, oy + j dy)), held at its edge values beyond
// the nodes; h == nullptr: no height field.  on == 0: the horizontal plane z = z_top.
struct SurfB {
    const double *__restrict__ h;
    int32_t on, nx, ny, pad;
    double sx, sy, ox, oy, dx, dy;
    // the same in FP32 for the FP32-mixed event tests: the heights, the slopes as float-float
    // pairs, the node origin, spacing and its inverse
    const float *__restrict__ hf;
    float sxh, sxl, syh, syl, oxf, oyf, dxf, dyf, inv_dxf, inv_dyf;
};

// A layered medium whose inner boundaries may be tilted planes or height-field surfaces.
struct MediumSurfaces : MediumLayered {
    SurfB B[RP_MAX_LAYERS];
};

template <class M>
constexpr bool is_layered_v = std::is_base_of<MediumLayered, M>::value;
template <class M>
constexpr bool has_spheres_v = std::is_same<M, MediumSpheres>::value;
template <class M>
constexpr bool has_surfaces_v = std::is_same<M, MediumSurfaces>::value;

// Depth of boundary k at (x, y) and (gx, gy non-NULL) its slopes dzb/dx, dzb/dy, in FP64 with
// the FP64 reference's operations, unfused.
__device__ __forceinline__ double surf_depth(const MediumSurfaces &m, int k, double x, double y,
                                             double *gx, double *gy)
{
    const SurfB &B = m.B[k];
    double z = m.top[k].d, sx = 0.0, sy = 0.0;
    if (B.on) {
        z = __dadd_rn(z, __dadd_rn(__dmul_rn(B.sx, x), __dmul_rn(B.sy, y)));
        sx = B.sx;
        sy = B.sy;
        if (B.h) {
            const double u_raw = __ddiv_rn(__dsub_rn(x, B.ox), B.dx);
            const double v_raw = __ddiv_rn(__dsub_rn(y, B.oy), B.dy);
            const double u = fmin(fmax(u_raw, 0.0), (double)(B.nx - 1));
            const double v = fmin(fmax(v_raw, 0.0), (double)(B.ny - 1));
            int i = (int)floor(u), j = (int)floor(v);
            if (i > B.nx - 2) i = B.nx - 2;
            if (j > B.ny - 2) j = B.ny - 2;
            const double fu = __dsub_rn(u, (double)i), fv = __dsub_rn(v, (double)j);
            const double *r0 = B.h + (size_t)j * B.nx + i, *r1 = r0 + B.nx;
            const double h00 = r0[0], h10 = r0[1], h01 = r1[0], h11 = r1[1];
            const double gu = __dsub_rn(1.0, fu), gv = __dsub_rn(1.0, fv);
            if (gx) {
                *gx = (u_raw >= 0.0 && u_raw <= (double)(B.nx - 1))
                          ? __ddiv_rn(__dadd_rn(__dmul_rn(gv, __dsub_rn(h10, h00)),
                                                __dmul_rn(fv, __dsub_rn(h11, h01))), B.dx)
                          : 0.0;
                *gy = (v_raw >= 0.0 && v_raw <= (double)(B.ny - 1))
                          ? __ddiv_rn(__dadd_rn(__dmul_rn(gu, __dsub_rn(h01, h00)),
                                                __dmul_rn(fu, __dsub_rn(h11, h10))), B.dy)
                          : 0.0;
                sx = __dadd_rn(sx, *gx);
                sy = __dadd_rn(sy, *gy);
            }
            const double H = __dadd_rn(
                __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(gu, gv), h00), __dmul_rn(__dmul_rn(fu, gv), h10)),
                          __dmul_rn(__dmul_rn(gu, fv), h01)),
                __dmul_rn(__dmul_rn(fu, fv), h11));
            z = __dadd_rn(z, H);
        }
    }
    if (gx) {
        *gx = sx;
        *gy = sy;
    }
    return z;
}

// True if boundary k of the medium exists and is a tilted plane or height field.
__device__ __forceinline__ bool surf_on(const MediumSurfaces &m, int k)
{
    return k >= 1 && k < m.n_layers && m.B[k].on;
}

// Layer of the point r (FP64; once per ray): the last boundary at or above it.
__device__ __forceinline__ int layer_at(const MediumSurfaces &m, const double r[3])
{
    int k = 0;
    for (int j = 1; j < m.n_layers; ++j)
        if (r[2] >= surf_depth(m, j, r[0], r[1], nullptr, nullptr)) k = j;
    return k;
}

__device__ __forceinline__ int layer_of(const MediumLayered &m, double z)
{
    int k = 0;
    for (int j = 1; j < m.n_layers; ++j)
        if (z >= m.top[j].d) k = j;
    return k;
}

// The same for a depth held as float-float (z = hi + lo), on the FP32 pipe.
__device__ __forceinline__ int layer_of_ff(const MediumLayered &m, float hi, float lo)
{
    int k = 0;
    for (int j = 1; j < m.n_layers; ++j)
        if (__fadd_rn(__fsub_rn(hi, m.top[j].hi), __fsub_rn(lo, m.top[j].lo)) >= 0.0f) k = j;
    return k;
}

// Region containing r (FP64; once per ray): inside sphere j, else the layer of the depth.
__device__ __forceinline__ int region_of(const MediumSpheres &m, const double r[3])
{
    for (int j = 0; j < m.n_sph; ++j) {
        const SphereB &S = m.S[j];
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) d2 = __dadd_rn(d2, __dmul_rn(r[a] - S.c[a], r[a] - S.c[a]));
        if (d2 < __dmul_rn(S.R, S.R)) return RP_MAX_LAYERS + j;
    }
    return layer_of(m, r[2]);
}

// n(z) and dn/dz of layer k in FP64 (used by the boundary split in both policies).
__device__ __forceinline__ void layer_eval_d(const MediumLayered &m, int k, double z, double &n,
                                             double &dndz)
{
    const LayerC &L = m.L[k];
    if (!L.has_exp) {
        n = L.n0 + L.off;
        dndz = 0.0;
        return;
    }
    double e = exp(-z * L.inv_z0);
    n = L.n0 - L.dn * e + L.off;
    dndz = L.gcoef * e;
}

// The constants of the layer a ray travels in and of the two planes bounding it, held in
// registers for the ray's whole life (a ray never changes layer: crossing a plane casts a
// secondary in the other layer).  Lanes of a warp in different layers then never read the
// medium description with divergent indices in the per-step loop.
template <class P>
struct LayerR {
    typename P::R n0, mdn, off, minv, gcoef;  // n = n0 + mdn e + off, dn/dz = gcoef e,
                                              // e = exp(minv z); constant layer: mdn = minv = 0
    PlaneC top, bot;                          // planes above / below (+-1e30 when absent)
};

template <class P>
__device__ __forceinline__ void load_layer(LayerR<P> &c, const MediumLayered &m, int k)
{
    const LayerC &L = m.L[k];
    if constexpr (P::kFF) {
        c.n0 = L.n0f;
        c.mdn = L.has_exp ? -L.dnf : 0.0f;
        c.off = L.offf;
        c.minv = L.has_exp ? -L.inv_z0f : 0.0f;
        c.gcoef = L.has_exp ? L.gcoeff : 0.0f;
    } else {
        c.n0 = L.n0;
        c.mdn = L.has_exp ? -L.dn : 0.0;
        c.off = L.off;
        c.minv = L.has_exp ? -L.inv_z0 : 0.0;
        c.gcoef = L.has_exp ? L.gcoef : 0.0;
    }
    PlaneC none_top, none_bot;
    none_top.d = -1e30;
    none_top.hi = -1e30f;
    none_top.lo = 0.0f;
    none_bot.d = 1e30;
    none_bot.hi = 1e30f;
    none_bot.lo = 0.0f;
    // a sphere's inside (k >= RP_MAX_LAYERS) has no planes: the ray meets its sphere first
    c.top = (k > 0 && k < RP_MAX_LAYERS) ? m.top[k] : none_top;
    c.bot = k + 1 < m.n_layers ? m.top[k + 1] : none_bot;
}
template <class P>
__device__ __forceinline__ void load_layer(LayerR<P> &, const MediumGrid &, int)
{
}

// Layered analytic medium: only the stage depth matters.
template <class P>
__device__ __forceinline__ void medium_eval(const MediumLayered &, const LayerR<P> &c,
                                            const typename P::R r[3], typename P::R &n,
                                            typename P::R g[3])
{
    typedef typename P::R R;
    g[0] = R(0);
    g[1] = R(0);
    if constexpr (P::kFF) {
        const float e = expf(r[2] * c.minv);
        n = __fadd_rn(__fmaf_rn(c.mdn, e, c.n0), c.off);
        g[2] = c.gcoef * e;
    } else {
        const double e = exp(r[2] * c.minv);
        n = c.n0 + c.mdn * e + c.off;
        g[2] = c.gcoef * e;
    }
}

// Gridded medium: trilinear interpolation of the four FP32 node channels, clamped to the box.
template <class P>
__device__ __forceinline__ void medium_eval(const MediumGrid &m, const LayerR<P> &,
                                            const typename P::R r[3], typename P::R &n,
                                            typename P::R g[3])
{
    typedef typename P::R R;
    const int dims[3] = {m.nx, m.ny, m.nz};
    int idx[3];
    R w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R f;
        if constexpr (P::kFF)
            f = (r[a] - m.orgf[a]) * m.inv_spf;
        else
            f = (r[a] - m.org[a]) * m.inv_sp;
        const R top = R(dims[a] - 1);
        f = fmax(f, R(0));  // also maps NaN to 0: the index below always stays in the box
        f = fmin(f, top);
        int i = (int)floor(f);
        if (i < 0) i = 0;
        if (i > dims[a] - 2) i = dims[a] - 2;
        idx[a] = i;
        w[a] = f - R(i);
    }
    const size_t sx = 1, sy = (size_t)m.nx, sz = (size_t)m.nx * (size_t)m.ny;
    const size_t b = (size_t)idx[2] * sz + (size_t)idx[1] * sy + (size_t)idx[0];
    float4 c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const size_t o = b + ((q >> 2) & 1) * sz + ((q >> 1) & 1) * sy + (q & 1) * sx;
        c[q] = __ldg(&m.g[o]);
    }
    R v[4];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        R e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // q = 2 dz + dy
            float a0 = ch == 0 ? c[2 * q].x : ch == 1 ? c[2 * q].y : ch == 2 ? c[2 * q].z : c[2 * q].w;
            float a1 = ch == 0   ? c[2 * q + 1].x
                       : ch == 1 ? c[2 * q + 1].y
                       : ch == 2 ? c[2 * q + 1].z
                                 : c[2 * q + 1].w;
            e[q] = R(a0) + w[0] * (R(a1) - R(a0));
        }
        R f0 = e[0] + w[1] * (e[1] - e[0]);
        R f1 = e[2] + w[1] * (e[3] - e[2]);
        v[ch] = f0 + w[2] * (f1 - f0);
    }
    n = v[0];
    g[0] = v[1];
    g[1] = v[2];
    g[2] = v[3];
}

// ---------------------------------------------------------------------------------------
// One Cash-Karp step of the ray system from (r0, t0) with step h.
//   y = (r, t, T);  r' = t;  t' = (g - (g.t) t)/n  [projected]  or  g/n  [paraxial];
//   T' = n / c0.
// Outputs the fifth-order increments dr, dt, dT and the error measures
//   er = |sum_i (b5_i - b4_i) k_r,i|,   et = h |sum_i (b5_i - b4_i) k_t,i|.
// Sums run over the stages in ascending order, as in the FP64 reference.
// ---------------------------------------------------------------------------------------
// Cash-Karp step of Eq. 1 as written, d/ds (n t) = grad n, on the state (r, p = n t, T):
// r' = p / |p|, p' = grad n, T' = n / c0 (FP64 only: a cross-check of the projected form).
// The stages run on p from p0 = n(r0) t0 (n(r0) is stage 0's index); the direction increment
// is p5 / |p5| - t0 and the direction error h |sum (b5 - b4) k_p| / n(r0).
template <class P, class M>
__device__ __forceinline__ void ck_step_momentum(const M &med, const LayerR<P> &lc,
                                                 const typename P::V &r0, const typename P::V &t0v,
                                                 double h, double dr[3], double dt[3],
                                                 double &dT, double &er, double &et)
{
    double p0[3] = {0.0, 0.0, 0.0}, kr[6][3], kp[6][3], n0 = 1.0;
    double sr[3] = {0.0, 0.0, 0.0}, sp_[3] = {0.0, 0.0, 0.0}, sT = 0.0;
    double dr_e[3] = {0.0, 0.0, 0.0}, dp_e[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double rs[3], ps[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double ar = 0.0, ap = 0.0;
#pragma unroll
            for (int j = 0; j < i; ++j) {
                ar += ck_a(i, j) * kr[j][c];
                ap += ck_a(i, j) * kp[j][c];
            }
            rs[c] = P::get(r0, c) + h * ar;
            ps[c] = p0[c] + h * ap;
        }
        double n, g[3];
        medium_eval<P>(med, lc, rs, n, g);
        if (i == 0) {
            n0 = n;
#pragma unroll
            for (int c = 0; c < 3; ++c) ps[c] = p0[c] = n0 * P::get(t0v, c);
        }
        const double q = sqrt(ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            kr[i][c] = ps[c] / q;
            kp[i][c] = g[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sr[c] += ck_b5(i) * kr[i][c];
            sp_[c] += ck_b5(i) * kp[i][c];
            dr_e[c] += ck_db(i) * kr[i][c];
            dp_e[c] += ck_db(i) * kp[i][c];
        }
        sT += ck_b5(i) * n;
    }
    double p5[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dr[c] = h * sr[c];
        p5[c] = p0[c] + h * sp_[c];
    }
    const double q5 = sqrt(p5[0] * p5[0] + p5[1] * p5[1] + p5[2] * p5[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) dt[c] = p5[c] / q5 - P::get(t0v, c);
    dT = h * (sT * kInvC0);
    er = sqrt(dr_e[0] * dr_e[0] + dr_e[1] * dr_e[1] + dr_e[2] * dr_e[2]);
    et = h * sqrt(dp_e[0] * dp_e[0] + dp_e[1] * dp_e[1] + dp_e[2] * dp_e[2]) / n0;
}

// Cash-Karp step for stratified media (planes and spheres whose regions have z-only index
// profiles), where grad n = (0, 0, g), in both precisions.  The horizontal direction components
// then obey the same linear equation, t_c' = kap t_c with kap = -(g t_z / n) (projected form;
// 0 for the paraxial one), so every stage's horizontal components are the step's start
// values times one common factor, t_c,i = t0_c phi_i with phi_i = 1 + h sum_j a_ij kap_j, and
// their slopes are t0_c kap_i.  The stages carry the scalars (phi, kap, t_z, t_z') instead of
// two more vector components: the same Runge-Kutta step in exact arithmetic, with fewer
// operations and registers (in FP64 its results differ from the general form's by rounding
// only).  The error measures are returned as ck_step returns them: squared in FP32-mixed mode.
template <class P, class M>
__device__ __forceinline__ void ck_step_vgrad(const M &med, const LayerR<P> &lc, int form,
                                              const typename P::V &r0, const typename P::V &t0v,
                                              typename P::R h, typename P::R dr[3],
                                              typename P::R dt[3], typename P::R &dT,
                                              typename P::R &er, typename P::R &et)
{
    typedef typename P::R R;
    const R tx = P::base(t0v, 0), ty = P::base(t0v, 1), tz0 = P::base(t0v, 2);
    R kap[6], tz[6], ktz[6];
    R s_phi = R(0), s_kap = R(0), s_tz = R(0), s_ktz = R(0), sT = R(0);
    R e_phi = R(0), e_kap = R(0), e_tz = R(0), e_ktz = R(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        R a_kap = R(0), a_tz = R(0), a_ktz = R(0);
#pragma unroll
        for (int j = 0; j < i; ++j) {
            a_kap += P::c(ck_a(i, j)) * kap[j];
            a_tz += P::c(ck_a(i, j)) * tz[j];
            a_ktz += P::c(ck_a(i, j)) * ktz[j];
        }
        const R phi = R(1) + h * a_kap;
        tz[i] = tz0 + h * a_ktz;
        const R rs[3] = {R(0), R(0), P::base(r0, 2) + h * a_tz};
        R n, g[3];
        medium_eval<P>(med, lc, rs, n, g);
        const R inv_n = P::rcp(n);
        if (form == RP_RHS_PROJECTED) {
            const R gt = g[2] * tz[i];
            kap[i] = -(gt * phi) * inv_n;
            ktz[i] = (g[2] - gt * tz[i]) * inv_n;
        } else {
            kap[i] = R(0);
            ktz[i] = g[2] * inv_n;
        }
        if (ck_b5(i) != 0.0) {
            s_phi += P::c(ck_b5(i)) * phi;
            s_kap += P::c(ck_b5(i)) * kap[i];
            s_tz += P::c(ck_b5(i)) * tz[i];
            s_ktz += P::c(ck_b5(i)) * ktz[i];
            sT += P::c(ck_b5(i)) * n;
        }
        if (ck_db(i) != 0.0) {
            e_phi += P::c(ck_db(i)) * phi;
            e_kap += P::c(ck_db(i)) * kap[i];
            e_tz += P::c(ck_db(i)) * tz[i];
            e_ktz += P::c(ck_db(i)) * ktz[i];
        }
    }
    const R hphi = h * s_phi, hkap = h * s_kap;
    dr[0] = tx * hphi;
    dr[1] = ty * hphi;
    dr[2] = h * s_tz;
    dt[0] = tx * hkap;
    dt[1] = ty * hkap;
    dt[2] = h * s_ktz;
    if constexpr (P::kFF) {
        // the stages used the high word of the direction; since sum_i b5_i = 1 its low word
        // contributes exactly h * t_lo to the position increment
#pragma unroll
        for (int c = 0; c < 3; ++c) dr[c] = __fmaf_rn(h, t0v.lo[c], dr[c]);
    }
    dT = h * (sT * P::c(kInvC0));
    const R th2 = tx * tx + ty * ty;
    if constexpr (P::kFF) {
        // squared error measures, as ck_step returns them in FP32-mixed mode
        er = th2 * (e_phi * e_phi) + e_tz * e_tz;
        et = (h * h) * (th2 * (e_kap * e_kap) + e_ktz * e_ktz);
    } else {
        er = P::sqrt_(th2 * (e_phi * e_phi) + e_tz * e_tz);
        et = h * P::sqrt_(th2 * (e_kap * e_kap) + e_ktz * e_ktz);
    }
}

template <class P, class M>
__device__ __forceinline__ void ck_step(const M &med, const LayerR<P> &lc, int form,
                                        const typename P::V &r0, const typename P::V &t0v,
                                        typename P::R h, typename P::R dr[3],
                                        typename P::R dt[3], typename P::R &dT,
                                        typename P::R &er, typename P::R &et)
{
    typedef typename P::R R;
    if constexpr (!P::kFF) {
        if (form == RP_RHS_MOMENTUM) {
            ck_step_momentum<P, M>(med, lc, r0, t0v, h, dr, dt, dT, er, et);
            return;
        }
    }
    if constexpr (is_layered_v<M>) {
        ck_step_vgrad<P, M>(med, lc, form, r0, t0v, h, dr, dt, dT, er, et);
        return;
    }
    R t0[3] = {P::base(t0v, 0), P::base(t0v, 1), P::base(t0v, 2)};
    R ts[6][3], kt[6][3];
    R sr[3] = {R(0), R(0), R(0)}, st[3] = {R(0), R(0), R(0)}, sT = R(0);
    R dr_e[3] = {R(0), R(0), R(0)}, dt_e[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        R rs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R ar = R(0), at = R(0);
#pragma unroll
            for (int j = 0; j < i; ++j) {
                ar += P::c(ck_a(i, j)) * ts[j][c];
                at += P::c(ck_a(i, j)) * kt[j][c];
            }
            rs[c] = P::base(r0, c) + h * ar;
            ts[i][c] = t0[c] + h * at;
        }
        R n, g[3];
        medium_eval<P>(med, lc, rs, n, g);
        R inv_n = P::rcp(n);
        if constexpr (is_layered_v<M>) {
            // stratified medium: grad n = (0, 0, g_z); the zero terms are dropped
            if (form == RP_RHS_PROJECTED) {
                const R gt = g[2] * ts[i][2];
                kt[i][0] = -(gt * ts[i][0]) * inv_n;
                kt[i][1] = -(gt * ts[i][1]) * inv_n;
                kt[i][2] = (g[2] - gt * ts[i][2]) * inv_n;
            } else {
                kt[i][0] = R(0);
                kt[i][1] = R(0);
                kt[i][2] = g[2] * inv_n;
            }
        } else if (form == RP_RHS_PROJECTED) {
            R gt = g[0] * ts[i][0] + g[1] * ts[i][1] + g[2] * ts[i][2];
#pragma unroll
            for (int c = 0; c < 3; ++c) kt[i][c] = (g[c] - gt * ts[i][c]) * inv_n;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) kt[i][c] = g[c] * inv_n;
        }
        if (ck_b5(i) != 0.0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sr[c] += P::c(ck_b5(i)) * ts[i][c];
                st[c] += P::c(ck_b5(i)) * kt[i][c];
            }
            sT += P::c(ck_b5(i)) * n;
        }
        if (ck_db(i) != 0.0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dr_e[c] += P::c(ck_db(i)) * ts[i][c];
                dt_e[c] += P::c(ck_db(i)) * kt[i][c];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dr[c] = h * sr[c];
        dt[c] = h * st[c];
    }
    if constexpr (P::kFF) {
        // the stages used the high word of the direction; since sum_i b5_i = 1 its low word
        // contributes exactly h * t_lo to the position increment
#pragma unroll
        for (int c = 0; c < 3; ++c) dr[c] = __fmaf_rn(h, t0v.lo[c], dr[c]);
    }
    dT = h * (sT * P::c(kInvC0));
    if constexpr (P::kFF) {
        // FP32-mixed: squared norms (the step control compares and scales squares, sparing two
        // square roots per step)
        er = dr_e[0] * dr_e[0] + dr_e[1] * dr_e[1] + dr_e[2] * dr_e[2];
        et = (h * h) * (dt_e[0] * dt_e[0] + dt_e[1] * dt_e[1] + dt_e[2] * dt_e[2]);
    } else {
        er = P::sqrt_(dr_e[0] * dr_e[0] + dr_e[1] * dr_e[1] + dr_e[2] * dr_e[2]);
        et = h * P::sqrt_(dt_e[0] * dt_e[0] + dt_e[1] * dt_e[1] + dt_e[2] * dt_e[2]);
    }
}

// ---------------------------------------------------------------------------------------
// Boundary module in FP64 (Sec. 2): reflection, Snell refraction, Fresnel amplitudes.
// nrm points toward the incident side.  Returns tir.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void normalise3(double v[3])
{
    double q = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= q;
    v[1] /= q;
    v[2] /= q;
}

__device__ __forceinline__ bool split_dirs(const double t[3], const double nrm[3], double n1,
                                           double n2, int pol, double t_refl[3],
                                           double t_refr[3], double &r, double &tau)
{
    double cos_i = -(t[0] * nrm[0] + t[1] * nrm[1] + t[2] * nrm[2]);
    if (cos_i < 0.0) cos_i = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) t_refl[a] = t[a] + 2.0 * cos_i * nrm[a];
    normalise3(t_refl);
    double eta = n1 / n2;
    double sin2_t = eta * eta * (1.0 - cos_i * cos_i);
    if (sin2_t > 1.0) {
        r = 1.0;  // total internal reflection: |r| = 1, phase not tracked
        tau = 0.0;
        return true;
    }
    double cos_t = sqrt(1.0 - sin2_t);
#pragma unroll
    for (int a = 0; a < 3; ++a) t_refr[a] = eta * t[a] + (eta * cos_i - cos_t) * nrm[a];
    normalise3(t_refr);
    double rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
    double ts = 2.0 * n1 * cos_i / (n1 * cos_i + n2 * cos_t);
    double rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);
    double tp = 2.0 * n1 * cos_i / (n2 * cos_i + n1 * cos_t);
    if (pol == RP_POL_S) {
        r = rs;
        tau = ts;
    } else if (pol == RP_POL_P) {
        r = rp;
        tau = tp;
    } else {
        double Rr = 0.5 * (rs * rs + rp * rp);
        r = sqrt(Rr);
        tau = sqrt(1.0 - Rr);
    }
    return false;
}

// ---------------------------------------------------------------------------------------
// Receivers: spheres binned in a uniform cell grid (see Receivers); a chord is tested against
// the spheres listed in the cell of its midpoint.
// ---------------------------------------------------------------------------------------
struct SphereC {
    PlaneC c[3];
    double R;
    float Rf;
    int32_t idx;
};

// Receivers are binned in a uniform grid of cells; every sphere is listed in each cell that
// its centre box, inflated by R + h_max / 2 (+ rounding pad), overlaps.  A step chord is no
// longer than h_max, so a sphere it meets has its centre within R + h_max / 2 of the chord's
// midpoint: the midpoint's cell lists every candidate, usually none.
struct Receivers {
    const SphereC *__restrict__ s;
    const int2 *__restrict__ cell;  // [begin, end) into items, per cell (x fastest)
    const int *__restrict__ items;  // sphere indices
    int32_t n, nx, ny, nz;
    float org[3], inv_cell;
    float hi[3];                    // far corner of the grid
};

// ---------------------------------------------------------------------------------------
// Per-call device control block (counters live in device memory, zeroed per call)
// ---------------------------------------------------------------------------------------
struct Ctrl {
    unsigned long long claim[RP_MAX_LAYERS + 8];
    unsigned long long seg_begin[RP_MAX_LAYERS + 8], seg_end[RP_MAX_LAYERS + 8];
    unsigned long long out_count, q_tail, n_hits, n_secondary;
    unsigned long long steps_acc, steps_rej, steps_root;
    unsigned int flags, pad;
};

enum { FLAG_BAD_INPUT = 1, FLAG_OUT_OVERFLOW = 2, FLAG_QUEUE_OVERFLOW = 4,
       FLAG_HIT_OVERFLOW = 8, FLAG_ROOT_CAP = 16 };

// Queued secondary ray (start state).
struct QRec {
    double r[3], t[3];
    double T, s, A, A0;
    double h;
    long long id, parent;
    int32_t layer, gen, seq;
    int32_t status;  // RP_ST_ALIVE: to be traced; otherwise a finished record to write out
};

// ---------------------------------------------------------------------------------------
// Lane state
// ---------------------------------------------------------------------------------------
enum { MODE_NORMAL = 0, MODE_PROBE = 1, MODE_ILLINOIS = 2 };
enum { EV_NONE = 0, EV_TOP = 1, EV_BOTTOM = 2, EV_STOP = 3, EV_SPH = 4 };  // EV_SPH + j: sphere j

template <class P>
struct Lane {
    typedef typename P::R R;
    typename P::V r, t;
    typename P::S T, s;  // travel time, arc length
    double A, A0;
    R h, h_next, h_try;
    R ra, rb, ga, gb;  // root bracket
    PlaneC stop;       // stop plane offset along stop_axis
    R stop_sign;       // orientation: the event distance is stop_sign * (r[axis] - offset)
    PlaneC mp;         // path budget of this ray (max_path)
    int32_t stop_axis;
    long long id, parent;
    int32_t mode, ev, side, it, last;
    int32_t layer, gen, seq;
    int32_t n_acc, n_rej, n_root, n_refl, n_turn, root_fail;
    int32_t status;
    int32_t stk;   // entries on this thread's private stack of pending secondaries
    int32_t pend;  // boundary event waiting for its split (EV_TOP / EV_BOTTOM), else 0
    int32_t tail;  // the launch's input was exhausted when this ray started: secondaries go
                   // to the global queue, spreading the last chains over the next launch
    LayerR<P> lc;  // the ray's layer and its bounding planes
};

// Parameters shared by every lane of a launch.
template <class P>
struct StepParams {
    typedef typename P::R R;
    R tol, inv_tol, inv_tol2, h_min, h_max, eps_b;  // inv_tol2 = 1/tol^2, capped at 1e30
    double max_path, max_time, min_amp;
    PlaneC mp, mt;  // max_path and max_time as float-float constants
    int32_t use_max_time, use_min_amp;
    int32_t rhs_form, polarization, max_generation, use_stop;
    int32_t stop_axis;  // 0, 1, 2 (the stop normal is +/- a coordinate axis)
    float stop_dir;     // +1 or -1: sign of the normal along stop_axis
    long long max_steps;
    unsigned int service_idle;      // idle lane-iterations that trigger a service phase
    int32_t flush_min;              // stack records left that a thread hands to the queue
                                    // once the wave's input has run out
};

// Offset of the candidate r + dr from the stop plane along the stop axis (selected without
// dynamic indexing so that the state stays in registers).
template <class P>
__device__ __forceinline__ typename P::R stop_rel(const Lane<P> &L, const StepParams<P> &,
                                                  const typename P::R dr[3])
{
    return L.stop_axis == 0   ? P::rel(L.r, 0, dr[0], L.stop)
           : L.stop_axis == 1 ? P::rel(L.r, 1, dr[1], L.stop)
                              : P::rel(L.r, 2, dr[2], L.stop);
}

template <class P>
__device__ __forceinline__ void set_trial(Lane<P> &L, const StepParams<P> &sp)
{
    typedef typename P::R R;
    L.last = 0;
    if constexpr (P::kFF) {
        const R rem = -P::sdiff(L.s, L.mp);  // max_path - s
        if (L.h >= rem) {
            L.h_try = rem;
            L.last = 1;
        } else {
            L.h_try = L.h;
        }
    } else {
        if (L.s + L.h >= L.mp.d) {
            L.h_try = L.mp.d - L.s;
            L.last = 1;
        } else {
            L.h_try = L.h;
        }
    }
    L.mode = MODE_NORMAL;
}

// Signed distance to an event plane for the candidate state r + dr (positive on the ray's
// own side).
template <class P>
__device__ __forceinline__ typename P::R event_g(const MediumLayered &m, const Lane<P> &L,
                                                 const StepParams<P> &sp, int kind,
                                                 const typename P::R dr[3])
{
    typedef typename P::R R;
    if (kind == EV_TOP) return P::rel(L.r, 2, dr[2], L.lc.top);
    if (kind == EV_BOTTOM) return -P::rel(L.r, 2, dr[2], L.lc.bot);
    return L.stop_sign * stop_rel(L, sp, dr);
}
template <class P>
__device__ __forceinline__ typename P::R event_g(const MediumGrid &, const Lane<P> &L,
                                                 const StepParams<P> &sp, int,
                                                 const typename P::R dr[3])
{
    return L.stop_sign * stop_rel(L, sp, dr);
}

// Distance |r + dr - c| - R of a candidate point from sphere S's surface.  FP64: the operations
// of the FP64 reference, unfused.  FP32-mixed: |w|^2 accumulated in float-float from the
// float-float position (w = r - c + dr with the rounding of r.hi - c.hi kept), then
// (|w|^2 - R^2) / (|w| + R), accurate to a few ulps of the distance itself.
template <class P>
__device__ __forceinline__ typename P::R sphere_dist(const typename P::V &r,
                                                     const typename P::R dr[3], const SphereB &S)
{
    if constexpr (!P::kFF) {
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double w = __dsub_rn(__dadd_rn(r.v[a], dr[a]), S.c[a]);
            d2 = __dadd_rn(d2, __dmul_rn(w, w));
        }
        return __dsub_rn(sqrt(d2), S.R);
    } else {
        float sh = 0.0f, sl = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float d0, e0;
            two_sum(r.hi[a], -S.cc[a].hi, d0, e0);
            const float wl0 = __fadd_rn(__fadd_rn(__fsub_rn(r.lo[a], S.cc[a].lo), dr[a]), e0);
            float wh, wl;
            two_sum(d0, wl0, wh, wl);
            const float p = __fmul_rn(wh, wh);
            const float pe = __fmaf_rn(wh, wh, -p);
            float s1, e1;
            two_sum(sh, p, s1, e1);
            sh = s1;
            sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(e1, pe), __fmul_rn(2.0f * wh, wl)));
        }
        const float g2 = __fadd_rn(__fsub_rn(sh, S.R2h), __fsub_rn(sl, S.R2l));
        return g2 / __fadd_rn(sqrtf(sh), S.Rf);
    }
}

// Signed distance to an event surface of a medium with spheres: the sphere's surface,
// positive on the ray's own side (outside, or inside its own sphere), or a plane as above.
template <class P>
__device__ __forceinline__ typename P::R event_g(const MediumSpheres &m, const Lane<P> &L,
                                                 const StepParams<P> &sp, int kind,
                                                 const typename P::R dr[3])
{
    if (kind >= EV_SPH) {
        const int j = kind - EV_SPH;
        const typename P::R g = sphere_dist<P>(L.r, dr, m.S[j]);
        return (L.layer == RP_MAX_LAYERS + j) ? -g : g;
    }
    return event_g<P>(static_cast<const MediumLayered &>(m), L, sp, kind, dr);
}

// Bilinear height field of SurfB B at the point x = xh + xl, y = yh + yl (float-float), in FP32:
// the cell is found from the point's offset from the node origin, and the offset within the
// cell is formed exactly (TwoSum, FMA residual) before it is scaled, so that the interpolation
// weights are accurate to ~1e-7 of a cell whatever the distance from the origin; held at the
// edge values beyond the nodes, as the FP64 form.
__device__ __forceinline__ float cell_coord(float ph, float pl, float o, float d, float inv_d,
                                            int n, int &i)
{
    float a, e;
    two_sum(ph, -o, a, e);
    e += pl;
    const float u = (a + e) * inv_d;
    if (!(u > 0.0f)) {  // below the first node (or NaN): the edge value
        i = 0;
        return 0.0f;
    }
    if (u >= (float)(n - 1)) {
        i = n - 2;
        return 1.0f;
    }
    i = min((int)floorf(u), n - 2);
    const float c = (float)i * d, ce = fmaf((float)i, d, -c);  // i d = c + ce exactly
    const float f = (((a - c) - ce) + e) * inv_d;
    return fminf(fmaxf(f, 0.0f), 1.0f);
}

__device__ __forceinline__ float height_ff(const SurfB &B, float xh, float xl, float yh, float yl)
{
    int i, j;
    const float fu = cell_coord(xh, xl, B.oxf, B.dxf, B.inv_dxf, B.nx, i);
    const float fv = cell_coord(yh, yl, B.oyf, B.dyf, B.inv_dyf, B.ny, j);
    const float *r0 = B.hf + (size_t)j * B.nx + i, *r1 = r0 + B.nx;
    const float gu = 1.0f - fu, gv = 1.0f - fv;
    return gv * (gu * __ldg(r0) + fu * __ldg(r0 + 1)) + fv * (gu * __ldg(r1) + fu * __ldg(r1 + 1));
}

// Vertical offset z - zb(x, y) of the candidate point r + dr from boundary k, for the
// FP32-mixed policy: float-float arithmetic on the FP32 pipe (TwoSum for the large terms
// z - z_top - s_x x - s_y y, which nearly cancel near the surface; FMA residuals of the slope
// products), the height field in FP32 relative to its cell.
__device__ __forceinline__ float surf_offset_ff(const MediumSurfaces &m, int k,
                                                const PrecF32::V &r, const float dr[3])
{
    const SurfB &B = m.B[k];
    const PlaneC &zt = m.top[k];
    float s, e, p, pe, s2, e2;
    two_sum(r.hi[2], -zt.hi, s, e);
    float small = e + (r.lo[2] - zt.lo) + dr[2];
    p = B.sxh * r.hi[0];
    pe = fmaf(B.sxh, r.hi[0], -p);
    two_sum(s, -p, s2, e2);
    small += e2 - pe - (B.sxh * (r.lo[0] + dr[0]) + B.sxl * r.hi[0]);
    p = B.syh * r.hi[1];
    pe = fmaf(B.syh, r.hi[1], -p);
    two_sum(s2, -p, s, e);
    small += e - pe - (B.syh * (r.lo[1] + dr[1]) + B.syl * r.hi[1]);
    float g = s + small;
    if (B.hf) g -= height_ff(B, r.hi[0], r.lo[0] + dr[0], r.hi[1], r.lo[1] + dr[1]);
    return g;
}

// Signed vertical offset from a layer boundary of a medium with surfaces, positive on the
// ray's own side (z - zb below the boundary, zb - z above it), for the candidate r + dr: in
// FP64 with the FP64 reference's operations (FP64 policy), in float-float on the FP32 pipe
// (FP32-mixed policy); horizontal planes keep the plane form.
template <class P>
__device__ __forceinline__ typename P::R event_g(const MediumSurfaces &m, const Lane<P> &L,
                                                 const StepParams<P> &sp, int kind,
                                                 const typename P::R dr[3])
{
    if (kind == EV_TOP || kind == EV_BOTTOM) {
        const int k = (kind == EV_TOP) ? L.layer : L.layer + 1;
        if (surf_on(m, k)) {
            if constexpr (P::kFF) {
                const float g = surf_offset_ff(m, k, L.r, dr);
                return (kind == EV_TOP) ? g : -g;
            } else {
                const double x = P::get(L.r, 0) + (double)dr[0];
                const double y = P::get(L.r, 1) + (double)dr[1];
                const double z = P::get(L.r, 2) + (double)dr[2];
                const double zb = surf_depth(m, k, x, y, nullptr, nullptr);
                return (typename P::R)((kind == EV_TOP) ? __dsub_rn(z, zb) : __dsub_rn(zb, z));
            }
        }
    }
    return event_g<P>(static_cast<const MediumLayered &>(m), L, sp, kind, dr);
}

__device__ __forceinline__ bool is_layered(const MediumLayered &) { return true; }
__device__ __forceinline__ bool is_layered(const MediumGrid &) { return false; }
__device__ __forceinline__ int n_layers(const MediumLayered &m) { return m.n_layers; }
__device__ __forceinline__ int n_layers(const MediumGrid &) { return 1; }

// Stop-plane side sign at the start of a ray: positive side is where the ray starts.
template <class P>
__device__ __forceinline__ void init_stop(Lane<P> &L, const StepParams<P> &sp)
{
    typedef typename P::R R;
    if (sp.use_stop) {
        // the start side counts as positive; f = n . r - d with n = stop_dir along the axis
        const R zero[3] = {R(0), R(0), R(0)};
        const R f = R(sp.stop_dir) * stop_rel(L, sp, zero);
        L.stop_sign = ((f <= R(0)) ? R(-1) : R(1)) * R(sp.stop_dir);
    } else {
        L.stop_sign = R(1);
    }
}

// Hooks the kernels provide: where a secondary goes and what a receiver hit writes.
constexpr int kStackDepth = 8;  // secondaries a thread keeps for itself before spilling
                                // (the fixed-scratch entry point may use fewer)

struct Sinks {
    Ctrl *ctrl;
    QRec *queue;
    unsigned long long q_cap;
    QRec *stack;  // stack_depth records per thread of the launch
    int32_t stack_depth;
    unsigned long long *warp_clock;  // per warp of wave 0: start and end (globaltimer, ns)
    // output arrays for rays recorded directly (transmitted into absorbing layers)
    rp_ray_out out;
    // hits
    rp_hits hits;
    Receivers rx;
    int32_t has_rx;
};

// Writes one finished ray record.
template <class P>
__device__ __forceinline__ void write_ray(const rp_ray_out &o, long long id, const Lane<P> &L,
                                          Ctrl *ctrl)
{
    if (id >= o.capacity) {
        atomicOr(&ctrl->flags, (unsigned)FLAG_OUT_OVERFLOW);
        return;
    }
    const long long cap = o.capacity;
#pragma unroll
    for (int a = 0; a < 3; ++a) o.end_pos[a * cap + id] = P::get(L.r, a);
    if (o.end_dir) {
#pragma unroll
        for (int a = 0; a < 3; ++a) o.end_dir[a * cap + id] = P::get(L.t, a);
    }
    if (o.path) o.path[id] = P::sget(L.s);
    if (o.time) o.time[id] = P::sget(L.T);
    if (o.amp) o.amp[id] = L.A;
    if (o.status) o.status[id] = L.status;
    if (o.generation) o.generation[id] = L.gen;
    if (o.seq) o.seq[id] = L.seq;
    if (o.layer) o.layer[id] = L.layer;
    if (o.parent) o.parent[id] = L.parent;
    if (o.n_acc) o.n_acc[id] = L.n_acc;
    if (o.n_rej) o.n_rej[id] = L.n_rej;
    if (o.n_root) o.n_root[id] = L.n_root;
    if (o.n_refl) o.n_refl[id] = L.n_refl;
    if (o.n_turn) o.n_turn[id] = L.n_turn;
}

// Receiver test on the committed chord (state L before the commit -> r1 = r + dr): a hit is
// recorded when the chord enters a sphere; quantities are interpolated linearly along it.
// Culling: the receiver grid cell of the chord's midpoint lists the candidates; only they get
// the exact chord-sphere intersection.
template <class P>
__device__ __forceinline__ void receivers_on_chord(const Sinks &sk, const Lane<P> &L,
                                                   const StepParams<P> &sp,
                                                   const typename P::R dr[3],
                                                   const typename P::R dt[3], typename P::R dT,
                                                   typename P::R hc, bool to_max_path)
{
    typedef typename P::R R;
    const Receivers &rx = sk.rx;
    float m[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        m[a] = (P::kFF ? (float)P::base(L.r, a) : (float)P::get(L.r, a)) + 0.5f * (float)dr[a];
    if (m[0] < rx.org[0] || m[1] < rx.org[1] || m[2] < rx.org[2] || m[0] >= rx.hi[0] ||
        m[1] >= rx.hi[1] || m[2] >= rx.hi[2])
        return;  // outside every receiver's reach
    const int ix = min(rx.nx - 1, (int)((m[0] - rx.org[0]) * rx.inv_cell));
    const int iy = min(rx.ny - 1, (int)((m[1] - rx.org[1]) * rx.inv_cell));
    const int iz = min(rx.nz - 1, (int)((m[2] - rx.org[2]) * rx.inv_cell));
    const int2 span = __ldg(&rx.cell[((size_t)iz * rx.ny + iy) * rx.nx + ix]);
    const R zero = R(0);
    for (int q = span.x; q < span.y; ++q) {
        const int j = __ldg(&rx.items[q]);
        const SphereC &S = rx.s[j];
        R w[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            w[a] = P::rel(L.r, a, zero, S.c[a]);   // r0 - c
            R w1 = P::rel(L.r, a, dr[a], S.c[a]);  // r1 - c
            d[a] = P::kFF ? (w1 - w[a]) : dr[a];
        }
        R Rs = P::kFF ? R(S.Rf) : R(S.R);
        R qa = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        R qb = R(2) * (d[0] * w[0] + d[1] * w[1] + d[2] * w[2]);
        R qc = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] - Rs * Rs;
        if (qc <= R(0) || qa == R(0)) continue;
        R disc = qb * qb - R(4) * qa * qc;
        if (disc < R(0)) continue;
        R lam = (-qb - P::sqrt_(disc)) / (R(2) * qa);
        if (lam < R(0) || lam > R(1)) continue;
        unsigned long long k = atomicAdd(&sk.ctrl->n_hits, 1ull);
        if (k >= (unsigned long long)sk.hits.capacity) {
            atomicOr(&sk.ctrl->flags, (unsigned)FLAG_HIT_OVERFLOW);
            continue;
        }
        const long long cap = sk.hits.capacity;
        const double l = (double)lam;
        const double T0 = P::sget(L.T), s0 = P::sget(L.s);
        const double ds = to_max_path ? L.mp.d - s0 : (double)hc;
        if (sk.hits.ray) sk.hits.ray[k] = L.id;
        if (sk.hits.receiver) sk.hits.receiver[k] = S.idx;
        if (sk.hits.time) sk.hits.time[k] = T0 + l * (double)dT;
        if (sk.hits.path) sk.hits.path[k] = s0 + l * ds;
        if (sk.hits.amp) sk.hits.amp[k] = L.A;
        double dir[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double r0 = P::get(L.r, a);
            if (sk.hits.pos) sk.hits.pos[a * cap + k] = r0 + l * (double)d[a];
            double t0 = P::get(L.t, a);
            double t1 = t0 + (double)dt[a];
            dir[a] = t0 + l * (t1 - t0);
        }
        if (sk.hits.dir) {
            normalise3(dir);
#pragma unroll
            for (int a = 0; a < 3; ++a) sk.hits.dir[a * cap + k] = dir[a];
        }
    }
}

// Float-float renormalisation of a direction whose norm is 1 + delta (paraxial form).
__device__ __forceinline__ void ff_renormalise(PrecF32::V &t)
{
    float S = 0.0f, E = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p = t.hi[a] * t.hi[a];
        float e = __fmaf_rn(t.hi[a], t.hi[a], -p);
        float s, e2;
        two_sum(S, p, s, e2);
        S = s;
        E += e + e2 + 2.0f * t.hi[a] * t.lo[a];
    }
    float delta = (S - 1.0f) + E;  // |t|^2 - 1
    float q = sqrtf(1.0f + delta);
    float phi = -delta / (q * (1.0f + q));  // 1/|t| - 1
#pragma unroll
    for (int a = 0; a < 3; ++a) ff_add(t.hi[a], t.lo[a], t.hi[a] * phi);
}

// Records a secondary that is not traced (refracted into an absorbing layer, or dropped
// because the queue is full) at the intersection point.
template <class P>
__device__ __forceinline__ void record_secondary(const Sinks &sk, const Lane<P> &L,
                                                 unsigned long long id, int other, double amp,
                                                 const double t_refr[3], int status)
{
    Lane<P> S = L;
    S.id = (long long)id;
    S.parent = L.id;
    S.seq = L.n_refl;
    S.gen = L.gen + 1;
    S.layer = other;
    S.A = amp;
    S.status = status;
    S.n_acc = S.n_rej = S.n_root = S.n_refl = S.n_turn = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) P::set(S.t, a, t_refr[a]);
    write_ray<P>(sk.out, S.id, S, sk.ctrl);
}

__device__ __forceinline__ QRec *thread_stack(const Sinks &sk)
{
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    return sk.stack + tid * (size_t)sk.stack_depth;
}

// Keeps a secondary for later tracing: on the thread's private stack (no atomics, traced by
// this same thread once its current ray ends) or, when that is full, on the global queue
// that the next launch drains.
template <class P>
__device__ __forceinline__ void queue_secondary(const Sinks &sk, Lane<P> &L,
                                                unsigned long long id, int other, double amp,
                                                const double t_refr[3], int status)
{
    QRec *slot;
    if (L.stk < sk.stack_depth && (!L.tail || status != RP_ST_ALIVE)) {
        slot = thread_stack(sk) + L.stk;
        ++L.stk;
    } else {
        const unsigned long long q = atomicAdd(&sk.ctrl->q_tail, 1ull);
        if (q >= sk.q_cap) {
            atomicOr(&sk.ctrl->flags, (unsigned)FLAG_QUEUE_OVERFLOW);
            record_secondary<P>(sk, L, id, other, amp, t_refr, RP_ST_QUEUE_FULL);
            return;
        }
        slot = &sk.queue[q];
    }
    QRec &Q = *slot;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Q.r[a] = P::get(L.r, a);
        Q.t[a] = t_refr[a];
    }
    Q.T = P::sget(L.T);
    Q.s = P::sget(L.s);
    Q.A = amp;
    Q.A0 = L.A0;
    Q.id = (long long)id;
    Q.parent = L.id;
    Q.h = (double)L.h;
    Q.layer = other;
    Q.gen = L.gen + 1;
    Q.seq = L.n_refl;
    Q.status = status;
}

// Boundary split at the horizontal plane between the ray's layer and `other` (Sec. 2,
// boundary module): the ray is reflected and continues with A r; a secondary with the
// refracted direction and A tau is cast from the intersection point unless the incidence is
// beyond the critical angle, the generation cap is reached, or A tau is already below the
// amplitude threshold (such a ray would be discarded at once).
template <class P>
__device__ __forceinline__ void split_at_plane(const MediumLayered &med, Lane<P> &L,
                                               const StepParams<P> &sp, const Sinks &sk, int ev)
{
    const int other = (ev == EV_TOP) ? L.layer - 1 : L.layer + 1;
    const double nz = (ev == EV_TOP) ? 1.0 : -1.0;  // normal toward the incident side
    const bool spawn_allowed = L.gen < sp.max_generation;
    const int pk = (ev == EV_TOP) ? L.layer : L.layer + 1;  // plane index
    // n on the ray's side (n1) and on the far side (n2) of the plane, evaluated on the host
    const double n1d = (ev == EV_TOP) ? med.n_below[pk] : med.n_above[pk];
    const double n2d = (ev == EV_TOP) ? med.n_above[pk] : med.n_below[pk];
    if constexpr (!P::kFF) {
        // FP64 path: the same operations as the FP64 reference
        const double n1 = n1d, n2 = n2d;
        const double nrm[3] = {0.0, 0.0, nz};
        double t[3] = {P::get(L.t, 0), P::get(L.t, 1), P::get(L.t, 2)};
        double t_refl[3], t_refr[3], rr, tau;
        bool tir = split_dirs(t, nrm, n1, n2, sp.polarization, t_refl, t_refr, rr, tau);
        const double amp = L.A * tau;
        const bool weak = sp.use_min_amp && fabs(amp) < sp.min_amp * fabs(L.A0);
        if (!tir && spawn_allowed && !weak) {
            const unsigned long long id = atomicAdd(&sk.ctrl->out_count, 1ull);
            atomicAdd(&sk.ctrl->n_secondary, 1ull);
            queue_secondary<P>(sk, L, id, other, amp, t_refr,
                               med.L[other].absorb ? RP_ST_TRANSMITTED : RP_ST_ALIVE);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) P::set(L.t, a, t_refl[a]);
        L.A *= rr;
    } else {
        // FP32-mixed path: incidence geometry and Fresnel factors in FP32 (for a horizontal
        // plane the reflection only flips t_z, exactly); the direction of a traced
        // secondary is built in FP64
        const float n1 = (ev == EV_TOP) ? med.n_below_f[pk] : med.n_above_f[pk];
        const float n2 = (ev == EV_TOP) ? med.n_above_f[pk] : med.n_below_f[pk];
        const float tz = L.t.hi[2] + L.t.lo[2];
        float cos_i = -(tz * (float)nz);
        const bool toward = cos_i > 0.0f;
        cos_i = fmaxf(cos_i, 0.0f);
        const float eta = n1 / n2;
        const float sin2_t = eta * eta * (1.0f - cos_i * cos_i);
        float rr = 1.0f, tau = 0.0f;
        const bool tir = sin2_t > 1.0f;
        float cos_t = 0.0f;
        if (!tir) {
            cos_t = sqrtf(1.0f - sin2_t);
            const float rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
            const float ts = 2.0f * n1 * cos_i / (n1 * cos_i + n2 * cos_t);
            const float rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);
            const float tp = 2.0f * n1 * cos_i / (n2 * cos_i + n1 * cos_t);
            if (sp.polarization == RP_POL_S) {
                rr = rs;
                tau = ts;
            } else if (sp.polarization == RP_POL_P) {
                rr = rp;
                tau = tp;
            } else {
                const float Rr = 0.5f * (rs * rs + rp * rp);
                rr = sqrtf(Rr);
                tau = sqrtf(1.0f - Rr);
            }
        }
        const double amp = L.A * (double)tau;
        const bool weak = sp.use_min_amp && fabs(amp) < sp.min_amp * fabs(L.A0);
        if (!tir && spawn_allowed && !weak) {
            const unsigned long long id = atomicAdd(&sk.ctrl->out_count, 1ull);
            atomicAdd(&sk.ctrl->n_secondary, 1ull);
            double t_refr[3];
            if (med.L[other].absorb) {
                const float tf[3] = {eta * L.t.hi[0], eta * L.t.hi[1],
                                     eta * tz + (eta * cos_i - cos_t) * (float)nz};
                const float q = sqrtf(tf[0] * tf[0] + tf[1] * tf[1] + tf[2] * tf[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a) t_refr[a] = (double)(tf[a] / q);
                queue_secondary<P>(sk, L, id, other, amp, t_refr, RP_ST_TRANSMITTED);
            } else {
                // traced secondary: Snell's law in FP64 (horizontal plane: the tangential
                // part scales by n1/n2, the normal part is -cos(theta_t) along the normal)
                const double etad = (ev == EV_TOP) ? med.eta_up[pk] : med.eta_down[pk];
                const double ci = fmax(-(P::get(L.t, 2) * nz), 0.0);
                const double ct = sqrt(fmax(1.0 - etad * etad * (1.0 - ci * ci), 0.0));
                t_refr[0] = etad * P::get(L.t, 0);
                t_refr[1] = etad * P::get(L.t, 1);
                t_refr[2] = -ct * nz;
                queue_secondary<P>(sk, L, id, other, amp, t_refr, RP_ST_ALIVE);
            }
        }
        if (toward) {
            L.t.hi[2] = -L.t.hi[2];
            L.t.lo[2] = -L.t.lo[2];
        }
        L.A *= (double)rr;
    }
}

// Boundary split at a tilted or height-field boundary (boundary shapes beyond the plane, the
// paragraph after Fig. 1), in FP64 for both policies: the local normal (-dzb/dx, -dzb/dy, 1)
// / |...| turned toward the incident side, both layers' indices at the point, Snell and
// Fresnel as at a plane; the reflected ray continues, the refracted one is cast into the other
// layer.
template <class P>
__device__ __forceinline__ void split_at_surface(const MediumSurfaces &med, Lane<P> &L,
                                                 const StepParams<P> &sp, const Sinks &sk, int ev)
{
    const int k = (ev == EV_TOP) ? L.layer : L.layer + 1;
    const int other = (ev == EV_TOP) ? L.layer - 1 : L.layer + 1;
    double bx, by;
    if constexpr (P::kFF) {
        // FP32-mixed landing, completed as at a plane (land_correction): the end point sat
        // L.ga above or below the surface before it was put on it vertically; the ray is taken
        // back along itself by u = g / (d/ds of z - zb) = g / (t_z - bx t_x - by t_y), to first
        // order, and put back on the surface at its new (x, y)
        const double x0 = P::get(L.r, 0), y0 = P::get(L.r, 1);
        surf_depth(med, k, x0, y0, &bx, &by);
        const double t0[3] = {P::get(L.t, 0), P::get(L.t, 1), P::get(L.t, 2)};
        const double D = t0[2] - bx * t0[0] - by * t0[1];
        const double u = (double)L.ga / D;
        if (fabs(u) <= 0.1) {
            double n, dndz;
            layer_eval_d(med, L.layer, P::get(L.r, 2), n, dndz);
            const double kap = dndz / n;
            const double x1 = x0 - u * t0[0], y1 = y0 - u * t0[1];
            P::set(L.r, 0, x1);
            P::set(L.r, 1, y1);
            P::set(L.r, 2, surf_depth(med, k, x1, y1, &bx, &by));
            P::set(L.t, 0, t0[0] + u * kap * t0[2] * t0[0]);
            P::set(L.t, 1, t0[1] + u * kap * t0[2] * t0[1]);
            P::set(L.t, 2, t0[2] - u * kap * (1.0 - t0[2] * t0[2]));
            P::sadd(L.s, (float)-u);
            P::sadd(L.T, (float)(-u * n * kInvC0));
        }
    }
    const double r[3] = {P::get(L.r, 0), P::get(L.r, 1), P::get(L.r, 2)};
    surf_depth(med, k, r[0], r[1], &bx, &by);
    const double q = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), 1.0));
    const double sg = (ev == EV_TOP) ? 1.0 : -1.0;
    const double nrm[3] = {__ddiv_rn(-sg * bx, q), __ddiv_rn(-sg * by, q), __ddiv_rn(sg, q)};
    double n1, n2, dd;
    layer_eval_d(med, L.layer, r[2], n1, dd);
    layer_eval_d(med, other, r[2], n2, dd);
    double t[3] = {P::get(L.t, 0), P::get(L.t, 1), P::get(L.t, 2)};
    double t_refl[3], t_refr[3], rr, tau;
    const bool tir = split_dirs(t, nrm, n1, n2, sp.polarization, t_refl, t_refr, rr, tau);
    const double amp = L.A * tau;
    const bool weak = sp.use_min_amp && fabs(amp) < sp.min_amp * fabs(L.A0);
    if (!tir && L.gen < sp.max_generation && !weak) {
        const unsigned long long id = atomicAdd(&sk.ctrl->out_count, 1ull);
        atomicAdd(&sk.ctrl->n_secondary, 1ull);
        queue_secondary<P>(sk, L, id, other, amp, t_refr,
                           med.L[other].absorb ? RP_ST_TRANSMITTED : RP_ST_ALIVE);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) P::set(L.t, a, t_refl[a]);
    L.A *= rr;
}

// The landing point r + dr put radially onto sphere S (the FP64 reference's operations); *g,
// if given, receives the point's signed distance from the surface before it was moved.
template <class P>
__device__ __forceinline__ void sphere_snap(const SphereB &S, const typename P::V &r,
                                            const typename P::R dr[3], double out[3],
                                            double *g = nullptr)
{
    double w[3], d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w[a] = __dsub_rn(__dadd_rn(P::get(r, a), (double)dr[a]), S.c[a]);
        d2 = __dadd_rn(d2, __dmul_rn(w[a], w[a]));
    }
    const double d = sqrt(d2);
    if (g) *g = d - S.R;
    const double q = S.R / d;
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = __dadd_rn(S.c[a], __dmul_rn(q, w[a]));
}

// Boundary split at sphere j's surface (curved boundaries, the paragraph after Fig. 1), in
// FP64 for both policies (splits are rare): the local normal (r - c) / |r - c| turned toward
// the incident side, the indices of the two regions at the point, Snell and Fresnel as at a
// plane; the reflected ray continues, the refracted secondary starts in the other region.
template <class P>
__device__ __forceinline__ void split_at_sphere(const MediumSpheres &med, Lane<P> &L,
                                                const StepParams<P> &sp, const Sinks &sk, int j)
{
    const SphereB &S = med.S[j];
    const bool inside = L.layer == RP_MAX_LAYERS + j;
    if constexpr (P::kFF) {
        // FP32-mixed landing, completed as at a plane (land_correction): the end point sat
        // L.ga outside (> 0) or inside the sphere before it was put on it radially; the ray is
        // taken back along itself by u = g / (d/ds of |r - c|) = g / (t . m), m the outward
        // normal, to first order (the point stays on the sphere within u^2 / 2R); direction,
        // arc length and travel time follow as at a plane (t' = k (e_z - t_z t),
        // k = (dn/dz) / n on the ray's side).  Small corrections: FP32 on the float-float state.
        const float invR = __fdividef(1.0f, S.Rf);
        float m[3], t0[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            m[a] = ((L.r.hi[a] - S.cc[a].hi) + (L.r.lo[a] - S.cc[a].lo)) * invR;
            t0[a] = L.t.hi[a] + L.t.lo[a];
        }
        const float D = t0[0] * m[0] + t0[1] * m[1] + t0[2] * m[2];
        const float u = __fdividef(L.ga, D);  // a correction term: 2 ulp suffice
        if (fabsf(u) <= 0.1f) {
            float n, gr[3];
            const float z3[3] = {0.0f, 0.0f, L.r.hi[2] + L.r.lo[2]};
            medium_eval<P>(med, L.lc, z3, n, gr);
            const float k = __fdividef(gr[2], n);
#pragma unroll
            for (int a = 0; a < 3; ++a) P::add(L.r, a, L.ga * m[a] - u * t0[a]);
            P::add(L.t, 0, u * k * t0[2] * t0[0]);
            P::add(L.t, 1, u * k * t0[2] * t0[1]);
            P::add(L.t, 2, -u * k * (1.0f - t0[2] * t0[2]));
            P::sadd(L.s, -u);
            P::sadd(L.T, -u * n * (float)kInvC0);
        }
    }
    double r[3], w[3], d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r[a] = P::get(L.r, a);
        w[a] = __dsub_rn(r[a], S.c[a]);
        d2 = __dadd_rn(d2, __dmul_rn(w[a], w[a]));
    }
    const double d = sqrt(d2);
    double nrm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nrm[a] = (inside ? -1.0 : 1.0) * w[a] / d;
    const int other = inside ? layer_of(med, r[2]) : RP_MAX_LAYERS + j;
    double n1, n2, dd;
    layer_eval_d(med, L.layer, r[2], n1, dd);
    layer_eval_d(med, other, r[2], n2, dd);
    double t[3] = {P::get(L.t, 0), P::get(L.t, 1), P::get(L.t, 2)};
    double t_refl[3], t_refr[3], rr, tau;
    const bool tir = split_dirs(t, nrm, n1, n2, sp.polarization, t_refl, t_refr, rr, tau);
    const double amp = L.A * tau;
    const bool weak = sp.use_min_amp && fabs(amp) < sp.min_amp * fabs(L.A0);
    if (!tir && L.gen < sp.max_generation && !weak) {
        const unsigned long long id = atomicAdd(&sk.ctrl->out_count, 1ull);
        atomicAdd(&sk.ctrl->n_secondary, 1ull);
        queue_secondary<P>(sk, L, id, other, amp, t_refr,
                           med.L[other].absorb ? RP_ST_TRANSMITTED : RP_ST_ALIVE);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) P::set(L.t, a, t_refl[a]);
    L.A *= rr;
}

// Commit of the candidate state (r + dr, t + dt, T + dT) after a step of length hc; ev is the
// event the step landed on (EV_NONE: an ordinary accepted step).  Performs receivers, split,
// stop and break conditions.  Returns true if the ray finished.
template <class P, class M>
__device__ __forceinline__ bool commit(const M &med, Lane<P> &L, const StepParams<P> &sp,
                                       const Sinks &sk, typename P::R hc,
                                       const typename P::R dr_in[3], const typename P::R dt[3],
                                       typename P::R dT, int ev)
{
    typedef typename P::R R;
    R dr[3] = {dr_in[0], dr_in[1], dr_in[2]};
    // landing: move the candidate onto the plane by adjusting the increment
    bool on_surface = false;  // landing on a tilted or height-field boundary
    if (ev == EV_TOP || ev == EV_BOTTOM) {
        if constexpr (has_surfaces_v<M>) {
            const int k = (ev == EV_TOP) ? L.layer : L.layer + 1;
            if (surf_on(med, k)) {
                on_surface = true;
                const double zs = surf_depth(med, k, P::get(L.r, 0) + (double)dr[0],
                                             P::get(L.r, 1) + (double)dr[1], nullptr, nullptr);
                if constexpr (P::kFF)  // landing residual, for the correction at the split
                    L.ga = (R)((P::get(L.r, 2) + (double)dr[2]) - zs);
                dr[2] = (R)(zs - P::get(L.r, 2));
            }
        }
        if constexpr (is_layered_v<M>) {
            if (!on_surface) {
                const PlaneC &pl = (ev == EV_TOP) ? L.lc.top : L.lc.bot;
                const R g = P::rel(L.r, 2, dr[2], pl);
                if constexpr (P::kFF) L.ga = g;  // landing residual, for land_correction
                dr[2] = dr[2] - g;
            }
        }
    } else if (ev == EV_STOP) {
        const R off = stop_rel(L, sp, dr);
        if (L.stop_axis == 0)
            dr[0] -= off;
        else if (L.stop_axis == 1)
            dr[1] -= off;
        else
            dr[2] -= off;
    }
    double sn[3] = {0.0, 0.0, 0.0};  // a sphere landing: the point put on the surface
    if constexpr (has_spheres_v<M>) {
        if (ev >= EV_SPH) {
            double g;
            sphere_snap<P>(med.S[ev - EV_SPH], L.r, dr, sn, &g);
            if constexpr (P::kFF) L.ga = (R)g;  // landing residual, for the split's correction
#pragma unroll
            for (int a = 0; a < 3; ++a) dr[a] = (R)(sn[a] - P::get(L.r, a));
        }
    }
    const bool to_max_path = L.last && ev == EV_NONE;
    if (sk.has_rx) receivers_on_chord<P>(sk, L, sp, dr, dt, dT, hc, to_max_path);
    {
        R tz1 = P::base(L.t, 2) + dt[2];
        if ((P::base(L.t, 2) > R(0)) != (tz1 > R(0))) ++L.n_turn;
    }
    // apply
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P::add(L.r, a, dr[a]);
        P::add(L.t, a, dt[a]);
    }
    if (ev == EV_TOP || ev == EV_BOTTOM) {
        if constexpr (has_surfaces_v<M>) {
            if (on_surface)  // put on the surface vertically, at the landing point's (x, y)
                P::set(L.r, 2, surf_depth(med, (ev == EV_TOP) ? L.layer : L.layer + 1,
                                          P::get(L.r, 0), P::get(L.r, 1), nullptr, nullptr));
            else
                P::snap(L.r, 2, (ev == EV_TOP) ? L.lc.top : L.lc.bot);
        } else if constexpr (is_layered_v<M>) {
            P::snap(L.r, 2, (ev == EV_TOP) ? L.lc.top : L.lc.bot);
        }
    } else if (ev == EV_STOP) {
        if (L.stop_axis == 0)
            P::snap(L.r, 0, L.stop);
        else if (L.stop_axis == 1)
            P::snap(L.r, 1, L.stop);
        else
            P::snap(L.r, 2, L.stop);
    }
    if constexpr (has_spheres_v<M>) {
        if (ev >= EV_SPH) {
#pragma unroll
            for (int a = 0; a < 3; ++a) P::set(L.r, a, sn[a]);
        }
    }
    if constexpr (P::kFF) {
        if (sp.rhs_form == RP_RHS_PARAXIAL) ff_renormalise(L.t);
    } else {
        double q = sqrt(L.t.v[0] * L.t.v[0] + L.t.v[1] * L.t.v[1] + L.t.v[2] * L.t.v[2]);
        L.t.v[0] /= q;
        L.t.v[1] /= q;
        L.t.v[2] /= q;
    }
    P::sadd(L.T, dT);
    if (to_max_path)
        P::sset(L.s, L.mp.d);
    else
        P::sadd(L.s, hc);
    ++L.n_acc;
    L.h = L.h_next;

    if (ev == EV_TOP || ev == EV_BOTTOM || ev >= EV_SPH) {
        if constexpr (is_layered_v<M>) {
            // the split itself is done by finish_split, batched across the warp
            L.pend = ev;
            return false;
        }
    } else if (ev == EV_STOP) {
        L.status = RP_ST_REACHED_STOP;
        return true;
    }
    // break conditions, in the reference's order (|A| changes only at splits)
    if (to_max_path) {
        L.status = RP_ST_MAX_PATH;
    } else if (sp.use_max_time && P::sdiff(L.T, sp.mt) >= R(0)) {
        L.status = RP_ST_MAX_TIME;
    } else if constexpr (!is_layered_v<M>) {
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R zero = R(0);
            inside = inside && !(P::rel(L.r, a, zero, med.lo_c[a]) < R(0) ||
                                 P::rel(L.r, a, zero, med.hi_c[a]) > R(0));
        }
        if (!inside) L.status = RP_ST_LEFT_DOMAIN;
    }
    if (L.status != RP_ST_ALIVE) return true;
    set_trial(L, sp);
    return false;
}

// FP32-mixed landing on a plane, completed in the service phase before the split.  The landing
// search stops once the step's end is within eps_b (2e-6 m) of the plane, offset g along the
// normal (kept in L.ga by commit), and commit then puts the end onto the plane along the normal
// alone; that leaves an along-track error of u = g / t_z, a tenth of a millimetre per
// reflection at grazing incidence (t_z ~ 0.01), where FP64 lands within 1e-9 m.  Here the ray
// is taken back along itself by u, to first order: position r - u t (on the plane, as the
// normal's part of u t is g), direction t - u t' with the ray equation's t' = k (e_z - t_z t),
// k = (dn/dz) / n on the ray's side of the plane (host-evaluated per plane, like n), arc
// length s - u and travel time T - u n / c0.  |u| is capped at 0.1 m, where the neglected
// terms (u^2 times the ray's curvature) are ~1e-8 m.
template <class P>
__device__ __forceinline__ void land_correction(const MediumLayered &med, Lane<P> &L)
{
    if constexpr (P::kFF) {
        const float tz = L.t.hi[2] + L.t.lo[2];
        const float u = __fdividef(L.ga, tz);  // a correction term: 2 ulp suffice
        if (!(fabsf(u) <= 0.1f)) return;
        const int pk = (L.pend == EV_TOP) ? L.layer : L.layer + 1;
        const float n1 = (L.pend == EV_TOP) ? med.n_below_f[pk] : med.n_above_f[pk];
        const float k = (L.pend == EV_TOP) ? med.kap_below_f[pk] : med.kap_above_f[pk];
        const float tx = L.t.hi[0], ty = L.t.hi[1];
        P::add(L.r, 0, -u * tx);
        P::add(L.r, 1, -u * ty);
        P::add(L.t, 0, u * k * tz * tx);
        P::add(L.t, 1, u * k * tz * ty);
        P::add(L.t, 2, -u * k * (1.0f - tz * tz));
        P::sadd(L.s, -u);
        P::sadd(L.T, -u * n1 * (float)kInvC0);
    }
}

// Boundary split of a ray parked on a plane by commit (Sec. 2, boundary module), followed by
// the break conditions that the reference checks after a split.  Returns true if the ray
// finished.
template <class P>
__device__ __forceinline__ bool finish_split(const MediumLayered &med, Lane<P> &L,
                                             const StepParams<P> &sp, const Sinks &sk)
{
    typedef typename P::R R;
    land_correction<P>(med, L);
    split_at_plane<P>(med, L, sp, sk, L.pend);
    ++L.n_refl;
    L.pend = 0;
    if (sp.use_max_time && P::sdiff(L.T, sp.mt) >= R(0))
        L.status = RP_ST_MAX_TIME;
    else if (sp.use_min_amp && fabs(L.A) < sp.min_amp * fabs(L.A0))
        L.status = RP_ST_MIN_AMP;
    if (L.status != RP_ST_ALIVE) return true;
    set_trial(L, sp);
    return false;
}
template <class P>
__device__ __forceinline__ bool finish_split(const MediumSpheres &med, Lane<P> &L,
                                             const StepParams<P> &sp, const Sinks &sk)
{
    typedef typename P::R R;
    if (L.pend >= EV_SPH) {
        split_at_sphere<P>(med, L, sp, sk, L.pend - EV_SPH);
    } else {
        land_correction<P>(med, L);
        split_at_plane<P>(med, L, sp, sk, L.pend);
    }
    ++L.n_refl;
    L.pend = 0;
    if (sp.use_max_time && P::sdiff(L.T, sp.mt) >= R(0))
        L.status = RP_ST_MAX_TIME;
    else if (sp.use_min_amp && fabs(L.A) < sp.min_amp * fabs(L.A0))
        L.status = RP_ST_MIN_AMP;
    if (L.status != RP_ST_ALIVE) return true;
    set_trial(L, sp);
    return false;
}
template <class P>
__device__ __forceinline__ bool finish_split(const MediumSurfaces &med, Lane<P> &L,
                                             const StepParams<P> &sp, const Sinks &sk)
{
    typedef typename P::R R;
    if (surf_on(med, (L.pend == EV_TOP) ? L.layer : L.layer + 1)) {
        split_at_surface<P>(med, L, sp, sk, L.pend);
    } else {
        land_correction<P>(med, L);
        split_at_plane<P>(med, L, sp, sk, L.pend);
    }
    ++L.n_refl;
    L.pend = 0;
    if (sp.use_max_time && P::sdiff(L.T, sp.mt) >= R(0))
        L.status = RP_ST_MAX_TIME;
    else if (sp.use_min_amp && fabs(L.A) < sp.min_amp * fabs(L.A0))
        L.status = RP_ST_MIN_AMP;
    if (L.status != RP_ST_ALIVE) return true;
    set_trial(L, sp);
    return false;
}
template <class P>
__device__ __forceinline__ bool finish_split(const MediumGrid &, Lane<P> &, const StepParams<P> &,
                                             const Sinks &)
{
    return false;  // gridded media have no boundaries
}

// Regula-falsi point of the current bracket (bisection if it falls outside).
template <class P>
__device__ __forceinline__ typename P::R rf_point(const Lane<P> &L)
{
    typedef typename P::R R;
    R c = L.rb - L.gb * (L.rb - L.ra) / (L.gb - L.ga);
    if (!(c > L.ra && c < L.rb)) c = R(0.5) * (L.ra + L.rb);
    return c;
}

// One iteration of a lane: one Cash-Karp evaluation and the state-machine update.
// Returns true when the ray has finished (L.status set).  Every branch that accepts the step
// leads to the one call of commit at the end, so that its code is inlined once.
template <class P, class M>
__device__ __forceinline__ bool advance(const M &med, Lane<P> &L, const StepParams<P> &sp,
                                        const Sinks &sk)
{
    typedef typename P::R R;
    if (L.mode == MODE_NORMAL && (long long)L.n_acc + L.n_rej + L.n_root >= sp.max_steps) {
        L.status = RP_ST_MAX_STEPS;
        return true;
    }
    const R hc = L.h_try;
    R dr[3], dt[3], dT, er, et;
    ck_step<P, M>(med, L.lc, sp.rhs_form, L.r, L.t, hc, dr, dt, dT, er, et);

    int cev = -1;  // the event the accepted step lands on (EV_NONE: none); -1: no commit
    if (L.mode == MODE_NORMAL) {
        // e = max(er, et) / tol; the FP32-mixed step returns squared norms, so there e holds
        // e^2 and the exponents of the step law are halved
        constexpr R kq = P::kFF ? R(0.5) : R(1);
        const R e = (er > et ? er : et) * (P::kFF ? sp.inv_tol2 : sp.inv_tol);
        if (!(e <= R(1)) && hc > sp.h_min) {
            ++L.n_rej;
            R fac = R(0.9) * P::pow_(e, R(-0.25) * kq);
            if (!(fac >= R(0.1))) fac = R(0.1);
            R hn = hc * fac;
            L.h = hn < sp.h_min ? sp.h_min : hn;
            set_trial(L, sp);
            return false;
        }
        R grow = (e == R(0)) ? R(5) : R(0.9) * P::pow_(e, R(-0.2) * kq);
        if (grow > R(5)) grow = R(5);
        R hn = hc * grow;
        hn = hn < sp.h_min ? sp.h_min : hn;
        hn = hn > sp.h_max ? sp.h_max : hn;
        L.h_next = hn;

        // event detection: earliest crossed plane by linear fraction
        int ev = EV_NONE;
        R ev_frac = R(2), ev_g0 = R(0), ev_g1 = R(0);
        const R zero3[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int kind = EV_TOP; kind <= EV_STOP; ++kind) {
            if ((kind == EV_TOP || kind == EV_BOTTOM) && !is_layered(med)) continue;
            if (kind == EV_STOP && !sp.use_stop) continue;
            R g0, g1;
            if constexpr (has_surfaces_v<M>) {
                // a surface's offset costs a height-field lookup: the start's is needed only
                // when the end could trigger an event (the same events as evaluating both)
                g1 = event_g<P>(med, L, sp, kind, dr);
                if (g1 > sp.eps_b) continue;
                g0 = event_g<P>(med, L, sp, kind, zero3);
            } else {
                g0 = event_g<P>(med, L, sp, kind, zero3);
                g1 = event_g<P>(med, L, sp, kind, dr);
            }
            if (g1 < R(0) || (g1 <= sp.eps_b && g0 > sp.eps_b)) {
                R fr = (g0 > R(0)) ? g0 / (g0 - g1) : R(0);
                if (fr < ev_frac) {
                    ev = kind;
                    ev_frac = fr;
                    ev_g0 = g0;
                    ev_g1 = g1;
                }
            }
        }
        if constexpr (has_spheres_v<M>) {
            // sphere surfaces: every sphere from outside, only its own from inside one
            const bool inside = L.layer >= RP_MAX_LAYERS;
            for (int j = 0; j < med.n_sph; ++j) {
                if (inside && L.layer != RP_MAX_LAYERS + j) continue;
                R g1 = event_g<P>(med, L, sp, EV_SPH + j, dr);
                if (g1 > sp.eps_b) continue;  // no event whatever g0 is: spare its evaluation
                R g0 = event_g<P>(med, L, sp, EV_SPH + j, zero3);
                if (g1 < R(0) || (g1 <= sp.eps_b && g0 > sp.eps_b)) {
                    R fr = (g0 > R(0)) ? g0 / (g0 - g1) : R(0);
                    if (fr < ev_frac) {
                        ev = EV_SPH + j;
                        ev_frac = fr;
                        ev_g0 = g0;
                        ev_g1 = g1;
                    }
                }
            }
        }
        if (ev == EV_NONE) {
            cev = EV_NONE;
        } else {
            L.ev = ev;
            if (fabs(ev_g1) <= sp.eps_b || (ev_g0 <= sp.eps_b && hc <= sp.h_min)) {
                cev = ev;
            } else if (ev_g0 <= sp.eps_b) {
                L.mode = MODE_PROBE;
                L.rb = hc;
                L.gb = ev_g1;
                L.h_try = sp.h_min;
            } else {
                L.mode = MODE_ILLINOIS;
                L.ra = R(0);
                L.ga = ev_g0;
                L.rb = hc;
                L.gb = ev_g1;
                L.side = 0;
                L.it = 1;
                L.h_try = rf_point(L);
            }
        }
    } else {
        // root-search evaluation at hc
        ++L.n_root;
        const R gc = event_g<P>(med, L, sp, L.ev, dr);
        if (L.mode == MODE_PROBE) {
            if (gc <= sp.eps_b) {
                cev = L.ev;
            } else {
                L.ra = hc;
                L.ga = gc;
                L.mode = MODE_ILLINOIS;
                L.side = 0;
                L.it = 1;
                L.h_try = rf_point(L);
            }
        } else if (fabs(gc) <= sp.eps_b) {
            cev = L.ev;
        } else {
            if (gc > R(0)) {
                L.ra = hc;
                L.ga = gc;
                if (L.side == 1) L.gb *= R(0.5);
                L.side = 1;
            } else {
                L.rb = hc;
                L.gb = gc;
                if (L.side == -1) L.ga *= R(0.5);
                L.side = -1;
            }
            if (L.it == kRootMaxIter) {
                L.root_fail = 1;
                atomicOr(&sk.ctrl->flags, (unsigned)FLAG_ROOT_CAP);
                cev = L.ev;
            } else {
                ++L.it;
                L.h_try = rf_point(L);
            }
        }
    }
    if (cev < 0) return false;
    return commit<P, M>(med, L, sp, sk, hc, dr, dt, dT, cev);
}

}  // namespace rpk
