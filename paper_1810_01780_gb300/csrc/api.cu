// api.cu -- the C ABI entry points (rp.h): argument checks, media, workspace, errors.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "rp_internal.h"

namespace rph {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? RP_ERR_OOM : RP_ERR_CUDA;
}

Workspace &workspace(int device)
{
    static std::mutex mu;
    static std::map<int, Workspace *> ws;
    std::lock_guard<std::mutex> lock(mu);
    Workspace *&w = ws[device];
    if (!w) w = new Workspace();
    return *w;
}

int ensure_host_clock(Workspace &w, size_t bytes)
{
    if (w.host_clock_size >= bytes) return RP_OK;
    if (w.host_clock) cudaFreeHost(w.host_clock);
    w.host_clock = nullptr;
    w.host_clock_size = 0;
    RP_CUDA_TRY(cudaMallocHost(&w.host_clock, bytes));
    w.host_clock_size = bytes;
    return RP_OK;
}

int ensure_workspace(Workspace &w, size_t bytes)
{
    if (!w.host_ctrl) RP_CUDA_TRY(cudaMallocHost(&w.host_ctrl, 4096));
    if (w.size >= bytes) return RP_OK;
    if (w.ptr) {
        RP_CUDA_TRY(cudaDeviceSynchronize());
        RP_CUDA_TRY(cudaFree(w.ptr));
        w.ptr = nullptr;
        w.size = 0;
    }
    size_t sz = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&w.ptr, sz);
    if (e != cudaSuccess) {
        w.ptr = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    w.size = sz;
    return RP_OK;
}

int sm_count(int device)
{
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device]) return cached[device];
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    if (n <= 0) n = 1;
    if (device >= 0 && device < 64) cached[device] = n;
    return n;
}

int validate_params(const rp_trace_params *p, bool path_finding)
{
    if (!(p->tol > 0.0) || !(p->h_min > 0.0) || !(p->h_max >= p->h_min) || !(p->h0 > 0.0)) {
        set_error("params: need tol > 0, 0 < h_min <= h_max, h0 > 0");
        return RP_ERR_INVALID_ARG;
    }
    if (!path_finding && !(p->max_path > 0.0)) {
        set_error("params: need max_path > 0");
        return RP_ERR_INVALID_ARG;
    }
    if (!(p->eps_b > 0.0) || p->max_steps <= 0 || p->max_generation < 0 ||
        p->max_generation > 15) {
        set_error("params: need eps_b > 0, max_steps > 0, 0 <= max_generation <= 15");
        return RP_ERR_INVALID_ARG;
    }
    if (p->precision != RP_FP64 && p->precision != RP_FP32_MIXED) {
        set_error("params: unknown precision %d", p->precision);
        return RP_ERR_INVALID_ARG;
    }
    if (p->polarization < RP_POL_S || p->polarization > RP_POL_UNPOL ||
        (p->rhs_form != RP_RHS_PROJECTED && p->rhs_form != RP_RHS_PARAXIAL &&
         p->rhs_form != RP_RHS_MOMENTUM)) {
        set_error("params: bad polarization or rhs_form");
        return RP_ERR_INVALID_ARG;
    }
    if (p->rhs_form == RP_RHS_MOMENTUM && p->precision != RP_FP64) {
        set_error("params: the momentum form runs in RP_FP64 only");
        return RP_ERR_INVALID_ARG;
    }
    if (p->service_idle < 0 || p->flush_min < 0 || p->blocks_per_sm < 0 || p->block < 0 ||
        p->block > kBlockMax || p->block % 32 != 0) {
        set_error("params: need service_idle, flush_min, blocks_per_sm >= 0 and block 0 or a "
                  "multiple of 32 up to %d", kBlockMax);
        return RP_ERR_INVALID_ARG;
    }
    if (p->ray_order != RP_ORDER_COHERENT && p->ray_order != RP_ORDER_GIVEN) {
        set_error("params: ray_order must be RP_ORDER_COHERENT (0) or RP_ORDER_GIVEN (1)");
        return RP_ERR_INVALID_ARG;
    }
    return RP_OK;
}

// Non-horizontal boundaries of a layered medium (rp_surface): checked on the host, height
// fields copied into one device allocation (the caller's array may be on the host or the
// device), the kernel's SurfB records filled in.
int build_surfaces(rp_medium_s *m, const rp_medium_desc *d)
{
    m->n_surf = 0;
    if (d->n_surfaces == 0) return RP_OK;
    if (d->n_surfaces < 0 || d->n_surfaces > RP_MAX_LAYERS) {
        set_error("rp_medium_create: n_surfaces must be 0..%d", RP_MAX_LAYERS);
        return RP_ERR_INVALID_ARG;
    }
    if (d->n_spheres > 0) {
        set_error("rp_medium_create: a medium takes either spheres or surfaces");
        return RP_ERR_UNSUPPORTED;
    }
    size_t total = 0;
    bool taken[RP_MAX_LAYERS] = {false};
    for (int j = 0; j < d->n_surfaces; ++j) {
        const rp_surface &S = d->surfaces[j];
        bool ok = S.layer >= 1 && S.layer < d->n_layers && !taken[S.layer] && S.normal[2] > 0.0 &&
                  std::isfinite(S.normal[0]) && std::isfinite(S.normal[1]) &&
                  std::isfinite(S.normal[2]);
        if (ok && S.height)
            ok = S.nx >= 2 && S.ny >= 2 && S.spacing[0] > 0.0 && S.spacing[1] > 0.0 &&
                 std::isfinite(S.spacing[0]) && std::isfinite(S.spacing[1]) &&
                 std::isfinite(S.origin[0]) && std::isfinite(S.origin[1]) &&
                 (size_t)S.nx * (size_t)S.ny <= ((size_t)1 << 28);
        if (!ok) {
            set_error("rp_medium_create: surface %d: needs an inner boundary (1..n_layers-1) "
                      "not taken by another, normal[2] > 0, and a height field of >= 2 x 2 nodes "
                      "with positive spacing", j);
            return RP_ERR_INVALID_ARG;
        }
        taken[S.layer] = true;
        if (S.height) total += (size_t)S.nx * (size_t)S.ny;
    }
    std::vector<double> host(total);
    size_t at = 0;
    for (int j = 0; j < d->n_surfaces; ++j) {
        const rp_surface &S = d->surfaces[j];
        if (!S.height) continue;
        const size_t cnt = (size_t)S.nx * (size_t)S.ny;
        RP_CUDA_TRY(cudaMemcpy(host.data() + at, S.height, cnt * sizeof(double), cudaMemcpyDefault));
        for (size_t i = 0; i < cnt; ++i)
            if (!std::isfinite(host[at + i])) {
                set_error("rp_medium_create: surface %d has a non-finite height", j);
                return RP_ERR_INVALID_ARG;
            }
        at += cnt;
    }
    if (total) {
        cudaError_t e = cudaMalloc(&m->surf_dev, total * sizeof(double));
        if (e != cudaSuccess) {
            m->surf_dev = nullptr;
            return cuda_fail(e, "cudaMalloc(height fields)");
        }
        RP_CUDA_TRY(cudaMemcpy(m->surf_dev, host.data(), total * sizeof(double),
                               cudaMemcpyHostToDevice));
        std::vector<float> hostf(total);
        for (size_t i = 0; i < total; ++i) hostf[i] = (float)host[i];
        e = cudaMalloc(&m->surf_dev_f, total * sizeof(float));
        if (e != cudaSuccess) {
            m->surf_dev_f = nullptr;
            return cuda_fail(e, "cudaMalloc(height fields)");
        }
        RP_CUDA_TRY(cudaMemcpy(m->surf_dev_f, hostf.data(), total * sizeof(float),
                               cudaMemcpyHostToDevice));
    }
    at = 0;
    for (int j = 0; j < d->n_surfaces; ++j) {
        const rp_surface &S = d->surfaces[j];
        rpk::SurfB &B = m->surf[S.layer];
        B.on = 1;
        B.sx = -S.normal[0] / S.normal[2];
        B.sy = -S.normal[1] / S.normal[2];
        B.sxh = (float)B.sx;
        B.sxl = (float)(B.sx - (double)B.sxh);
        B.syh = (float)B.sy;
        B.syl = (float)(B.sy - (double)B.syh);
        B.h = nullptr;
        B.hf = nullptr;
        if (S.height) {
            B.h = m->surf_dev + at;
            B.hf = m->surf_dev_f + at;
            at += (size_t)S.nx * (size_t)S.ny;
            B.nx = S.nx;
            B.ny = S.ny;
            B.ox = S.origin[0];
            B.oy = S.origin[1];
            B.dx = S.spacing[0];
            B.dy = S.spacing[1];
            B.oxf = (float)B.ox;
            B.oyf = (float)B.oy;
            B.dxf = (float)B.dx;
            B.dyf = (float)B.dy;
            B.inv_dxf = (float)(1.0 / B.dx);
            B.inv_dyf = (float)(1.0 / B.dy);
        }
    }
    m->n_surf = d->n_surfaces;
    return RP_OK;
}

}  // namespace rph

using namespace rph;

extern "C" {

int rp_medium_create(const rp_medium_desc *d, void *stream, rp_medium_t *out)
{
    if (!d || !out) {
        set_error("rp_medium_create: null argument");
        return RP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    rp_medium_s *m = new (std::nothrow) rp_medium_s();
    if (!m) return RP_ERR_OOM;
    memset(&m->layered, 0, sizeof m->layered);
    memset(&m->grid, 0, sizeof m->grid);
    m->grid_dev = nullptr;
    // the descriptor is checked on the host before any CUDA call; the medium belongs to the
    // current device
    auto bind_device = [&]() -> int {
        cudaError_t e = cudaGetDevice(&m->device);
        if (e != cudaSuccess) {
            delete m;
            return cuda_fail(e, "cudaGetDevice");
        }
        return RP_OK;
    };
    m->kind = d->kind;
    if (d->kind == RP_MEDIUM_LAYERED) {
        if (d->n_layers < 1 || d->n_layers > RP_MAX_LAYERS) {
            delete m;
            set_error("rp_medium_create: n_layers must be 1..%d", RP_MAX_LAYERS);
            return RP_ERR_INVALID_ARG;
        }
        m->layered.n_layers = d->n_layers;
        for (int k = 0; k < d->n_layers; ++k) {
            const rp_layer &L = d->layers[k];
            if (k >= 2 && !(L.z_top > d->layers[k - 1].z_top)) {
                delete m;
                set_error("rp_medium_create: z_top must increase with the layer index");
                return RP_ERR_INVALID_ARG;
            }
            if (L.dn != 0.0 && !(L.z0 > 0.0)) {
                delete m;
                set_error("rp_medium_create: layer %d needs z0 > 0", k);
                return RP_ERR_INVALID_ARG;
            }
            if (!(L.n0 + L.offset > 0.0)) {
                delete m;
                set_error("rp_medium_create: layer %d has a non-positive index", k);
                return RP_ERR_INVALID_ARG;
            }
            rpk::LayerC &c = m->layered.L[k];
            c.n0 = L.n0;
            c.dn = L.dn;
            c.off = L.offset;
            c.has_exp = L.dn != 0.0;
            c.inv_z0 = c.has_exp ? 1.0 / L.z0 : 0.0;
            c.gcoef = c.has_exp ? L.dn / L.z0 : 0.0;
            c.n0f = (float)c.n0;
            c.dnf = (float)c.dn;
            c.offf = (float)c.off;
            c.inv_z0f = (float)c.inv_z0;
            c.gcoeff = (float)c.gcoef;
            c.absorb = L.absorb != 0;
            m->layered.top[k] = plane_const(k ? L.z_top : -1e300);
        }
        // refractive index on both sides of every plane, in FP64 on the host (the boundary
        // module needs them at every split)
        for (int k = 1; k < d->n_layers; ++k) {
            const double z = d->layers[k].z_top;
            for (int side = 0; side < 2; ++side) {
                const rp_layer &L = d->layers[side == 0 ? k - 1 : k];
                double n = L.dn == 0.0 ? L.n0 + L.offset : L.n0 - L.dn * exp(-z / L.z0) + L.offset;
                double dndz = L.dn == 0.0 ? 0.0 : L.dn / L.z0 * exp(-z / L.z0);
                if (side == 0) {
                    m->layered.n_above[k] = n;
                    m->layered.n_above_f[k] = (float)n;
                    m->layered.kap_above_f[k] = (float)(dndz / n);
                } else {
                    m->layered.n_below[k] = n;
                    m->layered.n_below_f[k] = (float)n;
                    m->layered.kap_below_f[k] = (float)(dndz / n);
                }
            }
            m->layered.eta_down[k] = m->layered.n_above[k] / m->layered.n_below[k];
            m->layered.eta_up[k] = m->layered.n_below[k] / m->layered.n_above[k];
        }
        // spheres: each strictly inside one layer, none overlapping another
        if (d->n_spheres < 0 || d->n_spheres > RP_MAX_SPHERES) {
            delete m;
            set_error("rp_medium_create: n_spheres must be 0..%d", RP_MAX_SPHERES);
            return RP_ERR_INVALID_ARG;
        }
        m->layered.n_sph = d->n_spheres;
        for (int j = 0; j < d->n_spheres; ++j) {
            const rp_sphere &S = d->spheres[j];
            bool ok = S.radius > 0.0 && std::isfinite(S.radius) && (S.n0 + S.offset > 0.0) &&
                      (S.dn == 0.0 || S.z0 > 0.0);
            for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(S.center[a]);
            for (int k = 1; ok && k < d->n_layers; ++k)  // no plane cuts the sphere
                ok = fabs(S.center[2] - d->layers[k].z_top) > S.radius;
            for (int i = 0; ok && i < j; ++i) {
                const rp_sphere &T = d->spheres[i];
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a)
                    d2 += (S.center[a] - T.center[a]) * (S.center[a] - T.center[a]);
                ok = sqrt(d2) > S.radius + T.radius;
            }
            if (!ok) {
                delete m;
                set_error("rp_medium_create: sphere %d: needs radius > 0, a positive index, z0 > "
                          "0 with dn != 0, no layer plane through it and no overlap", j);
                return RP_ERR_INVALID_ARG;
            }
            rpk::LayerC &c = m->layered.L[RP_MAX_LAYERS + j];
            c.n0 = S.n0;
            c.dn = S.dn;
            c.off = S.offset;
            c.has_exp = S.dn != 0.0;
            c.inv_z0 = c.has_exp ? 1.0 / S.z0 : 0.0;
            c.gcoef = c.has_exp ? S.dn / S.z0 : 0.0;
            c.n0f = (float)c.n0;
            c.dnf = (float)c.dn;
            c.offf = (float)c.off;
            c.inv_z0f = (float)c.inv_z0;
            c.gcoeff = (float)c.gcoef;
            c.absorb = S.absorb != 0;
            rpk::SphereB &B = m->layered.S[j];
            for (int a = 0; a < 3; ++a) {
                B.c[a] = S.center[a];
                B.cc[a] = plane_const(S.center[a]);
            }
            B.R = S.radius;
            const double R2 = S.radius * S.radius;
            B.R2h = (float)R2;
            B.R2l = (float)(R2 - (double)B.R2h);
            B.Rf = (float)S.radius;
            B.pad = 0.0f;
        }
        if (int rc = bind_device()) return rc;
        if (int rc = build_surfaces(m, d)) {
            if (m->surf_dev) cudaFree(m->surf_dev);
            if (m->surf_dev_f) cudaFree(m->surf_dev_f);
            delete m;
            return rc;
        }
    } else if (d->kind == RP_MEDIUM_GRID) {
        if (d->nx < 2 || d->ny < 2 || d->nz < 2 || !(d->spacing > 0.0) || !d->grid_n) {
            delete m;
            set_error("rp_medium_create: grid needs >= 2 nodes per axis, spacing > 0, data");
            return RP_ERR_INVALID_ARG;
        }
        rpk::MediumGrid &g = m->grid;
        g.nx = d->nx;
        g.ny = d->ny;
        g.nz = d->nz;
        const int dims[3] = {d->nx, d->ny, d->nz};
        for (int a = 0; a < 3; ++a) {
            g.org[a] = d->origin[a];
            g.orgf[a] = (float)d->origin[a];
            g.hi[a] = d->origin[a] + d->spacing * (double)(dims[a] - 1);
            g.lo_c[a] = plane_const(g.org[a]);
            g.hi_c[a] = plane_const(g.hi[a]);
        }
        g.inv_sp = 1.0 / d->spacing;
        g.inv_spf = (float)g.inv_sp;
        if (int rc = bind_device()) return rc;
        int rc = build_grid(m, d->grid_n, d->spacing, (cudaStream_t)stream);
        if (rc) {
            if (m->grid_dev) cudaFree(m->grid_dev);
            delete m;
            return rc;
        }
        g.g = m->grid_dev;
    } else {
        delete m;
        set_error("rp_medium_create: unknown kind %d", d->kind);
        return RP_ERR_INVALID_ARG;
    }
    *out = m;
    return RP_OK;
}

int rp_medium_destroy(rp_medium_t m)
{
    if (!m) return RP_OK;
    if (m->grid_dev) cudaFree(m->grid_dev);
    if (m->surf_dev) cudaFree(m->surf_dev);
    if (m->surf_dev_f) cudaFree(m->surf_dev_f);
    delete m;
    return RP_OK;
}

int rp_trace(rp_medium_t m, const rp_rays *in, const rp_receivers *rx, const rp_trace_params *p,
             rp_ray_out *out, rp_hits *hits, rp_stats *stats, void *stream)
{
    if (stats) memset(stats, 0, sizeof *stats);
    try {
        return run_trace(m, in, rx, p, out, hits, stats, (cudaStream_t)stream);
    } catch (...) {
        set_error("rp_trace: internal exception");
        return RP_ERR_CUDA;
    }
}

int rp_find_paths(rp_medium_t m, int64_t n_pairs, const double *z_s, const double *z_r,
                  const double *dist, const int32_t *n_angles, const rp_path_params *p,
                  rp_solutions *sol, rp_stats *stats, void *stream)
{
    if (stats) memset(stats, 0, sizeof *stats);
    try {
        return run_find_paths(m, n_pairs, z_s, z_r, dist, n_angles, p, sol, stats,
                              (cudaStream_t)stream);
    } catch (...) {
        set_error("rp_find_paths: internal exception");
        return RP_ERR_CUDA;
    }
}

int rp_surrogate_encode(int64_t n, const double *z_s, const double *z_r, const double *dist,
                        const rp_solutions *sol, int32_t max_sol, float *x, float *y, float *t,
                        void *stream)
{
    return run_surrogate_encode(n, z_s, z_r, dist, sol, max_sol, x, y, t, (cudaStream_t)stream);
}

int rp_surrogate_find_paths(rp_surrogate_t s, rp_medium_t m, int64_t n, const double *z_s,
                            const double *z_r, const double *dist, const int32_t *n_angles,
                            const rp_path_params *p, const rp_surrogate_params *sp,
                            rp_solutions *sol, rp_surrogate_stats *stats, void *stream)
{
    try {
        return run_surrogate_paths(s, m, n, z_s, z_r, dist, n_angles, p, sp, sol, stats,
                                   (cudaStream_t)stream);
    } catch (...) {
        set_error("rp_surrogate_find_paths: internal exception");
        return RP_ERR_OOM;
    }
}

int rp_last_error(char *buf, size_t len)
{
    const std::string &s = g_last_error;
    if (buf && len) {
        size_t k = s.size() < len - 1 ? s.size() : len - 1;
        memcpy(buf, s.data(), k);
        buf[k] = 0;
    }
    return (int)s.size();
}

const char *rp_version(void) { return "rp-gb300 0.1 (sm_103a)"; }

}  // extern "C"
