"""Host-side checks of the C ABI that run before any CUDA call, so they are exercised here
without a GPU: medium descriptors that rp_medium_create must refuse (RP_ERR_INVALID_ARG with a
message), and a valid one that passes them (RP_OK on a GPU, else the CUDA error of the first
device call)."""
import ctypes as C

import pytest

from paper_1810_01780_gb300 import _abi as A

RP_ERR_INVALID_ARG, RP_ERR_CUDA = -1, -2


def _layered(n_layers=2):
    d = A.MediumDesc()
    d.kind = A.MEDIUM_KIND["layered"]
    d.n_layers = n_layers
    for k in range(n_layers):
        L = d.layers[k]
        L.z_top, L.n0, L.dn, L.z0, L.offset, L.absorb = 100.0 * k, 1.78, 0.43, 75.0, 0.0, 0
    d.layers[0].n0, d.layers[0].dn, d.layers[0].absorb = 1.000293, 0.0, 1
    return d


def _create(d):
    h = C.c_void_p()
    rc = A.lib().rp_medium_create(C.byref(d), None, C.byref(h))
    if rc == 0:
        A.lib().rp_medium_destroy(h)
    return rc, A.last_error()


def _sphere(d, j, c, r):
    S = d.spheres[j]
    S.center[0], S.center[1], S.center[2] = c
    S.radius, S.n0, S.dn, S.z0, S.offset = r, 1.8, 0.0, 0.0, 0.0


def test_valid_descriptor_passes_the_host_checks():
    d = _layered(3)
    d.n_spheres = 1
    _sphere(d, 0, (0.0, 0.0, 300.0), 40.0)
    rc, msg = _create(d)
    assert rc in (0, RP_ERR_CUDA), (rc, msg)


@pytest.mark.parametrize("case", ["no_layers", "too_many_layers", "z_top_order", "z0", "index",
                                  "n_spheres", "sphere_radius", "sphere_cut", "sphere_overlap",
                                  "grid_nodes", "grid_spacing", "grid_data", "kind"])
def test_invalid_descriptors_are_refused_on_the_host(case):
    d = _layered(3)
    if case == "no_layers":
        d.n_layers = 0
    elif case == "too_many_layers":
        d.n_layers = A.MAX_LAYERS + 1
    elif case == "z_top_order":
        d.layers[2].z_top = 50.0  # below layer 1's top
    elif case == "z0":
        d.layers[1].z0 = 0.0
    elif case == "index":
        d.layers[1].n0, d.layers[1].dn = -1.0, 0.0
    elif case == "n_spheres":
        d.n_spheres = A.MAX_SPHERES + 1
    elif case == "sphere_radius":
        d.n_spheres = 1
        _sphere(d, 0, (0.0, 0.0, 300.0), 0.0)
    elif case == "sphere_cut":  # the plane at 200 m passes through the sphere
        d.n_spheres = 1
        _sphere(d, 0, (0.0, 0.0, 190.0), 40.0)
    elif case == "sphere_overlap":
        d.n_spheres = 2
        _sphere(d, 0, (0.0, 0.0, 400.0), 40.0)
        _sphere(d, 1, (50.0, 0.0, 400.0), 40.0)
    elif case.startswith("grid") or case == "kind":
        d = A.MediumDesc()
        d.kind = A.MEDIUM_KIND["grid"] if case != "kind" else 7
        d.nx = d.ny = d.nz = 4
        d.spacing = 4.0
        d.grid_n = C.c_void_p(1)  # never read: the checks refuse the descriptor first
        if case == "grid_nodes":
            d.nz = 1
        elif case == "grid_spacing":
            d.spacing = 0.0
        elif case == "grid_data":
            d.grid_n = None
    rc, msg = _create(d)
    assert rc == RP_ERR_INVALID_ARG, (case, rc, msg)
    assert msg.startswith("rp_medium_create:"), msg


# rp_trace refuses bad calls before it touches the medium or the device: a zeroed block stands
# in for the medium handle (never read on these paths) and the batch is empty.
_FAKE_MEDIUM = (C.c_char * 65536)()
_ANCHOR = (C.c_double * 4)()


def _trace(params, n=0, capacity=1, end_pos=True):
    rays = A.Rays()
    rays.n = n
    out = A.RayOut()
    out.capacity = capacity
    out.end_pos = C.cast(_ANCHOR, C.c_void_p) if end_pos else None
    st = A.Stats()
    rc = A.lib().rp_trace(C.cast(_FAKE_MEDIUM, C.c_void_p), C.byref(rays), None, C.byref(params),
                          C.byref(out), None, C.byref(st), None)
    return rc, A.last_error()


def _params(**kw):
    from paper_1810_01780_gb300 import api

    base = dict(tol=1e-6, h_min=1e-3, h_max=10.0, h0=1.0, max_path=100.0, max_generation=3)
    p = api.make_params({k: v for k, v in base.items()}, kw.pop("precision", "fp64"))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [dict(tol=0.0), dict(h_min=0.0), dict(h_max=1e-4),
                                 dict(h0=0.0), dict(max_path=0.0), dict(eps_b=0.0),
                                 dict(max_steps=0), dict(max_generation=16),
                                 dict(max_generation=-1), dict(precision=7),
                                 dict(polarization=9), dict(rhs_form=9),
                                 dict(rhs_form=A.RHS_FORM["momentum"],
                                      precision=A.PRECISION["fp32"]),
                                 dict(service_idle=-1), dict(flush_min=-1), dict(block=100),
                                 dict(block=288), dict(block=-32), dict(blocks_per_sm=-1)])
def test_rp_trace_refuses_bad_parameters(bad):
    p = _params()
    for k, v in bad.items():
        setattr(p, k, v)
    rc, msg = _trace(p)
    assert rc == RP_ERR_INVALID_ARG, (bad, rc, msg)
    assert msg.startswith("params:"), msg


def test_rp_trace_refuses_bad_stop_planes_and_buffers():
    p = _params()
    p.use_stop = 1
    p.stop_n[0], p.stop_n[1] = 1.0, 1.0  # not a coordinate axis
    assert _trace(p)[0] == RP_ERR_INVALID_ARG
    p.stop_n[1] = 0.0
    p.stop_n[0] = 0.5  # not unit
    assert _trace(p)[0] == RP_ERR_INVALID_ARG
    q = _params()
    assert _trace(q, end_pos=False)[0] == RP_ERR_INVALID_ARG  # no end_pos array
    rc, msg = _trace(q, n=4, capacity=4)  # rays without arrays
    assert rc == RP_ERR_INVALID_ARG and "ray arrays" in msg


def _find_paths(pp, n=4, count=True):
    arr = (C.c_double * 4)()
    ang = (C.c_int32 * 4)()
    sol = A.Solutions()
    sol.count = C.cast(ang, C.c_void_p) if count else None
    st = A.Stats()
    p = C.cast(arr, C.c_void_p)
    rc = A.lib().rp_find_paths(C.cast(_FAKE_MEDIUM, C.c_void_p), n, p, p, p,
                               C.cast(ang, C.c_void_p), C.byref(pp), C.byref(sol), C.byref(st),
                               None)
    return rc, A.last_error()


def _path_params(**kw):
    pp = A.PathParams()
    pp.trace = _params()
    pp.trace.max_path = 0.0  # the path finder sets its own per-pair budget
    pp.hit_tol, pp.max_iter, pp.max_sol = 0.1, 60, 4
    for k, v in kw.items():
        setattr(pp, k, v)
    return pp


@pytest.mark.parametrize("bad", [dict(hit_tol=0.0), dict(max_iter=0), dict(max_iter=201),
                                 dict(max_sol=0), dict(max_sol=9)])
def test_rp_find_paths_refuses_bad_parameters(bad):
    rc, msg = _find_paths(_path_params(**bad))
    assert rc == RP_ERR_INVALID_ARG and msg.startswith("rp_find_paths:"), (bad, rc, msg)


def test_rp_find_paths_refuses_bad_trace_parameters_and_arrays():
    pp = _path_params()
    pp.trace.tol = -1.0
    assert _find_paths(pp)[0] == RP_ERR_INVALID_ARG
    rc, msg = _find_paths(_path_params(), count=False)
    assert rc == RP_ERR_INVALID_ARG and "null" in msg
    assert _find_paths(_path_params(), n=-1)[0] == RP_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [dict(epochs=0), dict(batch=0), dict(batch=1 << 20),
                                 dict(lr=0.0), dict(lr_final=-1.0)])
def test_rp_surrogate_train_refuses_bad_schedules(bad):
    tp = A.TrainParams()
    tp.epochs, tp.batch, tp.lr, tp.lr_final, tp.seed = 1, 256, 1e-3, 0.0, 1
    for k, v in bad.items():
        setattr(tp, k, v)
    buf = C.cast((C.c_float * 16)(), C.c_void_p)
    loss = C.c_double()
    rc = A.lib().rp_surrogate_train(C.cast(_FAKE_MEDIUM, C.c_void_p), 1024, buf, buf, buf,
                                    C.byref(tp), C.byref(loss), None)
    assert rc == RP_ERR_INVALID_ARG, (bad, rc)
    assert A.last_error().startswith("rp_surrogate_train:")
