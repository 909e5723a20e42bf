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
