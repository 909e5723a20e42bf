"""Seeded synthetic workloads (inputs only; none of the method's arithmetic lives here).

Every generator draws from numpy's PCG64 with a fixed seed, so the CUDA path, the CPU oracle,
the tests and the benchmark all see the same arrays.  The shapes and distributions follow the
ray-tracing scenarios of the paper (Sec. 2: exponential ice profile n(z) = n0 - dn exp(-z/z0),
a reflecting ice-air surface, an internal layer boundary, receivers, gridded refractivity,
source-receiver geometries of the accuracy study) at the sizes of the five standard
workloads:

  ``small``     1,024 rays in the x-z plane from 200 m depth, launch angles 0..180 deg
  ``batched``   1,048,576 isotropic rays, two-layer ice with an internal boundary, 64 receivers
  ``grid``      256 x 256 x 512 FP32 refractivity grid (4 m) with Gaussian random perturbations,
                4,194,304 isotropic rays from 16 sources
  ``paths``     65,536 source-receiver pairs with 32..512 scan angles each
  ``surrogate`` 4,194,304 training pairs and 1,048,576 query pairs of the ``paths`` distribution
  ``spheres``   curved boundaries: two spherical inclusions in the ice, 1,048,576 rays
  ``fig1``      the paper's Fig. 1 example (firn layer over exponential ice, 5 us, A/A0 cut) as
                a fan of 1,048,576 rays
  ``surfaces``  non-horizontal boundaries: a tilted, rough ice surface (height field) and a
                tilted internal boundary, 1,048,576 rays

Conventions: z = depth (positive downward), angles from +z, positions in metres; ray arrays
are SoA with shape (3, n).
"""
from __future__ import annotations

import math

import numpy as np

N_AIR = 1.000293
ICE = dict(n0=1.788, dn=0.463, z0=75.0)

# ---------------------------------------------------------------------------------------
# media
# ---------------------------------------------------------------------------------------


def ice_with_surface(z0: float = 75.0, n_air: float = N_AIR) -> dict:
    """Air (absorbing: refracted rays are recorded and stop) above z = 0, exponential ice below."""
    return {"kind": "layered", "layers": [
        dict(n0=n_air, dn=0.0, z0=1.0, off=0.0, absorb=True),
        dict(z_top=0.0, n0=ICE["n0"], dn=ICE["dn"], z0=z0, off=0.0, absorb=False),
    ]}


def two_layer_ice(z_int: float = 100.0, jump: float = 0.02) -> dict:
    """Air above 0, exponential ice 0..z_int, the same profile + jump below z_int."""
    return {"kind": "layered", "layers": [
        dict(n0=N_AIR, dn=0.0, z0=1.0, off=0.0, absorb=True),
        dict(z_top=0.0, n0=ICE["n0"], dn=ICE["dn"], z0=ICE["z0"], off=0.0, absorb=False),
        dict(z_top=z_int, n0=ICE["n0"], dn=ICE["dn"], z0=ICE["z0"], off=jump, absorb=False),
    ]}


def single_profile(n0=1.788, dn=0.463, z0=75.0) -> dict:
    """One exponential layer continued to all depths (no boundary)."""
    return {"kind": "layered", "layers": [dict(n0=n0, dn=dn, z0=z0, off=0.0, absorb=False)]}


def firn_over_ice(n_firn: float = 1.5, z_firn: float = 10.0, z0: float = 71.4,
                  n_air: float = 1.0) -> dict:
    """The medium of the paper's Fig. 1: air (absorbing) above z = 0, a layer of constant index
    n_firn from 0 to z_firn, the exponential profile n0 - dn exp(-z/z0) below (z0 = 71.4 m)."""
    return {"kind": "layered", "layers": [
        dict(n0=n_air, dn=0.0, z0=1.0, off=0.0, absorb=True),
        dict(z_top=0.0, n0=n_firn, dn=0.0, z0=1.0, off=0.0, absorb=False),
        dict(z_top=z_firn, n0=ICE["n0"], dn=ICE["dn"], z0=z0, off=0.0, absorb=False),
    ]}


def ice_with_inclusions(n_air: float = N_AIR) -> dict:
    """Curved boundaries: the surface-bounded exponential ice with two spherical inclusions -- a
    lens of denser ice (the profile + 0.05) of radius 40 m centred at 300 m depth, and an air
    pocket (n = 1.0, traced) of radius 25 m at (150, 0, 500) m."""
    m = ice_with_surface(n_air=n_air)
    m["spheres"] = [
        dict(center=(0.0, 0.0, 300.0), radius=40.0, n0=ICE["n0"], dn=ICE["dn"], z0=ICE["z0"],
             off=0.05, absorb=False),
        dict(center=(150.0, 0.0, 500.0), radius=25.0, n0=1.0, dn=0.0, z0=1.0, off=0.0,
             absorb=False),
    ]
    return m


def rough_ice(n_air: float = N_AIR, seed: int = 8) -> dict:
    """Non-horizontal boundaries: the two-layer ice of ``two_layer_ice`` with its surface a
    plane tilted by 2 degrees (about the y axis) carrying a height field of seeded
    undulations -- a Gaussian random field of 0.3 m standard deviation and 8 m correlation
    length on 256 x 256 nodes at 2 m spacing around the origin -- and its internal boundary at
    100 m a plane tilted by 1 degree about the x axis."""
    m = two_layer_ice()
    h = gaussian_random_field((1, 256, 256), 2.0, 0.3, 8.0, seed)[0].astype(np.float64)
    a, b = math.radians(2.0), math.radians(1.0)
    m["surfaces"] = [
        dict(layer=1, normal=(math.sin(a), 0.0, math.cos(a)), height=h,
             origin=(-255.0, -255.0), spacing=(2.0, 2.0)),
        dict(layer=2, normal=(0.0, -math.sin(b), math.cos(b))),
    ]
    return m


def gaussian_random_field(shape, spacing, sigma, corr_len, seed) -> np.ndarray:
    """Seeded stationary Gaussian field with covariance sigma^2 exp(-r^2 / (2 l^2)).

    White noise is filtered in Fourier space by exp(-k^2 l^2 / 4) (the transform of the
    Gaussian kernel whose autocorrelation has the requested width) and rescaled to sample
    standard deviation sigma.  shape = (nz, ny, nx)."""
    import scipy.fft as sfft

    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape, dtype=np.float32)
    spec = sfft.rfftn(noise, workers=-1)
    del noise
    ks = [np.fft.fftfreq(s, d=spacing) * 2.0 * np.pi for s in shape[:-1]]
    ks.append(np.fft.rfftfreq(shape[-1], d=spacing) * 2.0 * np.pi)
    filt = None
    for ax, k in enumerate(ks):
        f = np.exp(-(k.astype(np.float32) ** 2) * (corr_len**2) / 4.0).astype(np.float32)
        sh = [1] * len(shape)
        sh[ax] = -1
        f = f.reshape(sh)
        filt = f if filt is None else filt * f
    spec *= filt
    field = sfft.irfftn(spec, s=shape, workers=-1).astype(np.float32)
    field *= np.float32(sigma / float(field.std()))
    return field


def grid_medium(nx=256, ny=256, nz=512, spacing=4.0, sigma=1e-3, corr_len=20.0, seed=3) -> dict:
    """FP32 node grid: exponential profile at each node depth + Gaussian perturbations."""
    origin = (-0.5 * spacing * (nx - 1), -0.5 * spacing * (ny - 1), 0.0)
    z = origin[2] + spacing * np.arange(nz, dtype=np.float64)
    prof = (ICE["n0"] - ICE["dn"] * np.exp(-z / ICE["z0"])).astype(np.float32)
    n = np.empty((nz, ny, nx), dtype=np.float32)
    n[:] = prof[:, None, None]
    if sigma > 0.0:
        n += gaussian_random_field((nz, ny, nx), spacing, sigma, corr_len, seed)
    return {"kind": "grid", "n": n, "origin": origin, "spacing": float(spacing)}


# ---------------------------------------------------------------------------------------
# rays
# ---------------------------------------------------------------------------------------


def fan_xz(n: int, depth: float = 200.0, lo_deg: float = 0.0, hi_deg: float = 180.0):
    """n rays from (0, 0, depth), launch angles linspace(lo, hi) inclusive, in the x-z plane."""
    th = np.radians(np.linspace(lo_deg, hi_deg, n))
    pos = np.zeros((3, n))
    pos[2] = depth
    d = np.stack([np.sin(th), np.zeros(n), np.cos(th)])
    return pos, d, np.ones(n)


def isotropic_dirs(rng, n):
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz])


def tilted_dirs(d, angle: float, seed: int):
    """The directions d (3, n) each rotated by `angle` rad about a seeded random axis
    perpendicular to it: the perturbed launch directions of the conditioning test (a ray whose
    result moves far under a tiny tilt is ill-conditioned)."""
    rng = np.random.default_rng(seed)
    d = d / np.linalg.norm(d, axis=0)
    a = rng.standard_normal(d.shape)
    a -= (a * d).sum(0) * d
    a /= np.linalg.norm(a, axis=0)
    return np.cos(angle) * d + np.sin(angle) * a


def isotropic_sources(n: int, seed: int, depth=(50.0, 1500.0), xy=400.0):
    """n rays, each from its own source (x, y ~ U[-xy, xy], depth ~ U[depth]), isotropic."""
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(-xy, xy, n), rng.uniform(-xy, xy, n),
                    rng.uniform(depth[0], depth[1], n)])
    return pos, isotropic_dirs(rng, n), np.ones(n)


def point_sources(n_src: int, per_src: int, seed: int, depth=(100.0, 1500.0), xy=200.0):
    """n_src point sources, per_src isotropic rays each (source-major order)."""
    rng = np.random.default_rng(seed)
    src = np.stack([rng.uniform(-xy, xy, n_src), rng.uniform(-xy, xy, n_src),
                    rng.uniform(depth[0], depth[1], n_src)])
    pos = np.repeat(src, per_src, axis=1)
    return pos, isotropic_dirs(rng, n_src * per_src), np.ones(n_src * per_src)


def receiver_lattice(radius: float = 1.0):
    """64 spheres: x, y in {-300, -100, 100, 300} m, depths {25, 75, 125, 175} m."""
    xs = np.array([-300.0, -100.0, 100.0, 300.0])
    zs = np.array([25.0, 75.0, 125.0, 175.0])
    c = np.array([[x, y, z] for z in zs for y in xs for x in xs])
    return c, np.full(len(c), radius)


def subsample(rays, idx):
    pos, d, a = rays
    return pos[:, idx].copy(), d[:, idx].copy(), a[idx].copy()


# ---------------------------------------------------------------------------------------
# source-receiver pairs
# ---------------------------------------------------------------------------------------


def pairs(n: int, seed: int, zs=(0.0, 2000.0), zr=(0.0, 200.0), dist=(0.0, 4000.0),
          angles=(32, 512)):
    rng = np.random.default_rng(seed)
    return dict(zs=rng.uniform(*zs, n), zr=rng.uniform(*zr, n), dist=rng.uniform(*dist, n),
                n_angles=rng.integers(angles[0], angles[1] + 1, n).astype(np.int32))


# ---------------------------------------------------------------------------------------
# the five standard workloads
# ---------------------------------------------------------------------------------------

TRACE_DEFAULTS = dict(tol=1e-6, h_min=1e-3, h_max=10.0, h0=10.0, max_time=0.0, min_amp=0.0,
                      eps_b=1e-9, max_generation=3, polarization="s", rhs_form="projected",
                      max_steps=200_000)


def small(n=1024):
    """1,024 rays in the x-z plane from 200 m depth; ice below an absorbing air layer."""
    return dict(name="small", medium=ice_with_surface(),
                params=dict(TRACE_DEFAULTS, max_path=2000.0),
                rays=fan_xz(n, 200.0), receivers=None)


def batched(n=1_048_576, seed=2):
    """Isotropic rays from sources at 50..1500 m, two-layer ice, 64 receivers, 3 km paths.

    Break conditions: the 3 km path limit and the amplitude threshold A/A0 < 0.05 of the
    paper's Fig. 1 example (without it, rays grazing the internal boundary cast a secondary
    of near-zero amplitude at every one of thousands of bounces); at most 1,000 attempted
    steps per ray (an ordinary ray needs at most ~330; only rays trapped at grazing incidence
    against the internal boundary reach the cap)."""
    return dict(name="batched", medium=two_layer_ice(),
                params=dict(TRACE_DEFAULTS, max_path=3000.0, min_amp=0.05, max_steps=1_000),
                rays=isotropic_sources(n, seed), receivers=receiver_lattice())


def gridded(n_src=16, per_src=262_144, seed=3, nx=256, ny=256, nz=512):
    """Gridded medium with random perturbations; FP32 stages, tolerance 1e-5."""
    return dict(name="grid", medium=grid_medium(nx, ny, nz, seed=seed),
                params=dict(TRACE_DEFAULTS, tol=1e-5, max_path=3000.0, max_generation=0),
                rays=point_sources(n_src, per_src, seed + 100), receivers=None)


def paths(n=65_536, seed=4):
    """Source-receiver pairs in exponential ice with a reflecting surface."""
    return dict(name="paths", medium=ice_with_surface(),
                params=dict(TRACE_DEFAULTS, max_path=10000.0, max_generation=0),
                pairs=pairs(n, seed), hit_tol=0.1, max_iter=60, max_sol=4)


def fig1(n=1_048_576):
    """The example of the paper's Fig. 1: rays in the x-z plane from 240 m depth (launch
    angles 0..180 deg), the firn-over-ice medium, followed to a propagation time of 5 us;
    rays whose amplitude falls below 0.05 of the initial one are discarded.  Secondaries up to
    generation 8 (the paper shows multiple reflections and states no cap)."""
    return dict(name="fig1", medium=firn_over_ice(),
                params=dict(TRACE_DEFAULTS, max_path=3000.0, max_time=5e-6, min_amp=0.05,
                            max_generation=8),
                rays=fan_xz(n, 240.0), receivers=None)


def spheres(n=1_048_576, seed=7):
    """Rays from sources around the two inclusions of ``ice_with_inclusions``: x uniform in
    -60..210 m, y in +-60 m, depth in 250..550 m, directions uniform on the sphere;
    generations <= 3, 2 km paths, the amplitude cut A/A0 < 0.05."""
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(-60.0, 210.0, n), rng.uniform(-60.0, 60.0, n),
                    rng.uniform(250.0, 550.0, n)])
    return dict(name="spheres", medium=ice_with_inclusions(),
                params=dict(TRACE_DEFAULTS, max_path=2000.0, min_amp=0.05, max_generation=3,
                            max_steps=1000),
                rays=(pos, isotropic_dirs(rng, n), np.ones(n)), receivers=None)


def surfaces(n=1_048_576, seed=9):
    """Rays around the tilted, rough ice surface and the tilted internal boundary of
    ``rough_ice``: sources x, y uniform in +-200 m, depth 20..300 m, directions uniform on the
    sphere; 2 km paths, A/A0 < 0.05, generations <= 3, at most 1000 attempted steps."""
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(-200.0, 200.0, n), rng.uniform(-200.0, 200.0, n),
                    rng.uniform(20.0, 300.0, n)])
    return dict(name="surfaces", medium=rough_ice(),
                params=dict(TRACE_DEFAULTS, max_path=2000.0, min_amp=0.05, max_generation=3,
                            max_steps=1000),
                rays=(pos, isotropic_dirs(rng, n), np.ones(n)), receivers=None)


def surrogate(n_train=4_194_304, n_query=1_048_576, seed=5):
    """Learned surrogate of the path finder: training pairs and queries drawn like ``paths``
    (independent seeds); training labels from the FP32 path finder at hit_tol 0.1 m; inference
    refines to a 5 mm miss and falls back to the path finder at the same tolerance."""
    base = paths(1)
    return dict(name="surrogate", medium=base["medium"], params=base["params"],
                train=pairs(n_train, seed), queries=pairs(n_query, seed + 1),
                label_hit_tol=0.1, hit_tol=0.005, max_iter=60, max_sol=4,
                schedule=dict(epochs=36, batch=8192, lr=4e-3, lr_final=2e-5, seed=seed),
                infer=dict(conf=0.99, refine_tol=0.005, refine_step=1e-3, max_step=0.05,
                           refine_iters=16, deflate=True))


# ---------------------------------------------------------------------------------------
# surrogate network: layer sizes and seeded initial weights (inputs of both sides)
# ---------------------------------------------------------------------------------------

MLP_DIMS = (3, 256, 256, 256, 256, 12)


def mlp_init(seed: int = 0, dims=MLP_DIMS):
    """Seeded initial weights W[l] (in, out) float32, uniform in +-sqrt(6 / fan_in) for the
    hidden layers and +-sqrt(1 / fan_in) for the output layer; zero biases."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for i in range(len(dims) - 1):
        lim = math.sqrt(6.0 / dims[i]) if i < len(dims) - 2 else math.sqrt(1.0 / dims[i])
        W.append(rng.uniform(-lim, lim, (dims[i], dims[i + 1])).astype(np.float32))
        b.append(np.zeros(dims[i + 1], dtype=np.float32))
    return W, b


def mlp_flatten(W, b):
    """Flat float32 parameter vector in the library's order: W0, b0, W1, b1, ..., W4, b4."""
    return np.concatenate([np.concatenate([w.ravel(), c.ravel()]) for w, c in zip(W, b)]).astype(
        np.float32)


def mlp_unflatten(flat, dims=MLP_DIMS):
    W, b, o = [], [], 0
    for i in range(len(dims) - 1):
        n = dims[i] * dims[i + 1]
        W.append(np.asarray(flat[o:o + n], dtype=np.float32).reshape(dims[i], dims[i + 1]))
        o += n
        b.append(np.asarray(flat[o:o + dims[i + 1]], dtype=np.float32))
        o += dims[i + 1]
    return W, b
