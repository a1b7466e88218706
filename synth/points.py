"""Seeded point-cloud and right-hand-side generators (no solver arithmetic)."""
import numpy as np


def cube(n, seed):
    """n points uniform in the unit cube [0,1]^3 (Section IV workload)."""
    return np.random.default_rng(seed).random((n, 3))


def _unit_vectors(rng, n):
    g = rng.standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def sphere_surface(n, rng):
    return _unit_vectors(rng, n)


def line(n, seed):
    """n points uniform on the segment [0,1] x {0} x {0}, sorted (1-D
    geometry, where weak admissibility gives the HSS structure)."""
    x = np.sort(np.random.default_rng(seed).random(n))
    return np.stack([x, np.zeros(n), np.zeros(n)], 1)


def sphere_ball(n, seed):
    """Half the points uniform on the unit sphere, half uniform in the ball."""
    rng = np.random.default_rng(seed)
    ns = n // 2
    surf = _unit_vectors(rng, ns)
    dirs = _unit_vectors(rng, n - ns)
    rad = rng.random(n - ns) ** (1.0 / 3.0)
    return np.concatenate([surf, dirs * rad[:, None]])


def cube_surface(n, rng):
    """Area-uniform points on the surface of the unit cube."""
    face = rng.integers(0, 6, n)
    uv = rng.random((n, 2))
    p = np.empty((n, 3))
    ax = face // 2
    side = (face % 2).astype(float)
    for a in range(3):
        sel = ax == a
        others = [b for b in range(3) if b != a]
        p[sel, a] = side[sel]
        p[sel, others[0]] = uv[sel, 0]
        p[sel, others[1]] = uv[sel, 1]
    return p


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoid_surface(n, rng, axes):
    """Area-uniform points on an axis-aligned ellipsoid surface (rejection on
    the sphere map with acceptance proportional to the local area element)."""
    a, b, c = axes
    out = []
    need = n
    gmax = max(b * c, a * c, a * b)
    while need > 0:
        u = _unit_vectors(rng, 2 * need + 16)
        g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        keep = rng.random(len(u)) * gmax < g
        u = u[keep][:need]
        out.append(u * np.array([a, b, c]))
        need -= len(u)
    return np.concatenate(out)


def torus_surface(n, rng, R, r):
    """Area-uniform points on a torus (acceptance (R + r cos v) / (R + r))."""
    out = []
    need = n
    while need > 0:
        m = 2 * need + 16
        u = rng.random(m) * 2 * np.pi
        v = rng.random(m) * 2 * np.pi
        keep = rng.random(m) * (R + r) < R + r * np.cos(v)
        u, v = u[keep][:need], v[keep][:need]
        w = R + r * np.cos(v)
        out.append(np.stack([w * np.cos(u), w * np.sin(u), r * np.sin(v)], 1))
        need -= len(u)
    return np.concatenate(out)


def _ellipsoid_area(a, b, c):
    p = 1.6075
    return 4 * np.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)


def surface_union(n, seed, n_ell=16, n_tor=16):
    """Union of random ellipsoid and torus surfaces in [0,4]^3; points are
    allotted to components in proportion to their area."""
    rng = np.random.default_rng(seed)
    comps = []
    for k in range(n_ell + n_tor):
        centre = rng.random(3) * 4.0
        rot = _rotation(rng)
        if k < n_ell:
            axes = 0.2 + 0.6 * rng.random(3)
            area = _ellipsoid_area(*axes)
            comps.append(("e", centre, rot, tuple(axes), area))
        else:
            R = 0.3 + 0.5 * rng.random()
            r = 0.05 + (R / 2 - 0.05) * rng.random()
            comps.append(("t", centre, rot, (R, r), 4 * np.pi ** 2 * R * r))
    areas = np.array([c[4] for c in comps])
    counts = np.floor(n * areas / areas.sum()).astype(int)
    counts[np.argmax(areas)] += n - counts.sum()
    pts = []
    for c, cnt in zip(comps, counts):
        if c[0] == "e":
            p = ellipsoid_surface(cnt, rng, c[3])
        else:
            p = torus_surface(cnt, rng, *c[3])
        pts.append(p @ c[2].T + c[1])
    return np.concatenate(pts)


def batched_problems(n_problems=64, base_seed=100, n_min=2048, n_max=65536):
    """Independent problems: N log-uniform in [n_min, n_max]; geometry drawn
    from cube surface / sphere surface / ellipsoid surface."""
    probs = []
    for p in range(n_problems):
        rng = np.random.default_rng(base_seed + p)
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        geo = int(rng.integers(0, 3))
        if geo == 0:
            x = cube_surface(n, rng)
        elif geo == 1:
            x = sphere_surface(n, rng)
        else:
            x = ellipsoid_surface(n, rng, tuple(0.5 + 1.5 * rng.random(3)))
        nrhs = int(rng.integers(1, 257))
        probs.append(dict(points=x, nrhs=nrhs, geometry=("cube", "sphere", "ellipsoid")[geo]))
    return probs


def rhs(n, nrhs, seed):
    """Right-hand sides ~ N(0,1), column-major (n x nrhs)."""
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((n, nrhs)))


def workload(name, scale=1.0):
    """Named workloads.  ``scale`` < 1 shrinks N (for quick checks) keeping
    the geometry and kernel."""
    def sz(n):
        return max(64, int(n * scale))
    if name == "cube4k":
        return dict(points=cube(sz(4096), 0), kernel="laplace", leaf=256, eta=1.0, tol=1e-8,
                    max_rank=128, rhs_seed=1)
    if name == "sphereball64k":
        return dict(points=sphere_ball(sz(65536), 2), kernel="yukawa", leaf=256, eta=1.0,
                    tol=1e-10, max_rank=128, rhs_seed=3)
    if name == "surfaces1m":
        return dict(points=surface_union(sz(1 << 20), 4), kernel="laplace", leaf=256, eta=1.0,
                    tol=1e-6, max_rank=128, rhs_seed=40)
    if name == "matern256k":
        return dict(points=cube(sz(262144), 5), kernel="matern32", leaf=256, eta=1.0, tol=1e-8,
                    max_rank=128, rhs_seed=50)
    raise KeyError(name)
