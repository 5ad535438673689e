"""Seeded synthetic workloads shared by the CUDA path and the CPU oracle.

This module only *describes* problems: multi-patch geometries (spline control
points), degrees, element counts, Lame parameters, Dirichlet faces and seeded
random coefficient fields.  It contains none of the solver's arithmetic
(no basis evaluation, quadrature, assembly or linear algebra), so the CUDA
library and the oracle each build everything else on their own.

Layout conventions (Section 2.2, colexicographic ordering):
  * patch k has n_l = nel_l + p basis functions per direction l (open uniform
    knots, single interior knots, i.e. C^{p-1} splines);
  * control points are stored as ``ctrl[k]`` with shape (n3, n2, n1, d) in 3D
    and (n2, n1, d) in 2D, so that i1 is the fastest index;
  * a torn vector stacks patches, each patch stacks its d components, each
    component is an n3*n2*n1 block with i1 fastest;
  * faces are numbered f = 2*l + side (l = parametric direction, side 0 is
    eta_l = 0 and side 1 is eta_l = 1).

Geometry is defined by evaluating a map at the Greville abscissae of each
patch (the spline geometry *is* the problem).  Patches sharing a face get
bit-identical control points on it, so interfaces are watertight.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

STEEL_LAMBDA = 0.3 / 0.52   # E = 1, nu = 0.3 (Section 6)
STEEL_MU = 1.0 / 2.6


@dataclass
class Problem:
    """A conforming multi-patch elasticity problem (Sections 2-3)."""
    name: str
    dim: int
    degree: np.ndarray              # [npatch] int32
    nel: np.ndarray                 # [npatch, dim] int32
    ctrl: list                      # per patch float64 array, see module doc
    lame: np.ndarray                # [npatch, 2] float64: (lambda_k, mu_k)
    dirichlet_face: np.ndarray      # [npatch, 2*dim] uint8
    global_index: list = field(default_factory=list)  # per patch int64 node ids
    grid: tuple = ()                # patches per direction (structured layouts)
    # nested non-conforming interfaces (Section 2): (coarse patch, its face,
    # fine patch, its face), face = 2*direction + side; the fine face's knot
    # vectors refine the coarse face's in the same tangential order
    nested: list = field(default_factory=list)

    @property
    def npatch(self) -> int:
        return int(self.degree.shape[0])

    def n(self, k: int) -> tuple:
        """Basis counts (n1, n2[, n3]) of patch k."""
        return tuple(int(self.nel[k, l] + self.degree[k]) for l in range(self.dim))

    def ndof_patch(self, k: int) -> int:
        return self.dim * int(np.prod(self.n(k)))

    @property
    def ndof(self) -> int:
        return sum(self.ndof_patch(k) for k in range(self.npatch))

    def offsets(self) -> np.ndarray:
        off = np.zeros(self.npatch + 1, dtype=np.int64)
        for k in range(self.npatch):
            off[k + 1] = off[k] + self.ndof_patch(k)
        return off

    def ctrl_flat(self) -> np.ndarray:
        """All control points concatenated, [patch][i3][i2][i1][dim]."""
        return np.concatenate([c.reshape(-1) for c in self.ctrl]).astype(np.float64)


def _greville(nel: int, p: int) -> np.ndarray:
    """Knot averages of the open uniform knot vector (geometry placement only)."""
    knots = np.concatenate([np.zeros(p + 1), np.arange(1, nel) / nel, np.ones(p + 1)])
    n = nel + p
    g = np.array([knots[i + 1:i + p + 1].mean() for i in range(n)])
    g[0], g[-1] = 0.0, 1.0
    return g


def _patch_params(t0: float, t1: float, nel: int, p: int) -> np.ndarray:
    g = _greville(nel, p)
    x = t0 + (t1 - t0) * g
    x[0], x[-1] = t0, t1          # exact shared face coordinates
    return x


def _structured(name, dim, grid, nel_cols, p_of, geom, rng_geo=None, jitter=0.0,
                lame=(STEEL_LAMBDA, STEEL_MU)):
    """Structured grid of patches over the global parameter box [0,1]^dim.

    nel_cols[l][q] is the element count of column q in direction l (conforming),
    p_of is the common degree, geom maps global parameters (..., dim) to space.
    """
    npatch = int(np.prod(grid))
    breaks = [np.array([q / grid[l] for q in range(grid[l] + 1)]) for l in range(dim)]
    for l in range(dim):
        breaks[l][-1] = 1.0
    # global node lattice offsets per direction (for continuous random fields)
    goff = []
    for l in range(dim):
        o = [0]
        for q in range(grid[l]):
            o.append(o[-1] + nel_cols[l][q] + p_of - 1)
        goff.append(o)
    gsize = [goff[l][-1] + 1 for l in range(dim)]

    degree = np.full(npatch, p_of, dtype=np.int32)
    nel = np.zeros((npatch, dim), dtype=np.int32)
    ctrl, gidx = [], []
    dface = np.zeros((npatch, 2 * dim), dtype=np.uint8)
    for k in range(npatch):
        q = []
        r = k
        for l in range(dim):
            q.append(r % grid[l])
            r //= grid[l]
        params = []
        for l in range(dim):
            ne = nel_cols[l][q[l]]
            nel[k, l] = ne
            params.append(_patch_params(breaks[l][q[l]], breaks[l][q[l] + 1], ne, p_of))
            dface[k, 2 * l] = 1 if q[l] == 0 else 0
            dface[k, 2 * l + 1] = 1 if q[l] == grid[l] - 1 else 0
        mesh = np.meshgrid(*params[::-1], indexing="ij")       # (n3, n2, n1) order
        pts = np.stack(mesh[::-1], axis=-1)                     # [..., l] = eta_l
        x = geom(pts)
        if jitter > 0.0:
            inner = tuple(slice(1, -1) for _ in range(dim))
            hs = np.array([(breaks[l][q[l] + 1] - breaks[l][q[l]]) / nel[k, l]
                           for l in range(dim)])
            sub = x[inner]
            delta = rng_geo.uniform(-jitter, jitter, size=sub.shape) * hs
            x = x.copy()
            x[inner] = sub + delta
        ctrl.append(np.ascontiguousarray(x, dtype=np.float64))
        ranges = [np.arange(goff[l][q[l]], goff[l][q[l]] + nel[k, l] + p_of)
                  for l in range(dim)]
        gm = np.meshgrid(*ranges[::-1], indexing="ij")
        gid = np.zeros(gm[0].shape, dtype=np.int64)
        stride = 1
        for l in range(dim):
            gid += gm[dim - 1 - l] * stride
            stride *= gsize[l]
        gidx.append(gid)
    lam = np.tile(np.array(lame, dtype=np.float64), (npatch, 1))
    return Problem(name=name, dim=dim, degree=degree, nel=nel, ctrl=ctrl, lame=lam,
                   dirichlet_face=dface, global_index=gidx, grid=tuple(grid))


def unit_box(dim, grid, p, nel, *, jitter=0.0, seed=0, name=None):
    """[0,1]^dim split into `grid` identity-mapped patches (optionally jittered
    at control points that lie on no patch face)."""
    ss = np.random.SeedSequence(seed).spawn(3)
    rng_geo = np.random.default_rng(ss[0])
    nel_cols = [[nel] * grid[l] for l in range(dim)]
    return _structured(name or f"box{dim}d_{'x'.join(map(str, grid))}_p{p}_nel{nel}",
                       dim, grid, nel_cols, p, lambda e: e.copy(), rng_geo, jitter)


def quarter_annulus(grid=(6, 4, 3), p=3, nel=24, *, nel_cols=None, name=None):
    """Thick quarter annulus: radius 1..2, angle 0..pi/2, height 0..1.
    Direction 1 is the angle, 2 the radius, 3 the height."""
    def geom(e):
        th = 0.5 * math.pi * e[..., 0]
        r = 1.0 + e[..., 1]
        return np.stack([r * np.sin(th), r * np.cos(th), e[..., 2]], axis=-1)
    if nel_cols is None:
        nel_cols = [[nel] * grid[l] for l in range(3)]
    return _structured(name or f"annulus_p{p}", 3, grid, nel_cols, p, geom)


def twisted_box(grid=(8, 8, 4), p=4, nel=48, name=None):
    """Unit cube twisted by (pi/4)*z about the axis x = y = 1/2."""
    def geom(e):
        th = 0.25 * math.pi * e[..., 2]
        c, s = np.cos(th), np.sin(th)
        x, y = e[..., 0] - 0.5, e[..., 1] - 0.5
        return np.stack([0.5 + c * x - s * y, 0.5 + s * x + c * y, e[..., 2]], axis=-1)
    nel_cols = [[nel] * grid[l] for l in range(3)]
    return _structured(name or f"twist_p{p}_nel{nel}", 3, grid, nel_cols, p, geom)


def nested_box(dim=3, nels=(4, 8, 16), p=2, name=None) -> Problem:
    """The paper's non-conforming test layout (Section 6): the box
    (0,1) x (0,len(nels)) [x (0,1)] split along direction 2 into unit patches
    with nels[k] elements per direction in patch k, identity-mapped (the
    control points are the Greville abscissae, so each fine interface net is
    the knot-inserted coarse one).  Dirichlet conditions on the whole outer
    boundary; consecutive patches meet on a nested interface when their
    element counts divide one another.  Node ids are per patch (no node is
    shared), so body-force coefficient fields are per patch."""
    npatch = len(nels)
    degree = np.full(npatch, p, dtype=np.int32)
    nel = np.zeros((npatch, dim), dtype=np.int32)
    ctrl, gidx, nested = [], [], []
    dface = np.zeros((npatch, 2 * dim), dtype=np.uint8)
    base = 0
    for k, ne in enumerate(nels):
        nel[k, :] = ne
        params = [_patch_params(0.0, 1.0, ne, p) for _ in range(dim)]
        params[1] = params[1] + k
        mesh = np.meshgrid(*params[::-1], indexing="ij")
        ctrl.append(np.ascontiguousarray(np.stack(mesh[::-1], axis=-1), dtype=np.float64))
        n = ne + p
        gidx.append(base + np.arange(n ** dim, dtype=np.int64).reshape((n,) * dim))
        base += n ** dim
        for l in range(dim):
            for side in range(2):
                outer = l != 1 or (side == 0 and k == 0) or (side == 1 and k == npatch - 1)
                dface[k, 2 * l + side] = 1 if outer else 0
    for k in range(npatch - 1):
        a, b = nels[k], nels[k + 1]
        if a == b:
            continue
        if b % a == 0:
            nested.append((k, 3, k + 1, 2))
        elif a % b == 0:
            nested.append((k + 1, 2, k, 3))
        else:
            raise ValueError("consecutive element counts must divide one another")
    lam = np.tile(np.array((STEEL_LAMBDA, STEEL_MU), dtype=np.float64), (npatch, 1))
    return Problem(name=name or f"nested{dim}d_p{p}_" + "_".join(map(str, nels)), dim=dim,
                   degree=degree, nel=nel, ctrl=ctrl, lame=lam, dirichlet_face=dface,
                   global_index=gidx, grid=(1, npatch) + (1,) * (dim - 2), nested=nested)


def with_neumann(prob: Problem, faces, name=None) -> Problem:
    """Copy of a structured problem whose outer faces `faces` (parametric face
    indices f = 2*l + side: direction l, side 0 = lower, 1 = upper) carry the
    natural (zero-traction) condition instead of the homogeneous Dirichlet
    one.  Only the Dirichlet flags change."""
    import dataclasses
    df = prob.dirichlet_face.copy()
    for f in faces:
        df[:, f] = 0
    return dataclasses.replace(prob, dirichlet_face=df,
                               name=name or f"{prob.name}-neumann{''.join(map(str, faces))}")


NEL_CHOICES = (12, 16, 24, 32, 48)
P_CHOICES = (2, 3, 4, 5)


def config(name: str, seed: int = 0) -> Problem:
    """The paper-shaped workloads.

    C1  2D unit square, 2x2 patches, p=2, 8x8 elements, identity maps.
    C2  unit cube, 4x4x4 patches, p=3, 16^3 elements, interior jitter 10% of h.
    C3  quarter annulus 6x4x3 patches, element counts drawn per column from
        {12,16,24,32,48}, one degree drawn from {2,3,4,5} (conforming draws).
    C4  quarter annulus 6x4x3 patches, p=3, 24^3 elements.
    C5  twisted box 8x8x4 patches, p=4, 48^3 elements.
    Small variants (``*-small``, ``*-mid``) keep the geometry kind at oracle-friendly
    sizes; ``C2-quarter`` and ``C3-quarter`` hold a few full-size patches of C2 / C3.
    """
    if name == "C1":
        return unit_box(2, (2, 2), 2, 8, name="C1")
    if name == "C2":
        return unit_box(3, (4, 4, 4), 3, 16, jitter=0.1, seed=seed, name="C2")
    if name in ("C3", "C3-quarter"):
        rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(3)[1])
        grid = (6, 4, 3)
        cols = [[int(rng.choice(NEL_CHOICES)) for _ in range(grid[l])] for l in range(3)]
        p = int(rng.choice(P_CHOICES))
        if name == "C3-quarter":
            # nine of C3's patches, one per distinct (direction 1, direction 2)
            # column width, in one column of direction 3
            firsts = [sorted({c: i for i, c in reversed(list(enumerate(cols[l])))}.values())
                      for l in range(2)]
            sub = [[cols[0][i] for i in firsts[0]], [cols[1][i] for i in firsts[1]], cols[2][:1]]
            return quarter_annulus(tuple(len(c) for c in sub), p, nel_cols=sub, name=name)
        return quarter_annulus(grid, p, nel_cols=cols, name="C3")
    if name == "C4":
        return quarter_annulus((6, 4, 3), 3, 24, name="C4")
    if name == "C5":
        return twisted_box((8, 8, 4), 4, 48, name="C5")
    # oracle-sized variants of the same geometry kinds
    if name == "C2-small":
        return unit_box(3, (2, 2, 2), 3, 4, jitter=0.1, seed=seed, name=name)
    if name == "C2-quarter":   # C2 patches (p=3, 16^3 elements), 2x2x3 of them
        return unit_box(3, (2, 2, 3), 3, 16, jitter=0.1, seed=seed, name=name)
    if name == "C2-mid":
        return unit_box(3, (3, 3, 3), 3, 6, jitter=0.1, seed=seed, name=name)
    if name == "C3-mid":   # uneven columns at C3's degree, oracle-sized
        return quarter_annulus((2, 2, 1), 4, nel_cols=[[4, 6], [4, 6], [4]], name=name)
    if name == "C4-small":
        return quarter_annulus((3, 2, 2), 3, 3, name=name)
    if name == "C5-small":
        return twisted_box((2, 2, 2), 4, 3, name=name)
    if name == "C5-mid":   # C5 patches (p=4, 48^3 elements), 2x2x2 of them
        return twisted_box((2, 2, 2), 4, 48, name=name)
    if name == "C1-small":
        return unit_box(2, (2, 2), 2, 3, name=name)
    if name == "NC-small":   # nested interfaces, 2D, oracle-sized
        return nested_box(2, (2, 4, 8), 2, name=name)
    if name == "NC3-small":  # nested interfaces, 3D, oracle-sized
        return nested_box(3, (1, 2, 4), 2, name=name)
    if name == "NC3":        # the paper's non-conforming test (4, 8, 16 elements), p = 2
        return nested_box(3, (4, 8, 16), 2, name=name)
    raise KeyError(name)


def body_force_coeffs(prob: Problem, seed: int = 0) -> list:
    """Uniform[-1,1] nodal coefficients of a continuous body force field, one
    value per *global* node and component.  Returns per patch arrays shaped
    [dim, n3, n2, n1] (torn copies of the same global field)."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(3)[2])
    gmax = max(int(g.max()) for g in prob.global_index) + 1
    field_ = rng.uniform(-1.0, 1.0, size=(gmax, prob.dim))
    out = []
    for k in range(prob.npatch):
        c = field_[prob.global_index[k].reshape(-1)]            # [N, dim]
        out.append(np.ascontiguousarray(c.T.reshape((prob.dim,) + prob.global_index[k].shape)))
    return out


def torn_random(prob: Problem, seed: int, nrhs: int = 1) -> np.ndarray:
    """A seeded uniform[-1,1] vector in the torn space, [nrhs, N_dof]."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(3)[2])
    return rng.uniform(-1.0, 1.0, size=(nrhs, prob.ndof))


def fd_batch_shapes(seed: int = 0, npatch: int = 72) -> list:
    """Independent per-patch (n1, n2, n3, p) draws for the uneven batched FD
    workload (n_l = nel_l + p with nel_l from {12,...,48}, p from {2,...,5})."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(3)[1])
    shapes = []
    for _ in range(npatch):
        p = int(rng.choice(P_CHOICES))
        ne = [int(rng.choice(NEL_CHOICES)) for _ in range(3)]
        shapes.append((ne[0] + p, ne[1] + p, ne[2] + p, p))
    return shapes
