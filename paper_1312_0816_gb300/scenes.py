"""Seeded synthetic workloads: detector volumes and track baskets.

This module only *constructs* inputs. It holds none of the navigator's
arithmetic (no distance, safety, transform-of-tracks or reduction code): it
places shapes, draws rotations, and samples track positions and directions.
Both the CUDA path and the CPU oracle consume its arrays, so neither side ever
generates the other's inputs.

Shape parameter conventions (ROOT-style, the paper defers all shape details to
the ROOT geometry library, Sec. 3.1):

* Box  (kind 0): params = (dx, dy, dz, 0, 0)            half-lengths
* Tube (kind 1): params = (rmin, rmax, dz, 0, 0)        radii and half-z
* Cone (kind 2): params = (dz, rmin1, rmax1, rmin2, rmax2), radii 1 at -dz, 2 at +dz
* Tube segment (kind 3): params = (rmin, rmax, dz, sphi, dphi)
* Polycone (kind 4): params = (sphi, dphi, nz, offset, 0); the scene's plane
  table `pdata` holds at `offset` the nz plane positions z (increasing), then
  the nz inner radii, then the nz outer radii (a `Pcon` in a row spec)

A daughter is placed by a rotation R (row-major 3x3, local -> mother) and a
translation t: p_mother = R p_local + t.

Track pools follow the toy-detector protocol of Sec. 3.2: positions fill the
exclusive part of the mother (here: the mother minus a keep-out envelope around
every daughter), directions are isotropic unit vectors.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BOX, TUBE, CONE, TUBS, PCON = 0, 1, 2, 3, 4
KIND_NAMES = {BOX: "box", TUBE: "tube", CONE: "cone", TUBS: "tube segment", PCON: "polycone"}
MAX_PLANES = 32


@dataclasses.dataclass
class Pcon:
    """A polycone: nz planes z[0] < ... < z[nz-1] with radii rmin[k] <= rmax[k],
    cut to the azimuths [sphi, sphi + dphi]."""

    z: tuple
    rmin: tuple
    rmax: tuple
    sphi: float = 0.0
    dphi: float = 2.0 * math.pi

    def planes(self) -> np.ndarray:
        return np.concatenate([np.asarray(self.z, float), np.asarray(self.rmin, float), np.asarray(self.rmax, float)])

    @property
    def nz(self) -> int:
        return len(self.z)


@dataclasses.dataclass
class Scene:
    """One logical volume: a mother shape and its placed daughters."""

    name: str
    mother_kind: int
    mother_params: np.ndarray           # (5,) float64
    kinds: np.ndarray                   # (nd,) int32
    params: np.ndarray                  # (nd, 5) float64
    rot: np.ndarray                     # (nd, 9) float64, row-major local->mother
    trans: np.ndarray                   # (nd, 3) float64
    pdata: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))   # polycone planes

    @property
    def n_daughters(self) -> int:
        return int(self.kinds.shape[0])

    def planes_of(self, row) -> np.ndarray:
        """(3, nz) array z / rmin / rmax of a polycone row."""
        nz, off = int(row[2]), int(row[3])
        return self.pdata[off: off + 3 * nz].reshape(3, nz)

    def identity_mask(self) -> np.ndarray:
        eye = np.eye(3).reshape(9)
        return np.all(self.rot == eye[None, :], axis=1)

    def bounding_radius(self) -> np.ndarray:
        """Radius of a sphere about each daughter's origin enclosing it."""
        p = self.params
        r = np.empty(self.n_daughters)
        for j, k in enumerate(self.kinds):
            if k == BOX:
                r[j] = math.sqrt(p[j, 0] ** 2 + p[j, 1] ** 2 + p[j, 2] ** 2)
            elif k in (TUBE, TUBS):
                r[j] = math.sqrt(p[j, 1] ** 2 + p[j, 2] ** 2)
            elif k == PCON:
                z, _, rx = self.planes_of(p[j])
                r[j] = float(np.sqrt(rx * rx + z * z).max())
            else:
                r[j] = math.sqrt(max(p[j, 2], p[j, 4]) ** 2 + p[j, 0] ** 2)
        return r


@dataclasses.dataclass
class Tracks:
    """A basket in structure-of-arrays form (Sec. 2: contiguous per-field vectors)."""

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def fields(self):
        return (self.x, self.y, self.z, self.dx, self.dy, self.dz)

    def slice(self, a: int, b: int) -> "Tracks":
        return Tracks(*(f[a:b] for f in self.fields()))


# --------------------------------------------------------------------------
# rotations
# --------------------------------------------------------------------------

def euler_zxz(phi: float, theta: float, psi: float) -> np.ndarray:
    """R = Rz(phi) Rx(theta) Rz(psi), row-major (9,)."""
    c1, s1 = math.cos(phi), math.sin(phi)
    c2, s2 = math.cos(theta), math.sin(theta)
    c3, s3 = math.cos(psi), math.sin(psi)
    rz1 = np.array([[c1, -s1, 0.0], [s1, c1, 0.0], [0.0, 0.0, 1.0]])
    rx = np.array([[1.0, 0.0, 0.0], [0.0, c2, -s2], [0.0, s2, c2]])
    rz2 = np.array([[c3, -s3, 0.0], [s3, c3, 0.0], [0.0, 0.0, 1.0]])
    return (rz1 @ rx @ rz2).reshape(9)


def haar_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform (Haar) random rotation from ZXZ Euler angles with cos(theta) uniform."""
    phi = rng.uniform(0.0, 2.0 * math.pi)
    psi = rng.uniform(0.0, 2.0 * math.pi)
    theta = math.acos(rng.uniform(-1.0, 1.0))
    return euler_zxz(phi, theta, psi)


_EYE = np.eye(3).reshape(9)


def _scene(name, mkind, mparams, rows):
    kinds = np.array([r[0] for r in rows], dtype=np.int32)
    params = np.zeros((len(rows), 5))
    pdata = []

    def row_of(spec):
        out = np.zeros(5)
        if isinstance(spec, Pcon):
            off = sum(len(a) for a in pdata)
            pdata.append(spec.planes())
            out[:4] = (spec.sphi, spec.dphi, spec.nz, off)
        else:
            out[: len(spec)] = spec
        return out

    mp = row_of(mparams)
    for j, r in enumerate(rows):
        params[j] = row_of(r[1])
    rot = np.array([r[2] for r in rows], dtype=np.float64).reshape(len(rows), 9)
    trans = np.array([r[3] for r in rows], dtype=np.float64).reshape(len(rows), 3)
    pd = np.concatenate(pdata) if pdata else np.zeros(0)
    return Scene(name, int(mkind), mp, kinds, params, rot, trans, pd)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def box4(seed: int = 0) -> Scene:
    """Box mother (half 100 mm) with four axis-aligned boxes at (+-50, +-50, 0),
    half-lengths U[10, 20] per axis: the 1024-track basket case."""
    rng = np.random.default_rng(seed)
    rows = []
    for cx, cy in ((-50.0, -50.0), (50.0, -50.0), (-50.0, 50.0), (50.0, 50.0)):
        h = rng.uniform(10.0, 20.0, size=3)
        rows.append((BOX, h, _EYE, (cx, cy, 0.0)))
    return _scene("box4", BOX, (100.0, 100.0, 100.0), rows)


def toy40(seed: int = 1) -> Scene:
    """Toy detector after Sec. 3.2 (tube mother, beam-pipe/shield tubes, plates,
    endcap cones) grown to 40 daughters: 8 coaxial tube shells, 24 rotated boxes
    on a ring, 8 coaxial endcap cones."""
    rng = np.random.default_rng(seed)
    rows = []
    for k in range(8):
        rmin = 40.0 + 60.0 * k
        rows.append((TUBE, (rmin, rmin + 30.0, 1000.0), _EYE, (0.0, 0.0, 0.0)))
    for zc in (-600.0, 0.0, 600.0):
        for m in range(8):
            ph = math.radians(45.0 * m)
            h = rng.uniform(10.0, 60.0, size=3)
            rows.append((BOX, h, haar_rotation(rng), (750.0 * math.cos(ph), 750.0 * math.sin(ph), zc)))
    for zc in (-1400.0, -1300.0, -1200.0, -1100.0, 1100.0, 1200.0, 1300.0, 1400.0):
        rows.append((CONE, (40.0, 100.0, 800.0, 150.0, 900.0), _EYE, (0.0, 0.0, zc)))
    return _scene("toy40", TUBE, (0.0, 1000.0, 1500.0), rows)


def toy8(seed: int = 1) -> Scene:
    """The paper's own toy-detector composition (Sec. 3.2): tube mother, two tubes,
    four boxes, two cones."""
    rng = np.random.default_rng(seed)
    rows = [(TUBE, (40.0, 70.0, 1000.0), _EYE, (0.0, 0.0, 0.0)),
            (TUBE, (100.0, 130.0, 1000.0), _EYE, (0.0, 0.0, 0.0))]
    for m in range(4):
        ph = math.radians(90.0 * m)
        h = rng.uniform(10.0, 60.0, size=3)
        rows.append((BOX, h, haar_rotation(rng), (750.0 * math.cos(ph), 750.0 * math.sin(ph), 0.0)))
    for zc in (-1300.0, 1300.0):
        rows.append((CONE, (40.0, 100.0, 800.0, 150.0, 900.0), _EYE, (0.0, 0.0, zc)))
    return _scene("toy8", TUBE, (0.0, 1000.0, 1500.0), rows)


def diff3() -> Scene:
    """Box mother with one rotated box, tube and cone: exercises every shape-parameter
    gradient of the adjoint."""
    rows = [
        (BOX, (15.0, 10.0, 12.0), euler_zxz(0.3, 0.7, 1.1), (-50.0, 40.0, 10.0)),
        (TUBE, (5.0, 20.0, 25.0), euler_zxz(1.3, 0.4, 0.2), (50.0, 40.0, -10.0)),
        (CONE, (20.0, 0.0, 15.0, 5.0, 25.0), euler_zxz(2.1, 1.2, 0.5), (0.0, -50.0, 0.0)),
    ]
    return _scene("diff3", BOX, (100.0, 100.0, 100.0), rows)


def seg4() -> Scene:
    """Box mother (half 100 mm) with four tube segments (Sec. 3.1 lists the
    segmented tube among the ported shapes): a solid quarter-ish wedge, a
    half shell, a shell of 258 degrees (a non-convex wedge) and a whole turn;
    two of them rotated."""
    rows = [
        (TUBS, (0.0, 30.0, 20.0, 0.3, 1.2), euler_zxz(0.4, 0.9, 1.7), (-50.0, -50.0, 0.0)),
        (TUBS, (10.0, 25.0, 15.0, 2.0, math.pi), _EYE, (50.0, -50.0, 0.0)),
        (TUBS, (5.0, 30.0, 20.0, -1.0, 4.5), euler_zxz(2.2, 0.5, 0.3), (-50.0, 50.0, 0.0)),
        (TUBS, (0.0, 20.0, 25.0, 0.0, 2.0 * math.pi), _EYE, (50.0, 50.0, 0.0)),
    ]
    return _scene("seg4", BOX, (100.0, 100.0, 100.0), rows)


def pcon4() -> Scene:
    """Box mother (half 100 mm) with four polycones (Sec. 3.1: connected cone
    and tube sections): a solid bobbin (flanges, slopes and a waist: not
    convex), a shell whose hole widens in the middle, a polycone cut to a
    non-convex wedge with inner apexes on its end planes, and a cone segment
    (two planes, a convex wedge); two of them rotated."""
    rows = [
        (PCON, Pcon((-30.0, -25.0, -20.0, 20.0, 25.0, 30.0), (0.0,) * 6, (25.0, 25.0, 10.0, 10.0, 25.0, 25.0)),
         _EYE, (-50.0, -50.0, 0.0)),
        (PCON, Pcon((-25.0, -5.0, 5.0, 25.0), (5.0, 10.0, 10.0, 5.0), (15.0, 20.0, 20.0, 15.0)),
         euler_zxz(0.4, 0.9, 1.7), (50.0, -50.0, 0.0)),
        (PCON, Pcon((-20.0, 0.0, 20.0), (0.0, 5.0, 0.0), (20.0, 25.0, 15.0), -1.0, 4.2), _EYE, (-50.0, 50.0, 0.0)),
        (PCON, Pcon((-20.0, 20.0), (0.0, 5.0), (20.0, 10.0), 0.5, 1.3), euler_zxz(2.2, 0.5, 0.3),
         (50.0, 50.0, 0.0)),
    ]
    return _scene("pcon4", BOX, (100.0, 100.0, 100.0), rows)


def pconm() -> Scene:
    """A polycone mother with a waist (not convex: z from -100 to 100 mm,
    outer radius 80 mm narrowing to 40 mm at z = 0) holding a tube on the
    axis, two boxes in the flanges and a cone segment."""
    rows = [
        (TUBE, (0.0, 10.0, 60.0), _EYE, (0.0, 0.0, 0.0)),
        (BOX, (15.0, 10.0, 12.0), euler_zxz(0.3, 0.7, 1.1), (45.0, 10.0, -70.0)),
        (BOX, (10.0, 10.0, 10.0), _EYE, (-40.0, -30.0, 70.0)),
        (PCON, Pcon((-10.0, 10.0), (0.0, 5.0), (15.0, 8.0), 0.5, 1.3), euler_zxz(1.0, 0.4, 0.2), (0.0, 55.0, 75.0)),
    ]
    return _scene("pconm", PCON, Pcon((-100.0, -40.0, 0.0, 40.0, 100.0), (0.0,) * 5, (80.0, 80.0, 40.0, 80.0, 80.0)),
                  rows)


def grid512(seed: int = 5) -> Scene:
    """Box mother (half 800 mm) with 512 daughters on an 8x8x8 grid (pitch 200 mm):
    boxes or tubes by a seeded coin, random rotations."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(8):
        for j in range(8):
            for k in range(8):
                c = (-700.0 + 200.0 * i, -700.0 + 200.0 * j, -700.0 + 200.0 * k)
                if rng.uniform() < 0.5:
                    rows.append((BOX, rng.uniform(20.0, 50.0, size=3), haar_rotation(rng), c))
                else:
                    rmin = rng.uniform(0.0, 20.0)
                    rows.append((TUBE, (rmin, rng.uniform(30.0, 60.0), rng.uniform(20.0, 60.0)),
                                 haar_rotation(rng), c))
    return _scene("grid512", BOX, (800.0, 800.0, 800.0), rows)


def cell_volume(seed: int, nd: int, mother_box: bool) -> Scene:
    """One logical volume of the batched workload: nd mixed daughters, one per
    cell of a g^3 grid inscribed in the mother, random kinds and rotations."""
    rng = np.random.default_rng(seed)
    if mother_box:
        mk, mp, half = BOX, (600.0, 600.0, 600.0), 590.0
    else:
        mk, mp, half = TUBE, (0.0, 700.0, 700.0), 700.0 / math.sqrt(2.0) - 5.0
    g = int(math.ceil(nd ** (1.0 / 3.0) - 1e-9))
    while g ** 3 < nd:
        g += 1
    pitch = 2.0 * half / g
    cells = rng.permutation(g ** 3)[:nd]
    rows = []
    for c in cells:
        i, j, k = c // (g * g), (c // g) % g, c % g
        ctr = (-half + pitch * (i + 0.5), -half + pitch * (j + 0.5), -half + pitch * (k + 0.5))
        kind = int(rng.integers(0, 3))
        if kind == BOX:
            prm = rng.uniform(0.1, 0.25, size=3) * pitch
        elif kind == TUBE:
            rmax = rng.uniform(0.15, 0.3) * pitch
            prm = (rng.uniform(0.0, 0.6) * rmax, rmax, rng.uniform(0.1, 0.3) * pitch)
        else:
            r1, r2 = rng.uniform(0.05, 0.3, size=2) * pitch
            prm = (rng.uniform(0.1, 0.3) * pitch, rng.uniform(0.0, 0.6) * r1, r1,
                   rng.uniform(0.0, 0.6) * r2, r2)
        rows.append((kind, prm, haar_rotation(rng), ctr))
    return _scene(f"cell{nd}", mk, mp, rows)


def batched64(seed: int = 3, n_volumes: int = 64, total: int = 1 << 22):
    """64 logical volumes (box / tube mothers alternately, 4..200 daughters each)
    and a list of baskets (volume, size) with sizes log-uniform in [16, 65536],
    drawn until the total reaches `total` tracks."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(4, 201, size=n_volumes)
    vols = [cell_volume(seed * 1000 + v, int(counts[v]), v % 2 == 0) for v in range(n_volumes)]
    baskets = []
    acc = 0
    while acc < total:
        v = int(rng.integers(0, n_volumes))
        size = int(round(math.exp(rng.uniform(math.log(16.0), math.log(65536.0)))))
        size = min(size, total - acc)
        baskets.append((v, size))
        acc += size
    return vols, baskets


SCENES = {"box4": box4, "toy40": toy40, "toy8": toy8, "diff3": diff3, "grid512": grid512, "seg4": seg4,
          "pcon4": pcon4, "pconm": pconm}


# --------------------------------------------------------------------------
# track sampling
# --------------------------------------------------------------------------

def isotropic(rng: np.random.Generator, n: int):
    cz = rng.uniform(-1.0, 1.0, size=n)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=n)
    st = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return st * np.cos(ph), st * np.sin(ph), cz


def _sample_mother(rng, scene: Scene, n: int):
    """Uniform points in the mother's interior, by construction (no test)."""
    mp = scene.mother_params
    if scene.mother_kind == BOX:
        return (rng.uniform(-mp[0], mp[0], n), rng.uniform(-mp[1], mp[1], n),
                rng.uniform(-mp[2], mp[2], n))
    if scene.mother_kind == TUBE:
        rmin, rmax, dz = mp[0], mp[1], mp[2]
        r = np.sqrt(rng.uniform(rmin * rmin, rmax * rmax, n))
        ph = rng.uniform(0.0, 2.0 * math.pi, n)
        return r * np.cos(ph), r * np.sin(ph), rng.uniform(-dz, dz, n)
    if scene.mother_kind == PCON:
        # inside by construction, not uniform in volume: a section, a height
        # in it, a radius between its interpolated radii, an azimuth in the
        # wedge
        z, rn, rx = scene.planes_of(mp)
        k = rng.integers(0, z.shape[0] - 1, n)
        f = rng.uniform(0.0, 1.0, n)
        lo = rn[k] + (rn[k + 1] - rn[k]) * f
        hi = rx[k] + (rx[k + 1] - rx[k]) * f
        r = np.sqrt(rng.uniform(lo * lo, hi * hi))
        ph = mp[0] + mp[1] * rng.uniform(0.0, 1.0, n)
        return r * np.cos(ph), r * np.sin(ph), z[k] + (z[k + 1] - z[k]) * f
    raise ValueError("track sampling supports box, tube and polycone mothers")


def keepout_mask(scene: Scene, x, y, z, margin: float = 1e-6) -> np.ndarray:
    """True where a point lies in the keep-out envelope of some daughter.

    Envelopes are deliberately coarse: an axis-aligned box for unrotated boxes,
    an axis-aligned annulus slab for unrotated tubes/cones, and the bounding
    sphere for every rotated daughter.  The pool therefore covers the exclusive
    part of the mother minus a thin shell around rotated daughters."""
    from scipy.spatial import cKDTree

    n = x.shape[0]
    out = np.zeros(n, dtype=bool)
    ident = scene.identity_mask()
    p = scene.params
    t = scene.trans
    rad = scene.bounding_radius()
    for j in np.nonzero(ident)[0]:
        lx, ly, lz = x - t[j, 0], y - t[j, 1], z - t[j, 2]
        k = scene.kinds[j]
        if k == BOX:
            m = (np.abs(lx) <= p[j, 0] + margin) & (np.abs(ly) <= p[j, 1] + margin) & \
                (np.abs(lz) <= p[j, 2] + margin)
        else:
            if k in (TUBE, TUBS):   # a segment lies inside its whole tube
                rlo, rhi, hz = p[j, 0], p[j, 1], p[j, 2]
            elif k == PCON:         # a polycone lies inside its bounding tube
                zp, rn, rx = scene.planes_of(p[j])
                rlo, rhi, hz = float(rn.min()), float(rx.max()), 0.5 * float(zp[-1] - zp[0])
                lz = lz - 0.5 * float(zp[-1] + zp[0])
            else:
                rlo, rhi, hz = min(p[j, 1], p[j, 3]), max(p[j, 2], p[j, 4]), p[j, 0]
            rr = lx * lx + ly * ly
            lo = max(rlo - margin, 0.0)
            m = (np.abs(lz) <= hz + margin) & (rr <= (rhi + margin) ** 2) & (rr >= lo * lo)
            if rlo - margin <= 0.0:
                m = (np.abs(lz) <= hz + margin) & (rr <= (rhi + margin) ** 2)
        out |= m
    rot_idx = np.nonzero(~ident)[0]
    if rot_idx.size:
        tree = cKDTree(t[rot_idx])
        rmax = float(rad[rot_idx].max()) + margin
        kq = min(8, rot_idx.size)
        pts = np.stack([x, y, z], axis=1)
        dist, idx = tree.query(pts, k=kq, distance_upper_bound=rmax)
        if kq == 1:
            dist, idx = dist[:, None], idx[:, None]
        valid = idx < rot_idx.size
        safe_idx = np.where(valid, idx, 0)
        rj = rad[rot_idx][safe_idx] + margin
        out |= np.any(valid & (dist <= rj), axis=1)
    return out


def sample_tracks(scene: Scene, n: int, seed: int, exclusive: bool = True) -> Tracks:
    """n tracks uniform in the mother (minus daughter keep-out envelopes when
    `exclusive`), isotropic unit directions."""
    rng = np.random.default_rng(seed)
    xs, ys, zs = [], [], []
    have = 0
    while have < n:
        m = max(1024, int((n - have) * 1.5))
        x, y, z = _sample_mother(rng, scene, m)
        if exclusive and scene.n_daughters:
            keep = ~keepout_mask(scene, x, y, z)
            x, y, z = x[keep], y[keep], z[keep]
        xs.append(x)
        ys.append(y)
        zs.append(z)
        have += x.shape[0]
    x = np.concatenate(xs)[:n]
    y = np.concatenate(ys)[:n]
    z = np.concatenate(zs)[:n]
    dx, dy, dz = isotropic(rng, n)
    return Tracks(x.copy(), y.copy(), z.copy(), dx, dy, dz)


def pool_baskets(pool_n: int, basket: int, repeats: int, seed: int):
    """The benchmark protocol of Sec. 3.2: `repeats` baskets of `basket`
    consecutive tracks, each starting at a random offset in a pool."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, pool_n - basket + 1, size=repeats)


def batched_tracks(vols, baskets, seed: int):
    """Concatenated SoA tracks for a basket list; returns Tracks and an int64
    array of (volume, offset, count) rows."""
    parts = []
    rows = []
    off = 0
    for b, (v, size) in enumerate(baskets):
        parts.append(sample_tracks(vols[v], size, seed * 100003 + b))
        rows.append((v, off, size))
        off += size
    fields = [np.concatenate([getattr(p, f) for p in parts]) for f in ("x", "y", "z", "dx", "dy", "dz")]
    return Tracks(*fields), np.array(rows, dtype=np.int64)


# --------------------------------------------------------------------------
# adversarial rays: grazing, edge and corner hits on a chosen daughter
# --------------------------------------------------------------------------

def adversarial_tracks(scene: Scene, n: int, seed: int, jitter: float = 1e-7) -> Tracks:
    """Rays aimed at feature points of randomly chosen daughters: tangent to
    cylinders and cones, at box edges and corners, nearly parallel to faces.
    The target is a constructed point on the feature (with a relative jitter
    of about `jitter`), the start is backed off along the ray by 1..200 mm and
    kept only if it lies well inside the mother and outside every keep-out
    envelope."""
    rng = np.random.default_rng(seed)
    out_p, out_v = [], []
    have = 0
    rounds = 0
    while have < n and rounds < 200:
        rounds += 1
        m = max(4096, 2 * (n - have))
        j = rng.integers(0, scene.n_daughters, size=m)
        kind = scene.kinds[j]
        prm = scene.params[j]
        mode = rng.integers(0, 3, size=m)
        q = np.zeros((m, 3))
        v = np.stack(isotropic(rng, m), axis=1)
        # boxes: corner (mode 0), edge (1), face with a nearly parallel ray (2)
        b = kind == BOX
        if b.any():
            h = prm[b, :3]
            sg = rng.choice([-1.0, 1.0], size=h.shape)
            qb = sg * h
            mb = mode[b]
            free = rng.integers(0, 3, size=qb.shape[0])
            u = rng.uniform(-1.0, 1.0, size=qb.shape)
            rows = np.arange(qb.shape[0])
            e = mb == 1
            qb[rows[e], free[e]] = (u * h)[rows[e], free[e]]
            f = mb == 2
            for ax in range(3):
                sel = f & (free != ax)
                qb[sel, ax] = (u * h)[sel, ax]
            vb = v[b]
            vb[rows[f], free[f]] *= 1e-6
            q[b] = qb
            v[b] = vb
        # polycones: a section; a line tangent to its outer or inner cone
        # (mode 0), a point on that cone (1) or on the rim of one of its planes
        # (2); azimuths in the wedge, half of modes 1 and 2 on a phi face
        pcn = np.nonzero(kind == PCON)[0]
        for i in pcn:
            zp, rn, rx = scene.planes_of(prm[i])
            k = int(rng.integers(0, zp.shape[0] - 1))
            f = float(rng.choice([0.0, 1.0])) if mode[i] == 2 else float(rng.uniform())
            rr = rx if (rng.uniform() < 0.6 or rn[k] + rn[k + 1] == 0.0) else rn
            r = rr[k] + (rr[k + 1] - rr[k]) * f
            zc = zp[k] + (zp[k + 1] - zp[k]) * f
            slope = (rr[k + 1] - rr[k]) / (zp[k + 1] - zp[k])
            fr = float(rng.uniform())
            if mode[i] != 0 and prm[i, 1] < 2.0 * math.pi and rng.uniform() < 0.5:
                fr = float(rng.choice([0.0, 1.0]))
            ph = prm[i, 0] + prm[i, 1] * fr
            radial = np.array([math.cos(ph), math.sin(ph), 0.0])
            q[i] = radial * r + np.array([0.0, 0.0, zc])
            if mode[i] == 0:
                tang = np.array([-math.sin(ph), math.cos(ph), 0.0])
                gen = np.array([slope * radial[0], slope * radial[1], 1.0])
                gen /= np.linalg.norm(gen)
                a = rng.uniform(-1.0, 1.0)
                v[i] = tang * math.sqrt(max(0.0, 1.0 - a * a)) + gen * a
        # tubes, tube segments and cones: tangent lines (mode 0) or rim
        # points (1, 2); on a segment the points lie in its wedge, half of the
        # rim points on the edges of its phi faces
        c = ~b & (kind != PCON)
        if c.any():
            pc = prm[c]
            kc = kind[c]
            mc = mode[c]
            tubelike = (kc == TUBE) | (kc == TUBS)
            hz = np.where(tubelike, pc[:, 2], pc[:, 0])
            zc = np.where(mc == 2, rng.choice([-1.0, 1.0], size=hz.shape) * hz, rng.uniform(-1, 1, size=hz.shape) * hz)
            use_outer = rng.uniform(size=hz.shape) < 0.6
            tube_r = np.where(use_outer | (pc[:, 0] == 0.0), pc[:, 1], pc[:, 0])
            outer_c = use_outer | ((pc[:, 1] + pc[:, 3]) == 0.0)
            r1 = np.where(outer_c, pc[:, 2], pc[:, 1])
            r2 = np.where(outer_c, pc[:, 4], pc[:, 3])
            cone_r = r1 + (r2 - r1) * (zc + hz) / (2.0 * hz)
            slope = np.where(kc == CONE, (r2 - r1) / np.where(kc == CONE, 2.0 * hz, 1.0), 0.0)
            r = np.where(tubelike, tube_r, cone_r)
            ph = rng.uniform(0.0, 2.0 * math.pi, size=hz.shape)
            seg = kc == TUBS
            if seg.any():
                f0, dphi = pc[seg, 3], pc[seg, 4]
                at_face = (mc[seg] != 0) & (rng.uniform(size=f0.shape) < 0.5)
                end = np.where(rng.uniform(size=f0.shape) < 0.5, 0.0, 1.0)
                ph[seg] = f0 + dphi * np.where(at_face, end, rng.uniform(size=f0.shape))
            radial = np.stack([np.cos(ph), np.sin(ph), np.zeros_like(ph)], 1)
            tang = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], 1)
            qc = radial * r[:, None]
            qc[:, 2] = zc
            gen = np.stack([slope * radial[:, 0], slope * radial[:, 1], np.ones_like(ph)], 1)
            gen /= np.linalg.norm(gen, axis=1, keepdims=True)
            a = rng.uniform(-1.0, 1.0, size=hz.shape)
            vt = tang * np.sqrt(np.maximum(0.0, 1.0 - a * a))[:, None] + gen * a[:, None]
            vc = np.where((mc == 0)[:, None], vt, v[c])
            q[c] = qc
            v[c] = vc
        q = q * (1.0 + jitter * rng.uniform(-1.0, 1.0, size=q.shape))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        R = scene.rot[j].reshape(m, 3, 3)
        qw = np.einsum("nij,nj->ni", R, q) + scene.trans[j]
        vw = np.einsum("nij,nj->ni", R, v)
        back = rng.uniform(1.0, 200.0, size=m)
        start = qw - back[:, None] * vw
        mp = scene.mother_params
        if scene.mother_kind == BOX:
            inside = np.all(np.abs(start) < 0.999 * mp[:3], axis=1)
        elif scene.mother_kind == PCON:
            # the tube inscribed in the polycone (its least outer and largest
            # inner radius over its z-range) lies inside it; whole turns only
            zp, rn, rx = scene.planes_of(mp)
            rr = start[:, 0] ** 2 + start[:, 1] ** 2
            inside = (rr < (0.999 * rx.min()) ** 2) & (rr > (1.001 * rn.max()) ** 2) & \
                     (start[:, 2] > zp[0] + 1e-3 * (zp[-1] - zp[0])) & (start[:, 2] < zp[-1] - 1e-3 * (zp[-1] - zp[0]))
            assert mp[1] >= 2.0 * math.pi
        else:
            inside = (start[:, 0] ** 2 + start[:, 1] ** 2 < (0.999 * mp[1]) ** 2) & \
                     (np.abs(start[:, 2]) < 0.999 * mp[2])
        ok = inside & ~keepout_mask(scene, start[:, 0], start[:, 1], start[:, 2])
        out_p.append(start[ok])
        out_v.append(vw[ok])
        have += int(ok.sum())
    if have < n:
        raise RuntimeError("adversarial sampler could not place enough rays")
    P = np.concatenate(out_p)[:n]
    V = np.concatenate(out_v)[:n]
    return Tracks(P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy(), V[:, 0].copy(), V[:, 1].copy(), V[:, 2].copy())


# --------------------------------------------------------------------------
# a tree of logical volumes (final localisation after a step)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class World:
    """A tree of logical volumes.  Volume v's daughter j is an instance of
    volume child[v][j], whose mother solid equals that daughter's solid; the
    frame of the root volume is the frame of the tracks."""

    volumes: list          # Scene per logical volume
    child: list            # per volume: child volume index per daughter
    root: int = 0

    def flat(self) -> dict:
        """The volumes' arrays concatenated; polycone rows point into one
        concatenated plane table."""
        nd = np.array([v.n_daughters for v in self.volumes], dtype=np.int32)
        doff = np.concatenate([[0], np.cumsum(nd)[:-1]]).astype(np.int32)
        mparams, params, pdata, base = [], [], [], 0
        for v in self.volumes:
            mp = v.mother_params.astype(np.float64).copy()
            if v.mother_kind == PCON:
                mp[3] += base
            pr = v.params.astype(np.float64).copy().reshape(-1, 5)
            pr[v.kinds == PCON, 3] += base
            mparams.append(mp)
            params.append(pr)
            pdata.append(np.asarray(v.pdata, dtype=np.float64))
            base += v.pdata.shape[0]
        cat = lambda f, w: (np.concatenate([f(v) for v in self.volumes]) if nd.sum() else np.zeros((0, w)))
        return {
            "mkind": np.array([v.mother_kind for v in self.volumes], dtype=np.int32),
            "mparams": np.stack(mparams),
            "nd": nd, "doff": doff,
            "kinds": np.concatenate([v.kinds for v in self.volumes]).astype(np.int32),
            "params": np.concatenate(params).reshape(-1, 5),
            "pdata": np.concatenate(pdata) if base else np.zeros(0),
            "rot": cat(lambda v: v.rot, 9).reshape(-1, 9).astype(np.float64),
            "trans": cat(lambda v: v.trans, 3).reshape(-1, 3).astype(np.float64),
            "child": np.concatenate([np.asarray(c, dtype=np.int32) for c in self.child]).astype(np.int32),
            "root": int(self.root),
        }

    def check(self):
        for v, vol in enumerate(self.volumes):
            assert len(self.child[v]) == vol.n_daughters
            for j, c in enumerate(self.child[v]):
                cv = self.volumes[c]
                assert cv.mother_kind == vol.kinds[j], (v, j)
                if vol.kinds[j] == PCON:
                    assert np.array_equal(cv.mother_params[:3], vol.params[j, :3]), (v, j)
                    assert np.array_equal(cv.planes_of(cv.mother_params), vol.planes_of(vol.params[j])), (v, j)
                else:
                    assert np.array_equal(cv.mother_params, vol.params[j]), (v, j)


def leaf(kind, params, name="leaf") -> Scene:
    """A logical volume with no daughters (params: a row, or a Pcon)."""
    return _scene(name, kind, params, [])


def _rot_z(phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.array([c, -s, 0.0, s, c, 0.0, 0.0, 0.0, 1.0])


def world_toy(seed: int = 1) -> World:
    """Three levels below a hall: the toy detector of Sec. 3.2 (40 daughters)
    placed in a box hall (half 1600 x 1600 x 2000 mm) beside 4 racks (boxes
    holding a tube); every tube shell of the detector holds 8 sensor boxes,
    every rotated box holds two sub-boxes; cones and the rest are leaves.
    162 placed volumes, non-overlapping by construction."""
    toy = toy40(seed)
    vols, child = [], []

    def add(scene, kids):
        vols.append(scene)
        child.append(list(kids))
        return len(vols) - 1

    sensor = add(leaf(BOX, (8.0, 8.0, 100.0), "sensor"), [])
    cone = add(leaf(CONE, toy.params[32], "endcap"), [])
    rack_tube = add(leaf(TUBE, (0.0, 50.0, 300.0), "rack_tube"), [])
    rack = add(_scene("rack", BOX, (100.0, 100.0, 400.0), [(TUBE, (0.0, 50.0, 300.0), _EYE, (0.0, 0.0, 0.0))]),
               [rack_tube])
    det_kids = []
    for j in range(toy.n_daughters):
        k, p = int(toy.kinds[j]), toy.params[j]
        if k == TUBE:
            mid = 0.5 * (p[0] + p[1])
            rows = []
            for m in range(8):
                ph = math.radians(45.0 * m)
                rows.append((BOX, (8.0, 8.0, 100.0), _rot_z(ph),
                             (mid * math.cos(ph), mid * math.sin(ph), 400.0 * (-1) ** m)))
            sh = _scene(f"shell{j}", TUBE, p[:3], rows)
            det_kids.append(add(sh, [sensor] * 8))
        elif k == BOX:
            h = p[:3]
            sub = add(leaf(BOX, (h[0] / 4, h[1] / 2, h[2] / 2), f"sub{j}"), [])
            rows = [(BOX, (h[0] / 4, h[1] / 2, h[2] / 2), _EYE, (s * h[0] / 2, 0.0, 0.0)) for s in (-1.0, 1.0)]
            det_kids.append(add(_scene(f"box{j}", BOX, h, rows), [sub, sub]))
        else:
            det_kids.append(cone)
    det = add(Scene("detector", toy.mother_kind, toy.mother_params, toy.kinds, toy.params, toy.rot, toy.trans),
              det_kids)
    rows = [(TUBE, toy.mother_params[:3], _EYE, (0.0, 0.0, 0.0))]
    for cx, cy in ((1350.0, 0.0), (-1350.0, 0.0), (0.0, 1350.0), (0.0, -1350.0)):
        rows.append((BOX, (100.0, 100.0, 400.0), _EYE, (cx, cy, 0.0)))
    hall = add(_scene("hall", BOX, (1600.0, 1600.0, 2000.0), rows), [det, rack, rack, rack, rack])
    w = World(vols, child, root=hall)
    w.check()
    return w


def world_pcon() -> World:
    """A box hall (half 400 mm) holding: the polycone vessel of `pconm`
    (rotated; its tube, two boxes and cone segment as leaves), a box holding
    a polycone shell whose wall holds a small box, and a polycone bobbin
    leaf.  Non-overlapping by construction."""
    vols, child = [], []

    def add(scene, kids):
        vols.append(scene)
        child.append(list(kids))
        return len(vols) - 1

    vessel_sc = pconm()
    kids = []
    for j in range(vessel_sc.n_daughters):
        k, row = int(vessel_sc.kinds[j]), vessel_sc.params[j]
        if k == PCON:
            z, rn, rx = vessel_sc.planes_of(row)
            kids.append(add(leaf(PCON, Pcon(tuple(z), tuple(rn), tuple(rx), row[0], row[1]), f"v{j}"), []))
        else:
            kids.append(add(leaf(k, row, f"v{j}"), []))
    vessel = add(vessel_sc, kids)
    wall_box = add(leaf(BOX, (4.0, 4.0, 10.0), "wall_box"), [])
    shell_pc = Pcon((-60.0, -20.0, 20.0, 60.0), (20.0, 30.0, 30.0, 20.0), (40.0, 50.0, 50.0, 40.0))
    shell = add(_scene("pshell", PCON, shell_pc, [(BOX, (4.0, 4.0, 10.0), _EYE, (40.0, 0.0, 0.0))]), [wall_box])
    holder = add(_scene("holder", BOX, (80.0, 80.0, 80.0), [(PCON, shell_pc, euler_zxz(0.3, 0.0, 0.0), (0.0, 0.0, 0.0))]),
                 [shell])
    bob_pc = Pcon((-30.0, -25.0, -20.0, 20.0, 25.0, 30.0), (0.0,) * 6, (25.0, 25.0, 10.0, 10.0, 25.0, 25.0))
    bobbin = add(leaf(PCON, bob_pc, "bobbin"), [])
    rows = [(PCON, Pcon((-100.0, -40.0, 0.0, 40.0, 100.0), (0.0,) * 5, (80.0, 80.0, 40.0, 80.0, 80.0)),
             euler_zxz(0.5, 1.1, 0.2), (-150.0, 0.0, 0.0)),
            (BOX, (80.0, 80.0, 80.0), _EYE, (200.0, 150.0, 0.0)),
            (PCON, bob_pc, euler_zxz(1.2, 0.6, 0.0), (150.0, -200.0, 100.0))]
    hall = add(_scene("phall", BOX, (400.0, 400.0, 400.0), rows), [vessel, holder, bobbin])
    w = World(vols, child, root=hall)
    w.check()
    return w


def world_points(world: World, n: int, seed: int) -> Tracks:
    """n points uniform in the root volume's bounding box (the root is a box
    here), isotropic unit directions."""
    rng = np.random.default_rng(seed)
    r = world.volumes[world.root]
    assert r.mother_kind == BOX
    h = r.mother_params[:3]
    x = rng.uniform(-h[0], h[0], n)
    y = rng.uniform(-h[1], h[1], n)
    z = rng.uniform(-h[2], h[2], n)
    dx, dy, dz = isotropic(rng, n)
    return Tracks(x, y, z, dx, dy, dz)
