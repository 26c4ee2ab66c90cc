"""High-precision crossing of a navigator step's winning surface (test helper).

For a track, its winning solid (mother or daughter) and the surface tag the
oracle reports, this module evaluates in mpmath (212-bit significands) the
exact parameter at which the line p + s d, carried exactly into the solid's
frame, crosses that surface -- the root nearest a given step.  It also
evaluates the same root in plain binary64 arithmetic with a deliberately
different operation order and no error-free tricks (the textbook quadratic
formula), as a stand-in for "some FP64 implementation".  Both serve to pin
the oracle's a-priori error bound of the step; neither is used elsewhere.

Surface tags (as the oracle tags the endpoints of its line sets): box faces
0..5 = -x,+x,-y,+y,-z,+z; 4/5 the -z/+z planes of tubes, cones, tube
segments and polycones (the first / last plane); 6 the outer and 7 the inner
surface of tubes and cones; 8/9 the phi faces at sphi and sphi + dphi; for a
polycone 16 + 2k the outer and 17 + 2k the inner surface of section k.
"""
import math

import mpmath

PREC = 212


def _into(R, t, P, D, mp):
    """x = R^T (P - t), u = R^T D for a row-major placement (R, t), exactly."""
    R = [mp.mpf(float(a)) for a in R]
    t = [mp.mpf(float(a)) for a in t]
    w = [P[k] - t[k] for k in range(3)]
    x = [R[k] * w[0] + R[3 + k] * w[1] + R[6 + k] * w[2] for k in range(3)]
    u = [R[k] * D[0] + R[3 + k] * D[1] + R[6 + k] * D[2] for k in range(3)]
    return x, u


def _frame(scene, j, p, d, mp, chain=()):
    """Local point and direction (exact, mp) of track (p, d) in solid j, after
    the placements of `chain` (root first) have brought it into the scene."""
    P = [mp.mpf(float(a)) for a in p]
    D = [mp.mpf(float(a)) for a in d]
    for R, t in chain:
        P, D = _into(R, t, P, D, mp)
    if j < 0:
        return P, D
    return _into(scene.rot[j], scene.trans[j], P, D, mp)


def _solid(scene, j):
    if j < 0:
        kind, row = int(scene.mother_kind), scene.mother_params
    else:
        kind, row = int(scene.kinds[j]), scene.params[j]
    planes = scene.planes_of(row) if kind == 4 else None
    return kind, [float(a) for a in row], planes


def _surface(kind, row, planes, face, mp):
    """('lin', axis or normal, target) or ('quad', a, b) with the radius line
    R(z) = a + b z (b = 0 for a cylinder), in mp numbers."""
    if kind == 0:
        ax = face // 2
        h = mp.mpf(row[ax])
        return ("plane", ax, -h if face % 2 == 0 else h)
    if face in (4, 5):
        if kind in (1, 3):
            dz = mp.mpf(row[2])
            return ("plane", 2, -dz if face == 4 else dz)
        if kind == 2:
            dz = mp.mpf(row[0])
            return ("plane", 2, -dz if face == 4 else dz)
        z = planes[0]
        return ("plane", 2, mp.mpf(float(z[0] if face == 4 else z[-1])))
    if face in (8, 9):
        sphi, dphi = (row[3], row[4]) if kind == 3 else (row[0], row[1])
        if face == 8:
            a = mp.mpf(sphi)
            n = (-mp.sin(a), mp.cos(a))
        else:
            a = mp.mpf(sphi) + mp.mpf(dphi)
            n = (mp.sin(a), -mp.cos(a))
        return ("phi", n)
    if kind in (1, 3):
        return ("quad", mp.mpf(row[1] if face == 6 else row[0]), mp.mpf(0))
    if kind == 2:
        dz = mp.mpf(row[0])
        r1, r2 = (row[2], row[4]) if face == 6 else (row[1], row[3])
        r1, r2 = mp.mpf(r1), mp.mpf(r2)
        return ("quad", (r1 + r2) / 2, (r2 - r1) / (2 * dz))
    z, rmin, rmax = planes
    k = (face - 16) // 2
    rr = rmax if face % 2 == 0 else rmin
    z0, z1 = mp.mpf(float(z[k])), mp.mpf(float(z[k + 1]))
    r0, r1 = mp.mpf(float(rr[k])), mp.mpf(float(rr[k + 1]))
    b = (r1 - r0) / (z1 - z0)
    return ("quad", r0 - b * z0, b)


def _roots(surf, x, u, mp):
    """Roots of the surface equation along x + s u; (roots, real)."""
    if surf[0] == "plane":
        ax, c = surf[1], surf[2]
        if u[ax] == 0:
            return [], True
        return [(c - x[ax]) / u[ax]], True
    if surf[0] == "phi":
        n = surf[1]
        den = n[0] * u[0] + n[1] * u[1]
        if den == 0:
            return [], True
        return [-(n[0] * x[0] + n[1] * x[1]) / den], True
    a, b = surf[1], surf[2]
    r0 = a + b * x[2]
    rs = b * u[2]
    A = u[0] ** 2 + u[1] ** 2 - rs * rs
    B = x[0] * u[0] + x[1] * u[1] - r0 * rs
    C = x[0] ** 2 + x[1] ** 2 - r0 * r0
    if A == 0:
        return ([-C / (2 * B)] if B != 0 else []), True
    D = B * B - A * C
    if D < 0:
        return [-B / A], False   # no crossing: the closest approach instead
    sq = mp.sqrt(D)
    return [(-B - sq) / A, (-B + sq) / A], True


def exact_root(scene, j, face, p, d, near, chain=()):
    """Exact crossing of surface `face` of solid j (-1 the mother) nearest to
    `near`, as a float, and whether the line really meets the surface.
    `chain`: placements (R, t), root first, that carry the track from the
    world into the scene's frame (a node of a geometry tree)."""
    mp = mpmath.mp
    old = mp.prec
    mp.prec = PREC
    try:
        kind, row, planes = _solid(scene, j)
        x, u = _frame(scene, j, p, d, mp, chain)
        rts, real = _roots(_surface(kind, row, planes, face, mp), x, u, mp)
        if not rts:
            return math.nan, real
        s = min(rts, key=lambda r: abs(r - near))
        return float(s), real
    finally:
        mp.prec = old


def _into_plain(R, t, p, d):
    R = [float(a) for a in R]
    t = [float(a) for a in t]
    w = [p[k] - t[k] for k in range(3)]
    x = [(R[6 + k] * w[2] + R[3 + k] * w[1]) + R[k] * w[0] for k in range(3)]
    u = [(R[6 + k] * d[2] + R[3 + k] * d[1]) + R[k] * d[0] for k in range(3)]
    return x, u


def compose(chain):
    """The placements of a chain (root first) composed into one world
    transform in binary64, as a geometry tree's builder does: G <- G * (R, t)
    (rotation G R, translation G t + t_G)."""
    G = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0]
    tG = [0.0, 0.0, 0.0]
    for R, t in chain:
        R = [float(a) for a in R]
        t = [float(a) for a in t]
        Rc = [G[3 * a] * R[b] + G[3 * a + 1] * R[3 + b] + G[3 * a + 2] * R[6 + b] for a in range(3) for b in range(3)]
        tc = [G[3 * a] * t[0] + G[3 * a + 1] * t[1] + G[3 * a + 2] * t[2] + tG[a] for a in range(3)]
        G, tG = Rc, tc
    return G, tG


def plain_root(scene, j, face, p, d, near, chain=(), composed=False):
    """The same root in plain binary64: transforms summed in the reverse
    order, applied level by level (composed=True: the chain composed into one
    transform first), quadric coefficients and discriminant B*B - A*C without
    error-free products, roots by the cancellation-free textbook pair."""
    kind, row, planes = _solid(scene, j)
    x = [float(a) for a in p]
    u = [float(a) for a in d]
    if composed and chain:
        x, u = _into_plain(*compose(chain), x, u)
    else:
        for R, t in chain:
            x, u = _into_plain(R, t, x, u)
    if j >= 0:
        x, u = _into_plain(scene.rot[j], scene.trans[j], x, u)

    class F:   # binary64 stand-in for the mp namespace of _surface
        pi = math.pi
        mpf = staticmethod(float)
        sin = staticmethod(math.sin)
        cos = staticmethod(math.cos)

    surf = _surface(kind, row, planes, face, F)
    if surf[0] != "quad":
        rts, _ = _roots(surf, x, u, F)
    else:
        a, b = surf[1], surf[2]
        r0 = a + b * x[2]
        rs = b * u[2]
        A = u[0] * u[0] + u[1] * u[1] - rs * rs
        B = x[0] * u[0] + x[1] * u[1] - r0 * rs
        C = x[0] * x[0] + x[1] * x[1] - r0 * r0
        if A == 0.0:
            rts = [-C / (2.0 * B)] if B != 0.0 else []
        else:
            D = max(B * B - A * C, 0.0)
            q = -(B + math.copysign(math.sqrt(D), B))
            rts = [q / A] + ([C / q] if q != 0.0 else [])
    if not rts:
        return math.nan
    return min(rts, key=lambda r: abs(r - near))
