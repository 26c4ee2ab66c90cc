"""Pins of the oracle's geometry tree: node numbering, Locate, and the step
followed by final localisation (entering a daughter, leaving into the
parent, entering a touching sibling, leaving the root), on hand-built trees
whose answers are exact, plus invariants on the toy world."""
import numpy as np
import pytest

from helpers import tracks_from
from paper_1312_0816_gb300 import scenes

EYE = np.eye(3).reshape(9)


def world(volumes, child, root=0):
    w = scenes.World(volumes, child, root)
    w.check()
    return w


def vol(kind, params, rows, name="v"):
    if not rows:
        return scenes.leaf(kind, params, name)
    return scenes._scene(name, kind, params, rows)


def nested_boxes():
    """world box 1000 > A box 100 at the origin > B box 10 at (50, 0, 0)."""
    B = vol(0, (10.0, 10.0, 10.0), [], "B")
    A = vol(0, (100.0, 100.0, 100.0), [(0, (10.0, 10.0, 10.0), EYE, (50.0, 0.0, 0.0))], "A")
    W = vol(0, (1000.0, 1000.0, 1000.0), [(0, (100.0, 100.0, 100.0), EYE, (0.0, 0.0, 0.0))], "W")
    return world([W, A, B], [[1], [2], []])


def walk(orc, w, p, d, steps):
    p = np.array(p, dtype=float)
    d = np.array(d, dtype=float)
    node = orc.world_locate(w, tracks_from(p, d))[0]
    out = [int(node)]
    seq = []
    blocked = np.array([-1], dtype=np.int32)
    for _ in range(steps):
        s, nn, blocked = orc.world_step(w, tracks_from(p, d), np.array([node], dtype=np.int32), blocked)
        seq.append((float(s[0]), int(nn[0])))
        if nn[0] < 0:
            break
        p = p + s[0] * d
        node = nn[0]
    return out[0], seq


def test_node_numbering_is_breadth_first(orc):
    leafb = vol(0, (1.0, 1.0, 1.0), [])
    mid = vol(0, (10.0, 10.0, 10.0), [(0, (1.0, 1.0, 1.0), EYE, (-5.0, 0, 0)), (0, (1.0, 1.0, 1.0), EYE, (5.0, 0, 0))])
    top = vol(0, (100.0, 100.0, 100.0), [(0, (10.0, 10.0, 10.0), EYE, (-50.0, 0, 0)),
                                         (0, (10.0, 10.0, 10.0), EYE, (50.0, 0, 0))])
    w = world([top, mid, leafb], [[1, 1], [2, 2], []])
    t = orc.world_nodes(w)
    assert list(t["lv"]) == [0, 1, 1, 2, 2, 2, 2]
    assert list(t["parent"]) == [-1, 0, 0, 1, 1, 2, 2]
    assert list(t["slot"]) == [-1, 0, 1, 0, 1, 0, 1]
    assert list(t["first"]) == [1, 3, 5, 7, 7, 7, 7]


def test_nested_boxes_walk(orc):
    w = nested_boxes()
    start, seq = walk(orc, w, (-500.0, 0.0, 0.0), (1.0, 0.0, 0.0), 8)
    assert start == 0
    # world -> A (400), A -> B (140), B -> A (20), A -> world (40), leave (900)
    assert seq == [(400.0, 1), (140.0, 2), (20.0, 1), (40.0, 0), (900.0, -1)]


def test_locate(orc):
    w = nested_boxes()
    p = np.array([[50.0, 0, 0], [60.0, 10.0, 10.0], [61.0, 0, 0], [0.0, 0, 0], [500.0, 0, 0], [1000.0, 0, 0],
                  [1000.5, 0, 0], [np.nan, 0, 0]])
    node = orc.world_locate(w, tracks_from(p, np.tile([1.0, 0, 0], (len(p), 1))))
    # closed solids: a point on B's corner is in B; on the world's face, in the world
    assert list(node) == [2, 2, 1, 1, 0, 0, -1, -2]


def test_touching_siblings(orc):
    """Leaving A through a face it shares with C enters C directly."""
    A = vol(0, (10.0, 10.0, 10.0), [], "A")
    C = vol(0, (10.0, 10.0, 10.0), [], "C")
    W = vol(0, (1000.0, 1000.0, 1000.0), [(0, (10.0, 10.0, 10.0), EYE, (-10.0, 0.0, 0.0)),
                                          (0, (10.0, 10.0, 10.0), EYE, (10.0, 0.0, 0.0))], "W")
    w = world([W, A, C], [[1, 2], [], []])
    start, seq = walk(orc, w, (-15.0, 0.0, 0.0), (1.0, 0.0, 0.0), 4)
    assert start == 1
    assert seq[0] == (15.0, 2)
    assert seq[1] == (20.0, 0)
    # the other way: C -> A
    start, seq = walk(orc, w, (15.0, 3.0, 0.0), (-1.0, 0.0, 0.0), 2)
    assert start == 2 and seq[0] == (15.0, 1)


def test_daughter_on_the_mother_face(orc):
    """A touches the world's +x face: leaving A there lands on the world's
    (closed) boundary, inside the world; the next step is 0 and leaves."""
    A = vol(0, (100.0, 100.0, 100.0), [], "A")
    W = vol(0, (1000.0, 1000.0, 1000.0), [(0, (100.0, 100.0, 100.0), EYE, (900.0, 0.0, 0.0))], "W")
    w = world([W, A], [[1], []])
    start, seq = walk(orc, w, (950.0, 0.0, 0.0), (1.0, 0.0, 0.0), 3)
    assert start == 1
    assert seq == [(50.0, 0), (0.0, -1)]


def test_rotated_tube_and_entry_into_grandchild(orc):
    """A tube whose axis is the world x axis (rotation about y by 90 deg)
    holding a box at its local +z end; a ray along x goes world -> tube ->
    box -> tube -> world."""
    Ry = np.array([0.0, 0.0, 1.0, 0.0, 1.0, 0.0, -1.0, 0.0, 0.0])   # local z -> world x
    box = vol(0, (5.0, 5.0, 10.0), [], "box")
    tube = vol(1, (0.0, 50.0, 100.0), [(0, (5.0, 5.0, 10.0), EYE, (0.0, 0.0, 80.0))], "tube")
    W = vol(0, (1000.0, 1000.0, 1000.0), [(1, (0.0, 50.0, 100.0), Ry, (0.0, 0.0, 0.0))], "W")
    w = world([W, tube, box], [[1], [2], []])
    start, seq = walk(orc, w, (-500.0, 0.0, 0.0), (1.0, 0.0, 0.0), 6)
    assert start == 0
    steps = [s for s, _ in seq]
    nodes = [n for _, n in seq]
    assert nodes == [1, 2, 1, 0, -1]
    assert np.allclose(steps, [400.0, 170.0, 20.0, 10.0, 900.0], rtol=0, atol=1e-12)


def test_exit_through_grandparent(orc):
    """B touches A's face, which lies inside the world: leaving B there
    climbs to A, whose closed solid holds the point, so the track is in A;
    one more zero step leaves A into the world."""
    B = vol(0, (10.0, 10.0, 10.0), [], "B")
    A = vol(0, (100.0, 100.0, 100.0), [(0, (10.0, 10.0, 10.0), EYE, (90.0, 0.0, 0.0))], "A")
    W = vol(0, (1000.0, 1000.0, 1000.0), [(0, (100.0, 100.0, 100.0), EYE, (0.0, 0.0, 0.0))], "W")
    w = world([W, A, B], [[1], [2], []])
    start, seq = walk(orc, w, (95.0, 0.0, 0.0), (1.0, 0.0, 0.0), 3)
    assert start == 2
    assert seq[:3] == [(5.0, 1), (0.0, 0), (900.0, -1)]


@pytest.mark.parametrize("make,min_total", [(scenes.world_toy, 2000), (scenes.world_pcon, 500)], ids=["toy", "pcon"])
def test_toy_world_invariants(orc, make, min_total):
    """After every step the track is in another node (entering moves down the
    tree, leaving never returns the node left), and a point advanced 1e-6 mm
    past the boundary locates to the new node unless it lies within 1e-6 mm
    of another surface."""
    w = make()
    t = orc.world_nodes(w)
    parent = t["parent"]

    def below(a, b):   # a strictly below b
        while a > 0:
            a = parent[a]
            if a == b:
                return True
        return False

    tr = scenes.world_points(w, 4000, 21)
    node = orc.world_locate(w, tr)
    blk = np.full(tr.n, -1, dtype=np.int32)
    agree = total = down = 0
    for _ in range(4):
        s, nn, blk = orc.world_step(w, tr, node, blk)
        ok = (node >= 0) & (nn >= 0)
        assert np.all(nn[ok] != node[ok])
        down += sum(below(int(a), int(b)) for a, b in zip(nn[ok], node[ok]))
        adv = scenes.Tracks(tr.x + (s + 1e-6) * tr.dx, tr.y + (s + 1e-6) * tr.dy, tr.z + (s + 1e-6) * tr.dz,
                            tr.dx, tr.dy, tr.dz)
        loc = orc.world_locate(w, adv)
        agree += int(np.sum(loc[ok] == nn[ok]))
        total += int(ok.sum())
        tr = scenes.Tracks(tr.x + np.where(ok, s, 0) * tr.dx, tr.y + np.where(ok, s, 0) * tr.dy,
                           tr.z + np.where(ok, s, 0) * tr.dz, tr.dx, tr.dy, tr.dz)
        node = np.where(ok, nn, -1).astype(np.int32)
    assert total > min_total and 0 < down < total
    assert agree / total > 0.995


@pytest.mark.parametrize("make", [scenes.world_toy, scenes.world_pcon], ids=["toy", "pcon"])
def test_transport_makes_progress(orc, make):
    """Transporting tracks step after step through the toy world: no track
    ping-pongs across a surface (never more than two zero steps in a row),
    every track eventually leaves the root, and the path length of a track
    equals the distance from its start to where it left the hall."""
    w = make()
    tr = scenes.world_points(w, 3000, 22)
    x0 = np.stack([tr.x, tr.y, tr.z], 1)
    node = orc.world_locate(w, tr)
    flag = np.full(tr.n, -1, dtype=np.int32)
    zeros = np.zeros(tr.n, dtype=int)
    path = np.zeros(tr.n)
    alive = node >= 0
    for _ in range(60):
        if not alive.any():
            break
        s, nn, fl = orc.world_step(w, tr, node, flag)
        s = np.where(alive, s, 0.0)
        assert np.all(nn[alive] != -2)
        zeros = np.where(alive & (s == 0.0), zeros + 1, 0)
        assert zeros.max() <= 2
        path += s
        tr = scenes.Tracks(tr.x + s * tr.dx, tr.y + s * tr.dy, tr.z + s * tr.dz, tr.dx, tr.dy, tr.dz)
        node = np.where(alive, nn, -1).astype(np.int32)
        flag = fl
        alive = node >= 0
    assert not alive.any()
    x1 = np.stack([tr.x, tr.y, tr.z], 1)
    assert np.allclose(path, np.linalg.norm(x1 - x0, axis=1), rtol=0, atol=1e-9)
    h = w.volumes[w.root].mother_params[:3]
    assert np.all(np.isclose(np.abs(x1), h, rtol=0, atol=1e-9).any(axis=1))
