"""The geometry tree on the GPU: node numbering, Locate, and transport steps
(step of Fig. 1 in the track's node + final localisation) against the
oracle, both modes bit for bit identical to each other.

Transport runs several steps; at every step the oracle gets the GPU's state
(position, node, flag) as input, so differences cannot accumulate.  Bars:
every step within max(1e-9 mm, err) of the oracle's, err the oracle's
a-priori FP64 error bound of that step, which adds the rounding of the
placements that bring the world point into its node level by level (the GPU
applies one composed transform per node instead; pinned against exact
crossings in test_oracle_errbound.py); node and flag exact except on tracks
whose oracle answer changes when the start point moves by 1e-9 mm (a
boundary point within rounding of another surface), which must be rare.
"""
import numpy as np
import pytest

from helpers import tracks_from
from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EYE = np.eye(3).reshape(9)


@pytest.fixture(scope="module")
def g():
    import paper_1312_0816_gb300 as pkg

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    return pkg


def build(g, w):
    vols = [g.geo_build_volume(v) for v in w.volumes]
    return g.geo_build_world(vols, w.child, w.root), vols


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def gpu_step(g, W, tr, node, flag, mode):
    s, n, f = g.geo_world_step(W, *(dev(x) for x in tr.fields()), dev(node, torch.int32),
                               dev(flag, torch.int32), mode=mode)
    torch.cuda.synchronize()
    return s.cpu().numpy(), n.cpu().numpy(), f.cpu().numpy()


def unstable(orc, w, tr, node, flag, want_node):
    """Tracks whose oracle node changes when the start moves by 1e-9 mm."""
    bad = np.zeros(tr.n, dtype=bool)
    for k in range(3):
        for e in (-1e-9, 1e-9):
            f = [tr.x.copy(), tr.y.copy(), tr.z.copy()]
            f[k] = f[k] + e
            _, n2, _ = orc.world_step(w, scenes.Tracks(*f, tr.dx, tr.dy, tr.dz), node, flag)
            bad |= n2 != want_node
    return bad


def test_node_table_and_locate(g, orc):
    w = scenes.world_toy()
    W, vols = build(g, w)
    t = g.geo_world_nodes(W)
    ot = orc.world_nodes(w)
    for k in ("lv", "parent", "slot", "first"):
        assert np.array_equal(t[k], ot[k]), k
    assert W.n_nodes == len(ot["lv"]) and W.max_depth == 3
    tr = scenes.world_points(w, 200000, 3)
    node = g.geo_world_locate(W, dev(tr.x), dev(tr.y), dev(tr.z)).cpu().numpy()
    assert np.array_equal(node, orc.world_locate(w, tr))
    bad = tracks_from(np.array([[np.nan, 0, 0], [5000.0, 0, 0]]), np.array([[1.0, 0, 0], [1.0, 0, 0]]))
    nb = g.geo_world_locate(W, dev(bad.x), dev(bad.y), dev(bad.z)).cpu().numpy()
    assert list(nb) == [-2, -1]


@pytest.mark.parametrize("make,seed,min_checked", [(scenes.world_toy, 5, 100000), (scenes.world_toy, 6, 100000),
                                                  (scenes.world_pcon, 5, 50000)], ids=["toy5", "toy6", "pcon5"])
def test_transport_matches_oracle(g, orc, make, seed, min_checked):
    w = make()
    W, vols = build(g, w)
    tr = scenes.world_points(w, 50000, seed)
    node = orc.world_locate(w, tr)
    flag = np.full(tr.n, -1, dtype=np.int32)
    exempt_total = checked = 0
    for it in range(10):
        alive = node >= 0
        if not alive.any():
            break
        s0, n0, f0 = gpu_step(g, W, tr, node, flag, 0)
        s1, n1, f1 = gpu_step(g, W, tr, node, flag, 1)
        assert np.array_equal(s0.view(np.int64)[alive], s1.view(np.int64)[alive]), it
        assert np.array_equal(n0, n1) and np.array_equal(f0, f1), it
        os_, on, of, info = orc.world_step(w, tr, node, flag, info=True)
        d = np.abs(s0 - os_)[alive]
        tol = np.maximum(1e-9, info["err"])[alive]
        assert np.all(d <= tol), (it, np.nonzero(d > tol)[0][:5], d.max())
        diff = alive & ((n0 != on) | (f0 != of))
        if diff.any():
            ex = unstable(orc, w, tr, node, flag, on)
            assert not np.any(diff & ~ex), (it, np.nonzero(diff & ~ex)[0][:5])
            exempt_total += int(diff.sum())
        checked += int(alive.sum())
        s = np.where(alive, s0, 0.0)
        tr = scenes.Tracks(tr.x + s * tr.dx, tr.y + s * tr.dy, tr.z + s * tr.dz, tr.dx, tr.dy, tr.dz)
        node = np.where(alive, n0, -1).astype(np.int32)
        flag = np.where(alive, f0, -1).astype(np.int32)
    assert checked > min_checked
    assert exempt_total <= 1e-4 * checked


@pytest.mark.parametrize("make", [scenes.world_toy, scenes.world_pcon], ids=["toy", "pcon"])
def test_transport_until_every_track_leaves(g, make):
    """GPU-only transport of the world until every track has left the hall:
    no ping-pong on a surface (at most two zero steps in a row) and the
    summed steps equal the straight distance travelled."""
    w = make()
    W, vols = build(g, w)
    tr = scenes.world_points(w, 1 << 16, 8)
    x = [dev(f) for f in tr.fields()]
    p0 = torch.stack(x[:3]).clone()
    node = g.geo_world_locate(W, *x[:3])
    flag = torch.full_like(node, -1)
    zeros = torch.zeros_like(node)
    path = torch.zeros_like(x[0])
    for _ in range(80):
        alive = node >= 0
        if not bool(alive.any()):
            break
        s, nn, ff = g.geo_world_step(W, *x, node, flag, mode=1)
        assert not bool(((nn == -2) & alive).any())
        s = torch.where(alive, s, torch.zeros_like(s))
        zeros = torch.where(alive & (s == 0), zeros + 1, torch.zeros_like(zeros))
        assert int(zeros.max()) <= 2
        path += s
        for k in range(3):
            x[k] = x[k] + s * x[3 + k]
        node = torch.where(alive, nn, torch.full_like(nn, -1))
        flag = torch.where(alive, ff, torch.full_like(ff, -1))
    assert not bool((node >= 0).any())
    dist = torch.linalg.norm(torch.stack(x[:3]) - p0, dim=0)
    assert float((path - dist).abs().max()) <= 1e-9


def test_invalid_state_and_single_volume(g, orc):
    box = scenes.leaf(0, (100.0, 100.0, 100.0), "box")
    w = scenes.World([box], [[]], 0)
    W, vols = build(g, w)
    tr = tracks_from(np.array([[0.0, 0, 0], [0.0, 0, 0], [0.0, 0, 0], [500.0, 0, 0]]),
                     np.array([[1.0, 0, 0], [0.0, 0, 0], [0.0, 1.0, 0], [1.0, 0, 0]]))
    node = np.array([0, 0, 7, 0], dtype=np.int32)
    flag = np.full(4, -1, dtype=np.int32)
    s, n, f = gpu_step(g, W, tr, node, flag, 1)
    assert s[0] == 100.0 and n[0] == -1                  # leaves the root
    assert np.isnan(s[1]) and n[1] == -2                 # zero direction
    assert np.isnan(s[2]) and n[2] == -2                 # no such node
    assert s[3] == 0.0 and n[3] == -2                    # not inside its node


def test_grouping_paths_give_the_same_answers(g):
    """The step groups tracks by logical volume with a shared-memory
    histogram up to 8192 keys and with global atomics above; unused logical
    volumes appended to the list only add keys, so both trees give the same
    bits."""
    w = scenes.world_toy()
    W1, vols1 = build(g, w)
    extra = [g.geo_build_volume(scenes.leaf(0, (1.0, 1.0, 1.0))) for _ in range(8200)]
    W2 = g.geo_build_world(vols1 + extra, list(w.child) + [[]] * len(extra), w.root)
    tr = scenes.world_points(w, 1 << 16, 9)
    x = [dev(f) for f in tr.fields()]
    node = g.geo_world_locate(W1, *x[:3])
    flag = torch.full_like(node, -1)
    for _ in range(3):
        a = g.geo_world_step(W1, *x, node, flag, mode=1)
        b = g.geo_world_step(W2, *x, node, flag, mode=1)
        torch.cuda.synchronize()
        assert torch.equal(a[0].nan_to_num(-7.0), b[0].nan_to_num(-7.0))
        assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
        alive = node >= 0
        s = torch.where(alive, a[0], torch.zeros_like(a[0]))
        for k in range(3):
            x[k] = x[k] + s * x[3 + k]
        node = torch.where(alive, a[1], torch.full_like(a[1], -1))
        flag = torch.where(alive, a[2], torch.full_like(a[2], -1))
    W2.close()
    for v in extra:
        v.close()
