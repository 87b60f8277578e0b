"""Learned-culler cascade: box -> neural bound -> exact test, against the plain box ->
exact path and against brute force over every sphere of the scene (oracle)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _brute(ms, rays):
    # every sphere of the scene at once, in world coordinates on the world grid
    sc = I.Scene(ms.centres, ms.radii, None, ms.qexp)
    return O.label(I.RAY3, rays, sc).astype(bool)


def _plain(nb, ws, rays_d, n):
    import torch
    off, off_d, pair_ray, _, st = nb.cascade_bin(ws, rays_d, canonical=False)
    hits = torch.zeros(nb.n_words(n), dtype=torch.int32, device="cuda")
    est = torch.zeros(nb.CASCADE_STATS.itemsize, dtype=torch.uint8, device="cuda")
    nb.cascade_exact(ws, rays_d, pair_ray, off_d, int(off[-1]), ray_hits=hits, stats=est)
    return nb.bits_to_numpy(hits, n), st, nb._read(est, nb.CASCADE_STATS)


def test_plain_path_equals_brute_force(nb):
    ms = I.make_multi_scene(11, 24, 32)
    rays = I.sample_world_rays(12, 60_000)
    ws = nb.WorldScene(ms)
    got, st, est = _plain(nb, ws, _dev(rays), len(rays))
    assert np.array_equal(got, _brute(ms, rays))
    assert est["exact_pairs"] == st["aabb_pairs"]
    assert st["aabb_pairs"] >= est["hit_pairs"] > 0


def test_canonical_binning_keeps_every_hitting_pair(nb):
    import torch
    ms = I.make_multi_scene(21, 24, 32)
    rays = I.sample_world_rays(22, 60_000)
    ws = nb.WorldScene(ms)
    rd = _dev(rays)
    n = len(rays)
    off, off_d, pair_ray, pair_q, st = nb.cascade_bin(ws, rd, canonical=True)
    assert st["ball_pairs"] <= st["aabb_pairs"]
    hits = torch.zeros(nb.n_words(n), dtype=torch.int32, device="cuda")
    nb.cascade_exact(ws, rd, pair_ray, off_d, int(off[-1]), ray_hits=hits)
    assert np.array_equal(nb.bits_to_numpy(hits, n), _brute(ms, rays))
    # canonical rays start on the radius-2 ball around the object's centre
    pr = pair_ray.cpu().numpy()
    q = pair_q.cpu().numpy()
    live = pr != -1
    r = np.linalg.norm(q[live, :3].astype(np.float64), axis=1)
    assert np.all(np.abs(r - 2.0) < 1e-4)


def _object_of_rows(off):
    k = np.zeros(int(off[-1]), dtype=np.int64)
    for j in range(len(off) - 1):
        k[off[j]:off[j + 1]] = j
    return k


@pytest.mark.parametrize("K,indexed", [(24, False), (24, True), (300, True)])
def test_canonical_rays_equal_the_oracle_bit_for_bit(nb, K, indexed):
    """Every binned pair's network input (the ray in the object's frame, origin moved to
    its entry into the radius-2 ball) equals the oracle's replay of the defined FP32
    sequence bit for bit, and the oracle says the ray meets the ball."""
    ms = I.make_multi_scene(61 + K, K, 32)
    rays = I.sample_world_rays(62 + K, 40_003)
    ws = nb.WorldScene(ms)
    ix = nb.CascadeIndex(ws) if indexed else None
    off, _, pair_ray, pair_q, st = nb.cascade_bin(ws, _dev(rays), canonical=True, index=ix)
    pr = pair_ray.cpu().numpy()[:int(off[-1])]
    q = pair_q.cpu().numpy()[:int(off[-1])]
    live = pr != -1
    assert live.sum() == st["ball_pairs"] > 0
    k = _object_of_rows(off)[live]
    want, met = O.canonical_ray(rays[pr[live]], ms.obj_centre[k], float(ms.ball_radius))
    assert np.all(met)
    assert np.array_equal(q[live].view(np.uint32), want.view(np.uint32))
    if ix is not None:
        ix.close()


def test_cascade_end_to_end_equals_plain_and_avoids_exact_tests(nb):
    """16 objects, one trained 6->128x3->1 ray network each (split-FP16 queries), the
    thresholds calibrated on the cascade's own pairs: the cascade finds exactly the hits
    of the plain path and runs fewer exact tests."""
    import torch
    K = 16
    widths = [6, 128, 128, 128, 1]
    ms = I.make_multi_scene(31, K, 32)
    ws = nb.WorldScene(ms)
    B, W, T = 4096, 8, 400
    shapes = [nb.Shape(ms.local_scene(k)) for k in range(K)]
    pools = [_dev(I.sample_queries(I.RAY3, 3100 + k, B * W)) for k in range(K)]
    pbits = [nb.label(shapes[k], I.RAY3, pools[k]) for k in range(K)]
    batches = [(torch.cat([pools[k][j * B:(j + 1) * B] for k in range(K)]).contiguous(),
                torch.cat([pbits[k][j * B // 32:(j + 1) * B // 32] for k in range(K)]).contiguous())
               for j in range(W)]
    plan = nb.Plan(np.arange(K + 1, dtype=np.int64) * B, chunk_rows=4096)
    g = nb.Group(widths, K, infer_prec="f16x3")
    g.set_params(np.stack([I.init_params(3200 + k, widths) for k in range(K)]))
    for t in range(T):
        qd, bd = batches[t % W]
        g.train_step(plan, qd, bd, 1.0 + 99.0 * t / (T - 1))

    n = 100_000
    rays = I.sample_world_rays(33, n)
    rd = _dev(rays)
    off, off_d, pair_ray, pair_q, st = nb.cascade_bin(ws, rd, canonical=True)
    rows = int(off[-1])
    pair_lab = torch.zeros(nb.n_words(rows), dtype=torch.int32, device="cuda")
    nb.cascade_exact(ws, rd, pair_ray, off_d, rows, pair_hits=pair_lab)
    pplan = nb.Plan(off, chunk_rows=2048)
    g.calibrate(pplan, pair_q, pair_lab)
    neural = g.query(pplan, pair_q, margin=0.05)
    hits = torch.zeros(nb.n_words(n), dtype=torch.int32, device="cuda")
    est = torch.zeros(nb.CASCADE_STATS.itemsize, dtype=torch.uint8, device="cuda")
    nb.cascade_exact(ws, rd, pair_ray, off_d, rows, pass_bits=neural, ray_hits=hits, stats=est)
    casc = nb.bits_to_numpy(hits, n)
    plain, pst, pest = _plain(nb, ws, rd, n)
    e = nb._read(est, nb.CASCADE_STATS)
    assert np.array_equal(casc, plain), int(np.sum(plain & ~casc))
    assert np.array_equal(plain, _brute(ms, rays))
    assert e["exact_pairs"] < pest["exact_pairs"]
    # the network never excluded a pair that hits
    lab = nb.bits_to_numpy(pair_lab, rows)
    dec = nb.bits_to_numpy(neural, rows)
    live = pair_ray.cpu().numpy() != -1
    assert not np.any(lab & ~dec & live)


def _segments(off, pair_ray, pair_q=None):
    """per object: its rows sorted by ray (the order within an object is free)"""
    pr = pair_ray.cpu().numpy()
    q = None if pair_q is None else pair_q.cpu().numpy()
    out = []
    for k in range(len(off) - 1):
        seg = pr[off[k]:off[k + 1]]
        live = seg != -1
        o = np.argsort(seg[live], kind="stable")
        rows = np.nonzero(live)[0][o]
        out.append((seg[rows], None if q is None else q[off[k] + rows]))
    return out


@pytest.mark.parametrize("K,canonical", [(1, True), (24, False), (24, True), (300, True), (2048, False),
                                         (4096, True)])
def test_indexed_binning_equals_every_box(nb, K, canonical):
    ms = I.make_multi_scene(41 + K, K, 32)
    rays = I.sample_world_rays(42 + K, 50_000).astype(np.float32)
    # a slice of axis-parallel rays from object box faces
    rng = np.random.default_rng(43)
    m = 2000
    k = rng.integers(0, K, m)
    rays[:m, :3] = np.where(rng.random((m, 3)) < 0.5, ms.aabb[k, :3], ms.aabb[k, 3:])
    rays[:m, 3:] = 0
    rays[np.arange(m), 3 + rng.integers(0, 3, m)] = rng.choice([-1.0, 1.0], m)
    ws = nb.WorldScene(ms)
    ix = nb.CascadeIndex(ws)
    rd = _dev(rays)
    a = nb.cascade_bin(ws, rd, canonical=canonical)
    b = nb.cascade_bin(ws, rd, canonical=canonical, index=ix)
    assert np.array_equal(a[0], b[0])  # same counts, hence the same offsets
    assert a[4]["aabb_pairs"] == b[4]["aabb_pairs"] > 0
    assert a[4]["ball_pairs"] == b[4]["ball_pairs"]
    for (ra, qa), (rb, qb) in zip(_segments(a[0], a[2], a[3]), _segments(b[0], b[2], b[3])):
        assert np.array_equal(ra, rb)
        if canonical:
            assert np.array_equal(qa.view(np.uint32), qb.view(np.uint32))
    ix.close()


def test_indexed_plain_path_equals_brute_force(nb):
    import torch
    ms = I.make_multi_scene(51, 200, 32)
    rays = I.sample_world_rays(52, 80_001)
    ws = nb.WorldScene(ms)
    ix = nb.CascadeIndex(ws)
    rd = _dev(rays)
    n = len(rays)
    off, off_d, pair_ray, _, st = nb.cascade_bin(ws, rd, canonical=False, index=ix)
    hits = torch.zeros(nb.n_words(n), dtype=torch.int32, device="cuda")
    nb.cascade_exact(ws, rd, pair_ray, off_d, int(off[-1]), ray_hits=hits)
    assert np.array_equal(nb.bits_to_numpy(hits, n), _brute(ms, rays))
    # no rays: counts zero, nothing written
    e = nb.cascade_bin(ws, rd[:0], canonical=True, index=ix)
    assert int(e[0][-1]) == 0
    # an index of another scene is refused
    other = nb.WorldScene(I.make_multi_scene(53, 7, 4))
    with pytest.raises(nb.NBError):
        nb.cascade_bin(other, rd, canonical=False, index=ix)
    ix.close()
