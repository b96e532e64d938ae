"""The seeded synthetic inputs (workloads/): deterministic for a seed, and
drawn from the stated distributions (uneven batch of 256 double
integrators, box-SDF obstacles, Poisson request stream), with targets that
are what their formulas say."""
import numpy as np

import workloads as W


def test_grid_nodes_and_spacing():
    gd = W.grid([5, 3], [-2.0, 0.0], [2.0, 1.0])
    x0, x1 = W.node_coords(gd)
    assert np.allclose(x0, [-2, -1, 0, 1, 2]) and np.allclose(x1, [0, 0.5, 1])
    assert W.num_cells(gd) == 15


def test_strip_targets():
    gd, _, l = W.di_config(41)
    X = W.mesh(gd)[0]
    assert np.array_equal(l, 1.0 - np.abs(X))
    assert np.array_equal(W.target_outside(gd, 0, 2.0), np.abs(X) - 2.0)


def test_box_sdf_by_brute_force():
    rng = np.random.Generator(np.random.PCG64(5))
    c, h = [0.3, -0.2], [0.4, 0.25]
    # The box boundary, densely sampled.
    t = np.linspace(-1.0, 1.0, 4001)
    bx = np.concatenate([c[0] + h[0] * t, c[0] + h[0] * t, np.full_like(t, c[0] - h[0]),
                         np.full_like(t, c[0] + h[0])])
    by = np.concatenate([np.full_like(t, c[1] - h[1]), np.full_like(t, c[1] + h[1]),
                         c[1] + h[1] * t, c[1] + h[1] * t])
    p = rng.uniform(-1.5, 1.5, (2, 300))
    d = W.box_sdf([p[0], p[1]], c, h)
    dist = np.sqrt((p[0][:, None] - bx[None]) ** 2 + (p[1][:, None] - by[None]) ** 2).min(axis=1)
    inside = (np.abs(p[0] - c[0]) <= h[0]) & (np.abs(p[1] - c[1]) <= h[1])
    assert np.all(d[inside] <= 0) and np.all(d[~inside] > 0)
    assert np.allclose(np.abs(d), dist, atol=2e-3)  # boundary sampled at 2e-4 .. 4e-4 spacing
    # Union of boxes: the minimum of the distances.
    gd = W.grid([31, 31], [-2, -2], [2, 2])
    boxes = [(c, h), ([-1.0, 1.0], [0.2, 0.3])]
    pts = W.mesh(gd)
    assert np.array_equal(W.target_boxes(gd, boxes),
                          np.minimum(W.box_sdf(pts, *boxes[0]), W.box_sdf(pts, *boxes[1])))


def test_batch_instances_recipe():
    a = W.batch_instances(count=256, seed=1903)
    b = W.batch_instances(count=256, seed=1903)
    assert [x["grid"]["n"] for x in a] == [x["grid"]["n"] for x in b]
    assert [x["boxes"] for x in a] == [x["boxes"] for x in b]
    sides = np.array([x["grid"]["n"][0] for x in a])
    assert all(x["grid"]["n"][0] == x["grid"]["n"][1] for x in a)
    assert sides.min() >= 101 and sides.max() <= 501
    # E[s^2] = 301^2 + (401^2 - 1)/12 = 104001 for s ~ U{101..501}: about 26.6 M nodes.
    total = int((sides.astype(np.int64) ** 2).sum())
    assert abs(total - 256 * 104001) < 0.12 * 256 * 104001
    um = np.array([x["umax"] for x in a])
    dm = np.array([x["dmax"] for x in a])
    assert um.min() >= 0.5 and um.max() <= 2.0 and dm.min() >= 0.0 and dm.max() <= 0.3
    nb = np.array([len(x["boxes"]) for x in a])
    assert set(nb.tolist()) == {1, 2, 3}
    for x in a:
        for c, h in x["boxes"]:
            assert all(-1.5 <= v <= 1.5 for v in c) and all(0.1 <= v <= 0.5 for v in h)
        d = x["dyn"]
        assert d["uhi"][0] == x["umax"] and d["dhi"][0] == x["dmax"]
    assert W.batch_instances(count=4, seed=1)[0]["boxes"] != a[0]["boxes"]


def test_poisson_requests_recipe():
    reqs = W.poisson_requests(rate=50.0, duration=60.0, seed=7715)
    n = len(reqs)
    assert abs(n - 3000) < 4 * np.sqrt(3000)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] <= 60.0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50) < 4 * (1 / 50) / np.sqrt(n)
    # exponential gaps: the coefficient of variation is 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    quad = [r for r in reqs if r["kind"] == "quad4d"]
    di = [r for r in reqs if r["kind"] == "di"]
    assert abs(len(quad) / n - 0.5) < 0.05 and len(quad) + len(di) == n
    assert all(31 <= r["side"] <= 61 for r in quad) and all(201 <= r["side"] <= 1001 for r in di)
    for r in reqs:
        if r["change"] == "mass":
            assert 1.0 <= r["value"] <= 1.5
        else:
            assert r["change"] == "disturbance" and 0.0 <= r["value"] <= 0.3
    assert W.poisson_requests(rate=50.0, duration=60.0, seed=7715) == reqs
    assert len(W.poisson_requests(rate=50.0, duration=60.0, seed=7715, max_requests=10)) == 10
