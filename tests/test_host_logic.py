"""Host-side logic that needs no GPU: the seeded input generators (cameras,
perturbation, isosurface sampling and its memory order), the autotuner's
selection and cache, the benchmark's reading of recorded ncu traffic, the
CPU binning reference of the GPU parity tests against brute force, the
reference-set recipe (orientation, KNN scale, Lambertian colour, packing)
and the benchmark's clock sampler (against a stand-in nvidia-smi)."""
import hashlib
import math
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2509_05216_gb300 import autotune, inputs  # noqa: E402


def test_orbit_cameras_look_at_the_origin_from_the_radius():
    r = 4.0
    cams = inputs.orbit_cameras(5, 3, r, 64, 48)
    assert len(cams) == 15
    for c in cams:
        vm = c["viewmat"]
        # the origin lies on the optical axis (+z, camera looks forward) at depth r
        o = vm[:3, :3] @ np.zeros(3) + vm[:3, 3]
        assert np.allclose(o[:2], 0.0, atol=1e-5) and abs(o[2] - r) < 1e-5
        # rows of the rotation are orthonormal (FP32-rounded)
        assert np.allclose(vm[:3, :3] @ vm[:3, :3].T, np.eye(3), atol=1e-6)
        assert c["fx"] == pytest.approx(64 / (2 * math.tan(math.radians(30.0))), rel=1e-6)
        assert (c["cx"], c["cy"]) == (31.5, 23.5)
    # elevations are evenly spaced inside (-75, 75) degrees: no camera at a pole
    ups = [abs(np.linalg.inv(c["viewmat"])[2, 3]) / r for c in cams]
    assert max(ups) < math.sin(math.radians(75.0))


def test_perturbation_is_seeded_and_bounded():
    scene = inputs.random_scene(300, 1, 7)
    p = scene["params"].copy()
    p[:, :5] = 0.0  # zero entries take the additive form
    scene = dict(scene, params=p)
    a = inputs.perturb(scene, 11)
    b = inputs.perturb(scene, 11)
    c = inputs.perturb(scene, 12)
    n = scene["n"]
    assert np.array_equal(a["params"], b["params"])
    assert not np.array_equal(a["params"], c["params"])
    x = p[:, :n].astype(np.float64)
    y = a["params"][:, :n].astype(np.float64)
    nz = x != 0.0
    # p' = p (1 + 0.05 u), u in [-1, 1]: relative change at most 5 %
    assert np.all(np.abs(y[nz] - x[nz]) <= 0.05 * np.abs(x[nz]) * (1 + 1e-6) + 1e-7)
    # p = 0: p' = 0.05 u
    assert np.all(np.abs(y[~nz]) <= 0.05 + 1e-7) and np.any(y[~nz] != 0.0)
    # padding columns beyond n are untouched
    assert np.array_equal(a["params"][:, n:], p[:, n:])


def test_isosurface_samples_lie_on_the_level_set_in_cell_order():
    lo, hi, res, n = -2.0 * math.pi, 2.0 * math.pi, 12, 3000
    pts = inputs._sample_isosurface(inputs._gyroid_fg, lo, hi, 0.0, n, seed=3, res=res, device="cpu")
    again = inputs._sample_isosurface(inputs._gyroid_fg, lo, hi, 0.0, n, seed=3, res=res, device="cpu")
    assert pts.shape == (n, 3) and np.array_equal(pts, again)
    f, _ = inputs._gyroid_fg(torch.from_numpy(pts))
    assert float(f.abs().max()) < 1e-6
    assert np.all((pts >= lo) & (pts <= hi))
    # contour-filter order: by sampling cell, x fastest, then y, then z
    h = (hi - lo) / res
    cell = np.clip(np.floor((pts - lo) / h).astype(np.int64), 0, res - 1)
    key = (cell[:, 2] * res + cell[:, 1]) * res + cell[:, 0]
    assert np.all(np.diff(key) >= 0)
    # so that neighbours in memory are near in space: consecutive points are
    # far closer than random pairs
    step = np.linalg.norm(np.diff(pts, axis=0), axis=1).mean()
    rng = np.random.default_rng(0)
    i, j = rng.integers(0, n, size=(2, 2000))
    assert step < 0.25 * np.linalg.norm(pts[i] - pts[j], axis=1).mean()


class _FakeCtx:
    def __init__(self):
        self.options = {}

    def gs_set_option(self, opt, value):
        self.options[opt] = value


def test_autotuner_keeps_the_fastest_value_of_each_option_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("GS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    ctx = _FakeCtx()
    cost = {1: {2: 5.0, 8: 3.0, 4: 4.0}, 2: {0: 2.0, 2: 1.0}}
    calls = []

    def fake_time(step, reps=3):
        calls.append(dict(ctx.options))
        return sum(cost[o][v] for o, v in ctx.options.items() if o in cost)

    monkeypatch.setattr(autotune, "time_step", fake_time)
    cands = {1: [2, 8, 4], 2: [0, 2]}
    chosen = autotune.tune([ctx], lambda: None, "key-a", candidates=cands, rounds=2)
    assert chosen == {1: 8, 2: 2}
    assert ctx.options == {1: 8, 2: 2}
    # every candidate was timed in each of the two rounds
    assert len(calls) == 2 * (3 + 2)
    # a second tune of the same workload takes the cached choice without timing
    calls.clear()
    ctx2 = _FakeCtx()
    assert autotune.tune([ctx2], lambda: None, "key-a", candidates=cands) == {1: 8, 2: 2}
    assert calls == [] and ctx2.options == {1: 8, 2: 2}


def test_compositing_work_counts_contributing_pairs_at_full_cost():
    """The compositing roofline charges the full per-pair arithmetic only to
    contributing pairs and the alpha test to the other walked entries."""
    assert bench.raster_work("bwd", 100, 30) == bench.RASTER_OPS_BWD * 30 + bench.RASTER_OPS_TEST * 70
    assert bench.raster_work("fwd", 100, 30) == bench.RASTER_OPS_FWD * 30 + bench.RASTER_OPS_TEST * 70
    assert bench.raster_work("bwd", 50, 50) == bench.RASTER_OPS_BWD * 50
    kind, work = bench.algorithmic_work("raster_bwd", 10, 59, 2, 100, (1000, 200), 64)
    assert kind == "alu" and work == bench.raster_work("bwd", 1000, 200)
    assert bench.RASTER_OPS_TEST < bench.RASTER_OPS_FWD < bench.RASTER_OPS_BWD


def test_cpu_binning_reference_equals_brute_force():
    """The vectorised CPU binning that the GPU parity tests compare against,
    checked against a plain loop over (view, Gaussian, tile) -- keeping a
    tile of the radius' rect if the alpha box reaches one of its pixels,
    tested tile by tile -- and a sort of (key, Gaussian) pairs on small
    random inputs (empty rects, rects clipped at the image border, boxes
    narrower and wider than the rect, a box that reaches nothing, equal
    depths)."""
    from tests.gpu_helpers import cpu_cut_rect, cpu_rect, expected_binning
    rng = np.random.default_rng(5)
    cams = [inputs.pinhole(np.eye(4), 70, 45), inputs.pinhole(np.eye(4), 33, 80)]
    n, stride = 40, 48
    B = len(cams)
    rec0 = np.zeros((B * stride, 4), np.float32)
    rec2 = np.zeros((B * stride, 4), np.float32)
    rec3 = np.zeros((B * stride, 4), np.int32)
    for v, c in enumerate(cams):
        sl = slice(v * stride, v * stride + n)
        rec0[sl, 0] = rng.uniform(-20, c["width"] + 20, n)
        rec0[sl, 1] = rng.uniform(-20, c["height"] + 20, n)
        rad = rng.integers(0, 30, n)
        rec2[sl, 1] = rng.uniform(0.0, 45.0, n)
        rec2[sl, 2] = rng.uniform(0.0, 45.0, n)
        rec2[sl.start, 1] = -3.0e38  # reaches no pixel
        x0, x1, y0, y1 = cpu_cut_rect(rec0[sl, 0], rec0[sl, 1], rad, rec2[sl, 1], rec2[sl, 2], c["width"],
                                      c["height"])
        tiles = np.maximum(x1 - x0, 0) * np.maximum(y1 - y0, 0)
        rec3[sl, 0] = rad
        rec3[sl, 1] = tiles
        rec2[sl, 3] = rng.choice(np.float32([1.5, 2.25, 3.0, 7.0]), n)  # many equal depths
    keys, vals, ranges, per_view = expected_binning(rec0, rec2, rec3, cams, n, stride)

    pairs, tile_off = [], 0
    ref_per_view = []
    for v, c in enumerate(cams):
        gw, gh = (c["width"] + 15) // 16, (c["height"] + 15) // 16
        count = 0
        for g in range(n):
            o = v * stride + g
            if rec3[o, 1] == 0:
                continue
            x0, x1, y0, y1 = (int(t[0]) for t in cpu_rect(rec0[o:o + 1, 0], rec0[o:o + 1, 1],
                                                          rec3[o:o + 1, 0].astype(np.int64),
                                                          c["width"], c["height"]))
            d = int(np.float32(rec2[o, 3]).view(np.uint32))
            f32 = np.float32
            mx, my, hx, hy = f32(rec0[o, 0]), f32(rec0[o, 1]), f32(rec2[o, 1]), f32(rec2[o, 2])
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    # a pixel of the tile inside the box (the compositing's FP32 sums)
                    if not (f32(16 * tx) <= mx + hx and f32(16 * tx + 15) >= mx - hx and
                            f32(16 * ty) <= my + hy and f32(16 * ty + 15) >= my - hy):
                        continue
                    pairs.append((((tile_off + ty * gw + tx) << 32) | d, g))
                    count += 1
        ref_per_view.append(count)
        tile_off += gw * gh
    pairs.sort()  # by key, then Gaussian index (the stable order of equal keys)
    assert list(per_view) == ref_per_view
    assert [int(k) for k in keys] == [p[0] for p in pairs]
    assert [int(x) for x in vals] == [p[1] for p in pairs]
    ref_ranges = np.zeros((tile_off, 2), np.int64)
    for i, (k, _) in enumerate(pairs):
        b = k >> 32
        if i == 0 or (pairs[i - 1][0] >> 32) != b:
            ref_ranges[b, 0] = i
        ref_ranges[b, 1] = i + 1
    assert np.array_equal(ranges, ref_ranges)


def _rotation(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_surface_gaussians_are_oriented_scaled_and_lit_as_stated():
    """The reference-set recipe: rotation taking +z onto the surface normal,
    KNN scale, Lambertian DC grey under the SH colour rule."""
    rng = np.random.default_rng(8)
    nrm = rng.normal(size=(200, 3))
    nrm[0] = (0.0, 0.0, -1.0)  # the antipodal case
    nrm[1] = (0.0, 0.0, 1.0)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    q = inputs._quat_z_to(nrm)
    for qi, ni in zip(q, nrm):
        assert np.allclose(_rotation(qi) @ np.array([0.0, 0.0, 1.0]), ni, atol=1e-9)
    # the colour of the DC term alone: rgb = Y00 sh0 + 0.5 = 0.1 + 0.9 max(0, n.l)
    y00 = 1.0 / (2.0 * math.sqrt(math.pi))
    light = np.ones(3) / math.sqrt(3.0)
    grey = y00 * inputs._lambert_dc(nrm) + 0.5
    assert np.allclose(grey, 0.1 + 0.9 * np.maximum(0.0, nrm @ light), atol=1e-12)
    # KNN scale against brute force
    pts = rng.uniform(-1, 1, size=(300, 3))
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    ref = 0.5 * np.log(np.sort(d2, axis=1)[:, :3].mean(1))
    assert np.allclose(inputs.knn_log_scale(pts), ref, atol=1e-12)


def test_parameter_planes_round_trip():
    rng = np.random.default_rng(9)
    n, k = 13, 16
    arrays = dict(means=rng.normal(size=(n, 3)), log_scales=rng.normal(size=(n, 3)),
                  quats=rng.normal(size=(n, 4)), opacity_logits=rng.normal(size=n),
                  sh=rng.normal(size=(n, k, 3)))
    scene = inputs.pack_params(**arrays)
    assert scene["deg"] == 3 and scene["params"].shape == (59, 16)
    assert np.all(scene["params"][:, n:] == 0.0)
    back = inputs.unpack_params(scene)
    for name, a in arrays.items():
        assert np.array_equal(back[name], a.astype(np.float32)), name


def test_clock_sampler_waits_for_samples_and_summarises_the_region(tmp_path, monkeypatch):
    """The benchmark's clock record, against a stand-in nvidia-smi that
    prints one CSV line every 20 ms (the first after 150 ms, like the real
    tool's start-up)."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nsleep 0.15\nwhile true; do\n"
                    "  echo '0, 2070, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.02\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    import time
    with bench.ClockSampler(0, interval_ms=20) as clk:
        assert clk.rows, "the region starts only after the first sample"
        time.sleep(0.2)
    s = clk.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] >= 3
    # no nvidia-smi at all: the record says so and the region is not delayed
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    t0 = time.time()
    with bench.ClockSampler(0) as clk:
        pass
    assert time.time() - t0 < 1.0
    assert clk.summary()["reasons"] == ["unavailable"]


def test_clock_sampler_falls_back_to_the_usual_interval(tmp_path, monkeypatch):
    """A tool that refuses the short interval: the sampler restarts it at
    200 ms and still records the region."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\ncase \"$*\" in *'-lms 200'*) ;; *) exit 2 ;; esac\nwhile true; do\n"
                    "  echo '0, 1980, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "  sleep 0.05\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    import time
    with bench.ClockSampler(0, interval_ms=50) as clk:
        time.sleep(0.15)
    s = clk.summary()
    assert s["sm_mhz"] == 1980.0 and s["reasons"] == [] and s["samples"] >= 2
