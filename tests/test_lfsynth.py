"""The input generators: seeded, shaped like the workloads, and the two renderers agree."""
import numpy as np

import lfsynth


def test_torch_renderer_matches_numpy_renderer_without_noise():
    p = lfsynth.bench_params(U=3, V=5, H=40, W=56)
    v0, _ = lfsynth.voronoi_scene(p, 77, 8, (-3.4, 3.4), 0.5, 4.0, 0.0)
    v1 = lfsynth.voronoi_scene_torch(p, 77, 8, (-3.4, 3.4), 0.5, 4.0, 0.0).numpy()
    assert v1.shape == (5, 3, 40, 56) and v1.dtype == np.float32
    assert np.max(np.abs(v0 - v1)) <= 1e-6


def test_torch_renderer_is_seeded():
    p = lfsynth.tiny_params(U=3, V=3, H=24, W=24)
    a = lfsynth.voronoi_scene_torch(p, 5, 4, (-1.5, 1.5), 0.3, 2.0, 0.01).numpy()
    b = lfsynth.voronoi_scene_torch(p, 5, 4, (-1.5, 1.5), 0.3, 2.0, 0.01).numpy()
    c = lfsynth.voronoi_scene_torch(p, 6, 4, (-1.5, 1.5), 0.3, 2.0, 0.01).numpy()
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0


def test_batch_mix_covers_shapes_labels_and_census():
    ps = [lfsynth.batch_params(i) for i in range(64)]
    shapes = {(p.U, p.V, p.H, p.W) for p in ps}
    assert shapes == {(5, 5, 256, 256), (9, 9, 512, 512), (4, 4, 720, 1280), (15, 15, 434, 625)}
    assert {p.coarse_labels for p in ps} == {16, 32, 64, 128}
    assert {p.census_w for p in ps} == {5, 7}
    combos = {(p.U, p.census_w, p.coarse_labels) for p in ps}
    assert len(combos) == 32                      # every class meets every census and label count


def test_real_world_shaped_workloads():
    for f, shape in [(lfsynth.epfl, (3, 3, 60, 80)), (lfsynth.middlebury, (1, 7, 50, 70))]:
        V, U, H, W = shape
        p0 = f.__name__ == "epfl" and lfsynth.epfl_params(H=H, W=W) or lfsynth.middlebury_params(H=H, W=W)
        views, gt, p = f(params=p0)
        assert views.shape == shape and views.dtype == np.float32
        assert gt.shape == (H, W) and p.dmin <= gt.min() and gt.max() <= p.dmax
    assert lfsynth.middlebury_params().boundless == 1   # boundary-less search (Sec. IV-E)
