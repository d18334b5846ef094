"""The synthetic generator: determinism, pixel-subset consistency, and the
noise and scene statistics its recipe states."""
import numpy as np

from cogsynth import Scene, sm64, workload


def test_splitmix64_reference_values():
    # splitmix64 of the sequence started at 0 (Steele, Lea, Flood 2014): the
    # generator's first outputs are the finaliser of 1*gamma, 2*gamma, ...
    assert sm64(0) == 0xE220A8397B1DCDAF
    assert sm64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_render_is_deterministic_and_subset_consistent():
    sc = Scene(64, 48, 3, kind="dynamic", n_train=10, fg_frac=0.05, switch_at=5)
    a, ga = sc.render(17)
    b, gb = Scene(64, 48, 3, kind="dynamic", n_train=10, fg_frac=0.05, switch_at=5).render(17)
    assert np.array_equal(a, b) and np.array_equal(ga, gb)
    pix = np.array([0, 7, 1000, 64 * 48 - 1])
    c, gc = sc.render(17, pix)
    assert np.array_equal(c, a[pix]) and np.array_equal(gc, ga[pix])


def test_noise_level_matches_per_pixel_sigma():
    sc = Scene(32, 32, 1, kind="rects", n_train=400)
    f, _ = sc.frames(0, 300)                     # training frames: no objects
    sd = f.astype(np.float64).std(axis=0).mean(axis=1)
    want = sc.sig16 / 16.0
    assert np.all((want >= 2) & (want <= 6))
    assert abs(np.mean(sd / want) - 1.0) < 0.03


def test_workload_shapes_and_foreground():
    w = workload("qvga_rects")
    sc = w["scene"]
    f, g = sc.render(w["n_train"] + 10)
    assert f.shape == (160 * 120, 3)
    assert 0.01 < (g > 0).mean() < 0.08
    f0, g0 = sc.render(5)
    assert (g0 == 0).all()
    v = workload("vga_dynamic")["scene"]
    assert 0.07 < (v.blob_id >= 0).mean() < 0.12
    d_before = v.frame_desc(500 + 599)["offset"]
    d_after = v.frame_desc(500 + 600)["offset"]
    assert d_before == 0 and d_after == 60
