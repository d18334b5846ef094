"""Pins of the oracle's spatio-temporal grouping (Sec. 2, "Clustering
Similar Background - Spatio-Temporal Grouping", Eq. 3) against closed forms,
invariants and brute force -- never against the oracle itself nor the CUDA
path.

The reading pinned here: the features are the population standard
deviations, over the warm-up updates at training frames 1..N-1, of the
dominant mode's mean variance and weight, coded as round(64 sd_v) and
round(65536 sd_w); K-means with K = 3 on the codes scaled by their standard
deviations (1 for a constant code), first centroids at mean - sd, mean,
mean + sd (sd = 0 for a constant code); the Eq. 3 core is
the set of pixels strictly within their cluster's mean +- standard deviation
on both codes.
"""
import math

import numpy as np
import pytest

from oracle import Oracle, default_params, group_assign, group_centroids, group_cluster, group_init


def _const_frames(values, N):
    """N frames in which pixel p holds the grey value values[p]."""
    v = np.asarray(values, dtype=np.uint8)
    return np.repeat(np.repeat(v[None, :, None], 3, axis=2), N, axis=0)


def _decay_series(var_init, alpha, var_min, N):
    """A constant pixel's only live component: matched every frame with a
    zero residual, so v_t = max(var_min, (1 - alpha) v_{t-1}) and its weight
    stays 1 (Eq. 2)."""
    v, out = var_init, []
    for _ in range(1, N):
        v = max(var_min, (1.0 - alpha) * v)
        out.append(v)
    return np.array(out)


def _code(sd, scale):
    return min(65535, math.floor(sd * scale + 0.5))


@pytest.mark.parametrize("alpha,N", [(0.01, 200), (0.05, 100)])
def test_constant_pixel_features_closed_form(alpha, N):
    # the second case reaches the variance floor (225 * 0.95^t < 4 from t = 79)
    p = default_params(4, 1, 3)
    p.update(flags=0, alpha=alpha)
    o = Oracle(p)
    cv, cw = o.group_features(_const_frames([0, 37, 128, 255], N))
    series = _decay_series(225.0, alpha, 4.0, N)
    want = _code(float(np.sqrt(np.mean((series - series.mean()) ** 2))), 64.0)
    assert list(cv) == [want] * 4
    assert list(cw) == [0] * 4     # the dominant weight stays exactly 1


def test_feature_code_saturates():
    # spread above 1024 levels^2: 64 sd > 65535
    p = default_params(1, 1, 2)
    p.update(flags=0, alpha=0.05, var_init=8000.0, var_max=8000.0)
    o = Oracle(p)
    cv, _ = o.group_features(_const_frames([90], 100))
    series = _decay_series(8000.0, 0.05, 4.0, 100)
    assert 64.0 * series.std() > 65535
    assert cv[0] == 65535


def test_features_are_per_pixel():
    # a pixel's features depend on its own history only: permuting the
    # pixels permutes the codes
    rng = np.random.default_rng(5)
    N, P = 40, 24
    base = rng.integers(0, 256, (1, P, 3))
    frames = np.clip(base + rng.integers(-40, 41, (N, P, 3)) * rng.integers(0, 2, (N, P, 1)), 0, 255).astype(np.uint8)
    perm = rng.permutation(P)
    p = default_params(P, 1, 3)
    p.update(flags=0)
    a = Oracle(p).group_features(frames)
    b = Oracle(p).group_features(frames[:, perm])
    assert np.array_equal(a[0][perm], b[0]) and np.array_equal(a[1][perm], b[1])


def test_two_training_frames_give_zero_spread():
    p = default_params(3, 2, 3)
    p.update(flags=0)
    rng = np.random.default_rng(1)
    cv, cw = Oracle(p).group_features(rng.integers(0, 256, (2, 6, 3), dtype=np.uint8))
    assert not cv.any() and not cw.any()   # one update: a one-point series


# ------------------------------------------------------------------ K-means
def _blobs(rng, centres, n_each, spread):
    v, w, who = [], [], []
    for i, (cv, cw) in enumerate(centres):
        v.append(rng.integers(cv - spread, cv + spread + 1, n_each))
        w.append(rng.integers(cw - spread, cw + spread + 1, n_each))
        who.append(np.full(n_each, i))
    return np.concatenate(v), np.concatenate(w), np.concatenate(who)


def test_separated_blobs_are_recovered():
    rng = np.random.default_rng(2)
    v, w, who = _blobs(rng, [(200, 300), (6000, 9000), (30000, 40000)], 50, 20)
    labels, r = group_cluster(v, w)
    cl = labels & 3
    for i in range(3):
        assert len(set(cl[who == i])) == 1
    assert len(set(cl)) == 3
    assert r["converged"] == 1


def _bruteforce_check(v, w, labels, r):
    """Every pixel sits at the nearest final centroid (scaled distance), the
    centroids are their members' means, the cores follow Eq. 3; pixels
    within FP64 rounding of a tie or of a band edge are exempt."""
    x = np.stack([v, w], 1).astype(np.float64)
    sd = x.std(axis=0)
    sd[sd == 0] = 1.0
    cl = (labels & 3).astype(int)
    cent = np.array([x[cl == j].mean(axis=0) if (cl == j).any() else [np.nan, np.nan] for j in range(3)])
    d = np.stack([(((x - cent[j]) / sd) ** 2).sum(1) if (cl == j).any() else np.full(len(x), np.inf)
                  for j in range(3)], 1)
    best = d.min(1)
    clear = np.sort(d, 1)[:, 1] - best > 1e-9 * (1 + best)
    assert np.array_equal(d.argmin(1)[clear], cl[clear])
    for j in range(3):
        m = cl == j
        if not m.any():
            continue
        mu, sg = x[m].mean(0), x[m].std(0)
        assert np.allclose(mu, r["centroid"][j], rtol=1e-12, atol=1e-9)
        dev = np.abs(x[m] - mu)
        core = (dev < sg).all(1)
        edge = (np.abs(dev - sg) <= 1e-9 * (1 + sg)).any(1)
        assert np.array_equal(core[~edge], (labels[m] & 0x80).astype(bool)[~edge])
        assert r["n_core"][j] == int((labels[m] & 0x80).astype(bool).sum())
        assert r["n"][j] == int(m.sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kmeans_fixed_point_and_cores_bruteforce(seed):
    rng = np.random.default_rng(seed)
    P = 3000
    v = np.minimum(rng.gamma(2.0, 800.0, P), 65535).astype(np.uint16)
    w = np.minimum(rng.gamma(1.5, 3000.0, P), 65535).astype(np.uint16)
    labels, r = group_cluster(v, w)
    assert r["converged"] == 1
    _bruteforce_check(v, w, labels, r)


def test_separated_blobs_have_no_near_assignment():
    rng = np.random.default_rng(3)
    v, w, _ = _blobs(rng, [(200, 300), (6000, 9000), (30000, 40000)], 50, 20)
    _, r = group_cluster(v, w)
    assert r["n_near"] == 0


def test_init_closed_form():
    # codes v = 0, 2 (mean 1, population sd 1), w constant 5 (scale 1,
    # spread 0): centroids (0, 5), (1, 5), (2, 5)
    c, sd = group_init(np.array([0, 2], np.uint16), np.array([5, 5], np.uint16))
    assert sd.tolist() == [1.0, 1.0]
    assert c.tolist() == [[0.0, 5.0], [1.0, 5.0], [2.0, 5.0]]


def test_centroids_are_member_means_and_empty_keeps():
    v = np.array([1, 3, 10, 20, 30], np.uint16)
    w = np.array([4, 8, 0, 0, 3], np.uint16)
    lab = np.array([0, 0, 2, 2, 0x82], np.uint8)     # a core bit does not change the cluster
    c = group_centroids(v, w, lab, np.array([[7.0, 7.0], [-3.5, 11.25], [0.0, 0.0]]))
    assert c.tolist() == [[2.0, 6.0], [-3.5, 11.25], [20.0, 1.0]]


def test_assign_hand_worked_tie_and_margin():
    # centroids (100, 100), (200, 100), (1000, 1000), unit scales: the
    # pixel (150, 100) is 2500 from both of the first two (a tie: cluster
    # 0, near); (149, 100) is 2401 against 2601 (clear, cluster 0);
    # (151, 100) the mirror (clear, cluster 1); (999, 1000) clear, cluster 2
    c = np.array([[100.0, 100.0], [200.0, 100.0], [1000.0, 1000.0]])
    v = np.array([150, 149, 151, 999], np.uint16)
    w = np.array([100, 100, 100, 1000], np.uint16)
    lab, near = group_assign(v, w, c, np.array([1.0, 1.0]))
    assert lab.tolist() == [0, 0, 1, 2]
    assert near.tolist() == [True, False, False, False]


def test_assign_scales_each_feature():
    # with scales (100, 1) the w difference dominates: (500, 10) is
    # (0.01^2 + 0) from (499, 10) and (0 + 3^2) from (500, 13)
    c = np.array([[499.0, 10.0], [500.0, 13.0], [0.0, 0.0]])
    lab, near = group_assign(np.array([500], np.uint16), np.array([10], np.uint16), c, np.array([100.0, 1.0]))
    assert lab.tolist() == [0] and not near[0]
    # with scales (1, 100): 1^2 from the first, 0.03^2 from the second
    lab, _ = group_assign(np.array([500], np.uint16), np.array([10], np.uint16), c, np.array([1.0, 100.0]))
    assert lab.tolist() == [1]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_assign_bruteforce_and_single_precision_flips_are_near(seed):
    # FP64 labels equal a brute-force argmin away from ties; every pixel
    # whose decision a single-precision evaluation (centroid and reciprocal
    # scales rounded to float32 once, each operation rounded, ties to the
    # lower cluster) takes differently is in the near record.  Large codes
    # with small scales stress the rounding of the centroids.
    rng = np.random.default_rng(seed)
    P = 200000
    if seed % 2:
        v = rng.integers(60000, 65536, P).astype(np.uint16)
        w = rng.integers(0, 300, P).astype(np.uint16)
        sd = np.array([rng.uniform(3, 20), rng.uniform(50, 90)])
        c = np.stack([rng.uniform(60000, 65535, 3), rng.uniform(0, 300, 3)], 1)
    else:
        v = np.minimum(rng.gamma(2.0, 800.0, P), 65535).astype(np.uint16)
        w = np.minimum(rng.gamma(1.5, 3000.0, P), 65535).astype(np.uint16)
        sd = np.array([v.astype(float).std(), w.astype(float).std()])
        c = np.stack([rng.uniform(0, 4000, 3), rng.uniform(0, 9000, 3)], 1)
    lab, near = group_assign(v, w, c, sd)
    x = np.stack([v, w], 1).astype(np.float64)
    d = np.stack([(((x - c[j]) / sd) ** 2).sum(1) for j in range(3)], 1)
    ds = np.sort(d, 1)
    tie = ds[:, 1] - ds[:, 0] <= 1e-9 * (1 + ds[:, 0])
    assert np.array_equal(lab[~tie], d.argmin(1)[~tie])
    assert near[tie].all()
    flips = _fp32_labels(v, w, c, sd) != lab
    assert near[flips].all(), np.flatnonzero(flips & ~near)[:5]
    assert near.mean() < 0.01


def _fp32_labels(v, w, c, sd):
    """The assignment evaluated in single precision: centroids and
    reciprocal scales rounded to float32 once, each operation rounded, the
    first minimum taken (ties to the lower cluster)."""
    cf = c.astype(np.float32)
    isd = (1.0 / sd).astype(np.float32)
    d32 = np.empty((len(v), 3), np.float32)
    for j in range(3):
        tv = (v.astype(np.float32) - cf[j, 0]) * isd[0]
        tw = (w.astype(np.float32) - cf[j, 1]) * isd[1]
        d32[:, j] = tv * tv + tw * tw
    return d32.argmin(1)


def test_single_precision_near_ties_are_in_the_near_record():
    # pixels on (or a hair off) the bisector of two centroids placed around
    # a large code value: the rounding of the centroids to float32 flips
    # many decisions, and every flip must be in the near record
    rng = np.random.default_rng(0)
    flips_seen = 0
    for _ in range(300):
        m = int(rng.integers(1000, 65000))
        half = rng.uniform(0.5, 200)
        eta = rng.uniform(-2e-3, 2e-3) * (m / 65535)
        wc = rng.uniform(0, 60000)
        c = np.array([[m - half, wc], [m + half + eta, wc + rng.uniform(-1e-3, 1e-3)], [0.0, 0.0]])
        sd = np.array([rng.uniform(2, 50), rng.uniform(50, 3000)])
        v = np.full(64, m, np.uint16)
        w = rng.integers(0, 65536, 64).astype(np.uint16)
        lab, near = group_assign(v, w, c, sd)
        flips = _fp32_labels(v, w, c, sd) != lab
        assert near[flips].all()
        flips_seen += int(flips.sum())
    assert flips_seen > 1000     # the construction does reach the rounding


def test_constant_codes_form_one_cluster_with_empty_core():
    # all three centroids start on the one point: ties go to cluster 0; the
    # cluster's spread is 0, so no pixel is strictly inside Eq. 3
    labels, r = group_cluster(np.full(50, 700, np.uint16), np.full(50, 9, np.uint16))
    assert set(labels) == {0}
    assert r["n"] == [50, 0, 0] and r["n_core"] == [0, 0, 0]
    assert r["iterations"] == 1 and r["converged"] == 1


def test_single_pixel():
    labels, r = group_cluster(np.array([5], np.uint16), np.array([7], np.uint16))
    assert labels[0] == 0 and r["n"] == [1, 0, 0]


def test_constant_second_feature_splits_on_the_first():
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.integers(90, 111, 40), rng.integers(900, 1101, 40), rng.integers(5000, 5201, 40)])
    labels, r = group_cluster(v.astype(np.uint16), np.zeros(120, np.uint16))
    cl = labels & 3
    assert len(set(cl[:40])) == 1 and len(set(cl[40:80])) == 1 and len(set(cl[80:])) == 1
    assert len(set(cl)) == 3


# ------------------------------------------------------ shared parameters
def test_core_parameters_of_constant_scene():
    # constant pixels: the dominant mode ends at (weight 1, mean I,
    # variance max(var_min, 225 (1 - alpha)^(N-1))) on every channel
    N, vals = 60, [10, 50, 90, 130, 170, 210]
    p = default_params(6, 1, 3)
    p.update(flags=0)
    o = Oracle(p)
    o.train(_const_frames(vals, N))
    labels = np.array([0x80 | 0, 0x80 | 0, 0x80 | 2, 2, 0x80 | 2, 1], np.uint8)
    g = o.group_params(labels)
    vN = max(4.0, 225.0 * 0.99 ** (N - 1))
    assert g["w1"] == pytest.approx([1.0, 0.0, 1.0], abs=1e-12)
    assert g["mu1"][0] == pytest.approx([30.0] * 3, abs=1e-9)
    assert g["mu1"][2] == pytest.approx([130.0] * 3, abs=1e-9)    # (90 + 170) / 2, pixel 3 not core
    assert g["mu1"][1] == [0.0, 0.0, 0.0]                          # no core pixel
    assert g["v1"][0] == pytest.approx(vN, rel=1e-12) and g["v1"][2] == pytest.approx(vN, rel=1e-12)


def test_dominant_mode_switch_hand_worked():
    # A pixel at A = 50 for frames 0..M-1, then B = 200.  Hand-derived
    # dynamics (Eq. 2, alpha = 0.01, lambda = 2.5, w_init = 0.05, K = 3):
    #   frames 1..M-1: component 0 matches, w0 = 1, v0 <- max(4, 0.99 v0);
    #   frame M: nothing matches (150^2 > 6.25 v0, and the empty components
    #     sit at 0), the weights decay and the lowest-ranked component (the
    #     last of the zero keys) restarts at (B, 225, 0.05); renormalise;
    #   frames > M: component 2 matches (w2 <- 0.99 w2 + 0.01, v2 <- max(4,
    #     0.99 v2)), component 0 only decays (w0 <- 0.99 w0).
    # The dominant mode is the larger of w^2 / v between components 0 and 2.
    N, M = 200, 30
    w0, v0, w2, v2 = 1.0, 225.0, 0.0, 225.0
    sv, sw = [], []
    for t in range(1, N):
        if t < M:
            w0, v0 = 1.0, max(4.0, 0.99 * v0)
        elif t == M:
            s = 0.99 * w0 + 0.05
            w0, w2, v2 = 0.99 * w0 / s, 0.05 / s, 225.0
        else:
            w0, w2, v2 = 0.99 * w0, 0.99 * w2 + 0.01, max(4.0, 0.99 * v2)
            s = w0 + w2
            w0, w2 = w0 / s, w2 / s
        if w0 * w0 / v0 >= w2 * w2 / v2:
            sv.append(v0), sw.append(w0)
        else:
            sv.append(v2), sw.append(w2)
    assert sv[-1] != sv[M]   # the dominant mode does switch to B inside the series
    p = default_params(1, 1, 3)
    p.update(flags=0)
    frames = _const_frames([50], N)
    frames[M:] = 200
    cv, cw = Oracle(p).group_features(frames)
    assert cv[0] == _code(float(np.std(sv)), 64.0)
    assert cw[0] == _code(float(np.std(sw)), 65536.0)
