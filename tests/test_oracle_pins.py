"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every expected value here comes from a closed form, an invariant, a
brute-force evaluation of a definition, or a hand-worked case whose
arithmetic is written out beside it -- never from the oracle itself and
never from the CUDA path.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ORC_CONF, ORC_FD, ORC_ILLUM, ORC_RGA, Oracle, default_params, kde_weights

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ALL = ORC_FD | ORC_RGA | ORC_CONF | ORC_ILLUM


def _golden_ints(name):
    with open(os.path.join(GOLD, name)) as f:
        rows = [l for l in f if l.strip() and not l.startswith("#")]
    return [int(x) for x in rows[0].split()]


def one_pixel(K=3, flags=0, **over):
    p = default_params(1, 1, K)
    p.update(flags=flags, **over)
    return Oracle(p)


# --------------------------------------------------------------------- KDE
def test_kde_weights_match_rational_taylor_table():
    # Sec. 2 scene prior: Gaussian kernel, bandwidth 4, 3-bandwidth support
    assert list(kde_weights(4)) == _golden_ints("kde_weights_bw4.txt")


def test_kde_weights_semigroup_property():
    # exp(-a) exp(-b) = exp(-(a+b)): 3-4-5 and 6-8-10 triangles
    g = kde_weights(4)
    assert abs(g[3] * g[4] / 65536 - g[5]) <= 1.0
    assert abs(g[6] * g[8] / 65536 - g[10]) <= 1.0


@pytest.mark.parametrize("bw", [4, 1, 7])
@pytest.mark.parametrize("v", [0, 3, 100, 250, 255])
def test_kde_of_constant_training_is_the_normalised_kernel(v, bw):
    # all N training values equal v: k = N g[|u - v|], peak N g[0]; the
    # kernel's support is 3bw levels on each side
    o = one_pixel(kde_bw=bw)
    frames = np.full((6, 1, 3), v, np.uint8)
    o.train(frames)
    g = [math.floor(65536.0 * math.exp(-d * d / (2.0 * bw * bw)) + 0.5) for d in range(3 * bw + 1)]
    for c in range(3):
        q = o.state.kde[0, c]
        for u in range(256):
            d = abs(u - v)
            exp = (255 * g[d] + g[0] // 2) // g[0] if d <= 3 * bw else 0
            assert q[u] == exp, (u, v, bw)


def test_kde_bruteforce_direct_sum_over_samples():
    # the density at v is a sum over the training samples of g[|v - I_t|];
    # evaluated here sample by sample instead of through a histogram
    rng = np.random.default_rng(7)
    g = [int(x) for x in kde_weights(4)]
    for trial in range(20):
        N = int(rng.integers(2, 5))
        frames = rng.integers(0, 256, (N, 1, 3), dtype=np.uint8)
        if trial % 3 == 0:
            frames = np.clip(frames // 8 + 120, 0, 255).astype(np.uint8)
        o = one_pixel()
        o.train(frames)
        for c in range(3):
            k = [sum(g[abs(v - int(frames[t, 0, c]))] if abs(v - int(frames[t, 0, c])) <= 12 else 0
                     for t in range(N)) for v in range(256)]
            M = max(k)
            exp = [(255 * x + M // 2) // M for x in k]
            assert list(o.state.kde[0, c]) == exp


@pytest.mark.parametrize("bw", [4, 1, 7])
@pytest.mark.parametrize("v", [0, 100, 255])
def test_kde4_of_constant_training_is_the_kernel_on_15_levels(v, bw):
    # the 4-bit prior quantises the same density to 15 levels of its peak:
    # all N values equal v gives (15 g[d] + g[0]/2) div g[0], d = |u - v|
    o = one_pixel(kde_bw=bw, kde_bits=4)
    o.train(np.full((5, 1, 3), v, np.uint8))
    g = [math.floor(65536.0 * math.exp(-d * d / (2.0 * bw * bw)) + 0.5) for d in range(3 * bw + 1)]
    for c in range(3):
        q = o.state.kde[0, c]
        for u in range(256):
            d = abs(u - v)
            assert q[u] == ((15 * g[d] + g[0] // 2) // g[0] if d <= 3 * bw else 0), (u, v, bw)


def test_kde4_bruteforce_direct_sum_over_samples():
    # as the 8-bit brute force, with 15 levels: q = (15 k + M/2) div M
    rng = np.random.default_rng(11)
    g = [int(x) for x in kde_weights(4)]
    for trial in range(12):
        N = int(rng.integers(2, 6))
        frames = rng.integers(0, 256, (N, 1, 3), dtype=np.uint8)
        if trial % 2 == 0:
            frames = np.clip(frames // 6 + 100, 0, 255).astype(np.uint8)
        o = one_pixel(kde_bits=4)
        o.train(frames)
        for c in range(3):
            k = [sum(g[abs(v - int(frames[t, 0, c]))] if abs(v - int(frames[t, 0, c])) <= 12 else 0
                     for t in range(N)) for v in range(256)]
            M = max(k)
            assert list(o.state.kde[0, c]) == [(15 * x + M // 2) // M for x in k]


def test_kde4_and_kde8_round_the_same_density():
    # both widths round k/M to the nearest level: q8 = 255 k/M + e8 and
    # 17 q4 = 255 k/M + 17 e4 with |e| <= 1/2, so |17 q4 - q8| < 9; the top
    # 8-bit level (k/M >= 254.5/255) lies inside the top 4-bit level
    # (k/M >= 14.5/15)
    rng = np.random.default_rng(5)
    frames = rng.normal(128, 20, (40, 64, 3)).clip(0, 255).astype(np.uint8)
    o8 = Oracle(default_params(64, 1, 3))
    o4 = Oracle(dict(default_params(64, 1, 3), kde_bits=4))
    o8.train(frames)
    o4.train(frames)
    q8 = o8.state.kde.astype(int)
    q4 = o4.state.kde.astype(int)
    assert q4.max() == 15 and np.all(np.abs(17 * q4 - q8) <= 8)
    assert np.all(q4[q8 == 255] == 15) and np.all(q8[q4 < 15] < 255)


# ---------------------------------------------------------------- residues
def test_residue_classes_crafted_sequence():
    # Sec. 2 residue classes: R_t = max_c |I_t - I_{t-1}|; r1 = 10, r2 = 30.
    # channel-0 sequence: steps 0, 10, 11, 30, 31, 255 and back down 255, then 0s
    seq = [100, 100, 110, 121, 151, 182, 0, 255, 255, 255, 255]
    # residues: 0,10,11,30,31,182,255,0,0,0  -> n0 = 5 (0,10,0,0,0), n1 = 2 (11,30),
    # n2 = 3 (31,182,255); N-1 = 10
    frames = np.zeros((len(seq), 1, 3), np.uint8)
    frames[:, 0, 0] = seq
    frames[:, 0, 1] = 50          # other channels constant: residue 0
    o = one_pixel()
    o.train(frames)
    assert o.state.qa[0] == (255 * 5 + 5) // 10 == 128
    assert o.state.qb[0] == (255 * 3 + 5) // 10 == 77


def test_residue_weights_clamped_to_sum_255():
    # n0 = n2 = 1 of N-1 = 2: both round up to 128; b is clamped to 255 - a
    frames = np.zeros((3, 1, 3), np.uint8)
    frames[:, 0, 0] = [10, 10, 200]
    o = one_pixel()
    o.train(frames)
    assert o.state.qa[0] == 128 and o.state.qb[0] == 127


# ------------------------------------------------------ mixture closed forms
def test_static_pixel_variance_decay():
    # stages and confidence off, noiseless constant input: always background,
    # omega = (1, 0, 0) exactly, v_0 after n updates = max(v_min, v_init (1-a)^n)
    p = default_params(1, 1, 3)
    p["flags"] = 0
    o = Oracle(p)
    o.train(np.full((40, 1, 3), 90, np.uint8))
    n = 39
    for i in range(400):
        m, _, _, _ = o.apply(np.full((1, 3), 90, np.uint8))
        n += 1
        assert m[0] == 0
        assert list(o.state.w[0]) == [1.0, 0.0, 0.0]
        exp = max(p["var_min"], p["var_init"] * (1 - p["alpha"]) ** n)
        assert np.allclose(o.state.var[0, 0], exp, rtol=1e-12, atol=0)


def test_step_absorption_time():
    # a step from 100 to 200: no mode matches, so the pixel is foreground and
    # the weakest mode restarts at 200 with weight w_init; the old mode keeps
    # omega' = (1-a)/((1-a)+w_init) and decays by (1-a) per frame.  The pixel
    # turns background once the weight ranked before the new mode is <= T:
    # first at j = 1 + ceil(ln(T/omega') / ln(1-a)) frames after the step.
    p = default_params(1, 1, 3)
    p["flags"] = 0
    a, T, wi = p["alpha"], p["T_bg"], p["w_init"]
    wp = (1 - a) / ((1 - a) + wi)
    j_exp = 1 + math.ceil(math.log(T / wp) / math.log(1 - a))
    assert j_exp == 32
    for flags in (0, ORC_FD | ORC_RGA):
        p["flags"] = flags
        o = Oracle(p)
        o.train(np.full((300, 1, 3), 100, np.uint8))
        labels, stages = [], []
        for j in range(j_exp + 5):
            m, st, _, _ = o.apply(np.full((1, 3), 200, np.uint8))
            labels.append(int(m[0]))
            stages.append(int(st[0]))
        first_bg = labels.index(0)
        assert first_bg == j_exp
        assert all(x == 255 for x in labels[:first_bg])
        assert all(x == 0 for x in labels[first_bg:])
        if flags:
            # afterwards the value repeats, so the pixel leaves at stage 0
            assert stages[first_bg] == 2 and all(s == 0 for s in stages[first_bg + 1:])


def test_weights_stay_normalised():
    from cogsynth import Scene
    sc = Scene(24, 16, 11, kind="dynamic", n_train=30, fg_frac=0.1, switch_at=20)
    p = default_params(24, 16, 5)
    p["flags"] = ALL
    o = Oracle(p)
    tr, _ = sc.frames(0, 30)
    o.train(tr)
    for t in range(30, 90):
        f, _ = sc.render(t)
        o.apply(f)
        assert np.max(np.abs(o.state.w.sum(axis=1) - 1.0)) <= 1e-12
        assert o.state.w.min() >= 0.0


def test_cascade_with_everything_off_is_the_plain_mixture():
    # the cascade is a decomposition of the GMM: with every rejection stage
    # and modulation off it must reproduce the background-set form bit for bit
    from cogsynth import Scene
    sc = Scene(32, 20, 5, kind="dynamic", n_train=25, fg_frac=0.05, switch_at=10)
    for K in (1, 3, 5):
        p = default_params(32, 20, K)
        p["flags"] = 0
        o = Oracle(p)
        tr, _ = sc.frames(0, 25)
        o.train(tr)
        w, mu, var = o.state.w.copy(), o.state.mu.copy(), o.state.var.copy()
        for t in range(25, 60):
            f, _ = sc.render(t)
            m1, _, _, _ = o.apply(f)
            m2 = o.plain_gmm(w, mu, var, f)
            assert np.array_equal(m1, m2)
            assert np.array_equal(w, o.state.w)
            assert np.array_equal(mu, o.state.mu)
            assert np.array_equal(var, o.state.var)


def test_constant_input_confidence_recursion():
    # a repeating value leaves at stage 0 with instantaneous confidence 1, so
    # C_n = 1 - (1 - C_0)(1 - eta)^n
    p = default_params(1, 1, 3)
    p["flags"] = ORC_FD | ORC_CONF
    o = Oracle(p)
    o.train(np.full((10, 1, 3), 77, np.uint8))
    C0 = o.state.conf[0]
    assert C0 == 0.5
    for n in range(1, 60):
        _, st, _, _ = o.apply(np.full((1, 3), 77, np.uint8))
        assert st[0] == 0
        assert abs(o.state.conf[0] - (1 - (1 - C0) * (1 - p["eta"]) ** n)) <= 1e-12


def test_global_jump_flags_illumination_change():
    # > 70 % of the pixels jump by +60: foreground at the jump frame, the
    # counter of that frame flags the next one, which is forced to background
    W, H = 10, 10
    p = default_params(W, H, 3)
    p["flags"] = ALL
    o = Oracle(p)
    o.train(np.full((40, W * H, 3), 100, np.uint8))
    for _ in range(5):
        m, st, _, stats = o.apply(np.full((W * H, 3), 100, np.uint8))
        assert (m == 0).all() and stats["illum_flag"] == 0
    jump = np.full((W * H, 3), 100, np.uint8)
    jump[:80] = 160                     # 80 % of the pixels
    m, st, _, stats = o.apply(jump)
    assert (m[:80] == 255).all() and (m[80:] == 0).all()
    assert stats["illum_flag"] == 0 and stats["n_gmm"] == 80
    m, st, _, stats = o.apply(jump)
    assert stats["illum_flag"] == 1
    assert (m == 0).all() and (st[:80] == 4).all() and (st[80:] == 0).all()
    i = 0
    assert o.state.w[i].max() == p["w_illum"]
    assert abs(o.state.w[i].sum() - 1) <= 1e-12
    # frame s+1 still had 80 pixels at the mixture stage, so s+2 is flagged as
    # well; its pixels repeat their values and leave at stage 0 regardless
    m, st, _, stats = o.apply(jump)
    assert stats["illum_flag"] == 1 and (m == 0).all() and (st == 0).all()
    m, st, _, stats = o.apply(jump)
    assert stats["illum_flag"] == 0 and (m == 0).all() and (st == 0).all()


def test_global_jump_below_threshold_is_not_an_illumination_change():
    W, H = 10, 10
    p = default_params(W, H, 3)
    p["flags"] = ALL
    o = Oracle(p)
    o.train(np.full((40, W * H, 3), 100, np.uint8))
    jump = np.full((W * H, 3), 100, np.uint8)
    jump[:70] = 160                     # exactly 70 %: not above the threshold
    o.apply(jump)
    m, st, _, stats = o.apply(jump)
    assert stats["illum_flag"] == 0 and (m[:70] == 255).all()


def test_stage0_exit_leaves_model_untouched():
    from cogsynth import Scene
    sc = Scene(40, 30, 9, kind="dynamic", n_train=30, fg_frac=0.05)
    p = default_params(40, 30, 3)
    p["flags"] = ALL
    o = Oracle(p)
    tr, _ = sc.frames(0, 30)
    o.train(tr)
    for t in range(30, 45):
        before = o.state.copy()
        f, _ = sc.render(t)
        _, st, _, _ = o.apply(f)
        fd = st == 0
        assert fd.sum() > 100
        for name in ("w", "mu", "var", "rga_m", "rga_v"):
            assert np.array_equal(getattr(before, name)[fd], getattr(o.state, name)[fd])
        rga = st == 1
        for name in ("w", "mu", "var"):
            assert np.array_equal(getattr(before, name)[rga], getattr(o.state, name)[rga])


# ------------------------------------------------------- hand-worked pixels
def _hand_state(o, label=0, prev=(100, 100, 100)):
    s = o.state
    s.w[0] = [0.5, 0.3, 0.2]
    s.mu[0] = [[100, 100, 100], [50, 50, 50], [200, 200, 200]]
    s.var[0] = [[16, 16, 16], [4, 4, 4], [64, 64, 64]]
    s.rga_m[0] = [100, 100, 100]
    s.rga_v[0] = [16, 16, 16]
    s.conf[0] = 0.5
    s.label[0] = label
    s.prev[0] = prev
    s.kde[0] = 200
    s.qa[0], s.qb[0] = 153, 51
    s.illum[0] = 0


HAND = dict(alpha=0.25, var_min=1.0, var_max=1000.0, var_init=100.0, w_init=0.05)


def test_hand_gmm_match_second_ranked_is_background():
    # keys w^2/vbar: comp0 .25/16 = .015625, comp1 .09/4 = .0225, comp2 .04/64;
    # order 1, 0, 2.  I = (104,100,98): comp1 t = 54^2/25 >> 1; comp0 t = max(16,
    # 0, 4)/100 = .16 < 1 -> match at rank 2; weight before = .3 <= .7 -> BG.
    # update a = .25: w = (.75*.5+.25, .75*.3, .75*.2) = (.625, .225, .15);
    # mu0 = (101, 100, 99.5); v0 = (.75*16 + .25*3^2, .75*16, .75*16 + .25*1.5^2)
    #      = (14.25, 12, 12.5625); running average reseeded from comp0.
    o = one_pixel(flags=0, **HAND)
    _hand_state(o)
    m, st, _, stats = o.apply(np.array([[104, 100, 98]], np.uint8))
    assert m[0] == 0 and st[0] == 2 and stats["n_gmm"] == 1
    np.testing.assert_allclose(o.state.w[0], [0.625, 0.225, 0.15], rtol=1e-15)
    assert list(o.state.mu[0, 0]) == [101.0, 100.0, 99.5]
    assert list(o.state.var[0, 0]) == [14.25, 12.0, 12.5625]
    assert list(o.state.mu[0, 1]) == [50.0] * 3 and list(o.state.var[0, 2]) == [64.0] * 3
    assert list(o.state.rga_m[0]) == [101.0, 100.0, 99.5]
    assert list(o.state.rga_v[0]) == [14.25, 12.0, 12.5625]


def test_hand_gmm_no_match_replaces_weakest():
    # I = (0,255,0) matches nothing: FG; decay (.375,.225,.15), the lowest-ranked
    # comp2 becomes (I, v_init=100, w_init=.05); sum .65 -> (15/26, 9/26, 2/26)
    o = one_pixel(flags=0, **HAND)
    _hand_state(o)
    m, st, _, _ = o.apply(np.array([[0, 255, 0]], np.uint8))
    assert m[0] == 255 and st[0] == 3
    np.testing.assert_allclose(o.state.w[0], [15 / 26, 9 / 26, 2 / 26], rtol=1e-15)
    assert list(o.state.mu[0, 2]) == [0.0, 255.0, 0.0]
    assert list(o.state.var[0, 2]) == [100.0] * 3
    assert list(o.state.rga_m[0]) == [100.0] * 3      # FG: running average untouched


def test_hand_gmm_match_behind_too_much_weight_is_foreground():
    # I = comp2's mean: match at rank 3, weight before = .3 + .5 = .8 > .7 -> FG;
    # w = (.375, .225, .15 + .25) ; v2 = .75 * 64 = 48
    o = one_pixel(flags=0, **HAND)
    _hand_state(o)
    m, st, _, _ = o.apply(np.array([[200, 200, 200]], np.uint8))
    assert m[0] == 255 and st[0] == 3
    np.testing.assert_allclose(o.state.w[0], [0.375, 0.225, 0.4], rtol=1e-15)
    assert list(o.state.var[0, 2]) == [48.0] * 3


def test_hand_gmm_variance_clamped_at_the_top():
    # comp0 widened to v = 1000 = var_max: keys .25/1000, .09/4, .04/64 ->
    # order 1, 2, 0.  I = 179 on every channel: comp1 (50, 4) far; comp2
    # (200, 64): 21^2 = 441 > 6.25*64 = 400, no match; comp0: 79^2 = 6241 <
    # 6250 -> match at rank 3, weight before .3 + .2 = .5 <= .7 -> BG.
    # mu0 = 100 + .25*79 = 119.75; v0 = .75*1000 + .25*59.25^2 = 1627.640625
    # -> clamped to 1000; w = (.625, .225, .15)
    o = one_pixel(flags=0, **HAND)
    _hand_state(o)
    o.state.var[0, 0] = [1000.0] * 3
    m, st, _, _ = o.apply(np.array([[179, 179, 179]], np.uint8))
    assert m[0] == 0 and st[0] == 2
    assert list(o.state.mu[0, 0]) == [119.75] * 3
    assert list(o.state.var[0, 0]) == [1000.0] * 3
    np.testing.assert_allclose(o.state.w[0], [0.625, 0.225, 0.15], rtol=1e-15)


def test_hand_equal_keys_rank_the_lower_index_first():
    # two components with the same weight, mean and variance: equal keys, so
    # component 0 ranks first and takes the match; component 1 only decays
    o = one_pixel(K=2, flags=0, **HAND)
    s = o.state
    s.w[0] = [0.5, 0.5]
    s.mu[0] = [[100, 100, 100], [100, 100, 100]]
    s.var[0] = [[16, 16, 16], [16, 16, 16]]
    s.conf[0], s.label[0], s.prev[0], s.kde[0] = 0.5, 0, [100, 100, 100], 200
    m, _, _, _ = o.apply(np.array([[104, 104, 104]], np.uint8))
    assert m[0] == 0
    assert list(o.state.mu[0, 0]) == [101.0] * 3 and list(o.state.mu[0, 1]) == [100.0] * 3
    np.testing.assert_allclose(o.state.w[0], [0.625, 0.375], rtol=1e-15)


def test_hand_background_set_boundary_is_inclusive():
    # T = 0.5 and weights (0.5, 0.5) with component 0 ranked first (smaller
    # variance): a match at rank 2 has exactly T ranked before it -> BG
    # (weight before <= T); with T just below 0.5 the same match is FG
    for T, fg in ((0.5, 0), (0.4999, 255)):
        o = one_pixel(K=2, flags=0, **dict(HAND, T_bg=T))
        s = o.state
        s.w[0] = [0.5, 0.5]
        s.mu[0] = [[100, 100, 100], [200, 200, 200]]
        s.var[0] = [[16, 16, 16], [64, 64, 64]]
        s.conf[0], s.label[0], s.prev[0], s.kde[0] = 0.5, 0, [100, 100, 100], 200
        m, _, _, _ = o.apply(np.array([[200, 200, 200]], np.uint8))
        assert m[0] == fg, T


def test_hand_illumination_response():
    # the previous frame sent its one pixel to the mixture stage: 1 * 1000 >
    # 700 * 1 flags this frame.  I = (0, 255, 0) matches nothing: decay
    # (.375, .225, .15), comp2 restarts with w_init .05, renormalised to
    # (15, 9, 2)/26; the foreground decision becomes an illumination change:
    # comp2 takes w_illum = .75 and the others share .25 in proportion,
    # 15/24 * .25 = .15625 and 9/24 * .25 = .09375; the label is background
    o = one_pixel(flags=ORC_ILLUM, **HAND)
    _hand_state(o)
    o.state.illum[0] = 1
    m, st, _, stats = o.apply(np.array([[0, 255, 0]], np.uint8))
    assert m[0] == 0 and st[0] == 4 and stats["illum_flag"] == 1
    np.testing.assert_allclose(o.state.w[0], [0.15625, 0.09375, 0.75], rtol=1e-15)
    assert list(o.state.mu[0, 2]) == [0.0, 255.0, 0.0]
    # and without the flag the same frame is plain foreground
    o = one_pixel(flags=ORC_ILLUM, **HAND)
    _hand_state(o)
    m, st, _, stats = o.apply(np.array([[0, 255, 0]], np.uint8))
    assert m[0] == 255 and st[0] == 3 and stats["illum_flag"] == 0


def test_hand_rga_stage():
    # running average (100, 16): I = (104,100,98) -> t_r = .16 < 1 -> BG at stage 1,
    # same arithmetic as the matched mode above; the mixture is untouched
    o = one_pixel(flags=ORC_RGA, **HAND)
    _hand_state(o)
    m, st, _, stats = o.apply(np.array([[104, 100, 98]], np.uint8))
    assert m[0] == 0 and st[0] == 1 and stats["n_gmm"] == 0
    assert list(o.state.rga_m[0]) == [101.0, 100.0, 99.5]
    assert list(o.state.rga_v[0]) == [14.25, 12.0, 12.5625]
    assert list(o.state.w[0]) == [0.5, 0.3, 0.2]


def test_hand_fd_threshold_inclusive():
    # D = 8 <= tau_fd (0.5 + 0.5) = 8 -> stage 0; D = 9 -> falls through
    o = one_pixel(flags=ORC_FD, **HAND)
    _hand_state(o)
    _, st, near, _ = o.apply(np.array([[108, 95, 100]], np.uint8))
    assert st[0] == 0 and near[0] & 1
    _hand_state(o)
    _, st, _, _ = o.apply(np.array([[109, 100, 100]], np.uint8))
    assert st[0] == 2
    _hand_state(o, label=1)             # a foreground pixel never exits at stage 0
    _, st, _, _ = o.apply(np.array([[100, 100, 100]], np.uint8))
    assert st[0] != 0


def test_hand_confidence_terms():
    # a = 153/255 = .6, b = 51/255 = .2, g = .2; C- = .5, eta = 1/8
    # stage 1 (I = (104,100,98), J = (100,100,100)): D = 4, t_r = .16
    #   c = .6 + .2 (1 - 4/255) + .2 (1 - .16);  C = 7/8 * 1/2 + c / 8
    o = one_pixel(flags=ORC_RGA | ORC_CONF, **HAND)
    _hand_state(o)
    o.apply(np.array([[104, 100, 98]], np.uint8))
    c = Fraction(3, 5) + Fraction(1, 5) * (1 - Fraction(4, 255)) + Fraction(1, 5) * (1 - Fraction(4, 25))
    assert abs(o.state.conf[0] - float(Fraction(7, 16) + c / 8)) <= 1e-15
    # stage 2 with the prior at 200/255 everywhere: match comp0 (t = .16), D = 4
    #   c = .6 * 200/255 + .2 (1 - 4/255) + .2 (1 - .16)
    o = one_pixel(flags=ORC_CONF, **HAND)
    _hand_state(o)
    o.apply(np.array([[104, 100, 98]], np.uint8))
    c = Fraction(3, 5) * Fraction(200, 255) + Fraction(1, 5) * (1 - Fraction(4, 255)) \
        + Fraction(1, 5) * (1 - Fraction(4, 25))
    assert abs(o.state.conf[0] - float(Fraction(7, 16) + c / 8)) <= 1e-15
    # prior nullified (q = 5 < 13): the a term drops and b, g are renormalised
    #   c = (.2 (1 - 4/255) + .2 (1 - .16)) / .4
    o = one_pixel(flags=ORC_CONF, **HAND)
    _hand_state(o)
    o.state.kde[0] = 5
    o.apply(np.array([[104, 100, 98]], np.uint8))
    c = (Fraction(1, 5) * (1 - Fraction(4, 255)) + Fraction(1, 5) * (1 - Fraction(4, 25))) / Fraction(2, 5)
    assert abs(o.state.conf[0] - float(Fraction(7, 16) + c / 8)) <= 1e-15


def test_hand_confidence_prior_term_4bit():
    # the 4-bit prior enters as the fraction q / 15 of its peak: level 12
    # everywhere gives .6 * 12/15 in c, as the 8-bit level 204 = 17 * 12 does
    c_rest = Fraction(1, 5) * (1 - Fraction(4, 255)) + Fraction(1, 5) * (1 - Fraction(4, 25))
    for bits, level in ((4, 12), (8, 204)):
        o = one_pixel(flags=ORC_CONF, kde_bits=bits, **HAND)
        _hand_state(o)
        o.state.kde[0] = level
        o.apply(np.array([[104, 100, 98]], np.uint8))
        c = Fraction(3, 5) * Fraction(12, 15) + c_rest
        assert abs(o.state.conf[0] - float(Fraction(7, 16) + c / 8)) <= 1e-15, bits
    # nullified iff q / 15 < q_null / 255, i.e. 17 q < q_null: level 1 stays
    # at q_null = 17 (17 = 17) and drops at q_null = 18
    for q_null, dropped in ((17, False), (18, True), (13, False)):
        o = one_pixel(flags=ORC_CONF, kde_bits=4, q_null=q_null, **HAND)
        _hand_state(o)
        o.state.kde[0] = 1
        o.apply(np.array([[104, 100, 98]], np.uint8))
        c = c_rest / Fraction(2, 5) if dropped else Fraction(3, 5) * Fraction(1, 15) + c_rest
        assert abs(o.state.conf[0] - float(Fraction(7, 16) + c / 8)) <= 1e-15, q_null
    # level 0 is nullified at the default q_null = 13
    o = one_pixel(flags=ORC_CONF, kde_bits=4, **HAND)
    _hand_state(o)
    o.state.kde[0] = 0
    o.apply(np.array([[104, 100, 98]], np.uint8))
    assert abs(o.state.conf[0] - float(Fraction(7, 16) + c_rest / Fraction(2, 5) / 8)) <= 1e-15


@pytest.mark.parametrize("flags", [ORC_FD | ORC_RGA | ORC_CONF | ORC_ILLUM, ORC_CONF])
def test_kde4_equals_kde8_at_17_times_the_levels(flags):
    # the prior enters as q / Q: a 4-bit level q and the 8-bit level 17 q
    # are the same fraction of the peak (q/15 = 17q/255, both divisions
    # correctly rounded from one rational), and 255 q < 15 q_null exactly
    # when 17 q < q_null.  Runs from one random state, the 4-bit one with
    # levels q and the 8-bit one with 17 q, must agree bit for bit.
    from cog_harness import random_frame, random_state, set_oracle_state
    rng = np.random.default_rng(21)
    W, H, K = 31, 17, 3
    P = W * H
    st = random_state(rng, P, K, kde_bits=4)
    st8 = dict(st, kde=(17 * st["kde"].astype(np.uint16)).astype(np.uint8))
    runs = []
    for bits, state in ((4, st), (8, st8)):
        o = Oracle(dict(default_params(W, H, K), flags=flags, kde_bits=bits))
        set_oracle_state(o, state)
        runs.append(o)
    frames = [random_frame(np.random.default_rng(100 + t), st) for t in range(6)]
    for f in frames:
        r4, r8 = runs[0].apply(f), runs[1].apply(f)
        assert np.array_equal(r4[0], r8[0]) and np.array_equal(r4[1], r8[1])
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf", "label"):
        assert np.array_equal(getattr(runs[0].state, k), getattr(runs[1].state, k)), k


def test_kde_bits_other_than_8_or_4_rejected():
    with pytest.raises(Exception):
        one_pixel(kde_bits=6).train(np.zeros((3, 1, 3), np.uint8))


def test_confidence_modulates_rate_and_halts_rga():
    # C- = .95 >= c_halt: the running average does not move; the rate factor
    # (1.5 - C) applies to the mixture: a_eff = .25 * .55
    o = one_pixel(flags=ORC_RGA | ORC_CONF, **HAND)
    _hand_state(o)
    o.state.conf[0] = 0.95
    _, st, _, _ = o.apply(np.array([[104, 100, 98]], np.uint8))
    assert st[0] == 1 and list(o.state.rga_m[0]) == [100.0] * 3
    o = one_pixel(flags=ORC_CONF, **HAND)
    _hand_state(o)
    o.state.conf[0] = 0.95
    o.apply(np.array([[104, 100, 98]], np.uint8))
    ae = 0.25 * (1.5 - 0.95)
    assert abs(o.state.mu[0, 0, 0] - (100 + ae * 4)) <= 1e-12


def test_near_threshold_record():
    # t_r within 1e-4 of 1 is recorded; far from it is not
    o = one_pixel(flags=ORC_RGA, **HAND)
    _hand_state(o)
    o.state.rga_v[0] = [16 * 16 / 6.25 * (1 - 3e-5)] * 3   # t = 16^2 / (6.25 v) ~ 1 + 3e-5
    _, _, near, _ = o.apply(np.array([[116, 100, 100]], np.uint8))
    assert near[0] & 2
    _hand_state(o)
    _, _, near, _ = o.apply(np.array([[104, 100, 98]], np.uint8))
    assert near[0] == 0


def test_training_near_record():
    # two training frames; frame 1 differs from frame 0 by d on one channel,
    # and component 0 starts at (I_0, v_init).  With lambda^2 v_init = 256
    # the warm-up's match statistic is d^2 / 256: exactly 1 for d = 16 (a
    # decision on the threshold, recorded), 0.39 for d = 10 (not recorded)
    v = 256 / 6.25
    o = one_pixel(var_init=v)
    near = o.train(np.array([[[100, 100, 100]], [[116, 100, 100]]], np.uint8), want_near=True)
    assert near[0] & 4
    o = one_pixel(var_init=v)
    near = o.train(np.array([[[100, 100, 100]], [[110, 100, 100]]], np.uint8), want_near=True)
    assert near[0] == 0
    # constant training: every decision is far from its threshold
    o = one_pixel()
    assert (o.train(np.full((30, 1, 3), 90, np.uint8), want_near=True) == 0).all()


# ------------------------------------------------------ temporal sampling
from oracle import ORC_SAMPLE  # noqa: E402


def test_sampling_saturated_pixel_follows_its_block_phase():
    # Sec. 2 "Confidence based temporal sampling": once C >= c_skip a pixel
    # is looked at only on frames n with (n + p/64) % S == 0; before that it
    # is processed on every frame.  Two blocks (x = 0 and x = 64) have phases
    # one frame apart.
    S = 4
    p = default_params(128, 1, 3)
    p.update(flags=ORC_FD | ORC_CONF | ORC_SAMPLE, c_skip=0.95, skip_period=S)
    o = Oracle(p)
    o.train(np.full((10, 128, 3), 90, np.uint8))
    seen_skip = False
    for n in range(60):
        before = o.state.copy()
        _, st, _, stats = o.apply(np.full((128, 3), 90, np.uint8))
        for x, blk in ((0, 0), (64, 1)):
            Cm = before.conf[x]
            if Cm >= 0.95 and (n + blk) % S != 0:
                assert st[x] == 5
                seen_skip = True
                # skipped: every piece of state is unchanged
                assert o.state.conf[x] == Cm and o.state.label[x] == before.label[x]
                assert np.array_equal(o.state.prev[x], before.prev[x])
            else:
                assert st[x] == 0
        assert stats["n_stage"][5] == int((st == 5).sum())
    assert seen_skip
    # every pixel of a block shares its phase
    assert np.array_equal(st[:64], np.full(64, st[0])) and np.array_equal(st[64:], np.full(64, st[64]))


def test_sampling_delays_detection_by_less_than_one_period():
    S = 4
    p = default_params(1, 1, 3)
    p.update(flags=ORC_FD | ORC_RGA | ORC_CONF | ORC_SAMPLE, c_skip=0.95, skip_period=S)
    o = Oracle(p)
    o.train(np.full((10, 1, 3), 90, np.uint8))
    n = 0
    while not (o.state.conf[0] >= 0.95 and (n + 1) % S == 1):   # saturated, next frame off phase
        o.apply(np.full((1, 3), 90, np.uint8))
        n += 1
    # an object arrives on an off-phase frame: the label is carried until the
    # block's next phase frame, where the object is detected
    labels = []
    for k in range(S):
        m, st, _, _ = o.apply(np.full((1, 3), 200, np.uint8))
        labels.append((int(m[0]), int(st[0]), (n + k) % S))
    first = next(i for i, (lab, _, _) in enumerate(labels) if lab == 255)
    assert labels[first][2] == 0 and first <= S - 1
    assert all(s == 5 for _, s, _ in labels[:first])


def test_sampling_needs_confidence_below_threshold_processed_every_frame():
    p = default_params(1, 1, 3)
    p.update(flags=ORC_FD | ORC_CONF | ORC_SAMPLE, c_skip=0.999, skip_period=4)
    o = Oracle(p)
    o.train(np.full((10, 1, 3), 90, np.uint8))
    for n in range(20):           # C stays below 0.999 for these frames
        _, st, _, _ = o.apply(np.full((1, 3), 90, np.uint8))
        assert st[0] == 0


# ------------------------------------------------ stage 1 as the rank-1 mode
from oracle import ORC_MODE1  # noqa: E402


def test_mode1_writes_the_stage1_copy_back_on_the_transition():
    # hand state: keys .015625 (comp0), .0225 (comp1), .000625 (comp2), so the
    # rank-1 mode is comp1 (50, 4).  Stage 1 has moved its copy to
    # (52, 50, 50) / 5.  I = (150, 150, 150) fails stage 1 (t = 98^2 / 31.25)
    # and matches no mode (comp0: 50^2/100 = 25; comp2: 50^2/400 = 6.25), so
    # the weights decay, the lowest-ranked comp2 restarts at I, and comp1 --
    # unmatched -- keeps exactly the written-back copy (52, 50, 50) / 5.
    # Without the flag it would still read (50, 50, 50) / 4.
    for flags, mu1, v1 in ((ORC_RGA | ORC_MODE1, [52, 50, 50], 5.0), (ORC_RGA, [50, 50, 50], 4.0)):
        o = one_pixel(flags=flags, **HAND)
        _hand_state(o, label=1)
        o.state.top[0] = 1
        o.state.rga_m[0] = [52, 50, 50]
        o.state.rga_v[0] = [5, 5, 5]
        m, st, _, _ = o.apply(np.array([[150, 150, 150]], np.uint8))
        assert st[0] == 3 and m[0] == 255
        assert list(o.state.mu[0, 1]) == mu1 and list(o.state.var[0, 1]) == [v1] * 3
        assert list(o.state.mu[0, 2]) == [150, 150, 150]
    # with the flag the copy then follows the new rank-1 mode: weights
    # (.375, .225, .05)/.65 give keys .333/16, .12/5, .0059/100 -> comp1
    o = one_pixel(flags=ORC_RGA | ORC_MODE1, **HAND)
    _hand_state(o, label=1)
    o.state.top[0] = 1
    o.state.rga_m[0] = [52, 50, 50]
    o.state.rga_v[0] = [5, 5, 5]
    o.apply(np.array([[150, 150, 150]], np.uint8))
    assert o.state.top[0] == 1
    assert list(o.state.rga_m[0]) == [52, 50, 50] and list(o.state.rga_v[0]) == [5, 5, 5]


def test_mode1_copy_is_the_rank1_mode_after_every_stage2_visit():
    from cogsynth import Scene
    W, H, K = 24, 16, 3
    sc = Scene(W, H, 11, kind="dynamic", n_train=30, fg_frac=0.1, switch_at=20)
    p = default_params(W, H, K)
    p["flags"] = ALL | ORC_MODE1
    o = Oracle(p)
    tr, _ = sc.frames(0, 30)
    o.train(tr)
    s = o.state
    for t in range(30, 80):
        f, _ = sc.render(t)
        _, st, _, _ = o.apply(f)
        for q in np.nonzero(st >= 2)[0]:
            key = s.w[q] ** 2 / s.var[q].mean(axis=1)
            k1 = int(np.argmax(key))            # first maximum = lowest index on ties
            assert s.top[q] == k1
            assert np.array_equal(s.rga_m[q], s.mu[q, k1]) and np.array_equal(s.rga_v[q], s.var[q, k1])


def test_mode1_alone_is_the_plain_mixture():
    # with stage 1 off the copy is only ever set from the mixture, so the
    # write-back is the identity and the result is the plain mixture
    from cogsynth import Scene
    sc = Scene(32, 20, 5, kind="dynamic", n_train=25, fg_frac=0.05, switch_at=10)
    p = default_params(32, 20, 3)
    p["flags"] = ORC_MODE1
    o = Oracle(p)
    tr, _ = sc.frames(0, 25)
    o.train(tr)
    w, mu, var = o.state.w.copy(), o.state.mu.copy(), o.state.var.copy()
    for t in range(25, 60):
        f, _ = sc.render(t)
        m1, _, _, _ = o.apply(f)
        assert np.array_equal(m1, o.plain_gmm(w, mu, var, f))
        assert np.array_equal(mu, o.state.mu) and np.array_equal(var, o.state.var)


# ------------------------------------------------ per-channel mixtures
from oracle import ORC_PERCHAN  # noqa: E402


def test_perchan_on_gray_input_is_the_shared_mixture():
    # with R = G = B in every frame and every state, the three per-channel
    # mixtures are copies of the shared-weight one: same keys, matches,
    # updates and decisions, so masks, stage maps and means/variances agree
    # and each channel's weights equal the shared weights
    from cogsynth import Scene
    W, H, K = 40, 24, 3
    sc = Scene(W, H, 21, kind="dynamic", n_train=30, fg_frac=0.1, switch_at=15)
    fr, _ = sc.frames(0, 70)
    gray = np.repeat(fr[..., :1], 3, axis=-1)
    runs = []
    for extra in (0, ORC_PERCHAN):
        p = default_params(W, H, K)
        p["flags"] = ALL | extra
        o = Oracle(p)
        o.train(gray[:30])
        out = [o.apply(gray[t])[:2] for t in range(30, 70)]
        runs.append((o, out))
    (a, oa), (b, ob) = runs
    for (ma, sa), (mb, sb) in zip(oa, ob):
        assert np.array_equal(ma, mb) and np.array_equal(sa, sb)
    assert np.array_equal(a.state.mu, b.state.mu) and np.array_equal(a.state.var, b.state.var)
    for c in range(3):
        assert np.array_equal(b.state.wc[:, c, :], a.state.w)


def test_perchan_channels_are_independent():
    # with every other stage off each channel's mixture sees only its own
    # values: changing channel 1 leaves channels 0 and 2 bit-identical
    from cogsynth import Scene
    W, H, K = 32, 20, 3
    sc = Scene(W, H, 22, kind="dynamic", n_train=25, fg_frac=0.1, switch_at=12)
    fr, _ = sc.frames(0, 60)
    alt = fr.copy()
    alt[..., 1] = 255 - alt[..., 1]
    st = []
    for f in (fr, alt):
        p = default_params(W, H, K)
        p["flags"] = ORC_PERCHAN
        o = Oracle(p)
        o.train(f[:25])
        for t in range(25, 60):
            o.apply(f[t])
        st.append(o.state)
    for c in (0, 2):
        assert np.array_equal(st[0].wc[:, c], st[1].wc[:, c])
        assert np.array_equal(st[0].mu[:, :, c], st[1].mu[:, :, c])
        assert np.array_equal(st[0].var[:, :, c], st[1].var[:, :, c])
    assert not np.array_equal(st[0].wc[:, 1], st[1].wc[:, 1])


def test_hand_perchan_one_channel_behind_too_much_weight_is_foreground():
    # every channel: comp0 (100, v 16), comp1 (50, v 4), comp2 (200, v 64);
    # weights ch0 = ch2 = (.5, .3, .2), ch1 = (.2, .75, .05); I = (104, 100, 98)
    # ch0: keys .015625 / .0225 / .000625 -> order 1, 0, 2; comp0 matches at
    #      rank 2 (t = 16/100), S = .3 -> BG; w = (.625, .225, .15), mu0 = 101,
    #      v0 = .75*16 + .25*3^2 = 14.25
    # ch1: keys .0025 / .140625 / .0000390625 -> order 1, 0, 2; comp0 matches
    #      (t = 0), S = .75 > .7 -> FG; w = (.4, .5625, .0375), mu0 = 100, v0 = 12
    # ch2: as ch0 with t = 4/100: BG; mu0 = 99.5, v0 = .75*16 + .25*1.5^2 = 12.5625
    # the pixel is FG (one channel is); no transition update
    o = one_pixel(flags=ORC_PERCHAN, **HAND)
    _hand_state(o)
    o.state.wc[0, 0] = [0.5, 0.3, 0.2]
    o.state.wc[0, 1] = [0.2, 0.75, 0.05]
    o.state.wc[0, 2] = [0.5, 0.3, 0.2]
    rga0 = o.state.rga_m[0].copy()
    m, st, _, _ = o.apply(np.array([[104, 100, 98]], np.uint8))
    assert m[0] == 255 and st[0] == 3
    assert np.allclose(o.state.wc[0, 0], [0.625, 0.225, 0.15], rtol=0, atol=1e-15)
    assert np.allclose(o.state.wc[0, 1], [0.4, 0.5625, 0.0375], rtol=0, atol=1e-15)
    assert list(o.state.mu[0, 0]) == [101, 100, 99.5]
    assert list(o.state.var[0, 0]) == [14.25, 12, 12.5625]
    assert np.array_equal(o.state.rga_m[0], rga0)


def test_oracle_results_do_not_depend_on_its_thread_count():
    # OpenMP only distributes independent pixels (integer reductions): one
    # thread and several give identical training, masks, stage maps and state
    from cogsynth import Scene
    import oracle
    sc = Scene(48, 32, 11, kind="dynamic", n_train=20, fg_frac=0.1, switch_at=3)
    fr, _ = sc.frames(0, 30)
    out = []
    n0 = oracle.oracle_threads()
    try:
        for th in (1, max(2, n0)):
            oracle.set_threads(th)
            o = Oracle(default_params(48, 32, 3))
            o.train(fr[:20])
            res = [o.apply(fr[t])[:2] for t in range(20, 30)]
            out.append((res, o.state.w.copy(), o.state.var.copy(), o.state.kde.copy()))
    finally:
        oracle.set_threads(n0)
    (r1, w1, v1, k1), (r2, w2, v2, k2) = out
    for (m1, s1), (m2, s2) in zip(r1, r2):
        assert np.array_equal(m1, m2) and np.array_equal(s1, s2)
    assert np.array_equal(w1, w2) and np.array_equal(v1, v2) and np.array_equal(k1, k2)
