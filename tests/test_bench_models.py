"""The benchmark's algorithmic byte models (the numerators of every roofline
figure it reports) against the per-pixel tables they state, worked by hand.
Host logic only."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_cascade_bytes_fp16_k5():
    # every pixel: I 3 + J 3 + label 1 + C 2 read, mask 1 + label 1 + C 2
    # written = 13 B; past stage 0: qa|qb 2 + running average 12 = 14 B more;
    # at the mixture stage: 2 x 35 values x 2 B + 96 B prior sectors + 12 B
    # reseed = 248 B
    P, frames = 1000, 2
    st = {"n_stage": [1200, 500, 200, 80, 20, 0], "n_gmm": 300, "frames": frames}
    k1, k2 = bench.cog_bytes(st, P, 2, 5)
    past0 = 500 + 300
    assert k1 == frames * P * 13 + past0 * 26
    assert k2 == 300 * 248


def test_cascade_bytes_fp32_k3_and_skipped_pixels():
    # FP32 (e = 4): 9 + 2e = 17 B per pixel; a pixel skipped by the sampling
    # reads J, label and C and writes its mask: 3 + 1 + 4 + 1 = 9 B;
    # past stage 0: 2 + 12e = 50 B; mixture stage: 2 x 21 x 4 + 96 + 24 = 288 B
    P, frames = 100, 1
    st = {"n_stage": [40, 30, 10, 5, 0, 15], "n_gmm": 15, "frames": frames}
    k1, k2 = bench.cog_bytes(st, P, 4, 3)
    assert k1 == (100 - 15) * 17 + 15 * 9 + (30 + 15) * 50
    assert k2 == 15 * 288


def test_per_channel_record_bytes():
    # per-channel mixtures keep 9 values per component: 2 x 45 x 2 + 96 + 12
    st = {"n_stage": [0, 0, 0, 0, 0, 0], "n_gmm": 10, "frames": 1}
    _, k2 = bench.cog_bytes(st, 10, 2, 5, nv=9)
    assert k2 == 10 * (180 + 96 + 12)


def test_plain_mixture_bytes():
    # I 3 in, mask 1 out, 35 values in and out at 2 B: 144 B per pixel
    assert bench.plain_bytes(3, 1000, 2, 5) == 3 * 1000 * 144


def test_clip_bytes():
    # per pixel and launch: (J + label 4, C 2, running average 12 + 2)
    # read, written and copied to the undo log: 3 x 20 = 60 B; per pixel and
    # frame 4 B; per mixture-stage pixel 140 + 96 B
    st = {"frames": 32, "n_gmm": 50}
    assert bench.clip_bytes(st, 100, 2, 5, clips=1) == 100 * 60 + 32 * 100 * 4 + 50 * 236


def test_issue_peak_is_the_scheduler_count():
    # 152 SMs x 4 schedulers x 1 warp instruction per clock at 2070 MHz
    assert abs(bench.ISSUE_PEAK - 1.25856e12) < 1e6
