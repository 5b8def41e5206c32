"""Host logic of the learned-closure evaluation (no GPU): training windows and paired statistics."""

import math

import torch

from paper_2604_18536_b300 import les


def test_training_windows_cover_each_trajectory_at_the_stride():
    data = [(torch.arange(41.0).reshape(41, 1), 0.1), (torch.arange(41.0).reshape(41, 1) + 100, 0.2)]
    w = les.training_windows(data, 10, 5)
    assert len(w) == 2 * 7                      # starts 0, 5, ..., 30
    snaps, dt = w[3]
    assert snaps.shape[0] == 11 and snaps[0, 0].item() == 15.0 and snaps[-1, 0].item() == 25.0 and dt == 0.1
    assert w[7][0][0, 0].item() == 100.0 and w[7][1] == 0.2


def test_paired_difference_and_standard_error():
    base = [1.0, 2.0, 3.0, 4.0]
    other = [0.5, 1.0, 3.5, 2.0]
    p = les.paired(base, other)
    d = [0.5, 1.0, -0.5, 2.0]
    m = sum(d) / 4
    sd = math.sqrt(sum((x - m) ** 2 for x in d) / 3)
    assert abs(p["mean_diff"] - m) < 1e-15 and abs(p["se"] - sd / 2) < 1e-15
    assert p["wins"] == 3 and p["n"] == 4
