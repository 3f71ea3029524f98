"""Threshold calibration of the vetter (host logic)."""
import numpy as np

from paper_2509_26279_gb300 import vetting


def test_calibrate_picks_lowest_threshold_meeting_purity():
    logits = np.array([5.0, 4.0, 3.0, 2.0, 1.0, 0.0])
    labels = np.array([1, 1, 0, 1, 0, 0])
    # precision from the top: 1, 1, 2/3, 3/4, 3/5, 1/2
    assert vetting.calibrate(logits, labels, 0.75) == 2.0
    assert vetting.calibrate(logits, labels, 0.95) == 4.0
    assert vetting.calibrate(logits, labels, 0.5) == 0.0
    assert vetting.calibrate(logits, np.zeros(6), 0.5) == float("inf")


def test_vetted_keep_keeps_plain_threshold_candidates():
    keep = vetting.vetted_keep([30, 10, 10, 25], [-5.0, 2.0, -1.0, -9.0], 25, 0.5)
    assert keep.tolist() == [True, True, False, True]


def test_vetted_mask_is_a_superset_of_the_plain_threshold():
    counts = np.array([30, 10, 10, 25, 7])
    m = vetting.vetted_mask(counts, [1, 2, 3], [2.0, -1.0, -9.0], 25, 0.5)
    assert m.tolist() == [True, True, False, True, False]
