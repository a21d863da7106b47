"""Pins of the oracle's selection of salient regions (Sec. 2.3, end; Sec.
3.1) on hand-made candidate lists whose answers are written out here."""
import numpy as np


def C(x, y, z, r, source, H, W):
    return dict(x=x, y=y, z=z, r=r, source=source, H=H, W=W)


def keys(sel):
    return [(c["x"], c["y"], c["z"], c["r"], c["source"]) for c in sel]


def test_threshold_is_strict_and_scale_zero_is_dropped(ko):
    cands = [C(1, 1, 1, 5, 0, 2.0, 0.3), C(2, 2, 2, 5, 1, 1.5, 0.9), C(3, 3, 3, 0, 2, 3.0, 5.0),
             C(4, 4, 4, 6, 3, 1.5000000001, 0.1)]
    assert keys(ko.select_salient(cands, h_min=1.5, top_k=20)) == [(1, 1, 1, 5, 0), (4, 4, 4, 6, 3)]


def test_duplicates_merge_to_the_smallest_source(ko):
    cands = [C(5, 6, 7, 4, 9, 2.0, 0.5), C(5, 6, 7, 4, 2, 2.0, 0.5), C(5, 6, 7, 5, 1, 2.1, 0.4),
             C(5, 6, 7, 4, 7, 2.0, 0.5)]
    assert keys(ko.select_salient(cands, top_k=20)) == [(5, 6, 7, 4, 2), (5, 6, 7, 5, 1)]


def test_order_W_then_H_then_position(ko):
    cands = [C(0, 0, 1, 4, 0, 1.0, 0.5), C(0, 1, 0, 4, 1, 1.0, 0.5), C(1, 0, 0, 4, 2, 1.0, 0.5),
             C(0, 0, 0, 5, 3, 1.0, 0.5), C(0, 0, 0, 4, 4, 1.0, 0.5), C(9, 9, 9, 4, 5, 2.0, 0.5),
             C(9, 9, 9, 9, 6, 0.1, 0.7)]
    # W desc; among W = 0.5: H desc, then z, y, x, r ascending
    assert keys(ko.select_salient(cands, h_min=0.0, top_k=20)) == [
        (9, 9, 9, 9, 6), (9, 9, 9, 4, 5), (0, 0, 0, 4, 4), (0, 0, 0, 5, 3), (1, 0, 0, 4, 2),
        (0, 1, 0, 4, 1), (0, 0, 1, 4, 0)]


def test_top_k_cuts_after_merging(ko):
    cands = [C(i % 3, 0, 0, 4, i, 1.0, float(i % 3)) for i in range(30)]
    sel = ko.select_salient(cands, top_k=2)
    assert keys(sel) == [(2, 0, 0, 4, 2), (1, 0, 0, 4, 1)]
    assert ko.select_salient([], top_k=5) == []


def test_octant_candidates_carry_the_final_kb_evaluation(ko):
    res = {"xyz": np.array([[1, 2, 3], [4, 5, 6]], np.int32), "s": np.array([7, 0], np.uint8),
           "H": np.array([1.25, 0.0]), "W": np.array([0.5, 0.0])}
    assert ko.octant_candidates(res) == [C(1, 2, 3, 7, 0, 1.25, 0.5), C(4, 5, 6, 0, 1, 0.0, 0.0)]
