"""Host logic of the proposal-net evaluation: the flow-quality measure and the
equal-inlier comparison that the benchmark reports. CPU only."""
import numpy as np

from paper_1508_05151_gb300 import train


def test_flow_quality_threshold_and_mask():
    gt = np.zeros((1, 2, 3, 2))
    flow = np.zeros((1, 2, 3, 2), np.int16)
    flow[0, 0, 0] = (3, 0)      # endpoint error exactly 3: an inlier
    flow[0, 0, 1] = (2, 3)      # sqrt(13) > 3: an outlier
    flow[0, 0, 2] = (0, -4)     # 4: an outlier, but occluded
    flow[0, 1, 0] = (-1, 0)     # 1
    occ = np.zeros((1, 2, 3), bool)
    occ[0, 0, 2] = True
    inl, epe = train.flow_quality(flow, gt, occ)
    assert inl == 4 / 5
    assert np.isclose(epe, (3 + np.sqrt(13) + 1) / 5)


def _arms(**kw):
    return {"arms": {k: {"ms_per_pair": ms, "inliers_3px": inl} for k, (ms, inl) in kw.items()}}


def test_equal_inlier_point_picks_the_cheapest_arm_reaching_the_reference():
    ev = _arms(plain_rs3=(4.0, 0.90), plain_rs2=(3.8, 0.89),
               learned_rs1=(3.5, 0.85), learned_rs2=(3.7, 0.90), learned_rs3=(4.1, 0.91))
    eq = train.equal_inlier_point(ev)
    assert eq["arm"] == "learned_rs2"           # equal inliers count as reaching it
    assert eq["ms_per_pair"] == 3.7 and eq["ref_ms_per_pair"] == 4.0
    assert eq["speedup"] == round(4.0 / 3.7, 4)


def test_equal_inlier_point_none_when_no_learned_arm_reaches_it():
    ev = _arms(plain_rs3=(4.0, 0.92), plain_rs1=(3.0, 0.95), learned_rs3=(4.1, 0.91999))
    assert train.equal_inlier_point(ev) is None


def test_equal_inlier_point_defaults_to_the_largest_plain_budget():
    ev = _arms(plain_rs1=(3.0, 0.80), learned_rs1=(3.1, 0.81))
    eq = train.equal_inlier_point(ev)
    assert eq["ref"] == "plain_rs1" and eq["arm"] == "learned_rs1"
    ev = _arms(plain_rs1=(3.0, 0.80), plain_rs12=(5.0, 0.95), learned_rs1=(3.1, 0.81))
    assert train.equal_inlier_point(ev) is None


def test_paired_inlier_delta():
    gt = np.zeros((3, 1, 4, 2))
    occ = np.zeros((3, 1, 4), bool)
    a = np.zeros((3, 1, 4, 2), np.int16)
    b = np.zeros((3, 1, 4, 2), np.int16)
    b[0, 0, :1] = (9, 0)        # pair 0: a 4/4 inliers, b 3/4 -> +0.25
    a[1, 0, :2] = (0, 5)        # pair 1: a 2/4, b 4/4 -> -0.5
    occ[2, 0, 0] = True         # pair 2: equal -> 0 (the occluded pixel does not count)
    a[2, 0, 0] = (7, 7)
    d = train.paired_inlier_delta(a, b, gt, occ)
    diffs = np.array([0.25, -0.5, 0.0])
    assert d["pairs"] == 3
    assert np.isclose(d["mean"], diffs.mean())
    assert np.isclose(d["se"], diffs.std(ddof=1) / np.sqrt(3))
