"""The parity checker itself (CPU): the detection comparison used by the GPU
tests must accept exact agreement and genuine near-tie swaps, and reject a
wrong bin, a missing detection and a wrong power."""
import numpy as np
import pytest

from oracle import ofdm_oracle as o
from radar_cases import check_detections_vs_fp64


def _map():
    rng = np.random.default_rng(5)
    P = rng.random((32, 16)) * 1e-3
    P[4, 3], P[20, 12], P[11, 7] = 5.0, 3.0, 2.0
    P[27, 9] = 3.0 * (1 + 2e-6)          # near-tie with (20, 12): FP32 may order them either way
    return P


def _gpu(det, C):
    return [(int(r), int(s)) for r, s in zip(det.r, det.s)], det.power.astype(np.float32)


def test_exact_agreement_passes():
    P = _map()
    det = o.detect(P, o.DETECT_TOPK, 4)
    rs, pw = _gpu(det, P.shape[1])
    assert check_detections_vs_fp64(rs, pw, det, P) == 0


def test_near_tie_swap_accepted():
    P = _map()
    det = o.detect(P, o.DETECT_TOPK, 4)
    rs, pw = _gpu(det, P.shape[1])
    rs[1], rs[2] = rs[2], rs[1]
    pw[1], pw[2] = pw[2], pw[1]
    assert check_detections_vs_fp64(rs, pw, det, P) == 2


@pytest.mark.parametrize("mistake", ["wrong_bin", "dropped", "wrong_power", "non_peak_neighbour"])
def test_mistakes_rejected(mistake):
    P = _map()
    det = o.detect(P, o.DETECT_TOPK, 4)
    rs, pw = _gpu(det, P.shape[1])
    if mistake == "wrong_bin":
        rs[3] = (rs[3][0] + 5, rs[3][1])
    elif mistake == "dropped":
        rs, pw = rs[:3], pw[:3]
    elif mistake == "wrong_power":
        pw[0] *= 1.01
    else:                                 # the neighbour of a near-tie peak is not a peak
        rs[1] = (rs[1][0], rs[1][1] + 1)
    with pytest.raises(AssertionError):
        check_detections_vs_fp64(rs, pw, det, P)
