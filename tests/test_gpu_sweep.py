"""The Monte-Carlo RMSE-vs-SNR sweep at Table I's size (N = 2048, M = 560,
N_cp = 512) runs on the GPU for the three receivers; at high SNR every target
is found and the error is the off-grid rounding to the nearest bin (at most
half a bin, Eq. (19)).  The paper's comparison between the receivers is a
statistical observation, not a parity target."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_03883_gb300 import radar
    return radar, torch, torch.device("cuda:0")


def test_rmse_sweep_table1(env):
    import bench
    radar, torch, dev = env
    out = bench.rmse_sweep(radar, torch, dev, snrs=(20.0,), frames_per_snr=2)
    for form in ("zcp_dft_ce", "dft_ce", "ls"):
        assert out[form]["miss_rate"] == [0.0]
        assert out[form]["range_rmse_m"][0] <= 0.5 * out["range_resolution_m"] * (1 + 1e-9)
        assert out[form]["velocity_rmse_mps"][0] <= 0.5 * out["velocity_resolution_mps"] * (1 + 1e-9)
    # Table I's resolutions (Eq. (15) with N = 2048, M = 560, N_cp = 512): 30.52 cm and 0.67 m/s
    assert out["range_resolution_m"] == pytest.approx(0.3052, abs=5e-5)
    assert out["velocity_resolution_mps"] == pytest.approx(0.67, abs=5e-3)
    assert not math.isnan(out["zcp_dft_ce"]["range_rmse_m"][0])
