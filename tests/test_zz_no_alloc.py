"""The no-allocation entry point against the plan-based one.

ofdm_radar_process_noalloc serves callers that cannot allocate device
memory (and so cannot create a plan): its tables and workspace sit in a
fixed array inside the library.  Two calls in a row on fresh inputs must
give what ofdm_radar_process gives on the same inputs, within the chain's
tolerances.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from radar_cases import MAP_TOL, make_frames, oracle_params, plan_kwargs, rel_l2, stack_lk

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


def _outputs(radar, torch, dev, frames, Np, Mp, K):
    return (torch.full((frames, Np, Mp), -1.0, dtype=torch.float32, device=dev),
            torch.zeros((frames * K * radar.TARGET_BYTES,), dtype=torch.uint8, device=dev),
            torch.full((frames,), -1, dtype=torch.int32, device=dev),
            torch.full((frames,), -1, dtype=torch.int32, device=dev))


def test_noalloc_matches_plan_path_on_two_calls(env):
    radar, torch, dev = env
    frames = 12
    cfg, fr = make_frames(2, 2 * frames)
    p = oracle_params(cfg)
    params = radar.default_params(**plan_kwargs(p, frames))
    plan = radar.Plan(radar.default_params(**plan_kwargs(p, frames)))
    for call in range(2):
        chunk = fr[call * frames:(call + 1) * frames]
        Y = torch.from_numpy(stack_lk([f[2] for f in chunk])).to(dev)
        X = torch.from_numpy(stack_lk([f[0].A for f in chunk])).to(dev)
        ref = _outputs(radar, torch, dev, frames, cfg.N, cfg.M, p.max_targets)
        got = _outputs(radar, torch, dev, frames, cfg.N, cfg.M, p.max_targets)
        radar.ofdm_radar_process(plan, Y, X, frames, *ref)
        radar.ofdm_radar_process_noalloc(params, Y, X, frames, *got)
        torch.cuda.synchronize()
        m_ref, m_got = ref[0].cpu().numpy(), got[0].cpu().numpy()
        for i in range(frames):
            assert rel_l2(m_got[i], m_ref[i]) < MAP_TOL
        assert np.array_equal(got[2].cpu().numpy(), ref[2].cpu().numpy())
        assert np.array_equal(got[3].cpu().numpy(), ref[3].cpu().numpy())
        tr = radar.targets_view(ref[1], frames, p.max_targets)
        tg = radar.targets_view(got[1], frames, p.max_targets)
        for i in range(frames):
            n = int(ref[2][i])
            assert [(int(t["r"]), int(t["s"])) for t in tg[i][:n]] == \
                [(int(t["r"]), int(t["s"])) for t in tr[i][:n]]
            assert np.allclose(tg[i]["power"][:n], tr[i]["power"][:n], rtol=MAP_TOL)


def test_noalloc_rejects_requests_beyond_its_array(env):
    radar, torch, dev = env
    cfg, _ = make_frames(2, 1)
    p = oracle_params(cfg)
    params = radar.default_params(**plan_kwargs(p, 1))
    Y = torch.zeros((1, cfg.M, cfg.N), dtype=torch.complex64, device=dev)
    with pytest.raises(radar.OfdmError) as ei:
        radar.ofdm_radar_process_noalloc(params, Y, Y, 64)   # 64 * 130 * 256 cells > 2^20
    assert ei.value.code == -2
