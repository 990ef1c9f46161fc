"""The no-allocation entry point against the plan-based one and the oracle.

ofdm_radar_process_noalloc serves callers that cannot allocate device
memory (and so cannot create a plan): its tables and workspace sit in a
fixed array inside the library.  Two calls in a row on fresh inputs must
give what ofdm_radar_process gives on the same inputs, within the chain's
tolerances, and match the FP64 oracle; calls with other parameters must
rebuild the tables in the array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import (MAP_TOL, check_detections_vs_fp64, make_frames, oracle_params, plan_kwargs, rel_l2,
                         stack_lk)

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


def _compare_with_plan(radar, torch, dev, p, frames, fr):
    """One no-allocation call against a plan call on the same inputs; the
    first frame also against the oracle."""
    params = radar.default_params(**plan_kwargs(p, frames))
    plan = radar.Plan(radar.default_params(**plan_kwargs(p, frames)))
    Y = torch.from_numpy(stack_lk([f[2] for f in fr])).to(dev)
    X = torch.from_numpy(stack_lk([f[0].A for f in fr])).to(dev)
    ref = _outputs(radar, torch, dev, frames, p.Np, p.Mp, p.max_targets)
    got = _outputs(radar, torch, dev, frames, p.Np, p.Mp, p.max_targets)
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
    # the oracle on the first frame of the call
    frm, _, Yf = fr[0]
    want = o.process(Yf, frm.A, p)
    assert rel_l2(m_got[0], want["P"]) < MAP_TOL
    n = int(got[2][0])
    check_detections_vs_fp64([(int(t["r"]), int(t["s"])) for t in tg[0][:n]], tg[0]["power"][:n],
                             want["det"], want["P"])
    plan.close()


def test_noalloc_matches_plan_path_on_two_calls(env):
    radar, torch, dev = env
    frames = 12
    cfg, fr = make_frames(2, 2 * frames)
    p = oracle_params(cfg)
    for call in range(2):
        _compare_with_plan(radar, torch, dev, p, frames, fr[call * frames:(call + 1) * frames])


# Other parameter sets in a row: each call must rebuild the tables in the
# array (N >= 2048 pass twiddles, M' <= 32 roots, rect window, q' != 0,
# Doppler padding M' > M) and still agree with a plan built for it.
OTHER = [
    dict(N=2048, M=16, L_cp=256, window=o.WINDOW_RECT, zc_root=3, zc_q=3),
    dict(N=256, M=64, L_cp=32, window=o.WINDOW_HAMMING, zc_root=1, zc_q=0, M_pad=128),
    dict(N=1024, M=256, L_cp=128, window=o.WINDOW_HANN, zc_root=1, zc_q=0),
]


def test_noalloc_rebuilds_tables_when_parameters_change(env):
    radar, torch, dev = env
    for j, kw in enumerate(OTHER):
        base = syn.FrameConfig(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], qam=16, zc_root=kw["zc_root"], n_targets=3,
                               on_grid=False, amp_db=(-6.0, 0.0), snr_db=(0.0, 0.0), window=kw["window"],
                               detect_k=4)
        fr = []
        for f in range(2):
            d = syn.draw_frame(base, 9100 + 10 * j + f)
            Xp = o.zc_precode(d.A, kw["zc_root"], kw["zc_q"])
            fr.append((d, Xp, syn.received(d, Xp)))
        p = o.Params(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], zc_root=kw["zc_root"], zc_q=kw["zc_q"],
                     window=kw["window"], max_targets=4, M_pad=kw.get("M_pad", 0))
        _compare_with_plan(radar, torch, dev, p, 2, fr)


def test_noalloc_rejects_requests_beyond_its_array(env):
    radar, torch, dev = env
    cfg, _ = make_frames(2, 1)
    p = oracle_params(cfg)
    params = radar.default_params(**plan_kwargs(p, 1))
    Y = torch.zeros((1, cfg.M, cfg.N), dtype=torch.complex64, device=dev)
    with pytest.raises(radar.OfdmError) as ei:
        radar.ofdm_radar_process_noalloc(params, Y, Y, 64)   # 64 * 130 * 256 cells > 2^20
    assert ei.value.code == -2
    with pytest.raises(radar.OfdmError) as ei:
        radar.ofdm_radar_process_noalloc(params, Y, Y, 5000)  # more frames than the array holds
    assert ei.value.code == -2
