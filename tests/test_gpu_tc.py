"""The split-FP16 tensor-core column stage (precision OFDM_PREC_SPLIT_FP16)
against the FP64 oracle, through the C ABI.

Both 1024-point DFTs of the column stage (the ZC transform and DFT-CE's
inverse) run as 32-point DFT matrix products on the tensor cores with hi + lo
FP16 operands.  The gate is the split-precision one: periodogram relative L2
<= 1e-4, detected bins exact up to candidates within 1e-3 relative power.
Every frame of the benchmark batch is checked, plus the variants the kernel
supports and the inputs it must reject.
"""
import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import check_detections_vs_fp64, make_frames, oracle_params, plan_kwargs, rel_l2, stack_lk

pytestmark = pytest.mark.gpu

TC_TOL = 1e-4        # periodogram / strip relative L2 of the split-precision path
TC_NEAR_TIE = 1e-3   # relative power gap under which two detections may swap
TC_PEAK_TOL = 1e-3   # relative error of one detected peak's power
STATUS_TIMEOUT = 64  # OFDM_STATUS_TIMEOUT: a bounded wait inside the kernel ran out


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_03883_gb300 import radar
    return radar, torch, torch.device("cuda:0")


def tc_plan(radar, p, frames):
    return radar.Plan(precision=radar.PREC_SPLIT_FP16, **plan_kwargs(p, frames))


def run(env, p, fr, plan=None):
    radar, torch, dev = env
    frames = len(fr)
    plan = plan or tc_plan(radar, p, frames)
    Y = torch.from_numpy(stack_lk([f[2] for f in fr])).to(dev)
    X = torch.from_numpy(stack_lk([f[0].A if not p.x_is_precoded else f[1] for f in fr])).to(dev)
    out = radar.process(plan, Y, X)
    torch.cuda.synchronize()
    return dict(map=out["map"].cpu().numpy(), tg=radar.targets_view(out["targets"], frames, p.max_targets),
                n=out["n_targets"].cpu().numpy(), status=out["status"].cpu().numpy().view(np.uint32))


def check_frame(res, i, Y, A, p):
    ref = o.process(Y, A, p)
    assert rel_l2(res["map"][i], ref["P"]) < TC_TOL, f"frame {i}"
    n = int(res["n"][i])
    rs = [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]]
    check_detections_vs_fp64(rs, res["tg"][i]["power"][:n], ref["det"], ref["P"], near_tie=TC_NEAR_TIE,
                             peak_tol=TC_PEAK_TOL, map_tol=TC_TOL)
    assert int(res["status"][i]) & STATUS_TIMEOUT == 0


def test_tc_strip_matches_oracle(env):
    radar, torch, dev = env
    cfg, fr = make_frames(2, 3)
    p = oracle_params(cfg)
    plan = tc_plan(radar, p, 3)
    rows = plan.support_rows()
    Y = torch.from_numpy(stack_lk([f[2] for f in fr])).to(dev)
    X = torch.from_numpy(stack_lk([f[0].A for f in fr])).to(dev)
    strip = torch.empty((3, len(rows), cfg.M), dtype=torch.complex64, device=dev)
    radar.ofdm_radar_range_profile(plan, Y, X, 3, strip)
    torch.cuda.synchronize()
    s = strip.cpu().numpy()
    for i, (frm, Xp, Yf) in enumerate(fr):
        g = o.process(Yf, frm.A, p)["g"]
        assert rel_l2(s[i], g[rows, :]) < TC_TOL


def test_tc_every_bench_frame_matches_oracle(env):
    """64 frames of 1024 x 256 (the benchmark's launch), each in full."""
    cfg, fr = make_frames(2, 64)
    p = oracle_params(cfg)
    res = run(env, p, fr)
    for i, (frm, Xp, Y) in enumerate(fr):
        check_frame(res, i, Y, frm.A, p)


TC_VARIANTS = [
    ("no_zcp", dict(zc_root=0)),
    ("x_precoded", dict(x_is_precoded=True)),
    ("root3_q2", dict(zc_root=3, zc_q=2)),
    ("rect_lcp256", dict(window=o.WINDOW_RECT, L_cp=256)),
    ("hamming_lcp255", dict(window=o.WINDOW_HAMMING, L_cp=255)),
    ("hann_lcp5", dict(L_cp=5)),
    ("m16", dict(M=16)),
    ("doppler_pad", dict(M=64, M_pad=256)),
    ("threshold", dict(detect_mode=o.DETECT_THRESHOLD, max_targets=16)),
    ("m1024", dict(M=1024)),
]


@pytest.mark.parametrize("name,kw", TC_VARIANTS, ids=[v[0] for v in TC_VARIANTS])
def test_tc_variants(env, name, kw):
    N = 1024
    M = kw.get("M", 64)
    L = kw.get("L_cp", 128)
    zr, zq = kw.get("zc_root", 1), kw.get("zc_q", 0)
    base = syn.FrameConfig(N=N, M=M, L_cp=L, qam=16, zc_root=zr, n_targets=3 if L >= 8 else 0, on_grid=False,
                           amp_db=(-6.0, 0.0), snr_db=(0.0, 0.0), window=kw.get("window", o.WINDOW_HANN),
                           detect_k=4)
    fr = []
    for f in range(2):
        d = syn.draw_frame(base, 7700 + f)
        Xp = o.zc_precode(d.A, zr, zq) if zr else d.A
        fr.append((d, syn.as_complex64_values(Xp), syn.received(d, Xp)))
    p = o.Params(N=N, M=M, L_cp=L, zc_root=zr, zc_q=zq, window=base.window, max_targets=kw.get("max_targets", 4),
                 x_is_precoded=kw.get("x_is_precoded", False), M_pad=kw.get("M_pad", 0),
                 detect_mode=kw.get("detect_mode", o.DETECT_TOPK))
    res = run(env, p, fr)
    for i, (frm, Xp, Y) in enumerate(fr):
        check_frame(res, i, Y, Xp if p.x_is_precoded else frm.A, p)


def test_tc_single_frame_and_repeated_calls(env):
    """One frame (fewer tiles than warpgroups), then calls of other sizes on
    the same plan (the ticket counter carried across launches)."""
    radar, torch, dev = env
    cfg, fr = make_frames(2, 6)
    p = oracle_params(cfg)
    plan = tc_plan(radar, p, 6)
    for sl in (slice(0, 1), slice(1, 6), slice(0, 3)):
        sub = fr[sl]
        res = run(env, p, sub, plan=plan)
        for i, (frm, Xp, Y) in enumerate(sub):
            check_frame(res, i, Y, frm.A, p)


def test_tc_rejects_misaligned_buffers(env):
    radar, torch, dev = env
    cfg, fr = make_frames(2, 1)
    p = oracle_params(cfg)
    plan = tc_plan(radar, p, 1)
    n = cfg.N * cfg.M
    Y = torch.zeros((n + 1,), dtype=torch.complex64, device=dev)
    with pytest.raises(radar.OfdmError) as ei:
        radar.ofdm_radar_process(plan, Y[1:], Y[:n], 1)     # 8-byte offset: bulk copies need 16
    assert ei.value.code == -1
