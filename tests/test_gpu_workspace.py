"""Memory safety of the kernels without a sanitizer: every device buffer the
library allocates ends in a 256-byte canary that no kernel may write
(ofdm_radar_workspace_intact).  Every entry point runs on shapes that reach
its edge cases -- ragged tails, full supports, padded grids, grids that are
not powers of two, the largest N -- and no canary may change."""
import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import make_frames, oracle_params, plan_kwargs, stack_lk

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


def frames_for(p, n, seed):
    cfg = syn.FrameConfig(N=p.N, M=p.M, L_cp=p.L_cp, qam=16, zc_root=p.zc_root, n_targets=3, on_grid=False,
                          amp_db=(-6.0, 0.0), snr_db=(0.0, 0.0), window=p.window, detect_k=p.max_targets)
    out = []
    for f in range(n):
        d = syn.draw_frame(cfg, seed + f)
        Xp = o.zc_precode(d.A, p.zc_root) if p.zc_root else d.A
        out.append((d, syn.received(d, Xp)))
    return stack_lk([y for _, y in out]), stack_lk([d.A for d, _ in out])


CHAIN = [
    ("64x16_rect", dict(N=64, M=16, L_cp=8, window=o.WINDOW_RECT), 3),
    ("1024x256_hann", dict(N=1024, M=256, L_cp=128, window=o.WINDOW_HANN), 5),
    ("256x64_full", dict(N=256, M=64, L_cp=256, window=o.WINDOW_HAMMING), 3),
    ("128x32_Npad4", dict(N=128, M=32, L_cp=16, window=o.WINDOW_HANN, N_pad=512), 2),
    ("256x64_Mpad", dict(N=256, M=64, L_cp=32, window=o.WINDOW_HANN, M_pad=256), 2),
    ("256x100_general", dict(N=256, M=100, L_cp=32, window=o.WINDOW_HANN), 3),
    ("64x44_prime", dict(N=64, M=44, L_cp=8, window=o.WINDOW_RECT), 2),
    ("256x64_threshold", dict(N=256, M=64, L_cp=32, window=o.WINDOW_HANN, detect_mode=o.DETECT_THRESHOLD), 2),
    ("256x64_cfar", dict(N=256, M=64, L_cp=32, window=o.WINDOW_HANN, detect_mode=o.DETECT_CFAR, pfa=1e-6), 2),
    ("2048x64", dict(N=2048, M=64, L_cp=256, window=o.WINDOW_HANN), 2),
    ("4096x16", dict(N=4096, M=16, L_cp=512, window=o.WINDOW_HANN), 1),
]


@pytest.mark.parametrize("name,kw,frames", CHAIN, ids=[c[0] for c in CHAIN])
def test_chain_entry_points_keep_canaries(env, name, kw, frames):
    radar, torch, dev = env
    p = o.Params(zc_root=1, max_targets=8, **kw)
    Yh, Ah = frames_for(p, frames, 6100 + len(name))
    plan = radar.Plan(**plan_kwargs(p, frames))
    Y, X = torch.from_numpy(Yh).to(dev), torch.from_numpy(Ah).to(dev)
    out = radar.process(plan, Y, X)                                   # device buffers
    rows = plan.support_rows()
    strip = torch.empty((frames, len(rows), p.M), dtype=torch.complex64, device=dev)
    radar.ofdm_radar_range_profile(plan, Y, X, frames, strip)         # step entry points
    mp = torch.empty_like(out["map"])
    radar.ofdm_radar_doppler(plan, strip, frames, mp)
    radar.ofdm_radar_detect(plan, mp, frames, out["targets"], out["n_targets"], out["status"])
    hm = torch.empty(tuple(out["map"].shape), dtype=torch.float32).pin_memory()  # host path
    radar.ofdm_radar_process_host(plan, torch.from_numpy(Yh).pin_memory(), torch.from_numpy(Ah).pin_memory(),
                                  frames, hm)
    torch.cuda.synchronize()
    assert radar.ofdm_radar_workspace_intact()
    plan.close()


def test_other_entry_points_keep_canaries(env):
    radar, torch, dev = env
    # split-FP16 tensor-core column stage (ragged: 3 frames, M = 16)
    p = o.Params(N=1024, M=16, L_cp=128, zc_root=1, window=o.WINDOW_HANN, max_targets=4)
    Yh, Ah = frames_for(p, 3, 6300)
    tc = radar.Plan(precision=radar.PREC_SPLIT_FP16, **plan_kwargs(p, 3))
    radar.process(tc, torch.from_numpy(Yh).to(dev), torch.from_numpy(Ah).to(dev))
    # ZC precoding both ways, the transmit side
    A = torch.from_numpy(Ah).to(dev)
    Xp, back = torch.empty_like(A), torch.empty_like(A)
    radar.ofdm_zc_precode(tc, A, Xp, 3)
    radar.ofdm_zc_precode(tc, Xp, back, 3, inverse=True)
    papr = torch.empty((3, 16), dtype=torch.float32, device=dev)
    aci = torch.empty_like(papr)
    radar.ofdm_tx_amplifier(tc, Xp, 3, 4, 2.0, papr, aci)
    # FPS-SFT, with ZCP + DFT-CE and in the sampled-cells mode
    for zc, L in ((1, 128), (0, 1024)):
        p = o.Params(N=1024, M=1024, L_cp=L, zc_root=zc, window=o.WINDOW_RECT, max_targets=8)
        Yh, Ah = frames_for(p, 2, 6400 + zc)
        plan = radar.Plan(**plan_kwargs(p, 2))
        fp = radar.fps_default_params()
        rng = np.random.default_rng(6500 + zc)
        sl = np.zeros((2, fp.iterations, 2 + 2 * fp.offsets), dtype=np.int32)
        sl[:, :, 0] = rng.integers(0, 512, sl.shape[:2]) * 2 + 1
        sl[:, :, 1] = rng.integers(0, 512, sl.shape[:2]) * 2 + 1
        sl[:, :, 2::2] = rng.integers(0, 1024, sl[:, :, 2::2].shape)
        sl[:, :, 3::2] = rng.integers(0, 1024, sl[:, :, 3::2].shape)
        out = radar.alloc_outputs(plan, 2, dev, with_map=False)
        radar.ofdm_fps_sft(plan, torch.from_numpy(Yh).to(dev), torch.from_numpy(Ah).to(dev), 2, fp,
                           torch.from_numpy(sl).to(dev), out["targets"], out["n_targets"])
        plan.close()
    # learned proposal with an untrained network (its fallback runs too)
    p = o.Params(N=1024, M=256, L_cp=128, zc_root=1, window=o.WINDOW_HANN, max_targets=8)
    Yh, Ah = frames_for(p, 2, 6600)
    plan = radar.Plan(**plan_kwargs(p, 2))
    radar.ofdm_radar_learned_prepare(plan)
    theta = torch.from_numpy((np.random.default_rng(1).standard_normal(radar.ofdm_cnn_param_count()) * 0.1)
                             .astype(np.float32)).to(dev)
    out = radar.alloc_outputs(plan, 2, dev, with_map=False)
    radar.ofdm_radar_process_learned(plan, theta, torch.from_numpy(Yh).to(dev), torch.from_numpy(Ah).to(dev), 2,
                                     0.0, 8, out["targets"], out["n_targets"], out["status"])
    # batched frames of uneven shape, graph and direct launches
    descs, Ys, As, off = [], [], [], 0
    for i, (N, M, L) in enumerate(((256, 64, 32), (512, 128, 64), (256, 64, 32), (1024, 16, 128))):
        q = o.Params(N=N, M=M, L_cp=L, zc_root=1, window=o.WINDOW_HANN, max_targets=8)
        y, a = frames_for(q, 1, 6700 + i)
        Ys.append(y.ravel())
        As.append(a.ravel())
        descs.append((N, M, L, off, off))
        off += N * M
    Y = torch.from_numpy(np.concatenate(Ys)).to(dev)
    X = torch.from_numpy(np.concatenate(As)).to(dev)
    b = radar.Batch(radar.default_params(max_targets=8, window=o.WINDOW_HANN, zc_root=1), descs)
    mp = torch.empty((off,), dtype=torch.float32, device=dev)
    tg = torch.zeros((4 * 8 * radar.TARGET_BYTES,), dtype=torch.uint8, device=dev)
    nt = torch.zeros((4,), dtype=torch.int32, device=dev)
    st = torch.zeros((4,), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        for _ in range(2):
            b.process(Y, X, mp, tg, nt, st, s)
    b.process(Y, X, mp, tg, nt, st, 0)
    torch.cuda.synchronize()
    assert radar.ofdm_radar_workspace_intact()
    b.close()
    plan.close()
    tc.close()
