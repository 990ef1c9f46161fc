"""Batched frames of uneven shape (one graph replay for many frames)."""
import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import MAP_TOL, check_detections_vs_fp64, rel_l2

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


def mixed_batch(n_frames, seed=4000):
    """Uneven frames: N, M, L_cp = N/8, 1-16 targets, QPSK/16-QAM, SNR in [-15, 5] dB."""
    rng = np.random.default_rng(seed)
    shapes = syn.mixed_batch_shapes(rng, n_frames)
    frames = []
    for f, (N, M, L, K, q) in enumerate(shapes):
        cfg = syn.FrameConfig(N=N, M=M, L_cp=L, qam=q, zc_root=1, n_targets=K, on_grid=False,
                              amp_db=(-20.0, 0.0), snr_db=(-15.0, 5.0), window=1, detect_k=16)
        d = syn.draw_frame(cfg, seed + f)
        Xp = o.zc_precode(d.A, 1)
        frames.append((N, M, L, d, syn.received(d, Xp)))
    return frames


def pack(frames):
    Ys, Xs, descs, yx, mo = [], [], [], 0, 0
    for N, M, L, d, Y in frames:
        Ys.append(syn.to_lk(Y).ravel())
        Xs.append(syn.to_lk(d.A).ravel())
        descs.append((N, M, L, yx, mo))
        yx += N * M
        mo += N * M
    return np.concatenate(Ys), np.concatenate(Xs), descs, mo


def run_batch(env, frames, flags=0, repeats=1, stream=True):
    radar, torch, dev = env
    Yh, Xh, descs, nmap = pack(frames)
    K = 16
    params = radar.default_params(max_targets=K, window=1, zc_root=1)
    b = radar.Batch(params, descs, flags)
    Y, X = torch.from_numpy(Yh).to(dev), torch.from_numpy(Xh).to(dev)
    mp = torch.full((nmap,), -1.0, dtype=torch.float32, device=dev)
    tg = torch.zeros((len(frames) * K * radar.TARGET_BYTES,), dtype=torch.uint8, device=dev)
    nt = torch.zeros((len(frames),), dtype=torch.int32, device=dev)
    st = torch.zeros((len(frames),), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream() if stream else None
    for _ in range(repeats):
        if s is not None:
            with torch.cuda.stream(s):
                b.process(Y, X, mp, tg, nt, st, s)
        else:
            b.process(Y, X, mp, tg, nt, st, 0)
    torch.cuda.synchronize()
    return b, descs, mp.cpu().numpy(), radar.targets_view(tg, len(frames), K), nt.cpu().numpy()


def test_batch_matches_oracle_and_graph_replays(env):
    frames = mixed_batch(24)
    b, descs, mp, tv, nt = run_batch(env, frames, repeats=3)
    assert b.used_graph()
    groups = b.groups()
    assert sum(g[3] for g in groups) == 24 and len(groups) > 1
    for N, M, L, n, variant in groups:   # the tuner's pick among the launch shapes built for N
        assert variant in ((0, 4) if N < 1024 else (0, 4, 2) if N == 1024 else (2, 0)), (N, variant)
    for f in range(24):   # every frame of the batch
        N, M, L, d, Y = frames[f]
        p = o.Params(N=N, M=M, L_cp=L, zc_root=1, window=1, max_targets=16)
        ref = o.process(Y, d.A, p)
        got = mp[descs[f][4]:descs[f][4] + N * M].reshape(N, M)
        assert rel_l2(got, ref["P"]) < MAP_TOL, f"frame {f}"
        n = int(nt[f])
        check_detections_vs_fp64([(int(t["r"]), int(t["s"])) for t in tv[f][:n]], tv[f]["power"][:n],
                                 ref["det"], ref["P"])
        det32 = o.detect(got, o.DETECT_TOPK, 16)
        n = int(nt[f])
        assert [(int(t["r"]), int(t["s"])) for t in tv[f][:n]] == list(zip(det32.r.tolist(), det32.s.tolist()))


def test_batch_direct_launches_equal_graph(env):
    frames = mixed_batch(10, seed=4100)
    _, _, m1, t1, n1 = run_batch(env, frames, repeats=2)
    b2, _, m2, t2, n2 = run_batch(env, frames, flags=1)
    assert not b2.used_graph()
    assert np.array_equal(m1, m2) and np.array_equal(n1, n2)
    for f in range(10):
        assert np.array_equal(t1[f][:n1[f]], t2[f][:n2[f]])


def test_batch_falls_back_without_a_capturable_stream(env):
    frames = mixed_batch(4, seed=4200)
    b, _, m, _, n = run_batch(env, frames, stream=False)
    assert not b.used_graph()
    _, _, m2, _, n2 = run_batch(env, frames)
    assert np.array_equal(m, m2) and np.array_equal(n, n2)


def test_batch_rejects_bad_descriptors(env):
    radar, torch, dev = env
    params = radar.default_params(max_targets=4)
    with pytest.raises(radar.OfdmError):
        radar.Batch(params, [(1000, 64, 8, 0, 0)])
    with pytest.raises(radar.OfdmError):
        radar.Batch(params, [(256, 64, 32, 0, 2)])
