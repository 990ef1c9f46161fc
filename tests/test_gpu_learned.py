"""The learned proposal on the GPU: the CNN's own kernels against the FP64
oracle, the coarse map, exact refinement, the fallback and training."""
import os
import tempfile

import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import make_frames, oracle_params, plan_kwargs, rel_l2, stack_lk

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


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def cnn_gpu(env, theta, x, bf16):
    radar, torch, dev = env
    B, H, W = x.shape
    t = torch.from_numpy(theta.astype(np.float32)).to(dev)
    xd = torch.from_numpy(x.astype(np.float32)).to(dev)
    a1 = torch.empty((B, 16, H, W), device=dev)
    a2 = torch.empty_like(a1)
    z = torch.empty((B, H, W), device=dev)
    radar.ofdm_cnn_forward(t, bf16, xd, B, H, W, a1, a2, z)
    return t, xd, a1, a2, z


def test_cnn_forward_backward_match_oracle(env):
    radar, torch, dev = env
    rng = np.random.default_rng(3)
    theta = 0.3 * rng.standard_normal(o.cnn_n_params())
    x = rng.standard_normal((2, 20, 37))
    y = (rng.random((2, 20, 37)) < 0.1).astype(np.float32)
    t, xd, a1, a2, z = cnn_gpu(env, theta, x, 0)
    zr, saved = o.cnn_forward(x[:, None], theta.astype(np.float32).astype(np.float64))
    assert rel_l2(z.cpu().numpy(), zr[:, 0]) < 1e-5
    loss = torch.zeros((1,), device=dev)
    gz = torch.empty_like(z)
    radar.ofdm_cnn_bce(z, torch.from_numpy(y).to(dev), y.size, 8.0, loss, gz)
    lr_, gr = o.bce_logits(zr, y[:, None], 8.0)
    assert abs(float(loss) - lr_) < 1e-5 * abs(lr_)
    assert rel_l2(gz.cpu().numpy(), gr[:, 0]) < 1e-5
    ga1, ga2, g = torch.empty_like(a1), torch.empty_like(a2), torch.empty_like(t)
    radar.ofdm_cnn_backward(t, 0, xd, a1, a2, gz, 2, 20, 37, ga1, ga2, g)
    torch.cuda.synchronize()
    gref = o.cnn_backward(saved, theta.astype(np.float32).astype(np.float64), gr)
    assert rel_l2(g.cpu().numpy(), gref) < 1e-4


def test_cnn_bf16_inference(env):
    rng = np.random.default_rng(4)
    theta = 0.3 * rng.standard_normal(o.cnn_n_params())
    x = rng.standard_normal((1, 16, 16))
    *_, z = cnn_gpu(env, theta, x, 1)
    # weights in BF16, biases kept in FP32
    th = theta.astype(np.float32).astype(np.float64)
    off = 0
    for name, shp in o.CNN_SHAPES:
        n = int(np.prod(shp))
        if name[0] == "w":
            th[off:off + n] = bf16_round(theta[off:off + n])
        off += n
    zr, _ = o.cnn_forward(x[:, None], th)
    assert rel_l2(z.cpu().numpy(), zr[:, 0]) < 1e-5


def test_coarse_map_matches_oracle(env):
    radar, torch, dev = env
    cfg, fr = make_frames(2, 2)
    p = oracle_params(cfg)
    plan = radar.Plan(**plan_kwargs(p, 2))
    H, W = radar.ofdm_radar_learned_prepare(plan)
    Y = torch.from_numpy(stack_lk([f[2] for f in fr])).to(dev)
    X = torch.from_numpy(stack_lk([f[0].A for f in fr])).to(dev)
    x = torch.empty((2, H, W), device=dev)
    radar.ofdm_radar_coarse_map(plan, Y, X, 2, x)
    torch.cuda.synchronize()
    rows = plan.support_rows()
    for i, (frm, Xp, Yf) in enumerate(fr):
        g = o.process(Yf, frm.A, p)["g"][rows]
        assert np.max(np.abs(x[i].cpu().numpy() - o.coarse_map(g, p.window))) < 2e-5


def _learned(env, p, fr, theta, thr, cap):
    radar, torch, dev = env
    n = len(fr)
    plan = radar.Plan(**plan_kwargs(p, n))
    radar.ofdm_radar_learned_prepare(plan)
    Y = torch.from_numpy(stack_lk([f[2] for f in fr])).to(dev)
    X = torch.from_numpy(stack_lk([f[0].A for f in fr])).to(dev)
    out = radar.alloc_outputs(plan, n, dev, with_map=False)
    radar.ofdm_radar_process_learned(plan, torch.from_numpy(theta.astype(np.float32)).to(dev), Y, X, n, thr, cap,
                                     out["targets"], out["n_targets"], out["status"])
    ref = radar.alloc_outputs(plan, n, dev)
    radar.ofdm_radar_process(plan, Y, X, n, ref["map"], ref["targets"], ref["n_targets"], ref["status"])
    torch.cuda.synchronize()
    return (radar.targets_view(out["targets"], n, p.max_targets), out["n_targets"].cpu().numpy(),
            out["status"].cpu().numpy().view(np.uint32), ref)


def test_learned_refinement_is_exact(env):
    """Candidates from a network that flags every strong coarse cell (the
    identity map on x, threshold on x): every reported target is a local
    maximum of the oracle's periodogram with the oracle's power."""
    radar, torch, dev = env
    cfg, fr = make_frames(2, 2)
    p = oracle_params(cfg, max_targets=5)
    theta = np.zeros(o.cnn_n_params())
    # w1[0] centre = 1, w2[0][0] centre = 1, w3[0][0] centre = 1: logit = relu(relu(x))
    theta[4] = 1.0
    off_w2 = 16 * 9 + 16
    theta[off_w2 + 4] = 1.0
    off_w3 = off_w2 + 16 * 16 * 9 + 16
    theta[off_w3 + 4] = 1.0
    tv, nt, st, ref = _learned(env, p, fr, theta, 3.0, 64)
    for i, (frm, Xp, Y) in enumerate(fr):
        if st[i] & radar.STATUS_FALLBACK:
            continue
        P = o.process(Y, frm.A, p)["P"]
        lm = o.local_maxima(P)
        assert int(nt[i]) >= 1
        for t in tv[i][:int(nt[i])]:
            r, c = int(t["r"]), int(t["s"]) + p.M // 2
            assert lm[r, c]
            assert abs(float(t["power"]) - P[r, c]) < 2e-5 * P[r, c]


def test_learned_fallback_equals_plain(env):
    radar, torch, dev = env
    cfg, fr = make_frames(2, 3)
    p = oracle_params(cfg)
    theta = np.zeros(o.cnn_n_params())
    theta[-1] = 1.0              # b3 = 1: every cell's logit is 1 > 0 -> too many candidates
    tv, nt, st, ref = _learned(env, p, fr, theta, 0.0, 16)
    assert all(s & radar.STATUS_FALLBACK for s in st)
    assert np.array_equal(nt, ref["n_targets"].cpu().numpy())
    rv = radar.targets_view(ref["targets"], 3, p.max_targets)
    for i in range(3):
        assert np.array_equal(tv[i][:nt[i]], rv[i][:nt[i]])


def test_training_lowers_loss_and_checkpoint_roundtrip(env):
    radar, torch, dev = env
    from paper_2209_03883_gb300.learned import Trainer, coarse_labels
    cfg = syn.FrameConfig(N=1024, M=256, L_cp=128, qam=16, zc_root=1, n_targets=8, on_grid=False,
                          amp_db=(-10.0, 0.0), snr_db=(-10.0, 0.0), window=1)
    plan = radar.Plan(N=1024, M=256, L_cp=128, max_frames=8, max_targets=8)
    tr = Trainer(plan, torch, dev, seed=1)
    rows = plan.support_rows()

    def precode(A):
        out = torch.empty_like(A)
        radar.ofdm_zc_precode(plan, A, out, A.shape[0])
        return out

    losses = []
    for step in range(60):
        Y, A, truth = syn.draw_frames_torch(cfg, [90000 + 8 * step + i for i in range(8)], dev, precode)
        lab = coarse_labels(truth, 1024, 256, len(rows), rows[0], tr.Hc, tr.Mc)
        losses.append(float(tr.train_step(Y, A, lab)))
    assert np.mean(losses[-10:]) < 0.7 * np.mean(losses[:5])
    z1 = tr.logits(Y, A).clone()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "cnn.bin")
        tr.save(path)
        tr2 = Trainer(plan, torch, dev, seed=7)
        tr2.load(path)
        assert tr2.step == tr.step
        assert torch.equal(tr2.logits(Y, A), z1)


def test_checkpoint_resume_continues_the_loss_trajectory(env):
    """Resuming from a checkpoint (parameters, Adam moments and step count)
    continues training as if it had never stopped: a run interrupted after
    8 of 16 steps, reloaded into a trainer with other initial weights,
    reproduces the uninterrupted run's losses on the remaining steps and ends
    on the same parameters (up to the summation order of the gradient
    atomics)."""
    radar, torch, dev = env
    from paper_2209_03883_gb300.learned import Trainer, coarse_labels
    cfg = syn.FrameConfig(N=1024, M=256, L_cp=128, qam=16, zc_root=1, n_targets=8, on_grid=False,
                          amp_db=(-10.0, 0.0), snr_db=(-10.0, 0.0), window=1)
    plan = radar.Plan(N=1024, M=256, L_cp=128, max_frames=4, max_targets=8)
    rows = plan.support_rows()

    def precode(A):
        out = torch.empty_like(A)
        radar.ofdm_zc_precode(plan, A, out, A.shape[0])
        return out

    full = Trainer(plan, torch, dev, seed=3)
    batches = []
    for step in range(16):
        Y, A, truth = syn.draw_frames_torch(cfg, [95000 + 4 * step + i for i in range(4)], dev, precode)
        batches.append((Y, A, coarse_labels(truth, 1024, 256, len(rows), rows[0], full.Hc, full.Mc)))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "cnn.bin")
        loss_full = []
        for step, (Y, A, lab) in enumerate(batches):
            loss_full.append(float(full.train_step(Y, A, lab)))
            if step == 7:
                full.save(path)
        resumed = Trainer(plan, torch, dev, seed=11)
        assert not torch.equal(resumed.theta, full.theta)
        resumed.load(path)
        assert resumed.step == 8
        loss_resumed = [float(resumed.train_step(Y, A, lab)) for Y, A, lab in batches[8:]]
    assert resumed.step == full.step == 16
    np.testing.assert_allclose(loss_resumed, loss_full[8:], rtol=1e-3)
    rel = float(torch.linalg.vector_norm(resumed.theta - full.theta) / torch.linalg.vector_norm(full.theta))
    assert rel < 1e-3, rel


def test_trained_network_gain_over_the_plain_chain(env, capsys):
    """What the trained network gains over the chain without it, on held-out
    frames of the learned workload's shape (4096 x 1024, L_cp 512, 32 off-grid
    targets, SNR U[-15, 5] dB): frames/s of both forms and targets found
    within one bin.  The learned form replaces only the Doppler stage and the
    detection; the column stage (ZC transform, division, DFT-CE) is shared and
    is most of the plain form's time, which bounds the possible gain.  The test
    states the measured gain and that bound, and requires equal detection
    accuracy up to 1 % of the targets."""
    radar, torch, dev = env
    from paper_2209_03883_gb300.learned import Trainer, coarse_labels
    cfg = syn.CONFIGS[5]
    N, M, L, B = cfg.N, cfg.M, cfg.L_cp, 4
    tplan = radar.Plan(N=N, M=M, L_cp=L, max_frames=B, max_targets=cfg.detect_k)
    tr = Trainer(tplan, torch, dev, seed=5)
    rows = tplan.support_rows()

    def precode_with(plan):
        def f(A):
            out = torch.empty_like(A)
            radar.ofdm_zc_precode(plan, A, out, A.shape[0])
            return out
        return f

    for step in range(120):
        Y, A, truth = syn.draw_frames_torch(cfg, [5 * 1000 + 300 + B * step + i for i in range(B)], dev,
                                            precode_with(tplan))
        tr.train_step(Y, A, coarse_labels(truth, N, M, len(rows), rows[0], tr.Hc, tr.Mc))
    Yv, Av, _ = syn.draw_frames_torch(cfg, [5 * 1000 + 60 + i for i in range(B)], dev, precode_with(tplan))
    thr = float(torch.topk(tr.logits(Yv, Av).reshape(B, -1), 64, dim=1).values[:, -1].mean())
    n_eval = 8
    plan = radar.Plan(N=N, M=M, L_cp=L, max_frames=n_eval, max_targets=cfg.detect_k)
    radar.ofdm_radar_learned_prepare(plan)
    Y, A, truth = syn.draw_frames_torch(cfg, [5 * 1000 + 700 + f for f in range(n_eval)], dev, precode_with(plan))
    po = radar.alloc_outputs(plan, n_eval, dev, with_map=False)
    lo = radar.alloc_outputs(plan, n_eval, dev, with_map=False)
    plain = lambda: radar.ofdm_radar_process(plan, Y, A, n_eval, None, po["targets"], po["n_targets"], po["status"])
    learned = lambda: radar.ofdm_radar_process_learned(plan, tr.theta, Y, A, n_eval, thr, 256, lo["targets"],
                                                       lo["n_targets"], lo["status"])

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_plain, ms_learned = timed(plain), timed(learned)
    plan.timing_enable(True)
    plain()
    torch.cuda.synchronize()
    st = plan.timing_read()
    plan.timing_enable(False)
    col = st["column"][0]
    tail = sum(v[0] for k, v in st.items() if k != "column")
    bound = (col + tail) / col          # the learned stages for free

    def hits(o):
        tv = radar.targets_view(o["targets"], n_eval, cfg.detect_k)
        nt = o["n_targets"].cpu().numpy()
        h = 0
        for f, (rho, nu, _b, _snr) in enumerate(truth):
            got = [(int(t["r"]), int(t["s"])) for t in tv[f][:int(nt[f])]]
            for a_, b_ in zip(rho, nu):
                h += any(abs(r - a_) <= 1.0 and abs(((s - b_) + M // 2) % M - M // 2) <= 1.0 for r, s in got)
        return h

    hp, hl = hits(po), hits(lo)
    total = cfg.n_targets * n_eval
    gain = ms_plain / ms_learned
    with capsys.disabled():
        print(f"\nlearned vs plain on {n_eval} frames {N}x{M}: gain {gain:.3f}x "
              f"(plain {ms_plain:.3f} ms, learned {ms_learned:.3f} ms; bound if the learned stages were free "
              f"{bound:.3f}x), targets found {hl}/{total} learned vs {hp}/{total} plain")
    assert gain <= bound * 1.05
    assert hl >= hp - 0.01 * total
