"""GPU parity of the CUDA chain against the FP64 oracle, through the C ABI.

Every step is compared element by element on seeded frames: the ZC
transform, the range-profile strip (steps a1-a5), the full periodogram
(a6) and the detections (a7), on the five workloads' shapes (the largest
on sampled outputs) and on the edge cases of the method.
"""
import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import (MAP_TOL, check_detections_vs_fp64, make_frames, oracle_params,
                               plan_kwargs, rel_l2, stack_lk)

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


def to_dev(torch, dev, arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).to(dev)


def run_chain(env, p, Ys, As, with_map=True, plan=None):
    radar, torch, dev = env
    frames = len(Ys)
    plan = plan or radar.Plan(**plan_kwargs(p, frames))
    Y = to_dev(torch, dev, stack_lk(Ys))
    X = to_dev(torch, dev, stack_lk(As))
    out = radar.process(plan, Y, X, with_map=with_map)
    torch.cuda.synchronize()
    res = dict(plan=plan,
               map=out["map"].cpu().numpy() if with_map else None,
               tg=radar.targets_view(out["targets"], frames, p.max_targets),
               n=out["n_targets"].cpu().numpy(), status=out["status"].cpu().numpy().view(np.uint32),
               launches=plan.last_launch_count())
    return res


def gpu_strip(env, p, Ys, As):
    radar, torch, dev = env
    frames = len(Ys)
    plan = radar.Plan(**plan_kwargs(p, frames))
    rows = plan.support_rows()
    Y = to_dev(torch, dev, stack_lk(Ys))
    X = to_dev(torch, dev, stack_lk(As))
    strip = torch.empty((frames, len(rows), p.M), dtype=torch.complex64, device=dev)
    radar.ofdm_radar_range_profile(plan, Y, X, frames, strip)
    torch.cuda.synchronize()
    return rows, strip.cpu().numpy()


def oracle_strip(p, Y, A):
    ref = o.process(Y, A, p)
    return ref["g"], ref


# ------------------------------------------------------------------ ZC transform
@pytest.mark.parametrize("N,M,r,q", [(1024, 256, 1, 0), (256, 16, 3, 2), (64, 16, 5, 1),
                                     (4096, 16, 1, 0), (2048, 16, 7, 3)])
def test_zc_precode_forward_inverse(env, N, M, r, q):
    radar, torch, dev = env
    rng = np.random.default_rng(N + r)
    A = syn.as_complex64_values(syn.qam_symbols(rng, (N, M), 16))
    p = o.Params(N=N, M=M, L_cp=N // 8, zc_root=r, zc_q=q)
    plan = radar.Plan(**plan_kwargs(p, 1))
    Ad = to_dev(torch, dev, syn.to_lk(A)[None])
    Xd = torch.empty_like(Ad)
    Bd = torch.empty_like(Ad)
    radar.ofdm_zc_precode(plan, Ad, Xd, 1, inverse=False)
    radar.ofdm_zc_precode(plan, Xd, Bd, 1, inverse=True)
    torch.cuda.synchronize()
    want = o.zc_precode(A, r, q)
    got = Xd[0].cpu().numpy().T
    assert rel_l2(got, want) < MAP_TOL
    back = Bd[0].cpu().numpy().T
    assert rel_l2(back, o.zc_precode(got.astype(np.complex128), r, q, inverse=True)) < MAP_TOL
    assert rel_l2(back, A) < 2 * MAP_TOL


# ------------------------------------------------------------------ range profile (a1-a5)
@pytest.mark.parametrize("ci,frames", [(1, 1), (2, 2), (3, 1)])
def test_range_profile_matches_oracle(env, ci, frames):
    cfg, fr = make_frames(ci, frames)
    p = oracle_params(cfg)
    rows, strip = gpu_strip(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    for i, (frm, Xp, Y) in enumerate(fr):
        g, _ = oracle_strip(p, Y, frm.A)
        assert rel_l2(strip[i], g[rows, :]) < MAP_TOL
        others = np.setdiff1d(np.arange(cfg.N), rows)
        assert np.max(np.abs(g[others])) < 1e-9 * np.max(np.abs(g)), "oracle support mismatch"


# ------------------------------------------------------------------ full chain (a1-a7)
@pytest.mark.parametrize("ci,frames", [(1, 1), (2, 3), (3, 2)])
def test_chain_matches_oracle(env, ci, frames):
    cfg, fr = make_frames(ci, frames)
    p = oracle_params(cfg)
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    assert res["launches"] >= 2   # column + fused Doppler/detection (M' >= 64), else three kernels
    for i, (frm, Xp, Y) in enumerate(fr):
        ref = o.process(Y, frm.A, p)
        assert rel_l2(res["map"][i], ref["P"]) < MAP_TOL
        n = int(res["n"][i])
        rs = [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]]
        check_detections_vs_fp64(rs, res["tg"][i]["power"][:n], ref["det"], ref["P"])
        # the detection step itself is exact on the GPU's own map (same FP32 decisions)
        det32 = o.detect(res["map"][i], p.detect_mode, p.max_targets)
        assert rs == list(zip(det32.r.tolist(), det32.s.tolist()))
        assert np.array_equal(res["tg"][i]["power"][:n], det32.power.astype(np.float32))
        assert int(res["status"][i]) == det32.status


def test_chain_full_batch_every_frame(env):
    """The benchmark's launch: 64 frames of 1024 x 256 in one call, every
    frame checked in full against the oracle (map and detections)."""
    cfg, fr = make_frames(2, 64)
    p = oracle_params(cfg)
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    for i, (frm, Xp, Y) in enumerate(fr):
        ref = o.process(Y, frm.A, p)
        assert rel_l2(res["map"][i], ref["P"]) < MAP_TOL, f"frame {i}"
        n = int(res["n"][i])
        rs = [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]]
        check_detections_vs_fp64(rs, res["tg"][i]["power"][:n], ref["det"], ref["P"])
    # every frame finds its targets (one-bin tolerance for off-grid truth)
    hits = 0
    for i, (frm, _, _) in enumerate(fr):
        n = int(res["n"][i])
        got = [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]]
        for rho, nu in zip(frm.rho, frm.nu):
            hits += any(abs(r - rho) <= 1.0 and abs(((s - nu) + 128) % 256 - 128) <= 1.0 for r, s in got)
    assert hits >= 0.8 * 5 * 64


@pytest.mark.slow
def test_largest_workload_full_frame(env):
    """One whole 4096 x 1024 frame (L_cp = 512, 32 off-grid targets) through
    the chain: map and detections against the oracle."""
    cfg, fr = make_frames(5, 1)
    p = oracle_params(cfg)
    frm, Xp, Y = fr[0]
    res = run_chain(env, p, [Y], [frm.A])
    ref = o.process(Y, frm.A, p)
    assert rel_l2(res["map"][0], ref["P"]) < MAP_TOL
    n = int(res["n"][0])
    rs = [(int(t["r"]), int(t["s"])) for t in res["tg"][0][:n]]
    check_detections_vs_fp64(rs, res["tg"][0]["power"][:n], ref["det"], ref["P"])


def test_largest_workload_sampled(env):
    """4096 x 1024 with L_cp = 512: the strip is checked on sampled symbols
    against the oracle computed column by column."""
    radar, torch, dev = env
    cfg = syn.CONFIGS[5]
    fr = syn.draw_frame(cfg, syn.seed_for(5, 0))
    Xp = o.zc_precode(fr.A, 1)
    Y = syn.received(fr, Xp)
    p = oracle_params(cfg)
    rows, strip = gpu_strip(env, p, [Y], [fr.A])
    cols = [0, 1, 511, 1023]
    F, _ = o.ls_divide(Y[:, cols], Xp[:, cols])
    Hd, _ = o.dft_ce(F, p.L_cp)
    g = o.range_profile(Hd, o.window(p.N, p.window))
    assert rel_l2(strip[0][:, cols], g[rows, :]) < MAP_TOL


# ------------------------------------------------------------------ variants and edge cases
VARIANTS = [
    ("lcp_eq_N_rect", dict(N=64, M=16, L_cp=64, window=o.WINDOW_RECT)),
    ("lcp_eq_N_hann", dict(N=128, M=32, L_cp=128, window=o.WINDOW_HANN)),
    ("lcp_N_minus_1_hann", dict(N=64, M=64, L_cp=63, window=o.WINDOW_HANN)),
    ("hamming", dict(N=256, M=64, L_cp=32, window=o.WINDOW_HAMMING)),
    ("no_zcp", dict(N=512, M=128, L_cp=64, zc_root=0)),
    ("zc_root3_q2", dict(N=256, M=32, L_cp=32, zc_root=3, zc_q=2)),
    ("doppler_pad", dict(N=256, M=64, L_cp=32, M_pad=128)),
    ("n2048", dict(N=2048, M=64, L_cp=256)),
    ("n4096_m16", dict(N=4096, M=16, L_cp=512, window=o.WINDOW_RECT)),
    ("m32_direct", dict(N=128, M=32, L_cp=16)),
    ("lcp_1", dict(N=64, M=16, L_cp=1, window=o.WINDOW_HANN)),
    # N = 1024: the last DFT-CE half-pass is output-pruned for L_cp <= 128 only
    ("n1024_lcp200", dict(N=1024, M=32, L_cp=200)),
    ("n1024_lcp5_hamming", dict(N=1024, M=32, L_cp=5, window=o.WINDOW_HAMMING)),
    # full support: 1024 rows x 256 bins = 64 detection bands (two-level merge)
    ("n1024_full_rect", dict(N=1024, M=256, L_cp=1024, window=o.WINDOW_RECT)),
    ("m512", dict(N=256, M=512, L_cp=32)),
]


@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_variants(env, name, kw):
    base = syn.FrameConfig(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], qam=16,
                           zc_root=kw.get("zc_root", 1), n_targets=3, on_grid=False,
                           amp_db=(-6.0, 0.0), snr_db=(0.0, 0.0), window=kw.get("window", 1),
                           detect_k=4)
    if kw["L_cp"] < 8:
        base.n_targets = 0
    frames = 2
    fr = []
    for f in range(frames):
        d = syn.draw_frame(base, 7000 + f, n_targets=base.n_targets)
        Xp = o.zc_precode(d.A, base.zc_root, kw.get("zc_q", 0)) if base.zc_root else d.A
        fr.append((d, Xp, syn.received(d, Xp)))
    p = o.Params(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], zc_root=base.zc_root, zc_q=kw.get("zc_q", 0),
                 window=base.window, max_targets=4, M_pad=kw.get("M_pad", 0))
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    for i, (d, Xp, Y) in enumerate(fr):
        ref = o.process(Y, d.A, p)
        assert rel_l2(res["map"][i], ref["P"]) < MAP_TOL, name
        det32 = o.detect(res["map"][i], p.detect_mode, p.max_targets)
        n = int(res["n"][i])
        assert [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]] == \
            list(zip(det32.r.tolist(), det32.s.tolist()))


def test_x_is_precoded_equals_internal_precoding(env):
    cfg, fr = make_frames(1, 1)
    frm, Xp, Y = fr[0]
    p = oracle_params(cfg)
    a = run_chain(env, p, [Y], [frm.A])
    p2 = oracle_params(cfg, x_is_precoded=True)
    b = run_chain(env, p2, [Y], [Xp])
    assert rel_l2(b["map"][0], a["map"][0]) < MAP_TOL


def test_threshold_mode(env):
    cfg, fr = make_frames(2, 2)
    for noise_var in (-1.0, 40.0):
        p = oracle_params(cfg, detect_mode=o.DETECT_THRESHOLD, max_targets=16, noise_var=noise_var)
        res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
        rows = o.support_rows(p.N, p.L_cp, p.window)
        for i in range(2):
            P32 = res["map"][i]
            # the library takes P_fa as float32; the oracle gets the same value
            eta = o.threshold(P32, rows, float(np.float32(p.pfa)), p.noise_var)
            det32 = o.detect(P32, o.DETECT_THRESHOLD, p.max_targets, eta)
            n = int(res["n"][i])
            assert [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]] == \
                list(zip(det32.r.tolist(), det32.s.tolist()))
            assert int(res["status"][i]) == det32.status


def test_zero_and_nonfinite_cells_flagged(env):
    cfg, fr = make_frames(1, 2)
    p = oracle_params(cfg, zc_root=0)
    A0 = fr[0][0].A.copy()
    A0[5, 3] = 0.0                       # a zero transmit cell
    Y1 = fr[1][2].copy()
    Y1[7, 2] = np.nan                    # a non-finite received cell
    res = run_chain(env, p, [fr[0][2], Y1], [A0, fr[1][0].A])
    assert res["status"][0] & o.STATUS_ZERO_X
    assert not res["status"][0] & o.STATUS_NONFINITE
    assert res["status"][1] & o.STATUS_NONFINITE
    ref = o.process(fr[0][2], A0, p)     # F = 0 at the zero cell on both sides
    assert rel_l2(res["map"][0], ref["P"]) < MAP_TOL
    # status words do not leak into the next call on the same plan
    res2 = run_chain(env, p, [fr[0][2], fr[1][2]], [fr[0][0].A, fr[1][0].A], plan=res["plan"])
    assert (res2["status"] & (o.STATUS_ZERO_X | o.STATUS_NONFINITE) == 0).all()


def test_noiseless_point_target_lands_on_its_bin(env):
    N, M = 1024, 256
    rng = np.random.default_rng(11)
    A = syn.as_complex64_values(syn.qam_symbols(rng, (N, M), 16))
    Xp = o.zc_precode(A, 1)
    H = syn.channel([37.0], [-21.0], [1.0], N, M)
    p = o.Params(N=N, M=M, L_cp=128, window=o.WINDOW_HANN, max_targets=1)
    res = run_chain(env, p, [Xp * H], [A])
    t = res["tg"][0][0]
    assert (int(t["r"]), int(t["s"])) == (37, -21)
    assert abs(t["power"] - N * M / 16) < 1e-4 * N * M / 16
    Ts = o.symbol_time(N, 128, 240e3)
    dd, dv = o.resolution(N, M, 240e3, 77e9, Ts)
    assert t["range_m"] == pytest.approx(37 * dd, rel=1e-5)
    assert t["vel_mps"] == pytest.approx(-21 * dv, rel=1e-5)


def test_detect_entry_point_on_given_map(env):
    radar, torch, dev = env
    cfg, fr = make_frames(1, 1)
    p = oracle_params(cfg)
    ref = o.process(fr[0][2], fr[0][0].A, p)
    P32 = ref["P"].astype(np.float32)
    plan = radar.Plan(**plan_kwargs(p, 1))
    out = radar.alloc_outputs(plan, 1, dev, with_map=False)
    radar.ofdm_radar_detect(plan, to_dev(torch, dev, P32[None]), 1, out["targets"], out["n_targets"],
                            out["status"])
    torch.cuda.synchronize()
    det32 = o.detect(P32, p.detect_mode, p.max_targets)
    tg = radar.targets_view(out["targets"], 1, p.max_targets)[0]
    n = int(out["n_targets"][0])
    assert [(int(t["r"]), int(t["s"])) for t in tg[:n]] == list(zip(det32.r.tolist(), det32.s.tolist()))


@pytest.mark.parametrize("N,M,L,window", [(256, 100, 32, o.WINDOW_HANN), (64, 20, 64, o.WINDOW_RECT),
                                         (128, 44, 16, o.WINDOW_HAMMING)])
def test_detect_entry_point_general_grid(env, N, M, L, window):
    """ofdm_radar_detect on a given full map of a Doppler grid that is not a
    power of two (band detection on map rows, circular halo rows when the
    support is every row): top-K and threshold mode (median-estimated noise)
    exactly as the oracle's rule on the same float32 map."""
    radar, torch, dev = env
    base = syn.FrameConfig(N=N, M=M, L_cp=L, qam=16, zc_root=1, n_targets=3, on_grid=False, amp_db=(-6.0, 0.0),
                           snr_db=(0.0, 0.0), window=window, detect_k=8)
    d = syn.draw_frame(base, 8800 + N + M)
    Xp = o.zc_precode(d.A, 1)
    Y = syn.received(d, Xp)
    for mode in (o.DETECT_TOPK, o.DETECT_THRESHOLD):
        p = o.Params(N=N, M=M, L_cp=L, zc_root=1, window=window, max_targets=8, detect_mode=mode)
        P32 = o.process(Y, d.A, p)["P"].astype(np.float32)
        plan = radar.Plan(**plan_kwargs(p, 1))
        out = radar.alloc_outputs(plan, 1, dev, with_map=False)
        radar.ofdm_radar_detect(plan, to_dev(torch, dev, P32[None]), 1, out["targets"], out["n_targets"],
                                out["status"])
        torch.cuda.synchronize()
        rows = o.support_rows(N, L, window)
        eta = o.threshold(P32, rows, float(np.float32(p.pfa)), p.noise_var) if mode == o.DETECT_THRESHOLD else None
        det32 = o.detect(P32, mode, p.max_targets, eta)
        tg = radar.targets_view(out["targets"], 1, p.max_targets)[0]
        n = int(out["n_targets"][0])
        assert [(int(t["r"]), int(t["s"])) for t in tg[:n]] == list(zip(det32.r.tolist(), det32.s.tolist()))
        assert np.array_equal(tg["power"][:n], det32.power.astype(np.float32))
        assert int(out["status"][0]) == det32.status
        plan.close()


def test_misaligned_buffers_rejected(env):
    """Grids, maps and strips move in 16-byte pieces: a buffer that starts
    8 bytes off a 16-byte boundary is rejected before any launch, at every
    entry point that takes one (and the call after it still works)."""
    radar, torch, dev = env
    cfg, fr = make_frames(1, 1)
    p = oracle_params(cfg)
    plan = radar.Plan(**plan_kwargs(p, 1))
    n = cfg.N * cfg.M
    G = torch.zeros((2 * n + 2,), dtype=torch.complex64, device=dev)
    good, bad = G[:n], G[n + 1:2 * n + 1]                         # bad starts 8 bytes past a boundary
    mp = torch.zeros((plan.Np * plan.Mp + 4,), dtype=torch.float32, device=dev)
    out = radar.alloc_outputs(plan, 1, dev, with_map=False)
    calls = [
        lambda: radar.ofdm_radar_process(plan, bad, good, 1),
        lambda: radar.ofdm_radar_process(plan, good, bad, 1),
        lambda: radar.ofdm_radar_process(plan, good, good, 1, mp[2:2 + plan.Np * plan.Mp], out["targets"],
                                         out["n_targets"], out["status"]),
        lambda: radar.ofdm_radar_detect(plan, mp[2:2 + plan.Np * plan.Mp], 1, out["targets"], out["n_targets"],
                                        out["status"]),
        lambda: radar.ofdm_zc_precode(plan, bad, good, 1),
    ]
    for call in calls:
        with pytest.raises(radar.OfdmError) as ei:
            call()
        assert ei.value.code == -1
    Y, X = to_dev(torch, dev, stack_lk([fr[0][2]])), to_dev(torch, dev, stack_lk([fr[0][0].A]))
    radar.ofdm_radar_process(plan, Y, X, 1, None, out["targets"], out["n_targets"], out["status"])
    torch.cuda.synchronize()
    assert int(out["n_targets"][0]) > 0
    plan.close()


@pytest.mark.parametrize("config,frames", [(2, 8), (1, 37)])
def test_host_buffer_path_matches_device_path(env, config, frames):
    """Host buffers through the chunked three-stream pipeline equal the device
    path bit for bit; 37 frames give 13 chunks of 3 and a last chunk of 1."""
    radar, torch, dev = env
    cfg, fr = make_frames(config, frames)
    p = oracle_params(cfg)
    dres = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    plan = radar.Plan(**plan_kwargs(p, frames))
    Yh = torch.from_numpy(stack_lk([f[2] for f in fr])).pin_memory()
    Xh = torch.from_numpy(stack_lk([f[0].A for f in fr])).pin_memory()
    mh = torch.empty((frames, p.N, p.M), dtype=torch.float32).pin_memory()
    th = torch.zeros((frames * p.max_targets * radar.TARGET_BYTES,), dtype=torch.uint8).pin_memory()
    nh = torch.zeros((frames,), dtype=torch.int32).pin_memory()
    sh = torch.zeros((frames,), dtype=torch.int32).pin_memory()
    radar.ofdm_radar_process_host(plan, Yh, Xh, frames, mh, th, nh, sh)
    assert np.array_equal(mh.numpy(), dres["map"])
    assert np.array_equal(nh.numpy(), dres["n"])
    assert np.array_equal(sh.numpy().view(np.uint32), dres["status"])
    tv = radar.targets_view(th, frames, p.max_targets)
    for i in range(frames):
        n = int(nh[i])
        assert np.array_equal(tv[i][:n], dres["tg"][i][:n])


def test_frames_out_of_range_rejected(env):
    radar, torch, dev = env
    p = o.Params(N=64, M=16, L_cp=8)
    plan = radar.Plan(**plan_kwargs(p, 2))
    Y = torch.zeros((3, 16, 64), dtype=torch.complex64, device=dev)
    with pytest.raises(radar.OfdmError):
        radar.process(plan, Y, Y, frames=3)


def test_repeated_calls_on_one_plan(env):
    """Calls of different sizes on one plan (dynamically scheduled column
    kernel, ticket counter carried across calls) match a fresh plan each."""
    radar, torch, dev = env
    cfg, fr = make_frames(2, 8)
    p = oracle_params(cfg)
    plan = radar.Plan(**plan_kwargs(p, 8))
    for n in (8, 3, 5, 8):
        Ys, As = [f[2] for f in fr[:n]], [f[0].A for f in fr[:n]]
        a = run_chain(env, p, Ys, As, plan=plan)
        b = run_chain(env, p, Ys, As)
        assert np.array_equal(a["map"][:n], b["map"][:n])
        assert np.array_equal(a["n"][:n], b["n"][:n])


def test_detection_statistics_against_truth(env):
    """Miss rate and range / velocity RMSE of the GPU chain's estimates (Eq.
    (19)) against the generator's ground truth over 32 frames of 1024 x 256
    at -10 dB (off-grid targets: bin quantisation alone gives 1/sqrt(12) bin)."""
    cfg, fr = make_frames(2, 32)
    p = oracle_params(cfg)
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    Ts = o.symbol_time(cfg.N, cfg.L_cp, 240e3)
    dd, dv = o.resolution(cfg.N, cfg.M, 240e3, 77e9, Ts)
    errs_d, errs_v, n_true, hits = [], [], 0, 0
    for i, (frm, _, _) in enumerate(fr):
        tg = res["tg"][i][:int(res["n"][i])]
        for rho, nu in zip(frm.rho, frm.nu):
            n_true += 1
            best = None
            for t in tg:
                dr = t["r"] - rho
                ds = ((t["s"] - nu) + cfg.M / 2) % cfg.M - cfg.M / 2
                if abs(dr) <= 1.0 and abs(ds) <= 1.0 and (best is None or dr * dr + ds * ds < best[0]):
                    best = (dr * dr + ds * ds, t)
            if best:
                hits += 1
                t = best[1]
                errs_d.append(float(t["range_m"]) - rho * dd)
                errs_v.append(float(t["vel_mps"]) - nu * dv)
    assert hits >= 0.85 * n_true
    assert np.sqrt(np.mean(np.square(errs_d))) < 0.45 * dd
    assert np.sqrt(np.mean(np.square(errs_v))) < 0.45 * dv


# ------------------------------------------------------------------ range zero padding N' > N (Eq. (17))
PAD_CASES = [
    ("64_to_128_rect", dict(N=64, M=16, L_cp=8, N_pad=128, window=o.WINDOW_RECT)),
    ("128_to_512_hann", dict(N=128, M=32, L_cp=16, N_pad=512, window=o.WINDOW_HANN)),
    ("256_to_512_hamming_doppler_pad", dict(N=256, M=64, L_cp=32, N_pad=512, M_pad=128, window=o.WINDOW_HAMMING)),
    ("1024_to_2048_hann", dict(N=1024, M=64, L_cp=128, N_pad=2048, window=o.WINDOW_HANN)),
    ("512_to_4096_hann", dict(N=512, M=16, L_cp=64, N_pad=4096, window=o.WINDOW_HANN)),
]


@pytest.mark.parametrize("name,kw", PAD_CASES, ids=[c[0] for c in PAD_CASES])
def test_range_zero_padding(env, name, kw):
    """A padded range grid interpolates between bins, so every one of the N'
    rows carries signal: the strip (all N' rows), the map and the detections
    against the oracle's Eq. (17) with N' > N."""
    radar, torch, dev = env
    base = syn.FrameConfig(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], qam=16, zc_root=1, n_targets=3, on_grid=False,
                           amp_db=(-6.0, 0.0), snr_db=(0.0, 0.0), window=kw["window"], detect_k=4)
    fr = []
    for f in range(2):
        d = syn.draw_frame(base, 8100 + f)
        Xp = o.zc_precode(d.A, 1)
        fr.append((d, Xp, syn.received(d, Xp)))
    p = o.Params(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], zc_root=1, window=kw["window"], max_targets=4,
                 N_pad=kw["N_pad"], M_pad=kw.get("M_pad", 0))
    rows, strip = gpu_strip(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    assert rows == list(range(kw["N_pad"]))
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    for i, (frm, Xp, Y) in enumerate(fr):
        ref = o.process(Y, frm.A, p)
        g = o.range_profile(ref["Hd"], o.window(p.N, p.window), p.N_pad)
        assert rel_l2(strip[i], g) < MAP_TOL
        assert rel_l2(res["map"][i], ref["P"]) < MAP_TOL
        n = int(res["n"][i])
        rs = [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]]
        check_detections_vs_fp64(rs, res["tg"][i]["power"][:n], ref["det"], ref["P"])


# ------------------------------------------------------------------ CFAR detection (reading F, local noise level)
def _cfar_ratio(P, rows, r, c, guard, train, pfa):
    """P / (alpha(n) mean of the training cells) of one cell, in FP64."""
    R, C = P.shape
    on = np.zeros(R, dtype=bool)
    on[rows] = True
    w = guard + train
    tr = [P[(r + dr) % R, (c + dc) % C] for dr in range(-w, w + 1) for dc in range(-w, w + 1)
          if on[(r + dr) % R] and not (abs(dr) <= guard and abs(dc) <= guard)]
    return float(P[r, c]) / (o.cfar_alpha(len(tr), pfa) * float(np.mean(tr)))


@pytest.mark.parametrize("N,M,L,window,full", [(1024, 256, 128, o.WINDOW_HANN, False),
                                               (256, 64, 256, o.WINDOW_RECT, True),
                                               (512, 100, 64, o.WINDOW_HANN, False),    # M' = 100: general grid
                                               (128, 60, 128, o.WINDOW_RECT, True)])
def test_cfar_detection(env, N, M, L, window, full):
    """CFAR mode: the map against the FP64 oracle, and the detections exactly
    those of the oracle's CFAR rule applied to the GPU's own map, except cells
    whose statistic lies within 1e-4 of the threshold (FP32 training sums)."""
    base = syn.FrameConfig(N=N, M=M, L_cp=L, qam=16, zc_root=1, n_targets=4, on_grid=False, amp_db=(-10.0, 0.0),
                           snr_db=(-5.0, -5.0), window=window, detect_k=16)
    fr = []
    for f in range(2):
        d = syn.draw_frame(base, 8500 + f)
        Xp = o.zc_precode(d.A, 1)
        fr.append((d, Xp, syn.received(d, Xp)))
    p = o.Params(N=N, M=M, L_cp=L, zc_root=1, window=window, max_targets=32, detect_mode=o.DETECT_CFAR, pfa=1e-6,
                 cfar_guard=1, cfar_train=3)
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    rows = o.support_rows(N, L, window)
    assert (len(rows) == N) == full
    for i, (frm, Xp, Y) in enumerate(fr):
        ref = o.process(Y, frm.A, p)
        assert rel_l2(res["map"][i], ref["P"]) < MAP_TOL
        P32 = res["map"][i].astype(np.float64)
        want = o.cfar_detect(P32, rows, p.pfa, p.cfar_guard, p.cfar_train, p.max_targets)
        n = int(res["n"][i])
        assert want.count <= p.max_targets   # every detection is reported
        got = {(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]}
        exp = set(zip(want.r.tolist(), want.s.tolist()))
        for (r, s) in got ^ exp:
            ratio = _cfar_ratio(P32, rows, r, s + M // 2, p.cfar_guard, p.cfar_train, p.pfa)
            assert abs(ratio - 1.0) < 1e-4, f"({r}, {s}) decided differently, statistic {ratio}"
        # the strong targets are found (one-bin tolerance for off-grid truth)
        for rho, nu, b in zip(frm.rho, frm.nu, frm.b):
            if abs(b) ** 2 > 0.3:
                assert any(abs(r - rho) <= 1.0 and abs(((s - nu) + M // 2) % M - M // 2) <= 1.0 for r, s in got)


# ------------------------------------------------------------------ Doppler grids that are not powers of two
GENERAL_M = [
    ("table1_2048x560_hamming", dict(N=2048, M=560, L_cp=512, window=o.WINDOW_HAMMING, targets=5, frames=1)),
    ("64x20_rect", dict(N=64, M=20, L_cp=8, window=o.WINDOW_RECT, targets=2, frames=2)),
    ("256x100_hann", dict(N=256, M=100, L_cp=32, window=o.WINDOW_HANN, targets=3, frames=2)),
    ("128x48_pad60", dict(N=128, M=48, M_pad=60, L_cp=16, window=o.WINDOW_HANN, targets=2, frames=2)),
    ("256x100_threshold", dict(N=256, M=100, L_cp=32, window=o.WINDOW_HANN, targets=3, frames=2,
                               detect_mode=o.DETECT_THRESHOLD)),
    ("256x100_full_rect", dict(N=256, M=100, L_cp=256, window=o.WINDOW_RECT, targets=3, frames=2)),
    ("128x36_hann", dict(N=128, M=36, L_cp=16, window=o.WINDOW_HANN, targets=2, frames=2)),       # 3 x 3 x 4
    ("64x44_rect_prime11", dict(N=64, M=44, L_cp=8, window=o.WINDOW_RECT, targets=2, frames=2)),  # 11: two-factor
    ("512x1008_hamming", dict(N=512, M=1008, L_cp=64, window=o.WINDOW_HAMMING, targets=3, frames=1)),  # 7 3 3 16
]


@pytest.mark.parametrize("name,kw", GENERAL_M, ids=[c[0] for c in GENERAL_M])
def test_doppler_grid_not_a_power_of_two(env, name, kw):
    """M' = 560 = 2^4 5 7 (Table I) and other non-power-of-two Doppler grids:
    the mixed-radix Doppler transform (radices 7, 5, 3, 16, 8, 4), the
    two-factor form for a prime factor above 7 (M' = 44), and the general
    detection against the
    oracle (map, bins; the detection itself exactly on the GPU's own map)."""
    base = syn.FrameConfig(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], qam=16, zc_root=1, n_targets=kw["targets"],
                           on_grid=False, amp_db=(-6.0, 0.0), snr_db=(0.0, 0.0), window=kw["window"], detect_k=4)
    fr = []
    for f in range(kw["frames"]):
        d = syn.draw_frame(base, 8700 + f)
        Xp = o.zc_precode(d.A, 1)
        fr.append((d, Xp, syn.received(d, Xp)))
    p = o.Params(N=kw["N"], M=kw["M"], L_cp=kw["L_cp"], zc_root=1, window=kw["window"], max_targets=4,
                 M_pad=kw.get("M_pad", 0), detect_mode=kw.get("detect_mode", o.DETECT_TOPK))
    res = run_chain(env, p, [f[2] for f in fr], [f[0].A for f in fr])
    for i, (frm, Xp, Y) in enumerate(fr):
        ref = o.process(Y, frm.A, p)
        assert rel_l2(res["map"][i], ref["P"]) < MAP_TOL
        n = int(res["n"][i])
        rs = [(int(t["r"]), int(t["s"])) for t in res["tg"][i][:n]]
        if p.detect_mode == o.DETECT_TOPK:
            check_detections_vs_fp64(rs, res["tg"][i]["power"][:n], ref["det"], ref["P"])
        P32 = res["map"][i]
        eta = o.threshold(P32, ref["rows"], p.pfa, p.noise_var) if p.detect_mode == o.DETECT_THRESHOLD else None
        det32 = o.detect(P32, p.detect_mode, p.max_targets, eta)
        assert rs == list(zip(det32.r.tolist(), det32.s.tolist()))
        assert np.array_equal(res["tg"][i]["power"][:n], det32.power.astype(np.float32))
        assert int(res["status"][i]) == det32.status
