"""Shared helpers of the GPU parity tests: seeded frames, oracle runs and
comparisons.  Inputs come from ofdm_synth with the oracle's precoder; no
expected value ever comes from the CUDA path."""
from __future__ import annotations

import numpy as np

import ofdm_synth as syn
from oracle import ofdm_oracle as o

MAP_TOL = 1e-5      # relative L2 of the FP32 path against FP64 (periodogram and strip)
NEAR_TIE = 1e-5     # relative power gap under which two detections may swap


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_params(cfg: syn.FrameConfig, **kw) -> o.Params:
    d = dict(N=cfg.N, M=cfg.M, L_cp=cfg.L_cp, zc_root=cfg.zc_root, window=cfg.window,
             max_targets=cfg.detect_k)
    d.update(kw)
    return o.Params(**d)


def plan_kwargs(p: o.Params, frames: int) -> dict:
    return dict(N=p.N, M=p.M, N_pad=p.N_pad, M_pad=p.M_pad, L_cp=p.L_cp, n_cp=p.n_cp,
                zc_root=p.zc_root, zc_q=p.zc_q, x_is_precoded=int(p.x_is_precoded),
                window=p.window, detect_mode=p.detect_mode, max_targets=p.max_targets,
                max_frames=frames, pfa=p.pfa, noise_var=p.noise_var, fc_hz=p.fc_hz,
                df_hz=p.df_hz)


def make_frames(ci: int, frames: int, cfg: syn.FrameConfig | None = None, **draw_kw):
    """Seeded frames of workload `ci` with the oracle's ZC precoder."""
    cfg = cfg or syn.CONFIGS[ci]
    out = []
    for f in range(frames):
        fr = syn.draw_frame(cfg, syn.seed_for(ci, f), **draw_kw)
        Xp = o.zc_precode(fr.A, cfg.zc_root) if cfg.zc_root else fr.A
        out.append((fr, Xp, syn.received(fr, Xp)))
    return cfg, out


def stack_lk(arrs):
    return np.stack([syn.to_lk(a) for a in arrs])


def check_detections_vs_fp64(gpu_rs, gpu_pw, det: o.Detection):
    """Exact bin agreement with the FP64 oracle, except pairs of candidates
    whose oracle powers are within NEAR_TIE (relative) of each other."""
    want = list(zip(det.r.tolist(), det.s.tolist()))
    got = list(gpu_rs)
    if got == want:
        return 0
    # allow swaps only among near-ties, including the first unreported one
    pw = list(det.power) + ([det.next_power] if det.next_power else [])
    amb = 0
    for i, (g, w) in enumerate(zip(got, want)):
        if g != w:
            ref = pw[i]
            close = [j for j, q in enumerate(pw) if abs(q - ref) <= NEAR_TIE * ref]
            assert len(close) > 1, f"detection {i}: got {g}, oracle {want[i]} (no near-tie)"
            amb += 1
    return amb
