"""Shared helpers of the GPU parity tests: seeded frames, oracle runs and
comparisons.  Inputs come from ofdm_synth with the oracle's precoder; no
expected value ever comes from the CUDA path."""
from __future__ import annotations

import numpy as np

import ofdm_synth as syn
from oracle import ofdm_oracle as o

MAP_TOL = 1e-5      # relative L2 of the FP32 path against FP64 (periodogram and strip)
NEAR_TIE = 1e-5     # relative power gap under which two detections may swap
PEAK_TOL = 1e-4     # relative error of one detected peak's power against FP64


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
                df_hz=p.df_hz, cfar_guard=p.cfar_guard, cfar_train=p.cfar_train)


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


def check_detections_vs_fp64(gpu_rs, gpu_pw, det: o.Detection, P: np.ndarray, near_tie: float = NEAR_TIE,
                             peak_tol: float = PEAK_TOL, map_tol: float = MAP_TOL):
    """Exact bin agreement with the FP64 oracle up to near-ties.

    gpu_rs: the GPU's (r, s) bins in its reported order; gpu_pw: their powers;
    det: the oracle's detections on the FP64 map P ([r, c], c = s + M'/2).
    The GPU must report as many targets as the oracle.  Where its i-th bin
    differs from the oracle's, that bin must itself be a peak of the FP64 map
    (no neighbour above it by more than near_tie) whose FP64 power lies
    within near_tie of the oracle's i-th power: two candidates that FP32
    cannot order.  Every reported power must match the FP64 power of its bin
    to peak_tol (relative, plus map_tol of the strongest peak).  Returns the
    number of swapped positions."""
    want = list(zip(det.r.tolist(), det.s.tolist()))
    got = [(int(r), int(s)) for r, s in gpu_rs]
    assert len(got) == len(want), f"{len(got)} detections, oracle has {len(want)}"
    assert len(set(got)) == len(got), f"repeated detection in {got}"
    R, C = P.shape
    top = float(det.power[0]) if len(want) else 0.0
    amb = 0
    for i, (g, w) in enumerate(zip(got, want)):
        r, c = g[0] % R, (g[1] + C // 2) % C
        pg = float(P[r, c])
        if g != w:
            ref = float(det.power[i])
            assert abs(pg - ref) <= near_tie * ref, \
                f"detection {i}: got {g} (P {pg:.6e}), oracle {w} (P {ref:.6e}): not a near-tie"
            nb = max(float(P[(r + dr) % R, (c + dc) % C]) for dr in (-1, 0, 1) for dc in (-1, 0, 1)
                     if (dr, dc) != (0, 0))
            assert nb <= pg * (1 + near_tie), f"detection {i}: got {g}, not a peak of the FP64 map"
            amb += 1
        assert abs(float(gpu_pw[i]) - pg) <= peak_tol * pg + map_tol * top, \
            f"detection {i} at {g}: power {float(gpu_pw[i]):.6e}, FP64 {pg:.6e}"
    return amb
