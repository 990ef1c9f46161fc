"""Training and use of the learned proposal (not in the paper; its
conclusion names machine learning as future work).

Every arithmetic step -- coarse maps, CNN forward and backward, loss, Adam --
runs in the library's own kernels (include/ofdm_radar.h); torch only holds
device memory.  Frames come from ofdm_synth.draw_frames_torch.
"""
from __future__ import annotations

import struct

import numpy as np

from . import radar

MAGIC = b"OFDMCNN1"


def coarse_labels(truth, N, M, rows, row0, Hc, Mc):
    """One positive coarse cell per target: support row (r - row0) mod N pooled
    4x, Doppler bin rounded to the M/4-point grid, columns centred."""
    lab = np.zeros((len(truth), Hc, Mc), dtype=np.float32)
    for f, (rho, nu, _b, _snr) in enumerate(truth):
        for r, v in zip(rho, nu):
            ri = (int(round(r)) - row0) % N
            if ri >= rows:
                continue
            sc = int(round(v / 4.0))
            lab[f, ri // 4, (sc + Mc // 2) % Mc] = 1.0
    return lab


class Trainer:
    """Adam on the CNN parameters with the library's kernels."""

    def __init__(self, plan: radar.Plan, torch, device, seed=0, lr=3e-3, pos_weight=50.0):
        self.plan, self.torch, self.dev = plan, torch, device
        self.Hc, self.Mc = radar.ofdm_radar_learned_prepare(plan)
        self.P = radar.ofdm_cnn_param_count()
        rng = np.random.default_rng(seed)
        fan = [9, 9, 144, 144, 144, 144]
        theta = []
        for (name, shp), fi in zip((("w1", (16, 1, 3, 3)), ("b1", (16,)), ("w2", (16, 16, 3, 3)), ("b2", (16,)),
                                    ("w3", (1, 16, 3, 3)), ("b3", (1,))), fan):
            n = int(np.prod(shp))
            theta.append(rng.standard_normal(n) * np.sqrt(2.0 / fi) if name[0] == "w" else np.zeros(n))
        t = torch
        self.theta = t.from_numpy(np.concatenate(theta).astype(np.float32)).to(device)
        self.m = t.zeros_like(self.theta)
        self.v = t.zeros_like(self.theta)
        self.g = t.zeros_like(self.theta)
        self.step = 0
        self.seed = seed
        self.lr, self.pos_weight = lr, pos_weight

    def _buffers(self, B):
        t, dev = self.torch, self.dev
        shp = (B, 16, self.Hc, self.Mc)
        if getattr(self, "_B", None) != B:
            self._B = B
            self.x = t.empty((B, self.Hc, self.Mc), dtype=t.float32, device=dev)
            self.a1, self.a2 = t.empty(shp, device=dev), t.empty(shp, device=dev)
            self.ga1, self.ga2 = t.empty(shp, device=dev), t.empty(shp, device=dev)
            self.z = t.empty((B, self.Hc, self.Mc), device=dev)
            self.gz = t.empty_like(self.z)
            self.loss = t.zeros((1,), device=dev)

    def coarse(self, Y, A):
        B = Y.shape[0]
        self._buffers(B)
        radar.ofdm_radar_coarse_map(self.plan, Y, A, B, self.x)
        return self.x

    def train_step(self, Y, A, labels):
        B = Y.shape[0]
        self.coarse(Y, A)
        lab = self.torch.from_numpy(labels).to(self.dev)
        radar.ofdm_cnn_forward(self.theta, 1, self.x, B, self.Hc, self.Mc, self.a1, self.a2, self.z)
        radar.ofdm_cnn_bce(self.z, lab, lab.numel(), self.pos_weight, self.loss, self.gz)
        radar.ofdm_cnn_backward(self.theta, 1, self.x, self.a1, self.a2, self.gz, B, self.Hc, self.Mc,
                                self.ga1, self.ga2, self.g)
        self.step += 1
        radar.ofdm_cnn_adam(self.theta, self.g, self.m, self.v, self.P, self.step, self.lr)
        return self.loss

    def logits(self, Y, A):
        B = Y.shape[0]
        self.coarse(Y, A)
        radar.ofdm_cnn_forward(self.theta, 1, self.x, B, self.Hc, self.Mc, self.a1, self.a2, self.z)
        return self.z

    # -- checkpoint / resume: header, then little-endian float32 theta, m, v
    def save(self, path):
        with open(path, "wb") as f:
            f.write(MAGIC + struct.pack("<iiq", self.P, self.step, self.seed))
            for arr in (self.theta, self.m, self.v):
                f.write(arr.detach().cpu().numpy().astype("<f4").tobytes())

    def load(self, path):
        with open(path, "rb") as f:
            if f.read(8) != MAGIC:
                raise ValueError("not a CNN checkpoint")
            P, step, seed = struct.unpack("<iiq", f.read(16))
            if P != self.P:
                raise ValueError("parameter count mismatch")
            for arr in (self.theta, self.m, self.v):
                arr.copy_(self.torch.from_numpy(np.frombuffer(f.read(4 * P), dtype="<f4").copy()))
        self.step, self.seed = step, seed
