"""Seeded synthetic OFDM radar frames (inputs only).

The generator draws what a monostatic radar would face in the paper's
simplified model (Sec. II-B, the ICI-free form after Eq. (11) and Eq. (16)):
QAM data A, point targets (range bin rho, Doppler bin nu, complex amplitude b),
the channel H[k, l] = sum_p b_p e^{-j 2 pi k rho_p / N} e^{+j 2 pi l nu_p / M}
and complex AWGN Z.  The received grid is Y = X_p * H + Z, where X_p is the
transmitted (possibly ZC-precoded) grid.

It holds none of the receive chain's arithmetic: the precoder that maps A to
X_p is passed in by the caller (the oracle's in tests, the library's own in
the benchmark), so this module serves both sides without tying them.

Frames are returned in the paper's orientation (N x M, [k, l]); `to_lk`
gives the library's [l][k] complex64 layout.  The workloads' inputs are
complex64, so the QAM grid A and the received grid Y are rounded to
complex64-representable values here (held as complex128): the FP64 oracle
and the library then consume the same numbers, and the comparison measures
the chain's arithmetic, not the rounding of its inputs (which the LS division
amplifies at near-zero precoded cells).  Seeds follow
seed = 1000 * config_index + frame_index with numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 3.0e8


@dataclass
class FrameConfig:
    N: int
    M: int
    L_cp: int
    qam: int = 16                 # 4 or 16
    zc_root: int = 1              # 0 -> no precoding
    n_targets: int = 5
    on_grid: bool = False
    amp_db: tuple = (0.0, 0.0)    # |b| log-uniform in this dB range
    snr_db: tuple = (0.0, 0.0)    # per-frame SNR drawn uniformly in this range
    window: int = 1               # 0 rect, 1 Hann, 2 Hamming
    frames: int = 1
    detect_k: int = 5
    name: str = ""
    extra: dict = field(default_factory=dict)


# The five workloads.  Index = config number used in the seed.
CONFIGS = {
    1: FrameConfig(N=64, M=16, L_cp=8, qam=4, zc_root=1, n_targets=2, on_grid=True,
                   amp_db=(0.0, 0.0), snr_db=(0.0, 0.0), window=0, frames=1,
                   detect_k=2, name="small 64x16"),
    2: FrameConfig(N=1024, M=256, L_cp=128, qam=16, zc_root=1, n_targets=5,
                   on_grid=False, amp_db=(-20.0, 0.0), snr_db=(-10.0, -10.0),
                   window=1, frames=64, detect_k=5, name="1024x256 batch 64"),
    3: FrameConfig(N=1024, M=1024, L_cp=128, qam=16, zc_root=1, n_targets=8,
                   on_grid=True, amp_db=(0.0, 0.0), snr_db=(5.0, 5.0), window=0,
                   frames=32, detect_k=8, name="sparse 1024x1024"),
    5: FrameConfig(N=4096, M=1024, L_cp=512, qam=16, zc_root=1, n_targets=32,
                   on_grid=False, amp_db=(-20.0, 0.0), snr_db=(-15.0, 5.0),
                   window=1, frames=16, detect_k=32, name="learned 4096x1024"),
}


def seed_for(config_index: int, frame_index: int) -> int:
    return 1000 * config_index + frame_index


def qam_symbols(rng: np.random.Generator, shape, order: int) -> np.ndarray:
    """Unit-average-power square QAM (4 or 16 points), uniform over the points."""
    m = int(round(np.sqrt(order)))
    if m * m != order or m < 2:
        raise ValueError("square QAM order expected")
    levels = 2.0 * np.arange(m) - (m - 1)
    scale = np.sqrt(2.0 * (m * m - 1) / 3.0)
    i = rng.integers(0, m, size=shape)
    q = rng.integers(0, m, size=shape)
    return (levels[i] + 1j * levels[q]) / scale


def draw_targets(rng: np.random.Generator, n: int, N: int, M: int, L_cp: int,
                 on_grid: bool, amp_db=(0.0, 0.0), min_sep: float = 3.0):
    """Point targets inside the CP support (Eq. (13)).

    rho in [2, L_cp - 3] keeps each target and its window spill inside the
    kept taps; nu in [-M/2 + 2, M/2 - 3]; any two targets are at least
    `min_sep` bins apart in range or in Doppler.  |b| is log-uniform over
    amp_db, the phase uniform.
    """
    lo_r, hi_r = 2.0, max(2.0, L_cp - 3.0)
    lo_v, hi_v = -M / 2 + 2.0, M / 2 - 3.0
    rho, nu = [], []
    tries = 0
    while len(rho) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot place targets with the requested separation")
        if on_grid:
            r = float(rng.integers(int(lo_r), int(hi_r) + 1))
            v = float(rng.integers(int(lo_v), int(hi_v) + 1))
        else:
            r = float(rng.uniform(lo_r, hi_r))
            v = float(rng.uniform(lo_v, hi_v))
        if all(abs(r - a) >= min_sep or abs(v - b) >= min_sep for a, b in zip(rho, nu)):
            rho.append(r)
            nu.append(v)
    mag_db = rng.uniform(amp_db[0], amp_db[1], size=n) if amp_db[1] > amp_db[0] else np.full(n, amp_db[0])
    phase = rng.uniform(0.0, 2 * np.pi, size=n)
    b = 10.0 ** (mag_db / 20.0) * np.exp(1j * phase)
    return np.array(rho), np.array(nu), b


def channel(rho, nu, b, N: int, M: int) -> np.ndarray:
    """H[k, l] = sum_p b_p e^{-j2pi k rho_p / N} e^{+j2pi l nu_p / M} (Eq. (16))."""
    k = np.arange(N)[:, None]
    l = np.arange(M)[None, :]
    H = np.zeros((N, M), dtype=np.complex128)
    for r, v, a in zip(rho, nu, b):
        H += a * np.exp(-2j * np.pi * k * r / N) * np.exp(2j * np.pi * l * v / M)
    return H


def awgn(rng: np.random.Generator, shape, snr_db: float) -> np.ndarray:
    """Complex AWGN with variance 10^(-SNR/10) per cell (unit-power symbols)."""
    s2 = 10.0 ** (-snr_db / 10.0)
    return np.sqrt(s2 / 2.0) * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


@dataclass
class Frame:
    A: np.ndarray       # N x M transmitted QAM grid
    H: np.ndarray       # N x M channel
    Z: np.ndarray       # N x M noise
    rho: np.ndarray
    nu: np.ndarray
    b: np.ndarray
    snr_db: float
    seed: int


def draw_frame(cfg: FrameConfig, seed: int, N: int | None = None, M: int | None = None,
               L_cp: int | None = None, qam: int | None = None,
               n_targets: int | None = None, noise: bool = True) -> Frame:
    """Everything random about one frame, from one PCG64 stream."""
    N = N or cfg.N
    M = M or cfg.M
    L_cp = L_cp or cfg.L_cp
    qam = qam or cfg.qam
    n_targets = cfg.n_targets if n_targets is None else n_targets
    rng = np.random.Generator(np.random.PCG64(seed))
    A = as_complex64_values(qam_symbols(rng, (N, M), qam))
    rho, nu, b = draw_targets(rng, n_targets, N, M, L_cp, cfg.on_grid, cfg.amp_db)
    snr = float(rng.uniform(*cfg.snr_db)) if cfg.snr_db[1] > cfg.snr_db[0] else cfg.snr_db[0]
    Z = awgn(rng, (N, M), snr) if noise else np.zeros((N, M), dtype=np.complex128)
    return Frame(A=A, H=channel(rho, nu, b, N, M), Z=Z, rho=rho, nu=nu, b=b,
                 snr_db=snr, seed=seed)


def as_complex64_values(a: np.ndarray) -> np.ndarray:
    """The nearest complex64 values, held as complex128."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def received(frame: Frame, Xp: np.ndarray) -> np.ndarray:
    """Y = X_p * H + Z for the transmitted grid X_p chosen by the caller,
    rounded to complex64 values (the receiver's input type)."""
    return as_complex64_values(Xp * frame.H + frame.Z)


def to_lk(a: np.ndarray) -> np.ndarray:
    """[k, l] (N x M) -> the library's [l][k] complex64 layout (M x N)."""
    return np.ascontiguousarray(np.asarray(a).T.astype(np.complex64))


def from_lk(a: np.ndarray) -> np.ndarray:
    return np.asarray(a).T


def mixed_batch_shapes(rng: np.random.Generator, n_frames: int):
    """Per-frame (N, M, L_cp, n_targets, qam) of the uneven batch: N in
    {256..2048}, M in {64, 128, 256}, L_cp = N/8, 1-16 targets, QPSK/16-QAM."""
    Ns = rng.choice([256, 512, 1024, 2048], size=n_frames)
    Ms = rng.choice([64, 128, 256], size=n_frames)
    K = rng.integers(1, 17, size=n_frames)
    Q = rng.choice([4, 16], size=n_frames)
    return [(int(n), int(m), int(n) // 8, int(k), int(q)) for n, m, k, q in zip(Ns, Ms, K, Q)]


def draw_frames_torch(cfg: FrameConfig, seeds, device, precode):
    """A batch of frames generated on the device (for training and large
    benchmarks).  Same recipe as draw_frame -- QAM data, targets inside the CP
    support, H = sum_p b_p e^{-j2pi k rho/N} e^{+j2pi l nu/M}, AWGN -- with the
    per-frame randomness from PCG64 (targets, SNR) and torch's Philox
    generator seeded from the first seed (symbols, noise).  `precode` maps a
    [B][M][N] complex64 tensor of QAM grids to the transmitted grids.
    Returns Y, A (both [B][M][N] complex64 on the device) and the targets."""
    import torch
    B, N, M = len(seeds), cfg.N, cfg.M
    g = torch.Generator(device=device)
    g.manual_seed(int(seeds[0]))
    m = int(round(np.sqrt(cfg.qam)))
    levels = (2.0 * torch.arange(m, device=device) - (m - 1)) / np.sqrt(2.0 * (m * m - 1) / 3.0)
    iq = torch.randint(0, m, (2, B, M, N), generator=g, device=device)
    A = torch.complex(levels[iq[0]], levels[iq[1]]).to(torch.complex64)
    Xp = precode(A)
    k = torch.arange(N, device=device, dtype=torch.float64)
    l = torch.arange(M, device=device, dtype=torch.float64)
    Y = torch.empty_like(A)
    truth = []
    for i, sd in enumerate(seeds):
        rng = np.random.Generator(np.random.PCG64(int(sd)))
        rho, nu, b = draw_targets(rng, cfg.n_targets, N, M, cfg.L_cp, cfg.on_grid, cfg.amp_db)
        snr = float(rng.uniform(*cfg.snr_db)) if cfg.snr_db[1] > cfg.snr_db[0] else cfg.snr_db[0]
        H = torch.zeros((M, N), dtype=torch.complex128, device=device)
        for r, v, a in zip(rho, nu, b):
            H += complex(a) * torch.outer(torch.exp(2j * np.pi * l * v / M), torch.exp(-2j * np.pi * k * r / N))
        s2 = 10.0 ** (-snr / 10.0)
        Z = np.sqrt(s2 / 2.0) * torch.complex(torch.randn((M, N), generator=g, device=device, dtype=torch.float32),
                                              torch.randn((M, N), generator=g, device=device, dtype=torch.float32))
        Y[i] = (Xp[i].to(torch.complex128) * H).to(torch.complex64) + Z
        truth.append((rho, nu, b, snr))
    return Y, A, truth
