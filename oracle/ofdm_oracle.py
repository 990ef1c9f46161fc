"""FP64 CPU oracle of the OFDM monostatic radar receive chain.

Delamou, Noubir, Dang, Amhoud, "An Efficient OFDM-Based Monostatic Radar
Design for Multitarget Detection" (arXiv 2209.03883).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain definition that the
CUDA path is checked against.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product library never
does, and the two share no code, tables or constants.

Conventions
-----------
* Matrices follow the paper's orientation: a frame is an N x M array indexed
  [k, l], k = subcarrier (row), l = OFDM symbol (column) (Sec. II-B, Eq. (16)).
* Everything is complex128 / float64.  DFTs are explicit O(n^2) matrices built
  from exact integer index products, never an FFT.
* The range-Doppler map is indexed [r, c] with r = 0..N'-1 the range bin and
  c = s + M'/2 the column of Doppler bin s in [-M'/2, M'/2) (Eq. (17)).

Readings of the paper taken where it is silent or garbled (each also listed
in the design notes):
  A  the radar divides by the *precoded* grid X_p = Z_m A / sqrt(N).
  B  DFT-CE: IDFT carries 1/N, the DFT back carries no factor (Eqs. (20)-(22)).
  C  Z_m is N x N, so the ZC length is L = N^2; scaled by 1/sqrt(N) (unitary).
  D  Eq. (17): R' -> M', S' -> N'; Eq. (19): T_0 -> T_s, r <-> s swapped.
  E  periodic (DFT-even) Hann / Hamming windows, separable w_k * w_l.
  F  threshold eta = -sigma_P^2 ln(P_fa) (the printed sign is garbled).
  G  detections are 8-neighbour local maxima (circular in r and s), ordered by
     power descending then map index ascending.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 3.0e8  # speed of light used by the paper, Table I

WINDOW_RECT, WINDOW_HANN, WINDOW_HAMMING = 0, 1, 2
DETECT_TOPK, DETECT_THRESHOLD, DETECT_CFAR = 0, 1, 2

STATUS_ZERO_X = 1      # a precoded transmit cell was exactly zero
STATUS_NONFINITE = 2   # a non-finite input value was seen
STATUS_OVERFLOW = 4    # threshold mode found more targets than max_targets
STATUS_FEW_PEAKS = 8   # top-K mode found fewer than K local maxima


# --------------------------------------------------------------------------
# Zadoff-Chu sequence and matrix (Sec. III-B, Eqs. (23)-(24))
# --------------------------------------------------------------------------
def zc_sequence(L: int, r: int, q: int = 0) -> np.ndarray:
    """Zadoff-Chu sequence of length L with root r and shift q, Eq. (23).

    Even L:  exp(j 2 pi r / L * (k^2 / 2 + q k))  = exp(j pi m / L),
             m = r (k^2 + 2 q k) mod 2L.
    Odd L:   exp(j 2 pi r / L * (k (k + 1) / 2 + q k)) = exp(j 2 pi m / L),
             m = r (k (k + 1) / 2 + q k) mod L.
    The phase index m is reduced with exact int64 arithmetic, so the phase
    is exact before the one final exp.
    """
    if L <= 0:
        raise ValueError("L must be positive")
    if math.gcd(r, L) != 1:
        raise ValueError("ZC root must be coprime to L")
    if L >= 1 << 26:
        raise ValueError("L too large for exact int64 phase reduction")
    k = np.arange(L, dtype=np.int64)
    if L % 2 == 0:
        mod = 2 * L
        base = (k * k + 2 * (q % mod) * k) % mod          # k^2 + 2qk  (mod 2L)
        m = (base * (r % mod)) % mod                         # < 2^26 * 2^26
        return np.exp(1j * np.pi * m / L)
    mod = L
    base = (k * (k + 1) // 2 + (q % mod) * k) % mod        # k(k+1)/2 + qk  (mod L)
    m = (base * (r % mod)) % mod
    return np.exp(2j * np.pi * m / L)


def zc_matrix(N: int, r: int, q: int = 0) -> np.ndarray:
    """Square ZC matrix Z_m(i, j) = Z_seq(i D + j), D = sqrt(L), Eq. (24).

    Reading C: Z_m left-multiplies the N x M symbol grid, so D = N, L = N^2.
    """
    seq = zc_sequence(N * N, r, q)
    # Z_m(i, j) = seq[i N + j]: row-major reshape.
    return seq.reshape(N, N).copy()


def zc_precode(A: np.ndarray, r: int, q: int = 0, inverse: bool = False) -> np.ndarray:
    """ZC precoding A_p = Z_m A (Sec. III-B) and its undoing by Z_m^{-1}.

    Scaled by 1/sqrt(N) so that the transform is unitary (reading C); the
    inverse is then the conjugate transpose.  r = 0 means "no precoding".
    """
    A = np.asarray(A, dtype=np.complex128)
    if r == 0:
        return A.copy()
    N = A.shape[0]
    U = zc_matrix(N, r, q) / np.sqrt(N)
    if inverse:
        return U.conj().T @ A
    return U @ A


# --------------------------------------------------------------------------
# Radar processing (Sec. II-B.2) and DFT-CE (Sec. III-A)
# --------------------------------------------------------------------------
def ls_divide(Y: np.ndarray, X: np.ndarray):
    """LS spectral division h_{k,l} = y_{k,l} / x_{k,l}, Eq. (16).

    Cells whose transmit value is exactly zero give 0 and are counted.
    """
    Y = np.asarray(Y, dtype=np.complex128)
    X = np.asarray(X, dtype=np.complex128)
    zero = X == 0
    F = np.zeros_like(Y)
    F[~zero] = Y[~zero] / X[~zero]
    return F, int(zero.sum())


def dft_matrix(n: int) -> np.ndarray:
    """W[a, b] = exp(-j 2 pi a b / n), with a*b reduced mod n exactly."""
    idx = np.arange(n, dtype=np.int64)
    prod = np.outer(idx, idx) % n
    return np.exp(-2j * np.pi * prod / n)


def dft_ce(H: np.ndarray, L_cp: int):
    """DFT channel estimation, Eqs. (20)-(22), applied to every column.

    h = (1/N) W^H H          (IDFT over subcarriers, Eq. (20))
    h[n] = 0 for n >= L_cp   (keep the CP-long part, Eq. (21))
    H' = W h                 (DFT back, no factor -- reading B, Eq. (22))
    Returns (H', h_truncated).
    """
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    if not 1 <= L_cp <= N:
        raise ValueError("L_cp must be in [1, N]")
    W = dft_matrix(N)
    h = (W.conj() @ H) / N
    h[L_cp:, :] = 0
    return W @ h, h


def window(n: int, kind: int) -> np.ndarray:
    """Periodic window of length n (reading E): rect, Hann or Hamming (Sec. IV)."""
    k = np.arange(n, dtype=np.float64)
    if kind == WINDOW_RECT:
        return np.ones(n)
    if kind == WINDOW_HANN:
        return 0.5 - 0.5 * np.cos(2 * np.pi * k / n)
    if kind == WINDOW_HAMMING:
        return 0.54 - 0.46 * np.cos(2 * np.pi * k / n)
    raise ValueError("unknown window")


def range_profile(Hd: np.ndarray, w_k: np.ndarray, N_pad: int | None = None) -> np.ndarray:
    """Range transform of Eq. (17) alone: g[r, l] = sum_k w_k H'[k, l] e^{+j2pi k r / N'}."""
    N, M = Hd.shape
    N_pad = N if N_pad is None else N_pad
    G = np.zeros((N_pad, M), dtype=np.complex128)
    G[:N] = w_k[:, None] * Hd
    return dft_matrix(N_pad).conj() @ G


def periodogram(Hd: np.ndarray, w_k: np.ndarray, w_l: np.ndarray,
                N_pad: int | None = None, M_pad: int | None = None) -> np.ndarray:
    """Windowed 2D periodogram, Eq. (17), as an [r, c] map.

    P(s, r) = 1/(NM) |sum_k (sum_l h_{k,l} w_{k,l} e^{-j2pi l s/M'}) e^{+j2pi k r/N'}|^2
    with w_{k,l} = w_k w_l, h zero-padded to N' x M', and the Doppler axis
    reordered so that column c holds s = c - M'/2 (reading D).
    """
    N, M = Hd.shape
    N_pad = N if N_pad is None else N_pad
    M_pad = M if M_pad is None else M_pad
    if N_pad < N or M_pad < M:
        raise ValueError("padding must not shrink the grid")
    G = np.zeros((N_pad, M_pad), dtype=np.complex128)
    G[:N, :M] = np.outer(w_k, w_l) * Hd
    D = G @ dft_matrix(M_pad).T            # Doppler DFT over l  (e^{-j...})
    R = dft_matrix(N_pad).conj() @ D       # range IDFT over k  (e^{+j...}), no 1/N'
    P = np.abs(R) ** 2 / (N * M)
    out = np.empty_like(P)
    half = M_pad // 2
    for c in range(M_pad):
        s = c - half
        out[:, c] = P[:, s % M_pad]
    return out


# --------------------------------------------------------------------------
# Detection (Eqs. (18)-(19)) -- reading F and G
# --------------------------------------------------------------------------
def local_maxima(P: np.ndarray) -> np.ndarray:
    """8-neighbour local maxima of an [r, c] map, circular in both axes.

    A cell is a local maximum when P > 0 and, against every distinct
    neighbour n, P > P[n] or (P == P[n] and its flat index is smaller).
    """
    P = np.asarray(P)
    R, C = P.shape
    idx = np.arange(R * C, dtype=np.int64).reshape(R, C)
    ok = P > 0
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr == 0 and dc == 0:
                continue
            Pn = np.roll(P, (-dr, -dc), axis=(0, 1))
            In = np.roll(idx, (-dr, -dc), axis=(0, 1))
            same = In == idx
            ok &= same | (P > Pn) | ((P == Pn) & (idx < In))
    return ok


def support_rows(N: int, L_cp: int, window_kind: int) -> np.ndarray:
    """Range rows that can be non-zero after DFT-CE with N' = N (Eqs. (17), (21)).

    The truncated taps occupy r < L_cp; a periodic Hann/Hamming window over k
    spreads each tap to its two circular neighbours.
    """
    spread = 0 if window_kind == WINDOW_RECT else 2
    if L_cp + spread >= N:
        return np.arange(N)
    if window_kind == WINDOW_RECT:
        return np.arange(L_cp)
    return np.array([N - 1] + list(range(L_cp + 1)))


def threshold(P: np.ndarray, rows: np.ndarray, pfa: float, noise_var: float) -> np.floating:
    """Detection threshold eta = -sigma_P^2 ln(P_fa) of Eq. (18) (reading F).

    sigma_P^2 is the caller's noise level when noise_var > 0, otherwise the
    lower median of P over the given rows divided by ln 2 (the median of an
    exponential variable is its mean times ln 2).  The arithmetic is done in
    the map's own precision, so that a float32 map gives the float32 eta.
    """
    dt = P.dtype.type
    if noise_var > 0:
        return dt(noise_var) * dt(-math.log(pfa))
    vals = np.sort(P[rows, :].ravel())
    med = vals[(vals.size - 1) // 2]
    return dt(med) * dt(-math.log(pfa) / math.log(2.0))


@dataclass
class Detection:
    r: np.ndarray        # range bin 0..N'-1
    s: np.ndarray        # Doppler bin -M'/2..M'/2-1
    power: np.ndarray
    status: int = 0
    next_power: float = 0.0   # power of the first candidate not reported
    count: int = 0            # candidates found before truncation


def detect(P: np.ndarray, mode: int, max_targets: int, eta=None) -> Detection:
    """Peak picking on the map (Eq. (18)).

    mode DETECT_TOPK: the max_targets strongest local maxima.
    mode DETECT_THRESHOLD: local maxima with P >= eta, strongest first,
    at most max_targets of them.
    Order: power descending, then flat map index ascending (reading G).
    """
    R, C = P.shape
    lm = local_maxima(P)
    if mode == DETECT_THRESHOLD:
        lm &= P >= eta
    flat = np.flatnonzero(lm.ravel())
    vals = P.ravel()[flat]
    order = np.lexsort((flat, -vals.astype(np.float64)))
    flat, vals = flat[order], vals[order]
    status = 0
    if mode == DETECT_TOPK and flat.size < max_targets:
        status |= STATUS_FEW_PEAKS
    if mode == DETECT_THRESHOLD and flat.size > max_targets:
        status |= STATUS_OVERFLOW
    nxt = float(vals[max_targets]) if flat.size > max_targets else 0.0
    keep = flat[:max_targets]
    r = keep // C
    s = keep % C - C // 2
    return Detection(r=r, s=s, power=vals[:max_targets], status=status,
                     next_power=nxt, count=int(flat.size))


def cfar_alpha(n_train: int, pfa: float) -> float:
    """Cell-averaging CFAR multiplier: for a noise-only cell with exponential
    power and n_train independent training cells of the same mean,
    P[P > alpha * mean(training)] = (1 + alpha / n)^-n, which equals P_fa for
    alpha = n (P_fa^(-1/n) - 1) (-> -ln P_fa, the fixed-sigma threshold of
    Eq. (18), as n grows)."""
    return n_train * (pfa ** (-1.0 / n_train) - 1.0)


def cfar_detect(P: np.ndarray, rows: np.ndarray, pfa: float, guard: int, train: int, max_targets: int) -> Detection:
    """Detection with a locally estimated noise level (reading F made local,
    cell-averaging CFAR).  A cell of the support rows is a target when it is
    an 8-neighbour local maximum (reading G) and P >= alpha(n) * mean of its
    training cells: the cells within `guard + train` rows and columns of it
    but outside the (2 guard + 1)^2 guard square, circular in both axes, that
    lie on support rows (rows outside the DFT-CE support are zero by
    construction and carry no noise).  Order and cap as in detect()."""
    R, C = P.shape
    on_support = np.zeros(R, dtype=bool)
    on_support[rows] = True
    lm = local_maxima(P)
    w = guard + train
    hits = []
    for r in rows:
        for c in range(C):
            if not lm[r, c]:
                continue
            tot, n = 0.0, 0
            for dr in range(-w, w + 1):
                rr = (r + dr) % R
                if not on_support[rr]:
                    continue
                for dc in range(-w, w + 1):
                    if abs(dr) <= guard and abs(dc) <= guard:
                        continue
                    tot += float(P[rr, (c + dc) % C])
                    n += 1
            if n and P[r, c] >= cfar_alpha(n, pfa) * tot / n:
                hits.append(r * C + c)
    flat = np.array(sorted(hits), dtype=np.int64)
    vals = P.ravel()[flat] if flat.size else np.zeros(0)
    order = np.lexsort((flat, -vals.astype(np.float64)))
    flat, vals = flat[order], vals[order]
    status = STATUS_OVERFLOW if flat.size > max_targets else 0
    nxt = float(vals[max_targets]) if flat.size > max_targets else 0.0
    keep = flat[:max_targets]
    return Detection(r=keep // C, s=keep % C - C // 2, power=vals[:max_targets], status=status,
                     next_power=nxt, count=int(flat.size))


def symbol_time(N: int, n_cp: int, df_hz: float) -> float:
    """T_s = T + T_cp = (N + N_cp) / (N df), with T = 1/df (Sec. II-B)."""
    return (N + n_cp) / (N * df_hz)


def estimates(r, s, N_pad: int, M_pad: int, df_hz: float, fc_hz: float, Ts: float):
    """Eq. (19) (reading D): d = c r / (2 N' df), v = c s / (2 fc M' T_s)."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return C_LIGHT * r / (2 * N_pad * df_hz), C_LIGHT * s / (2 * fc_hz * M_pad * Ts)


def resolution(N: int, M: int, df_hz: float, fc_hz: float, Ts: float):
    """Eq. (15): range and velocity resolution."""
    return C_LIGHT / (2 * N * df_hz), C_LIGHT / (2 * M * fc_hz * Ts)


def unambiguous(df_hz: float, fc_hz: float, Ts: float):
    """Eq. (14): unambiguous range and velocity."""
    return C_LIGHT / (2 * df_hz), C_LIGHT / (2 * fc_hz * Ts)


# --------------------------------------------------------------------------
# Whole chain
# --------------------------------------------------------------------------
@dataclass
class Params:
    N: int
    M: int
    L_cp: int
    zc_root: int = 1
    zc_q: int = 0
    x_is_precoded: bool = False
    window: int = WINDOW_HANN
    detect_mode: int = DETECT_TOPK
    max_targets: int = 8
    pfa: float = 1e-2
    noise_var: float = -1.0
    N_pad: int = 0
    M_pad: int = 0
    n_cp: int = 0              # physical CP length for T_s; 0 -> L_cp
    cfar_guard: int = 1        # DETECT_CFAR: guard cells on each side
    cfar_train: int = 4        # DETECT_CFAR: training cells beyond the guard on each side
    fc_hz: float = 77e9
    df_hz: float = 240e3
    extra: dict = field(default_factory=dict)

    @property
    def Np(self):
        return self.N_pad or self.N

    @property
    def Mp(self):
        return self.M_pad or self.M


def process(Y: np.ndarray, A: np.ndarray, p: Params) -> dict:
    """The receive chain on one N x M frame, in the paper's order.

    ZC precoding of the known grid (Sec. III-B) -> LS division (Eq. (16)) ->
    DFT-CE (Eqs. (20)-(22)) -> windowed periodogram (Eq. (17)) ->
    detection (Eq. (18)) -> range / velocity estimates (Eq. (19)).
    """
    Y = np.asarray(Y, dtype=np.complex128)
    A = np.asarray(A, dtype=np.complex128)
    if p.zc_root and not p.x_is_precoded:
        Xp = zc_precode(A, p.zc_root, p.zc_q)
    else:
        Xp = A.copy()
    F, nzero = ls_divide(Y, Xp)
    Hd, h = dft_ce(F, p.L_cp)
    w_k = window(p.N, p.window)
    w_l = window(p.M, p.window)
    P = periodogram(Hd, w_k, w_l, p.Np, p.Mp)
    rows = support_rows(p.N, p.L_cp, p.window) if p.Np == p.N else np.arange(p.Np)
    eta = None
    if p.detect_mode == DETECT_THRESHOLD:
        eta = threshold(P, rows, p.pfa, p.noise_var)
    if p.detect_mode == DETECT_CFAR:
        det = cfar_detect(P, rows, p.pfa, p.cfar_guard, p.cfar_train, p.max_targets)
    else:
        det = detect(P, p.detect_mode, p.max_targets, eta)
    if nzero:
        det.status |= STATUS_ZERO_X
    Ts = symbol_time(p.N, p.n_cp or p.L_cp, p.df_hz)
    d, v = estimates(det.r, det.s, p.Np, p.Mp, p.df_hz, p.fc_hz, Ts)
    return dict(Xp=Xp, F=F, h=h, Hd=Hd, P=P, det=det, eta=eta, d=d, v=v,
                g=range_profile(Hd, w_k), rows=rows)


# --------------------------------------------------------------------------
# FPS-SFT (Sec. III-C) -- the sparse alternative to the 2D transform
# --------------------------------------------------------------------------
# The paper gives only the outline (I iterations, three or more Q-length
# slices per iteration, Q = lcm(N, M), a Q-point DFT per slice, frequencies
# recovered in one iteration removed from the next) and defers the details
# to its FPS-SFT reference.  This is our restatement from the
# projection-slice theorem, with the tolerances stated as parameters:
#   slice  s_j[n] = x[(a0 n + t0_j) mod N, (a1 n + t1_j) mod M], n < Q;
#   its Q-point DFT S_j[m] = (Q / (N M)) sum_f X[f] e^{+2pi i (f0 t0_j / N + f1 t1_j / M)}
#   over the frequencies f on the line a0 f0 Q/N + a1 f1 Q/M = m (mod Q),
#   X[f] = sum_{k,l} x[k,l] e^{-2pi i (f0 k / N + f1 l / M)} the 2D DFT.
# A bin holding one frequency is decoded by the maximum-likelihood search
# along its line (coherent sum over the T offsets), accepted when the
# coherence |sum_j S_j e^{-i theta_j}| / sum_j |S_j| passes `coherence_min`.

@dataclass
class FpsParams:
    iterations: int = 4
    offsets: int = 8
    max_recover: int = 32
    bin_pfa: float = 1e-6
    coherence_min: float = 0.95
    dynamic_range: float = 1e-10   # bins below this fraction of the strongest are not tested


def fps_line(m: int, a0: int, a1: int, N: int, M: int, Q: int):
    """Frequencies (f0, f1) whose slice bin is m: a0 f0 Q/N + a1 f1 Q/M = m (mod Q)."""
    out = []
    qn, qm = Q // N, Q // M
    for f0 in range(N):
        rest = (m - a0 * f0 * qn) % Q
        if rest % qm:
            continue
        # a1 f1 = rest / qm (mod M); a1 is odd, hence invertible mod M
        f1 = (pow(a1, -1, M) * (rest // qm)) % M
        out.append((f0, f1))
    return out


def fps_sft(x: np.ndarray, slice_params, fp: FpsParams):
    """FPS-SFT on an N x M signal x (here the DFT-CE estimate H').

    slice_params[i] = (a0, a1, [(t0_j, t1_j) for j < T]) for iteration i: the
    directions (odd) and offsets drawn by the caller.  Returns a list of
    (f0, f1, amplitude X[f]) in recovery order.
    """
    N, M = x.shape
    Q = math.lcm(N, M)
    rec = {}                      # (f0, f1) -> complex amplitude
    e_peak = 0.0
    for a0, a1, offs in slice_params:
        T = len(offs)
        n = np.arange(Q)
        S = []
        for t0, t1 in offs:
            s = x[(a0 * n + t0) % N, (a1 * n + t1) % M]
            S.append(dft_matrix(Q) @ s)                      # Q-point DFT of the slice
        S = np.array(S)
        # remove the frequencies already recovered (their bin in every slice)
        for (f0, f1), amp in rec.items():
            m = (a0 * f0 * (Q // N) + a1 * f1 * (Q // M)) % Q
            for j, (t0, t1) in enumerate(offs):
                ph = ((f0 * t0 * (Q // N) + f1 * t1 * (Q // M)) % Q) / Q
                S[j, m] -= (Q / (N * M)) * amp * np.exp(2j * np.pi * ph)
        E = np.mean(np.abs(S) ** 2, axis=0)                  # bin energy over the offsets
        thr = np.sort(E)[(Q - 1) // 2] / math.log(2.0) * (-math.log(fp.bin_pfa))
        e_peak = max(e_peak, float(E.max()))           # strongest bin of any iteration so far
        thr = max(thr, fp.dynamic_range * e_peak)
        found = []
        live = np.flatnonzero(E > thr)
        if live.size == 0:                 # nothing left above the noise: done
            break
        for m in live:
            best, bf = -1.0, None
            for f0, f1 in fps_line(int(m), a0, a1, N, M, Q):
                acc = 0j
                for j, (t0, t1) in enumerate(offs):
                    ph = ((f0 * t0 * (Q // N) + f1 * t1 * (Q // M)) % Q) / Q
                    acc += S[j, m] * np.exp(-2j * np.pi * ph)
                if abs(acc) > best:
                    best, bf = abs(acc), (f0, f1, acc)
            if bf is None or best < fp.coherence_min * np.sum(np.abs(S[:, m])):
                continue
            f0, f1, acc = bf
            found.append(((f0, f1), (N * M / Q) * acc / T))
        for key, amp in found:
            if key in rec:
                rec[key] += amp
            elif len(rec) < fp.max_recover:
                rec[key] = amp
    return [(f0, f1, a) for (f0, f1), a in rec.items()]


def fps_targets(rec, N: int, M: int, K: int):
    """Recovered frequencies as periodogram bins (Eq. (17) with a rect window):
    r = -f0 mod N (the range sum is an IDFT), s = f1 centred, P = |X|^2/(N M);
    ordered like detect(): power descending, then map index ascending."""
    rows = []
    for f0, f1, a in rec:
        r = (-f0) % N
        s = f1 - M if f1 >= M // 2 else f1
        rows.append((abs(a) ** 2 / (N * M), r * M + (s + M // 2), r, s))
    rows.sort(key=lambda t: (-t[0], t[1]))
    return rows[:K]


# --------------------------------------------------------------------------
# Learned proposal (not in the paper; its conclusion names machine learning
# as future work).  FP64 definition of the coarse map, the 3-layer CNN, its
# gradients and the training loss, for checking the GPU kernels.
# --------------------------------------------------------------------------
CNN_SHAPES = (("w1", (16, 1, 3, 3)), ("b1", (16,)), ("w2", (16, 16, 3, 3)), ("b2", (16,)),
              ("w3", (1, 16, 3, 3)), ("b3", (1,)))


def cnn_unflatten(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in CNN_SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def cnn_n_params() -> int:
    return sum(int(np.prod(s)) for _, s in CNN_SHAPES)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Same-size 3x3 convolution with zero padding: x [B, Ci, H, W], w [Co, Ci, 3, 3]."""
    B, Ci, H, W = x.shape
    xp = np.zeros((B, Ci, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((B, w.shape[0], H, W))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,bchw->bohw", w[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + W])
    return y + b[None, :, None, None]


def cnn_forward(x: np.ndarray, theta: np.ndarray):
    """conv(1->16)-ReLU-conv(16->16)-ReLU-conv(16->1): logits and saved activations."""
    p = cnn_unflatten(theta)
    z1 = conv3x3(x, p["w1"], p["b1"])
    a1 = np.maximum(z1, 0)
    z2 = conv3x3(a1, p["w2"], p["b2"])
    a2 = np.maximum(z2, 0)
    z3 = conv3x3(a2, p["w3"], p["b3"])
    return z3, (x, z1, a1, z2, a2)


def bce_logits(z: np.ndarray, y: np.ndarray, pos_weight: float):
    """Mean over cells of -[pw y log s(z) + (1 - y) log(1 - s(z))] and its gradient."""
    ls = -np.logaddexp(0.0, -z)            # log sigmoid(z)
    l1s = -np.logaddexp(0.0, z)            # log(1 - sigmoid(z))
    n = z.size
    loss = -np.sum(pos_weight * y * ls + (1 - y) * l1s) / n
    s = 1.0 / (1.0 + np.exp(-z))
    g = (pos_weight * y * (s - 1) + (1 - y) * s) / n
    return loss, g


def conv3x3_backward(x, w, gy):
    """Gradients of conv3x3 w.r.t. its input, weights and bias."""
    B, Ci, H, W = x.shape
    xp = np.zeros((B, Ci, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gy, xp[:, :, dy:dy + H, dx:dx + W])
            gxp[:, :, dy:dy + H, dx:dx + W] += np.einsum("oc,bohw->bchw", w[:, :, dy, dx], gy)
    return gxp[:, :, 1:-1, 1:-1], gw, gy.sum(axis=(0, 2, 3))


def cnn_backward(saved, theta, gz3):
    """Gradient of a loss w.r.t. the flat parameters, given dL/dlogits."""
    x, z1, a1, z2, a2 = saved
    p = cnn_unflatten(theta)
    ga2, gw3, gb3 = conv3x3_backward(a2, p["w3"], gz3)
    gz2 = ga2 * (z2 > 0)
    ga1, gw2, gb2 = conv3x3_backward(a1, p["w2"], gz2)
    gz1 = ga1 * (z1 > 0)
    _, gw1, gb1 = conv3x3_backward(x, p["w1"], gz1)
    g = {"w1": gw1, "b1": gb1, "w2": gw2, "b2": gb2, "w3": gw3, "b3": gb3}
    return np.concatenate([g[n].ravel() for n, _ in CNN_SHAPES])


def coarse_map(g_rows: np.ndarray, window_kind: int) -> np.ndarray:
    """The learned proposal's input from the support rows of the range profile
    g_rows [rows][M] (workspace order): an M/4-point Doppler DFT of the first M/4
    symbols with the window over those symbols, |.|^2, the maximum over each
    group of 4 rows, columns centred like the map, x = log(1 + C / mean C)."""
    rows, M = g_rows.shape
    Mc = M // 4
    w4 = window(Mc, window_kind)
    D = (g_rows[:, :Mc] * w4[None, :]) @ dft_matrix(Mc).T
    P = np.abs(D) ** 2
    Hc = (rows + 3) // 4
    C = np.zeros((Hc, Mc))
    for rc in range(Hc):
        C[rc] = P[4 * rc:4 * rc + 4].max(axis=0)
    Cs = np.empty_like(C)
    for c in range(Mc):
        Cs[:, c] = C[:, (c - Mc // 2) % Mc]
    return np.log1p(Cs / Cs.mean())


def papr(S: np.ndarray) -> np.ndarray:
    """PAPR of each OFDM symbol (column of S), Eq. (25), with the time signal of
    Eq. (1): x[n] = sum_k S[k] e^{+j 2 pi n k / N} (no 1/N).  Linear ratio."""
    S = np.asarray(S, dtype=np.complex128)
    x = dft_matrix(S.shape[0]).conj() @ S
    p = np.abs(x) ** 2
    return p.max(axis=0) / p.mean(axis=0)


# --------------------------------------------------------------------------
# Transmit side: PAPR through a nonlinear power amplifier (Sec. III-B)
# --------------------------------------------------------------------------
def hpa(x: np.ndarray, q: float = 2.0) -> np.ndarray:
    """Power amplifier of Sec. III-B: output modulus |x| / sqrt(1 + (|x| / (x_bar 10^(q/10)))^2)
    with the input phase kept (AM/AM only).  Reading: x_bar, "the mean of x",
    is the mean modulus of the symbol's time samples (the mean of the complex
    samples is about zero for an OFDM symbol); q is the state level (2)."""
    x = np.asarray(x, dtype=np.complex128)
    a = np.abs(x)
    sat = np.mean(a, axis=0, keepdims=True) * 10.0 ** (q / 10.0)
    g = 1.0 / np.sqrt(1.0 + (a / sat) ** 2)
    return x * g


def oversampled_time(S: np.ndarray, L: int) -> np.ndarray:
    """Time signal of each OFDM symbol (column of S) sampled L times per
    subcarrier spacing: subcarrier k sits at frequency k (k < N/2) or k - N
    (k >= N/2) of an L N-point grid, x[n] = sum_k S[k] e^{+j2pi f_k n / (L N)}
    (Eq. (1) with oversampling; L = 1 is Eq. (1) itself)."""
    S = np.asarray(S, dtype=np.complex128)
    N = S.shape[0]
    f = np.arange(N)
    f = np.where(f < N // 2, f, f + (L - 1) * N)          # bins of the L N grid
    Z = np.zeros((L * N,) + S.shape[1:], dtype=np.complex128)
    Z[f] = S
    return dft_matrix(L * N).conj() @ Z


def aci_ratio(y: np.ndarray, N: int) -> np.ndarray:
    """Share of the power of each oversampled symbol y (columns, L N samples)
    that falls outside the N occupied bins: the adjacent-channel interference
    that amplifier distortion creates (the spectrum study of Sec. III-B)."""
    Y = dft_matrix(y.shape[0]) @ np.asarray(y, dtype=np.complex128)
    LN = y.shape[0]
    occ = np.zeros(LN, dtype=bool)
    occ[:N // 2] = True
    occ[LN - N // 2:] = True
    p = np.abs(Y) ** 2
    return p[~occ].sum(axis=0) / p.sum(axis=0)


def tx_papr_aci(A: np.ndarray, zc_root: int, L: int = 4, q: float = 2.0, zc_q: int = 0):
    """Per OFDM symbol: PAPR (Eq. (25)) of the oversampled time signal of the
    transmitted grid (ZC-precoded when zc_root != 0) and the ACI ratio of the
    same signal after the amplifier."""
    Xp = zc_precode(A, zc_root, zc_q) if zc_root else np.asarray(A, dtype=np.complex128)
    x = oversampled_time(Xp, L)
    p = np.abs(x) ** 2
    return p.max(axis=0) / p.mean(axis=0), aci_ratio(hpa(x, q), A.shape[0])
