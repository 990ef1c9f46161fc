"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own formulas: closed forms,
invariants (CAZAC, unitarity, Parseval), brute force on tiny inputs, a
library routine on a special case, a time-domain simulation of the OFDM
link, and the numbers printed in the paper's Table I.  The last test plants
mistakes in the oracle and checks that these pins catch each one.
"""
import json
import math
import os

import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- ZC (Sec. III-B)
def _periodic_autocorr(x):
    L = x.size
    return np.array([np.vdot(x, np.roll(x, -tau)) for tau in range(L)])


def check_zc_cazac(L, r, q=0):
    z = o.zc_sequence(L, r, q)
    assert np.allclose(np.abs(z), 1.0, atol=1e-12)
    ac = _periodic_autocorr(z)
    assert abs(ac[0] - L) < 1e-9 * L
    assert np.max(np.abs(ac[1:])) < 1e-8 * L, "ZC periodic autocorrelation must vanish off zero lag"


@pytest.mark.parametrize("L,r,q", [(16, 1, 0), (64, 3, 0), (64, 5, 2), (1024, 1, 0),
                                   (1024, 7, 3), (13, 1, 0), (63, 2, 1), (139, 5, 0)])
def test_zc_cazac(L, r, q):
    check_zc_cazac(L, r, q)


def check_zc_unitary(N, r, q=0):
    Z = o.zc_matrix(N, r, q)
    assert np.allclose(Z @ Z.conj().T, N * np.eye(N), atol=1e-9 * N)


@pytest.mark.parametrize("N,r,q", [(4, 1, 0), (8, 3, 0), (16, 5, 1), (64, 1, 0), (64, 7, 2)])
def test_zc_matrix_unitary(N, r, q):
    check_zc_unitary(N, r, q)


def test_zc_precode_roundtrip_and_norm():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((32, 5)) + 1j * rng.standard_normal((32, 5))
    Xp = o.zc_precode(A, 3, 1)
    assert np.allclose(np.linalg.norm(Xp, axis=0), np.linalg.norm(A, axis=0))
    assert np.allclose(o.zc_precode(Xp, 3, 1, inverse=True), A)


def test_zc_matrix_entries_bruteforce():
    # Z_m(i, j) is the (iN + j)-th sequence entry; the sequence phase is
    # checked against a pure-python evaluation with fractions of 2*pi.
    from fractions import Fraction
    N, r, q = 4, 3, 1
    Z = o.zc_matrix(N, r, q)
    L = N * N
    for i in range(N):
        for j in range(N):
            k = i * N + j
            ph = Fraction(r, L) * (Fraction(k * k, 2) + q * k)   # turns (units of 2 pi)
            ph -= math.floor(ph)
            want = complex(math.cos(2 * math.pi * ph), math.sin(2 * math.pi * ph))
            assert abs(Z[i, j] - want) < 1e-12


# ---------------------------------------------------------------- DFTs
def _dft_loops(x, sign):
    n = len(x)
    return [sum(x[k] * complex(math.cos(sign * 2 * math.pi * j * k / n),
                               math.sin(sign * 2 * math.pi * j * k / n)) for k in range(n))
            for j in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 8, 16])
def test_dft_matrix_bruteforce(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    W = o.dft_matrix(n)
    assert np.allclose(W @ x, _dft_loops(list(x), -1), atol=1e-12)
    assert np.allclose(W.conj() @ x, _dft_loops(list(x), +1), atol=1e-12)


def test_dft_matrix_matches_library_fft():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    assert np.allclose(o.dft_matrix(256) @ x, np.fft.fft(x), atol=1e-9)


# ---------------------------------------------------------------- DFT-CE (Sec. III-A)
def check_dft_ce_identity():
    rng = np.random.default_rng(2)
    H = rng.standard_normal((32, 4)) + 1j * rng.standard_normal((32, 4))
    Hd, _ = o.dft_ce(H, 32)
    assert np.allclose(Hd, H, atol=1e-12), "DFT-CE with L_cp = N is the identity"


def test_dft_ce_identity():
    check_dft_ce_identity()


def test_dft_ce_keeps_on_grid_targets_in_cp():
    N, M = 64, 8
    H = syn.channel([3.0, 11.0], [1.0, -2.0], [1.0, 0.5j], N, M)
    Hd, h = o.dft_ce(H, 16)
    assert np.allclose(Hd, H, atol=1e-12)
    # a target beyond the CP part is removed entirely
    H2 = syn.channel([20.0], [0.0], [1.0], N, M)
    Hd2, _ = o.dft_ce(H2, 16)
    assert np.max(np.abs(Hd2)) < 1e-12


# ---------------------------------------------------------------- periodogram (Eq. (17))
def _noiseless_point(N, M, L_cp, rho, nu, b, zc_root, window):
    syn_rng = np.random.default_rng(7)
    A = syn.qam_symbols(syn_rng, (N, M), 16)
    Xp = o.zc_precode(A, zc_root) if zc_root else A
    H = syn.channel([rho], [nu], [b], N, M)
    Y = Xp * H
    p = o.Params(N=N, M=M, L_cp=L_cp, zc_root=zc_root, window=window, max_targets=1)
    return o.process(Y, A, p)


def check_point_target_rect(N=64, M=16, rho=5, nu=-3, zc_root=1):
    out = _noiseless_point(N, M, 8, rho, nu, 0.8 * np.exp(0.7j), zc_root, o.WINDOW_RECT)
    P = out["P"]
    c = nu + M // 2
    assert abs(P[rho, c] - N * M * 0.64) < 1e-9 * N * M
    Q = P.copy()
    Q[rho, c] = 0
    assert Q.max() < 1e-18 * N * M
    det = out["det"]
    assert (int(det.r[0]), int(det.s[0])) == (rho, nu)


@pytest.mark.parametrize("zc_root", [0, 1, 3])
def test_point_target_rect_closed_form(zc_root):
    check_point_target_rect(zc_root=zc_root)


def check_point_target_hann(N=64, M=32, rho=4, nu=6, window=o.WINDOW_HANN):
    out = _noiseless_point(N, M, 16, rho, nu, 1.0, 1, window)
    P = out["P"]
    c = nu + M // 2
    c0, c1 = (0.5, 0.25) if window == o.WINDOW_HANN else (0.54, 0.23)
    want = np.zeros_like(P)
    for dr, wr in ((-1, c1), (0, c0), (1, c1)):
        for dc, wc in ((-1, c1), (0, c0), (1, c1)):
            want[(rho + dr) % N, (c + dc) % M] = N * M * (wr * wc) ** 2
    assert np.allclose(P, want, atol=1e-9 * N * M)


@pytest.mark.parametrize("window", [o.WINDOW_HANN, o.WINDOW_HAMMING])
def test_point_target_window_closed_form(window):
    check_point_target_hann(window=window)


# ---------------------------------------------------------------- range profile (Eq. (17), inner sum)
def check_range_profile_point(window=o.WINDOW_HANN, N=64, M=16, rho=6, nu=3):
    """A noiseless on-grid target survives DFT-CE unchanged, so H'[k, l] =
    b e^{-j2pi k rho/N} e^{+j2pi l nu/M}.  With the periodic Hann window
    w_k = 1/2 - (e^{+j2pi k/N} + e^{-j2pi k/N})/4 the range sum
    sum_k w_k H'[k, l] e^{+j2pi k r/N} is N b e^{+j2pi l nu/M} times 1/2 at
    r = rho, -1/4 at r = rho -+ 1 and 0 elsewhere (orthogonality of the
    exponentials); Hamming gives 0.54 / -0.23; rect gives N at r = rho alone."""
    b = 0.9 * np.exp(0.4j)
    c0, c1 = {o.WINDOW_RECT: (1.0, 0.0), o.WINDOW_HANN: (0.5, -0.25),
              o.WINDOW_HAMMING: (0.54, -0.23)}[window]
    want = np.zeros((N, M), dtype=complex)
    ramp = np.exp(2j * np.pi * np.arange(M) * nu / M)
    want[rho] = c0 * N * b * ramp
    want[(rho - 1) % N] += c1 * N * b * ramp
    want[(rho + 1) % N] += c1 * N * b * ramp
    # through the whole chain (ZC precoding, division, DFT-CE) ...
    out = _noiseless_point(N, M, 16, rho, nu, b, 1, window)
    assert np.allclose(out["g"], want, atol=1e-9 * N)
    # ... and on the channel alone
    g = o.range_profile(syn.channel([rho], [nu], [b], N, M), o.window(N, window))
    assert np.allclose(g, want, atol=1e-9 * N)


@pytest.mark.parametrize("window", [o.WINDOW_RECT, o.WINDOW_HANN, o.WINDOW_HAMMING])
def test_range_profile_point_closed_form(window):
    check_range_profile_point(window)


def check_range_profile_then_doppler_is_periodogram(N=32, M=16, window=o.WINDOW_HANN):
    """Eq. (17) is the range sum followed by the windowed Doppler sum: the
    oracle's range profile, Doppler-summed term by term here, must give its
    periodogram (centred columns, 1/(NM))."""
    rng = np.random.default_rng(11)
    Hd = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    g = o.range_profile(Hd, o.window(N, window))
    w_l = o.window(M, window)
    P = o.periodogram(Hd, o.window(N, window), w_l)
    want = np.zeros((N, M))
    for r in range(N):
        for c in range(M):
            s = c - M // 2
            acc = 0j
            for l in range(M):
                acc += w_l[l] * g[r, l] * np.exp(-2j * np.pi * ((l * s) % M) / M)
            want[r, c] = abs(acc) ** 2 / (N * M)
    assert np.allclose(P, want, rtol=1e-10, atol=1e-12 * want.max())


@pytest.mark.parametrize("window", [o.WINDOW_RECT, o.WINDOW_HANN])
def test_range_profile_then_doppler_is_periodogram(window):
    check_range_profile_then_doppler_is_periodogram(window=window)


# ---------------------------------------------------------------- coarse map of the learned proposal
def check_coarse_map_point(window=o.WINDOW_HANN, N=64, M=64, L_cp=16, rho=6, nu_c=3):
    """One noiseless on-grid target whose Doppler bin nu = 4 nu_c falls on the
    coarse grid.  Its support rows carry amplitude alpha_j e^{+j2pi l nu/M};
    over the first M/4 symbols that is e^{+j2pi l nu_c/(M/4)}, so the windowed
    (M/4)-point DFT is alpha_j (M/4) beta(c) with beta the window's own DFT:
    1 at c = nu_c for rect; 1/2 at nu_c and -1/4 at nu_c -+ 1 for Hann.  The
    coarse cell is the maximum over each group of 4 workspace rows of
    |alpha_j (M/4) beta(c)|^2, columns centred (c + M/8), x = log(1 + C/mean C)."""
    b = 0.7 * np.exp(-1.1j)
    Mc = M // 4
    rows = o.support_rows(N, L_cp, window)
    alpha = {o.WINDOW_RECT: {0: 1.0}, o.WINDOW_HANN: {0: 0.5, -1: -0.25, 1: -0.25}}[window]
    beta = {o.WINDOW_RECT: {0: 1.0}, o.WINDOW_HANN: {0: 0.5, -1: -0.25, 1: -0.25}}[window]
    ramp = np.exp(2j * np.pi * np.arange(M) * (4 * nu_c) / M)
    g_rows = np.zeros((len(rows), M), dtype=complex)
    for j, r in enumerate(rows):
        d = (int(r) - rho + N // 2) % N - N // 2
        if d in alpha:
            g_rows[j] = alpha[d] * N * b * ramp
    Hc = (len(rows) + 3) // 4
    C = np.zeros((Hc, Mc))
    for j, r in enumerate(rows):
        d = (int(r) - rho + N // 2) % N - N // 2
        if d not in alpha:
            continue
        for dc, bc in beta.items():
            c = (nu_c + dc + Mc // 2) % Mc          # centred column
            C[j // 4, c] = max(C[j // 4, c], abs(alpha[d] * N * b * Mc * bc) ** 2)
    want = np.log1p(C / C.mean())
    got = o.coarse_map(g_rows, window)
    assert got.shape == (Hc, Mc)
    assert np.allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("window", [o.WINDOW_RECT, o.WINDOW_HANN])
def test_coarse_map_point_closed_form(window):
    check_coarse_map_point(window)


def test_coarse_map_rect_peak_value():
    """Rect windows: the only non-zero coarse cell holds log(1 + Hc Mc)."""
    N, M, L_cp, rho, nu_c = 64, 32, 16, 9, -2
    Mc, rows = M // 4, o.support_rows(N, L_cp, o.WINDOW_RECT)
    g = o.range_profile(syn.channel([rho], [4 * nu_c], [1.0], N, M), o.window(N, o.WINDOW_RECT))
    x = o.coarse_map(g[rows], o.WINDOW_RECT)
    Hc = (len(rows) + 3) // 4
    peak = (rho // 4, nu_c + Mc // 2)
    assert x[peak] == pytest.approx(math.log1p(Hc * Mc), rel=1e-12)
    x[peak] = 0
    assert np.max(np.abs(x)) < 1e-12


def test_parseval():
    rng = np.random.default_rng(3)
    N, M = 32, 16
    Hd = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    wk, wl = o.window(N, o.WINDOW_HANN), o.window(M, o.WINDOW_HANN)
    P = o.periodogram(Hd, wk, wl)
    G = np.outer(wk, wl) * Hd
    assert abs(P.sum() - np.sum(np.abs(G) ** 2)) < 1e-9 * P.sum()


def test_periodogram_bruteforce_tiny():
    rng = np.random.default_rng(4)
    N, M, Np, Mp = 4, 4, 8, 4
    h = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    wk, wl = o.window(N, o.WINDOW_HAMMING), o.window(M, o.WINDOW_HAMMING)
    P = o.periodogram(h, wk, wl, Np, Mp)
    for r in range(Np):
        for s in range(-Mp // 2, Mp // 2):
            acc = 0j
            for k in range(N):
                inner = 0j
                for l in range(M):
                    inner += h[k, l] * wk[k] * wl[l] * complex(
                        math.cos(-2 * math.pi * l * s / Mp), math.sin(-2 * math.pi * l * s / Mp))
                acc += inner * complex(math.cos(2 * math.pi * k * r / Np),
                                       math.sin(2 * math.pi * k * r / Np))
            assert abs(P[r, s + Mp // 2] - abs(acc) ** 2 / (N * M)) < 1e-10


def test_zero_padding_interpolates():
    rng = np.random.default_rng(5)
    N, M = 16, 8
    Hd = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    wk, wl = o.window(N, o.WINDOW_HANN), o.window(M, o.WINDOW_HANN)
    P = o.periodogram(Hd, wk, wl)
    P2 = o.periodogram(Hd, wk, wl, 2 * N, 2 * M)
    for r in range(N):
        for s in range(-M // 2, M // 2):
            assert abs(P2[2 * r, 2 * s + M] - P[r, s + M // 2]) < 1e-9 * (1 + P.max())


# ---------------------------------------------------------------- detection (Eqs. (18)-(19))
def _local_max_loops(P):
    R, C = P.shape
    out = np.zeros_like(P, dtype=bool)
    for r in range(R):
        for c in range(C):
            if not P[r, c] > 0:
                continue
            ok = True
            me = r * C + c
            for dr in (-1, 0, 1):
                for dc in (-1, 0, 1):
                    rr, cc = (r + dr) % R, (c + dc) % C
                    other = rr * C + cc
                    if other == me:
                        continue
                    if P[rr, cc] > P[r, c] or (P[rr, cc] == P[r, c] and other < me):
                        ok = False
            out[r, c] = ok
    return out


@pytest.mark.parametrize("shape,seed", [((8, 8), 0), ((5, 7), 1), ((2, 6), 2), ((16, 4), 3)])
def test_local_maxima_bruteforce(shape, seed):
    rng = np.random.default_rng(seed)
    P = np.round(rng.random(shape) * 4) / 4      # many exact ties
    P[0, 0] = 0
    assert np.array_equal(o.local_maxima(P), _local_max_loops(P))


def test_detect_order_ties_and_status():
    P = np.zeros((6, 6))
    P[1, 1] = P[4, 4] = 5.0       # tie: smaller flat index first
    P[1, 4] = 7.0
    det = o.detect(P, o.DETECT_TOPK, 3)
    assert list(zip(det.r, det.s)) == [(1, 1), (1, -2), (4, 1)]
    det = o.detect(P, o.DETECT_TOPK, 5)
    assert det.status & o.STATUS_FEW_PEAKS and det.r.size == 3
    det = o.detect(P, o.DETECT_THRESHOLD, 1, eta=5.0)
    assert det.status & o.STATUS_OVERFLOW and det.count == 3 and det.r.size == 1


def test_threshold_float32_lower_median():
    P = np.array([[4.0, 1.0, 3.0, 2.0]], dtype=np.float32)
    eta = o.threshold(P, np.array([0]), 1e-2, -1.0)
    assert eta.dtype == np.float32
    assert eta == np.float32(2.0) * np.float32(-math.log(1e-2) / math.log(2.0))


# ---------------------------------------------------------------- Table I (Eqs. (14)-(15), (19))
def test_table1_resolutions():
    g = json.load(open(os.path.join(GOLDEN, "table1.json")))
    p, pr = g["params"], g["printed"]
    assert p["N"] * p["df_hz"] == pytest.approx(p["B_hz"])
    Ts = o.symbol_time(p["N"], p["N_cp"], p["df_hz"])
    dd, dv = o.resolution(p["N"], p["M"], p["df_hz"], p["fc_hz"], Ts)
    assert abs(dd - pr["range_resolution_m"]["value"]) < pr["range_resolution_m"]["tol"]
    assert abs(dv - pr["velocity_resolution_mps"]["value"]) < pr["velocity_resolution_mps"]["tol"]
    assert abs(p["N_cp"] * dd - pr["max_range_m"]["value"]) < pr["max_range_m"]["tol"]
    # max range as the CP-limited delay c*T_cp/2 (Eq. (13))
    Tcp = 0.07 / p["df_hz"]
    assert abs(o.C_LIGHT * Tcp / 2 - pr["max_range_normal_cp_m"]["value"]) < pr["max_range_normal_cp_m"]["tol"]
    dun, vun = o.unambiguous(p["df_hz"], p["fc_hz"], Ts)
    assert dun == pytest.approx(p["N"] * dd) and vun == pytest.approx(p["M"] * dv)


def test_detected_bin_to_physics():
    # A noiseless on-grid target at (rho0, nu0) converts back to rho0*dd, nu0*dv.
    N, M = 64, 32
    out = _noiseless_point(N, M, 16, 9, -5, 1.0, 1, o.WINDOW_RECT)
    Ts = o.symbol_time(N, 16, 240e3)
    dd, dv = o.resolution(N, M, 240e3, 77e9, Ts)
    assert out["d"][0] == pytest.approx(9 * dd) and out["v"][0] == pytest.approx(-5 * dv)


# ---------------------------------------------------------------- time-domain link (Eqs. (1)-(2), (12))
def test_time_domain_link_matches_frequency_model():
    """OFDM modulation with CP, an integer-sample delay and a per-symbol Doppler
    phase, CP removal and FFT reproduce Y = X * H of the generator's model."""
    N, M, Ncp = 32, 6, 8
    rng = np.random.default_rng(6)
    A = syn.qam_symbols(rng, (N, M), 4)
    d, nu, b = 5, 1.5, 0.7 * np.exp(0.3j)
    n = np.arange(N)
    tx = []
    for l in range(M):
        x = np.array([sum(A[k, l] * np.exp(2j * np.pi * nn * k / N) for k in range(N)) for nn in n])
        tx.append(np.concatenate([x[-Ncp:], x]))          # CP + symbol, Eq. (2)
    tx = np.concatenate(tx)
    rx = np.zeros_like(tx)
    rx[d:] = tx[:-d]                                        # round-trip delay of d samples
    Y = np.zeros((N, M), dtype=complex)
    for l in range(M):
        seg = rx[l * (N + Ncp) + Ncp: (l + 1) * (N + Ncp)] * b * np.exp(2j * np.pi * l * nu / M)
        Y[:, l] = np.array([sum(seg[nn] * np.exp(-2j * np.pi * nn * k / N) for nn in n)
                            for k in range(N)]) / N
    H = syn.channel([d], [nu], [b], N, M)
    assert np.allclose(Y, A * H, atol=1e-9)


# ---------------------------------------------------------------- the pins bite
MUTATIONS = {
    "zc_phase_doubled": ("zc_sequence", lambda f: (lambda L, r, q=0: f(L, r, q) ** 2)),
    "dft_conjugated": ("dft_matrix", lambda f: (lambda n: f(n).conj())),
    "dft_ce_no_truncation": ("dft_ce", lambda f: (lambda H, L: f(H, H.shape[0]))),
    "dft_ce_extra_scale": ("dft_ce", lambda f: (lambda H, L: tuple(x / H.shape[0] for x in f(H, L)))),
    "window_symmetric": ("window", lambda f: (lambda n, k: f(n + 1, k)[:n] if k else f(n, k))),
    "range_profile_no_window": ("range_profile",
                                lambda f: (lambda Hd, w_k, N_pad=None: f(Hd, np.ones_like(w_k), N_pad))),
    "coarse_map_no_window": ("coarse_map", lambda f: (lambda g, k: f(g, o.WINDOW_RECT))),
    "coarse_map_unshifted": ("coarse_map", lambda f: (lambda g, k: np.roll(f(g, k), f(g, k).shape[1] // 2, axis=1))),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(name, monkeypatch):
    attr, wrap = MUTATIONS[name]
    monkeypatch.setattr(o, attr, wrap(getattr(o, attr)))
    checks = [lambda: check_zc_cazac(64, 3), lambda: check_zc_unitary(16, 3),
              check_dft_ce_identity, check_point_target_rect, check_point_target_hann,
              lambda: test_dft_ce_keeps_on_grid_targets_in_cp(),
              lambda: check_range_profile_point(o.WINDOW_HANN),
              lambda: check_range_profile_then_doppler_is_periodogram(),
              lambda: check_coarse_map_point(o.WINDOW_HANN), lambda: check_coarse_map_point(o.WINDOW_RECT)]
    caught = 0
    for c in checks:
        try:
            c()
        except (AssertionError, ValueError, IndexError):
            caught += 1
    assert caught > 0, f"planted mistake {name} went unnoticed"


@pytest.mark.parametrize("N,L,w", [(64, 8, 0), (64, 8, 1), (64, 62, 1), (64, 63, 1), (64, 64, 0), (64, 63, 0)])
def test_support_rows_cover_nonzero_rows_once(N, L, w):
    rng = np.random.default_rng(N + L)
    H = rng.standard_normal((N, 4)) + 1j * rng.standard_normal((N, 4))
    Hd, _ = o.dft_ce(H, L)
    g = o.range_profile(Hd, o.window(N, w))
    rows = o.support_rows(N, L, w)
    assert len(set(rows.tolist())) == len(rows)
    nz = np.flatnonzero(np.abs(g).max(axis=1) > 1e-9 * np.abs(g).max())
    assert set(nz.tolist()) <= set(rows.tolist())


# ---------------------------------------------------------------- FPS-SFT (Sec. III-C)
def _sparse_case(seed, N, M, K, iters=6, T=8):
    rng = np.random.default_rng(seed)
    F = set()
    while len(F) < K:
        F.add((int(rng.integers(N)), int(rng.integers(M))))
    X = np.zeros((N, M), complex)
    for f in F:
        X[f] = (rng.standard_normal() + 1j * rng.standard_normal()) * N * M
    # time-domain signal by brute-force inverse 2D DFT (pure sums, no FFT)
    k = np.arange(N)[:, None]
    l = np.arange(M)[None, :]
    x = np.zeros((N, M), complex)
    for (f0, f1) in F:
        x += X[f0, f1] * np.exp(2j * np.pi * (f0 * k / N + f1 * l / M)) / (N * M)
    sp = []
    for _ in range(iters):
        a0 = int(rng.integers(0, N // 2)) * 2 + 1
        a1 = int(rng.integers(0, M // 2)) * 2 + 1
        sp.append((a0, a1, [(int(rng.integers(N)), int(rng.integers(M))) for _ in range(T)]))
    return F, X, x, sp


def check_fps_exact(seed=3, N=64, M=16, K=5):
    F, X, x, sp = _sparse_case(seed, N, M, K)
    rec = o.fps_sft(x, sp, o.FpsParams())
    got = {(f0, f1): a for f0, f1, a in rec}
    assert sorted(got) == sorted(F)
    for f in F:
        assert abs(got[f] - X[f]) < 1e-8 * abs(X[f])


@pytest.mark.parametrize("seed,N,M,K", [(0, 64, 64, 1), (1, 64, 64, 8), (2, 64, 16, 7), (3, 64, 16, 5),
                                        (4, 32, 32, 4), (5, 128, 32, 6)])
def test_fps_sft_exact_recovery(seed, N, M, K):
    check_fps_exact(seed, N, M, K)


def test_fps_line_membership():
    # every frequency on a bin's line maps back to that bin, and the lines of
    # all bins partition the N x M grid
    N, M, Q, a0, a1 = 16, 8, 16, 3, 5
    seen = set()
    for m in range(Q):
        for f0, f1 in o.fps_line(m, a0, a1, N, M, Q):
            assert (a0 * f0 * (Q // N) + a1 * f1 * (Q // M)) % Q == m
            seen.add((f0, f1))
    assert len(seen) == N * M


def test_fps_sft_agrees_with_periodogram():
    # small noisy frame with strong on-grid targets, rect window (K-sparse map)
    cfg = syn.FrameConfig(N=64, M=16, L_cp=16, qam=16, zc_root=1, n_targets=3, on_grid=True,
                          amp_db=(0.0, 0.0), snr_db=(10.0, 10.0), window=0)
    fr = syn.draw_frame(cfg, 4242)
    Xp = o.zc_precode(fr.A, 1)
    p = o.Params(N=64, M=16, L_cp=16, zc_root=1, window=0, max_targets=3)
    ref = o.process(syn.received(fr, Xp), fr.A, p)
    rng = np.random.default_rng(9)
    sp = [(int(rng.integers(0, 32)) * 2 + 1, int(rng.integers(0, 8)) * 2 + 1,
           [(int(rng.integers(64)), int(rng.integers(16))) for _ in range(8)]) for _ in range(4)]
    tg = o.fps_targets(o.fps_sft(ref["Hd"], sp, o.FpsParams()), 64, 16, 3)
    assert sorted((r, s) for _, _, r, s in tg) == sorted(zip(ref["det"].r.tolist(), ref["det"].s.tolist()))


def test_fps_pin_catches_wrong_peeling_sign(monkeypatch):
    real = o.np.exp
    calls = {"n": 0}

    def bad_exp(z):
        # conjugate the phase of the peeling step (first use inside each removal)
        return real(np.conj(z)) if np.iscomplexobj(z) and np.ndim(z) == 0 else real(z)
    monkeypatch.setattr(o.np, "exp", bad_exp)
    with pytest.raises(AssertionError):
        check_fps_exact(1, 64, 64, 8)


# ---------------------------------------------------------------- learned proposal: the CNN
def _conv_loops(x, w, b):
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    y = np.zeros((B, Co, H, W))
    for bb in range(B):
        for o_ in range(Co):
            for i in range(H):
                for j in range(W):
                    acc = b[o_]
                    for c in range(Ci):
                        for dy in range(3):
                            for dx in range(3):
                                ii, jj = i + dy - 1, j + dx - 1
                                if 0 <= ii < H and 0 <= jj < W:
                                    acc += w[o_, c, dy, dx] * x[bb, c, ii, jj]
                    y[bb, o_, i, j] = acc
    return y


def test_conv3x3_matches_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 5, 6))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    assert np.allclose(o.conv3x3(x, w, b), _conv_loops(x, w, b))


def test_cnn_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = 0.3 * rng.standard_normal(o.cnn_n_params())
    x = rng.standard_normal((2, 1, 6, 7))
    y = (rng.random((2, 1, 6, 7)) < 0.2).astype(float)

    def loss(t):
        z, _ = o.cnn_forward(x, t)
        return o.bce_logits(z, y, 4.0)[0]

    z, saved = o.cnn_forward(x, theta)
    _, gz = o.bce_logits(z, y, 4.0)
    g = o.cnn_backward(saved, theta, gz)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


# ---------------------------------------------------------------- PAPR (Sec. III-B, Eq. (25))
def test_papr_closed_forms():
    N = 64
    single = np.zeros((N, 1), complex)
    single[5] = 1.0                       # one subcarrier: constant-modulus time signal
    assert o.papr(single)[0] == pytest.approx(1.0)
    flat = np.ones((N, 1), complex)       # all ones: x = N delta[n]
    assert o.papr(flat)[0] == pytest.approx(N)


def test_zc_precoding_lowers_papr():
    # The paper's claim (Sec. III-B): ZC precoding reduces the OFDM PAPR.
    rng = np.random.default_rng(0)
    A = syn.qam_symbols(rng, (128, 200), 16)
    p0 = 10 * np.log10(o.papr(A))
    p1 = 10 * np.log10(o.papr(o.zc_precode(A, 1)))
    assert np.median(p1) < np.median(p0) - 3.0
    assert np.quantile(p1, 0.99) < np.quantile(p0, 0.5)


# ---------------------------------------------------------------- amplifier and spectrum (Sec. III-B)
def test_hpa_limits():
    """Small inputs pass linearly; large ones saturate at x_bar 10^(q/10);
    the phase is kept."""
    x = np.ones((10001, 1), complex)
    x[0, 0] = 1e-6 * np.exp(0.3j)
    x[-1, 0] = 1e12 * np.exp(-2.0j)
    y = o.hpa(x, q=2.0)
    sat = np.mean(np.abs(x)) * 10 ** 0.2
    assert abs(y[0, 0] - x[0, 0]) < 1e-9 * abs(x[0, 0])
    assert abs(abs(y[-1, 0]) - sat) < 1e-6 * sat
    assert np.allclose(np.angle(y), np.angle(x))
    # f(a) = a / sqrt(1 + (a/s)^2) at a = s gives s / sqrt(2)
    z = np.full((4, 1), 3.0 + 0j)
    assert np.allclose(np.abs(o.hpa(z, 0.0)), 3.0 / np.sqrt(2.0))


def test_oversampled_time_matches_direct_sum():
    rng = np.random.default_rng(4)
    N, L = 8, 3
    S = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    x = o.oversampled_time(S, L)
    for n in range(L * N):
        for c in range(2):
            want = sum(S[k, c] * np.exp(2j * np.pi * (k if k < N // 2 else k - N) * n / (L * N)) for k in range(N))
            assert abs(x[n, c] - want) < 1e-9
    assert np.allclose(o.oversampled_time(S, 1), o.dft_matrix(N).conj() @ S)


def test_aci_closed_forms():
    """A single subcarrier has a constant-modulus time signal: the amplifier
    only scales it, so nothing leaks out of band; any signal without the
    amplifier has zero out-of-band power; a clipped two-tone signal leaks."""
    N, L = 16, 4
    one = np.zeros((N, 1), complex)
    one[3] = 1.0
    x = o.oversampled_time(one, L)
    assert o.aci_ratio(o.hpa(x), N)[0] < 1e-20
    rng = np.random.default_rng(2)
    S = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    assert np.all(o.aci_ratio(o.oversampled_time(S, L), N) < 1e-20)
    two = np.zeros((N, 1), complex)
    two[1] = two[5] = 1.0
    assert o.aci_ratio(o.hpa(o.oversampled_time(two, L), 0.0), N)[0] > 1e-4


def test_zc_precoding_lowers_amplifier_leakage():
    """The paper's claim (Sec. III-B): with ZC precoding the amplifier adds less
    adjacent-channel interference (statistical, 128 subcarriers)."""
    rng = np.random.default_rng(9)
    A = syn.qam_symbols(rng, (128, 64), 16)
    p0, a0 = o.tx_papr_aci(A, 0)
    p1, a1 = o.tx_papr_aci(A, 1)
    assert np.median(p1) < np.median(p0)
    assert np.median(a1) < np.median(a0)


# ---------------------------------------------------------------- CFAR detection (reading F, local noise level)
def test_cfar_alpha_gives_pfa_exactly():
    """For exponential noise, P[P > alpha * mean of n training cells] has the
    closed form (1 + alpha/n)^-n; alpha is chosen so that it equals P_fa."""
    for n in (8, 24, 112):
        for pfa in (1e-2, 1e-4):
            a = o.cfar_alpha(n, pfa)
            assert (1 + a / n) ** (-n) == pytest.approx(pfa, rel=1e-12)
    assert o.cfar_alpha(10 ** 6, 1e-2) == pytest.approx(-math.log(1e-2), rel=1e-5)


def test_cfar_false_alarm_rate_on_noise():
    """Monte-Carlo check of the closed form on an exponential-noise map: the
    fraction of cells above the CFAR threshold matches P_fa (local maxima and
    all); a strong on-grid peak is always detected."""
    rng = np.random.default_rng(5)
    R, C = 64, 64
    P = rng.exponential(1.0, size=(R, C))
    pfa = 0.05
    rows = np.arange(R)
    g, t = 1, 4
    exceed = 0
    w = g + t
    for r in range(R):
        for c in range(C):
            tr = [P[(r + dr) % R, (c + dc) % C] for dr in range(-w, w + 1) for dc in range(-w, w + 1)
                  if not (abs(dr) <= g and abs(dc) <= g)]
            exceed += P[r, c] >= o.cfar_alpha(len(tr), pfa) * np.mean(tr)
    assert abs(exceed / (R * C) - pfa) < 4 * math.sqrt(pfa * (1 - pfa) / (R * C)) + 0.01
    P[20, 30] = 100.0
    det = o.cfar_detect(P, rows, pfa, g, t, 64)
    assert (20, 30 - C // 2) in set(zip(det.r.tolist(), det.s.tolist()))


def test_cfar_bruteforce_tiny_and_support_edge():
    """Hand-built 6 x 8 map, support rows 0..3: the training mean of a peak
    next to the support edge uses only support rows."""
    P = np.full((6, 8), 1.0)
    P[4:] = 0.0                       # outside the support
    P[3, 2] = 50.0
    P[1, 6] = 5.0
    det = o.cfar_detect(P, np.arange(4), 0.1, 0, 1, 4)
    # (3, 2): training = 8 neighbours minus the 3 on row 4 (off support) -> 5 cells of 1
    a5 = o.cfar_alpha(5, 0.1)
    assert 50.0 >= a5 * 1.0
    # (1, 6): 8 training cells of 1 -> alpha(8) = 8 (10^(1/8) - 1) ~ 2.68 < 5
    got = set(zip(det.r.tolist(), det.s.tolist()))
    assert got == {(3, 2 - 4), (1, 6 - 4)}
    assert list(det.power) == [50.0, 5.0]
