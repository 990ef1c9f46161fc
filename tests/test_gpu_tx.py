"""Transmit side of Sec. III-B on the GPU (ofdm_tx_amplifier): PAPR of the
oversampled OFDM symbol and the out-of-band power the amplifier adds,
against the FP64 oracle on the same complex64 grid, and the paper's claim
that ZC precoding lowers both."""
import numpy as np
import pytest

import ofdm_synth as syn
from oracle import ofdm_oracle as o
from radar_cases import rel_l2

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


def gpu_tx(env, S, N, M, L, q):
    radar, torch, dev = env
    plan = radar.Plan(N=N, M=M, L_cp=N // 8, max_frames=1)
    Sd = torch.from_numpy(syn.to_lk(S)[None]).to(dev)
    papr = torch.empty((1, M), dtype=torch.float32, device=dev)
    aci = torch.empty((1, M), dtype=torch.float32, device=dev)
    radar.ofdm_tx_amplifier(plan, Sd, 1, L, q, papr, aci)
    torch.cuda.synchronize()
    return papr.cpu().numpy()[0], aci.cpu().numpy()[0]


def oracle_tx(S, L, q):
    x = o.oversampled_time(S, L)
    p = np.abs(x) ** 2
    return p.max(axis=0) / p.mean(axis=0), o.aci_ratio(o.hpa(x, q), S.shape[0])


@pytest.mark.parametrize("N,M,L,q,zc", [(128, 64, 4, 2.0, 1), (128, 64, 4, 2.0, 0), (1024, 16, 4, 2.0, 1),
                                        (64, 16, 1, 0.0, 0), (256, 16, 8, 4.0, 3)])
def test_tx_matches_oracle(env, N, M, L, q, zc):
    rng = np.random.default_rng(N + M + zc)
    A = syn.as_complex64_values(syn.qam_symbols(rng, (N, M), 16))
    S = syn.as_complex64_values(o.zc_precode(A, zc) if zc else A)
    papr, aci = gpu_tx(env, S, N, M, L, q)
    p_ref, a_ref = oracle_tx(S, L, q)
    assert rel_l2(papr, p_ref) < 1e-5
    if L > 1:
        assert rel_l2(aci, a_ref) < 1e-3
    else:
        assert np.all(aci == 0.0)   # no bins outside the band without oversampling


def test_zc_precoding_lowers_papr_and_leakage_on_gpu(env):
    """The paper's 128-subcarrier case: ZC precoding lowers both the PAPR and
    the amplifier's adjacent-channel leakage (medians over 256 symbols)."""
    rng = np.random.default_rng(12)
    A = syn.as_complex64_values(syn.qam_symbols(rng, (128, 256), 16))
    p0, a0 = gpu_tx(env, A, 128, 256, 4, 2.0)
    p1, a1 = gpu_tx(env, syn.as_complex64_values(o.zc_precode(A, 1)), 128, 256, 4, 2.0)
    assert np.median(p1) < np.median(p0)
    assert np.median(a1) < np.median(a0)
