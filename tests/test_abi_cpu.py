"""CPU-side checks of the C ABI: the library builds, loads and exports every
function the header declares; parameter validation rejects bad plans before
any device work.  No kernel is launched here."""
import ctypes

import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def radar():
    __graft_entry__.build()
    from paper_2209_03883_gb300 import radar as r
    return r


def test_exports_every_declared_function(radar):
    names = radar.declared_functions()
    assert len(names) >= 12
    lib = radar.lib()
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ofdm_radar.h but not exported"


def test_struct_layouts(radar):
    assert ctypes.sizeof(radar.Params) == 16 * 4 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(radar.Target) == 20


def test_default_params(radar):
    p = radar.default_params()
    assert p.zc_root == 1 and p.window == radar.WINDOW_HANN and p.max_targets == 8
    assert abs(p.pfa - 1e-2) < 1e-9 and p.fc_hz == 77e9 and p.df_hz == 240e3


BAD = [
    (dict(N=1000, M=256, L_cp=128), -2),      # N not a power of two
    (dict(N=8192, M=256, L_cp=128), -2),      # N too large
    (dict(N=1024, M=8, L_cp=128), -2),        # M too small
    (dict(N=1024, M=256, L_cp=0), -1),
    (dict(N=1024, M=256, L_cp=2048), -1),
    (dict(N=1024, M=256, L_cp=128, zc_root=2), -1),   # even root is not coprime to N^2
    (dict(N=1024, M=256, L_cp=128, window=7), -1),
    (dict(N=1024, M=256, L_cp=128, max_targets=0), -1),
    (dict(N=1024, M=256, L_cp=128, max_targets=33), -1),
    (dict(N=1024, M=256, L_cp=128, max_frames=0), -1),
    (dict(N=1024, M=256, L_cp=128, pfa=0.0), -1),
    (dict(N=1024, M=256, L_cp=128, N_pad=3072), -2),  # range padding: a power of two
    (dict(N=1024, M=256, L_cp=128, N_pad=8192), -2),  # range padding: N' <= 4096
    (dict(N=256, M=64, L_cp=32, N_pad=4096), -2),     # range padding: at most 8 N
    (dict(N=1024, M=256, L_cp=128, M_pad=200), -2),
]


@pytest.mark.parametrize("kw,code", BAD)
def test_plan_rejects_bad_params(radar, kw, code):
    with pytest.raises(radar.OfdmError) as ei:
        radar.Plan(**kw)
    assert ei.value.code == code


def test_null_arguments_rejected(radar):
    lib = radar.lib()
    assert lib.ofdm_radar_process(None, None, None, 1, None, None, None, None, None) == -1
    assert lib.ofdm_zc_precode(None, None, None, 1, 0, None) == -1
    assert lib.ofdm_radar_plan_create(None, None) == -1
    assert lib.ofdm_radar_strerror(-2).decode() == "unsupported size"


def test_more_struct_layouts(radar):
    assert ctypes.sizeof(radar.FrameDesc) == 32
    assert ctypes.sizeof(radar.FpsParams) == 24
    fp = radar.fps_default_params()
    assert (fp.iterations, fp.offsets, fp.max_recover) == (4, 8, 32)
    assert abs(fp.coherence_min - 0.95) < 1e-6


def test_batch_and_fps_reject_bad_input_before_any_launch(radar):
    lib = radar.lib()
    assert lib.ofdm_radar_batch_create(None, None, 0, 0, None) == -1
    assert lib.ofdm_fps_sft(None, None, None, 1, None, None, None, None, None) == -1
    assert lib.ofdm_radar_process_learned(None, None, None, None, 1, 0.0, 8, None, None, None, None) == -1
    assert radar.ofdm_cnn_param_count() == 16 * 9 + 16 + 16 * 16 * 9 + 16 + 16 * 9 + 1


def test_binding_checks_buffers_before_calling_the_library(radar):
    """dtype, contiguity, device and size are checked in the binding, so a
    float32 or transposed view never reaches a kernel (no GPU needed: host
    tensors are rejected for device arguments before any call)."""
    import torch
    p = radar.default_params(N=64, M=16, L_cp=8, max_targets=2)
    good = torch.zeros((1, 16, 64), dtype=torch.complex64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        radar.ofdm_radar_process_noalloc(p, good, good, 1)
    with pytest.raises(TypeError, match="complex64"):
        radar._buf(torch.zeros((1, 16, 64), dtype=torch.float32), "c64", 1024, "f", "Y")
    with pytest.raises(ValueError, match="contiguous"):
        radar._buf(torch.zeros((1, 64, 16), dtype=torch.complex64).transpose(1, 2), "c64", 1024, "f", "Y")
    with pytest.raises(ValueError, match="needs 2048"):
        radar._buf(good, "c64", 2048, "f", "Y", host=True)
    with pytest.raises(ValueError, match="CUDA tensor"):
        radar._chain_ptrs("f", 1, 64, 16, 64, 16, 2, good, good, None, None, None, None)
    assert radar._buf(good, "c64", 1024, "f", "Y", host=True).value == good.data_ptr()
    with pytest.raises(radar.OfdmError) as ei:
        radar._frames(0, "f")
    assert ei.value.code == -1


@pytest.mark.parametrize("kw,code", [
    (dict(N=2048, M=256, L_cp=128, precision=2), -2),   # split FP16: N = 1024 only
    (dict(N=1024, M=256, L_cp=256, precision=2), -2),   # Hann: rows up to L_cp need L_cp <= 255
    (dict(N=1024, M=256, L_cp=300, window=0, precision=2), -2),
    (dict(N=1024, M=256, L_cp=128, precision=1), -2),   # split BF16: not built
    (dict(N=1024, M=256, L_cp=128, precision=7), -1),
    (dict(N=1024, M=256, L_cp=128, detect_mode=2, cfar_guard=4, cfar_train=5), -1),   # guard + train <= 8
    (dict(N=1024, M=256, L_cp=128, detect_mode=2, cfar_train=0), -1),
    (dict(N=1024, M=256, L_cp=128, detect_mode=3), -1),
])
def test_precision_limits(radar, kw, code):
    with pytest.raises(radar.OfdmError) as ei:
        radar.Plan(**kw)
    assert ei.value.code == code
