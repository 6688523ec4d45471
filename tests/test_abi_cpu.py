"""Host-only checks of the C ABI: the library loads, exports every entry point that
include/lps_api.h declares, and rejects bad parameters before touching a GPU."""
import os
import re

import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.abi_layout import abi_to_mallat, bits_to_mallat, mallat_to_bits

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lps():
    from paper_1411_6206_gb300 import build, lps as L
    build.build()
    L.load()
    return L


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "lps_api.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lps_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lps):
    lib = lps.load()
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(lps.exported_symbols())


def test_params_defaults_and_status_strings(lps):
    p = lps.params_init()
    assert p.max_iters == 50 and p.wavelet_levels == 3 and p.fft_z == 1 and p.wavelet_dims == 2
    assert abs(p.lambda_L_rel - 0.01) < 1e-15 and abs(p.lambda_S_rel - 0.005) < 1e-15
    assert lps.status_string(0) == "LPS_OK"
    assert lps.status_string(-1) == "LPS_ERR_INVALID_ARG"
    assert lps.version() == 1


@pytest.mark.parametrize("bad,code", [
    (dict(nx=12), -1), (dict(ny=0), -1), (dict(ncoil=0), -1), (dict(wavelet_levels=4), -1),
    (dict(lambda_p=1.5), -1), (dict(layout=2), -1), (dict(layout=1), -8), (dict(precision=3), -1),
    (dict(nz=40), -8), (dict(ny=8 * 67), -8), (dict(max_iters=0), -1), (dict(coil_format=2), -1),
    (dict(wavelet_dims=1), -1), (dict(wavelet_dims=3, nz=12), -1), (dict(wavelet_dims=3, nz=6, wavelet_levels=2), -1),
    (dict(frame_slices=2), -1), (dict(layout=1, frame_slices=3), -1), (dict(layout=1, frame_slices=2, precision=1), -8),
    (dict(layout=1, frame_slices=2, nx_total=64), -8),
])
def test_plan_create_rejects_bad_params(lps, bad, code):
    kw = dict(nx=32, ny=32, nz=8, ncoil=2)
    kw.update(bad)
    p = lps.params_init(**kw)
    with pytest.raises(lps.LpsError) as e:
        lps.plan_create(p)
    assert e.value.code == code


def test_estimate_device_bytes(lps):
    p = lps.params_init(nx=128, ny=128, nz=16, ncoil=8)
    b = lps.estimate_device_bytes(p)
    N = 128 * 128 * 16
    assert 8 * N * 12 < b < 8 * N * 40
    assert lps.support_words(p) == N // 32


def test_half_precision_samples_are_an_extra_copy(lps):
    """LPS_DATA_FP16 keeps a binary16 copy of the hybrid samples: nx ncoil m 4 more bytes."""
    hdr = open(os.path.join(ROOT, "include", "lps_api.h")).read()
    assert re.search(r"#define LPS_DATA_FP32\s+0\b", hdr) and re.search(r"#define LPS_DATA_FP16\s+1\b", hdr)
    kw = dict(nx=128, ny=128, nz=16, ncoil=8)
    b32 = lps.estimate_device_bytes(lps.params_init(data_format=lps.DATA_FP32, **kw))
    b16 = lps.estimate_device_bytes(lps.params_init(data_format=lps.DATA_FP16, **kw))
    assert b16 > b32
    with pytest.raises(lps.LpsError):
        lps.plan_create(lps.params_init(data_format=2, **kw))


def test_half_precision_coil_maps_are_an_extra_copy(lps):
    """LPS_COILS_FP16 keeps a half-precision copy of the maps next to the rounded complex64
    ones: ncoil * N * 4 more bytes; the header and the binding agree on the constants."""
    hdr = open(os.path.join(ROOT, "include", "lps_api.h")).read()
    assert re.search(r"#define LPS_COILS_FP32\s+0\b", hdr) and re.search(r"#define LPS_COILS_FP16\s+1\b", hdr)
    kw = dict(nx=128, ny=128, nz=16, ncoil=8)
    b32 = lps.estimate_device_bytes(lps.params_init(coil_format=lps.COILS_FP32, **kw))
    b16 = lps.estimate_device_bytes(lps.params_init(coil_format=lps.COILS_FP16, **kw))
    assert b16 - b32 == 8 * 128 * 128 * 16 * 4


def test_frames_layout_is_the_per_frame_2d_encode(lps):
    """Layout "frames" (columns = frames of a 2D + time segment) takes the per-frame 2D encode:
    accepted with fft_z = 0 and planned like the slice layout with the per-slice encode; the
    header and the binding agree on the constants."""
    hdr = open(os.path.join(ROOT, "include", "lps_api.h")).read()
    assert re.search(r"#define LPS_LAYOUT_SLICES\s+0\b", hdr) and re.search(r"#define LPS_LAYOUT_FRAMES\s+1\b", hdr)
    assert (lps.LAYOUT_SLICES, lps.LAYOUT_FRAMES) == (0, 1)
    kw = dict(nx=64, ny=64, nz=12, ncoil=4, fft_z=0)
    bf = lps.estimate_device_bytes(lps.params_init(layout=lps.LAYOUT_FRAMES, **kw))
    bs = lps.estimate_device_bytes(lps.params_init(layout=lps.LAYOUT_SLICES, **kw))
    assert bf == bs > 0


@pytest.mark.parametrize("J", [1, 2, 3])
def test_abi_coefficient_order_is_blockwise_mallat(J):
    """The ABI order groups the coefficients of each 8x8 tile; inside it each 2^J block keeps
    its own Mallat layout. Check against the oracle's whole-plane transform."""
    rng = np.random.default_rng(0)
    nz, nx, ny = 2, 16, 24
    x = rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny))
    c = O.T(x, J)
    zz, ii, jj = abi_to_mallat(nz, nx, ny, J)
    assert len(set(zip(zz, ii, jj))) == nz * nx * ny            # a permutation
    vals = c[zz, ii, jj].reshape(nz, nx // 8, ny // 8, 8, 8)
    B = 1 << J
    for z in range(nz):
        for tx in range(nx // 8):
            for ty in range(ny // 8):
                tile = x[z, tx * 8:(tx + 1) * 8, ty * 8:(ty + 1) * 8]
                for su in range(8 // B):
                    for sv in range(8 // B):
                        blk = tile[su * B:(su + 1) * B, sv * B:(sv + 1) * B]
                        ref = O.haar2(blk, J)
                        got = vals[z, tx, ty, su * B:(su + 1) * B, sv * B:(sv + 1) * B]
                        assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("J", [1, 2, 3])
def test_abi_order_3d_is_blockwise_mallat(J):
    """With the 3D transform the ABI coefficient of slice z = bz 2^J + w, tile (tx, ty), (u, v)
    is coefficient (w, u', v') of the aligned 2^J x 2^J x 2^J block's own 3D transform."""
    rng = np.random.default_rng(3)
    nz, nx, ny = 16, 16, 8
    x = rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny))
    c = O.T3(x, J)
    zz, ii, jj = abi_to_mallat(nz, nx, ny, J, 3)
    assert len(set(zip(zz, ii, jj))) == nz * nx * ny
    vals = c[zz, ii, jj].reshape(nz, nx // 8, ny // 8, 8, 8)
    B = 1 << J
    for bz in range(nz // B):
        for tx in range(nx // 8):
            for ty in range(ny // 8):
                for su in range(8 // B):
                    for sv in range(8 // B):
                        x0, y0 = tx * 8 + su * B, ty * 8 + sv * B
                        ref = O.T3(x[bz * B:(bz + 1) * B, x0:x0 + B, y0:y0 + B], J)
                        got = vals[bz * B:(bz + 1) * B, tx, ty, su * B:(su + 1) * B, sv * B:(sv + 1) * B]
                        assert np.abs(got - ref).max() < 1e-12


def test_bitmap_pack_roundtrip():
    rng = np.random.default_rng(1)
    sup = rng.random((3, 16, 8)) < 0.3
    words = mallat_to_bits(sup, 3)
    assert words.dtype == np.uint32 and words.size == 3 * 16 * 8 // 32
    assert np.array_equal(bits_to_mallat(words, 3, 16, 8, 3), sup)
