"""The mixed path's FP64 -> FP32 input conversion (d2f_rn, exported as gr_cast_f32) is the IEEE
conversion: round to nearest, ties to even, float subnormals, overflow to infinity, NaN kept.  Checked
bitwise against numpy's host conversion and the GPU's own conversion (torch .to(float32), the hardware
cvt.rn.f32.f64) over random doubles of every magnitude, exact ties, both sides of the smallest normal
and of the subnormal range, and the top of the float range."""
import numpy as np
import pytest

from paper_2311_04989_gb300 import grstage as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()
    return torch


def _cases(rng):
    bits = []
    # random doubles over the whole exponent range (random sign, exponent, significand)
    bits.append(rng.integers(0, 2 ** 63, 200_000, dtype=np.uint64) | (rng.integers(0, 2, 200_000, dtype=np.uint64) << 63))
    # exponents that map into and around the float range
    e = rng.integers(860, 1160, 200_000).astype(np.uint64)
    m = rng.integers(0, 2 ** 52, 200_000, dtype=np.uint64)
    bits.append((e << 52) | m)
    # exact ties (low 29 bits 0x10000000) with even and odd kept LSB, and one ulp either side
    t = (e << 52) | (m & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    bits += [t, t - np.uint64(1), t + np.uint64(1), t | np.uint64(0x20000000)]
    # both sides of 2^-126, 2^-149, 2^-150 and FLT_MAX (+ half an ulp) by direct values
    special = [2.0 ** -126, np.nextafter(2.0 ** -126, 0), np.nextafter(2.0 ** -126, 1), 2.0 ** -149, 2.0 ** -150,
               np.nextafter(2.0 ** -150, 0), np.nextafter(2.0 ** -150, 1), 1.5 * 2.0 ** -149, 2.5 * 2.0 ** -149,
               3.5 * 2.0 ** -149, 2.0 ** -1074, 0.0, float(np.finfo(np.float32).max),
               float(np.finfo(np.float32).max) * (1 + 2.0 ** -25), float(np.finfo(np.float32).max) * (1 + 2.0 ** -24),
               np.nextafter(2.0 ** 128, 0), 2.0 ** 128, 1e300, np.inf, 1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24]
    s = np.array(special, dtype=np.float64)
    bits.append(np.concatenate([s, -s]).view(np.uint64))
    x = np.concatenate(bits).view(np.float64)
    return np.concatenate([x, np.array([np.nan, -np.nan])])


@pytest.mark.parametrize("offset", [0, 1])
def test_cast_is_the_ieee_conversion(torch, offset):
    rng = np.random.default_rng(2311)
    x = _cases(rng)[offset:]                  # offset 1: an odd length and an 8-byte-aligned start
    src = torch.from_numpy(x).cuda()
    dst = torch.empty(src.numel(), dtype=torch.float32, device="cuda")
    if offset:
        big = torch.zeros(src.numel() + 1, dtype=torch.float64, device="cuda")
        big[1:] = src
        src = big[1:]                         # not 16-byte aligned: the element-wise path
    G.gr_cast_f32(src, dst, torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = dst.cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        host = x.astype(np.float32)
    dev = src.to(torch.float32).cpu().numpy()
    nan = np.isnan(x)
    assert np.array_equal(np.isnan(got), nan)
    gb, hb, db = got.view(np.uint32), host.view(np.uint32), dev.view(np.uint32)
    bad = np.flatnonzero((gb != hb) & ~nan)
    assert bad.size == 0, [(x[i], hex(gb[i]), hex(hb[i])) for i in bad[:8]]
    assert np.array_equal(gb[~nan], db[~nan])
    # the cases reach the rounding rule's edges: ties, subnormals and overflow all occur
    assert np.any((got != 0) & (np.abs(got) < np.finfo(np.float32).tiny)) and np.any(np.isinf(got) & ~np.isinf(x))


def test_cast_rejects_a_negative_size(torch):
    import ctypes as C
    L = G.load()
    assert L.gr_cast_f32(None, None, C.c_int64(-1), None) == -1
    assert L.gr_cast_f32(None, None, C.c_int64(0), None) == 0
