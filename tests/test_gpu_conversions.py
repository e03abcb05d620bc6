"""The integer-built FP64 <-> FP32 conversions of the FP32 preconditioner
(every FP64 input element is narrowed to FP32 and every FP32 result widened
back on the hot path) against CUDA's own conversions, bit for bit, through
the aao_check_conversions self-test entry point.

The inputs are the cases where a hand-written IEEE-754 round-to-nearest-even
goes wrong first: exact ties (to even, both parities), a mantissa that
carries into the exponent, the top of the FP32 range (FLT_MAX and the values
that round to it or to infinity), the bottom of the normal range and the
FP32 subnormal results below it, FP64 subnormals, signed zeros, infinities,
NaN, and random doubles over the whole exponent range."""
import ctypes as C

import numpy as np
import pytest

from tests._helpers import need_gpu

pytestmark = pytest.mark.gpu


def _f64_cases():
    rng = np.random.default_rng(20240611)
    f = np.float32
    vals = []
    # ties: a float plus exactly half of its ulp (even and odd last bits)
    base = np.array([1.0, 1.0 + 2.0 ** -23, 1.5, 3.0 + 2.0 ** -22, 1e-30, 7.25e30, 0.1, 2.0 ** -126,
                     2.0 ** 127], dtype=np.float64)
    for b in base.astype(f).astype(np.float64):
        ulp = np.spacing(f(b)).astype(np.float64)
        vals += [b + ulp / 2, b - ulp / 4, b + ulp / 2 * (1 + 2.0 ** -29), b + ulp / 2 * (1 - 2.0 ** -29)]
    # mantissa carries into the exponent: just below a power of two
    for k in (-126, -60, -1, 0, 1, 20, 126):
        p = 2.0 ** k
        vals += [p * (1 - 2.0 ** -25), p * (1 - 2.0 ** -24), p * (1 - 2.0 ** -26), p * (1 - 2.0 ** -53)]
    # the top of the FP32 range
    fmax = float(np.finfo(f).max)
    half = 2.0 ** 103            # half an ulp of FLT_MAX (its ulp is 2^104)
    vals += [fmax, fmax + half * 0.5, fmax + half, fmax + half * (1 - 2.0 ** -20), 2 * fmax, 1e300]
    # the bottom: normal boundary, FP32 subnormal results, below the smallest
    tiny = float(np.finfo(f).tiny)
    vals += [tiny, tiny * (1 - 2.0 ** -25), tiny / 2, tiny / 3, 2.0 ** -149, 2.0 ** -150,
             2.0 ** -150 * 1.5, 2.0 ** -151, 1e-300]
    # FP64 subnormals, zeros, infinities, NaN
    vals += [5e-324, 2.2e-308, 0.0, np.inf, np.nan]
    v = np.array(vals, dtype=np.float64)
    v = np.concatenate([v, -v])
    # random bit patterns over the whole FP64 exponent range, and values near 1
    bits = rng.integers(0, 2 ** 63, size=20000, dtype=np.uint64)
    r1 = bits.view(np.float64)
    r2 = rng.standard_normal(20000) * np.exp2(rng.integers(-140, 130, size=20000))
    return np.concatenate([v, r1, -r1, r2])


def _f32_cases():
    rng = np.random.default_rng(7)
    f = np.float32
    v = np.array([0.0, 1.0, 1.5, np.finfo(f).max, np.finfo(f).tiny, np.finfo(f).tiny / 2, 1e-45,
                  np.inf, np.nan, 3.0e-39, 2.0 ** -126 * (1 - 2.0 ** -23)], dtype=f)
    v = np.concatenate([v, -v])
    r = rng.integers(0, 2 ** 32, size=40000, dtype=np.uint64).astype(np.uint32).view(f)
    return np.concatenate([v, r])


def _same_bits(a, b):
    """Equal bit patterns, with every NaN equal to every NaN."""
    nan = np.isnan(a) & np.isnan(b)
    ia = a.view(np.uint32 if a.dtype == np.float32 else np.uint64)
    ib = b.view(np.uint32 if b.dtype == np.float32 else np.uint64)
    return (ia == ib) | nan


def test_integer_conversions_match_cuda_bit_for_bit():
    torch = need_gpu()
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    x64 = torch.from_numpy(_f64_cases()).cuda()
    x32 = torch.from_numpy(_f32_cases()).cuda()
    lib32, ref32 = torch.empty(x64.numel(), dtype=torch.float32, device="cuda"), torch.empty(
        x64.numel(), dtype=torch.float32, device="cuda")
    lib64, ref64 = torch.empty(x32.numel(), dtype=torch.float64, device="cuda"), torch.empty(
        x32.numel(), dtype=torch.float64, device="cuda")
    st = lib.aao_check_conversions(
        C.c_void_p(x64.data_ptr()), x64.numel(), C.c_void_p(lib32.data_ptr()),
        C.c_void_p(ref32.data_ptr()), C.c_void_p(x32.data_ptr()), x32.numel(),
        C.c_void_p(lib64.data_ptr()), C.c_void_p(ref64.data_ptr()),
        C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    assert st == _capi.AAO_OK
    torch.cuda.synchronize()
    a, b = lib32.cpu().numpy(), ref32.cpu().numpy()
    bad = ~_same_bits(a, b)
    assert not bad.any(), list(zip(x64.cpu().numpy()[bad][:8], a[bad][:8], b[bad][:8]))
    a, b = lib64.cpu().numpy(), ref64.cpu().numpy()
    bad = ~_same_bits(a, b)
    assert not bad.any(), list(zip(x32.cpu().numpy()[bad][:8], a[bad][:8], b[bad][:8]))
    # CUDA's narrowing is the IEEE one numpy performs on the host
    with np.errstate(over="ignore", invalid="ignore"):
        want = _f64_cases().astype(np.float32)
    assert _same_bits(lib32.cpu().numpy(), want).all()


def test_conversion_check_rejects_bad_arguments():
    need_gpu()
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    assert lib.aao_check_conversions(None, -1, None, None, None, 0, None, None, None) == _capi.AAO_EINVAL
    assert lib.aao_check_conversions(None, 4, None, None, None, 0, None, None, None) == _capi.AAO_EINVAL
