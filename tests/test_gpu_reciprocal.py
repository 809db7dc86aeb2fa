"""Direct accuracy of the reciprocal approximations the force kernels inline.

The paper's summary proposes replacing the division of Algorithm 1 with a
hardware reciprocal approximation followed by a correction (section
"Summary and Discussion").  The kernels do so; the end-to-end force tests
would hide a defect of a few ulps, so each reciprocal is evaluated here on
over a million arguments through lj_eval_reciprocal and compared, element
by element, with IEEE division computed on the host in extended precision:

* the FP64 forms (FP32 seed + one third-order correction; reciprocal
  square root with two Newton steps)
  must be faithful, within 1 ulp of the exact value, over their whole
  range, and report "in range" exactly where the kernels rely on them;
* the integer-arithmetic reciprocal of the fixed-point FP64 kernels (FP32
  seed, second-order Newton step on the integer significands) must be
  within 0.5 + 2^-10 ulp -- correctly rounded but for arguments whose
  reciprocal lies within about 2^-12 ulp of a rounding midpoint;
* the double-float reciprocals (one entry per lane and the packed f32x2
  pair) must keep the relative error of double-float arithmetic, 2^-44;
* the FP32 reciprocal of the mixed kernels must be within 1 FP32 ulp.

Arguments: a dense log-uniform sweep over the r^2 the kernels see (and the
lambda-unit R of the double-float kernels), random mantissas over every
exponent of each range, significands next to 1 and to 2 (where the
double-float seed's significand carries into the exponent), and the
exponents at and beyond each range's ends.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ULP_BOUND_FP64 = 1.0
REL_BOUND_DF = 2.0 ** -44
ULP_BOUND_FP32 = 1.0


def _arguments(e_lo: int, e_hi: int, seed: int = 0) -> np.ndarray:
    """Positive doubles: a dense sweep, random mantissas at every exponent in
    [e_lo, e_hi], significands near 1 and 2, and the exponents e_lo - 2 ..
    e_lo + 1 and e_hi - 1 .. e_hi + 2 (just outside the range included)."""
    g = np.random.default_rng(seed)
    parts = [np.exp2(g.uniform(-8.0, 8.0, size=1 << 20))]
    exps = np.arange(e_lo - 2, e_hi + 3)
    m = g.uniform(1.0, 2.0, size=(exps.size, 256))
    parts.append((m * np.exp2(exps)[:, None]).ravel())
    k = np.arange(0, 512, dtype=np.float64)
    for e in np.concatenate([exps[:4], exps[-4:], np.arange(-6, 7)]):
        parts.append(np.ldexp(1.0 + k * 2.0 ** -52, int(e)))
        parts.append(np.ldexp(2.0 - (k + 1) * 2.0 ** -52, int(e)))
        # significands whose leading 24 bits are all ones (the FP32 head is
        # 2 - 2^-23) with every pattern of a few tail bits
        parts.append(np.ldexp(2.0 - 2.0 ** -23 + k * 2.0 ** -52, int(e)))
    a = np.concatenate(parts)
    return a[np.isfinite(a) & (a > 0)]


def _exponent(a: np.ndarray) -> np.ndarray:
    return ((a.view(np.int64) >> 52) & 0x7FF).astype(np.int64) - 1023


def _ulps(x: np.ndarray, exact: np.ndarray) -> np.ndarray:
    """|x - exact| in units of the double spacing at the exact value."""
    ulp = np.spacing(np.abs(exact.astype(np.float64)))
    return np.abs(x.astype(np.longdouble) - exact) / ulp.astype(np.longdouble)


def _run(lj, kind, a):
    out, ok = lj.lj_eval_reciprocal(kind, torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy(), ok.cpu().numpy().astype(bool)


def test_extended_precision_reference_is_available():
    # the host reference needs more than 53 significand bits
    assert np.finfo(np.longdouble).nmant >= 63


@pytest.mark.parametrize("kind_name,e_lo,e_hi", [("LJ_RCP_FP64_FAST", -126, 125)])
def test_fp64_reciprocal_is_faithful(cuda_lib, kind_name, e_lo, e_hi):
    lj = cuda_lib
    a = _arguments(e_lo, e_hi)
    assert a.size >= 1_000_000
    out, ok = _run(lj, getattr(lj, kind_name), a)
    ea = _exponent(a)
    want_ok = (ea >= e_lo) & (ea <= e_hi)
    assert np.array_equal(ok, want_ok), "range flag differs from the documented range"
    exact = np.longdouble(1) / a[ok].astype(np.longdouble)
    err = _ulps(out[ok, 0], exact)
    worst = float(err.max())
    print(f"{kind_name}: max error {worst:.3f} ulp over {int(ok.sum())} arguments")
    assert worst <= ULP_BOUND_FP64, f"{kind_name}: {worst:.3f} ulp at a = {a[ok][np.argmax(err)]!r}"


def test_fp64_integer_reciprocal_is_nearly_correctly_rounded(cuda_lib):
    lj = cuda_lib
    a = _arguments(-119, 119)
    assert a.size >= 1_000_000
    out, ok = _run(lj, lj.LJ_RCP_FP64_INT, a)
    ea = _exponent(a)
    assert np.array_equal(ok, (ea >= -119) & (ea <= 119)), \
        "range flag differs from the documented range"
    exact = np.longdouble(1) / a[ok].astype(np.longdouble)
    err = _ulps(out[ok, 0], exact)
    worst = float(err.max())
    assert worst <= 0.5 + 2.0 ** -10, f"{worst:.6f} ulp at a = {a[ok][np.argmax(err)]!r}"
    # IEEE division on the host is correctly rounded.  On the random sweep
    # (the first 2^20 arguments) a miss needs 1/a within ~2^-12 ulp of a
    # midpoint: rare.  The structured significands are not counted: for
    # a = 2 - m 2^-52 with m odd, 1/a lies 2^-50 ulp or less from one.
    sweep = out[: 1 << 20, 0]
    missed = int(np.count_nonzero(sweep != 1.0 / a[: 1 << 20]))
    print(f"rcp_fp64_int: max error {worst:.6f} ulp over {int(ok.sum())} arguments, "
          f"{missed} of the 2^20 random ones not correctly rounded")
    assert missed <= 1e-3 * sweep.size


def test_fp64_rsqrt_is_faithful(cuda_lib):
    lj = cuda_lib
    a = _arguments(-119, 119)
    out, ok = _run(lj, lj.LJ_RSQRT_FP64, a)
    ea = _exponent(a)
    assert np.array_equal(ok, (ea >= -119) & (ea <= 119))
    exact = np.longdouble(1) / np.sqrt(a.astype(np.longdouble))
    err = _ulps(out[:, 0], exact)
    worst_in = float(err[ok].max())
    worst_out = float(err[~ok].max())
    print(f"rsqrt_fp64: max error {worst_in:.3f} ulp in range, {worst_out:.3f} outside "
          "(division fallback)")
    assert worst_in <= ULP_BOUND_FP64
    # outside the range the function divides by a rounded square root
    assert worst_out <= 2.0


@pytest.mark.parametrize("kind_name", ["LJ_RCP_DF", "LJ_RCP_DF2"])
def test_double_float_reciprocal(cuda_lib, kind_name):
    lj = cuda_lib
    g = np.random.default_rng(3)
    # the kernels' R (squared distance in lambda units, lambda in [r_c, 2 r_c))
    # lies in (2^-6, 1]; sweep wider, staying where every float is normal
    a = np.concatenate([np.exp2(g.uniform(-20.0, 20.0, size=1 << 20)),
                        _arguments(-6, 6)[: 1 << 18]])
    if kind_name == "LJ_RCP_DF2":
        a = a[:-1]  # odd length: the last lane carries one entry twice
    out, ok = _run(lj, getattr(lj, kind_name), a)
    assert ok.all()
    h = a.astype(np.float32).astype(np.float64)
    l = (a - h).astype(np.float32)
    x = h.astype(np.longdouble) + l.astype(np.longdouble)
    exact = np.longdouble(1) / x
    got = out[:, 0].astype(np.longdouble) + out[:, 1].astype(np.longdouble)
    rel = np.abs(got - exact) / exact
    worst = float(rel.max())
    print(f"{kind_name}: max relative error 2^{np.log2(worst):.2f}")
    assert worst <= REL_BOUND_DF
    # the result is a normalised double-float: |tail| <= ulp(head) / 2
    head = out[:, 0].astype(np.float32)
    assert np.all(np.abs(out[:, 1]) <= np.spacing(np.abs(head)).astype(np.float64) / 2)


def test_fp32_reciprocal_within_one_ulp(cuda_lib):
    lj = cuda_lib
    g = np.random.default_rng(5)
    a = np.concatenate([np.exp2(g.uniform(-60.0, 60.0, size=1 << 20)), _arguments(-8, 8)[: 1 << 18]])
    out, ok = _run(lj, lj.LJ_RCP_FP32, a)
    assert ok.all()
    af = a.astype(np.float32)
    exact = 1.0 / af.astype(np.float64)            # exact to 2^-53, far below an FP32 ulp
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    err = np.abs(out[:, 0] - exact) / ulp
    worst = float(err.max())
    print(f"rcp_fp32: max error {worst:.3f} FP32 ulp")
    assert worst <= ULP_BOUND_FP32
