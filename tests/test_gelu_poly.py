"""CPU pins of the inference kernels' GELU (Sec. 2.2 activation, exact form v Phi(v)).

The kernels evaluate GELU(v) = max(v, 0) - a Q(a), a = min(|v|, 6), with the Gaussian tail
Q(a) = exp(-a^2/2) S(a) and S a degree-7 polynomial in u = a/3 - 1 whose coefficients
live in csrc/gelu_poly.cuh (written by csrc/gelu_fit.py).  Here: the committed header is
what the generator writes; the formula, evaluated step by step in FP32 on the host, is
within 5e-6 (1 + |v|) of v Phi(v) computed with math.erf; and GELU(v) - GELU(-v) = v,
an identity of v Phi(v), holds to the rounding of the final FMA (two ulps of v)."""
import importlib.util
import io
import math
import pathlib
import re
from contextlib import redirect_stdout

import numpy as np
import pytest

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2604_27158_gb300" / "csrc"
F32 = np.float32


def _coefficients():
    text = (CSRC / "gelu_poly.cuh").read_text()
    deg = int(re.search(r"#define GELU_S_DEG (\d+)", text).group(1))
    body = re.search(r"#define GELU_S_COEFFS \{([^}]*)\}", text).group(1)
    c = [F32(float(x.strip().rstrip("f"))) for x in body.split(",")]
    assert len(c) == deg + 1
    return c


def _fma(a, b, c):
    # FP32 fused multiply-add: the product of two FP32 values is exact in FP64
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def gelu_kernel_formula(v):
    c = _coefficients()
    v = F32(v)
    a = min(abs(v), F32(6.0))
    u = _fma(a, F32(1.0 / 3.0), F32(-1.0))
    p = c[-1]
    for k in range(len(c) - 2, -1, -1):
        p = _fma(p, u, c[k])
    t = F32(F32(a * a) * F32(-0.72134752044448170))
    e = F32(2.0 ** np.float64(t))  # the kernels use ex2.approx (relative error < 2^-22)
    h = v if np.isnan(v) else max(v, F32(0.0))  # the kernels' NaN-propagating max.NaN
    return _fma(-a, F32(e * p), h)


def test_header_is_what_the_generator_writes():
    pytest.importorskip("scipy")
    spec = importlib.util.spec_from_file_location("gelu_fit", CSRC / "gelu_fit.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    buf = io.StringIO()
    with redirect_stdout(buf):
        mod.main()
    assert buf.getvalue() == (CSRC / "gelu_poly.cuh").read_text()


def test_formula_matches_exact_gelu():
    vs = np.concatenate([np.linspace(-12.0, 12.0, 40001), np.linspace(-1e-3, 1e-3, 201),
                         [-50.0, -6.0, -5.999, 5.999, 6.0, 50.0]]).astype(np.float32)
    worst = 0.0
    for v in vs.tolist():
        ref = 0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0)))
        worst = max(worst, abs(float(gelu_kernel_formula(v)) - ref) / (1.0 + abs(v)))
    assert worst < 5e-6, worst


def test_formula_symmetry_and_special_values():
    rng = np.random.default_rng(3)
    for v in rng.standard_normal(2000).astype(np.float32) * F32(4.0):
        d = np.float64(gelu_kernel_formula(v)) - np.float64(gelu_kernel_formula(-v))
        assert abs(d - np.float64(v)) <= 2.0 * np.spacing(abs(v)), (v, d)
    assert gelu_kernel_formula(0.0) == 0.0
    assert gelu_kernel_formula(np.inf) == np.inf
    assert np.isnan(gelu_kernel_formula(np.nan))
    # beyond the clamp the polynomial's value at a = 6 stands in for the (smaller) exact tail
    # (6 Q(6) = 5.9e-9); it stays far inside the bound 5e-6 (1 + |v|)
    assert abs(float(gelu_kernel_formula(-30.0))) < 5e-6
