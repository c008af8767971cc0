"""Writes gelu_poly.cuh: the polynomial behind the tensor-core kernels' GELU.

GELU(v) = v Phi(v) = max(v, 0) - a Q(a) with a = |v| and Q(a) = Phi(-a), the Gaussian
tail.  Q(a) = exp(-a^2 / 2) S(a) with S(a) = erfcx(a / sqrt 2) / 2 smooth and slowly
varying, so S is fitted by a polynomial of degree 7 in u = a / 3 - 1 on a in [0, 6]
(weighted least squares at Chebyshev nodes, weight exp(-a^2/2) max(a, 1/2): the
absolute error of a Q(a), which is what enters GELU), converted to monomial
coefficients and rounded to FP32.  Beyond a = 6, a Q(a) < 7e-9 and the kernels clamp a.

Run:  python gelu_fit.py > gelu_poly.cuh     (needs numpy and scipy)
"""
import numpy as np
from numpy.polynomial import chebyshev as C
from scipy.special import erfcx

DEG, A, NODES = 7, 6.0, 8000


def coefficients():
    u = np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)
    a = (u + 1.0) * A / 2.0
    w = np.exp(-a * a / 2.0) * np.maximum(a, 0.5)
    c = C.chebfit(u, 0.5 * erfcx(a / np.sqrt(2.0)), DEG, w=w)
    return C.cheb2poly(c).astype(np.float32)


def main():
    mono = coefficients()
    print("// Generated by gelu_fit.py: S(a) = erfcx(a / sqrt 2) / 2 ~ sum_k c_k u^k with")
    print(f"// c = GELU_S_COEFFS, u = a / 3 - 1, a in [0, {A:g}] (degree {DEG}, weighted least squares).")
    print("#pragma once")
    print(f"#define GELU_S_DEG {DEG}")
    body = ", ".join(f"{float(x):.9e}f" for x in mono)
    print(f"#define GELU_S_COEFFS {{{body}}}")


if __name__ == "__main__":
    main()
