// Generated by gelu_fit.py: S(a) = erfcx(a / sqrt 2) / 2 ~ sum_k c_k u^k with
// c = GELU_S_COEFFS, u = a / 3 - 1, a in [0, 6] (degree 7, weighted least squares).
#pragma once
#define GELU_S_DEG 7
#define GELU_S_COEFFS {1.215069219e-01f, -1.015912443e-01f, 9.520497173e-02f, -4.894383252e-02f, -7.289769500e-02f, -4.403705001e-01f, -4.892418981e-01f, -2.545098960e-01f}
