// Generated by gelu_fit.py: S(a) = erfcx(a / sqrt 2) / 2 ~ sum_k c_k u^k with
// c = GELU_S_COEFFS, u = a / 3 - 1, a in [0, 6] (degree 10, weighted least squares).
#pragma once
#define GELU_S_DEG 10
#define GELU_S_COEFFS {1.215115413e-01f, -1.032090634e-01f, 8.271647990e-02f, -6.052213535e-02f, 4.511024803e-02f, -5.191537365e-02f, -2.492748946e-02f, -1.331000403e-02f, 1.204707325e-01f, 1.375626922e-01f, 6.372436881e-02f}
