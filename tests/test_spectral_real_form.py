"""CPU pins of the real-form GEMMs behind the tensor-core y-DFT pair (Sec. 2.2 spectral layer).

The kernels never form complex products: the forward y-DFT is one real GEMM
D[(kx, c)][(a, q)] = sum_{(y, p)} X1[(kx, c)][(y, p)] Fy[(y, p)][(a, q)] over the
(Re, Im) pairs p of X1 and q of the result, and the inverse is
Zt[y][(k', o)] = sum_{(a, p)} Ty[y][(a, p)] Yb[(a, p)][(k', o)] with Yb the mixed modes
arranged as (Re Y, -Im Y) for k' = kx and (Im Y, Re Y) for k' = m + kx.  Here the
tables are built from those definitions in numpy and the two GEMMs are checked against
the complex sums they replace (the kept rows ky = 0..m-1 and H-m..H-1)."""
import numpy as np
import pytest


def kept_ky(a, H, m):
    return a if a < m else H - 2 * m + a


def fy_table(H, m):
    """Fy[(y, p)][(a, q)]: p = Re/Im of the input, q = Re/Im of the output mode a."""
    F = np.zeros((2 * H, 4 * m))
    for y in range(H):
        for a in range(2 * m):
            phi = 2 * np.pi * (kept_ky(a, H, m) * y % H) / H
            c, s = np.cos(phi), np.sin(phi)
            F[2 * y + 0, 2 * a + 0] = c    # Re x -> Re
            F[2 * y + 1, 2 * a + 0] = s    # Im x -> Re
            F[2 * y + 0, 2 * a + 1] = -s   # Re x -> Im
            F[2 * y + 1, 2 * a + 1] = c    # Im x -> Im
    return F


def ty_table(H, m):
    T = np.zeros((H, 4 * m))
    for y in range(H):
        for a in range(2 * m):
            phi = 2 * np.pi * (kept_ky(a, H, m) * y % H) / H
            T[y, 2 * a + 0] = np.cos(phi)
            T[y, 2 * a + 1] = np.sin(phi)
    return T


def yb_operand(Y, m):
    """Y[a][kx][o] complex -> Yb[(a, p)][(k', o)], k' < 2m."""
    A, _, C = Y.shape
    Yb = np.zeros((2 * A, 2 * m * C))
    for a in range(A):
        for kx in range(m):
            for o in range(C):
                y = Y[a, kx, o]
                Yb[2 * a + 0, kx * C + o] = y.real
                Yb[2 * a + 1, kx * C + o] = -y.imag
                Yb[2 * a + 0, (m + kx) * C + o] = y.imag
                Yb[2 * a + 1, (m + kx) * C + o] = y.real
    return Yb


@pytest.mark.parametrize("H,m,C", [(16, 4, 3), (24, 6, 2), (40, 5, 4)])
def test_forward_real_gemm_equals_kept_row_dft(H, m, C):
    rng = np.random.default_rng(H + m)
    X1 = rng.standard_normal((H, m, C)) + 1j * rng.standard_normal((H, m, C))
    # A operand: rows (kx, c), K = (y, Re/Im)
    A = np.zeros((m * C, 2 * H))
    A[:, 0::2] = X1.real.transpose(1, 2, 0).reshape(m * C, H)
    A[:, 1::2] = X1.imag.transpose(1, 2, 0).reshape(m * C, H)
    D = A @ fy_table(H, m)
    ref = np.fft.fft(X1, axis=0)  # sum_y X1 e^{-2 pi i ky y / H} for every ky
    for a in range(2 * m):
        got = D[:, 2 * a] + 1j * D[:, 2 * a + 1]
        np.testing.assert_allclose(got, ref[kept_ky(a, H, m)].reshape(m * C), rtol=0, atol=1e-11)


@pytest.mark.parametrize("H,m,C", [(16, 4, 3), (24, 6, 2), (40, 5, 4)])
def test_inverse_real_gemm_equals_kept_row_idft(H, m, C):
    rng = np.random.default_rng(7 * H + m)
    Y = rng.standard_normal((2 * m, m, C)) + 1j * rng.standard_normal((2 * m, m, C))
    Z = ty_table(H, m) @ yb_operand(Y, m)  # [y][(k', o)]
    for y in range(H):
        ref = np.zeros((m, C), complex)
        for a in range(2 * m):
            ref += Y[a] * np.exp(2j * np.pi * kept_ky(a, H, m) * y / H)
        np.testing.assert_allclose(Z[y, :m * C], ref.real.reshape(-1), rtol=0, atol=1e-11)
        np.testing.assert_allclose(Z[y, m * C:], ref.imag.reshape(-1), rtol=0, atol=1e-11)
