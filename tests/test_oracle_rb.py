"""Pins of the reduced-basis amplitude oracle (Sec. 3.E, RomanNet: A = alpha . B, then each
knot's vector rescaled to a given norm) against facts that do not come from the oracle: a
product worked by hand, the identity basis, the discrete Fourier basis (numpy's FFT), the
round trip through an orthonormal basis, linearity, and the norm of the rescaled vectors."""
import numpy as np
import pytest

import oracle


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_hand_worked_product():
    # alpha = (1+2i, 3-i); B = [[1, i, 0], [2, 0, -1]]:
    #   A_0 = (1+2i)*1 + (3-i)*2 = 7;  A_1 = (1+2i)*i = -2+i;  A_2 = (3-i)*(-1) = -3+i
    alpha = np.array([[1 + 2j, 3 - 1j]])
    B = np.array([[1, 1j, 0], [2, 0, -1]], dtype=complex)
    assert np.array_equal(oracle.rb_amplitudes(alpha, B), np.array([[7, -2 + 1j, -3 + 1j]]))
    # ||A||^2 = 49 + 5 + 10 = 64, so the target norm 2 scales A by 2/8 exactly
    got = oracle.rb_amplitudes(alpha, B, norms=[2.0])
    assert np.array_equal(got, np.array([[1.75, -0.5 + 0.25j, -0.75 + 0.25j]]))


def test_identity_basis_returns_alpha():
    rng = np.random.default_rng(1)
    alpha = _crandn(rng, 5, 17)
    assert np.array_equal(oracle.rb_amplitudes(alpha, np.eye(17, dtype=complex)), alpha)


def test_fourier_basis_matches_fft():
    # B_j,i = exp(-2 pi i j i / N): A_k is the length-N DFT of alpha_k zero-padded to N
    rng = np.random.default_rng(2)
    Nb, N = 9, 64
    alpha = _crandn(rng, 4, Nb)
    j, i = np.meshgrid(np.arange(Nb), np.arange(N), indexing="ij")
    B = np.exp(-2j * np.pi * j * i / N)
    want = np.fft.fft(alpha, n=N, axis=1)
    got = oracle.rb_amplitudes(alpha, B)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_orthonormal_basis_round_trip():
    # rows of B orthonormal (B B^H = I): projecting A back onto the basis returns alpha
    rng = np.random.default_rng(3)
    Nb, N = 12, 200
    q, _ = np.linalg.qr(_crandn(rng, N, Nb))
    B = q.T  # [Nb, N], B B^H = (Q^T)(conj Q) = conj(Q^H Q) = I
    alpha = _crandn(rng, 6, Nb)
    A = oracle.rb_amplitudes(alpha, B)
    back = A @ B.conj().T
    assert np.max(np.abs(back - alpha)) <= 1e-13 * np.max(np.abs(alpha))


def test_linear_in_alpha():
    rng = np.random.default_rng(4)
    B = _crandn(rng, 7, 31)
    a1, a2 = _crandn(rng, 3, 7), _crandn(rng, 3, 7)
    c1, c2 = 0.3 - 1.1j, 2.0 + 0.5j
    lhs = oracle.rb_amplitudes(c1 * a1 + c2 * a2, B)
    rhs = c1 * oracle.rb_amplitudes(a1, B) + c2 * oracle.rb_amplitudes(a2, B)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))


def test_renormalised_rows_have_the_target_norm_and_direction():
    rng = np.random.default_rng(5)
    B = _crandn(rng, 11, 90)
    alpha = _crandn(rng, 8, 11)
    alpha[3] = 0.0  # a zero vector stays zero
    nu = rng.uniform(0.1, 5.0, 8)
    raw = oracle.rb_amplitudes(alpha, B)
    got = oracle.rb_amplitudes(alpha, B, norms=nu)
    for k in range(8):
        if k == 3:
            assert np.all(got[k] == 0)
            continue
        assert abs(np.linalg.norm(got[k]) - nu[k]) <= 1e-14 * nu[k]
        # same direction: got = raw * (positive real factor)
        ratio = got[k] / raw[k]
        assert np.allclose(ratio, ratio[0], rtol=1e-14, atol=0)
        assert abs(ratio[0].imag) <= 1e-15 and ratio[0].real > 0


@pytest.mark.parametrize("shape", [(0, 3, 4), (1, 1, 1), (2, 1, 5), (3, 4, 1)])
def test_degenerate_shapes(shape):
    M, Nb, N = shape
    rng = np.random.default_rng(6)
    alpha, B = _crandn(rng, M, Nb), _crandn(rng, Nb, N)
    got = oracle.rb_amplitudes(alpha, B)
    assert got.shape == (M, N)
    # brute force from the definition, term by term
    for k in range(M):
        for i in range(N):
            want = sum(alpha[k, j] * B[j, i] for j in range(Nb))
            assert abs(got[k, i] - want) <= 1e-15 * max(1.0, abs(want)) * Nb
