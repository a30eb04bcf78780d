"""Pins of the oracle's divide and concur projections (idempotence, data
consistency, least squares by brute force, scale covariance, indexing)."""
import numpy as np
import pytest

from oracle import dft, ptycho


def _problem(seed=0, N=8, M=(20, 23), J=6):
    rng = np.random.default_rng(seed)
    O = (0.8 + 0.2 * rng.uniform(size=M)) * np.exp(1j * rng.uniform(-1, 1, size=M))
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    pos = np.stack([rng.integers(0, M[0] - N + 1, size=J),
                    rng.integers(0, M[1] - N + 1, size=J)], axis=1)
    x_true = ptycho.exit_waves(P, O, pos)
    I = np.stack([np.abs(np.fft.fft2(e)) ** 2 for e in x_true])
    return O, P, pos, I, rng


def test_divide_modulus_and_idempotence():
    O, P, pos, I, rng = _problem()
    x = rng.standard_normal((pos.shape[0], 8, 8)) + 1j * rng.standard_normal((pos.shape[0], 8, 8))
    sq = np.sqrt(I)
    y, _ = ptycho.project_D(x, sq)
    for j in range(len(pos)):
        np.testing.assert_allclose(np.abs(np.fft.fft2(y[j])), sq[j], atol=1e-10)
    y2, _ = ptycho.project_D(y, sq)
    np.testing.assert_allclose(y2, y, atol=1e-10)


def test_divide_leaves_consistent_waves():
    O, P, pos, I, _ = _problem(1)
    x = ptycho.exit_waves(P, O, pos)
    y, err = ptycho.project_D(x, np.sqrt(I))
    np.testing.assert_allclose(y, x, atol=1e-10)
    assert err < 1e-18 * I.sum() + 1e-20


def test_modulus_projection_at_zero():
    Psi = np.array([[0j, 3 + 4j]])
    out = ptycho.modulus_projection(Psi, np.array([[2.0, 10.0]]))
    np.testing.assert_allclose(out, [[2.0, 6 + 8j]])


def test_modulus_projection_is_nearest_point():
    # the projection onto {|z| = s} is the nearest point: brute force over phases
    rng = np.random.default_rng(3)
    for _ in range(20):
        z = complex(rng.standard_normal(), rng.standard_normal())
        s = float(rng.uniform(0.1, 3))
        out = ptycho.modulus_projection(np.array([z]), np.array([s]))[0]
        ph = np.linspace(0, 2 * np.pi, 20001)
        best = (s * np.exp(1j * ph))[np.argmin(np.abs(s * np.exp(1j * ph) - z))]
        assert abs(out - best) < 1e-3 * s
        assert abs(abs(out) - s) < 1e-12


def _object_lstsq(y, P, pos, M):
    N = P.shape[0]
    rows, rhs = [], []
    for j in range(len(pos)):
        for r0 in range(N):
            for r1 in range(N):
                a = np.zeros(M[0] * M[1], dtype=np.complex128)
                a[(pos[j, 0] + r0) * M[1] + pos[j, 1] + r1] = P[r0, r1]
                rows.append(a)
                rhs.append(y[j, r0, r1])
    sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    return sol.reshape(M)


def _probe_lstsq(y, O, pos, N):
    rows, rhs = [], []
    for j in range(len(pos)):
        for r0 in range(N):
            for r1 in range(N):
                a = np.zeros(N * N, dtype=np.complex128)
                a[r0 * N + r1] = O[pos[j, 0] + r0, pos[j, 1] + r1]
                rows.append(a)
                rhs.append(y[j, r0, r1])
    return np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0].reshape(N, N)


def test_concur_object_is_least_squares():
    rng = np.random.default_rng(5)
    M, N = (12, 12), 4
    pos = np.array([[0, 0], [3, 5], [8, 2], [6, 7]])
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    y = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    O = ptycho.concur_object(y, P, pos, M, alpha=0.0)
    np.testing.assert_allclose(O, _object_lstsq(y, P, pos, M), atol=1e-12)


def test_concur_probe_is_least_squares():
    rng = np.random.default_rng(6)
    M, N = (12, 12), 4
    pos = np.array([[0, 0], [3, 5], [8, 2], [6, 7], [1, 8]])
    O = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    y = rng.standard_normal((5, N, N)) + 1j * rng.standard_normal((5, N, N))
    P = ptycho.concur_probe(y, O, pos, alpha=0.0)
    np.testing.assert_allclose(P, _probe_lstsq(y, O, pos, N), atol=1e-12)


def test_concur_idempotent():
    O, P, pos, I, rng = _problem(2)
    y = rng.standard_normal((len(pos), 8, 8)) + 1j * rng.standard_normal((len(pos), 8, 8))
    prob = ptycho.Problem(I, pos, O * 0 + 1, P * 1.3, alpha=0.0)
    z1 = prob.project_C(y)
    z2 = prob.project_C(z1)
    np.testing.assert_allclose(z2, z1, atol=1e-10 * np.abs(z1).max())


def test_concur_scale_covariance():
    # P -> lam P with y fixed gives O -> O / lam, regulariser included
    O, P, pos, I, rng = _problem(3)
    y = rng.standard_normal((len(pos), 8, 8)) + 1j * rng.standard_normal((len(pos), 8, 8))
    lam = 2.0 - 1.5j
    O1 = ptycho.concur_object(y, P, pos, O.shape, alpha=1e-3)
    O2 = ptycho.concur_object(y, lam * P, pos, O.shape, alpha=1e-3)
    np.testing.assert_allclose(O2, O1 / lam, atol=1e-12)


def test_regularised_ratio_zero_guard():
    num = np.array([1 + 1j, 2.0, 0.0])
    den = np.array([1.0, 4.0, 0.0])
    out = ptycho.regularised_ratio(num, den, 0.0)
    np.testing.assert_allclose(out, [1 + 1j, 0.5, 0.0])
    out = ptycho.regularised_ratio(num, den, 0.25)
    np.testing.assert_allclose(out, [(1 + 1j) / 2.0, 2.0 / 5.0, 0.0])


def test_shift_invariance_of_indexing():
    O, P, pos, I, rng = _problem(4)
    shift = np.array([3, 5])
    O_big = np.zeros((O.shape[0] + 7, O.shape[1] + 9), dtype=np.complex128)
    O_big[3:3 + O.shape[0], 5:5 + O.shape[1]] = O
    np.testing.assert_array_equal(ptycho.exit_waves(P, O, pos),
                                  ptycho.exit_waves(P, O_big, pos + shift))
    y = ptycho.exit_waves(P, O, pos) * 1.1
    a = ptycho.concur_object(y, P, pos, O.shape, 0.0)
    b = ptycho.concur_object(y, P, pos + shift, O_big.shape, 0.0)
    np.testing.assert_array_equal(a, b[3:3 + O.shape[0], 5:5 + O.shape[1]])
