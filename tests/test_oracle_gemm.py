"""Pins of the FP64 oracle GEMM against results fixed by mathematics.

The oracle computes C = alpha*A*B + beta*C (paper, Section 2).  Each test below
checks it against something other than itself: closed forms (identity,
permutation, all-ones, rank-1 integer outer products), a product worked out by
hand, and exact rational arithmetic on small random inputs (the oracle must lie
within FP64's summation error bound of the exact result).  A dropped term, a
wrong sign, a transposed operand or a swapped stride fails at least one.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_hand_worked_product():
    # [[1, 2, 3], [4, 5, 6]] @ [[7, 8], [9, 10], [11, 12]], worked by hand:
    # row 0: 1*7 + 2*9 + 3*11 = 58,  1*8 + 2*10 + 3*12 = 64
    # row 1: 4*7 + 5*9 + 6*11 = 139, 4*8 + 5*10 + 6*12 = 154
    A = np.array([[1, 2, 3], [4, 5, 6]], np.float64)
    B = np.array([[7, 8], [9, 10], [11, 12]], np.float64)
    C, absC = oracle.gemm(A, B)
    assert C.tolist() == [[58, 64], [139, 154]]
    assert absC.tolist() == [[58, 64], [139, 154]]
    # sign flips change C but not |A||B|
    C2, abs2 = oracle.gemm(-A, B)
    assert C2.tolist() == [[-58, -64], [-139, -154]]
    assert abs2.tolist() == absC.tolist()


def test_alpha_beta_closed_form():
    # A = ones(2x4), B = ones(4x3): A@B = 4 everywhere; C_in = [[1,2,3],[4,5,6]].
    A = np.ones((2, 4))
    B = np.ones((4, 3))
    Cin = np.array([[1, 2, 3], [4, 5, 6]], np.float64)
    C, _ = oracle.gemm(A, B, alpha=2.0, beta=0.5, C_in=Cin)
    assert C.tolist() == [[8.5, 9.0, 9.5], [10.0, 10.5, 11.0]]
    C, _ = oracle.gemm(A, B, alpha=-1.0, beta=0.0, C_in=None)
    assert (C == -4).all()
    C, _ = oracle.gemm(A, B, alpha=0.0, beta=1.0, C_in=Cin)
    assert (C == Cin).all()


@pytest.mark.parametrize("m,n,k", [(7, 5, 3), (16, 33, 1), (1, 1, 100), (40, 24, 48)])
def test_identity_and_permutation(m, n, k):
    r = rng(m * 1000 + n * 10 + k)
    B = r.integers(-50, 50, size=(k, n)).astype(np.float64)
    # identity-like A (m x k with ones on the diagonal): C = first rows of B
    A = np.eye(m, k)
    C, _ = oracle.gemm(A, B)
    want = np.zeros((m, n))
    d = min(m, k)
    want[:d] = B[:d]
    assert (C == want).all()
    # permutation A (k x k): row i of C is row perm[i] of B
    perm = r.permutation(k)
    P = np.zeros((k, k))
    P[np.arange(k), perm] = 1.0
    C, _ = oracle.gemm(P, B)
    assert (C == B[perm]).all()
    # permutation on the right: column j of C is column perm2[j] of A
    A2 = r.integers(-9, 9, size=(m, k)).astype(np.float64)
    perm2 = r.permutation(k)
    Q = np.zeros((k, k))
    Q[perm2, np.arange(k)] = 1.0
    C, _ = oracle.gemm(A2, Q)
    assert (C == A2[:, perm2]).all()


@pytest.mark.parametrize("k", [1, 17, 4096, 65536])
def test_all_ones_gives_k(k):
    C, absC = oracle.gemm(np.ones((3, k)), np.ones((k, 2)))
    assert (C == k).all() and (absC == k).all()


def test_rank1_integer_outer_product():
    # A = u e^T-like: every column of A is u, every row of B is v / k-scaled so
    # that (A B)_ij = k * u_i * v_j exactly.
    r = rng(7)
    m, n, k = 12, 9, 31
    u = r.integers(-20, 21, size=m).astype(np.float64)
    v = r.integers(-20, 21, size=n).astype(np.float64)
    A = np.repeat(u[:, None], k, axis=1)
    B = np.repeat(v[None, :], k, axis=0)
    C, absC = oracle.gemm(A, B)
    assert (C == k * np.outer(u, v)).all()
    assert (absC == k * np.outer(np.abs(u), np.abs(v))).all()


def test_non_square_orientation():
    # A (2x3) with distinct entries and B (3x4) with distinct entries: a
    # transposed or mis-strided operand would give a different product shape or
    # values.  Expected values computed by exact integer arithmetic in Python.
    A = np.array([[1, -2, 3], [0, 4, -1]], np.float64)
    B = np.array([[2, 0, 1, -3], [1, 5, -2, 0], [4, -1, 0, 2]], np.float64)
    want = [[sum(int(A[i, l]) * int(B[l, j]) for l in range(3)) for j in range(4)]
            for i in range(2)]
    C, _ = oracle.gemm(A, B)
    assert C.shape == (2, 4)
    assert C.tolist() == want


def test_storage_orders_agree():
    # The same logical matrices stored row-major, column-major and as strided
    # views must give identical results (the oracle reads through strides).
    r = rng(11)
    A = r.standard_normal((13, 21))
    B = r.standard_normal((21, 6))
    C_ref, abs_ref = oracle.gemm(A, B)
    A_cm = np.asfortranarray(A)
    B_cm = np.asfortranarray(B)
    C1, a1 = oracle.gemm(A_cm, B_cm)
    assert (C1 == C_ref).all() and (a1 == abs_ref).all()
    big = r.standard_normal((40, 50))
    big[:13:1, :21] = A
    C2, _ = oracle.gemm(big[:13, :21], B)
    assert (C2 == C_ref).all()
    Bt = np.ascontiguousarray(B.T)        # B given as the transpose view of an n x k array
    C3, _ = oracle.gemm(A, Bt.T)
    assert (C3 == C_ref).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_rational_brute_force(seed):
    """Against exact arithmetic: inputs are random bf16-like dyadic values;
    Fractions give the exact sum; the oracle must be within the FP64
    summation bound k * 2^-53 * sum |a||b| (+ one rounding of alpha, beta)."""
    r = rng(seed)
    m, n, k = 5, 4, 37
    A = np.round(r.standard_normal((m, k)) * 256) / 256
    B = np.round(r.standard_normal((k, n)) * 128) / 128
    Cin = np.round(r.standard_normal((m, n)) * 64) / 64
    alpha, beta = 1.5, -0.75
    C, absC = oracle.gemm(A, B, alpha=alpha, beta=beta, C_in=Cin)
    for i in range(m):
        for j in range(n):
            exact = Fraction(alpha) * sum(Fraction(A[i, l]) * Fraction(B[l, j]) for l in range(k))
            exact += Fraction(beta) * Fraction(Cin[i, j])
            mag = sum(abs(Fraction(A[i, l]) * Fraction(B[l, j])) for l in range(k))
            bound = (k + 2) * 2.0 ** -53 * (abs(alpha) * float(mag) + abs(beta * Cin[i, j]))
            assert abs(Fraction(C[i, j]) - exact) <= Fraction(bound)
            assert absC[i, j] == pytest.approx(float(mag), rel=k * 2.0 ** -52)


def test_entries_match_full_product():
    r = rng(5)
    A = r.standard_normal((30, 70))
    B = r.standard_normal((70, 20))
    Cin = r.standard_normal((30, 20))
    C, absC = oracle.gemm(A, B, alpha=0.5, beta=2.0, C_in=Cin)
    rows = r.integers(0, 30, size=50)
    cols = r.integers(0, 20, size=50)
    e, ea = oracle.gemm_entries(rows, cols, A, B, alpha=0.5, beta=2.0, C_in=Cin)
    assert (e == C[rows, cols]).all() and (ea == absC[rows, cols]).all()


def test_input_validation():
    with pytest.raises(ValueError):
        oracle.gemm(np.ones((2, 3)), np.ones((4, 2)))
    with pytest.raises(TypeError):
        oracle.gemm(np.ones((2, 3), np.float32), np.ones((3, 2)))
    with pytest.raises(IndexError):
        oracle.gemm_entries([5], [0], np.ones((2, 3)), np.ones((3, 2)))


def test_empty_shapes():
    C, absC = oracle.gemm(np.ones((3, 0)), np.ones((0, 4)))
    assert (C == 0).all() and (absC == 0).all()
    C, _ = oracle.gemm(np.ones((0, 5)), np.ones((5, 4)))
    assert C.shape == (0, 4)
