"""Companion-matrix form of the lagged Fibonacci transition (Sec. 3.1), numpy.

Test infrastructure only (see the package docstring).  Independent of the C
polynomial code: it builds the matrix A exactly as printed in Sec. 3.1 and
multiplies integer matrices modulo 2^24 in int64 (entries < 2^24, so each
97-term dot product stays below 2^55).
"""
from __future__ import annotations

import numpy as np

R = 97
S = 33
MOD = 1 << 24


def companion() -> np.ndarray:
    """A = [[0 ... 0 a_0], [I_{r-1} | (a_1..a_{r-1})^T]] with a_0 = 1,
    a_{r-s} = -1 and all other a_i = 0 (Sec. 3.1)."""
    a = np.zeros(R, np.int64)
    a[0] = 1
    a[R - S] = MOD - 1          # -1 mod 2^24
    A = np.zeros((R, R), np.int64)
    A[:, R - 1] = a
    A[1:, : R - 1] = np.eye(R - 1, dtype=np.int64)
    return A


def matmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    return (X @ Y) % MOD


def matpow(A: np.ndarray, J: int) -> np.ndarray:
    """A^J by repeated multiplication (small J only: the plain definition)."""
    P = np.eye(R, dtype=np.int64)
    for _ in range(J):
        P = matmul(P, A)
    return P


def poly_of_matrix(b: np.ndarray, A: np.ndarray) -> np.ndarray:
    """P(A) = sum_i b_i A^i."""
    acc = np.zeros((R, R), np.int64)
    Ai = np.eye(R, dtype=np.int64)
    for i in range(R):
        acc = (acc + int(b[i]) * Ai) % MOD
        Ai = matmul(Ai, A)
    return acc


def row_times(u: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Row vector u (sequence order) times M, mod 2^24: F1(u) = uA."""
    return (np.asarray(u, np.int64) @ M) % MOD


def char_poly_check(A: np.ndarray) -> np.ndarray:
    """phi(A) = A^97 + A^64 - I, which Cayley-Hamilton says is zero."""
    A64 = matpow(A, 64)
    A97 = matmul(A64, matpow(A, 33))
    return (A97 + A64 - np.eye(R, dtype=np.int64)) % MOD
