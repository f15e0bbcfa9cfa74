"""The algorithm of the FP32 y-solve for the well-conditioned x-modes, modelled in numpy
(FP64) and checked against a direct solve of the same tridiagonal system.

For x-mode k the box solve needs (T_y + lambda_k - kappa^2) v = x with
T_y = tridiag(1, -2, 1) / h^2 and v_0 = v_N = 0 (Alg. 4, the system a sine transform along y
diagonalises).  The CUDA kernel splits each line into chunks, one per thread; a chunk's
forward and backward recursions start w points early from a zero state (the error decays
like |c*|^w, c* the fixed point of the elimination coefficient), and the first 64
coefficients of the line come from the closed form c'_j = c* (1 - c*^2j) / (1 - c*^(2j+2)).
The modes it takes are those with |c*| <= 0.825.  This model follows the same steps, so a
change of the threshold, the warm-up rule or the closed form that breaks the accuracy the
kernel relies on fails here, on the CPU."""
import math

import numpy as np
import pytest

CMAX, WMAX, EXACT = 0.825, 96, 64


def lam(k, N, h):
    return -(4.0 / h**2) * math.sin(math.pi * k / (2.0 * N)) ** 2


def first_mode(N, kappa2, h):
    for k in range(1, N):
        mu = 4.0 * math.sin(math.pi * k / (2.0 * N)) ** 2 + h * h * kappa2
        if 2.0 / ((2.0 + mu) + math.sqrt((2.0 + mu) ** 2 - 4.0)) <= CMAX:
            return k
    return N


def chunked_solve(x, N, shift, h, chunks):
    A = 1.0 / h**2
    D = -2.0 * A + shift
    cs = 2.0 * A / (D - math.sqrt(D * D - 4.0 * A * A))
    gs = cs / A
    w = min(WMAX, math.ceil(-18.42 / math.log(abs(cs))) + 1)
    q = cs ** (2.0 * np.arange(EXACT))
    cp = cs * (1.0 - q) / (1.0 - q * cs * cs)
    coef = lambda j: cp[j] if j < EXACT else cs
    inv = lambda j: cp[j] / A if j < EXACT else gs
    M = N // chunks
    buf = x.astype(float).copy()
    carry = []
    for L in range(chunks):                      # forward warm-ups read the input
        s1 = max(L * M, 1)
        y = 0.0
        for j in range(max(s1 - w, 1), s1):
            y = (buf[j] - A * y) * inv(j)
        carry.append(y)
    for L in range(chunks):
        y = carry[L]
        for j in range(max(L * M, 1), L * M + M):
            y = (buf[j] - A * y) * inv(j)
            buf[j] = y
    carry = []
    for L in range(chunks):                      # backward warm-ups read the forward results
        e = L * M + M
        v = 0.0
        for j in range(min(e - 1 + w, N - 1), e - 1, -1):
            v = buf[j] - coef(j) * v
        carry.append(v)
    out = np.zeros(N)
    for L in range(chunks):
        v = carry[L]
        for j in range(L * M + M - 1, max(L * M, 1) - 1, -1):
            v = buf[j] - coef(j) * v
            out[j] = v
    return out


def direct_solve(x, N, shift, h):
    n = N - 1
    T = (np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h**2
    v = np.zeros(N)
    v[1:] = np.linalg.solve(T + shift * np.eye(n), x[1:])
    return v


@pytest.mark.parametrize("N,kappa,chunks", [(64, 0.0, 32), (96, 1.0, 32), (256, 10.0, 32),
                                            (1024, 1.0, 32), (2048, 0.0, 64)])
def test_chunked_elimination_matches_a_direct_solve(N, kappa, chunks):
    h = 2.0 / N
    k0 = first_mode(N, kappa**2, h)
    assert 1 <= k0 < N // 8                      # most modes take the elimination
    rng = np.random.default_rng(N)
    for k in sorted({k0, (k0 + N) // 2, N - 1}):
        x = np.zeros(N)
        x[1:] = rng.standard_normal(N - 1)
        shift = lam(k, N, h) - kappa**2
        ref = direct_solve(x, N, shift, h)
        got = chunked_solve(x, N, shift, h, chunks)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-7, (k, err)               # warm-up truncation ~1e-8 at the threshold


def test_closed_form_coefficients_match_the_recursion():
    A, D = 1.0, -2.0371                          # |c*| just below the threshold
    cs = 2.0 * A / (D - math.sqrt(D * D - 4.0 * A * A))
    c = 0.0
    for j in range(1, 80):
        c = A / (D - A * c)
        q = cs ** (2 * j)
        assert abs(c - cs * (1 - q) / (1 - q * cs * cs)) < 1e-14
