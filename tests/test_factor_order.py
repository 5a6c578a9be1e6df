"""The column-parallel warp Cholesky of the device code (lane l holds the
lower-triangle elements l and l + 32; after column k every element (i, j),
j > k, takes -L[i][k] L[j][k] with the factors fetched from their lanes)
applies to every element the same fused multiply-adds in the same order as
the row-by-row algorithm, then the same square root or division, so both
give the same bits.  Checked here on the schedule itself, in float32 with
a correctly rounded fused multiply-add, for every DoF up to the limit."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def fma(a, b, c):
    """float32 fma: the exact a*b + c, rounded once."""
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    return F32(float(exact)) if abs(float(exact)) < 1e30 else F32(float(a) * float(b) + float(c))


def rowwise(d, S):
    L = np.zeros((d, d), F32)
    for i in range(d):
        for j in range(i + 1):
            s = F32(S[i, j])
            if i == j:
                s = F32(s + F32(1e-8))
            for k in range(j):
                s = fma(-L[i, k], L[j, k], s)
            L[i, j] = F32(np.sqrt(max(s, F32(1e-12)))) if i == j else F32(s / L[j, j])
    return L


def warp_schedule(d, S):
    nel = d * (d + 1) // 2
    own = {}                       # element index -> (i, j)
    v = {}
    for e in range(64):
        i = 0
        while (i + 1) * (i + 2) // 2 <= e:
            i += 1
        own[e] = (i, e - i * (i + 1) // 2)
        if e < nel:
            i, j = own[e]
            v[e] = F32(S[i, j])
            if i == j:
                v[e] = F32(v[e] + F32(1e-8))
    idx = lambda i, j: i * (i + 1) // 2 + j
    for k in range(d):
        v[idx(k, k)] = F32(np.sqrt(max(v[idx(k, k)], F32(1e-12))))
        lkk = v[idx(k, k)]
        for e in range(nel):
            i, j = own[e]
            if j == k and i > k:
                v[e] = F32(v[e] / lkk)
        snap = dict(v)             # column k is final; the trailing updates read it
        for e in range(nel):
            i, j = own[e]
            if j > k:
                v[e] = fma(-snap[idx(i, k)], snap[idx(j, k)], v[e])
    L = np.zeros((d, d), F32)
    for e in range(nel):
        L[own[e]] = v[e]
    return L


def test_warp_and_row_orders_give_the_same_bits():
    rng = np.random.default_rng(7)
    for d in range(1, 10):
        for t in range(6):
            A = rng.normal(size=(d, d))
            S = (A @ A.T + 0.05 * np.eye(d)).astype(F32)
            if t == 0:
                S = np.zeros((d, d), F32)          # every pivot floored
            if t == 1:
                S = (0.09 * np.eye(d)).astype(F32)  # the restart covariance sigma^2 I
            a, b = rowwise(d, S), warp_schedule(d, S)
            assert np.array_equal(a, b), (d, t)
            if t == 1:   # its factor is the diagonal the Shift writes for the restart slot
                x = F32(F32(0.09) + F32(1e-8))
                assert np.array_equal(a, np.diag(np.full(d, F32(np.sqrt(x)), F32))), d
