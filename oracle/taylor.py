"""Truncated three-variable Taylor arithmetic for the oracle (test infrastructure only).

The pair matrix elements of Sec. III (Eq. single_layer_yl_matrix_element) are
derivatives of the Stokes Green's function, G_ij = (delta_ij lap - d_i d_j) r
(Sec. III, Green's function equations), so every entry is a Cartesian
derivative of r or of 1/r.  The oracle obtains all of them at once by
expanding f(rho + h) = |rho + h|^nu as a polynomial in h:

    |rho + h|^nu = r^nu (1 + u)^(nu/2),  u = (2 rho.h + h.h) / r^2,

and summing the binomial series in u.  Because u has no constant term, the
series truncated at total degree K in h is exact up to that degree; the
derivative d^n f(rho) is n1! n2! n3! times the coefficient of h^n.
"""
import math
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def monomials(K):
    """All exponent triples with total degree <= K, graded order."""
    out = []
    for d in range(K + 1):
        for a in range(d, -1, -1):
            for b in range(d - a, -1, -1):
                out.append((a, b, d - a - b))
    return tuple(out)


@lru_cache(maxsize=None)
def mono_index(K):
    return {m: i for i, m in enumerate(monomials(K))}


@lru_cache(maxsize=None)
def _mul_table(K):
    """Index triples (ia, ib, ic) with mono[ia] + mono[ib] = mono[ic], degree <= K."""
    mons = monomials(K)
    idx = mono_index(K)
    ia, ib, ic = [], [], []
    for i, a in enumerate(mons):
        for j, b in enumerate(mons):
            c = (a[0] + b[0], a[1] + b[1], a[2] + b[2])
            if sum(c) <= K:
                ia.append(i)
                ib.append(j)
                ic.append(idx[c])
    return np.array(ia), np.array(ib), np.array(ic)


def mul(A, B, K):
    """Truncated product of polynomial batches A, B of shape (P, nmono(K))."""
    ia, ib, ic = _mul_table(K)
    prod = A[:, ia] * B[:, ib]
    return np.asarray(prod @ _scatter(K))


@lru_cache(maxsize=None)
def _scatter(K):
    """Sparse 0/1 matrix that sums product terms into their output monomial."""
    import scipy.sparse as sp
    ia, ib, ic = _mul_table(K)
    n = len(monomials(K))
    return sp.csr_matrix((np.ones(len(ic)), (np.arange(len(ic)), ic)), shape=(len(ic), n))


def derivatives(rho, nu, K):
    """All derivatives d^n |x|^nu at x = rho, |n| <= K.

    rho: (P, 3).  Returns (P, nmono(K)) in the order of ``monomials(K)``.
    """
    rho = np.atleast_2d(np.asarray(rho, float))
    P = rho.shape[0]
    mons = monomials(K)
    idx = mono_index(K)
    nm = len(mons)
    r2 = np.sum(rho * rho, axis=1)
    u = np.zeros((P, nm))
    for i in range(3):
        e = [0, 0, 0]
        e[i] = 1
        u[:, idx[tuple(e)]] = 2.0 * rho[:, i] / r2
        e[i] = 2
        u[:, idx[tuple(e)]] = 1.0 / r2
    series = np.zeros((P, nm))
    series[:, 0] = 1.0
    upow = np.zeros((P, nm))
    upow[:, 0] = 1.0
    binom = 1.0
    for k in range(1, K + 1):
        upow = mul(upow, u, K)
        binom *= (nu / 2.0 - (k - 1)) / k
        series += binom * upow
    fact = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) for a, b, c in mons])
    return series * (r2 ** (nu / 2.0))[:, None] * fact[None, :]
