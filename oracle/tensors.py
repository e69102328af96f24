"""Cartesian tensor machinery of the FP64 CPU oracle (test infrastructure only).

Nothing in the product path may import this module; it exists so that the
tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline can check the
CUDA path against a plain restatement of the paper.

Contents, each written from the definition it cites:

* STF projector Delta^(k): the orthogonal projector onto symmetric, traceless
  rank-k tensors (Sec. III, text after Eq. tensorial_spherical_harmonics_orthogonality).
  Built numerically: symmetriser, then the null space of the pair trace.
* Tensorial spherical harmonics Y^(l)(n) = (-1)^l r^(l+1) grad^(l) (1/r)
  (Sec. III, Eq. tensorial_spherical_harmonics_definition), evaluated as
  (2l-1)!! Delta^(l) n^l.
* The real orthonormal STF basis U^(k)_mu (mu = -k..k) that fixes the packed
  layout of every irreducible coefficient: U_mu . n^k = N_k Y^real_{k mu}(n),
  N_k^2 = 4 pi k!/(2k+1)!!, with real spherical harmonics without the
  Condon-Shortley phase (cos(mu phi) for mu > 0, sin(|mu| phi) for mu < 0).
  Obtained by least squares on sample directions.
* The irreducible (l sigma) embeddings of Sec. III, Eq. irred_velocity_coefficients:
  V^(L) = Delta V^(L0) - (L-1)/L Delta(eps . V^(L1)) + L(L-1)/(2(2L-1)) Delta(delta V^(L2)).
* The mode table (1s, 2a | 2s, 3t, 3a, 3s, 4t, 4a, 4s, 5t) and truncations.
"""
import itertools
import math

import numpy as np


def dfact(n):
    """Double factorial with (-1)!! = 0!! = 1."""
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


# ----------------------------------------------------------------------------
# full-tensor helpers (rank-k tensors as arrays of shape (3,)*k)
# ----------------------------------------------------------------------------

def _perm_matrix(k, perm):
    """Matrix that permutes the k indices of a flattened rank-k tensor."""
    n = 3 ** k
    M = np.zeros((n, n))
    for idx in itertools.product(range(3), repeat=k):
        src = np.ravel_multi_index(idx, (3,) * k)
        dst = np.ravel_multi_index(tuple(idx[p] for p in perm), (3,) * k)
        M[dst, src] = 1.0
    return M


_STF_CACHE = {}


def stf_projector(k):
    """Orthogonal projector (3^k x 3^k) onto symmetric traceless rank-k tensors."""
    if k in _STF_CACHE:
        return _STF_CACHE[k]
    if k == 0:
        P = np.ones((1, 1))
    elif k == 1:
        P = np.eye(3)
    else:
        perms = list(itertools.permutations(range(k)))
        S = sum(_perm_matrix(k, p) for p in perms) / len(perms)
        w, V = np.linalg.eigh(S)
        B = V[:, w > 0.5]                       # orthonormal basis of symmetric tensors
        # trace over the first two indices (enough for symmetric tensors)
        Tr = np.zeros((3 ** (k - 2), 3 ** k))
        for rest in itertools.product(range(3), repeat=k - 2):
            r = np.ravel_multi_index(rest, (3,) * (k - 2)) if k > 2 else 0
            for i in range(3):
                Tr[r, np.ravel_multi_index((i, i) + rest, (3,) * k)] = 1.0
        M = Tr @ B
        _, s, Vt = np.linalg.svd(M)
        rank = int(np.sum(s > 1e-10))
        C = Vt[rank:].T                          # null space coefficients
        basis = B @ C
        q, _ = np.linalg.qr(basis)
        P = q @ q.T
        assert q.shape[1] == 2 * k + 1
    _STF_CACHE[k] = P
    return P


def outer_power(n, k):
    """n^{(x)k} as a flat vector of length 3^k."""
    t = np.ones(1)
    for _ in range(k):
        t = np.kron(t, n)
    return t


def tsh(l, n):
    """Tensorial spherical harmonic Y^(l)(n) as a rank-l array, |n| = 1.

    Y^(l) = (-1)^l r^(l+1) grad^(l)(1/r) = (2l-1)!! Delta^(l) n^l.
    """
    flat = dfact(2 * l - 1) * (stf_projector(l) @ outer_power(np.asarray(n, float), l))
    return flat.reshape((3,) * l) if l > 0 else flat[0]


# ----------------------------------------------------------------------------
# real spherical harmonics and the packed STF basis
# ----------------------------------------------------------------------------

def _assoc_legendre_noCS(k, m, x):
    """P_k^m(x) = (1-x^2)^{m/2} d^m/dx^m P_k(x) (no Condon-Shortley phase)."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    Pk = np.polynomial.legendre.Legendre(c).convert(kind=np.polynomial.Polynomial)
    d = Pk.deriv(m) if m > 0 else Pk
    return (1.0 - x * x) ** (m / 2.0) * d(x)


def real_sh(k, mu, n):
    """Orthonormal real spherical harmonic Y_{k mu} at unit vectors n (..., 3)."""
    n = np.asarray(n, float)
    x, y, z = n[..., 0], n[..., 1], n[..., 2]
    phi = np.arctan2(y, x)
    m = abs(mu)
    norm = math.sqrt((2 * k + 1) / (4 * math.pi) * math.factorial(k - m) / math.factorial(k + m))
    P = _assoc_legendre_noCS(k, m, z)
    if mu == 0:
        return norm * P
    if mu > 0:
        return math.sqrt(2.0) * norm * P * np.cos(m * phi)
    return math.sqrt(2.0) * norm * P * np.sin(m * phi)


_U_CACHE = {}


def stf_basis(k):
    """Packed STF basis: array (2k+1, 3,...,3); row j is U^(k)_mu with mu = j - k.

    Defined by U_mu . n^k = N_k Y_{k mu}(n), N_k^2 = 4 pi k!/(2k+1)!!, which makes the
    rows orthonormal in the full contraction (Frobenius) inner product.
    """
    if k in _U_CACHE:
        return _U_CACHE[k]
    P = stf_projector(k)
    w, V = np.linalg.eigh(P)
    B = V[:, w > 0.5]                                   # 3^k x (2k+1)
    rng = np.random.default_rng(12345)
    pts = rng.normal(size=(400, 3))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    Nk = math.sqrt(4 * math.pi * math.factorial(k) / dfact(2 * k + 1))
    X = np.stack([outer_power(p, k) for p in pts]) @ B   # values of basis polys
    U = np.zeros((2 * k + 1, 3 ** k))
    for j, mu in enumerate(range(-k, k + 1)):
        target = Nk * real_sh(k, mu, pts)
        c, *_ = np.linalg.lstsq(X, target, rcond=None)
        assert np.max(np.abs(X @ c - target)) < 1e-10
        U[j] = B @ c
    U[np.abs(U) < 1e-13] = 0.0
    U = U.reshape((2 * k + 1,) + (3,) * k)
    _U_CACHE[k] = U
    return U


def pack_stf(T):
    """Packed coordinates (2k+1,) of an STF rank-k tensor T (Cartesian array)."""
    T = np.asarray(T, float)
    k = T.ndim
    U = stf_basis(k)
    return np.tensordot(U, T, axes=k) if k > 0 else np.array([float(T)])


def unpack_stf(y, k):
    """Cartesian STF rank-k tensor from packed coordinates y (2k+1,)."""
    U = stf_basis(k)
    return np.tensordot(np.asarray(y, float), U, axes=1)


# ----------------------------------------------------------------------------
# irreducible (l sigma) embeddings and the mode table
# ----------------------------------------------------------------------------

LEVI = np.zeros((3, 3, 3))
for (i, j, k), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                     (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
    LEVI[i, j, k] = s


def _project_tail(X):
    """Apply Delta^(L-1) to the last L-1 indices of the rank-L array X."""
    L = X.ndim
    if L <= 2:
        return X
    P = stf_projector(L - 1)
    flat = X.reshape(3, 3 ** (L - 1)) @ P.T
    return flat.reshape(X.shape)


def embed(L, sigma, T):
    """Reducible rank-L coefficient from its sigma part T (Eq. irred_velocity_coefficients).

    sigma = 0: T is STF of rank L;       term  Delta^(L) T
    sigma = 1: T is STF of rank L-1;     term -(L-1)/L Delta^(L-1)[eps_{i a1 g} T_{g a2..}]
    sigma = 2: T is STF of rank L-2;     term  L(L-1)/(2(2L-1)) Delta^(L-1)[delta_{i a1} T_{a2..}]
    """
    T = np.asarray(T, float)
    if sigma == 0:
        return T.copy()
    if sigma == 1:
        X = np.tensordot(LEVI, T, axes=([2], [0]))      # (i, a1, a2..)
        return -(L - 1) / L * _project_tail(X)
    if sigma == 2:
        X = np.multiply.outer(np.eye(3), T) if T.ndim > 0 else np.eye(3) * float(T)
        return L * (L - 1) / (2 * (2 * L - 1)) * _project_tail(X)
    raise ValueError(sigma)


# (name, L = rank of the reducible coefficient, sigma); irreducible rank k = L - sigma.
MODES = [("1s", 1, 0), ("2a", 2, 1),
         ("2s", 2, 0), ("3t", 3, 2),
         ("3a", 3, 1), ("3s", 3, 0), ("4t", 4, 2),
         ("4a", 4, 1), ("4s", 4, 0), ("5t", 5, 2),
         ("5a", 5, 1), ("5s", 5, 0), ("6t", 6, 2),
         ("6a", 6, 1), ("6s", 6, 0), ("7t", 7, 2)]
# truncation l<=L keeps MODES[2 : 2 + N_HMODES[L]] as higher modes: the nested sets
# {1s, 2a} + {ks, ka, (k+1)t : 2 <= k <= L}.  MINIMAL (code 40) is the paper's minimal
# truncation of Sec. IV: every mode of rank <= 4 (Y^(0..3)), 47 components per sphere
# (l <= 4 without 5t).
MINIMAL = 40
N_HMODES = {2: 2, 3: 5, 4: 8, 5: 11, 6: 14, MINIMAL: 7}


def modes_for(trunc):
    """(L modes, H modes) lists of (name, L, sigma) for truncation l <= trunc (or MINIMAL)."""
    return MODES[:2], MODES[2:2 + N_HMODES[trunc]]


def mode_dim(m):
    return 2 * (m[1] - m[2]) + 1


def h_of(trunc):
    return sum(mode_dim(m) for m in modes_for(trunc)[1])


class ModeBasis:
    """Orthonormal basis e_p of the embedded mode spaces for one truncation.

    For every mode (L, sigma) and every packed component mu, e = E_sigma(U_mu)/c with
    c = |E_sigma(U_mu)| (the same for all mu).  Internal coordinates x = c * y, where y
    are the packed coordinates of the paper's irreducible tensor V^(L sigma) / F^(L sigma).
    """

    def __init__(self, trunc):
        self.trunc = trunc
        self.lmodes, self.hmodes = modes_for(trunc)
        self.modes = self.lmodes + self.hmodes
        self.vectors = []      # list of (mode index, L, sigma, full tensor e)
        self.scale = []        # c per component
        self.mode_of = []
        for mi, (name, L, sigma) in enumerate(self.modes):
            k = L - sigma
            U = stf_basis(k)
            for mu in range(2 * k + 1):
                E = embed(L, sigma, U[mu])
                c = np.sqrt(np.sum(E * E))
                self.vectors.append(E / c)
                self.scale.append(c)
                self.mode_of.append(mi)
        self.scale = np.array(self.scale)
        self.mode_of = np.array(self.mode_of)
        self.rank = np.array([self.modes[m][1] for m in self.mode_of])
        self.d = len(self.vectors)
        self.nL = sum(mode_dim(m) for m in self.lmodes)
        self.h = self.d - self.nL
