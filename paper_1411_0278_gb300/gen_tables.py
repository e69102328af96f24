"""Build step: derive the pair-frame Galerkin tables and emit ``csrc/gbi_generated.cuh``.

The CUDA pair kernels evaluate every single-layer pair block
    G_nm^(l+1,l'+1) = a^(l+l') F_n^l F_m^l' grad_n^(l) grad_m^(l') G(R_n - R_m)
(Sec. III, Eq. single_layer_yl_matrix_element) in the frame in which
R_n - R_m points along +z.  There the block only couples mode components with
the same |mu| and reduces to constants times (a/r)^(l+l'+1) [alpha + beta (a/r)^2];
this script derives those constants exactly (rational arithmetic), together with

* the packed basis U^(k)_mu of symmetric traceless (STF) tensors, defined by
  U_mu . x^k = N_k r^k Y_{k mu}(x) with orthonormal real spherical harmonics
  (no Condon-Shortley phase, cos for mu > 0, sin for mu < 0), N_k^2 = 4 pi k!/(2k+1)!!;
* the (l sigma) embeddings of Sec. III, Eq. irred_velocity_coefficients
  (coefficients 1, -(L-1)/L, L(L-1)/(2(2L-1))), as vectors of harmonic polynomials;
* the rotation matrices of the packed basis about y (polynomials in cos, sin);
* the one-body self scalars g (Sec. III, same equation, m = n): the sphere
  average of Y^(l) (I - nn) Y^(l), integrated exactly over monomials.

Only the Python standard library is used (the GPU host has no sympy), so the
script runs on both build machines and its output is deterministic.
"""
import math
import os
import sys
from fractions import Fraction as Fr

# ----------------------------------------------------------------------------
# homogeneous polynomials in (x, y, z): dict {(a, b, c): coefficient}
# ----------------------------------------------------------------------------


def padd(*ps):
    out = {}
    for p in ps:
        for k, v in p.items():
            out[k] = out.get(k, 0) + v
    return {k: v for k, v in out.items() if v != 0}


def pscale(p, s):
    return {k: v * s for k, v in p.items() if v * s != 0}


def pmul(p, q):
    out = {}
    for k1, v1 in p.items():
        for k2, v2 in q.items():
            k = (k1[0] + k2[0], k1[1] + k2[1], k1[2] + k2[2])
            out[k] = out.get(k, 0) + v1 * v2
    return {k: v for k, v in out.items() if v != 0}


def pderiv(p, i):
    out = {}
    for k, v in p.items():
        if k[i] > 0:
            kk = list(k)
            kk[i] -= 1
            out[tuple(kk)] = out.get(tuple(kk), 0) + v * k[i]
    return {k: v for k, v in out.items() if v != 0}


def plap(p):
    return padd(*[pderiv(pderiv(p, i), i) for i in range(3)])


X = {(1, 0, 0): Fr(1)}
Y = {(0, 1, 0): Fr(1)}
Z = {(0, 0, 1): Fr(1)}
R2 = {(2, 0, 0): Fr(1), (0, 2, 0): Fr(1), (0, 0, 2): Fr(1)}
ONE = {(0, 0, 0): Fr(1)}
AXES = (X, Y, Z)


def ppow(p, n):
    out = ONE
    for _ in range(n):
        out = pmul(out, p)
    return out


def dfact(n):
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def frob(p, q, k):
    """Full-contraction inner product of the symmetric rank-k tensors of p and q."""
    s = 0
    for key, v in p.items():
        w = q.get(key)
        if w is not None:
            s += v * w * Fr(math.factorial(key[0]) * math.factorial(key[1]) * math.factorial(key[2]),
                            math.factorial(k))
    return s


def harmonic_part(p, d):
    """STF projection of a degree-d polynomial: sum_j (-1)^j (2d-2j-1)!!/((2d-1)!!(2j)!!) r^2j lap^j p."""
    out = {}
    term = p
    j = 0
    while term:
        coef = Fr((-1) ** j * dfact(2 * d - 2 * j - 1), dfact(2 * d - 1) * dfact(2 * j))
        out = padd(out, pscale(pmul(ppow(R2, j), term), coef))
        term = plap(term)
        j += 1
    return out


# ----------------------------------------------------------------------------
# packed STF basis: U_mu . x^k = nrm2 * S_{k mu}(x),  S with rational coefficients
# ----------------------------------------------------------------------------

def legendre_deriv_coeffs(k, m):
    """Coefficients c_j of d^m/dt^m P_k(t) = sum_j c_j t^(k-m-2j) (exact)."""
    # P_k(t) = 2^-k sum_j (-1)^j C(k,j) C(2k-2j,k) t^(k-2j)
    out = {}
    for j in range(k // 2 + 1):
        c = Fr((-1) ** j * math.comb(k, j) * math.comb(2 * k - 2 * j, k), 2 ** k)
        e = k - 2 * j
        if e >= m:
            out[e - m] = out.get(e - m, 0) + c * Fr(math.factorial(e), math.factorial(e - m))
    return out


def solid_harmonic(k, mu):
    """(unnormalised S, squared normalisation) with U_mu . x^k = sqrt(nrm2) S(x)."""
    m = abs(mu)
    # r^(k-m) (d^m P_k)(z/r) = sum_e c_e z^e r^(k-m-e)
    leg = {}
    for e, c in legendre_deriv_coeffs(k, m).items():
        leg = padd(leg, pscale(pmul(ppow(Z, e), ppow(R2, (k - m - e) // 2)), c))
    # (x + i y)^m: real part (mu >= 0) or imaginary part (mu < 0)
    cplx = {}
    for j in range(m + 1):
        c = math.comb(m, j)
        # i^j: j % 4 -> 1, i, -1, -i
        ph = j % 4
        if (mu >= 0 and ph in (0, 2)) or (mu < 0 and ph in (1, 3)):
            sgn = 1 if ph in (0, 1) else -1
            cplx = padd(cplx, pscale(pmul(ppow(X, m - j), ppow(Y, j)), Fr(sgn * c)))
    S = pmul(leg, cplx)
    # N_k^2 * (2k+1)/(4pi) (k-m)!/(k+m)! * (2 if m > 0)
    nrm2 = Fr(math.factorial(k) * (2 * k + 1) * math.factorial(k - m),
              dfact(2 * k + 1) * math.factorial(k + m)) * (2 if m > 0 else 1)
    return S, nrm2


# ----------------------------------------------------------------------------
# modes
# ----------------------------------------------------------------------------

MODES = [("1s", 1, 0), ("2a", 2, 1), ("2s", 2, 0), ("3t", 3, 2), ("3a", 3, 1), ("3s", 3, 0),
         ("4t", 4, 2), ("4a", 4, 1), ("4s", 4, 0), ("5t", 5, 2), ("5a", 5, 1), ("5s", 5, 0), ("6t", 6, 2)]
# truncation l <= L keeps the first NMODES[L] modes; code 40 is the paper's minimal
# truncation of Sec. IV (every mode of rank <= 4, 47 components: l <= 4 without 5t)
MINIMAL = 40
NMODES = {2: 4, 3: 7, 4: 10, 5: 13, MINIMAL: 9}
TRUNCS = (2, 3, 4, 5, MINIMAL)


class Comp:
    """One packed component: embedded tensor as 3 tail polynomials (exact) + norm^2."""

    def __init__(self, mode, mi, mu):
        name, L, sigma = mode
        k = L - sigma
        S, nrm2 = solid_harmonic(k, mu)
        self.name, self.L, self.sigma, self.k, self.mu, self.mode = name, L, sigma, k, mu, mi
        # tail polynomials of the unnormalised S, times sqrt(nrm2) implicitly
        if sigma == 0:
            tails = [pscale(pderiv(S, i), Fr(1, k)) for i in range(3)]
        elif sigma == 1:
            u = [pscale(pderiv(S, g), Fr(1, k)) for g in range(3)]
            # (x cross u)_i, already harmonic; coefficient -(L-1)/L
            cr = [padd(pmul(Y, u[2]), pscale(pmul(Z, u[1]), -1)),
                  padd(pmul(Z, u[0]), pscale(pmul(X, u[2]), -1)),
                  padd(pmul(X, u[1]), pscale(pmul(Y, u[0]), -1))]
            tails = [pscale(c, Fr(-(L - 1), L)) for c in cr]
        else:
            tails = [pscale(harmonic_part(pmul(AXES[i], S), L - 1), Fr(L * (L - 1), 2 * (2 * L - 1)))
                     for i in range(3)]
        self.tails = tails
        self.nrm2_basis = nrm2
        # |E(U)|^2 = nrm2 * sum_i frob(tail_i, tail_i)
        self.emb2 = nrm2 * sum(frob(t, t, L - 1) for t in tails)
        self.full = padd(*[pmul(AXES[i], tails[i]) for i in range(3)])   # P_E(x), degree L

    @property
    def scale(self):
        """c = |E_sigma(U_mu)|: internal coordinate x = c * packed y."""
        return math.sqrt(self.emb2)


def components(trunc):
    out = []
    for mi, mode in enumerate(MODES[:NMODES[trunc]]):
        k = mode[1] - mode[2]
        for mu in range(-k, k + 1):
            out.append(Comp(mode, mi, mu))
    return out


# ----------------------------------------------------------------------------
# derivatives of r^nu at (0, 0, 1), exact
# ----------------------------------------------------------------------------

_DER = {}


def deriv_at_z(nu, n):
    """d^n |x|^nu at x = (0,0,1) via the Taylor-coefficient recurrence
    |n| T_n = -(2|n| - nu - 2) T_{n-e_z} - (|n| - nu - 2) sum_i T_{n-2e_i},  d^n = n! T_n."""
    key = (nu, n)
    if key in _DER:
        return _DER[key]

    def T(n):
        if min(n) < 0:
            return Fr(0)
        if (nu, n, "T") in _DER:
            return _DER[(nu, n, "T")]
        s = sum(n)
        if s == 0:
            v = Fr(1)
        else:
            v = -(2 * s - nu - 2) * T((n[0], n[1], n[2] - 1))
            for i in range(3):
                nn = list(n)
                nn[i] -= 2
                v -= (s - nu - 2) * T(tuple(nn))
            v /= s
        _DER[(nu, n, "T")] = v
        return v

    val = T(n) * math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2])
    _DER[key] = val
    return val


def contract(poly, nu):
    return sum(v * deriv_at_z(nu, k) for k, v in poly.items())


# ----------------------------------------------------------------------------
# pair-frame couplings and self scalars
# ----------------------------------------------------------------------------

def couplings(trunc):
    """Nonzero (p, q, alpha, beta): C_pq = (1/a) (a/r)^(l+l'+1) (alpha + beta (a/r)^2)."""
    comps = components(trunc)
    out = []
    for p, cp in enumerate(comps):
        lp = cp.L - 1
        for q, cq in enumerate(comps):
            lq = cq.L - 1
            if abs(cp.mu) != abs(cq.mu):
                continue
            M1 = sum(contract(pmul(cp.tails[i], cq.tails[i]), -1) for i in range(3))
            W = pmul(cp.full, cq.full)
            M2 = contract(W, 1)
            M3 = contract(W, -1)
            sgn = (-1) ** lq
            alpha = sgn * (2 * M1 - M2)
            beta = -sgn * 2 * (Fr(1, 4 * lp + 6) + Fr(1, 4 * lq + 6)) * M3
            # normalisation: sqrt(nrm2_p nrm2_q) / (c_p c_q) = 1/sqrt(sum tails^2 products)
            f = math.sqrt(cp.nrm2_basis * cq.nrm2_basis / (cp.emb2 * cq.emb2))
            a_f = float(alpha) * f
            b_f = float(beta) * f
            if abs(a_f) > 1e-15 or abs(b_f) > 1e-15:
                out.append((p, q, a_f, b_f))
    return comps, out


def point_couplings(trunc):
    """(p, q, alpha, beta) of the 1s rows (p < 3) for a point target: the target has no
    radius, so only the source's finite-size operator F^l' = 1 + a^2/(4l'+6) lap remains
    in the beta term (the beta of couplings() carries both radii: its factor
    1/6 + 1/(4l'+6) becomes 1/(4l'+6))."""
    comps, cpl = couplings(trunc)
    out = []
    for (p, q, al, be) in cpl:
        if p >= 3:
            continue
        lq = comps[q].L - 1
        bp = be * (1.0 / (4 * lq + 6)) / (1.0 / 6 + 1.0 / (4 * lq + 6))
        out.append((p, q, al, bp))
    return comps, out


def sphere_mono(n):
    """int x^a y^b z^c dOmega / (4 pi), exact."""
    if any(v % 2 for v in n):
        return Fr(0)
    return Fr(dfact(n[0] - 1) * dfact(n[1] - 1) * dfact(n[2] - 1), dfact(sum(n) + 1))


def sphere_avg(p):
    return sum(v * sphere_mono(k) for k, v in p.items())


def self_scalar(c):
    """g for one component, in units of 1/a: <e, G_nn e> with
    G_nn = (2l+1)/(2 pi a) int Y (I - nn) Y dOmega and (e . Y^(l))_i = (2l-1)!! tail_i(n)."""
    l = c.L - 1
    t = c.tails
    sq = padd(*[pmul(t[i], t[i]) for i in range(3)])
    rad = padd(*[pmul(AXES[i], t[i]) for i in range(3)])
    avg = sphere_avg(sq) - sphere_avg(pmul(rad, rad))    # (1/4pi) int [...]
    # (2l+1)/(2 pi) * 4 pi * avg * ((2l-1)!!)^2 * nrm2 / emb2
    return float(Fr(2 * (2 * l + 1) * dfact(2 * l - 1) ** 2) * avg * c.nrm2_basis / c.emb2)


# ----------------------------------------------------------------------------
# rotation of the packed basis about the y axis
# ----------------------------------------------------------------------------

def rot_y_poly(k):
    """D^k_{mu nu}(R_y(beta)) = <U_mu, R.U_nu> as {(i, j): float} polynomials in (cos, sin).

    (R.U_nu) . x^k = U_nu . (R^T x)^k, R^T x = (c x - s z, y, s x + c z)."""
    basis = {mu: solid_harmonic(k, mu) for mu in range(-k, k + 1)}
    # substitution with coefficients in Q[c, s]: represent as dict {(a,b,c,i,j): coef}
    def subst(S):
        out = {}
        for (ax, by, cz), v in S.items():
            # (c x - s z)^ax y^by (s x + c z)^cz
            for j1 in range(ax + 1):          # j1 factors of (-s z)
                c1 = math.comb(ax, j1) * (-1) ** j1
                for j2 in range(cz + 1):      # j2 factors of (s x)
                    c2 = math.comb(cz, j2)
                    xp = (ax - j1) + j2
                    zp = j1 + (cz - j2)
                    ci = (ax - j1) + (cz - j2)
                    si = j1 + j2
                    key = (xp, by, zp, ci, si)
                    out[key] = out.get(key, 0) + v * c1 * c2
        return out
    D = {}
    for nu in range(-k, k + 1):
        Sn, n2 = basis[nu]
        sub = subst(Sn)
        for mu in range(-k, k + 1):
            Sm, m2 = basis[mu]
            poly = {}
            for (xp, by, zp, ci, si), v in sub.items():
                w = Sm.get((xp, by, zp))
                if w is None:
                    continue
                f = v * w * Fr(math.factorial(xp) * math.factorial(by) * math.factorial(zp), math.factorial(k))
                # reduce s^2 -> 1 - c^2
                terms = {(ci, si): f}
                while True:
                    red = {}
                    changed = False
                    for (a, b), coef in terms.items():
                        if b >= 2:
                            changed = True
                            red[(a, b - 2)] = red.get((a, b - 2), 0) + coef
                            red[(a + 2, b - 2)] = red.get((a + 2, b - 2), 0) - coef
                        else:
                            red[(a, b)] = red.get((a, b), 0) + coef
                    terms = red
                    if not changed:
                        break
                for kk, vv in terms.items():
                    poly[kk] = poly.get(kk, 0) + vv
            scale = math.sqrt(m2 * n2)
            poly = {kk: float(vv) * scale for kk, vv in poly.items() if vv != 0}
            if poly:
                D[(mu, nu)] = poly
    return D


# ----------------------------------------------------------------------------
# self checks (floating point) of the derived tables
# ----------------------------------------------------------------------------

def eval_poly_cs(poly, c, s):
    return sum(v * c ** i * s ** j for (i, j), v in poly.items())


def check_tables(maxk):
    import random
    rnd = random.Random(7)
    for k in range(1, maxk + 1):
        D = rot_y_poly(k)
        b = rnd.uniform(-3, 3)
        c, s = math.cos(b), math.sin(b)
        n = 2 * k + 1
        M = [[eval_poly_cs(D.get((mu, nu), {}), c, s) for nu in range(-k, k + 1)] for mu in range(-k, k + 1)]
        for i in range(n):
            for j in range(n):
                v = sum(M[t][i] * M[t][j] for t in range(n))
                assert abs(v - (i == j)) < 1e-12, (k, i, j, v)
        # orthonormal basis
        for mu in range(-k, k + 1):
            for nu in range(-k, k + 1):
                S1, a1 = solid_harmonic(k, mu)
                S2, a2 = solid_harmonic(k, nu)
                v = float(frob(S1, S2, k)) * math.sqrt(a1 * a2)
                assert abs(v - (mu == nu)) < 1e-12, (k, mu, nu, v)
                # traceless
            assert not plap(solid_harmonic(k, mu)[0])


# ----------------------------------------------------------------------------
# code emission
# ----------------------------------------------------------------------------

def fmt(v):
    return repr(float(v))


def fma_chain(terms):
    """C++ expression for the sum of products [(a, b), ...] as a chain of gbi_fmac calls:
    the first product is a plain multiply, every later one is fused into the sum."""
    if not terms:
        return "T(0)"
    a0, b0 = terms[0]
    expr = a0 if b0 is None else "%s * %s" % (a0, b0)
    for a, b in terms[1:]:
        expr = "(%s + %s)" % (expr, a) if b is None else "gbi_fmac(%s, %s, %s)" % (a, b, expr)
    return expr


def emit(path):
    lines = []
    w = lines.append
    w("// Generated by paper_1411_0278_gb300/gen_tables.py -- do not edit.")
    w("// Pair-frame single-layer Galerkin couplings, packed-basis rotations and")
    w("// self scalars for the truncations l<=2, 3, 4, 5 (mode sets 1s 2a | 2s 3t | 3a 3s 4t | 4a 4s 5t |")
    w("// 5a 5s 6t) and the minimal truncation 40 (every mode of rank <= 4: l<=4 without 5t).")
    w("#pragma once")
    w("")
    w("#include \"df.cuh\"   // gbi_fmac: a * b + c in the arithmetic of T")
    w("")
    maxk = 5
    check_tables(maxk)
    # rotation about y: gbi_dmat<k>(c, s, dm) fills the nonzero entries of D^k(R_y(beta))
    # (c = cos beta, s = sin beta); gbi_dapply<k>/gbi_dapplyT<k> apply it or its transpose.
    dm_terms = {}
    dm_nnz = {}
    for k in range(1, maxk + 1):
        D = rot_y_poly(k)
        entries = sorted(D.items())
        dm_terms[k] = sum(len(p) for _, p in entries)
        dm_nnz[k] = len(entries)
        w("static constexpr int gbi_dm%d_n = %d;" % (k, len(entries)))
        w("template <typename T> __host__ __device__ __forceinline__ void gbi_dmat%d(T c, T s, T* __restrict__ dm) {" % k)
        if k <= 4:
            w("  const T c2 = c * c; const T c3 = c2 * c; const T c4 = c2 * c2;")
            w("  const T cp[5] = {T(1), c, c2, c3, c4}; (void)cp;")
            w("  const T sp[5] = {s, c * s, c2 * s, c3 * s, c4 * s}; (void)sp;")
        else:
            w("  const T c2 = c * c; const T c3 = c2 * c; const T c4 = c2 * c2; const T c5 = c4 * c;")
            w("  const T cp[6] = {T(1), c, c2, c3, c4, c5}; (void)cp;")
            w("  const T sp[6] = {s, c * s, c2 * s, c3 * s, c4 * s, c5 * s}; (void)sp;")
        for e, ((mu, nu), poly) in enumerate(entries):
            terms = []
            for (i, j), v in sorted(poly.items()):
                mono = ("sp[%d]" % i) if j == 1 else (None if i == 0 else "cp[%d]" % i)
                if mono is not None and v in (1, -1):      # unit coefficient: no multiply
                    terms.append((mono if v == 1 else "(-%s)" % mono, None))
                else:
                    terms.append(("T(%s)" % fmt(v), mono))
            # put a constant term (no monomial) first, so that the chain starts from it
            terms.sort(key=lambda t: t[1] is not None)
            w("  dm[%d] = %s;   // (mu=%d, nu=%d)" % (e, fma_chain(terms), mu, nu))
        w("}")
        for transpose in (False, True):
            nm = "gbi_dapply%s%d" % ("T" if transpose else "", k)
            w("template <typename T> __host__ __device__ __forceinline__ void %s(const T* __restrict__ dm, const T* __restrict__ in, T* __restrict__ out) {" % nm)
            rows = {}
            for e, ((mu, nu), poly) in enumerate(entries):
                if transpose:
                    rows.setdefault(nu, []).append((e, mu))
                else:
                    rows.setdefault(mu, []).append((e, nu))
            for o in range(-k, k + 1):
                terms = rows.get(o, [])
                w("  out[%d] = %s;" % (o + k, fma_chain([("dm[%d]" % e, "in[%d]" % (i + k)) for e, i in terms])))
            w("}")
    w("")
    # packing helpers for the trap inputs: U_mu . v^2 (mu = -2..2) and the Cartesian
    # symmetric tensor sum_mu y_mu U_mu (xx, xy, xz, yy, yz, zz)
    w("template <typename T> __host__ __device__ __forceinline__ void gbi_pack2(T x, T y, T z, T* __restrict__ out) {")
    for mu in range(-2, 3):
        S, n2 = solid_harmonic(2, mu)
        sc = math.sqrt(n2)
        names = {(2, 0, 0): "x * x", (0, 2, 0): "y * y", (0, 0, 2): "z * z",
                 (1, 1, 0): "x * y", (1, 0, 1): "x * z", (0, 1, 1): "y * z"}
        expr = " + ".join("T(%s) * %s" % (fmt(float(v) * sc), names[kk]) for kk, v in sorted(S.items()))
        w("  out[%d] = %s;" % (mu + 2, expr))
    w("}")
    w("template <typename T> __host__ __device__ __forceinline__ void gbi_unpack2(const T* __restrict__ yv, T* __restrict__ s6) {")
    order = [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for idx, key in enumerate(order):
        terms = []
        for mu in range(-2, 3):
            S, n2 = solid_harmonic(2, mu)
            v = S.get(key, 0)
            if v:
                # tensor component = coef * n!/k!
                f = float(v) * math.sqrt(n2) * math.factorial(key[0]) * math.factorial(key[1]) * math.factorial(key[2]) / 2.0
                terms.append("T(%s) * yv[%d]" % (fmt(f), mu + 2))
        w("  s6[%d] = %s;" % (idx, " + ".join(terms) or "T(0)"))
    w("}")
    w("")
    for trunc in TRUNCS:
        comps, cpl = couplings(trunc)
        d = len(comps)
        modes = MODES[:NMODES[trunc]]
        if trunc == MINIMAL:
            w("// ---------------- minimal truncation (every mode of rank <= 4): %d components per sphere" % d)
        else:
            w("// ---------------- truncation l <= %d: %d components per sphere" % (trunc, d))
        w("struct GbiTrunc%d {" % trunc)
        w("  static constexpr int D = %d;      // components per sphere (L + H)" % d)
        w("  static constexpr int NL = 6;")
        w("  static constexpr int H = %d;" % (d - 6))
        w("  static constexpr int NMODE = %d;" % len(modes))
        w("  static constexpr int MAXK = %d;" % max(m[1] - m[2] for m in modes))
        ks = [m[1] - m[2] for m in modes]
        Ls = [m[1] for m in modes]
        offs = []
        o = 0
        for kk in ks:
            offs.append(o)
            o += 2 * kk + 1
        w("};")
        w("__host__ __device__ constexpr int gbi_t%d_k(int m) { constexpr int v[%d] = {%s}; return v[m]; }"
          % (trunc, len(ks), ", ".join(map(str, ks))))
        w("__host__ __device__ constexpr int gbi_t%d_L(int m) { constexpr int v[%d] = {%s}; return v[m]; }"
          % (trunc, len(Ls), ", ".join(map(str, Ls))))
        w("__host__ __device__ constexpr int gbi_t%d_off(int m) { constexpr int v[%d] = {%s}; return v[m]; }"
          % (trunc, len(offs), ", ".join(map(str, offs))))
        w("// internal coordinate x = scale * packed coordinate of the paper's irreducible tensor")
        w("static const double gbi_t%d_scale[%d] = {%s};" % (trunc, d, ", ".join(fmt(c.scale) for c in comps)))
        w("// self scalar g per component (units 1/a): 8 pi eta V = -g Q for an isolated sphere")
        w("static const double gbi_t%d_self[%d] = {%s};" % (trunc, d, ", ".join(fmt(self_scalar(c)) for c in comps)))
        # coupling code: y[p] = e^(lp+1) * sum_q (alpha + beta e2) xs[q],  xs[q] = e^lq x[q]
        for rows_name, rows in (("all", range(d)), ("L", range(6)), ("H", range(6, d))):
            for cols_name, cols in (("all", range(d)), ("L", range(6)), ("H", range(6, d))):
                nm = "gbi_t%d_couple_%s_%s" % (trunc, rows_name, cols_name)
                w("template <typename T> __host__ __device__ __forceinline__ void %s(T e2, const T* __restrict__ xs, T* __restrict__ y) {" % nm)
                w("  // xs[q] = (a/r)^l_q * x'_q in the pair frame; y[p] = sum_q (alpha_pq + beta_pq (a/r)^2) xs[q]")
                by_p = {}
                for (p, q, al, be) in cpl:
                    if p in rows and q in cols:
                        by_p.setdefault(p, []).append((q, al, be))
                for p in rows:
                    terms = by_p.get(p, [])
                    if not terms:
                        w("  y[%d] = T(0);" % p)
                        continue
                    ta = [("T(%s)" % fmt(al), "xs[%d]" % q) for q, al, be in terms if al != 0.0]
                    tb = [("T(%s)" % fmt(be), "xs[%d]" % q) for q, al, be in terms if be != 0.0]
                    if tb:
                        w("  y[%d] = gbi_fmac(e2, %s, %s);" % (p, fma_chain(tb), fma_chain(ta)))
                    else:
                        w("  y[%d] = %s;" % (p, fma_chain(ta)))
                w("}")
        # the flow at a point (a target of radius zero): the 1s rows from every column
        _, pcpl = point_couplings(trunc)
        w("template <typename T> __host__ __device__ __forceinline__ void gbi_t%d_couple_P_all(T e2, const T* __restrict__ xs, T* __restrict__ y) {" % trunc)
        w("  // point target: 1s rows only, beta from the source's finite-size operator alone")
        by_p = {}
        for (p, q, al, be) in pcpl:
            by_p.setdefault(p, []).append((q, al, be))
        for p in range(3):
            terms = by_p.get(p, [])
            ta = [("T(%s)" % fmt(al), "xs[%d]" % q) for q, al, be in terms if al != 0.0]
            tb = [("T(%s)" % fmt(be), "xs[%d]" % q) for q, al, be in terms if be != 0.0]
            if tb:
                w("  y[%d] = gbi_fmac(e2, %s, %s);" % (p, fma_chain(tb), fma_chain(ta)))
            else:
                w("  y[%d] = %s;" % (p, fma_chain(ta)))
        w("}")
        nnz = len(cpl)
        w("static constexpr int gbi_t%d_nnz = %d;   // pair-frame nonzeros (all rows, all columns)" % (trunc, nnz))
        # algorithmic flops per ordered pair of the pair-frame evaluation (FMA = 2, rsqrt = 1)
        flops = {}
        for rn, rows in (("all", range(d)), ("L", range(6)), ("H", range(6, d))):
            for cn, cols in (("all", range(d)), ("L", range(6)), ("H", range(6, d))):
                rmodes = sorted({comps[p].mode for p in rows})
                cmodes = sorted({comps[q].mode for q in cols})
                maxk_used = max(MODES[m][1] - MODES[m][2] for m in rmodes + cmodes)
                f = 9 + 5 + 1 + 3 + 3 + 1 + 2 + 2 + 2          # geometry, direction, angles
                f += 6 * max(0, maxk_used - 1)                   # cos/sin of multiple angles
                f += 7                                           # powers of a/r
                for kk in range(1, maxk_used + 1):               # rotation matrices about y
                    f += 6 + 2 * dm_terms[kk]
                # z and y rotations per block; the (a/r)^j scalings ride on the z rotation's
                # cos/sin factors (2 products per multiple angle and power j, shared by the
                # modes), plus one multiply (columns, l > 0) or FMA (rows) for the centre entry
                kmax_pow = {}
                for m in cmodes:
                    kk, j = MODES[m][1] - MODES[m][2], MODES[m][1] - 1
                    f += 6 * kk + 2 * dm_nnz[kk] + (1 if j > 0 else 0)
                    if j > 0:
                        kmax_pow[j] = max(kmax_pow.get(j, 0), kk)
                for m in rmodes:
                    kk, j = MODES[m][1] - MODES[m][2], MODES[m][1]
                    f += 6 * kk + 2 * dm_nnz[kk] + 1
                    kmax_pow[j] = max(kmax_pow.get(j, 0), kk)
                f += sum(2 * kk for kk in kmax_pow.values())
                for (p, q, al, be) in cpl:
                    if p in rows and q in cols:
                        f += (2 if al != 0.0 else 0) + (2 if be != 0.0 else 0)
                f += 2 * len(rows) + len(rows)                  # combine alpha/beta, accumulate
                flops[(rn, cn)] = f
        # the point rows (1s from every column): same count with the 1s row mode and the
        # point couplings
        cmodes = sorted({c.mode for c in comps})
        maxk_used = max(MODES[m][1] - MODES[m][2] for m in cmodes)
        fp = 9 + 5 + 1 + 3 + 3 + 1 + 2 + 2 + 2 + 6 * max(0, maxk_used - 1) + 7
        for kk in range(1, maxk_used + 1):
            fp += 6 + 2 * dm_terms[kk]
        kmax_pow = {}
        for m in cmodes:
            kk, j = MODES[m][1] - MODES[m][2], MODES[m][1] - 1
            fp += 6 * kk + 2 * dm_nnz[kk] + (1 if j > 0 else 0)
            if j > 0:
                kmax_pow[j] = max(kmax_pow.get(j, 0), kk)
        fp += 6 * 1 + 2 * dm_nnz[1] + 1
        kmax_pow[1] = max(kmax_pow.get(1, 0), 1)
        fp += sum(2 * kk for kk in kmax_pow.values())
        for (p, q, al, be) in pcpl:
            fp += (2 if al != 0.0 else 0) + (2 if be != 0.0 else 0)
        fp += 2 * 3 + 3
        w("static constexpr int gbi_t%d_flops_point = %d;   // per (point, sphere): 1s rows from all columns" % (trunc, fp))
        w("// algorithmic flops per ordered pair, [rows][cols] with 0 = all, 1 = L, 2 = H")
        w("static constexpr int gbi_t%d_flops[3][3] = {%s};" % (trunc, ", ".join(
            "{%s}" % ", ".join(str(flops[(rn, cn)]) for cn in ("all", "L", "H")) for rn in ("all", "L", "H"))))
        w("")
    text = "\n".join(lines) + "\n"
    with open(path, "w") as f:
        f.write(text)
    return text


def main(argv):
    here = os.path.dirname(os.path.abspath(__file__))
    out = argv[1] if len(argv) > 1 else os.path.join(here, "csrc", "gbi_generated.cuh")
    emit(out)


if __name__ == "__main__":
    main(sys.argv)
