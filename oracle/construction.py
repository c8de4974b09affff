"""Moment-matching construction of discrete equilibria (Sec. 3.1 and 3.2), in exact arithmetic.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The construction, in the paper's order:

1. A single-speed stencil DdQq has velocities c_q with components in {-1, 0, 1}
   (Sec. 2.3).  Only monomial moments xi_0^e0 xi_1^e1 ... with e_i in {0,1,2}
   are independent (moment aliasing, Sec. 3.1).
2. D2Q9 and D3Q27 use all 3^d exponent vectors; D3Q19 drops the eight of
   Eq. 21.  The moment matrix is M[e][q] = prod_i c_qi^e_i (Sec. 3.2).
3. The target moments are those of the continuous Maxwellian (Eq. 6) with
   theta = c_s^2 = 1/3 in lattice units.  They factorise into 1D moments
   {1, u_i, u_i^2 + 1/3}; the product is truncated at second order in u; the
   u-independent part is multiplied by rho and the rest by rho0 (Eq. 18 and
   Table 1 use the same split).
4. f_eq = M^{-1} m_eq, solved exactly.

Polynomials are dicts mapping (tag, exponents) to Fraction, where tag is
"rho" or "rho0" and exponents is a tuple of powers of (u_0, ..., u_{d-1}).
"""
from fractions import Fraction as Fr
import itertools

THETA = Fr(1, 3)

# Eq. 21: exponent vectors dropped for D3Q19
DROPPED_D3Q19 = {(1, 2, 2), (2, 1, 2), (2, 2, 1), (1, 1, 2), (1, 2, 1), (2, 1, 1), (1, 1, 1), (2, 2, 2)}


def stencil(name):
    """Velocities of D2Q9, D3Q19 or D3Q27 (Sec. 2.3), as tuples of ints."""
    if name == "D2Q9":
        return [c for c in itertools.product((-1, 0, 1), repeat=2)]
    if name == "D3Q27":
        return [c for c in itertools.product((-1, 0, 1), repeat=3)]
    if name == "D3Q19":
        return [c for c in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in c) <= 2]
    raise ValueError(name)


def exponents(name):
    d = 2 if name == "D2Q9" else 3
    exps = list(itertools.product((0, 1, 2), repeat=d))
    if name == "D3Q19":
        exps = [e for e in exps if e not in DROPPED_D3Q19]
    return exps


def moment_matrix(vels, exps):
    return [[Fr(_mono(c, e)) for c in vels] for e in exps]


def _mono(c, e):
    p = 1
    for ci, ei in zip(c, e):
        p *= ci ** ei
    return p


def _poly_mul(a, b, d):
    out = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, Fr(0)) + ca * cb
    return out


def maxwellian_moment(e, order=2):
    """Moment int xi^e f_Maxwell dxi / rho (Eq. 6, theta = 1/3) as a polynomial in u,
    truncated at total degree `order`, split into rho / rho0 parts."""
    d = len(e)
    poly = {tuple([0] * d): Fr(1)}
    for i, ei in enumerate(e):
        unit = [0] * d
        if ei == 0:
            one_d = {tuple(unit): Fr(1)}
        elif ei == 1:
            unit[i] = 1
            one_d = {tuple(unit): Fr(1)}
        else:
            sq = list(unit)
            sq[i] = 2
            one_d = {tuple(sq): Fr(1), tuple(unit): THETA}
        poly = _poly_mul(poly, one_d, d)
    out = {}
    for ex, coef in poly.items():
        if coef == 0 or sum(ex) > order:
            continue
        tag = "rho" if sum(ex) == 0 else "rho0"
        out[(tag, ex)] = out.get((tag, ex), Fr(0)) + coef
    return out


def inverse(M):
    """Exact Gauss-Jordan inverse of a square matrix of Fractions."""
    n = len(M)
    A = [list(row) + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        p = A[col][col]
        A[col] = [x / p for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return [row[n:] for row in A]


def determinant(M):
    n = len(M)
    A = [list(r) for r in M]
    det = Fr(1)
    for col in range(n):
        piv = next((r for r in range(col, n) if A[r][col] != 0), None)
        if piv is None:
            return Fr(0)
        if piv != col:
            A[col], A[piv] = A[piv], A[col]
            det = -det
        det *= A[col][col]
        for r in range(col + 1, n):
            f = A[r][col] / A[col][col]
            A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return det


def constructed_equilibrium(name, order=2):
    """Returns (velocities, [poly_q]) with f_eq_q = sum_e (M^-1)[q][e] m_eq_e (Sec. 3.2)."""
    vels = stencil(name)
    exps = exponents(name)
    M = moment_matrix(vels, exps)
    Minv = inverse(M)
    moms = [maxwellian_moment(e, order) for e in exps]
    polys = []
    for q in range(len(vels)):
        p = {}
        for k, m in enumerate(moms):
            a = Minv[q][k]
            if a == 0:
                continue
            for key, coef in m.items():
                p[key] = p.get(key, Fr(0)) + a * coef
        polys.append({k: v for k, v in p.items() if v != 0})
    return vels, polys


def evaluate(poly, rho, rho0, u):
    """Value of a rho/rho0 polynomial at (rho, rho0, u); exact for Fractions."""
    s = 0
    for (tag, ex), coef in poly.items():
        term = coef * (rho if tag == "rho" else rho0)
        for ui, ei in zip(u, ex):
            term = term * ui ** ei
        s = s + term
    return s
