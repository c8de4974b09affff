"""Pins of the oracle's equilibria (Eq. 14, Eq. 22) and of the moment-matching
construction (Sec. 3.1-3.2) against Table 1, the continuous Maxwellian (Eq. 6)
integrated by numpy's Gauss-Hermite rule, and the textbook second-order
equilibrium on full-neighbourhood stencils."""
import itertools
import json
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import construction as cons

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_moments.json")


def _terms_value(terms, roles, rho, rho0, u, max_order):
    s = 0.0
    for coef, dens, mono in terms:
        if sum(mono.values()) > max_order:
            continue
        t = float(Fr(coef)) * (rho if dens == "rho" else rho0)
        for role, p in mono.items():
            t *= u[roles[role]] ** p
        s += t
    return s


def _moment(c, f, e):
    return float((f * np.prod(c.astype(float) ** np.asarray(e), axis=1)).sum())


def _role_assignments(exps):
    """Distinct axis assignments for the roles of a Table 1 row."""
    seen = {}
    for perm in itertools.permutations(range(3)):
        roles = dict(zip("ijk", perm))
        e = [0, 0, 0]
        for r, p in exps.items():
            e[roles[r]] = p
        seen.setdefault(tuple(e), roles)
    return seen


def _d3q27_standard(rho, rho0, u):
    """Second-order part of Eq. 14 on D3Q27 with the tensor-product weights."""
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    vels = list(itertools.product((-1, 0, 1), repeat=3))
    c = np.array(vels)
    w = np.array([w1[a] * w1[b] * w1[d] for a, b, d in vels])
    cu = c @ u
    return c, w * rho + w * rho0 * (3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))


@pytest.mark.parametrize("rho0_is_rho", [False, True])
def test_table1_moments(rho0_is_rho):
    table = json.load(open(GOLDEN))
    c, _, _ = oracle.velocity_set()
    rng = np.random.default_rng(11)
    total = 0
    for trial in range(20):
        rho = 1.0 + rng.uniform(-0.05, 0.05)
        u = rng.uniform(-0.1, 0.1, 3)
        rho0 = rho if rho0_is_rho else 1.0
        feq = {
            "D3Q19-S": oracle.equilibrium(oracle.STANDARD, np.array([rho]), u.reshape(3, 1), rho0_is_rho)[0],
            "D3Q19-I": oracle.equilibrium(oracle.IMPROVED, np.array([rho]), u.reshape(3, 1), rho0_is_rho)[0],
        }
        c27, f27 = _d3q27_standard(rho, rho0, u)
        for row in table["rows"]:
            assign = _role_assignments(row["exponents"])
            if trial == 0:
                assert len(assign) == row["count"], row["name"]
                total += len(assign)
            for e, roles in assign.items():
                for model in ("D3Q19-S", "D3Q19-I"):
                    # the second-order equilibria match the table up to O(u^3)
                    want = _terms_value(row[model], roles, rho, rho0, u, 2)
                    got = _moment(c, feq[model], e)
                    assert got == pytest.approx(want, abs=2e-15), (row["name"], model, e)
                want = _terms_value(row.get("D3Q27_reading", row["D3Q27"]), roles, rho, rho0, u, 2)
                assert _moment(c27, f27, e) == pytest.approx(want, abs=2e-15), (row["name"], "D3Q27", e)
    assert total == 27


def test_table1_s_and_i_differ_only_in_pi_iijj():
    """The second-order difference I - S shows up in exactly the three Pi_iijj
    moments (row 7), with value rho0 u_k^2 / 6."""
    c, _, _ = oracle.velocity_set()
    u = np.array([0.03, -0.05, 0.07])
    fs = oracle.equilibrium(oracle.STANDARD, np.array([1.0]), u.reshape(3, 1))[0]
    fi = oracle.equilibrium(oracle.IMPROVED, np.array([1.0]), u.reshape(3, 1))[0]
    for e in itertools.product((0, 1, 2), repeat=3):
        d = _moment(c, fi - fs, e)
        if sorted(e) == [0, 2, 2]:
            k = e.index(0)
            assert d == pytest.approx(u[k] ** 2 / 6, rel=1e-12)
        else:
            assert abs(d) < 1e-16, e


def test_equilibrium_moment_conditions_eq18():
    """Eq. 18 a-c hold exactly for both D3Q19 equilibria (to rounding)."""
    c, _, _ = oracle.velocity_set()
    rng = np.random.default_rng(5)
    for kind in (oracle.STANDARD, oracle.IMPROVED):
        for rho0_is_rho in (False, True):
            rho = 1 + rng.uniform(-0.1, 0.1)
            u = rng.uniform(-0.1, 0.1, 3)
            rho0 = rho if rho0_is_rho else 1.0
            f = oracle.equilibrium(kind, np.array([rho]), u.reshape(3, 1), rho0_is_rho)[0]
            assert f.sum() == pytest.approx(rho, abs=1e-15)
            assert np.allclose(c.T @ f, rho0 * u, atol=1e-16)
            P = (c.T * f) @ c
            assert np.allclose(P, rho0 * np.outer(u, u) + np.eye(3) * rho / 3, atol=1e-16)


def test_maxwellian_moments_against_quadrature_of_eq6():
    """The construction's untruncated Maxwellian moments (products of the 1D
    moments 1, u, u^2 + theta) equal numerical moments of Eq. 6 with theta = 1/3,
    computed with a 20-point Gauss-Hermite rule (exact for these polynomials)."""
    x, wt = np.polynomial.hermite_e.hermegauss(20)
    wt = wt / math.sqrt(2 * math.pi)
    rng = np.random.default_rng(3)
    for _ in range(5):
        u = rng.uniform(-0.2, 0.2, 3)
        for e in itertools.product((0, 1, 2), repeat=3):
            num = 1.0
            for i in range(3):
                xi = u[i] + math.sqrt(1 / 3) * x
                num *= float((wt * xi ** e[i]).sum())
            poly = cons.maxwellian_moment(e, order=99)
            val = float(cons.evaluate(poly, 1.0, 1.0, [Fr(float(v)) for v in u]))
            assert val == pytest.approx(num, rel=1e-13, abs=1e-16)


def _rational_points(d, n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        rho = Fr(int(rng.integers(90, 110)), 100)
        rho0 = Fr(int(rng.integers(90, 110)), 100)
        u = [Fr(int(rng.integers(-20, 21)), int(rng.integers(50, 200))) for _ in range(d)]
        yield rho, rho0, u


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_construction_reproduces_standard_on_full_stencils(name):
    """Sec. 3.1-3.2: on D2Q9 and D3Q27 the construction (Maxwellian moments
    truncated at second order) gives the second-order part of Eq. 14 exactly."""
    vels, polys = cons.constructed_equilibrium(name)
    d = len(vels[0])
    w1 = {-1: Fr(1, 6), 0: Fr(2, 3), 1: Fr(1, 6)}
    for rho, rho0, u in _rational_points(d, 12, 1):
        uu = sum(x * x for x in u)
        for c, p in zip(vels, polys):
            w = Fr(1)
            for a in c:
                w *= w1[a]
            cu = sum(a * b for a, b in zip(c, u))
            std = w * rho + w * rho0 * (3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
            assert cons.evaluate(p, rho, rho0, u) == std


def test_construction_d3q19_matches_oracle_improved_equilibrium():
    """Sec. 3.2: the D3Q19 construction (Eq. 21 dropped moments) equals the
    closed form of Eq. 22 as implemented in the C oracle."""
    vels, polys = cons.constructed_equilibrium("D3Q19")
    M = cons.moment_matrix(vels, cons.exponents("D3Q19"))
    assert len(M) == 19 and cons.determinant(M) != 0
    c, _, _ = oracle.velocity_set()
    index = {tuple(int(a) for a in v): q for q, v in enumerate(c)}
    for rho, rho0, u in _rational_points(3, 12, 2):
        # rho0 = rho and rho0 = 1 are both covered by evaluating the oracle twice
        for rho0_is_rho in (False, True):
            r0 = rho if rho0_is_rho else Fr(1)
            f = oracle.equilibrium(oracle.IMPROVED, np.array([float(rho)]),
                                   np.array([float(x) for x in u]).reshape(3, 1), rho0_is_rho)[0]
            for v, p in zip(vels, polys):
                exact = cons.evaluate(p, rho, r0, u)
                assert f[index[v]] == pytest.approx(float(exact), abs=1e-16)


def test_construction_d3q19_is_not_the_standard_equilibrium():
    vels, polys = cons.constructed_equilibrium("D3Q19")
    c, _, _ = oracle.velocity_set()
    index = {tuple(int(a) for a in v): q for q, v in enumerate(c)}
    u = [Fr(1, 20), Fr(-1, 30), Fr(1, 25)]
    fs = oracle.equilibrium(oracle.STANDARD, np.array([1.0]), np.array([float(x) for x in u]).reshape(3, 1))[0]
    diff = max(abs(float(cons.evaluate(p, 1, 1, u)) - fs[index[v]]) for v, p in zip(vels, polys))
    assert diff > 1e-5


def test_d2q9_projection_of_improved_equilibrium():
    """Grouping D3Q19-I by (c_x, c_y) gives the D2Q9 equilibrium in (rho, u_x, u_y)
    for any u_z; D3Q19-S does so only at u_z = 0 (a consequence of Eq. 14, 22)."""
    c, _, _ = oracle.velocity_set()
    vels2, polys2 = cons.constructed_equilibrium("D2Q9")
    rng = np.random.default_rng(8)
    for _ in range(10):
        rho = 1 + rng.uniform(-0.05, 0.05)
        u = rng.uniform(-0.1, 0.1, 3)
        fi = oracle.equilibrium(oracle.IMPROVED, np.array([rho]), u.reshape(3, 1))[0]
        fs = oracle.equilibrium(oracle.STANDARD, np.array([rho]), u.reshape(3, 1))[0]
        u0 = u.copy()
        u0[2] = 0
        fs0 = oracle.equilibrium(oracle.STANDARD, np.array([rho]), u0.reshape(3, 1))[0]
        uf = [Fr(float(u[0])), Fr(float(u[1]))]
        worst_s = 0.0
        for v, p in zip(vels2, polys2):
            d2 = float(cons.evaluate(p, Fr(float(rho)), 1, uf))
            sel = [q for q in range(19) if (c[q, 0], c[q, 1]) == v]
            assert fi[sel].sum() == pytest.approx(d2, abs=1e-15)
            assert fs0[sel].sum() == pytest.approx(d2, abs=1e-15)
            worst_s = max(worst_s, abs(fs[sel].sum() - d2))
        assert worst_s > 1e-6 * u[2] ** 2 / 0.01
