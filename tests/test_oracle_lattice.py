"""Pins of the oracle's lattice tables, equilibrium, Guo forcing and BGK
collision against what the paper prints (Appendix A) and what the lattice
algebra fixes."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# Eq. (A.1) and Eq. (A.2), transcribed here independently of the oracle.
E_A1 = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]]).T
W_A2 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def load_M():
    """Eq. (A.3) as printed, with the reading of its garbled rows 13/14."""
    M = np.loadtxt(os.path.join(GOLD, "d3q19_M_eqA3.txt"))
    assert M.shape == (19, 19)
    assert np.linalg.matrix_rank(M) < 19  # the print is singular
    M = M.copy()
    M[13, 11:] = 0.0                     # p_xy: only the xy diagonals
    M[14, :] = 0.0
    M[14, 15:19] = [1, -1, -1, 1]        # p_yz: only the yz diagonals
    assert np.linalg.matrix_rank(M) == 19
    return M


def test_d3q19_tables_match_eq_A1_A2():
    e, w, opp = O.lattice(19)
    np.testing.assert_array_equal(e, E_A1)
    np.testing.assert_allclose(w, W_A2, rtol=0, atol=1e-16)
    for i in range(19):
        np.testing.assert_array_equal(e[opp[i]], -e[i])


def test_d2q9_is_inplane_subset():
    e, w, opp = O.lattice(9)
    sub = [0, 1, 2, 3, 4, 7, 8, 9, 10]
    np.testing.assert_array_equal(e, E_A1[sub])
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4,
                               atol=1e-16)
    for i in range(9):
        np.testing.assert_array_equal(e[opp[i]], -e[i])


@pytest.mark.parametrize("q", [9, 19])
def test_isotropy(q):
    e, w, _ = O.lattice(q)
    D = 2 if q == 9 else 3
    e = e[:, :D].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, e), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, e, e),
                               np.eye(D) / 3, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0,
                               atol=1e-16)
    d = np.eye(D)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(
        np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e), iso4, atol=1e-15)


def meq_A4(rho, rho0, u):
    """Eq. (A.4); m10 read as -(3/2) p_xx^eq with 3 p_xx^eq = m9 (the print's
    second equality drops that factor 1/3)."""
    ux, uy, uz = u
    u2 = ux * ux + uy * uy + uz * uz
    pxx3 = rho0 * (2 * ux * ux - uy * uy - uz * uz)
    pww = rho0 * (uy * uy - uz * uz)
    return np.array([
        rho, -11 * rho + 19 * rho0 * u2, 3 * rho - 5.5 * rho0 * u2,
        rho0 * ux, -2 / 3 * rho0 * ux, rho0 * uy, -2 / 3 * rho0 * uy,
        rho0 * uz, -2 / 3 * rho0 * uz,
        pxx3, -0.5 * pxx3, pww, -0.5 * pww,
        rho0 * ux * uy, rho0 * uy * uz, rho0 * ux * uz, 0, 0, 0])


def SF_A5(u, F):
    """Eq. (A.5) with every (1 - S/2) factor set to 1 (rates zero)."""
    ux, uy, uz = u
    Fx, Fy, Fz = F
    uF = ux * Fx + uy * Fy + uz * Fz
    return np.array([
        0, 38 * uF, -11 * uF, Fx, -2 / 3 * Fx, Fy, -2 / 3 * Fy, Fz,
        -2 / 3 * Fz,
        2 * (2 * ux * Fx - uy * Fy - uz * Fz), (-2 * ux * Fx + uy * Fy + uz * Fz),
        2 * (uy * Fy - uz * Fz), (-uy * Fy + uz * Fz),
        uy * Fx + ux * Fy, uz * Fy + uy * Fz, ux * Fz + uz * Fx, 0, 0, 0])


def random_pops(rng, q):
    _, w, _ = O.lattice(q)
    return w * (1.0 + 0.2 * rng.standard_normal(q))


def test_equilibrium_moments_are_eq_A4():
    """With S = 1 and F = 0 every non-conserved moment of the output is its
    equilibrium value (A.4); mass and momentum keep theirs."""
    rng = np.random.default_rng(1)
    M = load_M()
    for _ in range(20):
        f = random_pops(rng, 19)
        rho0 = 0.9 + 0.2 * rng.random()
        out, u = O.collide(19, f, np.zeros(3), S=1.0, rho0=rho0)
        m = M @ out
        meq = meq_A4(f.sum(), rho0, u)
        cons = [0, 3, 5, 7]
        non = [k for k in range(19) if k not in cons]
        np.testing.assert_allclose(m[non], meq[non], rtol=0, atol=1e-14)
        np.testing.assert_allclose(m[cons], (M @ f)[cons], rtol=0, atol=1e-14)


def test_guo_forcing_moments_are_eq_A5():
    rng = np.random.default_rng(2)
    M = load_M()
    for _ in range(20):
        f = random_pops(rng, 19)
        F = 1e-3 * rng.standard_normal(3)
        out, u = O.collide(19, f, F, S=0.0, rho0=1.0)
        np.testing.assert_allclose(M @ (out - f), SF_A5(u, F), rtol=0,
                                   atol=1e-15)


def S_eq4(S):
    """Eq. (4) read with 19 entries (the print has a spurious 0 before S_nu):
    diag(0, S_e, S_eps, 0, S_q, 0, S_q, 0, S_q, S_nu, S_pi, S_nu, S_pi,
    S_nu, S_nu, S_nu, S_m, S_m, S_m), here with every rate equal to S."""
    d = np.full(19, S)
    d[[0, 3, 5, 7]] = 0.0
    return np.diag(d)


def test_collision_is_eq2_in_moment_space():
    """Eq. (2) evaluated with the printed M (A.3), m_eq (A.4) and S^F (A.5,
    its (1 - S/2) factors with the rate of each moment, 1 for the conserved
    ones), read as f'' = f - M^-1 S (m - m_eq) + M^-1 S^F."""
    rng = np.random.default_rng(13)
    M = load_M()
    Minv = np.linalg.inv(M)
    for _ in range(30):
        f = random_pops(rng, 19)
        F = 1e-3 * rng.standard_normal(3)
        S = 0.4 + 1.5 * rng.random()
        rho0 = 0.9 + 0.2 * rng.random()
        out, u = O.collide(19, f, F, S, rho0)
        rho = f.sum()
        Sm = S_eq4(S)
        SF = SF_A5(u, F) * (1 - 0.5 * np.diag(Sm))
        expect = f - Minv @ (Sm @ (M @ f - meq_A4(rho, rho0, u))) + Minv @ SF
        np.testing.assert_allclose(out, expect, rtol=0, atol=2e-15)


@pytest.mark.parametrize("q", [9, 19])
def test_collision_conserves_mass_and_gains_F(q):
    """Mass is unchanged and momentum becomes exactly j + F for any rho and
    rho0 (conserved moments have rate 0 in Eq. 4); u is Eq. (22); the second
    moment of the equilibrium is rho/3 I + rho0 u u (He-Luo form)."""
    rng = np.random.default_rng(3)
    e, w, _ = O.lattice(q)
    D = 2 if q == 9 else 3
    ef = e.astype(float)
    for _ in range(20):
        f = random_pops(rng, q)
        F = np.zeros(3)
        F[:D] = 1e-3 * rng.standard_normal(D)
        S = 0.5 + 1.4 * rng.random()
        rho0 = 0.9 + 0.2 * rng.random()
        out, u = O.collide(q, f, F, S, rho0)
        rho = f.sum()
        j = ef.T @ f
        np.testing.assert_allclose(u, (j + 0.5 * F) / rho, atol=1e-16)
        assert abs(out.sum() - rho) < 1e-14
        np.testing.assert_allclose(ef.T @ out, j + F, atol=1e-15)
        feq, ueq = O.collide(q, f, np.zeros(3), 1.0, rho0)
        # with S = 1 and F = 0, out = feq + e.(j - rho0 u)/E2 where u = j/rho
        E2 = (ef[:, 0] ** 2).sum()
        feq = feq - ef @ (j - rho0 * ueq) / E2
        P = np.einsum("i,ia,ib->ab", feq, ef, ef)[:D, :D]
        np.testing.assert_allclose(
            P, rho / 3 * np.eye(D) + rho0 * np.outer(ueq, ueq)[:D, :D],
            atol=1e-15)
        np.testing.assert_allclose(feq.sum(), rho, atol=1e-15)
        np.testing.assert_allclose(ef.T @ feq, rho0 * ueq, atol=1e-15)
