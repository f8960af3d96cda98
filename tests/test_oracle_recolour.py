"""Pins of the oracle's recolouring, Eqs. (20)-(21), by moments that the
lattice's isotropy fixes, on random node states through a test-only oracle
entry that runs the collision and the recolouring alone.

With f''_i the post-collision populations and rho = rho^r + rho^b:
  - each colour keeps its mass: sum_i f^r'_i = rho^r (the segregation
    term sums to zero, sum_i w_i e_i = 0);
  - the segregation momentum is closed-form: sum_i e_i f^r'_i minus
    (rho^r/rho) sum_i e_i f''_i equals beta (rho^r rho^b / rho) n / 3,
    because sum_i w_i e_i e_i = I / 3 on D2Q9 and D3Q19;
  - its second moment vanishes (sum_i w_i e_i e_i e_i = 0);
  - with beta = 0 every direction splits in proportion rho^r / rho, and a
    pure phase keeps all of f''.
A dropped w_i, a factor rho instead of rho^r rho^b / rho, a sign swap
between the colours or a wrong beta fails the second pin by far (without
w_i the D3Q19 sum gives 10 n instead of n / 3)."""
import numpy as np
import pytest

from oracle import oracle as O

TOL = 1e-13


def lattice(q):
    """The oracle's velocities (in its order, which the populations follow)
    and weights. The moments below hold for any order; they fail if the
    velocity set were not isotropic to third order with these weights."""
    e, w, _ = O.lattice(q)
    return e.astype(np.float64), w


def random_state(q, shape, seed, pure_at=None):
    rng = np.random.default_rng(seed)
    e, w = lattice(q)
    nz, ny, nx = shape
    wb = w[:, None, None, None]
    fr = wb * rng.uniform(0.05, 1.0, (q,) + shape)
    fb = wb * rng.uniform(0.05, 1.0, (q,) + shape)
    if pure_at is not None:
        fb[(slice(None),) + pure_at] = 0.0
    ft = np.stack([fr, fb])
    rr, rb = fr.sum(0), fb.sum(0)
    phi = (rr - rb) / (rr + rb)
    n = rng.normal(size=(3,) + shape)
    if q == 9:
        n[2] = 0.0
    n /= np.sqrt((n * n).sum(0))
    F = 1e-4 * rng.normal(size=(3,) + shape)
    if q == 9:
        F[2] = 0.0
    return ft, rr, rb, phi, n, F


def recoloured(q, shape, beta, seed, pure_at=None):
    solid = np.zeros(shape, np.uint8)
    o = O.Oracle(q, solid, (True, True, True))
    o.set_params(tau_r=1.0, tau_b=0.7, beta=beta, gamma=0.01, rho0=1.0)
    ft, rr, rb, phi, n, F = random_state(q, shape, seed, pure_at)
    out = o.collide_recolour(ft, rr, rb, phi, n, F)
    return out, rr, rb, n


CASES = [(19, (3, 4, 5)), (9, (1, 4, 5))]


@pytest.mark.parametrize("q,shape", CASES, ids=["D3Q19", "D2Q9"])
@pytest.mark.parametrize("beta", [0.95, 0.5])
def test_colour_masses_kept(q, shape, beta):
    out, rr, rb, _ = recoloured(q, shape, beta, 3)
    np.testing.assert_allclose(out[0].sum(0), rr, rtol=TOL, atol=0)
    np.testing.assert_allclose(out[1].sum(0), rb, rtol=TOL, atol=0)


@pytest.mark.parametrize("q,shape", CASES, ids=["D3Q19", "D2Q9"])
@pytest.mark.parametrize("beta", [0.95, 0.5, 0.1])
def test_segregation_momentum_closed_form(q, shape, beta):
    out, rr, rb, n = recoloured(q, shape, beta, 5)
    e, _ = lattice(q)
    rho = rr + rb
    fpp = out[0] + out[1]
    jr = np.einsum("ia,i...->a...", e, out[0])
    j = np.einsum("ia,i...->a...", e, fpp)
    seg = jr - rr / rho * j
    want = beta / 3.0 * rr * rb / rho * n
    scale = np.abs(want).max()
    assert np.abs(seg - want).max() <= TOL * scale
    # the plausible slips are far off: beta doubled, rho for rho^r rho^b/rho
    assert np.abs(seg - 2 * want).max() > 0.3 * scale
    assert np.abs(seg - beta / 3.0 * rho * n).max() > 0.3 * scale


@pytest.mark.parametrize("q,shape", CASES, ids=["D3Q19", "D2Q9"])
def test_segregation_second_moment_vanishes(q, shape):
    beta = 0.95
    out, rr, rb, _ = recoloured(q, shape, beta, 7)
    e, _ = lattice(q)
    rho = rr + rb
    dev = out[0] - rr / rho * (out[0] + out[1])
    m2 = np.einsum("ia,ib,i...->ab...", e, e, dev)
    scale = (beta * rr * rb / rho).max()
    assert np.abs(m2).max() <= TOL * scale


@pytest.mark.parametrize("q,shape", CASES, ids=["D3Q19", "D2Q9"])
def test_beta_zero_splits_in_proportion(q, shape):
    out, rr, rb, _ = recoloured(q, shape, 0.0, 11)
    rho = rr + rb
    np.testing.assert_allclose(out[0], rr / rho * (out[0] + out[1]),
                               rtol=TOL, atol=TOL * np.abs(out).max())


@pytest.mark.parametrize("q,shape", CASES, ids=["D3Q19", "D2Q9"])
def test_pure_phase_keeps_everything(q, shape):
    at = (0, 1, 2)
    out, rr, rb, _ = recoloured(q, shape, 0.95, 13, pure_at=at)
    sel = (slice(None),) + at
    assert np.all(out[1][sel] == 0.0)
    assert np.all(out[0][sel] > 0.0)
