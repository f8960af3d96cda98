"""Pins of the oracle's Zou-He boundaries against Appendix B as printed."""
import numpy as np
import pytest

from oracle import oracle as O


def box_oracle(shape, periodic, axis, zeta_r=0.7, rho_in=1.03, rho_out=0.98):
    rng = np.random.default_rng(11)
    solid = np.zeros(shape, np.uint8)
    o = O.Oracle(19, solid, periodic)
    _, w, _ = O.lattice(19)
    f = (w[None, :, None, None, None]
         * (0.5 + rng.random((2, 19) + shape)))
    o.pops = f
    o.set_params(zou_he=0, flow_axis=axis)
    raw = o.stream_only()
    o.set_params(zou_he=1, flow_axis=axis, rho_in=rho_in, rho_out=rho_out,
                 zeta_r=zeta_r)
    zh = o.stream_only()
    return raw, zh


def test_generic_axis_z_is_appendix_B():
    """Flow along z: the rebuilt populations must equal Eqs. (B.1)-(B.8) at
    the inlet and (B.9)-(B.18) at the outlet, written out here as printed."""
    shape = (6, 4, 5)  # (nz, ny, nx)
    zeta = (0.7, 0.3)
    rho_in, rho_out = 1.03, 0.98
    raw, zh = box_oracle(shape, (True, True, False), 2, zeta[0], rho_in, rho_out)
    nz = shape[0]
    for s in range(2):
        f = raw[s, :, 0]  # (19, ny, nx) at z = 0
        u = rho_in * zeta[s] - (f[0] + f[1] + f[2] + f[3] + f[4] + f[7] + f[8]
                                + f[9] + f[10] + 2 * (f[6] + f[13] + f[14]
                                                      + f[17] + f[18]))
        Nx = 0.5 * (f[1] + f[7] + f[9] - (f[2] + f[8] + f[10]))
        Ny = 0.5 * (f[3] + f[7] + f[8] - (f[4] + f[9] + f[10]))
        expect = f.copy()
        expect[5] = f[6] + u / 3
        expect[11] = f[14] + u / 6 - Nx
        expect[12] = f[13] + u / 6 + Nx
        expect[15] = f[18] + u / 6 - Ny
        expect[16] = f[17] + u / 6 + Ny
        np.testing.assert_allclose(zh[s, :, 0], expect, rtol=0, atol=1e-15)
    ft = raw[0, :, nz - 1] + raw[1, :, nz - 1]
    ut = -rho_out + (ft[0] + ft[1] + ft[2] + ft[3] + ft[4] + ft[7] + ft[8]
                     + ft[9] + ft[10] + 2 * (ft[5] + ft[11] + ft[12] + ft[15]
                                             + ft[16]))
    rr = raw[0, :, nz - 2].sum(0)
    rb = raw[1, :, nz - 2].sum(0)
    phi_out = (rr - rb) / (rr + rb)                          # Eq. (39)
    chi = (0.5 * (1 + phi_out), 0.5 * (1 - phi_out))         # (B.12), (B.13)
    for s in range(2):
        f = raw[s, :, nz - 1]
        Nx = 0.5 * (f[1] + f[7] + f[9] - (f[2] + f[8] + f[10]))
        Ny = 0.5 * (f[3] + f[7] + f[8] - (f[4] + f[9] + f[10]))
        uc = ut * chi[s]
        expect = f.copy()
        expect[6] = f[5] - uc / 3
        expect[13] = f[12] - uc / 6 - Nx
        expect[14] = f[11] - uc / 6 + Nx
        expect[17] = f[16] - uc / 6 - Ny
        expect[18] = f[15] - uc / 6 + Ny
        np.testing.assert_allclose(zh[s, :, nz - 1], expect, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(zh[:, :, 1:nz - 1], raw[:, :, 1:nz - 1])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_prescribed_densities_and_zero_tangential_momentum(axis):
    shape = (6, 7, 8)
    periodic = [True, True, True]
    periodic[axis] = False
    zeta_r, rho_in, rho_out = 0.8, 1.02, 0.97
    raw, zh = box_oracle(shape, tuple(periodic), axis, zeta_r, rho_in, rho_out)
    e, _, _ = O.lattice(19)
    sl_in = [slice(None)] * 3
    sl_out = [slice(None)] * 3
    ax_np = 2 - axis
    sl_in[ax_np] = 0
    sl_out[ax_np] = shape[ax_np] - 1
    fin = zh[(slice(None), slice(None)) + tuple(sl_in)]
    fout = zh[(slice(None), slice(None)) + tuple(sl_out)]
    np.testing.assert_allclose(fin[0].sum(0), rho_in * zeta_r, atol=1e-14)
    np.testing.assert_allclose(fin[1].sum(0), rho_in * (1 - zeta_r), atol=1e-14)
    np.testing.assert_allclose(fout.sum((0, 1)), rho_out, atol=1e-14)
    for t in range(3):
        if t == axis:
            continue
        for s in range(2):
            np.testing.assert_allclose(np.tensordot(e[:, t], fin[s], 1), 0,
                                       atol=1e-15)
            np.testing.assert_allclose(np.tensordot(e[:, t], fout[s], 1), 0,
                                       atol=1e-15)


def test_d2q9_zou_he_densities():
    rng = np.random.default_rng(12)
    solid = np.zeros((1, 6, 9), np.uint8)
    o = O.Oracle(9, solid, (False, True, True))
    _, w, _ = O.lattice(9)
    o.pops = w[None, :, None, None, None] * (0.5 + rng.random((2, 9, 1, 6, 9)))
    o.set_params(zou_he=1, flow_axis=0, rho_in=1.02, rho_out=0.99, zeta_r=1.0)
    zh = o.stream_only()
    np.testing.assert_allclose(zh[0, :, 0, :, 0].sum(0), 1.02, atol=1e-14)
    np.testing.assert_allclose(zh[1, :, 0, :, 0].sum(0), 0.0, atol=1e-14)
    np.testing.assert_allclose(zh[:, :, 0, :, 8].sum((0, 1)), 0.99, atol=1e-14)
