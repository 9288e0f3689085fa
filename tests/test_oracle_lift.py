"""Pins of the lifting / projection oracle (oracle/lift.py) against what the paper and the
mathematics fix: the field lift conserves |v| under the projection, the reconstruction inverts the
lift on bin-centred angles and quantises other angles to within half a bin, the lift commutes with
a quarter turn of the plane, and the signed interpolation is odd in its inputs and reduces to a
closed form for identical inputs (dense kernel matrix from the group law)."""
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle
from tests import refmath

if os.environ.get("SE2OT_ORACLE_LIFT"):
    # a planted-mistake copy of oracle/lift.py, loaded in the oracle package (the mutation test)
    _spec = importlib.util.spec_from_file_location("oracle._lift_under_test", os.environ["SE2OT_ORACLE_LIFT"])
    lift = importlib.util.module_from_spec(_spec)
    lift.__package__ = "oracle"
    _spec.loader.exec_module(lift)
else:
    from oracle import lift

RNG = np.random.default_rng(4242)
W = (1.0, 3.0, 0.5)


def _field(ny, nx, angles=None):
    mag = RNG.uniform(0.1, 1.0, size=(ny, nx))
    psi = RNG.uniform(-math.pi, math.pi, size=(ny, nx)) if angles is None else angles
    return np.stack([mag * np.cos(psi), mag * np.sin(psi)], axis=-1), mag, psi


def test_projection_of_the_lift_is_the_magnitude():
    v, mag, _ = _field(7, 9)
    U = lift.lift_field(v, 16)
    np.testing.assert_allclose(lift.project(U), mag, rtol=1e-14)
    assert (np.count_nonzero(U, axis=-1) == 1).all()


@pytest.mark.parametrize("nt", [4, 8, 16])
def test_reconstruction_inverts_the_lift_on_bin_centres(nt):
    k = RNG.integers(0, nt, size=(6, 5))
    v, _, _ = _field(6, 5, angles=2 * math.pi * k / nt)
    np.testing.assert_allclose(lift.reconstruct_field(lift.lift_field(v, nt)), v, atol=1e-14)


def test_reconstruction_quantises_to_half_a_bin_and_ties_go_up():
    nt = 16
    v, mag, psi = _field(8, 8)
    r = lift.reconstruct_field(lift.lift_field(v, nt))
    np.testing.assert_allclose(np.hypot(r[..., 0], r[..., 1]), mag, rtol=1e-14)
    d = np.angle(np.exp(1j * (np.arctan2(r[..., 1], r[..., 0]) - psi)))
    assert np.abs(d).max() <= math.pi / nt + 1e-12
    half = np.array([[[math.cos(math.pi / nt), math.sin(math.pi / nt)]]])   # exactly between bins 0 and 1
    assert lift.lift_field(half, nt)[0, 0, 1] == 1.0


def test_lift_commutes_with_a_quarter_turn():
    """Rotating the field by 90 degrees about the grid centre (positions and vectors) lifts to
    the quarter-turned score with orientations shifted by nt/4."""
    nt = 8
    v, _, _ = _field(6, 6)
    # out[y', x'] with x' = N-1-y, y' = x, vector rotated by +90 degrees
    vr = np.flip(np.swapaxes(v, 0, 1), axis=1)
    vr = np.stack([-vr[..., 1], vr[..., 0]], axis=-1)
    np.testing.assert_allclose(lift.lift_field(vr, nt), refmath.rot90(lift.lift_field(v, nt)), atol=1e-14)


def _dense_K(g):
    return np.exp(refmath.dense_log_kernel(g.nx, g.ny, g.nth, g.r,
                                           lambda x, y, t: oracle.rho_b2(x, y, t, (g.w1, g.w2, g.w3)),
                                           g.eps, g.periodic))


def test_signed_interpolation_is_odd_and_has_the_identical_input_closed_form():
    g = oracle.Grid(6, 6, 4, 2, W, 0.05)
    U = RNG.normal(size=g.shape)
    V = RNG.normal(size=g.shape)
    b = lift.interpolate_signed(g, U, V, 0.3, 12)
    np.testing.assert_allclose(lift.interpolate_signed(g, -U, -V, 0.3, 12), -b, rtol=1e-14)
    # identical inputs: every barycenter iterate is K(nu / K 1) (nu = the normalised part)
    K = _dense_K(g)
    k1 = K @ np.ones(g.V)
    want = np.zeros(g.shape[:2])
    for part, sign in ((np.maximum(U, 0), 1.0), (-np.minimum(U, 0), -1.0)):
        m = part.sum()
        nu = part + 1e-6 * part.max()          # the floored, normalised part
        nu = nu / nu.sum()
        phi = (K @ (nu.reshape(-1) / k1)).reshape(g.shape)
        want += sign * m * phi.sum(axis=-1)
    np.testing.assert_allclose(lift.interpolate_signed(g, U, U, 0.7, 5), want, rtol=1e-11, atol=1e-13)


def test_signed_interpolation_at_t0_uses_the_first_inputs_masses():
    """t = 0: the weights are (1, 0), so every barycenter iterate of a part is K(nu0 / K 1) (the
    one-hot closed form of the scaling iterations), and the result is m0+ P(K(nu0+ / K 1)) -
    m0- P(K(nu0- / K 1)) with the first input's part masses, whatever the second input is."""
    g = oracle.Grid(6, 6, 4, 2, W, 0.05)
    U = RNG.normal(size=g.shape)
    V = 3.0 * RNG.normal(size=g.shape) + 0.5        # other part masses on the second side
    K = _dense_K(g)
    k1 = K @ np.ones(g.V)
    want = np.zeros(g.shape[:2])
    for part, sign in ((np.maximum(U, 0), 1.0), (-np.minimum(U, 0), -1.0)):
        nu = part + 1e-6 * part.max()
        nu = nu / nu.sum()
        want += sign * part.sum() * (K @ (nu.reshape(-1) / k1)).reshape(g.shape).sum(axis=-1)
    np.testing.assert_allclose(lift.interpolate_signed(g, U, V, 0.0, 6), want, rtol=1e-11, atol=1e-13)
