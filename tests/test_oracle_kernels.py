"""Pins of the oracle's Peskin kernels, interpolation J and spreading S.

What the paper fixes (Sec. II.A Eq. dV_JS / adjoint_cond; Sec. III.A.1
Eq. JS_invariance and the text after it): unit sum, zero first moment and a
position-independent sum of squares; dV = 8 dV_f for the 3-point kernel; S is the
dV_f^-1 weighted transpose of J.  Closed-form values are Peskin's.
"""
import itertools

import numpy as np
import pytest

from oracle import icm


@pytest.mark.parametrize("kernel", [3, 4])
def test_moment_conditions(kernel):
    rng = np.random.default_rng(11)
    s = rng.uniform(-50.0, 50.0, size=10_000)
    nodes, w = icm.stencil_1d(s, kernel)
    r = s[:, None] - nodes
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose((r * w).sum(axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose((w ** 2).sum(axis=1), icm.kernel_sum_sq(kernel), atol=1e-14)


def test_four_point_even_odd_condition():
    """The 4-point kernel also has equal even and odd sums (1/2 each)."""
    s = np.random.default_rng(12).uniform(-9.0, 9.0, size=5000)
    nodes, w = icm.stencil_1d(s, 4)
    even = np.where(nodes % 2 == 0, w, 0.0).sum(axis=1)
    np.testing.assert_allclose(even, 0.5, atol=1e-14)


def test_closed_form_values_and_support():
    np.testing.assert_allclose(icm.phi3(np.array([0.0, 1.0, 0.5])), [2 / 3, 1 / 6, 0.5], atol=1e-15)
    # at integer r the 4-point nodes 0, +-1 carry 1/2, 1/4, 1/4 (unit sum, sum of squares 3/8)
    np.testing.assert_allclose(icm.phi4(np.array([0.0, 1.0])), [0.5, 0.25], atol=1e-15)
    assert icm.phi3(np.array([1.5, 1.6, -2.0])).tolist() == [0.0, 0.0, 0.0]
    assert icm.phi4(np.array([2.0, 2.5, -3.0])).tolist() == [0.0, 0.0, 0.0]
    # continuity at the branch points
    for f, b in ((icm.phi3, 0.5), (icm.phi4, 1.0)):
        lo, hi = f(np.array([b - 1e-12, b + 1e-12]))
        assert abs(lo - hi) < 1e-9


def test_blob_volume_three_point_is_eight_cells():
    """Sec. III.A.1: the 3-point kernel gives dV = 8 dV_f in three dimensions."""
    for h in (1.0, 0.5, 2.0):
        assert icm.blob_volume(3, h) == pytest.approx(8.0 * h ** 3, rel=1e-15)
    assert icm.blob_volume(4, 1.0) == pytest.approx((8.0 / 3.0) ** 3, rel=1e-15)


def _brute_force_interp(field, q, kernel, h):
    """J v by visiting every node of the grid with the minimum-image offset."""
    nz, ny, nx = field.shape[1:]
    sizes = (nx, ny, nz)
    out = np.zeros(3)
    for comp in range(3):
        off = icm.component_offsets(comp)
        for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
            wgt = 1.0
            for ax, idx in enumerate((i, j, k)):
                pos = (idx + off[ax]) * h
                d = q[ax] - pos
                L = sizes[ax] * h
                d -= L * np.round(d / L)
                wgt *= float(icm.phi(kernel, np.array([d / h]))[0])
            out[comp] += wgt * field[comp, k, j, i]
    return out


@pytest.mark.parametrize("kernel", [3, 4])
def test_interpolation_against_brute_force(kernel):
    """Node selection, staggering offsets and periodic wrap of J on an 8^3 grid."""
    rng = np.random.default_rng(13)
    h = 0.7
    field = rng.standard_normal((3, 8, 8, 8))
    qs = np.vstack([rng.uniform(0, 8 * h, size=(3, 3)),
                    [[0.0, 0.0, 0.0], [8 * h - 1e-9, 0.5 * h, 0.25 * h], [0.5 * h, 1.5 * h, 7.5 * h]]])
    got = icm.interpolate(field, qs, kernel, h)
    for b in range(qs.shape[0]):
        np.testing.assert_allclose(got[b], _brute_force_interp(field, qs[b], kernel, h), atol=1e-13)


@pytest.mark.parametrize("kernel", [3, 4])
def test_interpolation_is_exact_for_linear_fields(kernel):
    """Zeroth and first moments make J exact for linear functions sampled at the faces."""
    h = 0.5
    n = 16
    grad = np.array([[0.3, -1.1, 0.7], [2.0, 0.1, -0.4], [-0.6, 0.9, 1.3]])
    field = np.zeros((3, n, n, n))
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for c in range(3):
        off = icm.component_offsets(c)
        pos = [(i + off[0]) * h, (j + off[1]) * h, (k + off[2]) * h]
        field[c] = 0.25 + sum(grad[c, a] * pos[a] for a in range(3))
    rng = np.random.default_rng(14)
    q = rng.uniform(3 * h, (n - 3) * h, size=(20, 3))   # away from the periodic seam
    got = icm.interpolate(field, q, kernel, h)
    want = 0.25 + q @ grad.T
    np.testing.assert_allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("kernel", [3, 4])
def test_spreading_is_weighted_adjoint_of_interpolation(kernel):
    """Eq. adjoint_cond: (J v) . F = dV_f sum_k v_k . (S F)_k."""
    rng = np.random.default_rng(15)
    h = 0.8
    shape = (10, 8, 12)
    v = rng.standard_normal((3,) + shape)
    q = rng.uniform(0, 1, size=(7, 3)) * np.array([12, 8, 10]) * h
    F = rng.standard_normal((7, 3))
    lhs = np.sum(icm.interpolate(v, q, kernel, h) * F)
    rhs = h ** 3 * np.sum(v * icm.spread(F, q, kernel, h, shape))
    assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("kernel", [3, 4])
def test_JS_is_inverse_blob_volume(kernel):
    """Eq. dV_JS: J S = dV^-1 I at every position (translational invariance)."""
    rng = np.random.default_rng(16)
    h = 1.0
    shape = (12, 12, 12)
    dv = icm.blob_volume(kernel, h)
    for q in rng.uniform(0, 12, size=(25, 3)):
        F = rng.standard_normal(3)
        got = icm.interpolate(icm.spread(F[None], q[None], kernel, h, shape), q[None], kernel, h)[0]
        np.testing.assert_allclose(got, F / dv, rtol=1e-13, atol=1e-15)


def test_spread_total_force():
    """sum_k (S F)_k dV_f = sum_i F_i (unit sum of the kernel)."""
    rng = np.random.default_rng(17)
    shape = (8, 9, 10)
    q = rng.uniform(0, 8, size=(5, 3))
    F = rng.standard_normal((5, 3))
    f = icm.spread(F, q, 4, 1.0, shape)
    np.testing.assert_allclose(f.reshape(3, -1).sum(axis=1), F.sum(axis=0), atol=1e-13)
