"""Pins for the contour quadrature (Sec. 2.2-2.3): inversion of transforms
with known originals, at the convergence rate the paper states
(O(e^{-c N_z}), c = log 3.89)."""
import numpy as np
import pytest

from oracle import contour


@pytest.mark.parametrize("a", [0.0, 0.05, 1.0, 7.5, 50.0])
@pytest.mark.parametrize("t", [10.0, 100.0, 1e3, 1e4])
def test_inverse_of_one_over_z_plus_a(a, t):
    # L{e^{-a t}} = 1/(z + a)
    approx = contour.invert_scalar(lambda z: 1.0 / (z + a), t, 24)
    assert abs(approx - np.exp(-a * t)) < 1e-12


@pytest.mark.parametrize("t", [1.0, 10.0, 1e4])
def test_unit_step(t):
    # L{1} = 1/z
    assert abs(contour.invert_scalar(lambda z: 1.0 / z, t, 16) - 1.0) < 3e-9


def test_ramp_and_oscillation():
    # L{t} = 1/z^2 ; L{sin(w t)} = w / (z^2 + w^2) (pole pair inside the contour)
    t = 3.0
    assert abs(contour.invert_scalar(lambda z: 1.0 / z ** 2, t, 24) - t) < 1e-11
    w = 0.7
    assert abs(contour.invert_scalar(lambda z: w / (z ** 2 + w ** 2), t, 32) - np.sin(w * t)) < 1e-9


def test_convergence_rate_3_89():
    """max error over a and t of inverting 1/(z + a) decays like 3.89^{-N_z}."""
    errs = []
    Ns = [8, 12, 16, 20]
    for N in Ns:
        e = 0.0
        for t in (10.0, 100.0, 1e3, 1e4):
            for a in (0.0, 0.01, 0.1, 1.0, 10.0, 50.0):
                e = max(e, abs(contour.invert_scalar(lambda z: 1.0 / (z + a), t, N) - np.exp(-a * t)))
        errs.append(e)
    errs = np.array(errs)
    rate = np.exp(-np.polyfit(Ns, np.log(errs), 1)[0])
    assert 3.3 < rate < 4.6, (rate, errs)
    # and the absolute level: within a modest constant of 3.89^{-N}
    assert np.all(errs < 30.0 * 3.89 ** (-np.array(Ns, dtype=float)))
    assert errs[2] < 1e-8   # N_z = 16 reaches 1e-8, which config 1 relies on


def test_full_vs_half_sum():
    t = 50.0
    F = lambda z: 1.0 / (z + 0.3) + 2.0 / (z + 0.01)
    z, w = contour.nodes_weights(t, 20, half=False)
    full = np.sum(w * F(z))
    assert abs(full.imag) < 1e-13
    assert abs(full.real - contour.invert_scalar(F, t, 20)) < 1e-13


def test_nodes_are_conjugate_pairs_and_scale_with_Nz_over_t():
    zf, _ = contour.nodes_weights(7.0, 16, half=False)
    d = np.abs(zf[:, None] - np.conj(zf)[None, :]).min(axis=1)
    assert d.max() < 1e-12
    z1, _ = contour.nodes_weights(10.0, 16)
    z2, _ = contour.nodes_weights(20.0, 16)
    assert np.allclose(z1, 2.0 * z2)
    z3, _ = contour.nodes_weights(10.0, 32)
    assert np.all(z3.imag > 0)
    # contour encloses the negative real axis: left end well left of 0, crossing right of 0
    zf16, _ = contour.nodes_weights(1.0, 16, half=False)
    assert zf16.real.min() < -10 and zf16.real.max() > 0


def test_tau_schedule():
    z = np.array([1 + 1j, -2 + 0.5j, 3 + 0.1j])
    s = contour.tau_schedule(z, "flexible", 12)
    assert list(s[:5]) == [-2 + 0.5j] * 3 + [3 + 0.1j] * 2
    assert list(s[5:10]) == list(s[:5])
    assert np.all(contour.tau_schedule(z, "single", 4) == -2 + 0.5j)
