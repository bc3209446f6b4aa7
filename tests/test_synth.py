"""The seeded synthetic inputs have the structure the input recipe states.

The generator feeds both the CUDA path and the oracle, so a mistake in it
would go unnoticed by the parity tests.  Checked here directly, in numpy,
from the definitions: the coarse face velocity is discretely divergence-free
on every coarse cell (periodic or walled, uniform or tanh-stretched z), the
wall-normal velocity vanishes on the plates (and on side walls), the field
is rescaled to the requested rms over all coarse faces, the draw is
reproducible from its seed, and the initial scalar is the conduction profile
plus Gaussian noise of the stated size.
"""
import numpy as np
import pytest

from paper_1805_03426_gb300 import synth


def _faces(nx, ny, nz, gamma):
    Xf = np.arange(nx + 1) / nx
    Yf = np.arange(ny + 1) / ny
    k = np.arange(nz + 1) / nz
    if gamma:
        Zf = 0.5 * (1.0 + np.tanh(gamma * (2.0 * k - 1.0)) / np.tanh(gamma))
    else:
        Zf = k.copy()
    return Xf, Yf, Zf


def _divergence(U, V, W, Xf, Yf, Zf, walls):
    """Net outward flux of every coarse cell over its volume."""
    DX, DY, DZ = np.diff(Xf), np.diff(Yf), np.diff(Zf)
    ay = DY[None, :, None] * DZ[:, None, None]          # area of an x-face
    ax = DX[None, None, :] * DZ[:, None, None]          # area of a y-face
    az = DX[None, None, :] * DY[None, :, None]          # area of a z-face
    if walls:
        fx = (U[:, :, 1:] - U[:, :, :-1]) * ay
        fy = (V[:, 1:, :] - V[:, :-1, :]) * ax
    else:
        fx = (np.roll(U, -1, axis=2) - U) * ay
        fy = (np.roll(V, -1, axis=1) - V) * ax
    fz = (W[1:] - W[:-1]) * az
    vol = DX[None, None, :] * DY[None, :, None] * DZ[:, None, None]
    return (fx + fy + fz) / vol


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("gamma", [0.0, 1.5])
def test_coarse_velocity_is_discretely_divergence_free(walls, gamma):
    nx, ny, nz = 16, 12, 10
    Xf, Yf, Zf = _faces(nx, ny, nz, gamma)
    U, V, W = synth.coarse_velocity(1805, Xf, Yf, Zf, rms=0.1, walls=walls)
    w = 1 if walls else 0
    assert U.shape == (nz, ny, nx + w) and V.shape == (nz, ny + w, nx) and W.shape == (nz + 1, ny, nx)
    div = _divergence(U, V, W, Xf, Yf, Zf, walls)
    # scale: the largest single-face flux over the smallest cell
    scale = max(np.abs(U).max() / np.diff(Xf).min(), np.abs(V).max() / np.diff(Yf).min(),
                np.abs(W).max() / np.diff(Zf).min())
    assert np.abs(div).max() <= 1e-13 * scale
    # and the field is not trivially zero
    assert np.abs(U).max() > 1e-3 and np.abs(V).max() > 1e-3 and np.abs(W).max() > 1e-3


@pytest.mark.parametrize("walls", [False, True])
def test_wall_normal_velocity_vanishes(walls):
    Xf, Yf, Zf = _faces(12, 12, 8, 1.5)
    U, V, W = synth.coarse_velocity(7, Xf, Yf, Zf, rms=0.2, walls=walls)
    assert np.all(W[0] == 0.0) and np.all(W[-1] == 0.0)
    if walls:
        assert np.all(U[:, :, 0] == 0.0) and np.all(U[:, :, -1] == 0.0)
        assert np.all(V[:, 0, :] == 0.0) and np.all(V[:, -1, :] == 0.0)


@pytest.mark.parametrize("rms", [0.1, 0.2])
def test_rms_over_all_coarse_faces(rms):
    Xf, Yf, Zf = _faces(16, 16, 12, 1.5)
    U, V, W = synth.coarse_velocity(11, Xf, Yf, Zf, rms=rms)
    got = np.sqrt(np.mean(U ** 2) + np.mean(V ** 2) + np.mean(W ** 2))
    assert abs(got - rms) <= 1e-14 * rms


def test_draws_are_reproducible_from_the_seed():
    Xf, Yf, Zf = _faces(8, 8, 6, 1.5)
    a = synth.coarse_velocity(3, Xf, Yf, Zf)
    b = synth.coarse_velocity(3, Xf, Yf, Zf)
    c = synth.coarse_velocity(4, Xf, Yf, Zf)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[0], c[0])


def test_initial_scalar_is_conduction_plus_noise():
    nz, ny, nx, noise = 24, 32, 32, 1e-2
    zf = _faces(1, 1, nz, 1.5)[2]
    zc = 0.5 * (zf[1:] + zf[:-1])
    T = synth.initial_scalar(5, zc, ny, nx, noise=noise)
    assert T.shape == (nz, ny, nx)
    dev = T - (0.5 - zc)[:, None, None]
    # N(0, noise^2) over 24576 draws: mean within ~5 standard errors, std within 3 %
    assert abs(dev.mean()) < 5 * noise / np.sqrt(dev.size)
    assert abs(dev.std() / noise - 1.0) < 0.03
    assert np.array_equal(T, synth.initial_scalar(5, zc, ny, nx, noise=noise))
