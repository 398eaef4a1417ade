"""Pins of the oracle's hand-written adjoint of the COLA model (transpose of §2.1/§2.2 with continuous
CIC weights): every linear or linearised piece passes a dot-product test against central finite
differences of the forward, and the whole gradient of the density loss with respect to the white
noise matches central finite differences (eps = 1e-3) on 32 random lattice sites."""

import numpy as np
import pytest

import cola_inputs
from oracle import adjoint, cosmology, lpt
from oracle.cosmology import Params

P = Params(box=128.0, np_side=8, nmesh=16, nstep=10)
NGRID = 8


def _fd_dot(fun, x0, direction, lam, h):
    plus, minus = fun(x0 + h * direction), fun(x0 - h * direction)
    return float(np.sum(lam * (plus - minus)) / (2 * h))


def test_grid_delta_adjoint_dot_product():
    rng = np.random.default_rng(1)
    s = rng.normal(0, 2.0, (3, 8 ** 3))
    lam = rng.normal(size=(NGRID,) * 3)
    ds = rng.normal(size=s.shape)
    fd = _fd_dot(lambda x: adjoint.grid_delta(x, 8, 16, NGRID), s, ds, lam, 1e-6)
    an = float(np.sum(adjoint.grid_delta_adjoint(s, 8, 16, NGRID, lam) * ds))
    assert an == pytest.approx(fd, rel=1e-6)


def test_pm_force_adjoint_dot_product():
    rng = np.random.default_rng(2)
    s = rng.normal(0, 1.5, (3, 8 ** 3))
    lam = rng.normal(size=s.shape)
    ds = rng.normal(size=s.shape)
    fd = _fd_dot(lambda x: adjoint.pm_force_exact(x, 8, 16, 1.7), s, ds, lam, 1e-6)
    an = float(np.sum(adjoint.pm_force_adjoint(s, lam, 8, 16, 1.7) * ds))
    assert an == pytest.approx(fd, rel=1e-6)


def test_lpt_adjoint_dot_product():
    rng = np.random.default_rng(3)
    w = cola_inputs.white_noise(8, seed=2).astype(np.float64)
    l1, l2 = rng.normal(size=(3, 8 ** 3)), rng.normal(size=(3, 8 ** 3))
    dw = rng.normal(size=w.shape)
    h = 1e-4

    def both(x):
        a, b = lpt.displacements(x, P)
        return np.concatenate([a, b])

    fd = _fd_dot(both, w, dw, np.concatenate([l1, l2]), h)
    an = float(np.sum(adjoint.lpt_adjoint(w, l1, l2, P) * dw))
    assert an == pytest.approx(fd, rel=1e-7)


def test_gradient_matches_central_differences_on_32_sites():
    w = cola_inputs.white_noise(8, seed=4).astype(np.float64)
    target = adjoint.grid_delta(adjoint.forward(cola_inputs.white_noise(8, seed=5), P)["s"], 8, 16, NGRID)
    lval, grad = adjoint.gradient(w, P, NGRID, target)
    assert lval == pytest.approx(adjoint.loss(w, P, NGRID, target), rel=1e-12)
    sites = np.random.default_rng(6).choice(w.size, 32, replace=False)
    eps = 1e-3
    fd = []
    for j in sites:
        e = np.zeros_like(w)
        e[j] = eps
        fd.append((adjoint.loss(w + e, P, NGRID, target) - adjoint.loss(w - e, P, NGRID, target)) / (2 * eps))
    fd = np.array(fd)
    err = np.abs(grad[sites] - fd) / np.abs(fd).max()
    assert err.max() < 2e-3, err.max()
    assert np.corrcoef(grad[sites], fd)[0, 1] > 0.9999
