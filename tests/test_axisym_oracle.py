"""Pins of the oracle's axisymmetric form (Sec. 2, Eqs. gpe-pressure-two-phase-axisym,
gpe-momentum-two-phase-axisym-z and -r, che-axisym, div-v-axisym, chem-pot-axisym).

x is the radius r (axis on the low-x side), y the axis coordinate z.  The pins are:
- exactness on quadratics in r of every term the axisymmetric form adds (the central
  differences and the isotropic stencils are exact there, so the discrete operator
  must return the cylindrical operator's value to rounding);
- the Hagen-Poiseuille profile u_z = G (R^2 - r^2) / (4 nu), reached at second order;
- the decay rate M k^2 (8a + kappa k^2) of a small Bessel mode J0(k r) of phi about
  phi = 1, the linearised Cahn-Hilliard equation in cylindrical coordinates, reached
  at second order.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2011_00814_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _prm(nx=16, ny=4, dx=0.5, **kw):
    kw.setdefault("bc", ("freeslip", "periodic", "periodic"))
    return inputs.base_params(2, nx, ny, dx=dx, rhoL=1.3, rhoG=1.3, etaL=0.7, etaG=0.7, sigma=0.0,
                              axisym=1, **kw)


def _radii(prm):
    i = np.arange(prm["nx"])
    rc = np.broadcast_to((i + 0.5) * prm["dx"], (prm["ny"], prm["nx"]))
    rf = np.broadcast_to(i * prm["dx"], (prm["ny"], prm["nx"]))
    return rc, rf


def _state(prm, **f):
    shp = (prm["ny"], prm["nx"])
    st = {k: np.zeros(shp) for k in ("p", "u", "v")}
    st["phi"] = np.ones(shp)
    st.update({k: np.array(v, dtype=float) for k, v in f.items()})
    st.setdefault("mu", oracle.mu(prm, st["phi"]))
    return st


def test_mu_and_ch_rate_exact_on_r_squared():
    # lap(r^2) + (1/r) d(r^2)/dr = 2 + 2 = 4 in the cylindrical Laplacian
    prm = _prm()
    rc, _ = _radii(prm)
    c = 1e-3
    phi = 1.0 + c * rc**2
    a, kappa = 3.0 / (4.0 * prm["W"]), 3.0 * prm["W"] / 8.0
    want = 4.0 * a * phi * (phi * phi - 1.0) - kappa * 4.0 * c
    got = oracle.mu(prm, phi)
    # the outer column mirrors r^2 about the wall, where it is not even
    assert np.max(np.abs(got[:, :-1] - want[:, :-1])) < 1e-13
    mu = c * rc**2
    L = oracle.ch_rhs(prm, np.ones_like(mu), mu, [np.zeros_like(mu)] * 2)
    assert np.max(np.abs(L[:, :-1] - prm["M"] * 4.0 * c)) < 1e-14
    # the planar operator misses half of it: the pin is sensitive to the 1/r term
    flat = dict(prm, axisym=0)
    assert abs(oracle.ch_rhs(flat, np.ones_like(mu), mu, [np.zeros_like(mu)] * 2)[0, 3]
               - prm["M"] * 2.0 * c) < 1e-14


def test_pressure_rate_exact():
    prm = _prm()
    rc, rf = _radii(prm)
    nu, rho, cs2 = 0.7 / 1.3, 1.3, prm["cs"] ** 2
    # diffusion: d/dr(nu dp/dr) + (nu/r) dp/dr of p = c r^2 is 4 nu c
    c = 0.01
    Lp = oracle.flow_rhs(prm, _state(prm, p=c * rc**2))[0]
    assert np.max(np.abs(Lp[:, :-1] - 4.0 * nu * c)) < 1e-14
    # divergence: u_r = c r has div u = du_r/dr + u_r/r = 2c
    Lp = oracle.flow_rhs(prm, _state(prm, u=c * rf))[0]
    assert np.max(np.abs(Lp[:, :-1] + rho * cs2 * 2.0 * c)) < 1e-14


def test_axial_momentum_rate_exact():
    # eta (d2/dr2 + (1/r) d/dr) u_z of u_z = c r^2 is 4 eta c
    prm = _prm()
    rc, _ = _radii(prm)
    c = 0.01
    Lv = oracle.flow_rhs(prm, _state(prm, v=c * rc**2))[2]
    assert np.max(np.abs(Lv[:, :-1] - 4.0 * 0.7 * c / 1.3)) < 1e-14


def test_radial_momentum_rate_exact():
    # 2 d/dr(eta du_r/dr) + (eta/r)(du_r/dr - u_r/r) of u_r = c r^2 is (4 + 1) eta c;
    # the advection u_r du_r/dr is even in c and drops out of the odd part
    prm = _prm(bulk_visc=0)
    _, rf = _radii(prm)
    c = 0.01
    Lu_p = oracle.flow_rhs(prm, _state(prm, u=c * rf**2))[1]
    Lu_m = oracle.flow_rhs(prm, _state(prm, u=-c * rf**2))[1]
    odd = 0.5 * (Lu_p - Lu_m)
    assert np.all(odd[:, 0] == 0.0)  # the axis face is never updated
    assert np.max(np.abs(odd[:, 1:-1] - 5.0 * 0.7 * c / 1.3)) < 1e-14


@pytest.mark.parametrize("dx", [0.25, 0.125])
def test_bulk_term_uses_the_axisymmetric_divergence(dx):
    # d/dr(eta_b div u), div u = du_r/dr + u_r/r = 3 c r for u_r = c r^2: the bulk
    # contribution tends to 3 eta c at second order at a fixed radius
    errs = []
    for h in (dx, dx / 2):
        nx = int(round(4.0 / h))
        prm1, prm0 = _prm(nx=nx, dx=h), _prm(nx=nx, dx=h, bulk_visc=0)
        _, rf = _radii(prm1)
        st = _state(prm1, u=0.01 * rf**2)
        i = int(round(2.0 / h))  # the face at r = 2
        b = (oracle.flow_rhs(prm1, st)[1] - oracle.flow_rhs(prm0, st)[1])[0, i]
        errs.append(abs(b * 1.3 / (0.7 * 0.01) - 3.0))
    assert errs[0] < 0.01 and errs[1] < errs[0] / 3.5, errs


def _poiseuille_error(nx):
    R, nu, G = 1.0, 1.0, 1.0
    dx = R / nx
    prm = inputs.base_params(2, nx, 2, dx=dx, dt=0.1 * dx * dx / nu, cs=1.0, rhoL=1.0, rhoG=1.0,
                             etaL=nu, etaG=nu, sigma=0.0, g=(0.0, G, 0.0), rho_ref=0.0,
                             bc=("noslip", "periodic", "periodic"), axisym=1)
    rc, _ = _radii(prm)
    exact = G * (R * R - rc**2) / (4.0 * nu)
    st = oracle.step(prm, _state(prm, v=exact), int(round(2.0 / prm["dt"])))
    assert np.max(np.abs(st["u"])) == 0.0 and np.max(np.abs(st["p"])) == 0.0
    return np.max(np.abs(st["v"] - exact)) / np.max(exact)


def test_hagen_poiseuille_second_order():
    e8, e16 = _poiseuille_error(8), _poiseuille_error(16)
    assert e16 < 5e-3 and e16 < e8 / 3.5, (e8, e16)


def _bessel_decay_error(nx):
    from scipy.special import j0, jn_zeros

    R, W, M = 1.0, 1.0, 0.01
    dx = R / nx
    k = jn_zeros(1, 1)[0] / R  # J0'(kR) = 0: no flux through the outer wall
    a, kappa = 3.0 / (4.0 * W), 3.0 * W / 8.0
    lam = M * k * k * (8.0 * a + kappa * k * k)
    lam_max = 8.0 / (dx * dx)
    dt = 0.5 / (M * lam_max * (8.0 * a + kappa * lam_max))
    t_end = 0.5
    n = int(math.ceil(t_end / dt))
    dt = t_end / n
    prm = inputs.base_params(2, nx, 2, dx=dx, dt=dt, cs=1.0, rhoL=1.0, rhoG=1.0, etaL=0.1, etaG=0.1,
                             sigma=0.0, M=M, W=W, bc=("freeslip", "periodic", "periodic"), axisym=1,
                             ch_scheme=2)
    rc, _ = _radii(prm)
    eps = 1e-7
    mode = j0(k * rc)
    st = oracle.step(prm, _state(prm, phi=1.0 + eps * mode), n)
    amp = np.sum(rc * (st["phi"] - 1.0) * mode) / np.sum(rc * eps * mode * mode)
    rate = -math.log(amp) / t_end
    return abs(rate / lam - 1.0)


def test_ch_bessel_mode_decay_second_order():
    e8, e16 = _bessel_decay_error(8), _bessel_decay_error(16)
    assert e16 < 1e-2 and e16 < e8 / 3.0, (e8, e16)
