"""The explicit stability limits of `gpe2p_stability_limits` (host-only) against
the amplification factors of the linearised step.

For a uniform state the flow step multiplies every Fourier mode by
P3(dt A(theta)), A the symbol of the flow operator (derived by hand in
`test_oracle_pins.py` and pinned there against the oracle), and the CH step by
P2 or P4 of dt M lam (f'' - kappa lam).  Each limit is checked in a regime where
it is the binding one: just below it no mode grows, a little above it some
mode does.  The scan over theta is finer than the library's own.  Between
walls and in the axisymmetric form, where Fourier modes are not eigenmodes,
the same is checked against the eigenvalues of the oracle's own linearised
operator assembled on a small grid.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2011_00814_gb300 import build, gpe2p, inputs
from tests.test_oracle_pins import ch_polynomial, flow_symbol, iso_laplacian_symbol, rk3_amplification

pytestmark = pytest.mark.usefixtures("lib")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gpe2p.lib()


def _thetas(dim, n):
    ax = np.linspace(0.0, math.pi, n)
    if dim == 2:
        return [(a, b) for a in ax for b in ax]
    return [(a, b, c) for a in ax for b in ax for c in ax]


def _flow_growth(prm, dt, phi0=1.0, n=25):
    """Largest spectral radius of the RK3 amplification over the theta scan."""
    worst = 0.0
    for th in _thetas(prm["dim"], n):
        G = rk3_amplification(dt * flow_symbol(prm, th, phi0))
        worst = max(worst, np.max(np.abs(np.linalg.eigvals(G))))
    return worst


VISCOUS_CASES = [(2, 1), (2, 0), (3, 1), (3, 0)]


@pytest.mark.parametrize("dim,bulk", VISCOUS_CASES)
def test_viscous_limit_is_the_real_axis_bound(dim, bulk):
    # one phase, slow sound: the viscous modes bind, the acoustic limit is far away
    prm = inputs.base_params(dim, 8, 8, 8, dx=0.5, cs=0.01, rhoL=1.3, rhoG=1.3, etaL=0.2, etaG=0.2,
                             bulk_visc=bulk)
    ac, vi, ch = gpe2p.stability_limits(prm)
    assert vi < 0.05 * ac
    assert _flow_growth(prm, 0.999 * vi) <= 1.0 + 1e-9
    assert _flow_growth(prm, 1.03 * vi) > 1.0 + 1e-4


@pytest.mark.parametrize("dim,pavg", [(2, 1), (2, 0), (3, 1), (3, 0)])
def test_acoustic_limit_is_the_imaginary_axis_bound(dim, pavg):
    # no viscosity: the acoustic modes sit on the imaginary axis
    prm = inputs.base_params(dim, 8, 8, 8, dx=0.5, cs=1.7, rhoL=1.3, rhoG=1.3, etaL=0.0, etaG=0.0,
                             p_average=pavg)
    ac, vi, ch = gpe2p.stability_limits(prm)
    assert math.isinf(vi)
    assert _flow_growth(prm, 0.999 * ac) <= 1.0 + 1e-9
    assert _flow_growth(prm, 1.03 * ac) > 1.0 + 1e-4


@pytest.mark.parametrize("dim,iso,scheme", [(2, 9, 2), (2, 9, 4), (3, 15, 4), (3, 19, 2), (3, 27, 4)])
def test_ch_limit_is_the_real_axis_bound(dim, iso, scheme):
    prm = inputs.base_params(dim, 8, 8, 8, dx=0.5, M=0.02, W=1.5, iso=iso, ch_scheme=scheme)
    _, _, lim = gpe2p.stability_limits(prm)
    a_, kappa = 3.0 / (4.0 * prm["W"]), 3.0 * prm["W"] / 8.0
    fpp = 8.0 * a_  # f''(phi) = 4a (3 phi^2 - 1) is largest in the bulk, |phi| = 1

    def growth(dt):
        worst = 0.0
        for th in _thetas(dim, 49 if dim == 2 else 25):
            lam = iso_laplacian_symbol(dim, iso, th, prm["dx"])
            worst = max(worst, abs(ch_polynomial(dt * prm["M"] * lam * (fpp - kappa * lam), scheme)))
        return worst

    assert growth(0.999 * lim) <= 1.0 + 1e-9
    assert growth(1.03 * lim) > 1.0 + 1e-4


# ---------------------------------------------------------------------------
# walls and the axisymmetric form: the spectrum of the oracle's own operator
# ---------------------------------------------------------------------------
# Between walls and in the axisymmetric form the Fourier modes are not
# eigenmodes.  There the linear operator of the oracle's rates about a uniform
# state at rest is assembled column by column on a small grid, and the limits
# are checked against its eigenvalues.

def _flow_jacobian(prm, phi0=1.0):
    import oracle
    dim = prm["dim"]
    shp = (prm["nz"], prm["ny"], prm["nx"]) if dim == 3 else (prm["ny"], prm["nx"])
    names = ["p", "u", "v", "w"][: dim + 1]
    N = int(np.prod(shp))
    phi = np.full(shp, phi0)
    mu = oracle.mu(prm, phi)
    J = np.zeros(((dim + 1) * N, (dim + 1) * N))
    for a, nm in enumerate(names):
        for q in range(N):
            st = {k: np.zeros(shp) for k in names}
            st[nm].flat[q] = 1.0  # the rates are linear at rest (convection is quadratic)
            st["phi"], st["mu"] = phi, mu
            J[:, a * N + q] = np.concatenate([r.ravel() for r in oracle.flow_rhs(prm, st)])
    return np.linalg.eigvals(J)


def _ch_jacobian(prm, phi0=1.0, h=1e-6):
    import oracle
    shp = (prm["ny"], prm["nx"])
    phi = np.full(shp, phi0)
    uh = [np.zeros(shp), np.zeros(shp)]
    r0 = oracle.ch_rhs(prm, phi, oracle.mu(prm, phi), uh)
    J = np.zeros((phi.size, phi.size))
    for q in range(phi.size):
        p = phi.copy()
        p.flat[q] += h
        J[:, q] = ((oracle.ch_rhs(prm, p, oracle.mu(prm, p), uh) - r0) / h).ravel()
    return np.linalg.eigvals(J)


def _rk3(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


BOUNDED_FLOW_CASES = [
    (2, ("noslip", "noslip", "periodic"), 0),
    (2, ("freeslip", "periodic", "periodic"), 0),
    (2, ("noslip", "noslip", "periodic"), 1),
    (2, ("freeslip", "freeslip", "periodic"), 1),
    (3, ("noslip", "periodic", "freeslip"), 0),
]


@pytest.mark.parametrize("dim,bc,axisym", BOUNDED_FLOW_CASES)
def test_flow_limits_hold_between_walls_and_about_the_axis(dim, bc, axisym):
    # no mode grows just below each limit; a little above it one does (within
    # 15 % on the small 3D box, whose wall modes stop short of theta = pi)
    shape = (8, 12, 1) if dim == 2 else (4, 4, 6)
    over = 1.03 if dim == 2 else 1.15
    common = dict(dx=0.5, rhoL=1.3, rhoG=1.3, bc=bc, axisym=axisym)
    for regime, kw in (("viscous", dict(cs=0.01, etaL=0.2, etaG=0.2)),
                       ("acoustic", dict(cs=1.7, etaL=0.0, etaG=0.0))):
        prm = inputs.base_params(dim, *shape, **common, **kw)
        ac, vi, _ = gpe2p.stability_limits(prm)
        lim = vi if regime == "viscous" else ac
        lam = _flow_jacobian(prm)
        assert np.max(np.abs(_rk3(0.999 * lim * lam))) <= 1.0 + 1e-9, regime
        assert np.max(np.abs(_rk3(over * lim * lam))) > 1.0 + 1e-3, regime


@pytest.mark.parametrize("bc,axisym,scheme", [(("noslip", "noslip", "periodic"), 0, 2),
                                              (("noslip", "freeslip", "periodic"), 1, 2),
                                              (("freeslip", "noslip", "periodic"), 1, 4)])
def test_ch_limit_holds_between_walls_and_about_the_axis(bc, axisym, scheme):
    prm = inputs.base_params(2, 8, 12, dx=0.5, M=0.02, W=1.5, bc=bc, axisym=axisym, ch_scheme=scheme)
    _, _, lim = gpe2p.stability_limits(prm)
    lam = _ch_jacobian(prm)

    def growth(dt):
        z = dt * lam
        return np.max(np.abs(ch_polynomial(z, scheme)))

    assert growth(0.999 * lim) <= 1.0 + 1e-7
    assert growth(1.03 * lim) > 1.0 + 1e-3
