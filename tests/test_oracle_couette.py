"""Pin of the oracle's Navier-Stokes terms against an exact viscous solution: the steady
compressible Couette flow of Sec. 5.2 with its source term (Problem.source_weak), solved by
Newton from the interpolated exact state (steady: no time term), converges to the exact flow at
the rates the paper prints for HDG (Table t:CouetteConvergence_HDG) and with errors of the size
it prints (tests/golden/couette_hdg_errors.txt).

Setting: Re0 = 0.1, M0 = 0.15, Pr = 0.71 on (0, 1)^2; the exact state is given on the walls
y = 0, 1 (b_h = vhat - v_b). The flow does not depend on x and the x-axis is periodic: with the
given state on x = 0, 1 too, the state over-determines the pressure at the inflow and outflow
and the density and energy errors converge at a pre-asymptotic rate (about 1 to 1.5 for k = 1
at L/h = 4 to 32), which the paper's table does not show. The errors then stay within a factor
of 5 of the printed ones (measured ratios: k = 1: rho 1.02, momentum 2.9, rho E 0.89, tau 1.03,
f 1.6; k = 2: 2.4, 2.8, 2.4, 1.3, 4.1); a wrong sign or factor in a viscous term, a source not
consistent with the flux, or a heat flux taken from the wrong state leaves O(1) errors that do
not converge. With the continuous IEDG and EDG traces the gradients converge one order lower,
as the paper states for them."""
import pathlib

import numpy as np
import pytest

import workloads as wl
from oracle import physics as ph
from oracle.hdg import Problem, consistent_Q, face_states, interpolate_state, newton_solve
from oracle.mesh import BC_STATE, Mesh

GOLDEN = pathlib.Path(__file__).parent / "golden"
PHYS = ph.Physics(mach=0.15, reynolds=0.1, prandtl=0.71)
NAMES = ("rho", "momentum", "rhoE", "tau", "f")


def _paper_table():
    rows = {}
    for line in (GOLDEN / "couette_hdg_errors.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, n, *err = line.split()
            rows[(int(k), int(n))] = np.array([float(x) for x in err])
    return rows


def _exact_viscous(xq):
    """tau_xy = mu V_x' and the heat flux f_y = -kappa T' of the exact flow (all else zero)."""
    yb = xq[:, 1]
    dvx = np.log1p(yb) + yb / (1.0 + yb)
    dT = 0.05 + 0.5 * PHYS.prandtl * (PHYS.gamma - 1.0) * PHYS.mach ** 2 * (1.0 - 2.0 * yb)
    tau = np.zeros((len(yb), 2, 2))
    tau[:, 0, 1] = tau[:, 1, 0] = PHYS.mu * dvx
    f = np.zeros((len(yb), 2))
    f[:, 1] = -PHYS.kappa * dT
    return tau, f


def couette_errors(n, p, scheme="hdg"):
    """Steady Newton solve on the n x n mesh of degree p; L2 errors of (rho, momentum, rho E,
    L tau / mu, L f / mu) over the domain and the Newton result."""
    mesh = Mesh(2, n, 0.0, 1.0, p, bc=[("periodic", "periodic"), ("state", "state")])
    prob = Problem(mesh, PHYS, scheme=scheme)
    prim = lambda x: wl.couette_field(x, PHYS.mach, PHYS.prandtl)
    V, Vh = interpolate_state(prob, prim)
    prob.boundary_state = face_states(prob, V)
    src = np.stack([prob.source_weak(e, wl.couette_source(mesh.xnode[e], PHYS.mu)) for e in range(mesh.E)])
    res = newton_solve(prob, consistent_Q(prob, V, Vh), V, Vh, 0.0, src, tol=1e-12, max_it=8)
    err = np.zeros(5)
    for e in range(mesh.E):
        T = prob.tables(e)
        xq = mesh.X[e, 0] + mesh.ref.qp @ mesh.J[e].T
        rho, vel, pr = prim(xq)
        du = ph.u_of_v(T.phi @ res.V[e], PHYS.gamma) - ph.u_of_primitives(rho, vel, pr, PHYS.gamma)
        vh = T.phi @ res.V[e]
        G = -ph.viscous_flux(vh, np.einsum("ga,amk->gmk", T.phi, res.Q[e]), PHYS)   # (0, tau, tau V - f)
        tau = G[:, 1:3, :]
        f = np.einsum("gi,gij->gj", -vh[:, 1:3] / vh[:, 3:4], tau) - G[:, 3, :]
        tau_e, f_e = _exact_viscous(xq)
        err += T.W @ np.c_[du[:, 0] ** 2, du[:, 1] ** 2 + du[:, 2] ** 2, du[:, 3] ** 2,
                           np.sum((tau - tau_e) ** 2, axis=(1, 2)) / PHYS.mu ** 2,
                           np.sum((f - f_e) ** 2, axis=1) / PHYS.mu ** 2]
    return np.sqrt(err), res, prob


def test_couette_source_balances_the_exact_flux():
    """The source is the divergence of the exact flux: integrated against w = 1 over a strip
    y0 < y < y1, (s, 1) equals the jump of the y-flux (F + G)_y between the strip's edges."""
    y0, y1 = 0.2, 0.7
    t, w = np.polynomial.legendre.leggauss(40)
    y = 0.5 * (y1 - y0) * t + 0.5 * (y1 + y0)
    xq = np.c_[np.zeros_like(y), y]
    total = 0.5 * (y1 - y0) * (w @ wl.couette_source(xq, PHYS.mu))

    def flux_y(yy):
        x = np.array([[0.0, yy]])
        rho, vel, p = wl.couette_field(x, PHYS.mach, PHYS.prandtl)
        F = ph.inviscid_flux_prim(rho, vel, p, PHYS.gamma)[0][:, 1]          # F [m, d], y column
        tau, f = _exact_viscous(x)
        Gy = -np.r_[0.0, tau[0, :, 1], vel[0] @ tau[0, :, 1] - f[0, 1]]
        return F + Gy
    assert np.allclose(total, flux_y(y1) - flux_y(y0), rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("p,min_order", [(1, (1.85, 1.85, 1.85, 1.5, 1.85)),
                                         (2, (2.0, 2.75, 2.0, 2.3, 2.75))])
def test_couette_converges_at_the_paper_rates(p, min_order):
    """L/h = 4 and 8. The paper's rates (L/h = 8 -> 16): k = 1: 2.29, 1.98, 2.19, 1.73, 1.99;
    k = 2: 2.47, 2.98, 2.47, 2.72, 2.97 (density and energy are below k + 1 there too)."""
    e4, _, _ = couette_errors(4, p)
    e8, res, prob = couette_errors(8, p)
    assert res.res_norms[-1] <= 1e-12 * max(1.0, res.res_norms[0]) and res.iters <= 4
    order = np.log2(e4 / e8)
    for name, o, lo in zip(NAMES, order, min_order):
        assert o >= lo, (name, order)
    printed = _paper_table()[(p, 8)]
    ratio = e8 / printed
    assert np.all((ratio > 0.2) & (ratio < 5.0)), dict(zip(NAMES, ratio))
    wall = prob.mesh.face_bc == BC_STATE          # the trace takes the wall state
    assert np.abs(res.Vhat[wall] - prob.boundary_state[wall]).max() <= 1e-12 * np.abs(res.Vhat).max()


@pytest.mark.parametrize("scheme", ["iedg", "edg"])
def test_couette_gradients_of_the_continuous_traces_converge_one_order_lower(scheme):
    """Sec. 5.2: unlike HDG, whose gradients q_h converge at the optimal order k + 1 (above), IEDG
    and EDG give the solution at order k + 1 but the gradients at order k only. k = 1, L/h = 4
    and 8: momentum at >= 1.8 (measured 1.92 IEDG, 1.98 EDG), stress and heat flux between 0.6
    and 1.3 (measured 0.81 / 0.84 IEDG, 0.99 / 1.00 EDG; HDG 1.69 / 2.01)."""
    e4, _, _ = couette_errors(4, 1, scheme)
    e8, res, _ = couette_errors(8, 1, scheme)
    assert res.res_norms[-1] <= 1e-12 * max(1.0, res.res_norms[0])
    order = np.log2(e4 / e8)
    assert order[1] >= 1.8, order
    assert np.all((order[3:] > 0.6) & (order[3:] < 1.3)), order
