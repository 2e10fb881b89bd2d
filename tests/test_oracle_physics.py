"""Pins of the oracle's pointwise physics against definitions the paper fixes:
v = dH/du (Sec. 2.3), the entropy-flux identity (Eq. entropyFluxIdentity), symmetry
and definiteness of A0 and of A_n A0 (Sec. 4.1), lambda_max as the largest eigenvalue
magnitude of A_n (Eq. sLxF), the jump entropy identity (Lemma 1, Appendix A) and the
Newtonian / Fourier closures (Eq. closuresNS)."""
import numpy as np
import pytest

from oracle import physics as ph

G = 1.4
H = 1e-30


def random_states(rng, n, d):
    rho = rng.uniform(0.5, 2.0, n)
    vel = rng.normal(0, 1.0, (n, d))
    p = rng.uniform(0.5, 3.0, n)
    return rho, vel, p


def cs_jac(f, x):
    """Complex-step Jacobian of f at a single point x [k] -> [..., k]."""
    cols = []
    for j in range(x.shape[-1]):
        xc = x.astype(np.complex128).copy()
        xc[j] += 1j * H
        cols.append(np.imag(f(xc)) / H)
    return np.stack(cols, axis=-1)


@pytest.mark.parametrize("d", [2, 3])
def test_round_trip(d):
    rng = np.random.default_rng(1)
    rho, vel, p = random_states(rng, 200, d)
    u = ph.u_of_primitives(rho, vel, p, G)
    v = ph.v_of_u(u, G)
    assert np.all(v[:, -1] < 0)
    u2 = ph.u_of_v(v, G)
    assert np.max(np.abs(u2 - u) / np.abs(u).max(axis=1, keepdims=True)) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_entropy_variables_are_gradient_of_H(d):
    """v(u) as printed equals dH/du for H = -rho s (complex step of H)."""
    rng = np.random.default_rng(2)
    rho, vel, p = random_states(rng, 20, d)
    u = ph.u_of_primitives(rho, vel, p, G)
    for k in range(20):
        grad = cs_jac(lambda x: ph.entropy_H(x, G), u[k])
        v = ph.v_of_u(u[k], G)
        assert np.allclose(grad, v, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_A0_and_flux_jacobian_symmetry(d):
    rng = np.random.default_rng(3)
    rho, vel, p = random_states(rng, 20, d)
    u = ph.u_of_primitives(rho, vel, p, G)
    v = ph.v_of_u(u, G)
    A0 = ph.A0_of_v(v, G)
    for k in range(20):
        # du_of_v against complex step of u_of_v
        A0cs = cs_jac(lambda x: ph.u_of_v(x, G), v[k])
        assert np.allclose(A0[k], A0cs, rtol=1e-13, atol=1e-12 * np.abs(A0cs).max())
        assert np.allclose(A0[k], A0[k].T, atol=1e-12 * np.abs(A0[k]).max())
        assert np.linalg.eigvalsh(A0[k]).min() > 0
        nrm = rng.normal(size=d); nrm /= np.linalg.norm(nrm)
        An = cs_jac(lambda x: ph.inviscid_flux_u(x, G) @ nrm, u[k])       # dF_n/du
        At = An @ A0[k]
        assert np.allclose(At, At.T, atol=1e-12 * np.abs(At).max())
        # lambda_max = largest |eigenvalue| of A_n
        ev = np.abs(np.linalg.eigvals(An)).max()
        assert abs(ph.lambda_max(v[k], nrm, G) - ev) < 1e-12 * ev
        # entropy-flux identity: dF_ent,n/du = v^T dF_n/du
        dFe = cs_jac(lambda x: ph.entropy_flux(x, G) @ nrm, u[k])
        assert np.allclose(dFe, v[k] @ An, atol=1e-12 * np.abs(dFe).max())


@pytest.mark.parametrize("d", [2, 3])
def test_jump_entropy_identity(d):
    """Lemma 1 (Appendix A): -[F_ent,n] + 1/2 (v1+v2).[F_n] = 1/2 dv^T Sigma dv with
    Sigma = int_0^1 (1-2 theta) A~_n(v(theta)) d theta on the straight path."""
    rng = np.random.default_rng(4)
    xg, wg = np.polynomial.legendre.leggauss(20)
    th, wt = (xg + 1) / 2, wg / 2
    for _ in range(10):
        rho, vel, p = random_states(rng, 2, d)
        v1, v2 = ph.v_of_u(ph.u_of_primitives(rho, vel, p, G), G)
        nrm = rng.normal(size=d); nrm /= np.linalg.norm(nrm)
        Fn = lambda v: ph.inviscid_flux_v(v, G) @ nrm
        Fe = lambda v: ph.entropy_flux(ph.u_of_v(v, G), G) @ nrm
        lhs = -(Fe(v2) - Fe(v1)) + 0.5 * (v1 + v2) @ (Fn(v2) - Fn(v1))
        Sig = sum(w * (1 - 2 * t) * cs_jac(Fn, v1 + t * (v2 - v1)) for t, w in zip(th, wt))
        dv = v2 - v1
        rhs = 0.5 * dv @ Sig @ dv
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs)), (lhs, rhs)


@pytest.mark.parametrize("d", [2, 3])
def test_viscous_flux_closures(d):
    """G(v, q) with q = grad v of a smooth field equals -(0, tau, V.tau + kappa grad T)
    with tau, f from Eq. closuresNS evaluated on the primitive gradients directly."""
    rng = np.random.default_rng(5)
    phys = ph.Physics(gamma=G, mach=0.4, reynolds=100.0, prandtl=0.72)
    for _ in range(10):
        rho0, vel0, p0 = [a[0] for a in random_states(rng, 1, d)]
        gr, gV, gp = rng.normal(size=d), rng.normal(size=(d, d)), rng.normal(size=d)

        def prim_v(x):                       # entropy variables of a linear primitive field
            rho = rho0 + gr @ x
            vel = vel0 + gV @ x
            p = p0 + gp @ x
            return ph.v_of_u(ph.u_of_primitives(rho, vel, p, G), G)

        x0 = np.zeros(d)
        v = prim_v(x0)
        q = cs_jac(prim_v, x0)               # [m, d] = grad v
        Gv = ph.viscous_flux(v, q, phys)
        mu, kap, cv = phys.mu, phys.kappa, phys.cv
        gradT = (gp * rho0 - p0 * gr) / (rho0 ** 2 * (G - 1) * cv)
        tau = mu * (gV + gV.T - 2.0 / 3.0 * np.trace(gV) * np.eye(d))
        ref = -np.vstack([np.zeros(d), tau, vel0 @ tau + kap * gradT])
        assert np.allclose(Gv, ref, atol=1e-12 * np.abs(ref).max())
        # K~ = -dG/dq is symmetric positive semi-definite (Sec. 4.4, Prop. 2)
        m = d + 2
        K = -cs_jac(lambda qq: ph.viscous_flux(v, qq.reshape(m, d), phys).reshape(-1),
                    q.reshape(-1))
        assert np.allclose(K, K.T, atol=1e-12 * np.abs(K).max())
        assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > -1e-12 * np.abs(K).max()
