"""GPU parity of the variants of the scheme with the oracle, element by element: the viscous
numerical flux of Eq. numericalFluxNS_1 (ghat = G(v, q) . n), the power-law viscosity of Sec. 5.6
(mu = mu_ref (T / T_inf)^(3/4)), both together, the symmetric variable stabilization matrix
sigma_S = |A_n| A0 of Eq. symStab, and the entropy diagnostics of Eq. PiS."""
import dataclasses

import numpy as np
import pytest

from hdg_cases import CASES, GpuCase, oracle_hist, oracle_setup, rel_fro

pytestmark = pytest.mark.gpu

TOL_BLOCK = 1e-10
TOL_RES = 1e-12
VARIANTS = {"option1": dict(visc_flux=1), "power_law": dict(mu_exponent=0.75),
            "both": dict(visc_flux=1, mu_exponent=0.75), "sigma_s": dict(stabilization="s")}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("name", ["ns2d_p3", "ns3d_p2", "euler2d_p2"])
def test_variant_assemble_condense_matches_oracle(name, variant, precision):
    if CASES[name].reynolds == 0 and variant != "sigma_s":
        pytest.skip("viscous variant")
    case = dataclasses.replace(CASES[name], **VARIANTS[variant])
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    hist_o = oracle_hist(prob, V, case)
    gc.assemble(gc.history(), precision=precision)
    assert int(gc.status.abs().sum()) == 0
    S, g, R = gc.S.cpu().numpy(), gc.g.cpu().numpy(), gc.R.cpu().numpy()
    nv = gc.info["nv"]
    # the variant is exercised: the default scheme's blocks differ
    base = GpuCase(CASES[name])
    base.assemble(base.history(), precision=precision)
    assert rel_fro(S, base.S.cpu().numpy()) > 1e-8
    for e in sorted({0, 3, prob.mesh.E - 1}):
        L = prob.condense(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e), case.mass_coef,
                          hist_o[e])
        nq = L["Rl"].size - nv
        Rv = L["Rl"][nq:]
        scale = max(np.abs(Rv).max(), np.abs(L["Rt"]).max(), np.abs(hist_o[e]).max(), 1.0)
        assert np.abs(Rv - R[e, :nv]).max() <= TOL_RES * scale, (e, "R_v")
        assert np.abs(L["Rt"] - R[e, nv:]).max() <= TOL_RES * scale, (e, "R_t")
        assert rel_fro(S[e], L["S"]) < TOL_BLOCK, (e, rel_fro(S[e], L["S"]))
        assert rel_fro(g[e], L["g"]) < TOL_BLOCK, (e, rel_fro(g[e], L["g"]))


@pytest.mark.parametrize("name,omega", [("euler2d_p2", 0.0), ("ns2d_p3", 0.0), ("ns3d_p2", 0.75)])
def test_entropy_production_matches_oracle(name, omega):
    """int rho s and (1/c_v) int (Phi / T + kappa |grad T|^2 / T^2) from (v_h, q_h) (q_h of
    Eq. hDG_NS0 with the perturbed trace) against the oracle's sums over the same quadrature."""
    case = dataclasses.replace(CASES[name], mu_exponent=omega)
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    if Q is None:
        Q = np.zeros(V.shape + (prob.d,))
    s_gpu, p_gpu = gc.hdg.hdg_entropy_production(gc.ctx.handle, gc.V, gc.Vhat)
    s_ora, p_ora = prob.entropy_production_terms(Q, V)
    assert abs(s_gpu - s_ora) <= 1e-12 * abs(s_ora)
    if case.reynolds > 0:
        assert p_ora > 0 and abs(p_gpu - p_ora) <= 1e-10 * p_ora
    else:
        assert p_gpu == 0.0 and p_ora == 0.0
