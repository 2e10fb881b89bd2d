"""GPU parity of the boundary terms b_h (Eqs. hDG2 / hDG_NS2; BC_STATE and BC_SLIP) with the
oracle: the element blocks of bounded meshes (every element with a boundary face, and a few
interior ones; HDG and IEDG trace spaces) in both precisions, with sigma_SLF and sigma_S on the
slip walls; EDG's strongly imposed rows; BDF1 Newton steps (dense and GMRES trace solves) to the
oracle's state on all three trace spaces; the boundary state is read from the context's copy and
a missing state is an error."""
import dataclasses

import numpy as np
import pytest

from hdg_cases import CASES, GpuCase, oracle_hist, oracle_setup, rel_fro

pytestmark = pytest.mark.gpu

TOL_BLOCK = 1e-10
TOL_RES = 1e-12

BC_CASES = {
    # inflow / outflow sides with the given state, slip walls along the flow
    "euler2d_state_slip": dataclasses.replace(CASES["euler2d_p2"], bc=(("state", "state"), ("slip", "slip"))),
    # sigma_S (blocks only: at a slip wall V.n = 0 and sigma_S loses the rank of its entropy and
    # shear part, so the assembled trace system is singular there)
    "euler2d_slip_sigma_s": dataclasses.replace(CASES["euler2d_p2"], bc=(("slip", "slip"), ("periodic", "periodic")),
                                                stabilization="s", vinf=(1.0, 0.5), psi=1.0),
    "euler2d_state_sigma_s": dataclasses.replace(CASES["euler2d_p2"], bc=(("state", "state"), ("periodic", "periodic")),
                                                 stabilization="s", vinf=(1.0, 0.5), psi=1.0),
    "ns2d_state": dataclasses.replace(CASES["ns2d_p3"], bc=(("state", "state"), ("periodic", "periodic"))),
    "ns3d_state": dataclasses.replace(CASES["ns3d_p2"], bc=(("periodic", "periodic"), ("periodic", "periodic"),
                                                             ("state", "state"))),
    # IEDG (Sec. 3.4): continuous on the interior faces, each boundary face with its own nodes
    "ns2d_state_iedg": dataclasses.replace(CASES["ns2d_p3"], bc=(("state", "state"), ("periodic", "periodic")),
                                           scheme="iedg"),
    "euler2d_state_slip_iedg": dataclasses.replace(CASES["euler2d_p2"], bc=(("state", "state"), ("slip", "slip")),
                                                   scheme="iedg"),
}
# EDG: the continuous trace takes the state strongly at the nodes of the state faces (their rows
# of S and g are the identity and vhat - v_b once per node, zero at the node's other occurrences)
EDG_CASES = {
    "ns2d_state_edg": dataclasses.replace(CASES["ns2d_p3"], bc=(("state", "state"), ("periodic", "periodic")),
                                          scheme="edg"),
    "euler2d_state_edg": dataclasses.replace(CASES["euler2d_p2"], bc=(("state", "state"), ("state", "state")),
                                             scheme="edg"),
}


def _boundary_elements(prob):
    m = prob.mesh
    return sorted({s[0][0] for F, s in enumerate(m.face_elems) if m.face_bc[F] != 0})


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(BC_CASES))
def test_bc_assemble_condense_matches_oracle(name, precision):
    case = BC_CASES[name]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    hist_o = oracle_hist(prob, V, case)
    gc.assemble(gc.history(), precision=precision)
    assert int(gc.status.abs().sum()) == 0
    S, g, R = gc.S.cpu().numpy(), gc.g.cpu().numpy(), gc.R.cpu().numpy()
    nv = gc.info["nv"]
    assert gc.info["n_boundary_faces"] == int(np.sum(prob.mesh.face_bc != 0)) > 0
    elems = _boundary_elements(prob)
    elems = elems[:: max(1, len(elems) // 24)] + [e for e in (0, prob.mesh.E // 2) if e not in elems]
    for e in elems:
        L = prob.condense(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e), case.mass_coef,
                          hist_o[e])
        nq = L["Rl"].size - nv
        Rv = L["Rl"][nq:]
        scale = max(np.abs(Rv).max(), np.abs(L["Rt"]).max(), np.abs(hist_o[e]).max(), 1.0)
        assert np.abs(Rv - R[e, :nv]).max() <= TOL_RES * scale, (e, "R_v")
        assert np.abs(L["Rt"] - R[e, nv:]).max() <= TOL_RES * scale, (e, "R_t")
        assert rel_fro(S[e], L["S"]) < TOL_BLOCK, (e, rel_fro(S[e], L["S"]))
        assert rel_fro(g[e], L["g"]) < TOL_BLOCK, (e, rel_fro(g[e], L["g"]))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(EDG_CASES))
def test_edg_strong_state_rows_match_oracle(name, precision):
    """Element blocks of EDG with boundaries: the rows of the trace nodes on state faces are the
    identity (on the node's first occurrence over (element, local face, face node)) or zero, with
    g = vhat - v_b there or zero; every other row equals the oracle's condensation."""
    case = EDG_CASES[name]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    hist_o = oracle_hist(prob, V, case)
    gc.assemble(gc.history(), precision=precision)
    assert int(gc.status.abs().sum()) == 0
    S, g = gc.S.cpu().numpy(), gc.g.cpu().numpy()
    m = prob.m
    nodes, vb = prob.dirichlet_nodes()
    vb_of = dict(zip(nodes.tolist(), vb))
    flat = prob.edg_index.reshape(-1)
    _, first_at = np.unique(flat, return_index=True)
    designated = np.zeros(flat.size, dtype=bool)
    designated[first_at] = True
    per = prob.edg_index[0].size
    elems = sorted({int(k) // per for k in np.flatnonzero(np.isin(flat, nodes))})
    elems = elems[:: max(1, len(elems) // 16)] + [0, prob.mesh.E // 2]
    for e in elems:
        L = prob.condense(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e), case.mass_coef, hist_o[e])
        loc = prob.edg_index[e].reshape(-1)
        dir_row = np.repeat(np.isin(loc, nodes), m)
        keep = ~dir_row
        if keep.any():
            assert rel_fro(S[e][keep], L["S"][keep]) < TOL_BLOCK, e
            assert rel_fro(g[e][keep], L["g"][keep]) < TOL_BLOCK, e
        for j in np.flatnonzero(np.isin(loc, nodes)):
            rows = j * m + np.arange(m)
            expect = np.zeros((m, S.shape[-1]))
            gexp = np.zeros(m)
            if designated[e * per + j]:
                expect[np.arange(m), rows] = 1.0
                gexp = Vh[loc[j]] - vb_of[int(loc[j])]
            assert np.array_equal(S[e][rows], expect), (e, j)
            assert np.abs(g[e][rows] - gexp).max() <= 1e-14 * max(1.0, np.abs(Vh).max()), (e, j)


@pytest.mark.parametrize("name,precision,solver", [("euler2d_state_slip", 0, "dense"),
                                                    ("euler2d_state_slip", 1, "gmres"),
                                                    ("euler2d_state_sigma_s", 0, "gmres"),
                                                    ("ns2d_state", 1, "gmres"),
                                                    ("euler2d_state_slip_iedg", 0, "dense"),
                                                    ("ns2d_state_iedg", 1, "gmres"),
                                                    ("euler2d_state_edg", 0, "dense"),
                                                    ("ns2d_state_edg", 1, "gmres")])
def test_bc_newton_step_matches_oracle(name, precision, solver):
    """One BDF1 step (dt = 0.05) to |R| <= 1e-10 max(1, |R0|): the same number of Newton updates
    and the same state as the oracle's step (dense trace solves)."""
    from oracle.hdg import time_step
    case = dataclasses.replace({**BC_CASES, **EDG_CASES}[name], noise=0.0)
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    dt = 0.05
    res = time_step(prob, Q, V, Vh, [V], 1, dt, tol=1e-10, max_it=10)
    hdg = gc.hdg
    method = hdg.HDG_SOLVER_DENSE if solver == "dense" else hdg.HDG_SOLVER_GMRES
    hdg.hdg_ctx_set_trace_solver(gc.ctx.handle, method, 1e-13, 2000)
    V_gpu, Vh_gpu = gc.V.clone(), gc.Vhat.clone()
    it, rn = hdg.hdg_newton_step(gc.ctx.handle, V_gpu, Vh_gpu, gc.V, None, dt, 1, precision, 1e-10, 10)
    assert it == res.iters, (it, res.iters)
    assert rel_fro(V_gpu.cpu().numpy(), res.V) < 1e-10
    assert rel_fro(Vh_gpu.cpu().numpy(), res.Vhat) < 1e-10
    vh = Vh_gpu.cpu().numpy()
    for F in np.flatnonzero(prob.mesh.face_bc == 1):   # the trace takes the boundary state on the state faces
        e, f = prob.mesh.face_elems[F][0]
        vb = prob.boundary_state[F][prob.mesh.fnode_map[e, f]]
        assert np.abs(prob.gather_trace(vh, e)[f] - vb).max() <= 1e-12 * np.abs(vb).max()


def test_missing_boundary_state_is_an_error():
    from paper_1808_05066_gb300 import hdg
    import torch
    case = BC_CASES["ns2d_state"]
    mesh = hdg.Mesh(case.dim, case.n, 0.0, case.L, case.p, bc=case.bc)
    ctx = hdg.Context(mesh, 1.4, case.mach, case.reynolds, case.prandtl, 0)
    i = mesh.info
    dev = torch.device("cuda", 0)
    V = torch.zeros((i["n_elem"], i["Np"], i["m"]), dtype=torch.float64, device=dev)
    V[..., -1] = -1.0
    Vh = torch.zeros((i["n_faces"], i["Nf"], i["m"]), dtype=torch.float64, device=dev)
    Vh[..., -1] = -1.0
    S = torch.empty((i["n_elem"], i["nt"], i["nt"]), dtype=torch.float64, device=dev)
    g = torch.empty((i["n_elem"], i["nt"]), dtype=torch.float64, device=dev)
    rec = torch.empty((i["n_elem"], i["nv"] * i["nt"] + i["nv"]), dtype=torch.float64, device=dev)
    R = torch.empty((i["n_elem"], i["nv"] + i["nt"]), dtype=torch.float64, device=dev)
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_assemble_condense(ctx.handle, V, Vh, None, 0.0, 0, S, g, rec, R, None)
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    torch.cuda.synchronize()
