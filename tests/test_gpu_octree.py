"""Octree brick grid on the GPU against the FP64 octree oracle
(oracle/octree.py) on the same seeded inputs.

Bars: bricks, levels, Morton order, node kinds, inside flags and the
crossing list bit-exact; pure-row edge weights bit-exact; operator apply
within 1e-12 (FP64) and 1e-5 (FP32) relative; right-hand side within 1e-13;
the converged solution to a true residual of 1e-8 under the oracle's
operator; energies within 1e-6."""
import numpy as np
import pytest

import pb_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_09323_gb300 import build
    build.build()
    import paper_2502_09323_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def O(orc):
    from oracle import octree
    return octree


CASES = {
    # name: (atoms, octree spec kwargs, params kwargs)
    "born3": (lambda: np.array([[0.0, 0.0, 0.0, 2.0, 1.0]]),
              dict(h_fine=0.5, h_bulk=2.0, refine_dist=3.0, n0=2, origin=(-16.0, -16.0, -16.0)),
              dict(eps_in=1.0, eps_out=80.0, ionic_strength_M=0.0, bc=1)),
    "mol": (lambda: pb_inputs.globular_molecule(30, seed=31),
            dict(h_fine=0.5, h_bulk=1.0, refine_dist=2.0, fill=2.0),
            dict(bc=2)),
    # the workload's levels (0.25 / 0.5 / 1 A, refined within 3 A) on 250
    # atoms: 3,114 bricks and 1.5M unknowns, so the persistent brick kernels
    # run many blocks, split the transition rows over many blocks and drain
    # a work-queue tail
    "mid250": (lambda: pb_inputs.globular_molecule(250, seed=77),
               dict(h_fine=0.25, h_bulk=1.0, refine_dist=3.0, fill=1.5),
               dict(bc=2)),
    # de-refined domain (Sec. 3.4): tight box at 0.5 A, 2 A far field,
    # perfil about 15 %, homogeneous Dirichlet values
    "deref": (lambda: pb_inputs.globular_molecule(20, seed=41),
              dict(h_fine=0.25, h_bulk=2.0, refine_dist=3.0, fill=1 / 0.15, h_tight=0.5,
                   tight_fill=1.1),
              dict(bc=0)),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, pb, O):
    atoms_fn, skw, pkw = CASES[request.param]
    atoms = atoms_fn()
    spec = pb.OctreeSpec(**skw)
    okw = dict(h_fine=skw["h_fine"], h_bulk=skw["h_bulk"], refine_dist=skw["refine_dist"])
    if skw.get("h_tight"):
        okw.update(h_tight=skw["h_tight"], tight_fill=skw["tight_fill"])
    if skw.get("n0", 0) > 0:
        tree = O.build(atoms, origin=np.array(skw["origin"]), n0=skw["n0"], **okw)
    else:
        tree = O.build(atoms, fill=skw["fill"], **okw)
    params = pb.Params(**pkw)
    ref = O.solve_problem(atoms, tree, eps_in=params.eps_in, eps_out=params.eps_out,
                          ionic_strength_M=params.ionic_strength_M, bc=params.bc, rtol=1e-12)
    g = pb.pb_build_grid(spec, atoms)
    s = pb.pb_assemble_coeffs(g, params)
    return dict(name=request.param, atoms=atoms, tree=tree, ref=ref, g=g, s=s, params=params)


def test_bricks_and_node_kinds(pb, O, case):
    g, tree, ref = case["g"], case["tree"], case["ref"]
    info = g.info
    assert info.kind == 1 and info.n_bricks == tree.nb and info.n_nodes == 512 * tree.nb
    assert info.n_levels == tree.Lmax + 1
    br = pb.pb_get_array(g, "oct_bricks")
    assert np.array_equal(br[:, :3], tree.blow) and np.array_equal(br[:, 3], tree.blevel)
    kind = pb.pb_get_array(g, "oct_kind")
    P = tree.slot_positions()
    okind = O.node_kind(tree, P)
    gk = np.where(kind == 3, 0, kind)  # both row kinds are regular unknowns
    assert np.array_equal(gk, okind)
    unk = np.zeros(len(P), bool)
    unk[ref["unk_slot"]] = True
    assert np.array_equal(kind == 0, unk & (kind != 3))
    assert np.array_equal((kind == 0) | (kind == 3), unk)
    op = ref["op"]
    NL1 = tree.NL + 1
    sk = (P[:, 2] * NL1 + P[:, 1]) * NL1 + P[:, 0]
    sidx = np.searchsorted(op["key"], sk)
    assert np.array_equal(pb.pb_get_array(g, "inside"), op["inside"][sidx])


def test_crossing_list_bit_exact(pb, O, case):
    g, tree, ref = case["g"], case["tree"], case["ref"]
    cr = O.crossing_edges(tree, ref["op"], case["atoms"])
    assert np.array_equal(pb.pb_get_array(g, "cross_id"), cr["ids_octree"])
    assert np.array_equal(pb.pb_get_array(g, "cross_alpha"), cr["alpha"])
    assert np.array_equal(pb.pb_get_array(g, "cross_rp"), cr["rp"])
    assert np.array_equal(pb.pb_get_array(g, "cross_sign"), cr["sign"])
    assert np.array_equal(pb.pb_get_array(g, "mc_weight"), cr["mc_w"])
    assert np.array_equal(pb.pb_get_array(g, "mc_normal"), cr["mc_n"])


def _unknown_map(case):
    tree, ref = case["tree"], case["ref"]
    return ref["unk_slot"], 512 * tree.nb


def test_operator_coefficients_and_rhs(pb, O, case):
    s, tree, ref = case["s"], case["tree"], case["ref"]
    unk, N = _unknown_map(case)
    A = ref["A"]
    diag = pb.pb_get_array(s, "diag")
    assert np.max(np.abs(diag[unk] - A.diagonal())) <= 1e-14 * np.max(np.abs(A.diagonal()))
    f = pb.pb_get_array(s, "rhs")
    assert np.max(np.abs(f[unk] - ref["f"])) <= 1e-13 * np.max(np.abs(ref["f"]))
    # pure-row edge weights: the element-form weight of edges inside four
    # same-level cells, bit for bit
    op = ref["op"]
    e = op["edges"]
    full = e["count"] == 4
    P = tree.slot_positions()
    NL1 = tree.NL + 1
    sk = (P[:, 2] * NL1 + P[:, 1]) * NL1 + P[:, 0]
    slot_of_pos = np.full(len(op["pos"]), -1)
    slot_of_pos[np.searchsorted(op["key"], sk)] = np.arange(len(P))
    W = [pb.pb_get_array(s, k) for k in ("Wx", "Wy", "Wz")]
    a = e["a"][full]
    d = e["d"][full]
    sl = slot_of_pos[a]
    lev = tree.blevel[np.clip(sl, 0, None) // 512]
    ok = (sl >= 0) & (lev == e["level"][full])
    got = np.array([W[dd][ss] for dd, ss in zip(d[ok], sl[ok])])
    assert np.array_equal(got, e["W"][full][ok])


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_operator_apply(pb, case, prec, tol):
    import torch
    s, ref = case["s"], case["ref"]
    unk, N = _unknown_map(case)
    xu = pb_inputs.random_field(len(unk), seed=5)
    x = np.zeros(N)
    x[unk] = xu
    dt = torch.float64 if prec == 0 else torch.float32
    y = pb.pb_apply(s, torch.tensor(x, dtype=dt, device="cuda"), precision=prec).double().cpu().numpy()
    yref = ref["A"] @ xu
    assert np.max(np.abs(y[unk] - yref)) <= tol * np.max(np.abs(yref))
    other = np.ones(N, bool)
    other[unk] = False
    assert np.all(y[other] == 0.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_residual_and_energy(pb, case, prec):
    s, ref = case["s"], case["ref"]
    unk, N = _unknown_map(case)
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    st = pb.pb_solve(s, pb.SolveOpts(precision=prec, rtol=1e-10))
    assert st["status"] == 0 and st["true_rel_res"] <= 1e-10
    assert st["dof"] == len(unk)
    phi = pb.pb_get_phi(s)
    r = ref["f"] - ref["A"] @ phi[unk]
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(ref["f"])
    # boundary and hanging values match the oracle's P x + x_b
    tree = case["tree"]
    op = ref["op"]
    P = tree.slot_positions()
    NL1 = tree.NL + 1
    sidx = np.searchsorted(op["key"], (P[:, 2] * NL1 + P[:, 1]) * NL1 + P[:, 0])
    refphi = ref["phi_pos"][sidx]
    assert np.max(np.abs(phi - refphi)) <= 1e-6 * np.max(np.abs(refphi))
    e = pb.pb_energy(s)
    er = ref["energy"]
    for k in ("e_pol", "e_ion_flux", "e_ion_surf", "e_coul", "e_total", "e_ion_mc"):
        assert abs(e[k] - er[k]) <= 1e-6 * max(abs(er[k]), 1e-3 * abs(er["e_pol"])), k


def test_surface_coulomb_terms(pb, O, case, orc):
    """Phi, Psi along the edge and Psi along the analytic surface normal at
    the octree's crossing points against the oracle's FP64 sums.  The
    crossing list in slot order makes the kernel's target blocks compact, so
    these take the per-block-origin form of the differences (and the axis
    form of Psi) that the uniform cases mostly do not."""
    s, tree, ref, atoms = case["s"], case["tree"], case["ref"], case["atoms"]
    pb.pb_coulomb_terms(s, pb.CT_SURFACE)
    cr = O.crossing_edges(tree, ref["op"], atoms)
    flux = cr["sign"] != 0
    rp = cr["rp"][flux]
    Phi = pb.pb_get_array(s, "phi_surf")[flux]
    Psi = pb.pb_get_array(s, "psi_surf")[flux]
    PsiN = pb.pb_get_array(s, "psi_n")[flux]
    P_ref = orc.coulomb_phi(rp, atoms)
    S_ref = orc.coulomb_psi(rp, cr["d"][flux].astype(np.int8), cr["sign"][flux], atoms)
    N_ref = orc.coulomb_psi_n(rp, cr["mc_n"][flux], atoms)
    # FP32 error bound: relative to the sum of absolute contributions
    # (evaluated in chunks of targets to bound the memory of the distances)
    absq = np.abs(atoms[:, 4])[None, :]
    for c0 in range(0, len(rp), 8192):
        sl = slice(c0, c0 + 8192)
        r = np.linalg.norm(rp[sl, None, :] - atoms[None, :, :3], axis=2)
        s1, s2 = (absq / r).sum(1), (absq / r ** 2).sum(1)
        assert np.max(np.abs(Phi[sl] - P_ref[sl]) / s1) <= 2e-6
        assert np.max(np.abs(Psi[sl] - S_ref[sl]) / s2) <= 2e-6
        assert np.max(np.abs(PsiN[sl] - N_ref[sl]) / s2) <= 2e-6


def test_born_on_octree_gpu(pb, orc):
    atoms = np.array([[0.0, 0.0, 0.0, 2.0, 1.0]])
    g = pb.pb_build_grid(pb.OctreeSpec(h_fine=0.25, h_bulk=1.0, refine_dist=3.0, n0=4,
                                       origin=(-16.0, -16.0, -16.0)), atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params(eps_in=1.0, eps_out=80.0, ionic_strength_M=0.0, bc=1))
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    st = pb.pb_solve(s, pb.SolveOpts(precision=pb.MIXED, rtol=1e-10))
    assert st["status"] == 0
    e = pb.pb_energy(s)
    lB, _ = orc.units(298.15, 0.0, 80.0)
    exact = 0.5 * (1.0 / 80.0 - 1.0) * lB / 2.0
    assert abs(e["e_pol"] / exact - 1.0) < 1e-7
    assert abs(e["flux_charge"] - 1.0) < 1e-7


def test_octree_argument_errors(pb):
    atoms = np.array([[0.0, 0.0, 0.0, 2.0, 1.0]])
    with pytest.raises(pb.PBError) as ei:
        pb.pb_build_grid(pb.OctreeSpec(h_fine=0.5, h_bulk=2.0, refine_dist=1.0), atoms)
    assert ei.value.code == -1
    with pytest.raises(pb.PBError):
        pb.pb_build_grid(pb.OctreeSpec(h_fine=0.5, h_bulk=1.5, refine_dist=3.0), atoms)

def test_octree_in_a_batch_equals_alone(pb):
    """pb_solve_batch takes octree systems beside uniform ones: each result
    is the same bits as its own pb_solve."""
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-9)

    def systems():
        a = pb_inputs.globular_molecule(60, seed=91)
        go = pb.pb_build_grid(pb.OctreeSpec(h_fine=0.5, h_bulk=1.0, refine_dist=3.0, fill=1.5), a)
        gu = pb.pb_build_grid(pb.GridSpec(n=(49, 49, 49), fill=1.6), a)
        return [pb.pb_assemble_coeffs(go, pb.Params()), pb.pb_assemble_coeffs(gu, pb.Params())]

    alone = systems()
    ref = [(pb.pb_solve(s, opts), pb.pb_get_phi(s)) for s in alone]
    mix = systems()
    stats = pb.pb_solve_batch(mix, opts)
    for s, st, (st_ref, phi) in zip(mix, stats, ref):
        assert st["status"] == 0 and st["true_rel_res"] <= 1e-9
        assert st["iters_inner"] == st_ref["iters_inner"]
        assert np.array_equal(pb.pb_get_phi(s), phi)
