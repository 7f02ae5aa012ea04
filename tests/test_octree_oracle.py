"""Pins of the octree oracle (oracle/octree.py) against facts outside itself:
brute-force geometry, the uniform grid it must reduce to, fields the scheme
reproduces exactly, and the Born closed form."""
import math

import numpy as np
import pytest

import pb_inputs


@pytest.fixture(scope="module")
def O(orc):
    from oracle import octree
    return octree


def _born_tree(O, hb=2.0):
    atoms = np.array([[0.0, 0.0, 0.0, 2.0, 1.0]])
    tree = O.build(atoms, 0.5, hb, 3.0, origin=np.array([-16.0, -16.0, -16.0]), n0=int(32 / (8 * hb)))
    return atoms, tree


def test_tree_structure(O):
    atoms = pb_inputs.globular_molecule(12, seed=11)
    tree = O.build(atoms, 0.5, 2.0, 3.0, fill=2.0)
    lv, low, NL = tree.blevel, tree.blow, tree.NL
    side = 8 * tree.spacing(lv)
    # leaves tile the domain exactly (volumes add up, no two overlap)
    assert int(np.sum(side.astype(np.int64) ** 3)) == NL ** 3
    cover = np.zeros((NL // 8,) * 3, dtype=np.int64)
    for b in range(tree.nb):
        lo = low[b] // 8
        s = side[b] // 8
        cover[lo[0]:lo[0] + s, lo[1]:lo[1] + s, lo[2]:lo[2] + s] += 1
    assert np.all(cover == 1)
    # 2:1 balance over faces, edges and corners (finest-brick cells)
    f = tree.level_field
    n = f.shape[0]
    for off in np.ndindex(3, 3, 3):
        d = np.array(off) - 1
        a = f[max(0, d[0]):n + min(0, d[0]), max(0, d[1]):n + min(0, d[1]), max(0, d[2]):n + min(0, d[2])]
        b = f[max(0, -d[0]):n + min(0, -d[0]), max(0, -d[1]):n + min(0, -d[1]),
              max(0, -d[2]):n + min(0, -d[2])]
        assert np.all(np.abs(a - b) <= 1)
    # Morton order of the low corners
    codes = O.morton3(low[:, 0] // 8, low[:, 1] // 8, low[:, 2] // 8)
    assert np.all(np.diff(codes) > 0)
    # no coarse leaf lies near a sphere surface (else it would be split)
    coarse = lv < tree.Lmax
    for b in np.nonzero(coarse)[0]:
        assert not O.near_boxes(atoms, tree.origin, tree.h_fine, low[b:b + 1], int(side[b]), 3.0)[0]


def test_near_test_against_sampling(O):
    """The box test is the exact minimum of | |x - c| - R | over the box:
    compare with dense sampling of random boxes."""
    rng = np.random.Generator(np.random.PCG64(3))
    atoms = np.array([[0.3, -0.4, 0.2, 1.7, 0.0]])
    origin = np.zeros(3)
    for _ in range(60):
        low = rng.integers(-12, 8, size=(1, 3))
        side = int(rng.integers(1, 6))
        near = O.near_boxes(atoms, origin, 0.5, low, side, 1.0)[0]
        g = np.linspace(0.0, 1.0, 25)
        pts = origin + 0.5 * (low[0] + side * np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3))
        dist = np.abs(np.linalg.norm(pts - atoms[0, :3], axis=1) - 1.7)
        res = 0.5 * side * math.sqrt(3) / 24
        if dist.min() <= 1.0 - res:
            assert near
        if dist.min() > 1.0 + res:
            assert not near


def test_hanging_nodes(O):
    atoms, tree = _born_tree(O)
    pos, _ = O.corner_positions(tree)
    kind = O.node_kind(tree, pos)
    hang = pos[kind == 2]
    assert len(hang) > 0
    par, w = O.hanging_parents(tree, hang)
    assert np.allclose(w.sum(axis=1), 1.0)
    assert set(np.unique((w > 0).sum(axis=1))) <= {2, 4}
    pk = O.node_kind(tree, par.reshape(-1, 3)).reshape(-1, 4)
    assert np.all(pk[w > 0] != 2)
    # parents are the ends of the coarse edge / corners of the coarse face
    mid = (par * w[..., None]).sum(axis=1)
    assert np.array_equal(mid, hang)


def test_single_level_tree_is_the_uniform_grid(O, orc):
    """With h_fine = h_bulk the element form gives exactly the uniform
    operator: same classification, edge weights and masses bit for bit, same
    solution and energies up to summation order."""
    atoms = pb_inputs.globular_molecule(20, seed=7)
    h, n0 = 0.5, 3
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(0)
    hi = (atoms[:, :3] + atoms[:, 3:4]).max(0)
    o = 0.5 * (lo + hi) - 0.5 * n0 * 8 * h
    tree = O.build(atoms, h, h, 3.0, origin=o, n0=n0)
    res = O.solve_problem(atoms, tree, rtol=1e-12, bc=orc.BC_DH)
    n = 8 * n0 + 1
    ref = orc.solve_problem(atoms, orc.Grid((n,) * 3, o, h), rtol=1e-12, bc=orc.BC_DH)
    op = res["op"]
    pos = op["pos"]
    lin = (pos[:, 2] * n + pos[:, 1]) * n + pos[:, 0]
    assert np.array_equal(op["inside"], ref["inside"][lin])
    e = op["edges"]
    Wu = np.stack([ref["coef"]["Wx"], ref["coef"]["Wy"], ref["coef"]["Wz"]])
    full = e["count"] == 4
    assert np.array_equal(e["W"][full], Wu[e["d"], lin[e["a"]]][full])
    inter = op["kind"] == 0
    assert np.array_equal(op["mass"][inter], ref["coef"]["kap"][lin[inter]])
    assert np.max(np.abs(res["phi_pos"] - ref["phi"][lin])) <= 1e-12 * np.max(np.abs(ref["phi"]))
    for k in ("e_pol", "e_ion_flux", "e_ion_surf", "e_total", "e_ion_mc"):
        assert abs(res["energy"][k] - ref["energy"][k]) <= 1e-12 * abs(ref["energy"][k])
    # the crossing list is the uniform one (same alpha, r_p, sign), in slot
    # order, and so is its re-triangulated surface (weights, normals)
    cr = res["cross"]
    order = np.argsort(ref["cross"]["ids"])
    assert np.array_equal(np.sort(cr["ids"]), ref["cross"]["ids"][order])
    back = np.argsort(cr["ids"])
    for k in ("alpha", "rp", "sign"):
        assert np.array_equal(cr[k][back], ref["cross"][k][order])
    assert np.array_equal(cr["mc_w"][back], ref["mc"]["W"][order])
    assert np.array_equal(cr["mc_n"][back], ref["mc"]["normals"][order])


@pytest.mark.parametrize("field", ["constant", "linear"])
def test_constant_and_linear_fields_are_exact(O, field):
    """Uniform eps, no salt, no charge, Dirichlet data from a constant or
    linear field: the discrete solution is that field at every node,
    hanging ones included (P reproduces linear functions and the element
    form is exact on them)."""
    atoms = np.array([[0.0, 0.0, 0.0, 2.0, 0.0]])
    tree = O.build(atoms, 0.5, 2.0, 3.0, origin=np.array([-16.0, -16.0, -16.0]), n0=2)
    op = O.operator(tree, atoms, 2.0, 2.0, 0.0)
    P, unk, hinfo = O.interpolation(tree, op)
    K = op["K"]
    A = (P.T @ K @ P).tocsr()
    x = op["pos"].astype(np.float64)
    g = np.ones(len(x)) if field == "constant" else 0.3 * x[:, 0] - 0.7 * x[:, 1] + 0.2 * x[:, 2] + 1.0
    assert np.any(op["kind"] == 2)
    xb = O.boundary_field(tree, op, hinfo, np.where(op["kind"] == 1, g, 0.0))
    f = P.T @ (-(K @ xb))
    sol, it, rel, conv = O.jacobi_pcg(A, f, 1e-13)
    assert conv
    phi = P @ sol + xb
    assert np.max(np.abs(phi - g)) <= 1e-11 * np.max(np.abs(g))


def test_born_ion_on_octree_is_exact(O, orc):
    """Discrete Gauss identity: E_pol of a Born ion equals the closed form up
    to the solver tolerance on the octree too (three levels, hanging nodes)."""
    atoms, tree = _born_tree(O)
    assert len(np.unique(tree.blevel)) >= 2
    res = O.solve_problem(atoms, tree, eps_in=1.0, eps_out=80.0, ionic_strength_M=0.0,
                          bc=orc.BC_COULOMB, rtol=1e-12)
    lB, _ = orc.units(298.15, 0.0, 80.0)
    ref = 0.5 * (1.0 / 80.0 - 1.0) * lB / 2.0
    assert abs(res["energy"]["e_pol"] / ref - 1.0) < 1e-9
    assert abs(res["energy"]["flux_charge"] - 1.0) < 1e-9


def test_octree_operator_spd_and_direct_solve(O):
    # one refined corner brick among seven coarse ones (hanging nodes on
    # three of its faces), small enough for a dense factorisation
    atoms = np.array([[0.0, 0.0, 0.0, 1.5, 1.0], [0.6, 0.3, -0.4, 1.3, -0.5]])
    tree = O.build(atoms, 0.5, 1.0, 1.5, origin=np.array([-4.0, -4.0, -4.0]), n0=2)
    assert sorted(np.bincount(tree.blevel).tolist()) == [7, 8]
    res = O.solve_problem(atoms, tree, rtol=1e-13, with_energy=False)
    A = res["A"].toarray()
    # symmetric up to the summation order of P^T K P
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(0.5 * (A + A.T))
    x = np.linalg.solve(A, res["f"])
    assert np.max(np.abs(x - res["x"])) <= 1e-10 * np.max(np.abs(x))


def test_far_field_coarsening_is_small(O, orc):
    """The same ion in salt on the octree and on the uniform grid at h_fine:
    the Gauss-exact terms agree to rounding, the surface term to 1e-3."""
    atoms = np.array([[0.1, -0.2, 0.05, 2.0, 1.0]])
    o = np.array([-16.0, -16.0, -16.0])
    tree = O.build(atoms, 0.5, 1.0, 3.0, origin=o, n0=4)
    res = O.solve_problem(atoms, tree, eps_in=1.0, eps_out=80.0, rtol=1e-12, bc=orc.BC_DH)
    ref = orc.solve_problem(atoms, orc.Grid((65,) * 3, o, 0.5), eps_in=1.0, eps_out=80.0,
                            rtol=1e-12, bc=orc.BC_DH)
    for k in ("e_pol", "e_ion_flux"):
        assert abs(res["energy"][k] / ref["energy"][k] - 1.0) < 1e-12
    assert abs(res["energy"]["e_ion_surf"] / ref["energy"]["e_ion_surf"] - 1.0) < 1e-3


def test_derefined_domain_with_null_bc(O, orc):
    """Sec. 3.4: a tight box refined around the molecule and coarse cells out
    to a low perfil make homogeneous Dirichlet values accurate.  Kirkwood
    sphere (R = 2 A, q = 1 e, eps 2/80, 0.145 M): on a tight domain (perfil
    50 %) null boundary values miss the ionic energy entirely (error above
    100 %), Debye-Hueckel values do not (about 13 % at h = 0.5 A); on the
    de-refined domain (perfil 12.5 %, 1 A far-field cells) null values match
    the Debye-Hueckel result with a third of the unknowns of a uniform grid
    over the same box.  E_pol is exact (Gauss) in every case.  The
    re-triangulated-surface E_ion beats the staircase one there."""
    lB, kD = orc.units(298.15, 0.145, 80.0)
    e_pol = 0.5 * (1 / 80.0 - 1 / 2.0) * lB / 2.0
    e_ion = -0.5 * lB / 80.0 * kD / (1.0 + kD * 2.0)
    atoms = np.array([[0.0, 0.0, 0.0, 2.0, 1.0]])

    def run(bc, **kw):
        tree = O.build(atoms, **kw)
        r = O.solve_problem(atoms, tree, bc=bc, rtol=1e-11)
        e = r["energy"]
        assert abs(e["e_pol"] - e_pol) < 1e-9 * abs(e_pol)
        mc = (e["e_ion_mc"] + e["e_ion_flux"] - e_ion) / abs(e_ion)
        return tree, len(r["unk_slot"]), (e["e_ion_surf"] + e["e_ion_flux"] - e_ion) / abs(e_ion), mc

    _, _, tight_null, _ = run(orc.BC_ZERO, h_fine=0.5, h_bulk=0.5, refine_dist=3.0, fill=1.25)
    _, _, tight_dh, _ = run(orc.BC_DH, h_fine=0.5, h_bulk=0.5, refine_dist=3.0, fill=1.25)
    tree, unk, deref_null, deref_mc = run(orc.BC_ZERO, h_fine=0.5, h_bulk=4.0, refine_dist=3.0,
                                          fill=1 / 0.15, h_tight=0.5, tight_fill=1.25)
    assert abs(tight_null) > 1.0 and abs(tight_dh) < 0.2
    assert abs(deref_null) <= abs(tight_dh)
    # the first integral on the re-triangulated surface (Sec. 3.3.2) halves
    # the staircase error on the same de-refined domain
    assert abs(deref_mc) < 0.6 * abs(deref_null)
    # a coarser far field around the tight box at h_tight (the 2:1 balance
    # grades the cells brick by brick, 8 cells per brick and level)
    assert tree.Lmax == 3 and set(np.unique(tree.blevel)) == {2, 3}
    assert unk < (tree.NL - 1) ** 3 / 2
    # the tight box lies in bricks of cells no coarser than h_tight
    tlo, thi = O.tight_box(atoms, 1.25)
    P = tree.slot_positions()
    W = tree.world(P)
    inbox = np.all((W >= tlo) & (W <= thi), axis=1)
    assert np.all(tree.spacing(tree.blevel)[np.arange(len(P)) // 512][inbox] == 1)
