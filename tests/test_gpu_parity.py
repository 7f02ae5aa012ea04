"""GPU path vs the FP64 oracle on the same seeded inputs (small sizes that
still span several tiles and ragged tails).

Bars: grid classification and the crossing list bit-exact; FP64 coefficients
and the zero-BC right-hand side within 1e-14; FP64 operator apply within
1e-12 and FP32 apply within 1e-5 (relative infinity norm); converged phi to a
true FP64 residual <= 1e-8 (checked with the oracle's operator); energies
within 1e-6 of the oracle solved to 1e-12.
"""
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


def rel_inf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


CASES = {
    # name: (atoms, grid-spec kwargs, params kwargs)
    "cube33": (lambda: pb_inputs.globular_molecule(40, seed=101), dict(n=(33, 33, 33), fill=1.5),
               dict(bc=0)),
    "ragged": (lambda: pb_inputs.globular_molecule(60, seed=102), "explicit", dict(bc=2)),
}


def _explicit_grid(orc, atoms):
    """Non-cubic grid with nx > 128 (two x tiles, ragged tail) and explicit h."""
    h = 0.27
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(0) - 3.0
    ext = (atoms[:, :3] + atoms[:, 3:4]).max(0) + 3.0 - lo
    n = [int(np.ceil(e / h)) + 2 for e in ext]
    n[0] = max(n[0], 141)
    n[2] += 3
    return orc.Grid(tuple(n), lo, h)


@pytest.fixture(scope="module", params=list(CASES))
def case(request, pb, orc):
    atoms_fn, gspec, pkw = CASES[request.param]
    atoms = atoms_fn()
    if gspec == "explicit":
        og = _explicit_grid(orc, atoms)
        spec = pb.GridSpec(n=tuple(int(v) for v in og.n), origin=tuple(og.origin), h=og.h)
    else:
        spec = pb.GridSpec(**gspec)
        og = orc.place_grid(atoms, gspec["n"][0], gspec["fill"])
    params = pb.Params(**pkw)
    ref = orc.solve_problem(atoms, og, eps_in=params.eps_in, eps_out=params.eps_out,
                            ionic_strength_M=params.ionic_strength_M, bc=params.bc, rtol=1e-12)
    g = pb.pb_build_grid(spec, atoms)
    s = pb.pb_assemble_coeffs(g, params)
    return dict(name=request.param, atoms=atoms, og=og, spec=spec, params=params, ref=ref, g=g, s=s)


def test_grid_placement_and_classification(pb, case):
    og, g = case["og"], case["g"]
    assert tuple(g.info.n) == tuple(int(v) for v in og.n)
    assert g.info.h == og.h
    assert tuple(g.info.origin) == tuple(og.origin)
    inside = pb.pb_get_array(g, "inside")
    assert np.array_equal(inside, case["ref"]["inside"])
    assert g.info.n_inside == int(inside.sum())


def test_crossing_list_bit_exact(pb, case):
    g, cr = case["g"], case["ref"]["cross"]
    assert g.info.n_cross == len(cr["ids"]) > 0
    assert np.array_equal(pb.pb_get_array(g, "cross_id"), cr["ids"])
    assert np.array_equal(pb.pb_get_array(g, "cross_alpha"), cr["alpha"])
    assert np.array_equal(pb.pb_get_array(g, "cross_rp"), cr["rp"])
    assert np.array_equal(pb.pb_get_array(g, "cross_sign"), cr["sign"])
    assert g.info.n_flux == int((cr["sign"] != 0).sum())


@pytest.mark.parametrize("kind", ["placed", "snapped"])
def test_crossing_list_degenerate_geometry(pb, orc, kind):
    """Classification and crossing list bit-exact on inputs full of exact
    ties; the snapped molecule has coordinates on multiples of h/4 and radii
    on multiples of h/2."""
    h = 0.5
    atoms = pb_inputs.lattice_balls() if kind == "placed" else pb_inputs.snapped_molecule()
    og = orc.Grid((33, 33, 33), (-8.0, -8.0, -8.0), h)
    g = pb.pb_build_grid(pb.GridSpec(n=(33, 33, 33), origin=(-8.0, -8.0, -8.0), h=h), atoms)
    inside = orc.classify(og, atoms)
    cr = orc.crossing_edges(og, atoms, inside)
    assert np.array_equal(pb.pb_get_array(g, "inside"), inside)
    assert g.info.n_cross == len(cr["ids"]) > 0
    assert np.array_equal(pb.pb_get_array(g, "cross_id"), cr["ids"])
    assert np.array_equal(pb.pb_get_array(g, "cross_alpha"), cr["alpha"])
    assert np.array_equal(pb.pb_get_array(g, "cross_rp"), cr["rp"])
    assert np.array_equal(pb.pb_get_array(g, "cross_sign"), cr["sign"])
    if kind == "placed":
        # listed with alpha = 1: the surface passes through the end node
        assert np.any(cr["alpha"] == 1.0)
    g.free()


def test_coefficients(pb, case):
    s, ref = case["s"], case["ref"]
    for name in ("Wx", "Wy", "Wz"):
        assert np.array_equal(pb.pb_get_array(s, name), ref["coef"][name]), name
    assert rel_inf(pb.pb_get_array(s, "kappa"), ref["coef"]["kap"]) <= 1e-14
    assert rel_inf(pb.pb_get_array(s, "diag"), ref["coef"]["diag"]) <= 1e-14


def test_boundary_values_and_rhs(pb, case):
    s, ref = case["s"], case["ref"]
    bc = pb.pb_get_array(s, "bc")
    f = pb.pb_get_array(s, "rhs")
    if case["params"].bc == 0:
        assert not bc.any()
        assert rel_inf(f, ref["f"]) <= 1e-14
    else:
        # FP64 boundary sums: only the summation order differs from the oracle
        assert rel_inf(bc, ref["phib"]) <= 1e-13
        assert rel_inf(f, ref["f"]) <= 1e-13


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_operator_apply(pb, case, prec, tol):
    import torch
    s, og, ref = case["s"], case["og"], case["ref"]
    x = pb_inputs.random_field(og.N, seed=7)
    dt = torch.float64 if prec == 0 else torch.float32
    xt = torch.tensor(x, dtype=dt, device="cuda")
    y = pb.pb_apply(s, xt, precision=prec).double().cpu().numpy()
    from oracle import oracle as orc
    xin = xt.double().cpu().numpy()
    yref = orc.apply(og, ref["coef"], xin)
    assert rel_inf(y, yref) <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_residual_and_energy(pb, case, prec, orc):
    s, og, ref = case["s"], case["og"], case["ref"]
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    st = pb.pb_solve(s, pb.SolveOpts(precision=prec, rtol=1e-10))
    assert st["status"] == 0 and st["true_rel_res"] <= 1e-10
    phi = pb.pb_get_phi(s)
    # true residual of the GPU solution, evaluated by the oracle's operator
    x = phi - ref["phib"]
    r = ref["f"] - orc.apply(og, ref["coef"], x)
    n = og.n
    interior = np.zeros(og.shape_zyx(), bool)
    interior[1:-1, 1:-1, 1:-1] = True
    interior = interior.reshape(-1)
    rel = np.linalg.norm(r[interior]) / np.linalg.norm(ref["f"][interior])
    assert rel <= 1e-8
    e = pb.pb_energy(s)
    er = ref["energy"]
    for k in ("e_pol", "e_ion_flux", "e_ion_surf", "e_coul", "e_total", "e_ion_mc"):
        assert abs(e[k] - er[k]) <= 1e-6 * max(abs(er[k]), 1e-3 * abs(er["e_pol"])), k
    assert abs(e["flux_charge"] - case["atoms"][:, 4].sum()) < 1e-6 * np.abs(case["atoms"][:, 4]).sum()


def test_retriangulated_surface(pb, case, orc):
    """Marching-cubes vertex weights (T_j/3 sums) and analytic normals bit
    for bit; Psi along the normals within the compensated FP32 bound."""
    s, ref, atoms = case["s"], case["ref"], case["atoms"]
    pb.pb_coulomb_terms(s, pb.CT_SURFACE)
    cr = ref["cross"]
    W = pb.pb_get_array(s, "mc_weight")
    nrm = pb.pb_get_array(s, "mc_normal")
    assert np.array_equal(W, ref["mc"]["W"])
    assert np.array_equal(nrm, ref["mc"]["normals"])
    flux = cr["sign"] != 0
    psi = pb.pb_get_array(s, "psi_n")
    psi_ref = orc.coulomb_psi_n(cr["rp"][flux], nrm[flux], atoms)
    r = np.linalg.norm(cr["rp"][flux][:, None, :] - atoms[None, :, :3], axis=2)
    absq = np.abs(atoms[:, 4])[None, :]
    assert np.max(np.abs(psi[flux] - psi_ref) / (absq / r ** 2).sum(1)) <= 2e-6
    assert not psi[~flux].any()


def test_surface_coulomb_terms(pb, case, orc):
    s, ref, atoms = case["s"], case["ref"], case["atoms"]
    pb.pb_coulomb_terms(s, pb.CT_SURFACE)
    cr = ref["cross"]
    flux = cr["sign"] != 0
    Phi = pb.pb_get_array(s, "phi_surf")
    Psi = pb.pb_get_array(s, "psi_surf")
    P_ref = orc.coulomb_phi(cr["rp"][flux], atoms)
    dirs = (cr["ids"][flux] // case["og"].N).astype(np.int8)
    S_ref = orc.coulomb_psi(cr["rp"][flux], dirs, cr["sign"][flux], atoms)
    # FP32 error bound: relative to the sum of absolute contributions
    r = np.linalg.norm(cr["rp"][flux][:, None, :] - atoms[None, :, :3], axis=2)
    absq = np.abs(atoms[:, 4])[None, :]
    assert np.max(np.abs(Phi[flux] - P_ref) / (absq / r).sum(1)) <= 2e-6
    assert np.max(np.abs(Psi[flux] - S_ref) / (absq / r ** 2).sum(1)) <= 2e-6
    assert not Phi[~flux].any() and not Psi[~flux].any()


def test_born_ion_end_to_end(pb, orc):
    """Born ion (eps 1/80, R = 2 A, 65^3, h = 0.3125, Coulomb BC, FP64 PCG to
    1e-10): polarisation energy equals the closed form."""
    atoms = pb_inputs.born_ion()
    spec = pb.GridSpec(n=(65, 65, 65), origin=(0.0, 0.0, 0.0), h=0.3125)
    params = pb.Params(eps_in=1.0, eps_out=80.0, ionic_strength_M=0.0, bc=pb.BC_COULOMB)
    out = pb.solve_molecule(atoms, spec=spec, params=params,
                            opts=pb.SolveOpts(precision=pb.FP64, rtol=1e-10))
    lB, _ = orc.units(298.15, 0.0, 80.0)
    closed = 0.5 * (1 / 80.0 - 1.0) * lB / 2.0
    assert abs(out["energy"]["e_pol"] - closed) / abs(closed) < 1e-7
    out2 = pb.solve_molecule(atoms, spec=spec, params=params,
                             opts=pb.SolveOpts(precision=pb.MIXED, rtol=1e-10))
    assert abs(out2["energy"]["e_pol"] - closed) / abs(closed) < 1e-7


def test_argument_errors(pb):
    import math
    from paper_2502_09323_gb300 import PBError
    good = pb_inputs.globular_molecule(10, seed=3)
    bad = good.copy()
    bad[2, 3] = -1.0
    with pytest.raises(PBError, match="ARG"):
        pb.pb_build_grid(pb.GridSpec(n=(33, 33, 33)), bad)
    bad = good.copy()
    bad[1, 0] = math.nan
    with pytest.raises(PBError, match="ARG"):
        pb.pb_build_grid(pb.GridSpec(n=(33, 33, 33)), bad)
    # a charge whose trilinear cell touches the box boundary
    h = 0.5
    origin = tuple(good[0, :3] - 0.25 * h)
    with pytest.raises(PBError, match="ARG"):
        pb.pb_build_grid(pb.GridSpec(n=(40, 40, 40), origin=origin, h=h), good)
    g = pb.pb_build_grid(pb.GridSpec(n=(33, 33, 33)), good)
    with pytest.raises(PBError, match="ARG"):
        pb.pb_assemble_coeffs(g, pb.Params(eps_in=-2.0))
    s = pb.pb_assemble_coeffs(g, pb.Params())
    with pytest.raises(PBError, match="STATE"):
        pb.pb_energy(s)
    st = pb.pb_solve(s, pb.SolveOpts(precision=pb.FP64, rtol=1e-12, max_iter=3), check=False)
    assert st["rc"] == -4 and st["status"] == -4 and st["iters_inner"] <= 3 + 32
    import ctypes
    spec = pb.GridSpec(n=(33, 33, 33)).c()
    spec.kind = 1  # octree without h_fine / h_bulk
    h = ctypes.c_void_p()
    rc = pb._native.lib().pb_build_grid(ctypes.byref(spec), good.ctypes.data_as(ctypes.c_void_p),
                                        len(good), 0, None, ctypes.byref(h))
    assert rc == -1


def test_too_many_balls_on_one_edge(pb):
    """Sixty coincident uncharged balls cut the same listed edges: more than
    the 48 intervals one edge holds, reported as an argument error.  One ball
    fewer than the limit builds."""
    from paper_2502_09323_gb300 import PBError
    spec = pb.GridSpec(n=(33, 33, 33), origin=(-8.0, -8.0, -8.0), h=0.5)
    ball = [0.1, 0.2, 0.3, 1.3, 0.0]
    with pytest.raises(PBError, match="balls meet one listed grid edge"):
        pb.pb_build_grid(spec, np.array([ball] * 60))
    g = pb.pb_build_grid(spec, np.array([ball] * 48))
    assert g.info.n_cross > 0
    g.free()


@pytest.mark.parametrize("tw", [32, 64, 128])
def test_tile_widths(pb, case, tw, orc):
    """The mixed-precision solve with each tile width of the TMA-staged PCG
    kernels (tiles tw x 1024/tw points of a plane, fixed through
    pb_set_tuning) meets the true residual and the energies of the oracle."""
    s, og, ref = case["s"], case["og"], case["ref"]
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    pb.pb_set_tuning(s, pb.MIXED, 1, 8 + 10000 * tw)
    try:
        st = pb.pb_solve(s, pb.SolveOpts(precision=pb.MIXED, rtol=1e-10))
    finally:
        pb.pb_set_tuning(s, pb.MIXED, 1, 8)
    assert st["status"] == 0 and st["true_rel_res"] <= 1e-10
    assert st["kc"] // 10000 == tw and st["kc"] % 1000 == 8
    phi = pb.pb_get_phi(s)
    x = phi - ref["phib"]
    r = ref["f"] - orc.apply(og, ref["coef"], x)
    interior = np.zeros(og.shape_zyx(), bool)
    interior[1:-1, 1:-1, 1:-1] = True
    interior = interior.reshape(-1)
    assert np.linalg.norm(r[interior]) / np.linalg.norm(ref["f"][interior]) <= 1e-8
    e = pb.pb_energy(s)
    er = ref["energy"]
    for k in ("e_pol", "e_ion_flux", "e_coul", "e_total", "e_ion_mc"):
        assert abs(e[k] - er[k]) <= 1e-6 * max(abs(er[k]), 1e-3 * abs(er["e_pol"])), k


def test_tile_width_rejected(pb, case):
    from paper_2502_09323_gb300 import PBError
    with pytest.raises(PBError, match="ARG"):
        pb.pb_set_tuning(case["s"], pb.MIXED, 1, 8 + 10000 * 48)
