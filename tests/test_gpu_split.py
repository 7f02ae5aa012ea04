"""One system solved on several z-slabs (pb_solve_split): the multi-GPU
decomposition of the solve, with its halo exchanges and rank-ordered
reductions, run with every rank on this GPU.

One rank reproduces pb_solve bit for bit; two to five ranks (uneven slabs,
a ragged x extent) reach the requested true residual under the oracle's
operator and the oracle's energies within 1e-6."""
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
def case(pb, orc):
    atoms = pb_inputs.globular_molecule(80, seed=301)
    og = orc.Grid((141, 65, 61), (-21.0, -9.6, -9.0), 0.3)
    ref = orc.solve_problem(atoms, og, bc=orc.BC_DH, rtol=1e-12)
    spec = pb.GridSpec(n=tuple(int(v) for v in og.n), origin=tuple(og.origin), h=og.h)

    def system():
        g = pb.pb_build_grid(spec, atoms)
        s = pb.pb_assemble_coeffs(g, pb.Params(bc=pb.BC_DH))
        pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
        return s

    return dict(atoms=atoms, og=og, ref=ref, system=system)


def test_one_rank_is_the_single_solve(pb, case):
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-10)
    a = case["system"]()
    st = pb.pb_solve(a, opts)
    b = case["system"]()
    st1 = pb.pb_solve_split(b, 1, opts)
    assert st1["status"] == 0 and st1["iters_inner"] == st["iters_inner"]
    assert st1["true_rel_res"] == st["true_rel_res"]
    assert np.array_equal(pb.pb_get_phi(b), pb.pb_get_phi(a))


@pytest.mark.parametrize("ranks", [2, 3, 5])
def test_split_solve_matches_the_oracle(pb, orc, case, ranks):
    og, ref = case["og"], case["ref"]
    s = case["system"]()
    st = pb.pb_solve_split(s, ranks, pb.SolveOpts(precision=pb.MIXED, rtol=1e-10))
    assert st["status"] == 0 and st["true_rel_res"] <= 1e-10
    phi = pb.pb_get_phi(s)
    r = ref["f"] - orc.apply(og, ref["coef"], phi - ref["phib"])
    interior = np.zeros(og.shape_zyx(), bool)
    interior[1:-1, 1:-1, 1:-1] = True
    interior = interior.reshape(-1)
    assert np.linalg.norm(r[interior]) <= 1e-8 * np.linalg.norm(ref["f"][interior])
    # boundary nodes carry the system's own boundary values
    assert np.array_equal(phi[~interior], pb.pb_get_array(s, "bc")[~interior])
    e, er = pb.pb_energy(s), ref["energy"]
    for k in ("e_pol", "e_ion_flux", "e_ion_surf", "e_coul", "e_total", "e_ion_mc"):
        assert abs(e[k] - er[k]) <= 1e-6 * max(abs(er[k]), 1e-3 * abs(er["e_pol"])), k


def test_split_arguments(pb, case):
    from paper_2502_09323_gb300 import PBError
    s = case["system"]()
    with pytest.raises(PBError, match="ARG"):
        pb.pb_solve_split(s, 0, pb.SolveOpts(precision=pb.MIXED))
    with pytest.raises(PBError, match="ARG"):
        pb.pb_solve_split(s, 2, pb.SolveOpts(precision=pb.FP64))
