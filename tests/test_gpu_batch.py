"""Batched solves (pb_solve_batch): uneven systems in one launch table.

Each system must get exactly the same result (bitwise phi, same iteration
counts) alone through pb_solve and inside a batch with other systems, and
every batched solve must reach the requested true residual."""
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


SHAPES = [(33, 60, 201), (41, 120, 202), (49, 200, 203), (65, 300, 204), (37, 90, 205)]


def _systems(pb, shapes):
    out = []
    for n, na, seed in shapes:
        atoms = pb_inputs.globular_molecule(na, seed=seed)
        g = pb.pb_build_grid(pb.GridSpec(n=(n, n, n), fill=1.6), atoms)
        s = pb.pb_assemble_coeffs(g, pb.Params(bc=pb.BC_DH))
        pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
        out.append(s)
    return out


def test_batch_equals_alone_bitwise(pb):
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-9)
    alone = _systems(pb, SHAPES)
    ref = []
    for s in alone:
        st = pb.pb_solve(s, opts)
        ref.append((pb.pb_get_phi(s), st, pb.pb_energy(s)))
    batch = _systems(pb, SHAPES)
    stats = pb.pb_solve_batch(batch, opts)
    for s, st, (phi, st_ref, e_ref) in zip(batch, stats, ref):
        assert st["status"] == 0 and st["true_rel_res"] <= 1e-9
        assert st["iters_inner"] == st_ref["iters_inner"]
        assert np.array_equal(pb.pb_get_phi(s), phi)
        assert pb.pb_energy(s) == e_ref
    # a different mix (subset, other order) gives the same bits again
    mix = _systems(pb, [SHAPES[3], SHAPES[0]])
    stats = pb.pb_solve_batch(mix, opts)
    assert np.array_equal(pb.pb_get_phi(mix[0]), ref[3][0])
    assert np.array_equal(pb.pb_get_phi(mix[1]), ref[0][0])


def test_batch_of_one_and_errors(pb):
    from paper_2502_09323_gb300 import PBError
    (s,) = _systems(pb, [SHAPES[0]])
    st = pb.pb_solve_batch([s], pb.SolveOpts(precision=pb.MIXED, rtol=1e-8))
    assert st[0]["status"] == 0 and st[0]["true_rel_res"] <= 1e-8
    with pytest.raises(PBError, match="ARG"):
        pb.pb_solve_batch([s, s], pb.SolveOpts(precision=pb.MIXED))
    st = pb.pb_solve_batch([s], pb.SolveOpts(precision=pb.FP64, rtol=1e-8))
    assert st[0]["status"] == 0


def test_batch_narrow_tiles_equal_alone(pb):
    """Systems whose shapes run narrow tiles (32 x 32 and 64 x 16 points of a
    plane) beside one on 128 x 8 tiles: each gives the same bits alone and in
    the batch."""
    shapes = [(43, 80, 211), (57, 150, 212), (71, 220, 213)]
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-9)
    alone = _systems(pb, shapes)
    for s, tw in zip(alone, (32, 64, 128)):
        pb.pb_set_tuning(s, pb.MIXED, 1, 6 + 10000 * tw)
    ref = []
    for s, tw in zip(alone, (32, 64, 128)):
        st = pb.pb_solve(s, opts)
        assert st["status"] == 0 and st["kc"] // 10000 == tw
        ref.append((pb.pb_get_phi(s), st))
    batch = _systems(pb, shapes[::-1])
    stats = pb.pb_solve_batch(batch, opts)
    for s, st, (phi, st_ref) in zip(batch, stats, ref[::-1]):
        assert st["status"] == 0 and st["true_rel_res"] <= 1e-9
        assert st["kc"] == st_ref["kc"] and st["iters_inner"] == st_ref["iters_inner"]
        assert np.array_equal(pb.pb_get_phi(s), phi)
