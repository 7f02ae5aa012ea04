"""Failure paths triggered from the host (no GPU fault is ever made): a
time budget that runs out, an iteration cap, and a non-converging solve in
the serving engine.  Each returns its status with the statistics filled in,
and the library and the system stay usable afterwards."""
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


def _system(pb, n=97):
    atoms = pb_inputs.globular_molecule(400, seed=61)
    g = pb.pb_build_grid(pb.GridSpec(n=(n, n, n), fill=1.5), atoms)
    return pb.pb_assemble_coeffs(g, pb.Params())


@pytest.mark.parametrize("prec", [0, 1])
def test_time_budget_runs_out_then_solves(pb, prec):
    s = _system(pb)
    st = pb.pb_solve(s, pb.SolveOpts(precision=prec, rtol=1e-12, time_budget_s=1e-5), check=False)
    assert st["rc"] == -5 and st["status"] == -5
    assert "time budget" in pb.pb_last_error()
    st = pb.pb_solve(s, pb.SolveOpts(precision=prec, rtol=1e-8))
    assert st["status"] == 0 and st["true_rel_res"] <= 1e-8


@pytest.mark.parametrize("prec", [0, 1])
def test_iteration_cap_reports_noconv(pb, prec):
    s = _system(pb)
    st = pb.pb_solve(s, pb.SolveOpts(precision=prec, rtol=1e-10, max_iter=20), check=False)
    assert st["rc"] == -4 and st["status"] == -4
    assert 0 < st["iters_inner"] <= 20 and st["true_rel_res"] > 1e-10
    # the best iterate is kept and is better than the zero guess
    assert st["true_rel_res"] < 1.0
    st = pb.pb_solve(s, pb.SolveOpts(precision=prec, rtol=1e-8))
    assert st["status"] == 0


def test_octree_time_budget(pb):
    atoms = pb_inputs.globular_molecule(200, seed=62)
    g = pb.pb_build_grid(pb.OctreeSpec(h_fine=0.25, h_bulk=1.0, refine_dist=3.0), atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params())
    st = pb.pb_solve(s, pb.SolveOpts(precision=pb.MIXED, rtol=1e-12, time_budget_s=1e-5), check=False)
    assert st["rc"] == -5
    st = pb.pb_solve(s, pb.SolveOpts(precision=pb.MIXED, rtol=1e-8))
    assert st["status"] == 0


def test_engine_reports_noconv_and_keeps_serving(pb):
    import time
    with pb.Engine(capacity=2, opts=pb.SolveOpts(precision=pb.MIXED, rtol=1e-10, max_iter=15)) as eng:
        a, b = _system(pb, 65), _system(pb, 81)
        eng.submit(a)
        eng.submit(b)
        got = []
        t_end = time.time() + 60
        while len(got) < 2 and time.time() < t_end:
            got += eng.wait(timeout_s=0.05)
        assert len(got) == 2
        for r in got:
            assert r["stats"]["status"] == -4 and r["stats"]["iters_inner"] <= 15
        assert eng.query()["rc"] == 0
    st = pb.pb_solve(a, pb.SolveOpts(precision=pb.MIXED, rtol=1e-8))
    assert st["status"] == 0


def test_device_wait_limit_expires_then_solves(pb):
    """Every ring-slot wait of the FP32 PCG kernels is bounded.  With the
    bound set to zero polls the first wait gives up at once: the kernels stop,
    drain their own copies, reset their work counters and mark the solve with
    device status 3, which the host reports as PB_ERR_TIMEOUT -- for a single
    solve, a batch and a served system.  With the bound restored the same
    systems solve to the same bits as before."""
    import time
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-8)
    a, b = _system(pb, 65), _system(pb, 81)
    for s in (a, b):  # fixed tuning: no timing runs under the short bound
        pb.pb_set_tuning(s, pb.MIXED, 1, 8)
    ref = [pb.pb_solve(s, opts) for s in (a, b)]
    phi_ref = [pb.pb_get_phi(s) for s in (a, b)]
    try:
        pb.pb_set_wait_limit(0)
        st = pb.pb_solve(a, opts, check=False)
        assert st["rc"] == -5 and st["status"] == -5, st
        assert "device-side wait" in pb.pb_last_error()
        sts = pb.pb_solve_batch([a, b], opts, check=False)
        assert all(s["status"] == -5 for s in sts), sts
        with pb.Engine(capacity=2, opts=opts) as eng:
            eng.submit(b)
            got, t_end = [], time.time() + 60
            while not got and time.time() < t_end:
                got = eng.wait(timeout_s=0.05)
            assert len(got) == 1 and got[0]["stats"]["status"] == -5, got
    finally:
        pb.pb_set_wait_limit(-1)
    for s, r, p in zip((a, b), ref, phi_ref):
        st = pb.pb_solve(s, opts)
        assert st["status"] == 0 and st["true_rel_res"] <= 1e-8
        assert st["iters_inner"] == r["iters_inner"]
        assert np.array_equal(pb.pb_get_phi(s), p)
    sts = pb.pb_solve_batch([a, b], opts)
    for s, p in zip((a, b), phi_ref):
        assert np.array_equal(pb.pb_get_phi(s), p)


def test_batch_time_budget_runs_out_then_solves(pb):
    """A batch whose time budget runs out reports PB_ERR_TIMEOUT for the
    systems it did not finish, hands every system back, and the same systems
    then solve normally."""
    a, b = _system(pb, 65), _system(pb, 97)
    sts = pb.pb_solve_batch([a, b], pb.SolveOpts(precision=pb.MIXED, rtol=1e-12,
                                                 time_budget_s=1e-5), check=False)
    assert sts[0]["rc"] == -5 and any(s["status"] == -5 for s in sts)
    sts = pb.pb_solve_batch([a, b], pb.SolveOpts(precision=pb.MIXED, rtol=1e-8))
    assert all(s["status"] == 0 and s["true_rel_res"] <= 1e-8 for s in sts)
