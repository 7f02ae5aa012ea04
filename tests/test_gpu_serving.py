"""Continuous batching (pb_engine_*) and the serving loop on the GPU.

A solve must give the same bits alone and inside a running mix that other
requests join and leave while it iterates, and the same bits as pb_solve
(same z-chunk); the serving loop must stay inside its memory budget and its
energies must match the FP64 oracle within 1e-6."""
import time

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


# (n, atoms, seed): uneven sizes, several x tiles for the larger ones
SHAPES = [(65, 300, 301), (33, 60, 302), (49, 200, 303), (41, 120, 304), (57, 250, 305),
          (37, 90, 306), (45, 150, 307)]
OPTS = dict(rtol=1e-9)


def _system(pb, n, na, seed):
    atoms = pb_inputs.globular_molecule(na, seed=seed)
    g = pb.pb_build_grid(pb.GridSpec(n=(n, n, n), fill=1.6), atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params(bc=pb.BC_DH))
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    return s


@pytest.fixture(scope="module")
def reference(pb):
    """pb_solve of every shape (this also fixes each shape's z-chunk)."""
    out = []
    for shp in SHAPES:
        s = _system(pb, *shp)
        st = pb.pb_solve(s, pb.SolveOpts(precision=pb.MIXED, **OPTS))
        assert st["status"] == 0
        out.append((pb.pb_get_phi(s), st, pb.pb_energy(s)))
    return out


def _drain(eng, n, timeout=120.0):
    got = []
    t_end = time.time() + timeout
    while len(got) < n:
        assert time.time() < t_end, "engine did not finish"
        got += eng.wait(timeout_s=0.05)
    return got


def test_engine_alone_equals_pb_solve(pb, reference):
    with pb.Engine(capacity=4, opts=pb.SolveOpts(precision=pb.MIXED, **OPTS)) as eng:
        for shp, (phi, st_ref, e_ref) in zip(SHAPES, reference):
            s = _system(pb, *shp)
            t = eng.submit(s)
            (r,) = _drain(eng, 1)
            assert r["ticket"] == t and r["system"] is s
            st = r["stats"]
            assert st["status"] == 0 and st["true_rel_res"] <= 1e-9
            assert st["iters_inner"] == st_ref["iters_inner"]
            assert st["iters_outer"] == st_ref["iters_outer"]
            assert np.array_equal(pb.pb_get_phi(s), phi)
            assert pb.pb_energy(s) == e_ref


def test_engine_mix_with_joins_equals_alone(pb, reference):
    """Requests join while others iterate (capacity below the request count,
    so some wait for a slot); every result keeps its alone bits."""
    with pb.Engine(capacity=3, opts=pb.SolveOpts(precision=pb.MIXED, **OPTS)) as eng:
        systems = [_system(pb, *shp) for shp in SHAPES]
        tickets = {}
        got = []
        # two at once, the rest staggered while those run
        for i in (0, 1):
            tickets[eng.submit(systems[i])] = i
        for i in range(2, len(SHAPES)):
            time.sleep(0.002)
            got += eng.wait(timeout_s=0.0)
            tickets[eng.submit(systems[i])] = i
        got += _drain(eng, len(SHAPES) - len(got))
        q = eng.query()
        assert q["pending"] == 0 and q["active"] == 0 and q["rc"] == 0
    assert sorted(r["ticket"] for r in got) == sorted(tickets)
    for r in got:
        i = tickets[r["ticket"]]
        phi, st_ref, e_ref = reference[i]
        assert r["stats"]["status"] == 0
        assert r["stats"]["iters_inner"] == st_ref["iters_inner"]
        assert np.array_equal(pb.pb_get_phi(systems[i]), phi), i
        assert pb.pb_energy(systems[i]) == e_ref
    # the solves overlapped on the device: some request was admitted while
    # another one was still iterating
    spans = [(r["t_admit"], r["t_done"]) for r in got]
    overlap = any(a2 < d1 and a1 < d2 for k, (a1, d1) in enumerate(spans)
                  for (a2, d2) in spans[k + 1:])
    assert overlap


def test_engine_errors(pb):
    with pb.Engine(capacity=2, opts=pb.SolveOpts(precision=pb.MIXED, **OPTS)) as eng:
        s = _system(pb, *SHAPES[1])
        eng.submit(s)
        with pytest.raises(pb.PBError) as ei:
            eng.submit(s)
        assert ei.value.code == -1
        _drain(eng, 1)
        # once returned, the same system may be solved again (same bits)
        phi1 = pb.pb_get_phi(s)
        eng.submit(s)
        (r,) = _drain(eng, 1)
        assert r["stats"]["status"] == 0
        assert np.array_equal(pb.pb_get_phi(s), phi1)
    with pytest.raises(pb.PBError):
        pb.Engine(capacity=0)


def test_engine_destroy_with_work_in_flight(pb):
    """Destroying a busy engine hands its systems back; they stay usable."""
    eng = pb.Engine(capacity=1, opts=pb.SolveOpts(precision=pb.MIXED, **OPTS))
    systems = [_system(pb, *SHAPES[i]) for i in (0, 2)]
    for s in systems:
        eng.submit(s)
    eng.close()
    st = pb.pb_solve(systems[1], pb.SolveOpts(precision=pb.MIXED, **OPTS))
    assert st["status"] == 0


def test_server_poisson_stream_budget_and_oracle_energy(pb, orc):
    from paper_2502_09323_gb300 import serving
    rng_sizes = pb_inputs.batch_sizes(10, 5000, 60, 400)
    arrivals = pb_inputs.poisson_arrivals(10, rate_hz=200.0, seed=5000)
    reqs = []
    for j, (na, t) in enumerate(zip(rng_sizes, arrivals)):
        atoms = pb_inputs.globular_molecule(int(na), seed=5001 + j)
        reqs.append(serving.Request(rid=j, atoms=atoms, arrival_s=float(t)))
    specs = [serving.uniform_spec(r.atoms, h=0.5) for r in reqs]
    need = [serving.device_bytes_estimate(s, len(r.atoms)) for s, r in zip(specs, reqs)]
    budget = 2.5 * max(need)  # only two or three solves fit at once
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-10)
    with serving.Server(capacity=8, hbm_budget_bytes=budget, opts=opts, h=0.5,
                        keep_phi=True) as srv:
        recs = srv.run(reqs)
        assert srv.max_used <= budget
    assert len(recs) == len(reqs)
    summ = serving.latency_summary(recs)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0
    for r in recs:
        assert r["stats"]["status"] == 0 and r["stats"]["true_rel_res"] <= 1e-10
        assert r["latency_s"] >= r["engine_s"] > 0
    # energies of the smallest request against the FP64 oracle
    r = min(recs, key=lambda r: r["n"] * 10000 + r["atoms"])
    req = reqs[r["rid"]]
    spec = req.spec
    og = orc.Grid(tuple(spec.n), np.array(spec.origin), spec.h)
    ref = orc.solve_problem(req.atoms, og, rtol=1e-12)
    er = ref["energy"]
    for k in ("e_pol", "e_ion_flux", "e_ion_surf", "e_coul", "e_total"):
        assert abs(r["energy"][k] - er[k]) <= 1e-6 * max(abs(er[k]), 1e-3 * abs(er["e_pol"])), k
    # device memory of one request stays inside its estimate
    import torch
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    g = pb.pb_build_grid(spec, req.atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params())
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    with pb.Engine(capacity=1, opts=opts) as eng:
        eng.submit(s)
        _drain(eng, 1)
        torch.cuda.synchronize()
        used = torch.cuda.memory_allocated() - before
    assert used <= serving.device_bytes_estimate(spec, len(req.atoms))


def _octree_system(pb, na, seed):
    atoms = pb_inputs.globular_molecule(na, seed=seed)
    g = pb.pb_build_grid(pb.OctreeSpec(h_fine=0.5, h_bulk=1.0, refine_dist=2.0, fill=1.8), atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params(bc=pb.BC_DH))
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    return s


def test_engine_octree_beside_uniform_equals_pb_solve(pb, reference):
    """Octree systems are served beside uniform ones (their brick kernels run
    with every replay); each keeps the bits of its pb_solve."""
    oshapes = [(150, 401), (260, 402)]
    oref = []
    for na, seed in oshapes:
        s = _octree_system(pb, na, seed)
        st = pb.pb_solve(s, pb.SolveOpts(precision=pb.MIXED, **OPTS))
        assert st["status"] == 0
        oref.append((pb.pb_get_phi(s), st, pb.pb_energy(s)))
    with pb.Engine(capacity=3, opts=pb.SolveOpts(precision=pb.MIXED, **OPTS)) as eng:
        systems = {}
        for i, (na, seed) in enumerate(oshapes):
            systems[eng.submit(_octree_system(pb, na, seed))] = ("oct", i)
        for i in (1, 3):
            systems[eng.submit(_system(pb, *SHAPES[i]))] = ("uni", i)
        got = _drain(eng, 4)
    for r in got:
        kind, i = systems[r["ticket"]]
        phi, st_ref, e_ref = oref[i] if kind == "oct" else reference[i]
        assert r["stats"]["status"] == 0
        assert r["stats"]["iters_inner"] == st_ref["iters_inner"]
        assert r["stats"]["dof"] == st_ref["dof"]
        assert np.array_equal(pb.pb_get_phi(r["system"]), phi), (kind, i)
        assert pb.pb_energy(r["system"]) == e_ref


def test_server_octree_stream_within_budget(pb):
    import torch
    from paper_2502_09323_gb300 import serving
    sizes = pb_inputs.batch_sizes(6, 5100, 60, 400)
    arrivals = pb_inputs.poisson_arrivals(6, rate_hz=50.0, seed=5100)
    reqs = [serving.Request(rid=j, atoms=pb_inputs.globular_molecule(int(n), seed=5101 + j),
                            arrival_s=float(t)) for j, (n, t) in enumerate(zip(sizes, arrivals))]
    srv_kw = dict(h=0.5, grid="octree")
    need = [serving.device_bytes_estimate(serving.octree_spec(r.atoms, h_fine=0.5), len(r.atoms),
                                          r.atoms) for r in reqs]
    budget = 2.5 * max(need)
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-8)
    with serving.Server(capacity=4, hbm_budget_bytes=budget, opts=opts, **srv_kw) as srv:
        recs = srv.run(reqs)
        assert srv.max_used <= budget
    assert len(recs) == 6
    for r in recs:
        assert r["stats"]["status"] == 0 and r["stats"]["true_rel_res"] <= 1e-8
        assert r["energy"]["e_total"] != 0.0
    # the estimate covers the peak of one request (its build included)
    big = max(reqs, key=lambda r: len(r.atoms))
    spec = serving.octree_spec(big.atoms, h_fine=0.5)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    g = pb.pb_build_grid(spec, big.atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params())
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    pb.pb_solve(s, opts)
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated() - base
    assert peak <= serving.device_bytes_estimate(spec, len(big.atoms), big.atoms)
