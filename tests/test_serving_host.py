"""Host logic of the serving loop (no GPU): grid sizing, memory estimate,
FIFO admission under the slot and memory limits, latency bookkeeping.  The
engine is replaced by a fake whose solves take fixed wall-clock times."""
import time

import numpy as np

import pb_inputs
from paper_2502_09323_gb300 import serving


def test_uniform_spec_covers_the_molecule():
    for na, seed in ((300, 1), (3000, 2), (20000, 3)):
        atoms = pb_inputs.globular_molecule(na, seed=seed)
        spec = serving.uniform_spec(atoms, h=0.5, fill=1.5)
        n = spec.n[0]
        assert spec.n == (n, n, n) and n in serving.GRID_SIZES and (n - 1) % 32 == 0
        lo = (atoms[:, :3] - atoms[:, 3:4]).min(0)
        hi = (atoms[:, :3] + atoms[:, 3:4]).max(0)
        ext = (hi - lo).max()
        assert (n - 1) * 0.5 >= 1.5 * ext
        assert (n - 33) * 0.5 < 1.5 * ext  # the next smaller size would not do
        c = np.array(spec.origin) + 0.5 * 0.5 * (n - 1)
        assert np.allclose(c, 0.5 * (lo + hi))


def test_memory_estimate_grows_with_the_grid():
    a = serving.device_bytes_estimate(serving.GridSpec(n=(65, 65, 65)), 100)
    b = serving.device_bytes_estimate(serving.GridSpec(n=(129, 129, 129)), 100)
    assert b > 7 * (a - serving.FIXED_BYTES)
    # rows are padded to 16 nodes
    assert serving.device_bytes_estimate(serving.GridSpec(n=(65, 10, 10)), 0) == \
        serving.device_bytes_estimate(serving.GridSpec(n=(80, 10, 10)), 0)


class FakeEngine:
    def __init__(self, seconds_per_solve):
        self.dt = seconds_per_solve
        self.running = {}
        self.next = 1
        self.max_running = 0

    def submit(self, req):
        t = self.next
        self.next += 1
        self.running[t] = (req, time.perf_counter())
        self.max_running = max(self.max_running, len(self.running))
        return t

    def wait(self, timeout_s=0.0):
        t_end = time.perf_counter() + timeout_s
        while True:
            now = time.perf_counter()
            out = []
            for t, (req, t0) in list(self.running.items()):
                if now - t0 >= self.dt(req):
                    del self.running[t]
                    out.append({"ticket": t, "system": req, "stats": {"status": 0},
                                "t_admit": t0, "t_done": now})
            if out or now >= t_end:
                return out
            time.sleep(0.0005)


class FakeServer(serving.Server):
    def __init__(self, capacity, budget, dt):
        self.capacity, self.budget = capacity, budget
        self.h, self.fill = 0.5, 1.5
        self.engine = FakeEngine(dt)
        self.max_used = 0
        self.admitted = []

    def _admit(self, req, rec):
        rec["n"] = req.spec.n[0]
        self.admitted.append(req.rid)
        return self.engine.submit(req)

    def _finish(self, system, rec):
        pass


def test_admission_fifo_within_slots_and_budget():
    sizes = pb_inputs.batch_sizes(24, 77, 100, 3000)
    arrivals = pb_inputs.poisson_arrivals(24, rate_hz=400.0, seed=77)
    reqs = [serving.Request(rid=j, atoms=pb_inputs.globular_molecule(int(n), seed=100 + j),
                            arrival_s=float(t)) for j, (n, t) in enumerate(zip(sizes, arrivals))]
    need = {r.rid: serving.device_bytes_estimate(serving.uniform_spec(r.atoms), len(r.atoms))
            for r in reqs}
    budget = 3 * max(need.values())
    srv = FakeServer(capacity=4, budget=budget, dt=lambda req: 0.002 + 1e-6 * len(req.atoms))
    recs = srv.run(reqs)
    assert len(recs) == len(reqs)
    assert sorted(r["rid"] for r in recs) == list(range(len(reqs)))
    assert srv.admitted == sorted(srv.admitted, key=lambda j: reqs[j].arrival_s)  # FIFO
    assert srv.max_used <= budget
    assert srv.engine.max_running <= 4
    for r in recs:
        assert r["admit_s"] >= r["arrival_s"] - 1e-9
        assert r["done_s"] >= r["admit_s"] and r["latency_s"] == r["done_s"] - r["arrival_s"]
    s = serving.latency_summary(recs)
    assert s["requests"] == 24 and s["p99_ms"] >= s["p50_ms"] > 0 and s["solves_per_s"] > 0


def test_a_request_above_the_budget_is_refused():
    atoms = pb_inputs.globular_molecule(500, seed=5)
    srv = FakeServer(capacity=2, budget=1e6, dt=lambda req: 0.001)
    try:
        srv.run([serving.Request(rid=0, atoms=atoms, arrival_s=0.0)])
    except ValueError as e:
        assert "above the budget" in str(e)
    else:
        raise AssertionError("expected a refusal")


def test_octree_estimate_covers_the_transient_lattice_and_grows():
    """The octree estimate includes the build's finest-lattice pass (an inside
    byte per node and two bytes per edge, freed after the build) and grows
    with the molecule and with a finer finest level."""
    import math
    small = pb_inputs.globular_molecule(500, seed=6)
    big = pb_inputs.globular_molecule(4000, seed=7)
    for atoms in (small, big):
        spec = serving.octree_spec(atoms, h_fine=0.25)
        lo = (atoms[:, :3] - atoms[:, 3:4]).min(0)
        hi = (atoms[:, :3] + atoms[:, 3:4]).max(0)
        n0 = max(1, math.ceil(spec.fill * float((hi - lo).max()) / (8.0 * spec.h_bulk)))
        lattice = (n0 * 8.0 * spec.h_bulk / spec.h_fine + 1) ** 3
        assert serving.device_bytes_estimate(spec, len(atoms), atoms) > 7 * lattice
    e_small = serving.device_bytes_estimate(serving.octree_spec(small), len(small), small)
    e_big = serving.device_bytes_estimate(serving.octree_spec(big), len(big), big)
    assert e_big > e_small
    coarse = serving.device_bytes_estimate(serving.octree_spec(big, h_fine=0.5), len(big), big)
    assert e_big > coarse
