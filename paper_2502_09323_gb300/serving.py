"""Request loop for a stream of PB solves on one GPU (continuous batching).

Requests (one molecule each) arrive over time.  The loop admits a waiting
request when the engine has a free slot and the device-memory budget covers
the request's estimated footprint; it builds the request's grid,
coefficients and Coulomb terms on a side stream while the engine keeps every
admitted solve iterating, submits the system to the engine, and, when the
engine reports the solve finished, evaluates the energy, frees the system and
returns its memory to the budget.  Each request's latency runs from its
arrival to its energy.

Every computation runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import (CT_PAIRS, CT_SURFACE, Engine, GridSpec, OctreeSpec, Params, SolveOpts,
               pb_assemble_coeffs, pb_build_grid, pb_coulomb_terms, pb_energy, pb_get_phi)

# nodes per axis offered to uniform serving grids (32k + 1)
GRID_SIZES = tuple(range(65, 2049, 32))

# device bytes per padded node of one solve (FP64 faces, diagonal, rhs,
# boundary values, iterate; FP32 weights, code bytes and four FP32 solver
# vectors; grid classification), plus a fixed allowance for the crossing-edge
# list, per-block partial sums and the launch-table entry
BYTES_PER_NODE = 112
FIXED_BYTES = 16 << 20


def uniform_spec(atoms: np.ndarray, h: float = 0.5, fill: float = 1.5,
                 sizes=GRID_SIZES) -> GridSpec:
    """Uniform grid of spacing h covering fill x the molecular extent, with the
    smallest node count of ``sizes`` that reaches it, centred on the atoms'
    bounding box of the spheres."""
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(axis=0)
    hi = (atoms[:, :3] + atoms[:, 3:4]).max(axis=0)
    extent = float((hi - lo).max())
    need = math.ceil(fill * extent / h) + 1
    n = next((s for s in sizes if s >= need), None)
    if n is None:
        raise ValueError(f"molecule needs {need} nodes per axis, above the largest offered size")
    origin = 0.5 * (lo + hi) - 0.5 * h * (n - 1)
    return GridSpec(n=(n, n, n), origin=tuple(float(v) for v in origin), h=float(h), fill=0.0)


def octree_spec(atoms: np.ndarray, h_fine: float = 0.25, h_bulk: float = 1.0,
                refine_dist: float = 3.0, fill: float = 1.5) -> OctreeSpec:
    """Brick octree placed automatically around the atoms."""
    return OctreeSpec(h_fine=h_fine, h_bulk=h_bulk, refine_dist=refine_dist, fill=fill)


# octree: device bytes per node slot (the uniform set plus node kinds, inside
# flags and the transition-row map), bytes per listed edge, and listed edges
# per atom at 0.25 A (they scale with 1/h^2)
OCT_BYTES_PER_SLOT = 112
OCT_BYTES_PER_EDGE = 64
OCT_EDGES_PER_ATOM = 400


def _octree_estimate(spec: OctreeSpec, atoms: np.ndarray) -> int:
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(axis=0)
    hi = (atoms[:, :3] + atoms[:, 3:4]).max(axis=0)
    c = 0.5 * (lo + hi)
    extent = float((hi - lo).max())
    n0 = max(1, math.ceil(spec.fill * extent / (8.0 * spec.h_bulk)))
    side = n0 * 8.0 * spec.h_bulk
    reach = float(np.max(np.linalg.norm(atoms[:, :3] - c, axis=1) + atoms[:, 3]))
    levels = int(round(math.log2(spec.h_bulk / spec.h_fine)))
    slots = 0.0
    r = reach + spec.refine_dist
    h = spec.h_fine
    for _ in range(levels):
        # each level's region grows by two of its bricks (brick rounding, balance)
        r += 16.0 * h
        slots += 4.0 / 3.0 * math.pi * r ** 3 / h ** 3
        h *= 2.0
    slots += (side / spec.h_bulk) ** 3
    edges = OCT_EDGES_PER_ATOM * len(atoms) * (0.25 / spec.h_fine) ** 2
    # the build classifies the whole domain on the finest lattice (freed
    # after): an inside byte per node, listed-edge and covered-edge bytes per
    # edge, and a byte per node of margin
    transient = 8.0 * (side / spec.h_fine + 1) ** 3
    return int(OCT_BYTES_PER_SLOT * slots + OCT_BYTES_PER_EDGE * edges + transient) + FIXED_BYTES


def device_bytes_estimate(spec, n_atoms: int, atoms: np.ndarray | None = None) -> int:
    """Device memory of one request's system (octree specs need the atoms)."""
    if isinstance(spec, OctreeSpec):
        return _octree_estimate(spec, atoms)
    nx, ny, nz = spec.n
    sx = (nx + 15) // 16 * 16  # FP32 rows are padded to 16 elements
    return BYTES_PER_NODE * sx * ny * nz + 64 * n_atoms + FIXED_BYTES


@dataclasses.dataclass
class Request:
    rid: int
    atoms: np.ndarray
    arrival_s: float
    spec: GridSpec | None = None


class Server:
    """Serves requests through one :class:`Engine` under a device-memory budget."""

    def __init__(self, capacity: int = 64, hbm_budget_bytes: float = 150e9,
                 params: Params | None = None, opts: SolveOpts | None = None, h: float = 0.5,
                 fill: float = 1.5, energy: bool = True, keep_phi: bool = False,
                 grid: str = "uniform"):
        import torch
        self.torch = torch
        self.params = params or Params()
        self.opts = opts or SolveOpts()
        self.h, self.fill = h, fill
        if grid not in ("uniform", "octree"):
            raise ValueError("grid must be 'uniform' or 'octree'")
        self.grid = grid
        self.energy = energy
        self.keep_phi = keep_phi
        self.budget = float(hbm_budget_bytes)
        self.engine = Engine(capacity=capacity, opts=self.opts)
        self.capacity = capacity
        self.stream = torch.cuda.Stream()
        self.max_used = 0

    def close(self):
        self.engine.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def spec_for(self, atoms: np.ndarray):
        """The request's grid: uniform of spacing h, or a brick octree whose
        finest spacing is h."""
        if getattr(self, "grid", "uniform") == "octree":
            return octree_spec(atoms, h_fine=self.h, fill=self.fill)
        return uniform_spec(atoms, self.h, self.fill)

    def _admit(self, req: Request, rec: dict):
        spec = req.spec or self.spec_for(req.atoms)
        rec["n"] = spec.n[0] if isinstance(spec, GridSpec) else 0
        with self.torch.cuda.stream(self.stream):
            g = pb_build_grid(spec, req.atoms, self.stream)
            s = pb_assemble_coeffs(g, self.params, self.stream)
            if self.energy:
                pb_coulomb_terms(s, CT_SURFACE | CT_PAIRS, self.stream)
        return self.engine.submit(s, self.stream)

    def run(self, requests: list[Request], on_done=None) -> list[dict]:
        """Serve ``requests`` (arrival times relative to the call); returns one
        record per request in completion order."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        self.max_used = 0
        waiting: collections.deque = collections.deque()
        inflight: dict[int, tuple[Request, dict, int]] = {}
        used = 0
        done: list[dict] = []
        nxt = 0
        t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
                waiting.append(reqs[nxt])
                nxt += 1
            # admission: FIFO, while a slot is free and the budget allows
            while waiting and len(inflight) < self.capacity:
                req = waiting[0]
                spec = req.spec or self.spec_for(req.atoms)
                need = device_bytes_estimate(spec, len(req.atoms), req.atoms)
                if inflight and used + need > self.budget:
                    break
                if need > self.budget:
                    raise ValueError(f"request {req.rid} needs {need} bytes, above the budget")
                waiting.popleft()
                req.spec = spec
                rec = {"rid": req.rid, "atoms": len(req.atoms), "arrival_s": req.arrival_s,
                       "admit_s": time.perf_counter() - t0, "bytes": need}
                ticket = self._admit(req, rec)
                rec["submit_s"] = time.perf_counter() - t0
                inflight[ticket] = (req, rec, need)
                used += need
                self.max_used = max(self.max_used, used)
            # completions
            if inflight:
                # until a completion, or the next arrival
                wait = 0.01
                if nxt < len(reqs):
                    wait = max(0.0, min(wait, reqs[nxt].arrival_s - (time.perf_counter() - t0)))
                results = self.engine.wait(timeout_s=wait)
            else:
                results = []
                if nxt < len(reqs) and not waiting:
                    time.sleep(max(0.0, min(0.01, reqs[nxt].arrival_s - (time.perf_counter() - t0))))
            for r in results:
                req, rec, need = inflight.pop(r["ticket"])
                rec["stats"] = r["stats"]
                rec["engine_s"] = r["t_done"] - r["t_admit"]
                self._finish(r["system"], rec)
                rec["done_s"] = time.perf_counter() - t0
                rec["latency_s"] = rec["done_s"] - rec["arrival_s"]
                used -= need
                done.append(rec)
                if on_done:
                    on_done(rec)
            self.max_used = max(self.max_used, used)
        return done

    def _finish(self, system, rec: dict) -> None:
        """Energy (and, if kept, phi) of a finished solve; frees the system."""
        with self.torch.cuda.stream(self.stream):
            if self.energy and rec["stats"]["status"] in (0, -4):
                rec["energy"] = pb_energy(system, self.stream)
            if self.keep_phi:
                rec["phi"] = pb_get_phi(system, self.stream)
        grid = system.grid
        system.free()
        grid.free()


def latency_summary(records: list[dict]) -> dict:
    lat = np.array([r["latency_s"] for r in records])
    span = max(r["done_s"] for r in records) - min(r["arrival_s"] for r in records)
    return {"requests": len(records), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "solves_per_s": len(records) / span if span > 0 else float("nan")}
