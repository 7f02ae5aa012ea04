#!/usr/bin/env python3
"""Benchmark of the linear Poisson-Boltzmann hot path on GB300.

One step = one pass of the whole hot path for one synthetic molecule:
grid placement + classification + crossing edges (pb_build_grid), edge
weights + right-hand side (pb_assemble_coeffs), surface and pair Coulomb sums
(pb_coulomb_terms), mixed-precision Jacobi-PCG to a true FP64 residual of
1e-8 (pb_solve) and the energy terms (pb_energy).

Default workload: 2,000-atom globular molecule (seed 2), uniform 257^3 grid
spanning 1.5x the molecular extent, eps 2/80, 0.145 M salt, zero Dirichlet
boundary.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank solves its own copy of
the workload (independent problems, weak scaling, no data-path collective).
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (host cores only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s & DoF-iter/s (%HBM peak), p50/p99 latency vs plain FP64 CG at 1e-8 residual"
WORKLOADS = {
    "globular257": dict(n_atoms=2000, seed=2, n=257, fill=1.5, eps_in=2.0, eps_out=80.0,
                        ionic=0.145, bc=0, rtol=1e-8),
}
# Stream (read+write) bytes per interior node of one launch of each FP32 PCG
# kernel: direction kernel reads z, p_old (4 B each) and the code byte and
# writes p; update kernel reads p, x, z and the code byte, writes x, z.
ALG_BYTES_P32 = 4 * 3 + 1
ALG_BYTES_U32 = 4 * 5 + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="globular257", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-octree", action="store_true")
    ap.add_argument("--octree-only", action="store_true",
                    help="run only the octree workload (for profiling)")
    ap.add_argument("--octree-atoms", type=int, default=20000,
                    help="atoms of the octree workload (smaller for profiling captures)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-rate", type=float, default=None,
                    help="Poisson arrival rate (default 1.5/s on octree grids, 6/s on uniform)")
    ap.add_argument("--serve-grid", default="octree", choices=["octree", "uniform"])
    ap.add_argument("--grid-n", type=int, default=None,
                    help="nodes per axis of the uniform workload instead of its own (profiling "
                         "captures of smaller cases)")
    ap.add_argument("--profile-fp64", action="store_true",
                    help="run only W + K plain FP64 steps of the uniform workload (profiling)")
    ap.add_argument("--serve-sweep", default=None,
                    help="comma-separated Poisson rates (1/s): serve --serve-requests requests at "
                         "each rate and report every operating point (long; not in the default run)")
    ap.add_argument("--oracle-procs", type=int, default=None,
                    help="host processes for the oracle throughput of the batched workload "
                         "(default: the cores this process may use)")
    ap.add_argument("--tuning", default=None,
                    help="VARIANT:ZCHUNK for the FP32 PCG kernels instead of the autotuner "
                         "(e.g. 1:0 = TMA-staged persistent); for profiler runs")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.tmp.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle --
def oracle_sample(wl: dict, pcg_iters: int = 10, targets: int = 2000) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload and
    extrapolate one full solve: full setup (classification, crossing edges,
    coefficients, right-hand side) + `pcg_iters` PCG iterations scaled to the
    oracle's own iteration count to rtol (recorded by ``python -m
    oracle.calibrate``) + surface sums on `targets` flux points scaled to all
    of them + the full pair sum."""
    import numpy as np

    import pb_inputs
    from oracle import oracle as orc
    orc.build()
    atoms = pb_inputs.globular_molecule(wl["n_atoms"], seed=wl["seed"])
    t0 = time.perf_counter()
    g = orc.place_grid(atoms, wl["n"], wl["fill"])
    lB, kD = orc.units(298.15, wl["ionic"], wl["eps_out"])
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    coef = orc.assemble(g, inside, cross, wl["eps_in"], wl["eps_out"], kD)
    phib = orc.bc_values(g, atoms, lB, wl["eps_out"], wl["bc"], kD)
    f = orc.rhs(g, atoms, lB, coef, phib)
    t_setup = time.perf_counter() - t0
    # iteration time from two runs of different length: the difference
    # leaves out the first iterations' page faults and cold caches
    t0 = time.perf_counter()
    orc.pcg(g, coef, f, wl["rtol"], max_iter=2)
    t_short = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.pcg(g, coef, f, wl["rtol"], max_iter=2 + pcg_iters)
    t_iter = max(time.perf_counter() - t0 - t_short, 0.0) / pcg_iters
    flux = cross["sign"] != 0
    nflux = int(flux.sum())
    sel = np.flatnonzero(flux)[:: max(1, nflux // targets)][:targets]
    t0 = time.perf_counter()
    orc.coulomb_phi(cross["rp"][sel], atoms)
    orc.coulomb_psi(cross["rp"][sel], (cross["ids"][sel] // g.N).astype(np.int8),
                    cross["sign"][sel], atoms)
    t_surf = (time.perf_counter() - t0) * nflux / len(sel)
    t0 = time.perf_counter()
    orc.ecoul(atoms, lB, wl["eps_in"])
    t_pairs = time.perf_counter() - t0
    iters = oracle_iters()
    t_solve = t_setup + iters * t_iter + t_surf + t_pairs
    return {"t_setup": t_setup, "t_iter": t_iter, "iters": iters, "t_surface": t_surf,
            "t_pairs": t_pairs, "t_solve": t_solve, "nflux": nflux, "sampled_targets": len(sel),
            "pcg_iters_sampled": pcg_iters}


def oracle_record() -> dict:
    """The oracle's complete run on the default workload as recorded by
    ``python -m oracle.calibrate``: its Jacobi-PCG iteration count to a 1e-8
    true residual and the measured seconds of the whole pass (with the
    machine it ran on)."""
    with open(os.path.join(ROOT, "oracle", "iters_globular257.json")) as fh:
        return json.load(fh)


def oracle_iters() -> int:
    return int(oracle_record()["iters"])


def full_solve_check() -> dict | None:
    """The recorded, measured full oracle pass when it was taken on a machine
    of this architecture (the projection of the sample can be read against
    it)."""
    import platform
    rec = oracle_record()
    if rec.get("machine") != platform.machine() or "seconds_full" not in rec:
        return None
    return {"seconds_measured": rec["seconds_full"], "iters": rec["iters"],
            "machine": rec["machine"], "source": "oracle/iters_globular257.json "
            "(python -m oracle.calibrate: one complete oracle pass, grid to energy)"}


def cpu_baseline_obj(s: dict) -> dict:
    return {"value": 1.0 / s["t_solve"], "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"projection of one full solve from a measured sample: full FP64 setup "
                       f"({s['t_setup']:.1f} s), {s['pcg_iters_sampled']} PCG iterations after 2 "
                       f"({s['t_iter']:.3f} s each) scaled to the oracle's own {s['iters']}, "
                       f"surface sums on {s['sampled_targets']} of {s['nflux']} flux points "
                       f"scaled, full pair sum; one host core, single-threaded C"),
            "seconds_per_solve_est": s["t_solve"], "full_solve_check": full_solve_check()}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample(wl, pcg_iters=1, targets=200)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(wl))
    wall = time.perf_counter() - t0
    t_solve = statistics.mean(v["t_solve"] for v in vals)
    value = 1.0 / t_solve
    # each step is one measured sample (ms_per_step is its wall time); the
    # value projects one full solve from the samples
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_obj(args, wl),
            "cpu_baseline": dict(cpu_baseline_obj(vals[-1]), value=value),
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "value_kind": "projected seconds per full solve from the measured per-step samples",
            "projected_s_per_solve": t_solve, "sample_wall_s": wall}
    print(json.dumps(line))
    return 0


def config_obj(args, wl):
    return {"workload": f"globular molecule {wl['n_atoms']} atoms, uniform {wl['n']}^3 grid, "
                        f"fill {wl['fill']}, eps {wl['eps_in']:g}/{wl['eps_out']:g}, "
                        f"{wl['ionic']} M, zero Dirichlet BC, rtol {wl['rtol']:g}",
            "n_atoms": wl["n_atoms"], "grid": [wl["n"]] * 3, "seed": wl["seed"],
            "parallelism": f"independent problems x{args.gpus}",
            "l2": "inputs larger than L2 (working set ~1 GB per solve)"}


# ------------------------------------------------------------ batched --
BATCH_SIZES = (65, 97, 129, 161, 193)


def run_batched(args, pb, pb_inputs, torch):
    """256 uneven molecules (atom counts log-uniform in [200, 3000], molecule
    i seeded 4000 + i), uniform grids of spacing 0.5 A, solved to 1e-8 by
    one graph-launched batch; beside them the same systems solved one at a
    time by plain FP64 Jacobi-PCG."""
    from paper_2502_09323_gb300 import serving
    count = args.batch_count
    mols = pb_inputs.batch_molecules(count, 4000, 200, 3000)
    specs = [serving.uniform_spec(a, h=0.5, fill=1.5, sizes=BATCH_SIZES) for a in mols]
    params = pb.Params()
    systems = []
    for a, sp in zip(mols, specs):
        g = pb.pb_build_grid(sp, a)
        s = pb.pb_assemble_coeffs(g, params)
        pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
        systems.append(s)
    mixed = pb.SolveOpts(precision=pb.MIXED, rtol=1e-8)
    fp64 = pb.SolveOpts(precision=pb.FP64, rtol=1e-8)
    # warm-up: tune every grid shape once (both precisions)
    first = {}
    for i, sp in enumerate(specs):
        first.setdefault(sp.n, i)
    warm = [systems[i] for i in first.values()]
    pb.pb_solve_batch(warm, mixed)
    for s in warm:
        pb.pb_solve(s, fp64)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    st = pb.pb_solve_batch(systems, mixed)
    b.record(stream)
    torch.cuda.synchronize()
    t_mixed = a.elapsed_time(b) / 1e3
    e_mixed = [pb.pb_energy(s)["e_total"] for s in systems[:8]]
    a.record(stream)
    st64 = [pb.pb_solve(s, fp64) for s in systems]
    b.record(stream)
    torch.cuda.synchronize()
    t64 = a.elapsed_time(b) / 1e3
    e64 = [pb.pb_energy(s)["e_total"] for s in systems[:8]]
    # the oracle's throughput on a seeded subsample of the batch: every
    # sampled molecule is one complete oracle pass on the grid of its GPU
    # solve, in its own host process; the GPU energies of the same molecules
    # (mixed precision, from the batch above) are compared with the oracle's
    cpu = None
    if not args.no_cpu_baseline:
        import numpy as np
        rng = np.random.Generator(np.random.PCG64(4001))
        pick = sorted(int(i) for i in rng.choice(count, size=min(16, count), replace=False))
        procs = args.oracle_procs or min(host_cores(), len(pick))
        e_gpu = {}
        for i in pick:
            pb.pb_solve_batch([systems[i]], mixed)
            e_gpu[i] = pb.pb_energy(systems[i])["e_total"]
        jobs = [(mols[i], specs[i].n[0], specs[i].origin, specs[i].h) for i in pick]
        with oracle_pool(procs) as pool:
            t0 = time.perf_counter()
            res = list(pool.map(_oracle_uniform_job, jobs))
            wall = time.perf_counter() - t0
        secs = [r[0] for r in res]
        cpu = {"value": len(pick) / wall, "unit": "solves/s", "cores": procs, "kind": "oracle",
               "sample": (f"{len(pick)} of the {count} molecules (seeded choice, grids "
                          f"{sorted({specs[i].n[0] for i in pick})}), each one complete oracle "
                          f"pass (grid to energy, FP64 PCG to 1e-8) in its own process, {procs} "
                          f"processes on {host_cores()} host cores; value = sampled molecules / "
                          "wall time of the sample"),
               "sample_wall_s": wall, "seconds_per_molecule": secs,
               "projected_batch_s": sum(secs) / procs * count / len(pick),
               "energy_rel_diff_gpu_vs_oracle_max": max(
                   abs(e_gpu[i] - r[2]) / abs(r[2]) for i, r in zip(pick, res))}
    dof = [x["dof"] for x in st]
    iters = [x["iters_inner"] for x in st]
    shapes = {}
    for sp in specs:
        shapes[sp.n[0]] = shapes.get(sp.n[0], 0) + 1
    # the autotuner's tile width and z-chunk per grid shape
    tiles = {str(sp.n[0]): {"tile_width": x["kc"] // 10000, "z_chunk": x["kc"] % 1000}
             for sp, x in zip(specs, st)}
    out = {
        "workload": f"{count} globular molecules, atoms log-uniform [200, 3000] (seed 4000 + i), "
                    f"uniform grids h = 0.5 A, n in {list(BATCH_SIZES)}, fill 1.5, eps 2/80, "
                    "0.145 M, zero BC, rtol 1e-8",
        "grids": {str(k): v for k, v in sorted(shapes.items())},
        "tuned_tiles": dict(sorted(tiles.items(), key=lambda kv: int(kv[0]))),
        "solves_per_s": count / t_mixed, "seconds": t_mixed,
        "fp64_plain_solves_per_s": count / t64, "fp64_seconds": t64,
        "speedup_mixed_over_fp64": t64 / t_mixed,
        "dof_total": int(sum(dof)),
        "dof_iter_per_s": sum(d * i for d, i in zip(dof, iters)) / t_mixed,
        "iters_inner_mean": statistics.mean(iters),
        "true_rel_res_max": max(x["true_rel_res"] for x in st),
        "fp64_true_rel_res_max": max(x["true_rel_res"] for x in st64),
        "all_converged": all(x["status"] == 0 for x in st) and all(x["status"] == 0 for x in st64),
        "energy_rel_diff_mixed_vs_fp64_max": max(abs(m - f) / abs(f) for m, f in zip(e_mixed, e64)),
        "cpu_baseline": cpu,
    }
    del systems
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- octree --
OCTREE = dict(n_atoms=20000, seed=3, radius=45.0, h_fine=0.25, h_bulk=1.0, refine_dist=3.0,
              fill=1.5, rtol=1e-8)


def run_octree(args, pb, pb_inputs, torch, steps=3, warmup=1, fp64=True):
    """20,000-atom molecule (45 A ball, seed 3) on a 2:1-balanced brick
    octree: 0.25 A cells within 3 A of the atom spheres, 1 A bulk; whole hot
    path per step (build, coefficients, Coulomb terms, mixed solve to 1e-8,
    energy), and the plain FP64 solve of the same system."""
    import numpy as np
    wl = dict(OCTREE)
    if args.octree_atoms != wl["n_atoms"]:
        # same density: the ball radius scales with the cube root of the count
        wl["radius"] = wl["radius"] * (args.octree_atoms / wl["n_atoms"]) ** (1.0 / 3.0)
        wl["n_atoms"] = args.octree_atoms
    atoms = pb_inputs.globular_molecule(wl["n_atoms"], seed=wl["seed"], radius=wl["radius"])
    atoms_dev = torch.tensor(atoms, device="cuda")
    spec = pb.OctreeSpec(h_fine=wl["h_fine"], h_bulk=wl["h_bulk"], refine_dist=wl["refine_dist"],
                         fill=wl["fill"])
    params = pb.Params()

    ev_s0 = torch.cuda.Event(enable_timing=True)
    ev_s1 = torch.cuda.Event(enable_timing=True)

    def step(precision):
        g = pb.pb_build_grid(spec, atoms_dev)
        s = pb.pb_assemble_coeffs(g, params)
        pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
        # device time of the solve alone (the host-side figure of pb_solve
        # also counts the build and Coulomb kernels still queued at its call)
        ev_s0.record(torch.cuda.current_stream())
        st = pb.pb_solve(s, pb.SolveOpts(precision=precision, rtol=wl["rtol"]))
        ev_s1.record(torch.cuda.current_stream())
        return st, pb.pb_energy(s), s

    for _ in range(warmup):
        step(pb.MIXED)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s = None
    for _ in range(steps):
        s = None  # release the previous system's memory to the allocator first
        st, e, s = step(pb.MIXED)
    b.record(stream)
    torch.cuda.synchronize()
    t_step = a.elapsed_time(b) / 1e3 / steps
    t_solve = ev_s0.elapsed_time(ev_s1) / 1e3  # the last timed step's solve
    info = s.grid.info
    kinds = np.bincount(pb.pb_get_array(s.grid, "oct_kind"), minlength=4)
    out = {
        "workload": f"{wl['n_atoms']} atoms in a {wl['radius']:g} A ball (seed {wl['seed']}), brick octree "
                    f"h {wl['h_fine']:g}..{wl['h_bulk']:g} A, refined within {wl['refine_dist']:g} A of "
                    f"the atom spheres, fill {wl['fill']:g}, eps 2/80, 0.145 M, zero BC, rtol {wl['rtol']:g}",
        "bricks": int(info.n_bricks), "levels": int(info.n_levels), "slots": int(info.n_nodes),
        "dof": int(st["dof"]), "transition_rows": int(kinds[3]), "hanging": int(kinds[2]),
        "crossing_edges": int(info.n_cross),
        "solves_per_s": 1.0 / t_step, "ms_per_step": 1e3 * t_step,
        "solve_seconds": t_solve, "iters_inner": st["iters_inner"],
        "iters_outer": st["iters_outer"], "true_rel_res": st["true_rel_res"],
        "dof_iter_per_s": st["iters_inner"] * st["dof"] / t_solve,
        "energy_kT": e,
    }
    # live kernel timing of the brick kernels (pure rows)
    kt = {}
    for which, name in ((1, "update"), (0, "direction")):
        pb.pb_profile_kernels(s, pb.MIXED, which, 3)
        torch.cuda.synchronize()
        a.record(stream)
        pb.pb_profile_kernels(s, pb.MIXED, which, 20)
        b.record(stream)
        torch.cuda.synchronize()
        kt[name] = a.elapsed_time(b) / 1e3 / 20
    out["kernels"] = {
        "update_s": kt["update"], "direction_s": kt["direction"],
        "update_achieved_gbs": info.n_nodes * ALG_BYTES_U32 / kt["update"] / 1e9,
        "direction_achieved_gbs": info.n_nodes * ALG_BYTES_P32 / kt["direction"] / 1e9,
        "alg_bytes": "21 B (update) / 13 B (direction) per node slot"}
    if fp64:
        del s
        torch.cuda.synchronize()
        a.record(stream)
        st64, e64, s64 = step(pb.FP64)
        b.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / 1e3
        out["fp64_plain"] = {"solves_per_s": 1.0 / t64,
                             "solve_seconds": ev_s0.elapsed_time(ev_s1) / 1e3,
                             "iters": st64["iters_inner"], "true_rel_res": st64["true_rel_res"],
                             "e_total": e64["e_total"]}
        out["speedup_mixed_over_fp64"] = t64 / t_step
        out["energy_rel_diff_mixed_vs_fp64"] = abs(e["e_total"] - e64["e_total"]) / abs(e64["e_total"])
        del s64
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ serving --
def run_serving(args, pb, pb_inputs, torch):
    """Poisson stream of solves (atom counts log-uniform in [300, 50000],
    arrivals and counts seeded 5000, molecule j seeded 5000 + j) served with
    continuous batching under a 150 GB device-memory budget, on brick octrees
    of 0.25 A finest spacing (1 A bulk, refined within 3 A of the atom
    spheres), or on uniform grids of spacing 0.5 A."""
    from paper_2502_09323_gb300 import serving
    count = args.serve_requests
    octree = args.serve_grid == "octree"
    rate = args.serve_rate if args.serve_rate else (1.5 if octree else 6.0)
    h = 0.25 if octree else 0.5
    sizes = pb_inputs.batch_sizes(count, 5000, 300, 50000)
    arrivals = pb_inputs.poisson_arrivals(count, rate, seed=5000)
    reqs = [serving.Request(rid=j, atoms=pb_inputs.globular_molecule(int(n), seed=5000 + j),
                            arrival_s=float(t)) for j, (n, t) in enumerate(zip(sizes, arrivals))]
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-8)
    # warm-up: uniform grids let the autotuner see every grid shape of the
    # stream once; octree grids run one small solve through the engine
    shapes = [] if octree else sorted({serving.uniform_spec(r.atoms, h=h).n[0] for r in reqs})
    with pb.Engine(capacity=4, opts=opts) as eng:
        for n in shapes:
            one = pb_inputs.globular_molecule(40, seed=n)
            g = pb.pb_build_grid(pb.GridSpec(n=(n, n, n), origin=(-0.25 * (n - 1),) * 3, h=0.5),
                                 one)
            s = pb.pb_assemble_coeffs(g, pb.Params())
            eng.submit(s)
            while not eng.wait(timeout_s=0.1):
                pass
            del s, g
        if octree:
            one = pb_inputs.globular_molecule(300, seed=4999)
            g = pb.pb_build_grid(serving.octree_spec(one, h_fine=h), one)
            s = pb.pb_assemble_coeffs(g, pb.Params())
            eng.submit(s)
            while not eng.wait(timeout_s=0.1):
                pass
            del s, g
    torch.cuda.synchronize()
    launches0 = pb.pb_kernel_launches()
    with serving.Server(capacity=64, hbm_budget_bytes=150e9, opts=opts, h=h,
                        grid=args.serve_grid) as srv:
        recs = srv.run(reqs)
        max_used = srv.max_used
    launches = pb.pb_kernel_launches() - launches0
    summ = serving.latency_summary(recs)
    # one small request again with plain FP64 on the GPU: energy difference
    small = min(reqs, key=lambda r: len(r.atoms))
    g = pb.pb_build_grid(small.spec, small.atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params())
    pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
    pb.pb_solve(s, pb.SolveOpts(precision=pb.FP64, rtol=1e-10))
    e64 = pb.pb_energy(s)["e_total"]
    em = next(r for r in recs if r["rid"] == small.rid)["energy"]["e_total"]
    dofs = [r["stats"]["dof"] for r in recs]
    out = {
        "workload": f"{count} requests, Poisson arrivals at {rate:g}/s (seed 5000), "
                    "globular molecules with atoms log-uniform [300, 50000], "
                    + ("brick octrees h 0.25..1 A refined within 3 A of the atom spheres"
                       if octree else "uniform grids h = 0.5 A (32k+1 nodes per axis)")
                    + ", fill 1.5, mixed precision to 1e-8, 150 GB budget, 64 slots",
        "grid": args.serve_grid,
        "rate_hz": rate, **summ,
        "engine_mean_ms": 1e3 * statistics.mean(r["engine_s"] for r in recs),
        "max_budget_used_gb": max_used / 1e9,
        "dof_max": int(max(dofs)),
        "dof_total": int(sum(dofs)),
        "all_converged": all(r["stats"]["status"] == 0 for r in recs),
        "true_rel_res_max": max(r["stats"]["true_rel_res"] for r in recs),
        "energy_rel_diff_vs_fp64_gpu": abs(em - e64) / abs(e64),
        "gpu_launches": int(launches),
    }
    del s, g
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def _oracle_uniform_job(job):
    """One complete oracle pass (grid to energy) of one molecule on the grid
    of its GPU solve, in a worker process; returns (seconds, iterations,
    E_total)."""
    atoms, n, origin, h = job
    from oracle import oracle as orc
    g = orc.Grid((n, n, n), origin, h)
    t0 = time.perf_counter()
    r = orc.solve_problem(atoms, g, rtol=1e-8, with_energy=True)
    return time.perf_counter() - t0, int(r["iters"]), float(r["energy"]["e_total"])


def _oracle_octree_job(job):
    """Octree oracle pass (grid to energy) of one served molecule."""
    atoms, h_fine, h_bulk, refine_dist, fill = job
    from oracle import octree
    from oracle import oracle as orc
    orc.build()
    t0 = time.perf_counter()
    tree = octree.build(atoms, h_fine, h_bulk, refine_dist, fill=fill)
    r = octree.solve_problem(atoms, tree, rtol=1e-10)
    return time.perf_counter() - t0, float(r["energy"]["e_total"])


def oracle_pool(procs: int):
    """Worker processes for the oracle, started with spawn (never forked
    from a process that holds a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import oracle as orc
    orc.build()
    return cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_serve_sweep(args):
    """The serving workload at several Poisson rates (``inf``: every request
    arrives at once, the engine's saturation throughput); per rate the
    latency percentiles, throughput and budget used.  The two smallest
    requests are also solved by the octree oracle (FP64, rtol 1e-10) in host
    processes while the GPU serves, and their served energies are compared
    with it."""
    import torch

    import paper_2502_09323_gb300 as pb
    import pb_inputs
    from paper_2502_09323_gb300 import build, serving
    count = args.serve_requests
    rates = [float(r) for r in args.serve_sweep.split(",")]
    sizes = pb_inputs.batch_sizes(count, 5000, 300, 50000)
    mols = [pb_inputs.globular_molecule(int(n), seed=5000 + j) for j, n in enumerate(sizes)]
    small = sorted(range(count), key=lambda j: len(mols[j]))[:2]
    pool = oracle_pool(2)
    futs = {j: pool.submit(_oracle_octree_job, (mols[j], 0.25, 1.0, 3.0, 1.5)) for j in small}
    build.build()
    torch.cuda.set_device(0)
    opts = pb.SolveOpts(precision=pb.MIXED, rtol=1e-8)
    with pb.Engine(capacity=4, opts=opts) as eng:  # warm-up
        one = pb_inputs.globular_molecule(300, seed=4999)
        g = pb.pb_build_grid(serving.octree_spec(one), one)
        s = pb.pb_assemble_coeffs(g, pb.Params())
        eng.submit(s)
        while not eng.wait(timeout_s=0.1):
            pass
        del s, g
    points = []
    served_e = {}
    for rate in rates:
        if math.isinf(rate):
            arrivals = [0.0] * count
        else:
            arrivals = pb_inputs.poisson_arrivals(count, rate, seed=5000)
        reqs = [serving.Request(rid=j, atoms=mols[j], arrival_s=float(t))
                for j, t in enumerate(arrivals)]
        with serving.Server(capacity=64, hbm_budget_bytes=150e9, opts=opts, h=0.25,
                            grid="octree") as srv:
            recs = srv.run(reqs)
            max_used = srv.max_used
        for r in recs:
            if r["rid"] in small and r["rid"] not in served_e:
                served_e[r["rid"]] = r["energy"]["e_total"]
        summ = serving.latency_summary(recs)
        points.append({"rate_hz": rate if not math.isinf(rate) else "all at once", **summ,
                       "max_budget_used_gb": max_used / 1e9,
                       "all_converged": all(r["stats"]["status"] == 0 for r in recs),
                       "true_rel_res_max": max(r["stats"]["true_rel_res"] for r in recs)})
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    oracle = []
    for j in small:
        secs, e_orc = futs[j].result()
        oracle.append({"rid": j, "atoms": len(mols[j]), "e_total_served": served_e[j],
                       "e_total_oracle": e_orc, "rel_diff": abs(served_e[j] - e_orc) / abs(e_orc),
                       "oracle_seconds": secs})
    pool.shutdown()
    offered = [p["rate_hz"] for p in points]
    print(json.dumps({"serving_sweep": {
        "workload": f"{count} requests per rate, Poisson arrivals (seed 5000), globular molecules "
                    "with atoms log-uniform [300, 50000] (molecule j seeded 5000 + j), brick "
                    "octrees h 0.25..1 A refined within 3 A of the atom spheres, fill 1.5, mixed "
                    "precision to 1e-8, 150 GB budget, 64 slots",
        "rates_offered": offered, "points": points,
        "saturation_solves_per_s": max(p["solves_per_s"] for p in points),
        "energy_vs_octree_oracle": oracle}}))
    return 0


# ------------------------------------------------------------- ranks --
def max_over_ranks_of(v: float, dist, device) -> float:
    """Largest value over all ranks (the slowest rank's time); v itself
    without a process group."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps: int, world: int, elapsed_max_s: float) -> float:
    """Units processed by all ranks (one workload copy per rank and step)
    per second of the slowest rank."""
    return steps * world / elapsed_max_s


# ------------------------------------------------------------------ ours --
def run_ours(args, wl):
    import numpy as np
    import torch

    import paper_2502_09323_gb300 as pb
    import pb_inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2502_09323_gb300 import build
    build.build()

    atoms_np = pb_inputs.globular_molecule(wl["n_atoms"], seed=wl["seed"])
    atoms_dev = torch.tensor(atoms_np, device=dev)
    atoms_pin = torch.tensor(atoms_np).pin_memory()
    spec = pb.GridSpec(n=(wl["n"],) * 3, fill=wl["fill"])
    params = pb.Params(eps_in=wl["eps_in"], eps_out=wl["eps_out"], ionic_strength_M=wl["ionic"],
                       bc=wl["bc"])

    def step(atoms, precision):
        g = pb.pb_build_grid(spec, atoms)
        s = pb.pb_assemble_coeffs(g, params)
        if args.tuning and precision == pb.MIXED:
            v, kc = (int(t) for t in args.tuning.split(":"))
            pb.pb_set_tuning(s, pb.MIXED, v, kc)
        pb.pb_coulomb_terms(s, pb.CT_SURFACE | pb.CT_PAIRS)
        st = pb.pb_solve(s, pb.SolveOpts(precision=precision, rtol=wl["rtol"]))
        e = pb.pb_energy(s)
        return st, e, s

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return max_over_ranks_of(v, dist, dev)

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        st, e, s = step(atoms_dev, pb.MIXED)
        del s
    # ---- timed region (device-resident inputs)
    clocks = ClockSampler(dev.index)
    barrier()
    launches0 = pb.pb_kernel_launches()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    lat = []
    stats = []
    ev0.record(stream)
    s = last_sys = None
    for _ in range(args.steps):
        # the previous step's system is released first, so its device memory
        # returns to the caching allocator before this step allocates
        s = last_sys = None
        t0 = time.perf_counter()
        st, e, s = step(atoms_dev, pb.MIXED)
        lat.append(time.perf_counter() - t0)
        stats.append(st)
        last_sys = s
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = pb.pb_kernel_launches() - launches0
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    value = whole_job_rate(args.steps, world, elapsed)
    energy = e
    dof = stats[-1]["dof"]
    iters = statistics.mean(s_["iters_inner"] for s_ in stats)
    solve_s = statistics.mean(s_["seconds"] for s_ in stats)

    # ---- end to end through host buffers (pinned atoms in, energies out)
    barrier()
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        st2, e2, s2 = step(atoms_pin, pb.MIXED)
        del s2
    ev3.record(stream)
    barrier()
    e2e_elapsed = max_over_ranks(ev2.elapsed_time(ev3) / 1e3)

    # ---- plain FP64 Jacobi-PCG, same workload
    fp64 = None
    if not args.no_fp64:
        step(atoms_dev, pb.FP64)
        barrier()
        ev4 = torch.cuda.Event(enable_timing=True)
        ev5 = torch.cuda.Event(enable_timing=True)
        k64 = max(1, min(2, args.steps))
        ev4.record(stream)
        st64 = []
        s64 = None
        for _ in range(k64):
            s64 = None  # as in the mixed loop: the previous system is released first
            st_, e64, s64 = step(atoms_dev, pb.FP64)
            st64.append(st_)
        ev5.record(stream)
        barrier()
        t64 = max_over_ranks(ev4.elapsed_time(ev5) / 1e3)
        fp64 = {"solves_per_s": k64 * world / t64, "iters": st64[-1]["iters_inner"],
                "true_rel_res": st64[-1]["true_rel_res"],
                "dof_iter_per_s": st64[-1]["iters_inner"] * dof / st64[-1]["seconds"],
                "e_total": e64["e_total"]}
        fp64["speedup_mixed_over_fp64"] = value / fp64["solves_per_s"]

    # ---- live kernel timing for the roofline (FP32 update kernel = dominant)
    peak, peak_kind = load_peaks()
    reps = 40
    kt = {}
    for which, name in ((1, "update"), (0, "direction")):
        pb.pb_profile_kernels(last_sys, pb.MIXED, which, 3)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        pb.pb_profile_kernels(last_sys, pb.MIXED, which, reps)
        b.record(stream)
        torch.cuda.synchronize()
        kt[name] = a.elapsed_time(b) / 1e3 / reps
    bytes_u = dof * ALG_BYTES_U32
    achieved = bytes_u / kt["update"] / 1e9
    # DRAM bytes of one launch from the stored ncu capture of this kernel on
    # this workload (a profiler run is not a bench run); null without it
    traffic, traffic_source = None, None
    tpath = os.path.join(ROOT, "profiles", "stencil_update_fp32_globular257.json")
    if os.path.exists(tpath) and wl["n"] == 257:
        with open(tpath) as fh:
            rec = json.load(fh)
        traffic = rec.get("dram_bytes_per_launch")
        traffic_source = rec.get("source")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_source,
                "kernel": ("k_stencil_tma<MODE_U> (FP32 PCG update, TMA-staged, persistent)"
                           if stats[-1]["kc"] >= 1000 else
                           "k_stencil<float,CoefC32,MODE_U> (FP32 PCG update)"),
                "z_chunk": stats[-1]["kc"] % 1000,
                "tile_width": stats[-1]["kc"] // 10000 or None,
                "alg_bytes_per_launch": bytes_u, "launch_s": kt["update"],
                "peak_kind": f"{peak_kind} hbm_gbs",
                "direction_kernel": {"launch_s": kt["direction"],
                                     "achieved_gbs": dof * ALG_BYTES_P32 / kt["direction"] / 1e9}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_obj(oracle_sample(wl))

    octree = None if args.no_octree else run_octree(args, pb, pb_inputs, torch)
    batched = None if args.no_batched else run_batched(args, pb, pb_inputs, torch)
    serving_line = None if args.no_serving else run_serving(args, pb, pb_inputs, torch)

    lat_ms = sorted(1e3 * v for v in lat)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32 inner PCG + fp64 refinement", "data": "synthetic",
        "config": config_obj(args, wl),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_rate(args.steps, world, e2e_elapsed), "unit": "solves/s",
                "h2d_bytes_per_step": int(atoms_np.nbytes), "d2h_bytes_per_step": 48},
        "gpu_launches": int(launches),
        "clocks": clk,
        "dof": dof, "iters_inner": iters, "iters_outer": stats[-1]["iters_outer"],
        "true_rel_res": stats[-1]["true_rel_res"],
        "dof_iter_per_s": iters * dof / solve_s, "solve_seconds": solve_s,
        "latency_ms": {"p50": lat_ms[len(lat_ms) // 2],
                       "p99": lat_ms[min(len(lat_ms) - 1, math.ceil(0.99 * len(lat_ms)) - 1)]},
        "fp64_plain": fp64,
        "energy_kT": energy,
        "octree": octree,
        "batched": batched,
        "serving": serving_line,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_profile_fp64(args, wl):
    """W + K whole-path steps with the plain FP64 solver only (for profiler
    captures of its kernels); prints the solve statistics."""
    import torch

    import paper_2502_09323_gb300 as pb
    import pb_inputs
    from paper_2502_09323_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    atoms = torch.tensor(pb_inputs.globular_molecule(wl["n_atoms"], seed=wl["seed"]), device="cuda")
    spec = pb.GridSpec(n=(wl["n"],) * 3, fill=wl["fill"])
    params = pb.Params(eps_in=wl["eps_in"], eps_out=wl["eps_out"], ionic_strength_M=wl["ionic"],
                       bc=wl["bc"])
    out = []
    for i in range(args.warmup + args.steps):
        g = pb.pb_build_grid(spec, atoms)
        s = pb.pb_assemble_coeffs(g, params)
        st = pb.pb_solve(s, pb.SolveOpts(precision=pb.FP64, rtol=wl["rtol"]))
        if i >= args.warmup:
            out.append({k: st[k] for k in ("iters_inner", "true_rel_res", "seconds", "dof")})
        del s, g
    torch.cuda.synchronize()
    print(json.dumps({"profile_fp64": out, "grid": wl["n"]}))
    return 0


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.grid_n:
        wl = dict(wl, n=args.grid_n)
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.profile_fp64:
        return run_profile_fp64(args, wl)
    if args.serve_sweep:
        return run_serve_sweep(args)
    if args.octree_only:
        import torch

        import paper_2502_09323_gb300 as pb
        import pb_inputs
        from paper_2502_09323_gb300 import build
        build.build()
        torch.cuda.set_device(0)
        print(json.dumps({"octree": run_octree(args, pb, pb_inputs, torch, steps=args.steps,
                                               warmup=args.warmup, fp64=not args.no_fp64)}))
        return 0
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
