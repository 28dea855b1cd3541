#!/usr/bin/env python
"""Benchmark of the Coordinate Condensation hot path on one or more GB300s.

Workload (one "step"): quasistatic stretch of the jittered 32x32x32-cell
Kuhn cube (35 937 vertices, 196 608 tets; x = 0 face clamped, x = 1 face
pulled to 1.5), stable Neo-Hookean, 2-ring perturbation bases, coloured
Coordinate Condensation sweeps in mixed precision until the free gradient
norm drops by 1e-6 (max 800 sweeps), once for each E in {1e4, 1e5, 1e6, 1e7}.
Inputs are resident in HBM when a step starts; L2 is flushed between steps.

The metric is vertex-updates/s (free vertices x sweeps / solve time) and
time to tolerance; the same solves in plain float64 are timed beside them.
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
Multi-GPU (torchrun): each rank solves its own copy of the workload (weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# one BLAS thread per process: the oracle baseline below sets its own process
# count, and threaded BLAS inside each of its workers oversubscribes the cores
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ms to 1e-6 rel grad-norm & vertex-updates/s on 1 GB300, mixed/learned vs plain CC"
E_SWEEP = [1e4, 1e5, 1e6, 1e7]
DIMS = (32, 32, 32)
K_RING = 2
MAX_ITERS = 800
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flop/FMA x max SM clock
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "sweep_kernels_cube32.md")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(kernel_class, summary=None):
    """DRAM bytes per launch of a kernel class from a committed ncu summary
    (the sweep kernels' by default), or None when the kernel source changed
    since the capture (hash mismatch)."""
    import hashlib
    try:
        text = open(summary or PROFILE_SUMMARY).read()
    except OSError:
        return None
    for line in text.splitlines():
        if line.startswith("traffic:"):
            _, cls, nbytes, src, digest = line.split()
            if cls != kernel_class:
                continue
            path = os.path.join(ROOT, "paper_2510_12053_gb300", "csrc", src)
            try:
                cur = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
            except OSError:
                return None
            return float(nbytes) if cur == digest else None
    return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--nu", type=float, default=0.3)
    p.add_argument("--no-fp64", action="store_true", help="skip the plain float64 comparison solves")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--max-iters", type=int, default=MAX_ITERS, help="sweep cap per solve")
    p.add_argument("--check-every", type=int, default=8, help="sweeps between host residual checks")
    p.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of CUDA graphs")
    p.add_argument("--no-batch", action="store_true", help="skip the 256-mesh batched solve")
    p.add_argument("--headline", choices=["concurrent", "batch", "single"], default="concurrent",
                   help="time the configuration's four E solves side by side, each mesh on its own stream "
                        "(cc_solve_concurrent), as one 4-mesh batch (cc_solve_batch) or one mesh after another")
    p.add_argument("--batch-count", type=int, default=256)
    p.add_argument("--no-learned", action="store_true", help="skip the learned-basis workload")
    p.add_argument("--resolution-sweep", action="store_true",
                   help="add the SNH / FCR mesh-resolution sweep (8^3 .. 48^3 cubes)")
    p.add_argument("--resolution-max-iters", type=int, default=3000)
    p.add_argument("--large-beam", action="store_true",
                   help="add the throughput run on the 64x64x256-cell beam (1.09 M vertices)")
    p.add_argument("--large-sweeps", type=int, default=40)
    p.add_argument("--train-meshes", type=int, default=2000)
    p.add_argument("--train-steps", type=int, default=4000)
    p.add_argument("--train-batch", type=int, default=8192)
    p.add_argument("--learned-max-iters", type=int, default=2000, help="sweep cap of the 48^3 solves")
    p.add_argument("--no-nu045", action="store_true", help="skip the nu = 0.45 solves of the named configuration")
    p.add_argument("--cfg1-oracle", action="store_true",
                   help="add the oracle's CD / CC / JGS2 / Newton timings on the 8^3 cube (100 iterations each)")
    p.add_argument("--cpu-full-sweep", action="store_true",
                   help="add one whole coloured CC sweep of the oracle on the 32^3 cube, single-threaded")
    p.add_argument("--colors", choices=["lattice", "greedy"], default="lattice",
                   help="colouring of the coloured schedule: the Kuhn grid's (i+j+k) mod 4 (4 colours) or greedy (8)")
    p.add_argument("--no-cfg3", action="store_true",
                   help="skip the dynamic cantilever: 64x64x256 cells, 3-ring bases, backward Euler, 20 steps")
    p.add_argument("--cfg3-cells", type=str, default="64,64,256", help="beam cells nx,ny,nz")
    p.add_argument("--cfg3-steps", type=int, default=20)
    p.add_argument("--cfg3-sweeps", type=int, default=20, help="sweep cap per time step")
    return p.parse_args()


def scenes(nu):
    import meshgen
    return [meshgen.stretch_box(*DIMS, E=E, nu=nu, factor=1.5, jitter_amount=0.05, seed=0,
                                name=f"cube32_E{E:g}") for E in E_SWEEP]


COLORING = {"mode": "lattice"}


def colorize(mesh, scenes):
    """Colours a mesh (or a batch of meshes, in order) for the coloured
    schedule: the Kuhn grid's lattice colouring (i + j + k) mod 4 (four colour
    phases per sweep), or with --colors greedy the library's greedy colouring
    (eight on these grids)."""
    if COLORING["mode"] == "greedy":
        mesh.color()
        return
    import meshgen
    scs = scenes if isinstance(scenes, (list, tuple)) else [scenes]
    mesh.set_colors(np.concatenate([meshgen.lattice_colors(*sc.dims) for sc in scs]), num_colors=4)


def workload_config(nu, n, T, n_free):
    return {"workload": f"cube32_stretch: {DIMS[0]}x{DIMS[1]}x{DIMS[2]} cells x 6 tets ({n} vertices, {T} tets), "
                        f"jitter 5% seed 0, x=0 clamped, x=1 pulled to 1.5, SNH nu={nu}, E in {E_SWEEP}, "
                        f"{K_RING}-ring bases, coloured CC, tol 1e-6 rel grad-norm",
            "n_free": n_free, "k_ring": K_RING, "schedule": "colored", "update": "cc",
            "coloring": ("lattice (i+j+k) mod 4, 4 colours" if COLORING["mode"] == "lattice"
                         else "greedy in ascending id, 8 colours"),
            "nu": nu, "E_values": E_SWEEP, "cells": list(DIMS), "tol": 1e-6,
            "nu_note": "the named configuration's nu=0.45 diverges with 2-ring rest bases (oracle and GPU agree); "
                       "its outcome is reported under cfg_nu045",
            "l2": "flushed between steps (256 MiB write)", "inputs": "resident in HBM"}


# ----------------------------------------------------------------------------- clocks
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, nm in enumerate(names):
                    if r[3 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU)
# The float64 oracle timed on the host cores: one colour of a coloured CC
# sweep of the 32^3 cube, exactly as the oracle's sweep does it (gradient and
# Hessian assembly at the current x, then the local CC update of every free
# vertex of the colour, applied).  Bases (Eq. 5 on the 2-ring patch at rest)
# are built by the oracle beforehand and are not timed.  With several cores
# the local updates of the colour are split over worker processes (spawned;
# same-coloured vertices are independent), the assembly stays serial.
_OW = {}


def _ow_scene(nu):
    import meshgen
    return meshgen.stretch_box(*DIMS, E=E_SWEEP[1], nu=nu, factor=1.5, jitter_amount=0.05, seed=0)


def _ow_init(nu, bases=True):
    from oracle import fem, topology
    sc = _ow_scene(nu)
    pb = fem.problem_from_scene(sc)
    _OW["pb"] = pb
    if bases:
        _OW["nb"] = topology.vertex_neighbors(pb.n, pb.tets)
        _OW["H0"] = pb.hessian(pb.X)


def _ow_bases(verts):
    from oracle import subspace, topology
    pb, (nb_ptr, nb_idx), H0 = _OW["pb"], _OW["nb"], _OW["H0"]
    out = []
    for i in verts:
        S = np.array([j for j in topology.k_ring(int(i), K_RING, nb_ptr, nb_idx) if j != i and pb.free[j]],
                     dtype=np.int64)
        out.append((S, subspace.local_basis(H0, int(i), S)))
    return out


def _ow_updates(args):
    """Local CC updates of a chunk of the colour's vertices from g, H (and
    the bases) that the parent placed in shared memory."""
    import scipy.sparse as sps
    from multiprocessing import shared_memory
    from oracle import solvers
    verts, specs, shape = args
    handles = [shared_memory.SharedMemory(name=name) for name, _, _ in specs]
    try:
        views = [np.ndarray(shp, dtype=dt, buffer=h.buf) for h, (_, shp, dt) in zip(handles, specs)]
        data, indices, indptr, g, sptr, sidx, U = views
        H = sps.csr_matrix((data, indices, indptr), shape=shape, copy=False)
        d = np.empty((len(verts), 3))
        for k, (i, pos) in enumerate(verts):
            d[k] = solvers.local_update("cc", H, g, int(i), sidx[sptr[pos]:sptr[pos + 1]], U[sptr[pos]:sptr[pos + 1]])
        del H, data, indices, indptr, g, sptr, sidx, U, views
    finally:
        for h in handles:
            h.close()
    return d


class OracleColour:
    """Times the oracle on colour ``c`` of the 32^3 cube with ``cores``
    processes (1: in this process, no pool)."""

    def __init__(self, nu, cores, colour=0):
        from oracle import topology
        self.cores = max(1, int(cores))
        _ow_init(nu, bases=self.cores == 1)
        self.pb = _OW["pb"]
        self.x0 = _ow_scene(nu).x0
        import meshgen
        cols = meshgen.lattice_colors(*DIMS) if COLORING["mode"] == "lattice" else None
        topo = topology.Topology(self.pb.n, self.pb.tets, self.pb.free, colors=cols)
        self.verts = np.asarray(topo.color_classes(free_only=True)[colour], dtype=np.int64)
        self.pool = None
        self.shm = []
        chunks = np.array_split(self.verts, self.cores * 4)
        if self.cores > 1:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_ow_init, initargs=(nu,))
            parts = self.pool.map(_ow_bases, chunks)
        else:
            parts = [_ow_bases(c) for c in chunks]
        sb = [sb for part in parts for sb in part]
        self.sptr = np.zeros(len(sb) + 1, dtype=np.int64)
        self.sptr[1:] = np.cumsum([len(S) for S, _ in sb])
        self.sidx = np.concatenate([S for S, _ in sb]) if sb else np.zeros(0, np.int64)
        self.U = np.concatenate([U.reshape(-1, 3, 3) for _, U in sb]) if sb else np.zeros((0, 3, 3))
        self.chunks = [list(zip(c.tolist(), range(o, o + len(c))))
                       for c, o in zip(chunks, np.cumsum([0] + [len(c) for c in chunks[:-1]]))]

    def _put(self, name, a):
        from multiprocessing import shared_memory
        a = np.ascontiguousarray(a)
        h = shared_memory.SharedMemory(create=True, size=max(a.nbytes, 1))
        self.shm.append(h)
        np.ndarray(a.shape, dtype=a.dtype, buffer=h.buf)[...] = a
        return (h.name, a.shape, a.dtype.str)

    def step(self, x=None, serial=False):
        """One timed colour from x (default x0), its updates over the worker
        processes or (serial) in this process: returns (updates, seconds)."""
        from oracle import solvers
        x = np.array(self.x0 if x is None else x, dtype=np.float64, copy=True)
        t0 = time.perf_counter()
        g = self.pb.gradient(x)
        H = self.pb.hessian(x)
        if self.pool is None or serial:
            d = np.empty((len(self.verts), 3))
            for k, i in enumerate(self.verts):
                S = self.sidx[self.sptr[k]:self.sptr[k + 1]]
                d[k] = solvers.local_update("cc", H, g, int(i), S, self.U[self.sptr[k]:self.sptr[k + 1]])
        else:
            specs = [self._put("d", H.data), self._put("i", H.indices), self._put("p", H.indptr), self._put("g", g),
                     self._put("sp", self.sptr), self._put("si", self.sidx), self._put("U", self.U)]
            d = np.concatenate(self.pool.map(_ow_updates, [(c, specs, H.shape) for c in self.chunks]))
        x[self.verts] += d
        dt = time.perf_counter() - t0
        for h in self.shm:
            h.close()
            h.unlink()
        self.shm = []
        return len(self.verts), dt

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


def host_info():
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model") and model is None:
                model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def oracle_baseline(nu, cores=None, serial=True):
    """Measured oracle rate (vertex-updates/s) on colour 0 of the 32^3 cube:
    one timed colour with its updates over ``cores`` processes (default:
    every host core) and, with ``serial``, one timed colour in one process."""
    cores = os.cpu_count() if cores is None else cores
    oc = OracleColour(nu, cores)
    try:
        u, t = oc.step()
        out = {"value": u / t, "cores": oc.cores, "s": t, "updates": u}
        if serial:
            u1, t1 = oc.step(serial=True)
            out["single_thread"] = {"value": u1 / t1, "cores": 1, "s": t1, "updates": u1}
    finally:
        oc.close()
    return out


def cfg1_oracle_timings(max_iters=100):
    """The 8^3 cube (729 vertices, 3 072 tets; E = 1e5, nu = 0.45, 1.5x stretch,
    2-ring bases, float64) solved by the oracle with CD, CC and JGS2 sweeps
    (coloured) and Newton, ``max_iters`` iterations each: seconds, iterations
    run and the final relative residual (a divergence ends the run early)."""
    import meshgen
    from oracle import fem, solvers, subspace, topology
    sc = meshgen.cube8_stretch(E=1e5)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    t0 = time.perf_counter()
    sup, U = subspace.build_local_bases(pb, topo, K_RING)
    out = {"workload": f"cube8_stretch: 8x8x8 cells ({pb.n} vertices, {pb.T} tets), E=1e5, "
                       f"nu={sc.material.nu}, 1.5x, 2-ring bases, float64 oracle",
           "basis_build_s": time.perf_counter() - t0}
    for kind in ("cd", "cc", "jgs2", "newton"):
        t0 = time.perf_counter()
        try:
            with np.errstate(all="ignore"):
                if kind == "newton":
                    _, h = solvers.newton(pb, sc.x0, tol=1e-30, max_iters=max_iters)
                else:
                    _, h = solvers.solve(pb, topo, sup, U, sc.x0, kind=kind, tol=1e-30, max_iters=max_iters)
            g = np.asarray(h.grad_norm)
            rec = {"iterations": h.iterations, "rel_residual": float(g[-1] / g[0]),
                   "min_rel_residual": float(np.nanmin(g / g[0]))}
        except Exception as e:   # a diverged iteration (singular local solve) ends the run
            rec = {"iterations": None, "error": f"{type(e).__name__}: {e}"}
        rec["s"] = time.perf_counter() - t0
        out[kind] = rec
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    sc = _ow_scene(args.nu)
    n_free = int((sc.pinned == 0).sum())
    cores = os.cpu_count()
    oc = OracleColour(args.nu, cores)
    try:
        for _ in range(args.warmup):
            oc.step()
        ups, secs, per = 0, 0.0, []
        for _ in range(args.steps):
            u, t = oc.step()
            ups += u
            secs += t
            per.append(t)
    finally:
        oc.close()
    value = ups / secs
    sample = (f"per step: colour 0 of one coloured CC sweep of the full 32^3 cube ({len(oc.verts)} of {n_free} "
              f"free vertices): float64 gradient + Hessian assembly at x0 (serial), then every local CC update of "
              f"the colour over {cores} processes; 2-ring oracle bases built beforehand (untimed)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "vertex-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.nu, sc.n, sc.T, n_free),
        "cpu_baseline": {"value": value, "unit": "vertex-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "host": host_info(), "s_per_step": per},
        "e2e": {"value": value, "unit": "vertex-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- ranks
def reduce_over_ranks(x: float, world: int, device, op: str) -> float:
    """A host number reduced over all ranks ("max": the slowest rank's time;
    "sum": the units every rank processed).  One rank: x itself."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units: float, ms: float, world: int, device) -> float:
    """Units per second of the whole job: the units all ranks processed over
    the slowest rank's time."""
    total_units = reduce_over_ranks(units, world, device, "sum")
    slowest_ms = reduce_over_ranks(ms, world, device, "max")
    return total_units / (slowest_ms / 1e3)


# ----------------------------------------------------------------------------- GPU
def local_solve_flops(mesh):
    """Algorithmic float32 FLOPs of the coupling products per free vertex:
    2 x 27 per (j, l) block pair in S x S with H_jl != 0 (Y_j = sum H_jl U_l),
    2 x (27 + 9) per j in S (U_j^T Y_j and U_j^T g_j), 2 x 27 per l in S in
    row i (A).  Returns an array over vertices (0 for pinned)."""
    nb_ptr, nb_idx = mesh.export("nbr_ptr"), mesh.export("nbr_idx")
    sp, si = mesh.export("sup_ptr"), mesh.export("sup_idx")
    n = len(sp) - 1
    out = np.zeros(n)
    insup = np.zeros(n, dtype=bool)
    for i in range(n):
        S = si[sp[i]:sp[i + 1]]
        if len(S) == 0:
            continue
        insup[S] = True
        pairs = 0
        for j in S:
            row = nb_idx[nb_ptr[j]:nb_ptr[j + 1]]
            pairs += int(insup[row].sum()) + 1
        rowi = nb_idx[nb_ptr[i]:nb_ptr[i + 1]]
        out[i] = 2 * (27 * pairs + 36 * len(S) + 27 * int(insup[rowi].sum()))
        insup[S] = False
    return out


def gather_bytes_per_refresh(scene):
    """Algorithmic bytes of one row-gather launch (all free rows): per row the
    stored blocks it sums (per incident tet its 24-byte diagonal block and a
    36-byte block per other corner with a vertex id above the row's), its
    24-byte float-float gradient entries, its upper blocks written and its
    gradient written."""
    tets = np.asarray(scene.tets, dtype=np.int64)
    free = scene.pinned == 0
    n = scene.n
    ge = tets[:, None, :] >= tets[:, :, None]          # [T, v, w]: vid[w] >= vid[v]
    src = np.zeros(n)
    np.add.at(src, tets.ravel(), ge.sum(axis=2).ravel())
    val = np.bincount(tets.ravel(), minlength=n)
    nup = np.zeros(n)
    pairs = set()
    for a in range(4):
        for c in range(4):
            if a != c:
                pairs.update(zip(tets[:, a].tolist(), tets[:, c].tolist()))
    for (j, l) in pairs:
        if l > j:
            nup[j] += 1
    nup += 1
    per = (src - val) * 36 + val * 24 + val * 24 + nup * 36 + 24
    return float(per[free].sum())


# ids, slots, D_m^-1, V w, positions; gradient + 10 blocks (4 diagonal ones as 6 values, 6 others as 9)
TET_BYTES = 16 + 16 + 72 + 12 + 4 * 32 + 4 * 24 + 4 * (4 * 6 + 6 * 9)


def run_batch(args, stream, dev):
    """Batch of independent boxes (sides U{4..24} cells, E log-uniform
    [1e4, 1e7], nu U[0.30, 0.49], a random face clamped and the opposite one
    stretched by U[1.1, 1.8], seed 0) solved as one union with per-mesh
    convergence, CUDA-graph replay and autotuned launch shapes."""
    import torch
    import meshgen
    import paper_2510_12053_gb300 as cc
    scenes = meshgen.random_boxes(args.batch_count, seed=0)
    t0 = time.perf_counter()
    batch = cc.Mesh.from_scenes(scenes, stream=stream)
    colorize(batch, scenes)
    batch.build_subspace(K_RING)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    x0 = cc.to_soa(np.concatenate([sc.x0 for sc in scenes]), device=dev)
    tune = batch.autotune(x0, precision="mixed", sweeps=3)
    x = torch.empty_like(x0)
    x.copy_(x0)
    batch.solve_batch(x, precision="mixed", tol=1e-6, max_iters=16, check_every=8, use_graph=True)  # warm-up
    x.copy_(x0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    res = batch.solve_batch(x, precision="mixed", tol=1e-6, max_iters=args.max_iters // 2, check_every=8,
                            use_graph=True)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    nfree = np.array([int((sc.pinned == 0).sum()) for sc in scenes])
    applied = int((nfree * res["iterations"]).sum())
    nus = np.array([sc.material.nu for sc in scenes])

    def buckets(r):
        out = {}
        for name, sel in (("nu<0.35", nus < 0.35), ("nu>=0.35", nus >= 0.35)):
            st = r["status"][sel]
            out[name] = {"meshes": int(sel.sum()), "converged": int((st == 1).sum()),
                         "diverged": int((st == -1).sum()), "not_reached": int((st == 0).sum())}
        return out

    # the same batch with the per-mesh global line search (Sec. 4.4): meshes
    # that plain CC blows up take damped steps instead of diverging
    x.copy_(x0)
    torch.cuda.synchronize()
    ev0.record(stream)
    res_ls = batch.solve_batch(x, precision="mixed", tol=1e-6, max_iters=args.max_iters // 2, check_every=8,
                               line_search=True)
    ev1.record(stream)
    ev1.synchronize()
    ms_ls = ev0.elapsed_time(ev1)
    # launch gaps of the graph replay: 16 sweeps timed plain, then the same 16
    # sweeps with every kernel class timed by events; sum of kernel time vs wall
    x.copy_(x0)
    batch.solve_batch(x, precision="mixed", tol=0.0, max_iters=16, check_every=16, use_graph=True)
    x.copy_(x0)
    torch.cuda.synchronize()
    ev0.record(stream)
    batch.solve_batch(x, precision="mixed", tol=0.0, max_iters=16, check_every=16, use_graph=True)
    ev1.record(stream)
    ev1.synchronize()
    wall16 = ev0.elapsed_time(ev1)
    batch.profile_enable(True)
    x.copy_(x0)
    batch.solve_batch(x, precision="mixed", tol=0.0, max_iters=16, check_every=16, use_graph=True)
    x.copy_(x0)
    batch.solve_batch(x, precision="mixed", tol=0.0, max_iters=16, check_every=16, use_graph=True)
    torch.cuda.synchronize()
    prof = batch.profile_read()
    batch.profile_enable(False)
    kern16 = sum(prof[k]["ms"] for k in cc.PROFILE_CLASSES) / 2.0
    # the same meshes solved one after another (first 16, warm, launch by launch)
    loop_ms, loop_upd = 0.0, 0
    for sc in scenes[:16]:
        m = cc.Mesh.from_scene(sc, stream=stream)
        colorize(m, sc)
        m.build_subspace(K_RING)
        xs = cc.to_soa(sc.x0, device=dev)
        a, bq = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        try:
            r = m.solve_step(xs, precision="mixed", tol=1e-6, max_iters=args.max_iters // 2, check_every=8)
            iters = r.iterations
        except cc.CCError:   # a diverging mesh (non-finite update) ends its solve early
            iters = 0
        bq.record(stream)
        bq.synchronize()
        loop_ms += a.elapsed_time(bq)
        loop_upd += int((sc.pinned == 0).sum()) * iters
        m.close()
    out = {"meshes": len(scenes), "vertices": int(sum(sc.n for sc in scenes)),
           "tets": int(sum(sc.T for sc in scenes)), "setup_ms": setup_ms, "autotune": tune,
           "ms_until_all_stopped": ms, "sweeps_launched": int(res["sweeps"]),
           "converged": int((res["status"] == 1).sum()), "diverged": int((res["status"] == -1).sum()),
           "not_reached": int((res["status"] == 0).sum()), "by_nu": buckets(res),
           "applied_vertex_updates_per_s": applied / (ms / 1e3),
           "line_search": {"ms_until_all_stopped": ms_ls, "sweeps_launched": int(res_ls["sweeps"]),
                           "converged": int((res_ls["status"] == 1).sum()),
                           "diverged": int((res_ls["status"] == -1).sum()),
                           "not_reached": int((res_ls["status"] == 0).sum()), "by_nu": buckets(res_ls),
                           "max_sweeps": args.max_iters // 2},
           "graph_replay_16_sweeps": {"wall_ms": wall16, "sum_of_kernel_ms": kern16,
                                      "note": "kernel time summed over classes from event-timed replays; "
                                              "wall minus that sum bounds what a persistent kernel could save"},
           "looped_single_mesh_solves": {"meshes": 16, "ms": loop_ms,
                                         "vertex_updates_per_s": loop_upd / (loop_ms / 1e3)},
           "note": "nu >= 0.35 diverges with 2-ring rest bases; such meshes are frozen when their residual "
                   "exceeds 1e6 x its start; with the line search they stall instead (not reached)"}
    batch.close()
    return out


def mlp_flops(dims, rows, backward=False):
    """Algorithmic GEMM FLOPs of the network over ``rows`` rows: 2 rows N K
    per layer forward; backward adds the weight gradients (2 rows N K per
    layer) and the input gradients of every layer but the first."""
    nk = [dims[l + 1] * dims[l] for l in range(len(dims) - 1)]
    f = 2.0 * rows * sum(nk)
    if backward:
        f += 2.0 * rows * sum(nk) + 2.0 * rows * sum(nk[1:])
    return f


def run_resolution(args, stream, dev):
    """Mesh-resolution sweep with both materials: jittered n^3 stretch cubes
    (E = 1e5, nu = 0.3, 1.5x, seed 0) for n in 8..48, solved to 1e-6 with
    mixed-precision coloured CC on 2-ring rest bases; SNH and FCR with fixed
    bases, FCR with corotated bases.  Sweeps and time to tolerance per case."""
    import torch
    import meshgen
    import paper_2510_12053_gb300 as cc
    out = []
    for side in (8, 16, 24, 32, 48):
        sc = meshgen.stretch_box(side, side, side, E=1e5, nu=0.3, factor=1.5, jitter_amount=0.05, seed=0,
                                 name=f"cube{side}")
        n_free = int((sc.pinned == 0).sum())
        x0 = cc.to_soa(sc.x0, device=dev)
        for model, corot in (("snh", False), ("fcr", False), ("fcr", True)):
            m = cc.Mesh.from_scene(sc, stream=stream, model=model)
            colorize(m, sc)
            m.build_subspace(K_RING)
            x = x0.clone()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            rec = {"side": side, "n_free": n_free, "material": model, "corotated": corot}
            try:
                r = m.solve_step(x, precision="mixed", tol=1e-6, max_iters=args.resolution_max_iters,
                                 check_every=args.check_every, use_graph=not args.no_graph, corotated=corot)
                ev1.record(stream)
                ev1.synchronize()
                rec.update(sweeps=r.iterations, converged=r.converged, ms=ev0.elapsed_time(ev1),
                           rel_residual=r.g_final / r.g0)
            except cc.CCError as e:   # a diverging solve is reported, not fatal
                torch.cuda.synchronize()
                rec.update(sweeps=None, converged=False, error=str(e))
            m.close()
            out.append(rec)
    return out


def run_large(args, stream, dev):
    """Throughput on a mesh far larger than L2: the 64 x 64 x 256-cell beam
    (1 085 825 vertices, 6 291 456 tets) as a quasistatic 1.2x stretch along
    its long axis (SNH, E = 1e5, nu = 0.3, jitter 5%, seed 0), 2-ring bases,
    mixed-precision coloured CC for a fixed number of sweeps (the run measures
    rates, not convergence).  Per-class kernel time from CUDA events and the
    HBM rate of the gather and per-tet kernels on their algorithmic bytes."""
    import torch
    import meshgen
    import paper_2510_12053_gb300 as cc
    sc = meshgen.stretch_box(64, 64, 256, E=1e5, nu=0.3, factor=1.2, jitter_amount=0.05, seed=0, axis=2,
                             size=4.0, name="beam64x64x256")
    n_free = int((sc.pinned == 0).sum())
    t0 = time.perf_counter()
    m = cc.Mesh.from_scene(sc, stream=stream)
    colorize(m, sc)
    m.build_subspace(K_RING)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    x0 = cc.to_soa(sc.x0, device=dev)
    sweeps = args.large_sweeps
    m.solve_step(x0.clone(), precision="mixed", tol=1e-30, max_iters=4, check_every=4,
                 use_graph=not args.no_graph)   # warm-up (graph capture)
    m.profile_enable(True)
    x = x0.clone()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    r = m.solve_step(x, precision="mixed", tol=1e-30, max_iters=sweeps, check_every=sweeps,
                     use_graph=not args.no_graph)
    ev1.record(stream)
    ev1.synchronize()
    prof = m.profile_read()
    m.profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    ncol = int(m.info().num_colors)
    # algorithmic bytes (vectorised forms of the per-unit figures used for the cube)
    tets = np.asarray(sc.tets, dtype=np.int64)
    ge = tets[:, None, :] >= tets[:, :, None]
    src = np.zeros(sc.n)
    np.add.at(src, tets.ravel(), ge.sum(axis=2).ravel())
    val = np.bincount(tets.ravel(), minlength=sc.n)
    nbp, nbi = m.export("nbr_ptr"), m.export("nbr_idx")
    owner = np.repeat(np.arange(sc.n), np.diff(nbp))
    nup = np.bincount(owner[nbi > owner], minlength=sc.n) + 1
    free = sc.pinned == 0
    gather_bytes = float(((src - val) * 36 + val * 24 + val * 24 + nup * 36 + 24)[free].sum())
    free_corners = int((sc.pinned[sc.tets] == 0).sum())
    active_tets = int((sc.pinned[sc.tets] == 0).any(axis=1).sum())
    tet_refreshes = r.iterations * free_corners + active_tets
    gathers = r.iterations * ncol + 1
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    ga, te = prof["gather"], prof["tet_eval"]
    out = {"workload": f"beam 64x64x256 cells ({sc.n} vertices, {sc.T} tets), 1.2x stretch along z, SNH E=1e5 "
                       f"nu=0.3, jitter 5%, 2-ring bases, mixed coloured CC, {sweeps} sweeps",
           "n_free": n_free, "colors": ncol, "setup_s": setup_s, "sweeps": r.iterations, "ms": ms,
           "ms_per_sweep": ms / max(r.iterations, 1),
           "vertex_updates_per_s": n_free * r.iterations / (ms / 1e3),
           "kernel_ms": {k: round(prof[k]["ms"], 3) for k in cc.PROFILE_CLASSES},
           "peak_hbm_gbs": hbm, "peak_source": peak_src}
    if ga["ms"] > 0:
        a = gather_bytes * gathers / (ga["ms"] / 1e3) / 1e9
        out["gather_hbm"] = {"achieved_gbs": a, "frac": a / hbm, "bytes_per_launch": gather_bytes}
    if te["ms"] > 0:
        a = TET_BYTES * tet_refreshes / (te["ms"] / 1e3) / 1e9
        out["tet_eval_hbm"] = {"achieved_gbs": a, "frac": a / hbm, "bytes_per_tet": TET_BYTES}
    m.close()
    return out


def run_cfg3(args, stream, dev):
    """The dynamic cantilever as specified: 64 x 64 x 256 cells of 1/64 m
    (1 085 825 vertices, 6 291 456 tets), z = 0 face clamped, gravity -y 9.8,
    backward Euler dt = 1/60, SNH E = 1e7, nu = 0.45, rho = 1000, 3-ring rest
    bases, mixed-precision coloured CC, 20 steps with a fixed sweep cap per
    step (tolerance 1e-6 of each step's first residual).  Reports per step the
    sweeps, the residual reduction and the time; the sweep rate; and the sweep
    against the HBM roofline on its algorithmic bytes."""
    import torch
    import meshgen
    import paper_2510_12053_gb300 as cc
    nx, ny, nz = (int(v) for v in args.cfg3_cells.split(","))
    sc = meshgen.beam_dynamic(nx, ny, nz)
    n_free = int((sc.pinned == 0).sum())
    t0 = time.perf_counter()
    m = cc.Mesh.from_scene(sc, stream=stream)
    t_mesh = time.perf_counter() - t0
    colorize(m, sc)
    t_col = time.perf_counter() - t0 - t_mesh
    m.build_subspace(3)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = m.info()
    ncol = int(info.num_colors)
    t_sub = setup_s - t_mesh - t_col

    def run_steps(corotated, line_search=False):
        x = cc.to_soa(sc.X, device=dev)
        v = torch.zeros_like(x)
        steps = []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total_ms, total_sweeps = 0.0, 0
        for k in range(args.cfg3_steps):
            ev0.record(stream)
            try:
                r = m.solve_step(x, v, precision="mixed", tol=1e-6, max_iters=args.cfg3_sweeps,
                                 check_every=args.cfg3_sweeps, use_graph=not args.no_graph, corotated=corotated,
                                 line_search=line_search)
            except cc.CCError as e:
                torch.cuda.synchronize()
                steps.append({"step": k, "error": str(e)})
                break
            ev1.record(stream)
            ev1.synchronize()
            ms = ev0.elapsed_time(ev1)
            total_ms += ms
            total_sweeps += r.iterations
            steps.append({"step": k, "sweeps": r.iterations, "rel_residual": r.g_final / r.g0, "ms": ms,
                          "converged": r.converged})
        return steps, total_ms, total_sweeps

    plain_steps, total_ms, total_sweeps = run_steps(False)
    corot_steps, corot_ms, corot_sweeps = run_steps(True)
    ls_steps, ls_ms, ls_sweeps = run_steps(False, line_search=True)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    sweep_bytes = int(info.support_total) * 40 + 4 * sc.T * 56 + (ncol + 1) * sc.n * 24
    ms_sweep = total_ms / max(total_sweeps, 1)
    ach = sweep_bytes / (ms_sweep / 1e3) / 1e9 if total_sweeps else None
    m.close()
    return {"workload": f"cantilever {nx}x{ny}x{nz} cells of 1/64 m ({sc.n} vertices, {sc.T} tets), z=0 clamped, "
                        f"gravity -y, backward Euler dt=1/60, SNH E=1e7 nu=0.45 rho=1000, 3-ring rest bases, "
                        f"mixed coloured CC, {args.cfg3_steps} steps, at most {args.cfg3_sweeps} sweeps per step",
            "n_free": n_free, "colors": ncol, "support_mean": info.support_total / max(n_free, 1),
            "support_max": int(info.support_max), "setup_s": setup_s, "mesh_s": t_mesh, "color_s": t_col,
            "subspace_s": t_sub, "patches_solved": int(info.patch_solved), "patches_shared": int(info.patch_shared),
            "steps": plain_steps, "sweeps": total_sweeps, "ms": total_ms, "ms_per_sweep": ms_sweep,
            "corotated": {"steps": corot_steps, "sweeps": corot_sweeps, "ms": corot_ms,
                          "ms_per_sweep": corot_ms / max(corot_sweeps, 1)},
            "line_search": {"steps": ls_steps, "sweeps": ls_sweeps, "ms": ls_ms,
                            "note": "fixed bases with the global backtracking line search of Sec. 4.4 "
                                    "(energy evaluations included in ms)"},
            "vertex_updates_per_s": n_free * total_sweeps / (total_ms / 1e3) if total_ms else None,
            "sweep_roofline": {"bound": "hbm", "algorithmic_bytes_per_sweep": sweep_bytes, "achieved_gbs": ach,
                               "peak": hbm, "frac": ach / hbm if ach else None, "peak_source": peak_src}}


def run_learned(args, stream, dev):
    """Learned bases: train the network on computed 2-ring
    bases of jittered random boxes (sides U{4..12}, batch-family materials and
    boundary conditions, seed 0; the last 10% held out), then solve the
    48x48x48-cell stretch cube (E = 1e6, jitter 5%) with learned bases (with
    the per-vertex fallback), with computed bases, in plain float64 with
    computed bases, and with coordinate descent.  Wall time = basis
    acquisition + solve."""
    import torch
    import meshgen
    import paper_2510_12053_gb300 as cc
    from paper_2510_12053_gb300 import learned as cl
    peaks, peak_src = measured_peaks()
    dims = meshgen.mlp_dims()
    out = {"network": {"dims": dims, "params": meshgen.mlp_param_count(dims), "activation": "GELU (erf)",
                       "storage": "BF16 weights/activations, float32 accumulation and master weights"}}
    boxes = meshgen.training_boxes(args.train_meshes, seed=0, side_lo=4, side_hi=12)
    n_hold = max(1, len(boxes) // 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, T, counts = cl.training_set(boxes, stream=stream)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n_train = int(counts[:-n_hold].sum())
    Xtr, Ttr, Xho, Tho = X[:n_train], T[:n_train], X[n_train:], T[n_train:]
    net = cc.MLP(max_batch=args.train_batch, stream=stream)
    net.set_params(meshgen.mlp_init(dims, 1))
    ho0 = cl.evaluate(net, Xho, Tho)
    losses, train_s = cl.train(net, Xtr, Ttr, lambda s0, c, b, n: meshgen.batch_indices(17, s0, c, b, n),
                               steps=args.train_steps, batch=args.train_batch, lr=2e-3, lr_final=2e-5)
    ho1 = cl.evaluate(net, Xho, Tho)
    tr_flops = mlp_flops(dims, args.train_batch, backward=True) * args.train_steps
    out["training"] = {"meshes": len(boxes) - n_hold, "held_out_meshes": n_hold, "samples": n_train,
                       "held_out_samples": int(X.shape[0] - n_train), "data_generation_s": gen_s,
                       "steps": args.train_steps, "batch": args.train_batch, "train_s": train_s,
                       "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-50:].mean()),
                       "held_out_mse_before": ho0, "held_out_mse_after": ho1,
                       "target_mean_square": float((Tho ** 2).mean().item()),
                       "tflops": tr_flops / train_s / 1e12}
    del X, T, Xtr, Ttr, Xho, Tho

    sc = meshgen.cube48_stretch(E=1e6, nu=args.nu)
    x0 = cc.to_soa(sc.x0, device=dev)
    n_free = int((sc.pinned == 0).sum())

    def solve(mesh, precision, update="cc"):
        x = x0.clone()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        try:
            r = mesh.solve_step(x, update=update, precision=precision, tol=1e-6, max_iters=args.learned_max_iters,
                                check_every=args.check_every, use_graph=not args.no_graph, history=True)
        except cc.CCError as e:   # a diverging solve (non-finite residual) is reported, not fatal
            torch.cuda.synchronize()
            return {"ms": None, "sweeps": None, "converged": False, "error": str(e)}
        ev1.record(stream)
        ev1.synchronize()
        h = r.residuals[:r.iterations + 1]
        checked = [k for k in range(len(h)) if h[k] >= 0.0]   # residual read every check_every sweeps
        keep = checked[::max(1, len(checked) // 24)] + checked[-1:]
        curve = {int(k): float(h[k] / r.g0) for k in keep}
        return {"ms": ev0.elapsed_time(ev1), "sweeps": r.iterations, "converged": r.converged,
                "vertex_updates_per_s": n_free * r.iterations / (ev0.elapsed_time(ev1) / 1e3),
                "rel_residual_curve": curve}

    def fresh():
        m = cc.Mesh.from_scene(sc, stream=stream)
        colorize(m, sc)
        return m

    free = sc.pinned == 0

    def literal_fallbacks(mesh):
        """The workload text's fallback rule read literally: after one Jacobi
        sweep from x0 with the mesh's bases and one coordinate-descent sweep,
        count the free vertices whose gradient norm after the former exceeds
        the latter (evaluation only)."""
        norms = []
        for upd in ("cc", "cd"):
            xs = x0.clone()
            mesh.sweep(xs, update=upd, schedule="jacobi", precision="mixed")
            _, g, _ = mesh.energy_grad(xs, precision="fp64", want_grad=True)
            norms.append(torch.linalg.vector_norm(g, dim=0).cpu().numpy()[free])
        return int((norms[0] > norms[1]).sum())

    res = {}
    # computed bases (mixed), warm once then timed
    m = fresh()
    m.build_subspace(K_RING)
    solve(m, "mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.build_subspace(K_RING)
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    res["computed_mixed"] = dict(solve(m, "mixed"), acquisition_ms=build_ms,
                                 literal_rule_fallbacks=literal_fallbacks(m))
    res["plain_fp64"] = dict(solve(m, "fp64"), acquisition_ms=build_ms)
    m.close()
    # learned bases (mixed)
    m = fresh()
    m.build_learned_subspace(net)
    solve(m, "mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, rho = m.build_learned_subspace(net, tau=1.0, want_rho=True)
    torch.cuda.synchronize()
    acq_ms = 1e3 * (time.perf_counter() - t0)
    rq = np.quantile(rho.cpu().numpy(), [0.5, 0.9, 0.99, 1.0])
    lit = literal_fallbacks(m)
    res["learned_mixed"] = dict(solve(m, "mixed"), acquisition_ms=acq_ms,
                                literal_rule_fallbacks=lit, literal_rule_fallback_frac=lit / max(n_free, 1),
                                fallback=int(st["n_fallback"]), fallback_frac=st["n_fallback"] / max(st["n_free"], 1),
                                rho_mean=st["rho_mean"], rho_max_kept=st["rho_max"],
                                rho_quantiles={"p50": rq[0], "p90": rq[1], "p99": rq[2], "max": rq[3]},
                                acquisition_split_ms={k[3:]: st[k] for k in st if k.startswith("ms_")})
    # the network's forward pass alone on the cube's inputs (tensor pipe), L2
    # flushed before every timed pass; the one-kernel inference (default), the
    # SM-pair MMA variant and one GEMM launch per layer
    Xc, _ = m.learned_inputs()
    Yc = net.forward(Xc)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def time_forward(kind):
        net.set_fused(kind)
        for _ in range(3):
            net.forward(Xc, out=Yc)
        times = []
        for _ in range(10):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.forward(Xc, out=Yc)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        return statistics.median(times)

    per_layer_ms, pair_ms, inf_ms = time_forward(0), time_forward(2), time_forward(1)
    del flush
    inf_flop = mlp_flops(dims, Xc.shape[0])
    inf_tf = inf_flop / (inf_ms / 1e3) / 1e12
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    out["inference_roofline"] = {"kernel": "k_mlp_fused (every layer in one persistent tcgen05 kernel, activations in "
                                           "shared memory, SM pairs sharing weight tiles by TMA multicast)",
                                 "bound": "tensor", "achieved": inf_tf, "peak": bf16_peak, "unit": "TFLOP/s",
                                 "frac": inf_tf / bf16_peak, "rows": int(Xc.shape[0]), "ms": inf_ms,
                                 "l2": "flushed before every timed pass",
                                 "pair_mma_ms": pair_ms, "pair_mma_tflops": inf_flop / (pair_ms / 1e3) / 1e12,
                                 "per_layer_ms": per_layer_ms,
                                 "per_layer_tflops": inf_flop / (per_layer_ms / 1e3) / 1e12,
                                 "traffic": ncu_traffic("k_mlp_fused",
                                                        os.path.join(ROOT, "profiles", "mlp_gemm_cube48_rows.md")),
                                 "peak_source": peak_src + " (bf16, burst)"}
    m.close()
    # coordinate descent: the method without any subspace
    m = fresh()
    res["cd_mixed"] = dict(solve(m, "mixed", update="cd"), acquisition_ms=0.0)
    m.close()
    for v in res.values():
        v["wall_ms"] = v["acquisition_ms"] + v["ms"] if v.get("ms") is not None else None
    out["cube48"] = {"workload": f"cube48_stretch: 48x48x48 cells ({sc.n} vertices, {sc.T} tets), E=1e6, "
                                 f"nu={args.nu}, jitter 5%, tol 1e-6 rel grad-norm, "
                                 f"at most {args.learned_max_iters} sweeps", "n_free": n_free, **res}

    def ratio(a, b):
        wa, wb = res[a].get("wall_ms"), res[b].get("wall_ms")
        return wa / wb if (wa and wb and res[a]["converged"] and res[b]["converged"]) else None
    out["learned_vs_plain_fp64_wall"] = ratio("plain_fp64", "learned_mixed")
    out["learned_vs_computed_mixed_wall"] = ratio("computed_mixed", "learned_mixed")
    net.close()
    return out


SWEEP_KERNELS = ("k_tet_grad_mixed", "k_row_gather", "k_couple", "k_condense")


def sweep_ncu_traffic(ncol):
    """DRAM bytes of one sweep from the committed ncu summary (one launch of
    each sweep kernel per colour), or None when a kernel changed since."""
    t = [ncu_traffic(k) for k in SWEEP_KERNELS]
    return None if None in t else ncol * float(sum(t))


def per_class_rooflines(cls, meshes, scs, sweeps, tet_refreshes, row_gathers, flops_per_sweep, hbm, peak_src):
    """Every kernel class of the profiled step against its own bound."""
    roof = {}
    ls = cls["local_solve"]
    if ls["ms"] > 0:
        ach = flops_per_sweep * sweeps / (ls["ms"] / 1e3) / 1e12
        tr = [ncu_traffic("k_couple"), ncu_traffic("k_condense")]
        roof["local_solve"] = {"kernel": "k_couple + k_condense (coupling products + batched Schur solve)",
                               "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": ach / FP32_PEAK_TFLOPS,
                               "traffic": (tr[0] + tr[1]) if None not in tr else None,
                               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                               "algorithmic": f"{flops_per_sweep / meshes[0].info().n_free:.0f} FP32 flop per vertex per sweep",
                               "avg_launch_ms": ls["ms"] / max(ls["launches"] // 2, 1)}
    ga = cls["gather"]
    if ga["ms"] > 0:
        gb = gather_bytes_per_refresh(scs[0])
        ach = gb * row_gathers / (ga["ms"] / 1e3) / 1e9
        roof["gather"] = {"kernel": "k_row_gather (gradient + upper block rows of every free vertex)",
                          "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                          "traffic": ncu_traffic("k_row_gather"), "peak_source": peak_src,
                          "algorithmic": f"{gb / 1e6:.1f} MB per launch (counts the per-tet Hessian store, "
                                         f"which the sweep roofline treats as overhead)",
                          "avg_launch_ms": ga["ms"] / max(ga["launches"], 1)}
    te = cls["tet_eval"]
    if te["ms"] > 0:
        ach = TET_BYTES * tet_refreshes / (te["ms"] / 1e3) / 1e9
        roof["tet_eval"] = {"kernel": "k_tet_grad_mixed (float-float gradient + float32 Hessian blocks per tet)",
                            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                            "traffic": ncu_traffic("k_tet_grad_mixed"), "peak_source": peak_src,
                            "algorithmic": f"{TET_BYTES} B per refreshed tet",
                            "avg_launch_ms": te["ms"] / max(te["launches"], 1)}
    return roof


def run_nu045(args, stream, dev):
    """The named configuration as written: the 32^3 cube at nu = 0.45, the
    same four E values, mixed coloured CC to 1e-6 (at most max_iters sweeps).
    Reports each solve's outcome: converged, stopped at the cap (with its
    residual) or ended by a non-finite update (with the sweeps run before)."""
    import torch
    import paper_2510_12053_gb300 as cc
    out = []
    for sc in scenes(0.45):
        m = cc.Mesh.from_scene(sc, stream=stream)
        colorize(m, sc)
        m.build_subspace(K_RING)
        x = cc.to_soa(sc.x0, device=dev)
        rec = {"E": sc.material.E, "nu": 0.45}
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        hist = None
        try:
            r = m.solve_step(x, precision="mixed", tol=1e-6, max_iters=args.max_iters, check_every=args.check_every,
                             use_graph=not args.no_graph, history=True)
            ev1.record(stream)
            ev1.synchronize()
            hist = r.residuals
            rec.update(outcome="converged" if r.converged else "cap", sweeps=r.iterations,
                       rel_residual=r.g_final / r.g0, ms=ev0.elapsed_time(ev1))
        except cc.CCError as e:
            torch.cuda.synchronize()
            hist = getattr(e, "residuals", None)
            done = np.flatnonzero(hist >= 0) if hist is not None else np.zeros(0, int)
            rec.update(outcome="diverged", error=str(e),
                       sweeps_before_failure=int(done.max()) if done.size else None)
        if hist is not None:
            h = hist[np.isfinite(hist) & (hist >= 0)]
            rec["max_rel_residual"] = float(h.max() / h[0]) if h.size else None
        m.close()
        out.append(rec)
    return out


def oracle_full_sweep(nu):
    """One whole coloured CC sweep of the oracle (its own ``solvers.sweep``) on
    the 32^3 cube from x0, single-threaded; the 2-ring bases of every free
    vertex are built by the oracle first (timed separately)."""
    from oracle import fem, solvers, subspace, topology
    sc = _ow_scene(nu)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    t0 = time.perf_counter()
    sup, U = subspace.build_local_bases(pb, topo, K_RING)
    t_b = time.perf_counter() - t0
    st = solvers.Stats()
    t0 = time.perf_counter()
    solvers.sweep(pb, topo, sup, U, sc.x0, None, "cc", "colored", st)
    t_s = time.perf_counter() - t0
    n_free = int(pb.free.sum())
    return {"basis_build_s": t_b, "sweep_s": t_s, "updates": st.updates, "vertex_updates_per_s": st.updates / t_s,
            "cores": 1, "n_free": n_free, "host": host_info()}


def run_headline_batch(args, scs, n, n_free, x0s, flush, stream, dev, world, dist_barrier):
    """The configuration's four E solves as one 4-mesh batch (cc_build_batch /
    cc_solve_batch: one launch per kernel per colour covers all four meshes),
    timed under the same rules as the single-mesh solves: warm-up steps, L2
    flushed before every step, CUDA events on the launching stream, clocks
    sampled during the timed region; then the same through host buffers."""
    import torch
    import paper_2510_12053_gb300 as cc

    b4 = cc.Mesh.from_scenes(scs, stream=stream)
    colorize(b4, scs)
    b4.build_subspace(K_RING)
    nm = len(scs)
    xb0 = cc.to_soa(np.concatenate(x0s), device=dev)
    xb = torch.empty_like(xb0)

    def batch_step(src):
        xb.copy_(src, non_blocking=True)
        rb = b4.solve_batch(xb, precision="mixed", tol=1e-6, max_iters=args.max_iters,
                            check_every=args.check_every, use_graph=not args.no_graph)
        return int(rb["iterations"].sum()), bool((rb["status"] == 1).all()), rb["iterations"].tolist()

    for _ in range(args.warmup):
        batch_step(xb0)
    torch.cuda.synchronize()
    b4.profile_enable(False)   # resets the launch counters; no event timing inside the timed region
    clocks = Clocks(dev.index)
    dist_barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, sweeps, conv, iters = [], 0, True, None
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s_, c_, iters = batch_step(xb0)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        sweeps += s_
        conv &= c_
    torch.cuda.synchronize()
    dist_barrier()
    clk = clocks.stop()
    launches = b4.profile_read()["total_launches"]
    total_ms = sum(times)
    value = whole_job_rate(n_free * sweeps, total_ms, world, dev)
    total_ms = reduce_over_ranks(total_ms, world, dev, "max")

    # end to end: every step copies the four meshes' positions from pinned host
    # memory, solves, and copies the result back
    x_host = torch.empty(tuple(xb0.shape), dtype=torch.float64, pin_memory=True)
    x_host.copy_(xb0.cpu())
    out_host = torch.empty_like(x_host, pin_memory=True)
    e2e_ms, e2e_sweeps = [], 0
    torch.cuda.synchronize()
    dist_barrier()
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s_, _, _ = batch_step(x_host)
        out_host.copy_(xb, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        e2e_ms.append(ev0.elapsed_time(ev1))
        e2e_sweeps += s_
    torch.cuda.synchronize()
    dist_barrier()
    e2e_value = whole_job_rate(n_free * e2e_sweeps, sum(e2e_ms), world, dev)
    b4.close()
    return {"value": value, "total_ms": total_ms, "sweeps": sweeps, "converged": conv, "iterations": iters,
            "clocks": clk, "launches": launches, "meshes": nm,
            "e2e": {"value": e2e_value, "unit": "vertex-updates/s", "h2d_bytes_per_step": 24 * n * nm,
                    "d2h_bytes_per_step": 24 * n * nm}}


def run_headline_concurrent(args, scs, n, n_free, flush, stream, dev, world, dist_barrier):
    """The configuration's four E solves side by side (cc_solve_concurrent):
    each mesh on its own stream and host thread, so that one mesh's short
    colour kernels run while another's wait on their predecessors.  Timed
    under the same rules as the other headlines: warm-up steps, L2 flushed
    before every step, CUDA events recorded on the launching stream, which
    every mesh stream waits on at the start and which waits on every mesh
    stream at the end; clocks sampled during the timed region; then the same
    through host buffers."""
    import torch
    import paper_2510_12053_gb300 as cc

    nm = len(scs)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nm)]
    meshes = []
    for sc, st in zip(scs, streams):
        m = cc.Mesh.from_scene(sc, stream=st)
        colorize(m, sc)
        m.build_subspace(K_RING)
        meshes.append(m)
    x0s = [cc.to_soa(sc.x0, device=dev) for sc in scs]
    xs = [torch.empty_like(x) for x in x0s]
    torch.cuda.synchronize()

    def step(srcs, outs=None):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for st, x, src in zip(streams, xs, srcs):
            st.wait_event(ev0)
            with torch.cuda.stream(st):
                x.copy_(src, non_blocking=True)
        res = cc.solve_concurrent(meshes, xs, precision="mixed", tol=1e-6, max_iters=args.max_iters,
                                  check_every=args.check_every, use_graph=not args.no_graph)
        if outs is not None:
            for st, x, out in zip(streams, xs, outs):
                with torch.cuda.stream(st):
                    out.copy_(x, non_blocking=True)
        for st in streams:
            stream.wait_stream(st)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1), sum(r.iterations for r in res), all(r.converged for r in res), \
            [r.iterations for r in res]

    for _ in range(args.warmup):
        step(x0s)
    torch.cuda.synchronize()
    for m in meshes:
        m.profile_enable(False)   # resets the launch counters; no event timing inside the timed region
    clocks = Clocks(dev.index)
    dist_barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, sweeps, conv, iters = [], 0, True, None
    for _ in range(args.steps):
        flush.zero_()
        ms, s_, c_, iters = step(x0s)
        times.append(ms)
        sweeps += s_
        conv &= c_
    torch.cuda.synchronize()
    dist_barrier()
    clk = clocks.stop()
    launches = sum(m.profile_read()["total_launches"] for m in meshes)
    total_ms = sum(times)
    value = whole_job_rate(n_free * sweeps, total_ms, world, dev)
    total_ms = reduce_over_ranks(total_ms, world, dev, "max")

    # end to end: every step copies each mesh's positions from pinned host
    # memory on its stream, solves, and copies the results back
    x_host = [torch.empty(tuple(x.shape), dtype=torch.float64, pin_memory=True) for x in x0s]
    for h, x in zip(x_host, x0s):
        h.copy_(x.cpu())
    out_host = [torch.empty_like(h, pin_memory=True) for h in x_host]
    e2e_ms, e2e_sweeps = [], 0
    torch.cuda.synchronize()
    dist_barrier()
    for _ in range(args.steps):
        flush.zero_()
        ms, s_, _, _ = step(x_host, out_host)
        e2e_ms.append(ms)
        e2e_sweeps += s_
    torch.cuda.synchronize()
    dist_barrier()
    e2e_value = whole_job_rate(n_free * e2e_sweeps, sum(e2e_ms), world, dev)
    for m in meshes:
        m.close()
    return {"value": value, "total_ms": total_ms, "sweeps": sweeps, "converged": conv, "iterations": iters,
            "clocks": clk, "launches": launches, "meshes": nm,
            "e2e": {"value": e2e_value, "unit": "vertex-updates/s", "h2d_bytes_per_step": 24 * n * nm,
                    "d2h_bytes_per_step": 24 * n * nm}}


def run_ours(args, rank, world):
    import torch
    import paper_2510_12053_gb300 as cc

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    scs = scenes(args.nu)
    t_setup = time.perf_counter()
    meshes = []
    for sc in scs:
        m = cc.Mesh.from_scene(sc, stream=stream)
        colorize(m, sc)
        m.build_subspace(K_RING)
        meshes.append(m)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t_setup) / len(scs)
    n, T = scs[0].n, scs[0].T
    n_free = int((scs[0].pinned == 0).sum())
    x0 = cc.to_soa(scs[0].x0, device=dev)
    x = torch.empty_like(x0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def dist_barrier():
        if world > 1:
            torch.distributed.barrier()

    def one_step(precision):
        sweeps, conv = 0, True
        for m in meshes:
            x.copy_(x0)
            r = m.solve_step(x, precision=precision, tol=1e-6, max_iters=args.max_iters,
                             check_every=args.check_every, use_graph=not args.no_graph)
            sweeps += r.iterations
            conv &= r.converged
        return sweeps, conv

    for _ in range(args.warmup):
        one_step("mixed")
    torch.cuda.synchronize()
    for m in meshes:
        m.profile_enable(False)   # resets the launch counters; no event timing inside the timed region
    clocks = Clocks(dev.index)
    dist_barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, sweeps_total, all_conv = [], 0, True
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s, c = one_step("mixed")
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        sweeps_total += s
        all_conv &= c
    torch.cuda.synchronize()
    dist_barrier()
    wall_ms = 1e3 * (time.perf_counter() - t_wall)
    clk = clocks.stop()
    launches = sum(m.profile_read()["total_launches"] for m in meshes)
    total_ms = sum(times)
    updates = n_free * sweeps_total
    value = whole_job_rate(updates, total_ms, world, dev)
    total_ms = reduce_over_ranks(total_ms, world, dev, "max")
    sweeps_per_solve = sweeps_total / (args.steps * len(meshes))
    ms_per_sweep = total_ms / max(sweeps_total, 1)

    # per-class device time: one more step with event timing on, outside the timed region
    for m in meshes:
        m.profile_enable(True)
    flush.zero_()
    sweeps_prof, _ = one_step("mixed")
    torch.cuda.synchronize()
    prof = [m.profile_read() for m in meshes]
    for m in meshes:
        m.profile_enable(False)
    cls = {k: {"ms": sum(p[k]["ms"] for p in prof), "launches": sum(p[k]["launches"] for p in prof)}
           for k in cc.PROFILE_CLASSES}
    dominant = max(cc.PROFILE_CLASSES, key=lambda k: cls[k]["ms"])
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    ncol = int(meshes[0].info().num_colors)
    # units processed in the profiling step
    free_corners = int((scs[0].pinned[scs[0].tets] == 0).sum())
    active_tets = int((scs[0].pinned[scs[0].tets] == 0).any(axis=1).sum())
    tet_refreshes = sweeps_prof * free_corners + len(meshes) * active_tets
    row_gathers = sweeps_prof * ncol + len(meshes)
    fl = local_solve_flops(meshes[0])
    flops_per_sweep = float(fl.sum())

    # the sweep against the HBM roofline on its algorithmic bytes: bases and
    # support ids read once, tet ids / D_m^-1 / V_t for the four refreshes of
    # every tet, positions read once per colour and written once
    sup_total = int(meshes[0].info().support_total)
    b_u, b_d = 4, 4   # float32 bases and D_m^-1 on the mixed path
    sweep_bytes = sup_total * (9 * b_u + 4) + 4 * T * (16 + 9 * b_d + 4) + (ncol + 1) * n * 24
    sweep_ach = sweep_bytes / (ms_per_sweep / 1e3) / 1e9
    sweep_traffic = sweep_ncu_traffic(ncol)
    sweep_flops_rate = flops_per_sweep / (ms_per_sweep / 1e3) / 1e12
    roofline = {"kernel": "sweep", "bound": "hbm", "achieved": sweep_ach, "peak": hbm, "unit": "GB/s",
                "frac": sweep_ach / hbm, "traffic": sweep_traffic, "peak_source": peak_src + " (HBM copy)",
                "algorithmic": f"{sweep_bytes / 1e6:.1f} MB per {ncol}-colour sweep (bases {sup_total} blocks x 40 B, "
                               f"{T} tets x 4 refreshes x 56 B, positions {ncol + 1} x {n} x 24 B)",
                "ms_per_sweep": ms_per_sweep, "units": "one coloured sweep (every free vertex updated once)",
                "fp32_alu": {"achieved_tflops": sweep_flops_rate, "peak": FP32_PEAK_TFLOPS,
                             "frac": sweep_flops_rate / FP32_PEAK_TFLOPS,
                             "note": "coupling products only; peak derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}}
    roof = per_class_rooflines(cls, meshes, scs, sweeps_prof, tet_refreshes, row_gathers, flops_per_sweep,
                               hbm, peak_src)

    # plain float64 CC on the same solves
    fp64 = None
    if not args.no_fp64:
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s64, c64 = one_step("fp64")
        ev1.record(stream)
        ev1.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        fp64 = {"ms_to_tol_per_solve": ms64 / len(meshes), "sweeps_per_solve": s64 / len(meshes),
                "vertex_updates_per_s": n_free * s64 / (ms64 / 1e3), "converged": bool(c64)}

    # end to end through the public API with host buffers
    x_host = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
    x_host.copy_(torch.as_tensor(np.ascontiguousarray(scs[0].x0.T)))
    out_host = torch.empty_like(x_host, pin_memory=True)
    e2e_ms, e2e_sweeps = [], 0
    torch.cuda.synchronize()
    dist_barrier()
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for m in meshes:
            x.copy_(x_host, non_blocking=True)
            r = m.solve_step(x, precision="mixed", tol=1e-6, max_iters=args.max_iters,
                             check_every=args.check_every, use_graph=not args.no_graph)
            e2e_sweeps += r.iterations
            out_host.copy_(x, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        e2e_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    dist_barrier()
    e2e_value = whole_job_rate(n_free * e2e_sweeps, sum(e2e_ms), world, dev)
    for m in meshes:
        m.close()

    # the headline: the same four solves side by side on four streams, or as
    # one 4-mesh batch, timed like the above
    head = None
    if args.headline == "concurrent":
        head = run_headline_concurrent(args, scs, n, n_free, flush, stream, dev, world, dist_barrier)
    elif args.headline == "batch":
        head = run_headline_batch(args, scs, n, n_free, [sc.x0 for sc in scs], flush, stream, dev, world,
                                  dist_barrier)

    # the same four solves as one batch (cc_build_batch: one launch per kernel
    # per colour covers all four meshes), graph-replayed, after one warm-up solve
    batched4 = None
    if not args.no_batch and args.headline != "batch":
        b4 = cc.Mesh.from_scenes(scs, stream=stream)
        colorize(b4, scs)
        b4.build_subspace(K_RING)
        xb0 = cc.to_soa(np.concatenate([sc.x0 for sc in scs]), device=dev)
        xb = xb0.clone()
        b4.solve_batch(xb, precision="mixed", tol=1e-6, max_iters=args.max_iters, check_every=args.check_every,
                       use_graph=not args.no_graph)
        xb.copy_(xb0)
        flush.zero_()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        rb = b4.solve_batch(xb, precision="mixed", tol=1e-6, max_iters=args.max_iters, check_every=args.check_every,
                            use_graph=not args.no_graph)
        ev1.record(stream)
        ev1.synchronize()
        msb = ev0.elapsed_time(ev1)
        batched4 = {"ms_all_four": msb, "iterations": rb["iterations"].tolist(),
                    "converged": bool((rb["status"] == 1).all()),
                    "vertex_updates_per_s": n_free * float(rb["iterations"].sum()) / (msb / 1e3),
                    "ms_per_mesh_sweep": msb / float(rb["iterations"].sum()),
                    "note": "the headline's four E values solved together as one 4-mesh batch"}
        b4.close()

    # the same four solves with the greedy colouring (8 colours), for comparison
    greedy_cmp = None
    if COLORING["mode"] == "lattice" and not args.no_fp64:
        gms, gsw = 0.0, []
        for sc in scs:
            mg = cc.Mesh.from_scene(sc, stream=stream)
            mg.color()
            mg.build_subspace(K_RING)
            xg = x0.clone()
            mg.solve_step(xg, precision="mixed", tol=1e-6, max_iters=args.max_iters, check_every=args.check_every,
                          use_graph=not args.no_graph)   # warm-up (graph capture)
            xg.copy_(x0)
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            rg = mg.solve_step(xg, precision="mixed", tol=1e-6, max_iters=args.max_iters,
                               check_every=args.check_every, use_graph=not args.no_graph)
            ev1.record(stream)
            ev1.synchronize()
            gms += ev0.elapsed_time(ev1)
            gsw.append(rg.iterations)
            mg.close()
        greedy_cmp = {"colors": 8, "ms_to_tol_per_solve": gms / len(scs), "sweeps_per_solve": float(np.mean(gsw)),
                      "ms_per_sweep": gms / sum(gsw), "vertex_updates_per_s": n_free * sum(gsw) / (gms / 1e3)}

    nu045 = None if args.no_nu045 else run_nu045(args, stream, dev)
    batch_res = None
    if not args.no_batch:
        batch_res = run_batch(args, stream, dev)
    learned_res = None
    if not args.no_learned:
        learned_res = run_learned(args, stream, dev)
    resolution_res = run_resolution(args, stream, dev) if args.resolution_sweep else None
    large_res = run_large(args, stream, dev) if args.large_beam else None
    cfg3_res = None if args.no_cfg3 else run_cfg3(args, stream, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ob = oracle_baseline(args.nu)
        cpu = {"value": ob["value"], "unit": "vertex-updates/s", "cores": ob["cores"], "kind": "oracle",
               "sample": f"colour 0 of one coloured CC sweep of the full 32^3 cube ({ob['updates']} of {n_free} free "
                         f"vertices, E=1e5): float64 gradient + Hessian assembly at x0 (serial) and every local CC "
                         f"update of the colour over {ob['cores']} processes, {ob['s']:.1f} s; 2-ring oracle bases "
                         f"built beforehand (untimed)",
               "single_thread": ob.get("single_thread"), "host": host_info()}
    cfg1 = cfg1_oracle_timings() if (rank == 0 and args.cfg1_oracle) else None
    full_cpu = oracle_full_sweep(args.nu) if (rank == 0 and args.cpu_full_sweep) else None

    if rank == 0 and head is not None:
        # the single-mesh solves become a sub-object; the headline fields are the batch's
        single = {"value": value, "ms_per_step": total_ms / args.steps,
                  "ms_to_tol_per_solve": total_ms / (args.steps * len(meshes)), "ms_per_sweep": ms_per_sweep,
                  "sweep_hbm_frac": roofline["frac"], "e2e": e2e_value, "gpu_launches": launches, "clocks": clk,
                  "note": "the four E solves one mesh after another (cc_solve_step each)"}
        nm = head["meshes"]
        ms_sweep_b = head["total_ms"] / max(head["sweeps"], 1)
        ach_b = sweep_bytes / (ms_sweep_b / 1e3) / 1e9
        fl_b = flops_per_sweep / (ms_sweep_b / 1e3) / 1e12
        if args.headline == "batch":
            t_note = ("ncu DRAM bytes of the single-mesh launches per sweep; a batch launch processes the four "
                      "meshes' units, so per mesh-sweep the same bytes")
            u_note = (f"one coloured sweep of one mesh (every free vertex updated once); the batch's {nm} meshes "
                      "sweep together, one launch per kernel per colour")
            batched4 = {"note": "the headline (the four E values as one 4-mesh batch)",
                        "iterations": head["iterations"]}
        else:
            t_note = ("ncu DRAM bytes of the single-mesh launches per sweep; the concurrent solves launch the same "
                      "kernels with the same units, on four streams")
            u_note = (f"one coloured sweep of one mesh (every free vertex updated once); the {nm} meshes sweep "
                      "side by side, each on its own stream, so the time per mesh-sweep is the wall time over "
                      "all meshes' sweeps")
        roofline = dict(roofline, achieved=ach_b, frac=ach_b / hbm, ms_per_sweep=ms_sweep_b, traffic_note=t_note,
                        units=u_note,
                        fp32_alu=dict(roofline["fp32_alu"], achieved_tflops=fl_b, frac=fl_b / FP32_PEAK_TFLOPS))
        value, total_ms, launches, clk = head["value"], head["total_ms"], head["launches"], head["clocks"]
        sweeps_per_solve = head["sweeps"] / (args.steps * nm)
        all_conv = head["converged"]
        e2e_value = head["e2e"]["value"]
    if rank == 0:
        cfg = dict(workload_config(args.nu, n, T, n_free), parallelism=f"replicas x{world}")
        cfg["execution"] = {
            "concurrent": "the four E solves side by side (cc_solve_concurrent: each mesh on its own stream and "
                          "host thread; iterates and sweep counts bit for bit as solved alone)",
            "batch": "the four E solves as one 4-mesh batch (cc_solve_batch: one launch per kernel per colour for "
                     "all four; per-mesh iterates and sweep counts as solved alone)",
            "single": "the four E solves one mesh after another (cc_solve_step)"}[args.headline]
        line = {
            "metric": METRIC, "value": value, "unit": "vertex-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed (f32 + f32x2 + f64)",
            "data": "synthetic",
            "config": cfg,
            "ms_to_tol_per_solve": total_ms / (args.steps * len(meshes)),
            "sweeps_per_solve": sweeps_per_solve, "converged": bool(all_conv), "setup_ms_per_mesh": setup_ms,
            "plain_fp64": fp64,
            "speedup_vs_fp64": (fp64["ms_to_tol_per_solve"] / (total_ms / (args.steps * len(meshes))))
            if fp64 else None,
            "wall_ms_timed": wall_ms,
            "roofline": roofline,
            "roofline_all": roof,
            "kernel_ms_profiled_step": {k: round(v["ms"], 3) for k, v in cls.items()},
            "kernel_launches_profiled_step": {k: v["launches"] for k, v in cls.items()},
            "dominant_kernel_class": dominant,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "vertex-updates/s", "h2d_bytes_per_step": 24 * n * len(meshes),
                    "d2h_bytes_per_step": 24 * n * len(meshes)},
            "cpu_baseline": cpu,
            "cfg_nu045": nu045,
            "batched_four_solves": batched4,
            "greedy_coloring_solves": greedy_cmp,
            "batch": batch_res,
            "learned": learned_res,
        }
        if head is not None:
            line["single_mesh_solves"] = single
            line["profile_note"] = ("kernel_ms_profiled_step and roofline_all come from one more profiled "
                                    "single-mesh step (per-launch figures)")
        if resolution_res is not None:
            line["resolution"] = resolution_res
        if large_res is not None:
            line["large_beam"] = large_res
        if cfg3_res is not None:
            line["large_beam_k3_dynamic"] = cfg3_res
        if cfg1 is not None:
            line["cfg1_oracle"] = cfg1
        if full_cpu is not None:
            line["cpu_full_sweep"] = full_cpu
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    COLORING["mode"] = args.colors
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
