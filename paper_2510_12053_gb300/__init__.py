"""GB300-native Coordinate Condensation (arxiv 2510.12053): Python binding.

A thin ``ctypes`` layer over the C ABI in ``include/cc.h``.  It only
marshals arguments: every step of the sweep runs in the CUDA kernels of
``_lib/libcc_gb300.so``.  If that library is missing, importing works but
every call raises :class:`CCError` (there is no CPU fallback).

Device arrays are ``torch`` float64 CUDA tensors in SoA layout ``[3, n]``;
PyTorch supplies memory and streams only.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcc_gb300.so")

# cc_status
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_NOT_CONVERGED, ERR_STATE = range(8)
STATUS_NAMES = ["CC_OK", "CC_ERR_INVALID_ARG", "CC_ERR_CUDA", "CC_ERR_OOM", "CC_ERR_NUMERIC",
                "CC_ERR_TIMEOUT", "CC_ERR_NOT_CONVERGED", "CC_ERR_STATE"]
PREC = {"fp64": 0, "mixed": 1}
SCHED = {"colored": 0, "jacobi": 1}
UPDATE = {"cc": 0, "cd": 1, "jgs2": 2}
ARRAYS = {"vt_ptr": (0, np.int64), "vt_tet": (1, np.int32), "vt_corner": (2, np.int32),
          "nbr_ptr": (3, np.int64), "nbr_idx": (4, np.int32), "color": (5, np.int32),
          "sup_ptr": (6, np.int64), "sup_idx": (7, np.int32), "U": (8, np.float64),
          "mass": (9, np.float64)}


class CCError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class Material(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("rho", ctypes.c_double), ("model", ctypes.c_int32)]


MODEL = {"snh": 0, "fcr": 1}


class SweepOpts(ctypes.Structure):
    _fields_ = [("update", ctypes.c_int), ("schedule", ctypes.c_int), ("precision", ctypes.c_int),
                ("color_begin", ctypes.c_int32), ("color_end", ctypes.c_int32), ("corotated", ctypes.c_int32)]


class SweepStats(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int64), ("fallback_empty", ctypes.c_int64),
                ("fallback_reduced", ctypes.c_int64), ("fallback_schur", ctypes.c_int64)]


class StepOpts(ctypes.Structure):
    _fields_ = [("update", ctypes.c_int), ("schedule", ctypes.c_int), ("precision", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("min_iters", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("residual_history", ctypes.POINTER(ctypes.c_double)), ("corotated", ctypes.c_int32),
                ("restart_every", ctypes.c_int32), ("line_search", ctypes.c_int32)]


class StepStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("g0", ctypes.c_double),
                ("g_final", ctypes.c_double), ("energy_final", ctypes.c_double), ("sweeps", SweepStats)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("T", ctypes.c_int64), ("n_free", ctypes.c_int64),
                ("nnz_blocks", ctypes.c_int64), ("num_colors", ctypes.c_int32), ("k_ring", ctypes.c_int32),
                ("support_total", ctypes.c_int64), ("support_max", ctypes.c_int32),
                ("max_valence", ctypes.c_int32), ("patch_float64", ctypes.c_int64),
                ("patch_solved", ctypes.c_int64), ("patch_shared", ctypes.c_int64)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("tets", ctypes.c_void_p), ("T", ctypes.c_int64),
                ("pinned", ctypes.c_void_p), ("mat", Material)]


class BatchStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.POINTER(ctypes.c_int32)), ("status", ctypes.POINTER(ctypes.c_int32)),
                ("g0", ctypes.POINTER(ctypes.c_double)), ("g_final", ctypes.POINTER(ctypes.c_double)),
                ("sweeps", ctypes.c_int32), ("totals", SweepStats)]


class TuneResult(ctypes.Structure):
    _fields_ = [("couple_threads", ctypes.c_int32), ("couple_row_lanes", ctypes.c_int32),
                ("gather_warps", ctypes.c_int32), ("couple_ms", ctypes.c_double * 4),
                ("row_lanes_ms", ctypes.c_double * 4), ("gather_ms", ctypes.c_double * 3),
                ("rows_from_positions", ctypes.c_int32), ("fused_condense", ctypes.c_int32),
                ("variant_ms", ctypes.c_double * 4)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 5), ("launches", ctypes.c_int64 * 5), ("total_launches", ctypes.c_int64)]


class MlpConfig(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_int32), ("hidden", ctypes.c_int32), ("layers", ctypes.c_int32),
                ("d_out", ctypes.c_int32), ("max_batch", ctypes.c_int32)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


class LearnedStats(ctypes.Structure):
    _fields_ = [("n_free", ctypes.c_int64), ("n_fallback", ctypes.c_int64), ("rho_max", ctypes.c_double),
                ("rho_mean", ctypes.c_double), ("ms_supports", ctypes.c_double), ("ms_inputs", ctypes.c_double),
                ("ms_infer", ctypes.c_double), ("ms_assemble", ctypes.c_double), ("ms_residual", ctypes.c_double),
                ("ms_fallback", ctypes.c_double), ("ms_total", ctypes.c_double)]


PROFILE_CLASSES = ["tet_eval", "gather", "local_solve", "reduce", "other"]
LEARNED_D_IN, LEARNED_D_OUT, LEARNED_LDX = 258, 576, 264

_lib_handle = None

_P = ctypes.c_void_p
_SIGS = {
    "cc_build_mesh": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.POINTER(Material),
                                     ctypes.c_double, _P, _P, ctypes.POINTER(_P)]),
    "cc_destroy_mesh": (None, [_P]),
    "cc_color": (ctypes.c_int, [_P, _P, _P]),
    "cc_set_colors": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "cc_build_subspace": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cc_set_subspace": (ctypes.c_int, [_P, _P, _P, _P]),
    "cc_build_subspace_at": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "cc_energy_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "cc_sweep": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepStats)]),
    "cc_solve_step": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(StepOpts), ctypes.POINTER(StepStats)]),
    "cc_get_info": (ctypes.c_int, [_P, ctypes.POINTER(MeshInfo)]),
    "cc_export": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "cc_build_batch": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.c_int32, ctypes.c_double, _P, _P,
                                      ctypes.POINTER(_P)]),
    "cc_batch_offsets": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "cc_solve_batch": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(StepOpts), ctypes.POINTER(BatchStats)]),
    "cc_solve_concurrent": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, ctypes.POINTER(StepOpts),
                                           ctypes.POINTER(StepStats), _P]),
    "cc_autotune": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(TuneResult)]),
    "cc_gemm_bf16_tn": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _P]),
    "cc_mlp_activation": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "cc_mlp_create": (ctypes.c_int, [ctypes.POINTER(MlpConfig), _P, ctypes.POINTER(_P)]),
    "cc_mlp_destroy": (None, [_P]),
    "cc_mlp_param_count": (ctypes.c_int64, [_P]),
    "cc_mlp_set_params": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "cc_mlp_get_params": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "cc_mlp_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "cc_mlp_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "cc_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_int64]),
    "cc_mlp_set_fused": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cc_mlp_loss_grad": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_double), _P]),
    "cc_mlp_adam_step": (ctypes.c_int, [_P, _P, ctypes.POINTER(Adam)]),
    "cc_mlp_train": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int64, _P,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Adam), _P]),
    "cc_learned_inputs": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64)]),
    "cc_build_learned_subspace": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, ctypes.POINTER(LearnedStats)]),
    "cc_set_launch_shape": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "cc_set_sweep_variant": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "cc_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cc_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "cc_build_bases_noalloc": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P, _P, ctypes.c_int32, _P, _P]),
    "cc_last_error": (ctypes.c_char_p, []),
    "cc_version": (ctypes.c_char_p, []),
}


def lib():
    """The loaded C library (raises CCError if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise CCError(ERR_STATE, f"CUDA library not built ({LIB_PATH}); run "
                                     "`python -m paper_2510_12053_gb300.build`")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib_handle = h
    return _lib_handle


def _check(status: int):
    if status != OK:
        raise CCError(status, lib().cc_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev3n(t, n, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and tuple(t.shape) == (3, n)):
        raise CCError(ERR_INVALID_ARG, f"{name} must be a contiguous float64 CUDA tensor of shape (3, {n})")
    return t.data_ptr()


@dataclasses.dataclass
class SolveResult:
    iterations: int
    converged: bool
    g0: float
    g_final: float
    energy: float
    updates: int
    fallback_empty: int
    fallback_reduced: int
    fallback_schur: int
    residuals: Optional[np.ndarray] = None


class Mesh:
    """A tet mesh on the GPU (owns the library's ``cc_mesh``)."""

    def __init__(self, X, tets, pinned=None, *, E: float, nu: float, rho: float = 1000.0, h: float = 0.0,
                 gravity=None, stream=None, model: str = "snh"):
        X = np.ascontiguousarray(X, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.n, self.T = int(X.shape[0]), int(tets.shape[0])
        pin = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
        grav = None if gravity is None else np.ascontiguousarray(gravity, dtype=np.float64)
        mat = Material(E, nu, rho, MODEL[model])
        out = _P()
        self._h = None
        _check(lib().cc_build_mesh(X.ctypes.data, self.n, tets.ctypes.data, self.T,
                                   None if pin is None else pin.ctypes.data, ctypes.byref(mat), float(h),
                                   None if grav is None else grav.ctypes.data, _stream_ptr(stream),
                                   ctypes.byref(out)))
        self._h = out
        self.dynamic = h > 0.0

    @classmethod
    def from_scenes(cls, scenes, stream=None, model: str = "snh") -> "Mesh":
        """A batch: the disjoint union of several meshes, solved together
        (materials per mesh; time step and gravity of the first scene)."""
        keep = []
        descs = (MeshDesc * len(scenes))()
        for k, sc in enumerate(scenes):
            X = np.ascontiguousarray(sc.X, dtype=np.float64)
            T = np.ascontiguousarray(sc.tets, dtype=np.int32)
            P = np.ascontiguousarray(sc.pinned, dtype=np.uint8)
            keep += [X, T, P]
            m = sc.material
            descs[k] = MeshDesc(X.ctypes.data, X.shape[0], T.ctypes.data, T.shape[0], P.ctypes.data,
                                Material(m.E, m.nu, m.rho, MODEL[model]))
        grav = np.ascontiguousarray(scenes[0].gravity, dtype=np.float64)
        obj = cls.__new__(cls)
        obj._h = None
        out = _P()
        _check(lib().cc_build_batch(descs, len(scenes), float(scenes[0].h), grav.ctypes.data, _stream_ptr(stream),
                                    ctypes.byref(out)))
        obj._h = out
        obj.n = int(sum(sc.n for sc in scenes))
        obj.T = int(sum(sc.T for sc in scenes))
        obj.dynamic = scenes[0].h > 0.0
        return obj

    def batch_offsets(self) -> np.ndarray:
        cnt = ctypes.c_int32()
        _check(lib().cc_batch_offsets(self._h, None, ctypes.byref(cnt)))
        off = np.zeros(cnt.value + 1, dtype=np.int64)
        _check(lib().cc_batch_offsets(self._h, off.ctypes.data, ctypes.byref(cnt)))
        return off

    def solve_batch(self, x, v=None, *, update: str = "cc", schedule: str = "colored", precision: str = "mixed",
                    tol: float = 1e-6, max_iters: int = 200, min_iters: int = 0, check_every: int = 1,
                    use_graph: bool = False, corotated: bool = False, line_search: bool = False,
                    restart_every: int = 0) -> dict:
        B = len(self.batch_offsets()) - 1
        it = np.zeros(B, dtype=np.int32)
        status = np.zeros(B, dtype=np.int32)
        g0 = np.zeros(B)
        gf = np.zeros(B)
        st = BatchStats(it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        g0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        gf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, SweepStats())
        o = StepOpts(UPDATE[update], SCHED[schedule], PREC[precision], tol, max_iters, min_iters, check_every,
                     int(use_graph), None, int(corotated), int(restart_every), int(line_search))
        rc = lib().cc_solve_batch(self._h, _dev3n(x, self.n, "x"), _dev3n(v, self.n, "v"), ctypes.byref(o),
                                  ctypes.byref(st))
        if rc not in (OK, ERR_NOT_CONVERGED):
            _check(rc)
        return {"iterations": it, "status": status, "g0": g0, "g_final": gf, "sweeps": st.sweeps,
                "updates": st.totals.updates}

    @classmethod
    def from_scene(cls, scene, stream=None, model: str = "snh") -> "Mesh":
        m = scene.material
        return cls(scene.X, scene.tets, scene.pinned, E=m.E, nu=m.nu, rho=m.rho, h=scene.h,
                   gravity=scene.gravity, stream=stream, model=model)

    def close(self):
        if self._h is not None and self._h.value:
            lib().cc_destroy_mesh(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def color(self) -> np.ndarray:
        cols = np.empty(self.n, dtype=np.int32)
        nc = ctypes.c_int32()
        _check(lib().cc_color(self._h, cols.ctypes.data, ctypes.byref(nc)))
        return cols

    def set_colors(self, colors, num_colors: Optional[int] = None):
        """A caller's colouring (no two vertices of a tet alike), e.g. a Kuhn
        grid's lattice colouring (i + j + k) mod 4."""
        c = np.ascontiguousarray(colors, dtype=np.int32)
        _check(lib().cc_set_colors(self._h, c.ctypes.data, int(c.max()) + 1 if num_colors is None else int(num_colors)))

    def build_subspace(self, k: int):
        _check(lib().cc_build_subspace(self._h, int(k)))

    def build_subspace_at(self, x) -> int:
        """Restarted bases from the Hessian at x; returns how many patches kept their basis."""
        kept = ctypes.c_int64()
        _check(lib().cc_build_subspace_at(self._h, _dev3n(x, self.n, "x"), ctypes.byref(kept)))
        return kept.value

    def set_subspace(self, sup_ptr, sup_idx, U):
        sp = np.ascontiguousarray(sup_ptr, dtype=np.int64)
        si = np.ascontiguousarray(sup_idx, dtype=np.int32)
        Ub = np.ascontiguousarray(U, dtype=np.float64)
        _check(lib().cc_set_subspace(self._h, sp.ctypes.data, si.ctypes.data if si.size else None,
                                     Ub.ctypes.data))

    def learned_inputs(self, X=None, T=None, targets: bool = False):
        """Network inputs (and with ``targets`` the computed k = 2 bases in
        slot order) of every free vertex: (X [n_free, 264] bf16, T or None)."""
        import torch
        nf = int(self.info().n_free)
        if X is None:
            X = torch.empty((nf, LEARNED_LDX), dtype=torch.bfloat16, device="cuda")
        if targets and T is None:
            T = torch.empty((nf, LEARNED_D_OUT), dtype=torch.float32, device="cuda")
        rows = ctypes.c_int64()
        _check(lib().cc_learned_inputs(self._h, _dev(X, torch.bfloat16, "X", LEARNED_LDX), X.stride(0),
                                       _dev(T, torch.float32, "T", LEARNED_D_OUT) if T is not None else None,
                                       T.stride(0) if T is not None else 0, X.shape[0], ctypes.byref(rows)))
        return X, T

    def build_learned_subspace(self, net: "MLP", tau: float = 1.0, want_rho: bool = False):
        """Learned k = 2 bases with the per-vertex fallback; returns (stats dict, rho or None)."""
        import torch
        st = LearnedStats()
        rho = torch.empty(int(self.info().n_free), dtype=torch.float64, device="cuda") if want_rho else None
        _check(lib().cc_build_learned_subspace(self._h, net._h, float(tau), _ptr(rho), ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in LearnedStats._fields_}, rho

    def info(self) -> MeshInfo:
        inf = MeshInfo()
        _check(lib().cc_get_info(self._h, ctypes.byref(inf)))
        return inf

    def export(self, name: str) -> np.ndarray:
        which, dt = ARRAYS[name]
        cnt = ctypes.c_int64()
        _check(lib().cc_export(self._h, which, None, 0, ctypes.byref(cnt)))
        out = np.empty(max(cnt.value, 1), dtype=dt)
        _check(lib().cc_export(self._h, which, out.ctypes.data, out.size, ctypes.byref(cnt)))
        return out[:cnt.value]

    def autotune(self, x, xtilde=None, precision: str = "mixed", sweeps: int = 4) -> dict:
        """Pick the fastest launch shapes for this mesh (x is not modified)."""
        r = TuneResult()
        _check(lib().cc_autotune(self._h, _dev3n(x, self.n, "x"), _dev3n(xtilde, self.n, "xtilde"), PREC[precision],
                                 int(sweeps), ctypes.byref(r)))
        return {"couple_threads": r.couple_threads, "couple_row_lanes": r.couple_row_lanes,
                "gather_warps": r.gather_warps, "couple_ms": list(r.couple_ms),
                "row_lanes_ms": list(r.row_lanes_ms), "gather_ms": list(r.gather_ms),
                "rows_from_positions": r.rows_from_positions, "fused_condense": r.fused_condense,
                "variant_ms": list(r.variant_ms)}

    def set_launch_shape(self, couple_threads: int = 0, gather_warps: int = 0, couple_row_lanes: int = 0):
        """Pins the coupling kernel's threads per vertex (32 = one warp) and threads per block row,
        and the gather's warps per block (0 keeps a value)."""
        _check(lib().cc_set_launch_shape(self._h, int(couple_threads), int(gather_warps), int(couple_row_lanes)))

    def set_sweep_variant(self, rows_from_positions: int = -1, fused_condense: int = -1):
        """Chooses the sweep's kernel variants (1 on, 0 off, -1 keep)."""
        _check(lib().cc_set_sweep_variant(self._h, int(rows_from_positions), int(fused_condense)))

    def profile_enable(self, on: bool = True):
        _check(lib().cc_profile_enable(self._h, int(on)))

    def profile_read(self) -> dict:
        """Per-class device milliseconds and launch counts since the last read."""
        p = Profile()
        _check(lib().cc_profile_read(self._h, ctypes.byref(p)))
        out = {k: {"ms": p.ms[i], "launches": p.launches[i]} for i, k in enumerate(PROFILE_CLASSES)}
        out["total_launches"] = p.total_launches
        return out

    def energy_grad(self, x, xtilde=None, precision: str = "fp64", want_grad: bool = True):
        import torch
        gx = _dev3n(x, self.n, "x")
        gt = _dev3n(xtilde, self.n, "xtilde")
        grad = torch.empty_like(x) if want_grad else None
        e, gn = ctypes.c_double(), ctypes.c_double()
        _check(lib().cc_energy_grad(self._h, gx, gt, PREC[precision], ctypes.byref(e), _ptr(grad),
                                    ctypes.byref(gn)))
        return e.value, grad, gn.value

    def sweep(self, x, xtilde=None, update: str = "cc", schedule: str = "colored", precision: str = "fp64",
              color_begin: int = 0, color_end: int = -1, corotated: bool = False) -> SweepStats:
        o = SweepOpts(UPDATE[update], SCHED[schedule], PREC[precision], color_begin, color_end, int(corotated))
        st = SweepStats()
        _check(lib().cc_sweep(self._h, _dev3n(x, self.n, "x"), _dev3n(xtilde, self.n, "xtilde"),
                              ctypes.byref(o), ctypes.byref(st)))
        return st

    def solve_step(self, x, v=None, *, update: str = "cc", schedule: str = "colored", precision: str = "mixed",
                   tol: float = 1e-6, max_iters: int = 200, min_iters: int = 0, check_every: int = 1,
                   use_graph: bool = False, history: bool = False, corotated: bool = False,
                   line_search: bool = False, restart_every: int = 0) -> SolveResult:
        hist = np.full(max_iters + 1, -1.0) if history else None
        o = StepOpts(UPDATE[update], SCHED[schedule], PREC[precision], tol, max_iters, min_iters, check_every,
                     int(use_graph),
                     hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if hist is not None else None,
                     int(corotated), int(restart_every), int(line_search))
        st = StepStats()
        rc = lib().cc_solve_step(self._h, _dev3n(x, self.n, "x"), _dev3n(v, self.n, "v"), ctypes.byref(o),
                                 ctypes.byref(st))
        if rc not in (OK, ERR_NOT_CONVERGED):
            err = CCError(rc, lib().cc_last_error().decode())
            err.residuals = hist   # the residuals checked before the failure (-1 past it)
            raise err
        return SolveResult(st.iterations, bool(st.converged), st.g0, st.g_final, st.energy_final,
                           st.sweeps.updates, st.sweeps.fallback_empty, st.sweeps.fallback_reduced,
                           st.sweeps.fallback_schur, hist)


def solve_concurrent(meshes, xs, vs=None, *, update: str = "cc", schedule: str = "colored",
                     precision: str = "mixed", tol: float = 1e-6, max_iters: int = 200, min_iters: int = 0,
                     check_every: int = 1, use_graph: bool = False, history: bool = False,
                     corotated: bool = False, line_search: bool = False, restart_every: int = 0):
    """Mesh.solve_step on several meshes at once (cc_solve_concurrent): each mesh on
    its own stream and host thread, every mesh with the same options.  Returns one
    SolveResult per mesh (``converged`` False where max_iters came first); raises
    CCError for any other failure, with ``statuses`` (per mesh) attached."""
    count = len(meshes)
    if len(xs) != count or (vs is not None and len(vs) != count):
        raise CCError(ERR_INVALID_ARG, "one x (and v) per mesh")
    hists = [np.full(max_iters + 1, -1.0) if history else None for _ in range(count)]
    opts = (StepOpts * count)()
    for k in range(count):
        opts[k] = StepOpts(UPDATE[update], SCHED[schedule], PREC[precision], tol, max_iters, min_iters,
                           check_every, int(use_graph),
                           hists[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history else None,
                           int(corotated), int(restart_every), int(line_search))
    hs = (_P * count)(*[m._h for m in meshes])
    xp = (_P * count)(*[_dev3n(x, m.n, "x") for m, x in zip(meshes, xs)])
    vp = None if vs is None else (_P * count)(*[_dev3n(v, m.n, "v") for m, v in zip(meshes, vs)])
    st = (StepStats * count)()
    rcs = (ctypes.c_int * count)()
    rc = lib().cc_solve_concurrent(count, hs, xp, vp, opts, st, rcs)
    if rc not in (OK, ERR_NOT_CONVERGED):
        err = CCError(rc, lib().cc_last_error().decode())
        err.statuses = list(rcs)
        raise err
    return [SolveResult(s_.iterations, bool(s_.converged), s_.g0, s_.g_final, s_.energy_final, s_.sweeps.updates,
                        s_.sweeps.fallback_empty, s_.sweeps.fallback_reduced, s_.sweeps.fallback_schur, h)
            for s_, h in zip(st, hists)]


def gemm_bf16_tn(A, B, out=None, stream=None, n_tile: int = 0, k_splits: int = 0, one_tile_per_cta: bool = False):
    """C = A . B^T on the tcgen05 kernel (A [M, K], B [N, K] bf16 CUDA tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = out if out is not None else torch.empty((M, N), dtype=torch.float32, device=A.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().cc_gemm_bf16_tn(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), M, N, K, C.data_ptr(),
                                 C.stride(0), int(n_tile), int(k_splits), 1 if one_tile_per_cta else 0,
                                 _stream_ptr(st)))
    return C


def mlp_activation(x):
    """(erf, GELU, GELU') of a float32 CUDA tensor as the network's epilogues compute them."""
    import torch
    out = torch.empty((x.numel(), 3), dtype=torch.float32, device=x.device)
    _check(lib().cc_mlp_activation(x.data_ptr(), x.numel(), out.data_ptr(),
                                   _stream_ptr(torch.cuda.current_stream())))
    return out


def _dev(t, dtype, name, cols=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.dim() == 2 and t.stride(1) == 1):
        raise CCError(ERR_INVALID_ARG, f"{name} must be a row-major 2-D {dtype} CUDA tensor")
    if cols is not None and t.shape[1] < cols:
        raise CCError(ERR_INVALID_ARG, f"{name} needs at least {cols} columns")
    return t.data_ptr()


class MLP:
    """The subspace network on the GPU (owns the library's ``cc_mlp``)."""

    def __init__(self, d_in: int = LEARNED_D_IN, hidden: int = 256, layers: int = 3, d_out: int = LEARNED_D_OUT,
                 max_batch: int = 8192, stream=None):
        cfg = MlpConfig(d_in, hidden, layers, d_out, max_batch)
        out = _P()
        self._h = None
        _check(lib().cc_mlp_create(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(out)))
        self._h = out
        self.dims = [d_in] + [hidden] * layers + [d_out]
        self.max_batch = max_batch

    def close(self):
        if self._h is not None and self._h.value:
            lib().cc_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self) -> int:
        return int(lib().cc_mlp_param_count(self._h))

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().cc_mlp_set_params(self._h, p.ctypes.data, p.size))

    def save(self, path: str):
        _check(lib().cc_mlp_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        _check(lib().cc_mlp_load(self._h, os.fsencode(path)))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.param_count, dtype=np.float32)
        _check(lib().cc_mlp_get_params(self._h, p.ctypes.data, p.size))
        return p

    def set_fused(self, on=True):
        """Inference kernel: one kernel for every layer (True or 1: SM pairs share weight tiles by
        multicast; 2: SM-pair MMAs) or one GEMM per layer (False or 0)."""
        _check(lib().cc_mlp_set_fused(self._h, int(on)))

    def forward(self, X, out=None):
        """Y [rows, d_out] float32 for BF16 inputs X [rows, >= d_in] (row stride a multiple of 8)."""
        import torch
        rows = X.shape[0]
        Y = out if out is not None else torch.empty((rows, self.dims[-1]), dtype=torch.float32, device=X.device)
        _check(lib().cc_mlp_forward(self._h, _dev(X, torch.bfloat16, "X"), X.stride(0), rows,
                                    _dev(Y, torch.float32, "Y", self.dims[-1]), Y.stride(0)))
        return Y

    def loss_grad(self, X, T, want_grad: bool = True):
        """(mean squared error, gradient as a float32 CUDA tensor or None)."""
        import torch
        g = torch.empty(self.param_count, dtype=torch.float32, device=X.device) if want_grad else None
        loss = ctypes.c_double()
        _check(lib().cc_mlp_loss_grad(self._h, _dev(X, torch.bfloat16, "X"), X.stride(0),
                                      _dev(T, torch.float32, "T", self.dims[-1]), T.stride(0), X.shape[0],
                                      ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def adam_step(self, grad, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(lib().cc_mlp_adam_step(self._h, grad.data_ptr(), ctypes.byref(Adam(lr, beta1, beta2, eps))))

    def train(self, X, T, idx, batch: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> np.ndarray:
        """Steps over minibatches idx [steps, batch] (int32 CUDA tensor); returns the losses."""
        import torch
        steps = idx.shape[0]
        if not (idx.is_cuda and idx.dtype == torch.int32 and idx.is_contiguous() and idx.shape[1] == batch):
            raise CCError(ERR_INVALID_ARG, "idx must be a contiguous int32 CUDA tensor [steps, batch]")
        losses = np.zeros(max(steps, 1))
        _check(lib().cc_mlp_train(self._h, _dev(X, torch.bfloat16, "X"), X.stride(0),
                                  _dev(T, torch.float32, "T", self.dims[-1]), T.stride(0), X.shape[0],
                                  idx.data_ptr(), steps, batch, ctypes.byref(Adam(lr, beta1, beta2, eps)),
                                  losses.ctypes.data))
        return losses[:steps]


def version() -> str:
    return lib().cc_version().decode()


def to_soa(x_n3, device="cuda"):
    """[n, 3] array -> contiguous (3, n) float64 tensor on ``device``."""
    import torch
    return torch.as_tensor(np.ascontiguousarray(np.asarray(x_n3, dtype=np.float64).T), device=device).contiguous()


def from_soa(t) -> np.ndarray:
    """(3, n) tensor -> [n, 3] numpy array."""
    return t.detach().cpu().numpy().T.copy()
