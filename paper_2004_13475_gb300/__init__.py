"""Python binding of libfractal.so (C ABI in include/fractal.h).

Argument marshalling only: every step of the map and the workloads runs in
the library's CUDA kernels.  Tensors are used for device memory and streams;
any object with ``data_ptr()`` (a CUDA tensor) or a plain integer device
address is accepted.  There is no CPU path: importing works anywhere, but the
first call loads the library and raises if it was not built, and the library
itself needs a CUDA device.

Names follow the C ABI: ``fractal_map`` returns a :class:`Plan`; the step,
write and reduce calls take the plan first.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

FRACTAL_OK = 0
FRACTAL_EINVAL = -1
FRACTAL_ENOMEM = -2
FRACTAL_ECUDA = -3
FRACTAL_ETOOBIG = -4
FRACTAL_NOALLOC_MAX_PARTIALS = 65536

FRACTAL_LAMBDA = 0
FRACTAL_BB = 1
FRACTAL_U8 = 0
FRACTAL_F32 = 1
FRACTAL_DF = 2  # double-float (hi, lo) pairs (gradient path)
FRACTAL_MAX_LEVEL = 16

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfractal.so")

# Every entry point declared in include/fractal.h.
EXPORTS = (
    "fractal_strerror", "fractal_last_cuda_error", "fractal_map", "fractal_plan_destroy",
    "fractal_plan_get_info", "fractal_plan_set_cta_levels", "fractal_map_blocks",
    "fractal_map_write", "fractal_step_ca", "fractal_step_diffusion", "fractal_reduce",
    "fractal_reduce_async", "fractal_set_l2_fetch_granularity", "fractal_get_l2_fetch_granularity",
    "fractal_plan_set_schedule", "fractal_plan_device_status", "fractal_reduce_noalloc",
    "fractal_plan_autotune", "fractal_plan_set_steps_per_launch",
    "fractal_batch_create", "fractal_batch_destroy", "fractal_batch_bind", "fractal_batch_configure",
    "fractal_batch_step_diffusion", "fractal_batch_reduce", "fractal_batch_autotune",
    "fractal_batch_graph_capture", "fractal_batch_graph_launch", "fractal_batch_get_info",
    "fractal_step_diffusion_kappa", "fractal_adjoint_diffusion_step",
    "fractal_step_diffusion_kappa_f64", "fractal_adjoint_diffusion_step_f64",
    "fractal_step_ca_count", "fractal_step_diffusion_sum", "fractal_map_blocks_method",
    "fractal_pack", "fractal_unpack",
    "fractal_step_diffusion_kappa_df", "fractal_adjoint_diffusion_step_df", "fractal_step_diffusion_sums",
    "fractal_fused_box_blocks", "fractal_plan_selftest_wait", "fractal_debug_fail_allocs",
    "fractal_kappa_fused_limits", "fractal_kappa_trajectory_df", "fractal_kappa_trajectory_df_io",
    "fractal_kappa_gradient_df", "fractal_kappa_gradient_df_io", "fractal_nbb_map_blocks", "fractal_nbb_write",
    "fractal_nbb_step_ca", "fractal_nbb_reduce", "fractal_nbb_step_diffusion",
    "fractal_plan_set_kappa_fusion", "fractal_plan_records_bytes", "fractal_records_from_array",
    "fractal_records_to_array", "fractal_step_diffusion_records", "fractal_step_ca_records",
)

FRACTAL_SCHED_AUTO = 0
FRACTAL_SCHED_STAGED = 1
FRACTAL_SCHED_TMA = 2


class FractalError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _load()
        msg = lib.fractal_strerror(status).decode()
        cuda = lib.fractal_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f"; {cuda}" if cuda and status == FRACTAL_ECUDA else ""))
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32), ("rho", ctypes.c_int32), ("mode", ctypes.c_int32), ("r_b", ctypes.c_int32),
        ("n", ctypes.c_int64), ("n_b", ctypes.c_int64), ("grid_w", ctypes.c_int32), ("grid_h", ctypes.c_int32),
        ("member_tiles", ctypes.c_int64), ("members", ctypes.c_int64),
        ("cta_levels", ctypes.c_int32 * 2), ("ctas", ctypes.c_int64 * 2),
        ("threads", ctypes.c_int32 * 2), ("smem_bytes", ctypes.c_int32 * 2),
        ("tma", ctypes.c_int32 * 2), ("sched", ctypes.c_int32),
        ("steps_per_launch", ctypes.c_int32 * 2),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int32), ("k_min", ctypes.c_int32), ("k_max", ctypes.c_int32),
        ("supertile", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32), ("ctas", ctypes.c_int32),
        ("threads", ctypes.c_int32), ("smem_bytes", ctypes.c_int32), ("supertiles", ctypes.c_int64),
        ("members", ctypes.c_int64), ("bound", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, F, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_void_p
    sig = {
        "fractal_strerror": (ctypes.c_char_p, [I]),
        "fractal_last_cuda_error": (ctypes.c_char_p, []),
        "fractal_map": (I, [I, I, I, ctypes.POINTER(P)]),
        "fractal_plan_destroy": (I, [P]),
        "fractal_plan_get_info": (I, [P, ctypes.POINTER(PlanInfo)]),
        "fractal_plan_set_cta_levels": (I, [P, I, I]),
        "fractal_map_blocks": (I, [P, VP, VP]),
        "fractal_nbb_map_blocks": (I, [I, I, ctypes.POINTER(ctypes.c_int32), I, VP, VP]),
        "fractal_nbb_write": (I, [I, I, ctypes.POINTER(ctypes.c_int32), I, I, I, I, F, VP, VP]),
        "fractal_nbb_step_ca": (I, [I, I, ctypes.POINTER(ctypes.c_int32), I, I, I, VP, VP, I, VP]),
        "fractal_nbb_reduce": (I, [I, I, ctypes.POINTER(ctypes.c_int32), I, I, I, VP, VP, ctypes.c_int64, VP,
                                   VP]),
        "fractal_nbb_step_diffusion": (I, [I, I, ctypes.POINTER(ctypes.c_int32), I, I, I, VP, VP, F, I, VP]),
        "fractal_map_write": (I, [P, VP, I, D, VP]),
        "fractal_step_ca": (I, [P, VP, VP, I, VP]),
        "fractal_step_diffusion": (I, [P, VP, VP, F, I, VP]),
        "fractal_reduce": (I, [P, VP, I, ctypes.POINTER(D), VP]),
        "fractal_reduce_async": (I, [P, VP, I, VP, VP]),
        "fractal_set_l2_fetch_granularity": (I, [I]),
        "fractal_fused_box_blocks": (I, [I, I, I]),
        "fractal_get_l2_fetch_granularity": (I, [ctypes.POINTER(I)]),
        "fractal_plan_set_schedule": (I, [P, I]),
        "fractal_plan_device_status": (I, [P, ctypes.POINTER(I)]),
        "fractal_reduce_noalloc": (I, [I, I, VP, I, VP, VP]),
        "fractal_plan_autotune": (I, [P, I, VP, VP, I, ctypes.POINTER(F), VP]),
        "fractal_plan_set_steps_per_launch": (I, [P, I, I]),
        "fractal_batch_create": (I, [I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(P)]),
        "fractal_batch_destroy": (I, [P]),
        "fractal_batch_bind": (I, [P, ctypes.POINTER(VP), ctypes.POINTER(VP)]),
        "fractal_batch_configure": (I, [P, I, I]),
        "fractal_batch_step_diffusion": (I, [P, F, I, VP]),
        "fractal_batch_reduce": (I, [P, I, VP, VP]),
        "fractal_batch_autotune": (I, [P, F, I, ctypes.POINTER(F), VP]),
        "fractal_batch_graph_capture": (I, [P, F, I]),
        "fractal_batch_graph_launch": (I, [P, VP]),
        "fractal_batch_get_info": (I, [P, ctypes.POINTER(BatchInfo)]),
        "fractal_step_diffusion_kappa": (I, [P, VP, VP, VP, F, I, VP]),
        "fractal_adjoint_diffusion_step": (I, [P, VP, VP, VP, VP, VP, F, VP]),
        "fractal_step_diffusion_kappa_f64": (I, [P, VP, VP, VP, D, I, VP]),
        "fractal_step_ca_count": (I, [P, VP, VP, I, VP, VP]),
        "fractal_map_blocks_method": (I, [P, VP, I, VP]),
        "fractal_pack": (I, [P, VP, I, VP, VP]),
        "fractal_step_diffusion_kappa_df": (I, [P, VP, VP, VP, D, I, VP]),
        "fractal_adjoint_diffusion_step_df": (I, [P, VP, VP, VP, VP, VP, D, VP]),
        "fractal_unpack": (I, [P, VP, I, VP, VP]),
        "fractal_step_diffusion_sum": (I, [P, VP, VP, F, I, VP, VP]),
        "fractal_step_diffusion_sums": (I, [P, VP, VP, F, I, I, VP, VP]),
        "fractal_adjoint_diffusion_step_f64": (I, [P, VP, VP, VP, VP, VP, D, VP]),
        "fractal_plan_selftest_wait": (I, [P, ctypes.c_uint, VP]),
        "fractal_kappa_fused_limits": (I, [I, I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(I)]),
        "fractal_kappa_trajectory_df": (I, [P, VP, VP, VP, VP, D, I, VP]),
        "fractal_kappa_trajectory_df_io": (I, [P, VP, I, VP, I, VP, VP, D, I, VP]),
        "fractal_kappa_gradient_df": (I, [P, VP, VP, VP, D, I, VP]),
        "fractal_kappa_gradient_df_io": (I, [P, VP, VP, VP, I, VP, D, I, VP]),
        "fractal_plan_set_kappa_fusion": (I, [P, I]),
        "fractal_plan_records_bytes": (I, [P, I, ctypes.POINTER(ctypes.c_int64)]),
        "fractal_records_from_array": (I, [P, I, VP, VP, VP]),
        "fractal_records_to_array": (I, [P, I, VP, VP, VP]),
        "fractal_step_diffusion_records": (I, [P, VP, VP, F, I, I, VP, VP]),
        "fractal_step_ca_records": (I, [P, VP, VP, I, VP, VP]),
        "fractal_debug_fail_allocs": (I, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:  # pragma: no cover - torch absent
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(status: int, where: str) -> None:
    if status != FRACTAL_OK:
        raise FractalError(status, where)


class Plan:
    """Owner of a ``fractal_plan_t`` (freed on close / garbage collection)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("plan is closed")
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        _check(_load().fractal_plan_get_info(self.handle, ctypes.byref(inf)), "fractal_plan_get_info")
        return inf.as_dict()

    def close(self) -> None:
        if self._h:
            _load().fractal_plan_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fractal_map(k: int, rho: int, mode: int = FRACTAL_LAMBDA) -> Plan:
    h = ctypes.c_void_p()
    _check(_load().fractal_map(k, rho, mode, ctypes.byref(h)), "fractal_map")
    return Plan(h.value)


def fractal_plan_set_cta_levels(plan: Plan, dtype: int, levels: int) -> None:
    _check(_load().fractal_plan_set_cta_levels(plan.handle, dtype, levels), "fractal_plan_set_cta_levels")


def fractal_plan_set_schedule(plan: Plan, sched: int) -> None:
    _check(_load().fractal_plan_set_schedule(plan.handle, int(sched)), "fractal_plan_set_schedule")


def fractal_plan_autotune(plan: Plan, dtype: int, dev_in, dev_scratch, reps: int = 5, stream=None) -> float:
    """Pick the fastest staging and CTA shape for `dtype`; returns its mean step time (us).
    dev_in is only read, dev_scratch is overwritten."""
    best = ctypes.c_float(-1.0)
    _check(_load().fractal_plan_autotune(plan.handle, int(dtype), _ptr(dev_in), _ptr(dev_scratch), int(reps),
                                         ctypes.byref(best), _stream(stream)), "fractal_plan_autotune")
    return best.value


def fractal_plan_set_steps_per_launch(plan: Plan, dtype: int, spl: int) -> None:
    _check(_load().fractal_plan_set_steps_per_launch(plan.handle, int(dtype), int(spl)),
           "fractal_plan_set_steps_per_launch")


def fractal_plan_device_status(plan: Plan) -> int:
    v = ctypes.c_int()
    _check(_load().fractal_plan_device_status(plan.handle, ctypes.byref(v)), "fractal_plan_device_status")
    return v.value


def fractal_plan_selftest_wait(plan: Plan, spins: int = 1 << 16, stream=None) -> None:
    """Make the bounded device wait run out once (the plan's status becomes 1)."""
    _check(_load().fractal_plan_selftest_wait(plan.handle, int(spins), _stream(stream)), "fractal_plan_selftest_wait")


def fractal_debug_fail_allocs(after: int) -> None:
    """Fail the library's device allocation after `after` more successes (< 0: off)."""
    _check(_load().fractal_debug_fail_allocs(int(after)), "fractal_debug_fail_allocs")


def fractal_plan_records_bytes(plan: Plan, dtype: int) -> int:
    """Bytes of one state of `dtype` in the plan's record form (needs steps per launch > 1)."""
    v = ctypes.c_int64()
    _check(_load().fractal_plan_records_bytes(plan.handle, int(dtype), ctypes.byref(v)), "fractal_plan_records_bytes")
    return v.value


def fractal_records_from_array(plan: Plan, dtype: int, embedded, records, stream=None) -> None:
    _check(_load().fractal_records_from_array(plan.handle, int(dtype), _ptr(embedded), _ptr(records), _stream(stream)),
           "fractal_records_from_array")


def fractal_records_to_array(plan: Plan, dtype: int, records, embedded, stream=None) -> None:
    _check(_load().fractal_records_to_array(plan.handle, int(dtype), _ptr(records), _ptr(embedded), _stream(stream)),
           "fractal_records_to_array")


def fractal_step_diffusion_records(plan: Plan, rec_in, rec_out, coef: float, steps: int, every: int = 0,
                                   dev_sums=None, stream=None) -> None:
    """Diffusion steps from records rec_in to records rec_out (sums every `every` steps, default: once)."""
    _check(_load().fractal_step_diffusion_records(plan.handle, _ptr(rec_in), _ptr(rec_out), float(coef), int(steps),
                                                  int(every or steps), _ptr(dev_sums), _stream(stream)),
           "fractal_step_diffusion_records")


def fractal_step_ca_records(plan: Plan, rec_in, rec_out, steps: int, dev_count=None, stream=None) -> None:
    """Automaton steps from bit records rec_in to rec_out (alive count into dev_count, nullable)."""
    _check(_load().fractal_step_ca_records(plan.handle, _ptr(rec_in), _ptr(rec_out), int(steps), _ptr(dev_count),
                                           _stream(stream)), "fractal_step_ca_records")


def fractal_plan_set_kappa_fusion(plan: Plan, on: bool) -> None:
    """Temporal fusion of the double-float conductivity steps on (default) or off."""
    _check(_load().fractal_plan_set_kappa_fusion(plan.handle, 1 if on else 0), "fractal_plan_set_kappa_fusion")


def fractal_kappa_fused_limits(k: int, mode: int = FRACTAL_LAMBDA):
    """(floats of one recorded state, most steps per fused launch) of the
    double-float gradient path at level k; raises for k < 4."""
    rf = ctypes.c_int64()
    ms = ctypes.c_int()
    _check(_load().fractal_kappa_fused_limits(int(k), int(mode), ctypes.byref(rf), ctypes.byref(ms)),
           "fractal_kappa_fused_limits")
    return rf.value, ms.value


def fractal_kappa_trajectory_df(plan: Plan, dev_in, dev_out, dev_traj, dev_kappa, coef: float, steps: int,
                                stream=None) -> None:
    """`steps` fused double-float conductivity steps from dev_in, the states
    before each step into dev_traj (record form; nullable) and the result into
    dev_out (or, when dev_out is None, into trajectory state `steps`)."""
    _check(_load().fractal_kappa_trajectory_df(plan.handle, _ptr(dev_in), _ptr(dev_out), _ptr(dev_traj),
                                               _ptr(dev_kappa), float(coef), int(steps), _stream(stream)),
           "fractal_kappa_trajectory_df")


def fractal_kappa_trajectory_df_io(plan: Plan, dev_in, in_format: int, dev_out, out_format: int, dev_traj,
                                   dev_kappa, coef: float, steps: int, stream=None) -> None:
    """fractal_kappa_trajectory_df with the input and result formats chosen
    (FRACTAL_DF pairs or FRACTAL_F32 floats)."""
    _check(_load().fractal_kappa_trajectory_df_io(plan.handle, _ptr(dev_in), int(in_format), _ptr(dev_out),
                                                  int(out_format), _ptr(dev_traj), _ptr(dev_kappa), float(coef),
                                                  int(steps), _stream(stream)), "fractal_kappa_trajectory_df_io")


def fractal_kappa_gradient_df(plan: Plan, dev_utraj, dev_ptraj, dev_gkappa, coef: float, steps: int,
                              stream=None) -> None:
    """dJ/dkappa of a segment of `steps` steps from the recorded u and p trajectories (double-float)."""
    _check(_load().fractal_kappa_gradient_df(plan.handle, _ptr(dev_utraj), _ptr(dev_ptraj), _ptr(dev_gkappa),
                                             float(coef), int(steps), _stream(stream)), "fractal_kappa_gradient_df")


def fractal_kappa_gradient_df_io(plan: Plan, dev_utraj, dev_ptraj, dev_gkappa, accumulate: bool, dev_out_f32,
                                 coef: float, steps: int, stream=None) -> None:
    """dJ/dkappa of a segment added to dev_gkappa (accumulate) or from 0, into
    dev_gkappa (double-float) or, when given, dev_out_f32 (float32)."""
    _check(_load().fractal_kappa_gradient_df_io(plan.handle, _ptr(dev_utraj), _ptr(dev_ptraj), _ptr(dev_gkappa),
                                                1 if accumulate else 0, _ptr(dev_out_f32), float(coef), int(steps),
                                                _stream(stream)), "fractal_kappa_gradient_df_io")


def fractal_map_blocks(plan: Plan, dev_xy, stream=None) -> None:
    _check(_load().fractal_map_blocks(plan.handle, _ptr(dev_xy), _stream(stream)), "fractal_map_blocks")


def _nbb_cells(cells):
    flat = [int(v) for xy in cells for v in xy]
    return (ctypes.c_int32 * max(1, len(flat)))(*flat)


def fractal_nbb_map_blocks(s: int, cells, r: int, dev_xy, stream=None) -> None:
    """lambda(omega) of an NBB fractal (step: s and its k cells (x, y) in
    numbering order) for every block of the packed grid at level r: 2 k^r int32."""
    _check(_load().fractal_nbb_map_blocks(int(s), len(cells), _nbb_cells(cells), int(r), _ptr(dev_xy),
                                          _stream(stream)), "fractal_nbb_map_blocks")


def fractal_nbb_write(s: int, cells, r_b: int, j: int, mode: int, value: float, dev_buf, stream=None,
                      cta_levels: int = 0) -> None:
    """The single write on the level-(r_b + j) NBB fractal in tiles of side
    s^j: one CTA per tile (cta_levels = 0) or per super-tile of s^m x s^m tiles."""
    _check(_load().fractal_nbb_write(int(s), len(cells), _nbb_cells(cells), int(r_b), int(j), int(cta_levels),
                                     int(mode), float(value), _ptr(dev_buf), _stream(stream)), "fractal_nbb_write")


def fractal_nbb_step_ca(s: int, cells, r_b: int, j: int, mode: int, dev_a, dev_b, steps: int, stream=None):
    """`steps` B3/S23 steps on the level-(r_b + j) NBB fractal, one CTA per
    tile of side s^j; returns the buffer holding the result (dev_a for even steps)."""
    _check(_load().fractal_nbb_step_ca(int(s), len(cells), _nbb_cells(cells), int(r_b), int(j), int(mode),
                                       _ptr(dev_a), _ptr(dev_b), int(steps), _stream(stream)), "fractal_nbb_step_ca")
    return dev_a if steps % 2 == 0 else dev_b


def fractal_nbb_reduce(s: int, cells, r_b: int, j: int, mode: int, dev_buf, dev_partials, dev_out,
                       stream=None) -> None:
    """Sum over the members of the level-(r_b + j) NBB fractal into dev_out
    (FP64), one CTA per tile of side s^j; dev_partials: one double per CTA."""
    _check(_load().fractal_nbb_reduce(int(s), len(cells), _nbb_cells(cells), int(r_b), int(j), int(mode),
                                      _ptr(dev_buf), _ptr(dev_partials), int(dev_partials.numel()), _ptr(dev_out),
                                      _stream(stream)), "fractal_nbb_reduce")


def fractal_nbb_step_diffusion(s: int, cells, r_b: int, j: int, mode: int, dev_a, dev_b, coef: float, steps: int,
                               stream=None):
    """`steps` float32 diffusion steps on the level-(r_b + j) NBB fractal, one
    CTA per tile of side s^j; returns the buffer holding the result."""
    _check(_load().fractal_nbb_step_diffusion(int(s), len(cells), _nbb_cells(cells), int(r_b), int(j), int(mode),
                                              _ptr(dev_a), _ptr(dev_b), float(coef), int(steps), _stream(stream)),
           "fractal_nbb_step_diffusion")
    return dev_a if steps % 2 == 0 else dev_b


FRACTAL_MAP_BALLOT = 0
FRACTAL_MAP_SCALAR = 1
FRACTAL_MAP_MMA = 2


def fractal_map_blocks_method(plan: Plan, dev_xy, method: int, stream=None) -> None:
    _check(_load().fractal_map_blocks_method(plan.handle, _ptr(dev_xy), int(method), _stream(stream)),
           "fractal_map_blocks_method")


def fractal_map_write(plan: Plan, buf, dtype: int, value: float, stream=None) -> None:
    _check(_load().fractal_map_write(plan.handle, _ptr(buf), dtype, float(value), _stream(stream)),
           "fractal_map_write")


def fractal_step_ca(plan: Plan, a, b, steps: int, stream=None):
    """Run `steps` CA steps; returns whichever of (a, b) holds the result."""
    _check(_load().fractal_step_ca(plan.handle, _ptr(a), _ptr(b), int(steps), _stream(stream)),
           "fractal_step_ca")
    return a if steps % 2 == 0 else b


def fractal_step_diffusion(plan: Plan, a, b, coef: float, steps: int, stream=None):
    """Run `steps` diffusion steps with a = alpha*dt; returns the buffer holding the result."""
    _check(_load().fractal_step_diffusion(plan.handle, _ptr(a), _ptr(b), float(coef), int(steps),
                                          _stream(stream)), "fractal_step_diffusion")
    return a if steps % 2 == 0 else b


def fractal_step_ca_count(plan: Plan, a, b, steps: int, dev_count, stream=None):
    """CA steps, then the alive count of the result into the device double `dev_count`;
    returns the buffer holding the result."""
    _check(_load().fractal_step_ca_count(plan.handle, _ptr(a), _ptr(b), int(steps), _ptr(dev_count),
                                         _stream(stream)), "fractal_step_ca_count")
    return a if steps % 2 == 0 else b


def fractal_step_diffusion_sum(plan: Plan, a, b, coef: float, steps: int, dev_sum, stream=None):
    """Diffusion steps, then the member sum of the result into the device double `dev_sum`;
    returns the buffer holding the result."""
    _check(_load().fractal_step_diffusion_sum(plan.handle, _ptr(a), _ptr(b), float(coef), int(steps),
                                              _ptr(dev_sum), _stream(stream)), "fractal_step_diffusion_sum")
    return a if steps % 2 == 0 else b


def fractal_step_diffusion_sums(plan: Plan, a, b, coef: float, steps: int, every: int, dev_sums, stream=None):
    """Diffusion steps with the member sum after every `every` steps into the
    device doubles `dev_sums` (steps / every of them); returns the buffer
    holding the result."""
    _check(_load().fractal_step_diffusion_sums(plan.handle, _ptr(a), _ptr(b), float(coef), int(steps), int(every),
                                               _ptr(dev_sums), _stream(stream)), "fractal_step_diffusion_sums")
    return a if steps % 2 == 0 else b


def fractal_reduce(plan: Plan, buf, dtype: int, stream=None) -> float:
    out = ctypes.c_double()
    _check(_load().fractal_reduce(plan.handle, _ptr(buf), dtype, ctypes.byref(out), _stream(stream)),
           "fractal_reduce")
    return out.value


def fractal_reduce_async(plan: Plan, buf, dtype: int, dev_out, stream=None) -> None:
    _check(_load().fractal_reduce_async(plan.handle, _ptr(buf), dtype, _ptr(dev_out), _stream(stream)),
           "fractal_reduce_async")


def fractal_reduce_noalloc(k: int, rho: int, buf, dtype: int, dev_out, stream=None) -> None:
    """Sum over the members into the device double `dev_out` without any allocation
    (fixed scratch inside the library; see include/fractal.h)."""
    _check(_load().fractal_reduce_noalloc(int(k), int(rho), _ptr(buf), int(dtype), _ptr(dev_out),
                                          _stream(stream)), "fractal_reduce_noalloc")


def fractal_pack(plan: Plan, embedded, dtype: int, packed, stream=None) -> None:
    """Member tiles of `embedded` in lambda order into `packed` (member_tiles * rho^2 elements).

    Either buffer may be a pinned CPU tensor (mapped into the device's address
    space): the kernel then reads or writes host memory directly."""
    _check(_load().fractal_pack(plan.handle, _ptr(embedded), int(dtype), _ptr(packed), _stream(stream)),
           "fractal_pack")


def fractal_unpack(plan: Plan, packed, dtype: int, embedded, stream=None) -> None:
    """Inverse of fractal_pack: writes the member tiles of `embedded`."""
    _check(_load().fractal_unpack(plan.handle, _ptr(packed), int(dtype), _ptr(embedded), _stream(stream)),
           "fractal_unpack")


def fractal_fused_box_blocks(supertile: int, margin: int, reach: int) -> int:
    """Margin-box blocks a float32 fused launch stages per super-tile (host only)."""
    r = _load().fractal_fused_box_blocks(int(supertile), int(margin), int(reach))
    if r < 0:
        _check(r, "fractal_fused_box_blocks")
    return r


def fractal_set_l2_fetch_granularity(nbytes: int) -> None:
    _check(_load().fractal_set_l2_fetch_granularity(int(nbytes)), "fractal_set_l2_fetch_granularity")


def fractal_get_l2_fetch_granularity() -> int:
    v = ctypes.c_int()
    _check(_load().fractal_get_l2_fetch_granularity(ctypes.byref(v)), "fractal_get_l2_fetch_granularity")
    return v.value


def fractal_step_diffusion_kappa(plan: Plan, a, b, kappa, coef: float, steps: int, stream=None):
    """`steps` diffusion steps with per-cell conductivity `kappa` (float32 state);
    returns the buffer holding the result."""
    _check(_load().fractal_step_diffusion_kappa(plan.handle, _ptr(a), _ptr(b), _ptr(kappa), float(coef), int(steps),
                                                _stream(stream)), "fractal_step_diffusion_kappa")
    return a if steps % 2 == 0 else b


def fractal_step_diffusion_kappa_f64(plan: Plan, a, b, kappa, coef: float, steps: int, stream=None):
    """The same with a float64 state (a, b float64; kappa float32)."""
    _check(_load().fractal_step_diffusion_kappa_f64(plan.handle, _ptr(a), _ptr(b), _ptr(kappa), float(coef),
                                                    int(steps), _stream(stream)), "fractal_step_diffusion_kappa_f64")
    return a if steps % 2 == 0 else b


def fractal_adjoint_diffusion_step(plan: Plan, u, p_in, p_out, kappa, gkappa, coef: float, stream=None) -> None:
    """One reverse step: p_out = A p_in, gkappa (float64) += the step's dJ/dkappa (u = the forward state u_t)."""
    _check(_load().fractal_adjoint_diffusion_step(plan.handle, _ptr(u), _ptr(p_in), _ptr(p_out), _ptr(kappa),
                                                  _ptr(gkappa), float(coef), _stream(stream)),
           "fractal_adjoint_diffusion_step")


def fractal_adjoint_diffusion_step_f64(plan: Plan, u, p_in, p_out, kappa, gkappa, coef: float, stream=None) -> None:
    """The reverse step with float64 u and p."""
    _check(_load().fractal_adjoint_diffusion_step_f64(plan.handle, _ptr(u), _ptr(p_in), _ptr(p_out), _ptr(kappa),
                                                      _ptr(gkappa), float(coef), _stream(stream)),
           "fractal_adjoint_diffusion_step_f64")


def fractal_step_diffusion_kappa_df(plan: Plan, a, b, kappa, coef: float, steps: int, stream=None):
    """The same with a double-float state: a, b float32 tensors of 2 n^2
    elements, (hi, lo) per cell (value hi + lo); kappa float32."""
    _check(_load().fractal_step_diffusion_kappa_df(plan.handle, _ptr(a), _ptr(b), _ptr(kappa), float(coef),
                                                   int(steps), _stream(stream)), "fractal_step_diffusion_kappa_df")
    return a if steps % 2 == 0 else b


def fractal_adjoint_diffusion_step_df(plan: Plan, u, p_in, p_out, kappa, gkappa, coef: float, stream=None) -> None:
    """The reverse step with double-float u, p and gkappa ((hi, lo) pairs)."""
    _check(_load().fractal_adjoint_diffusion_step_df(plan.handle, _ptr(u), _ptr(p_in), _ptr(p_out), _ptr(kappa),
                                                     _ptr(gkappa), float(coef), _stream(stream)),
           "fractal_adjoint_diffusion_step_df")


class Batch:
    """Owner of a ``fractal_batch_t``: many gaskets of uneven levels advanced
    by one persistent launch (include/fractal.h, "Batches")."""

    def __init__(self, handle: int, ks):
        self._h = ctypes.c_void_p(handle)
        self.ks = list(ks)

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("batch is closed")
        return self._h

    def info(self) -> dict:
        inf = BatchInfo()
        _check(_load().fractal_batch_get_info(self.handle, ctypes.byref(inf)), "fractal_batch_get_info")
        return inf.as_dict()

    def close(self) -> None:
        if self._h:
            _load().fractal_batch_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fractal_batch_create(ks) -> Batch:
    arr = (ctypes.c_int32 * len(ks))(*[int(k) for k in ks])
    h = ctypes.c_void_p()
    _check(_load().fractal_batch_create(len(ks), arr, ctypes.byref(h)), "fractal_batch_create")
    return Batch(h.value, ks)


def fractal_batch_bind(batch: Batch, a_list, b_list) -> None:
    """a_list, b_list: per-instance device buffers (tensors or addresses)."""
    n = len(batch.ks)
    if len(a_list) != n or len(b_list) != n:
        raise ValueError("one buffer pair per instance")
    A = (ctypes.c_void_p * n)(*[_ptr(x) for x in a_list])
    B = (ctypes.c_void_p * n)(*[_ptr(x) for x in b_list])
    _check(_load().fractal_batch_bind(batch.handle, A, B), "fractal_batch_bind")


def fractal_batch_configure(batch: Batch, supertile: int, steps_per_launch: int) -> None:
    _check(_load().fractal_batch_configure(batch.handle, int(supertile), int(steps_per_launch)),
           "fractal_batch_configure")


def fractal_batch_step_diffusion(batch: Batch, coef: float, steps: int, stream=None) -> int:
    """Run `steps` steps on every instance; returns 0 if the results are in the
    a buffers, 1 if in the b buffers."""
    _check(_load().fractal_batch_step_diffusion(batch.handle, float(coef), int(steps), _stream(stream)),
           "fractal_batch_step_diffusion")
    return steps % 2


def fractal_batch_reduce(batch: Batch, which: int, dev_out, stream=None) -> None:
    _check(_load().fractal_batch_reduce(batch.handle, int(which), _ptr(dev_out), _stream(stream)),
           "fractal_batch_reduce")


def fractal_batch_autotune(batch: Batch, coef: float = 0.2, reps: int = 3, stream=None) -> float:
    best = ctypes.c_float(-1.0)
    _check(_load().fractal_batch_autotune(batch.handle, float(coef), int(reps), ctypes.byref(best),
                                          _stream(stream)), "fractal_batch_autotune")
    return best.value


def fractal_batch_graph_capture(batch: Batch, coef: float, steps: int) -> None:
    _check(_load().fractal_batch_graph_capture(batch.handle, float(coef), int(steps)), "fractal_batch_graph_capture")


def fractal_batch_graph_launch(batch: Batch, stream=None) -> None:
    _check(_load().fractal_batch_graph_launch(batch.handle, _stream(stream)), "fractal_batch_graph_launch")


def fractal_strerror(status: int) -> str:
    return _load().fractal_strerror(status).decode()


def fractal_last_cuda_error() -> str:
    return _load().fractal_last_cuda_error().decode()
