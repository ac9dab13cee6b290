"""Python binding of libmpt (the C ABI declared in include/mpt.h).

Argument marshalling only: every step of the path (enumeration, solve,
validation, compaction, adjoint) runs in the library's CUDA kernels.  PyTorch
provides device memory and streams.  There is no CPU fallback: if the library
is not built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading

import numpy as np
import torch

from . import build as _build

P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double

MPT_OK, MPT_ERR_ARG, MPT_ERR_CUDA, MPT_ERR_CAPACITY, MPT_ERR_TIMEOUT, MPT_ERR_UNSUPPORTED = range(6)
FP64_PLAIN, FP32, FP32_FP64REFINE = 0, 1, 2
PATH_CONVERGED, PATH_MAXITER, PATH_DIVERGED, PATH_STALLED, PATH_NONFINITE, PATH_EXCLUDED = range(6)
PATH_REFINED, PATH_PRESCREENED, PATH_FALLBACK = 0x10, 0x20, 0x40
TAU = 1e-20  # acceptance threshold on the cost of Eq. 15


class SceneDesc(C.Structure):
    _fields_ = [("n_obj", I32), ("obj_kind", P), ("obj_param", P), ("n_occ", I32), ("occ_kind", P),
                ("occ_param", P), ("scale", D)]


class FieldParams(C.Structure):
    _fields_ = [("wavenumber", D), ("e0", D), ("refl", D * 2), ("diff", D * 2)]


class Endpoints(C.Structure):
    _fields_ = [("tx", P), ("n_tx", I32), ("rx", P), ("n_rx", I32), ("pair_mode", I32)]


class Sampling(C.Structure):
    _fields_ = [("quota", I64 * 4), ("seed", U64), ("starts_curved", I32), ("force_edges_every", I32)]


class CandStruct(C.Structure):
    _fields_ = [("rec", P), ("capacity", I64), ("count", P), ("order_begin", P), ("init_seed", U64)]


class SolStruct(C.Structure):
    _fields_ = [("T", P), ("cost", P), ("status", P), ("iters", P), ("evals", P), ("T32", P), ("capacity", I64)]


class Schedule(C.Structure):
    _fields_ = [("block", I32), ("blocks_per_sm", I32), ("tile", I32), ("max_iters", I32),
                ("refine_steps", I32), ("mixed_orders", I32), ("refill_min", I32), ("prescreen", I32),
                ("fallback", I32), ("warp_orders", I32),
                ("exclude", I32)]


class PathStruct(C.Structure):
    _fields_ = [("cand", P), ("X", P), ("T", P), ("length", P), ("cost", P), ("capacity", I64)]


_lib = None
_lock = threading.Lock()

# Every symbol include/mpt.h declares.
SYMBOLS = ["mpt_ctx_create", "mpt_ctx_destroy", "mpt_ctx_sm_count", "mpt_ctx_check", "mpt_scene_upload",
           "mpt_scene_free", "mpt_enumerate", "mpt_candidate_count", "mpt_solve", "mpt_validate", "mpt_grad",
           "mpt_status_string", "mpt_flop_model", "mpt_validate_noalloc", "mpt_visibility", "mpt_field",
           "mpt_ctx_selftest_wait", "mpt_image_method", "mpt_autotune", "mpt_scene_shift_planes",
           "mpt_ctx_time_solver", "mpt_ctx_solver_ms"]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmpt.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libmpt.so is not built ({path}); run __graft_entry__.build()")
            L = C.CDLL(path)
            L.mpt_ctx_create.argtypes = [C.c_int, C.POINTER(P)]
            L.mpt_ctx_destroy.argtypes = [P]
            L.mpt_ctx_sm_count.argtypes = [P]
            L.mpt_ctx_check.argtypes = [P, P]
            L.mpt_ctx_selftest_wait.argtypes = [P, P]
            L.mpt_ctx_time_solver.argtypes = [P, C.c_int]
            L.mpt_ctx_solver_ms.argtypes = [P, C.c_int, C.POINTER(C.c_float)]
            L.mpt_scene_upload.argtypes = [P, C.POINTER(SceneDesc), C.POINTER(P)]
            L.mpt_scene_free.argtypes = [P]
            L.mpt_enumerate.argtypes = [P, P, C.POINTER(Endpoints), C.c_int, P, C.POINTER(Sampling),
                                        C.POINTER(CandStruct), P]
            L.mpt_visibility.argtypes = [P, P, P, P]
            L.mpt_field.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct), C.POINTER(PathStruct), P,
                                    C.POINTER(FieldParams), P, P]
            L.mpt_candidate_count.restype = I64
            L.mpt_candidate_count.argtypes = [P, C.POINTER(Endpoints), C.c_int, C.POINTER(Sampling)]
            L.mpt_solve.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct), C.c_int,
                                    C.POINTER(Schedule), C.POINTER(SolStruct), P]
            L.mpt_scene_shift_planes.argtypes = [P, P, P, P, P]
            L.mpt_autotune.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct), C.c_int,
                                       C.POINTER(SolStruct), C.POINTER(Schedule), C.POINTER(D), P]
            L.mpt_image_method.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct), C.POINTER(SolStruct),
                                           P]
            L.mpt_validate.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct), C.POINTER(SolStruct),
                                       D, C.POINTER(PathStruct), P, P]
            L.mpt_validate_noalloc.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct),
                                               C.POINTER(SolStruct), D, C.POINTER(PathStruct), P, P]
            L.mpt_grad.argtypes = [P, P, C.POINTER(Endpoints), C.POINTER(CandStruct), C.POINTER(PathStruct), P,
                                   P, P, P, P, P, P]
            L.mpt_status_string.restype = C.c_char_p
            L.mpt_status_string.argtypes = [C.c_int]
            L.mpt_flop_model.argtypes = [C.c_int, P, C.POINTER(D), C.POINTER(D), C.POINTER(D)]
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != MPT_OK:
        msg = lib().mpt_status_string(rc).decode()
        raise RuntimeError(f"{what}: {msg}")


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def status_string(rc: int) -> str:
    return lib().mpt_status_string(rc).decode()


def flop_model(kinds) -> tuple[float, float, float]:
    """(flops per Cholesky+solve, flops per evaluation, SFU ops per evaluation)."""
    k = np.ascontiguousarray(np.asarray(kinds, np.int32))
    fi, fe, sf = D(), D(), D()
    _check(lib().mpt_flop_model(len(k), k.ctypes.data_as(P), C.byref(fi), C.byref(fe), C.byref(sf)),
           "mpt_flop_model")
    return fi.value, fe.value, sf.value


class Context:
    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libmpt needs a CUDA GPU")
        self.device = device
        h = P()
        _check(lib().mpt_ctx_create(device, C.byref(h)), "mpt_ctx_create")
        self.h = h

    @property
    def sm_count(self) -> int:
        return int(lib().mpt_ctx_sm_count(self.h))

    def check(self, stream=None) -> int:
        return int(lib().mpt_ctx_check(self.h, _stream(stream)))

    def time_solver(self, on: bool) -> None:
        """mpt_ctx_time_solver: record events around each order's solver launch."""
        _check(lib().mpt_ctx_time_solver(self.h, 1 if on else 0), "mpt_ctx_time_solver")

    def solver_ms(self, order: int) -> float:
        """mpt_ctx_solver_ms: milliseconds of the last timed solver launch of `order`."""
        ms = C.c_float()
        _check(lib().mpt_ctx_solver_ms(self.h, order, C.byref(ms)), "mpt_ctx_solver_ms")
        return float(ms.value)

    def selftest_wait(self, stream=None) -> int:
        """Enqueue the bounded-wait self-test (mpt_ctx_selftest_wait)."""
        return int(lib().mpt_ctx_selftest_wait(self.h, _stream(stream)))

    def close(self):
        if self.h:
            lib().mpt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceScene:
    """A scene uploaded with mpt_scene_upload plus its TX/RX endpoints on the device."""

    def __init__(self, ctx: Context, scene, device: int | None = None, tx_host: torch.Tensor | None = None,
                 rx_host: torch.Tensor | None = None):
        self.ctx = ctx
        self.scene = scene.contiguous()
        s = self.scene
        desc = SceneDesc(s.n_obj, s.obj_kind.ctypes.data, s.obj_param.ctypes.data, s.n_occ,
                         s.occ_kind.ctypes.data if s.n_occ else None,
                         s.occ_param.ctypes.data if s.n_occ else None, s.scale)
        h = P()
        _check(lib().mpt_scene_upload(ctx.h, C.byref(desc), C.byref(h)), "mpt_scene_upload")
        self.h = h
        dev = torch.device("cuda", ctx.device if device is None else device)
        src_tx = tx_host if tx_host is not None else torch.as_tensor(s.tx, dtype=torch.float64)
        src_rx = rx_host if rx_host is not None else torch.as_tensor(s.rx, dtype=torch.float64)
        self.tx = src_tx.to(dev, non_blocking=True).contiguous()
        self.rx = src_rx.to(dev, non_blocking=True).contiguous()
        self.pair_mode = s.pair_mode

    def endpoints(self) -> Endpoints:
        return Endpoints(self.tx.data_ptr(), self.tx.shape[0], self.rx.data_ptr(), self.rx.shape[0], self.pair_mode)

    @property
    def n_pairs(self) -> int:
        return self.scene.n_pairs

    def free(self):
        if self.h:
            lib().mpt_scene_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class SceneView:
    """A scene already on the device with caller-provided device endpoints
    (float64 [n, 3] tensors, used in place): what the calls need of a
    DeviceScene, without copies."""

    def __init__(self, ctx: Context, scene, handle, tx: torch.Tensor, rx: torch.Tensor):
        self.ctx = ctx
        self.scene = scene
        self.h = handle
        self.tx = tx
        self.rx = rx
        self.pair_mode = scene.pair_mode

    def endpoints(self) -> Endpoints:
        return Endpoints(self.tx.data_ptr(), self.tx.shape[0], self.rx.data_ptr(), self.rx.shape[0], self.pair_mode)

    @property
    def n_pairs(self) -> int:
        return self.tx.shape[0] * self.rx.shape[0] if self.pair_mode == 0 else self.tx.shape[0]


def shift_planes(base: DeviceScene, dst: DeviceScene, delta: torch.Tensor, stream=None) -> None:
    """mpt_scene_shift_planes: dst <- base with plane i moved by delta[i]
    (device float64 [n_obj]) along its normal."""
    d = delta.detach().to(device=base.tx.device, dtype=torch.float64).contiguous()
    if stream is not None and d.data_ptr() != delta.data_ptr():
        d.record_stream(stream)  # a converted copy lives until the launch has read it
    _check(lib().mpt_scene_shift_planes(base.ctx.h, base.h, dst.h, C.c_void_p(d.data_ptr()), _stream(stream)),
           "mpt_scene_shift_planes")


def sampling_struct(spec) -> Sampling:
    q = list(spec.quota) + [0] * (4 - len(spec.quota))
    return Sampling((I64 * 4)(*q[:4]), spec.seed, spec.starts_curved, spec.force_edges_every)


@dataclasses.dataclass
class Candidates:
    rec: torch.Tensor  # int32 [cap, 4] (16-byte records)
    count: torch.Tensor  # int64 [1]
    order_begin: torch.Tensor  # int64 [5]
    capacity: int
    init_seed: int = 0

    def struct(self) -> CandStruct:
        return CandStruct(self.rec.data_ptr(), self.capacity, self.count.data_ptr(), self.order_begin.data_ptr(),
                          self.init_seed)


def candidate_count(ds: DeviceScene, max_order: int, spec) -> int:
    ep = ds.endpoints()
    sp = sampling_struct(spec)
    n = lib().mpt_candidate_count(ds.h, C.byref(ep), max_order, C.byref(sp))
    if n < 0:
        raise RuntimeError("mpt_candidate_count: bad arguments")
    return int(n)


def alloc_candidates(capacity: int, device, init_seed: int = 0) -> Candidates:
    cap = max(int(capacity), 1)
    return Candidates(torch.empty((cap, 4), dtype=torch.int32, device=device),
                      torch.zeros(1, dtype=torch.int64, device=device),
                      torch.zeros(5, dtype=torch.int64, device=device), cap, init_seed)


def visibility(ds: DeviceScene, stream=None) -> torch.Tensor:
    """Visibility matrix V (uint8 [n_obj, n_obj] on the scene's device), usable
    as the adjacency mask of enumerate_candidates."""
    n = ds.scene.n_obj
    V = torch.empty((n, n), dtype=torch.uint8, device=ds.tx.device)
    _check(lib().mpt_visibility(ds.ctx.h, ds.h, C.c_void_p(V.data_ptr()), _stream(stream)), "mpt_visibility")
    return V


def enumerate_candidates(ds: DeviceScene, max_order: int, spec, adj: torch.Tensor | None = None,
                         capacity: int | None = None, init_seed: int = 0, out: Candidates | None = None,
                         stream=None) -> Candidates:
    if out is not None:
        c = out
    else:
        if capacity is None:
            capacity = candidate_count(ds, max_order, spec)
        c = alloc_candidates(capacity, ds.tx.device, init_seed)
    ep = ds.endpoints()
    sp = sampling_struct(spec)
    cs = c.struct()
    _check(lib().mpt_enumerate(ds.ctx.h, ds.h, C.byref(ep), max_order, _ptr(adj), C.byref(sp), C.byref(cs),
                               _stream(stream)), "mpt_enumerate")
    return c


@dataclasses.dataclass
class Solutions:
    T: torch.Tensor  # float64 [8, cap]
    cost: torch.Tensor  # float64 [cap]
    status: torch.Tensor  # uint8 [cap]
    iters: torch.Tensor  # uint8 [cap]
    evals: torch.Tensor  # uint8 [cap]
    T32: torch.Tensor | None
    capacity: int

    def struct(self) -> SolStruct:
        return SolStruct(self.T.data_ptr(), self.cost.data_ptr(), self.status.data_ptr(), self.iters.data_ptr(),
                         self.evals.data_ptr(), self.T32.data_ptr() if self.T32 is not None else None,
                         self.capacity)


def alloc_solutions(capacity: int, device, keep_fp32: bool = False) -> Solutions:
    cap = max(int(capacity), 1)
    return Solutions(torch.zeros((8, cap), dtype=torch.float64, device=device),
                     torch.zeros(cap, dtype=torch.float64, device=device),
                     torch.zeros(cap, dtype=torch.uint8, device=device),
                     torch.zeros(cap, dtype=torch.uint8, device=device),
                     torch.zeros(cap, dtype=torch.uint8, device=device),
                     torch.zeros((8, cap), dtype=torch.float32, device=device) if keep_fp32 else None, cap)


def schedule_struct(block=128, blocks_per_sm=0, tile=0, max_iters=0, refine_steps=0, mixed_orders=0,
                    refill_min=0, prescreen=0, fallback=0, warp_orders=0, exclude=0) -> Schedule:
    return Schedule(block, blocks_per_sm, tile, max_iters, refine_steps, mixed_orders, refill_min, prescreen,
                    fallback, warp_orders, exclude)


def solve(ds: DeviceScene, cands: Candidates, precision: int = FP32_FP64REFINE, schedule: Schedule | None = None,
          out: Solutions | None = None, keep_fp32: bool = False, stream=None) -> Solutions:
    if out is None:
        out = alloc_solutions(cands.capacity, ds.tx.device, keep_fp32)
    ep = ds.endpoints()
    cs = cands.struct()
    ss = out.struct()
    _check(lib().mpt_solve(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), precision,
                           C.byref(schedule) if schedule is not None else None, C.byref(ss), _stream(stream)),
           "mpt_solve")
    return out


def autotune(ds: DeviceScene, cands: Candidates, precision: int = FP32_FP64REFINE, out: Solutions | None = None,
             stream=None) -> tuple[Schedule, float]:
    """mpt_autotune: the fastest schedule of mpt_solve for this workload and
    its time (ms); cached in the context by workload signature."""
    if out is None:
        out = alloc_solutions(cands.capacity, ds.tx.device)
    ep = ds.endpoints()
    cs = cands.struct()
    ss = out.struct()
    best = Schedule()
    ms = D()
    _check(lib().mpt_autotune(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), precision, C.byref(ss), C.byref(best),
                              C.byref(ms), _stream(stream)), "mpt_autotune")
    return best, ms.value


def schedule_dict(s: Schedule) -> dict:
    return {name: getattr(s, name) for name, _ in Schedule._fields_}


def image_method(ds: DeviceScene, cands: Candidates, out: Solutions | None = None, stream=None) -> Solutions:
    """Image method (Sec. III-A, Eqs. 5-6) for the reflection-only planar
    candidates, in the layout of solve(); validate() applies bounds and
    visibility."""
    if out is None:
        out = alloc_solutions(cands.capacity, ds.tx.device)
    ep = ds.endpoints()
    cs = cands.struct()
    ss = out.struct()
    _check(lib().mpt_image_method(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), C.byref(ss), _stream(stream)),
           "mpt_image_method")
    return out


@dataclasses.dataclass
class Paths:
    cand: torch.Tensor  # int64 [cap]
    X: torch.Tensor  # float64 [12, cap]
    T: torch.Tensor  # float64 [8, cap]
    length: torch.Tensor  # float64 [cap]
    cost: torch.Tensor  # float64 [cap]
    count: torch.Tensor  # int64 [1] (device)
    capacity: int

    def struct(self) -> PathStruct:
        return PathStruct(self.cand.data_ptr(), self.X.data_ptr(), self.T.data_ptr(), self.length.data_ptr(),
                          self.cost.data_ptr(), self.capacity)

    def n(self) -> int:
        return min(int(self.count.item()), self.capacity)


def alloc_paths(capacity: int, device) -> Paths:
    cap = max(int(capacity), 1)
    return Paths(torch.zeros(cap, dtype=torch.int64, device=device),
                 torch.zeros((12, cap), dtype=torch.float64, device=device),
                 torch.zeros((8, cap), dtype=torch.float64, device=device),
                 torch.zeros(cap, dtype=torch.float64, device=device),
                 torch.zeros(cap, dtype=torch.float64, device=device),
                 torch.zeros(1, dtype=torch.int64, device=device), cap)


def validate(ds: DeviceScene, cands: Candidates, sols: Solutions, tau: float = TAU, capacity: int | None = None,
             out: Paths | None = None, stream=None) -> Paths:
    if out is None:
        out = alloc_paths(capacity if capacity is not None else max(cands.capacity // 64, 1024), ds.tx.device)
    ep = ds.endpoints()
    cs = cands.struct()
    ss = sols.struct()
    ps = out.struct()
    _check(lib().mpt_validate(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), C.byref(ss), tau, C.byref(ps),
                              _ptr(out.count), _stream(stream)), "mpt_validate")
    return out


def field(ds: DeviceScene, cands: Candidates, paths: Paths, wavenumber: float, e0: float = 1.0,
          refl: complex = -1.0, diff: complex = 1.0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Received field per TX/RX pair (float64 [n_pairs, 2] = re, im), added into `out`."""
    if out is None:
        out = torch.zeros((ds.n_pairs, 2), dtype=torch.float64, device=ds.tx.device)
    fp = FieldParams(float(wavenumber), float(e0), (D * 2)(complex(refl).real, complex(refl).imag),
                     (D * 2)(complex(diff).real, complex(diff).imag))
    ep = ds.endpoints()
    cs = cands.struct()
    ps = paths.struct()
    _check(lib().mpt_field(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), C.byref(ps), C.c_void_p(paths.count.data_ptr()),
                           C.byref(fp), C.c_void_p(out.data_ptr()), _stream(stream)), "mpt_field")
    return out


def grad(ds: DeviceScene, cands: Candidates, paths: Paths, g_len: torch.Tensor, g_pts: torch.Tensor | None = None,
         g_tx: torch.Tensor | None = None, g_rx: torch.Tensor | None = None, g_obj: torch.Tensor | None = None,
         stream=None):
    """Accumulates d(sum g_len * L + g_pts . X)/d theta into g_tx [n_tx,3], g_rx [n_rx,3], g_obj [n_obj]."""
    dev = ds.tx.device
    if g_tx is None:
        g_tx = torch.zeros_like(ds.tx)
    if g_rx is None:
        g_rx = torch.zeros_like(ds.rx)
    if g_obj is None:
        g_obj = torch.zeros(ds.scene.n_obj, dtype=torch.float64, device=dev)
    ep = ds.endpoints()
    cs = cands.struct()
    ps = paths.struct()
    _check(lib().mpt_grad(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), C.byref(ps), _ptr(paths.count),
                          _ptr(g_len.contiguous()), _ptr(g_pts.contiguous() if g_pts is not None else None),
                          _ptr(g_tx), _ptr(g_rx), _ptr(g_obj), _stream(stream)), "mpt_grad")
    return g_tx, g_rx, g_obj


def decode_candidates(cands: Candidates, n: int | None = None):
    """Host decode of candidate records: (pair, ids[., 4] with -1, order, start)."""
    r = cands.rec[: (n if n is not None else cands.capacity)].cpu().numpy().view(np.uint32)
    pair = r[:, 0].astype(np.int64)
    ids = np.stack([r[:, 1] & 0xFFFF, r[:, 1] >> 16, r[:, 2] & 0xFFFF, r[:, 2] >> 16], 1).astype(np.int64)
    ids[ids == 0xFFFF] = -1
    order = (r[:, 3] & 0xFF).astype(np.int64)
    start = ((r[:, 3] >> 8) & 0xFF).astype(np.int64)
    return pair, ids, order, start


@dataclasses.dataclass
class TraceResult:
    cands: Candidates
    sols: Solutions
    paths: Paths


def trace(ds: DeviceScene, max_order: int, spec, precision: int = FP32_FP64REFINE, tau: float = TAU,
          path_capacity: int | None = None, schedule: Schedule | None = None, init_seed: int = 0,
          keep_fp32: bool = False, stream=None) -> TraceResult:
    """Algorithm 1 on the GPU: enumerate, solve, validate (compacted valid paths)."""
    cands = enumerate_candidates(ds, max_order, spec, init_seed=init_seed, stream=stream)
    sols = solve(ds, cands, precision, schedule, keep_fp32=keep_fp32, stream=stream)
    paths = validate(ds, cands, sols, tau, capacity=path_capacity, stream=stream)
    return TraceResult(cands, sols, paths)
