"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every function of the C library is exposed under its own name
(``lbm_create``, ``lbm_step`` ...), plus a small ``Lattice`` convenience class
that owns a context.  Device memory for results may be PyTorch CUDA tensors
(pass ``on_device=True`` and a tensor); the library's own stream can be
replaced by a PyTorch stream through ``stream=``.  No step of the method runs
in Python: if the CUDA library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = range(7)
LBM_PERIODIC, LBM_WALL, LBM_OPEN = 0, 1, 2
LBM_FP64, LBM_FP32_DEV, LBM_FP16_DEV = 0, 1, 2
LBM_RHOW_CONST, LBM_RHOW_LOCAL = 0, 1
LBM_REFILL_A1, LBM_REFILL_A2, LBM_REFILL_A3 = 1, 2, 3
LBM_PRESCRIBED, LBM_FREE = 0, 1
LBM_CME, LBM_GME = 0, 1
LBM_BGK, LBM_MRT = 0, 1
LBM_HALFWAY, LBM_INTERPOLATED = 0, 1

PRECISION_NAMES = {"fp64": LBM_FP64, "fp32": LBM_FP32_DEV, "fp16": LBM_FP16_DEV}


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


class lbm_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("u0", ctypes.c_double * 2), ("wall_ux", ctypes.c_double * 2),
        ("body_force", ctypes.c_double * 2), ("inflow_umax", ctypes.c_double),
        ("gravity", ctypes.c_double * 2), ("lub_range", ctypes.c_double),
        ("precision", ctypes.c_int32), ("rho_w_mode", ctypes.c_int32),
        ("refill", ctypes.c_int32), ("force_ring", ctypes.c_int32),
        ("device", ctypes.c_int32), ("motion_cme", ctypes.c_int32),
        ("relative_changes", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


class lbm_unet_config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("base", ctypes.c_int32), ("height", ctypes.c_int32),
                ("width", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("device", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p)]


class lbm_disk(ctypes.Structure):
    _fields_ = [
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("r", ctypes.c_double),
        ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("omega", ctypes.c_double),
        ("rho_s", ctypes.c_double), ("motion", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

_SIGNATURES = {
    "lbm_config_default": (None, [ctypes.POINTER(lbm_config)]),
    "lbm_create": (_I32, [ctypes.POINTER(lbm_config), ctypes.POINTER(_P)]),
    "lbm_destroy": (_I32, [_P]),
    "lbm_add_solid": (_I32, [_P, ctypes.POINTER(lbm_disk), ctypes.POINTER(_I32)]),
    "lbm_step": (_I32, [_P, _I64]),
    "lbm_sync": (_I32, [_P]),
    "lbm_forces": (_I32, [_P, _I32, _I64, _I64, _P, _I32]),
    "lbm_fields": (_I32, [_P, _P, _P, _P, _I32]),
    "lbm_fields_static": (_I32, [_P, _P, _P, _P]),
    "lbm_get_populations": (_I32, [_P, _P, _I32]),
    "lbm_set_populations": (_I32, [_P, _P, _I32]),
    "lbm_get_owner": (_I32, [_P, _P, _I32]),
    "lbm_get_solids": (_I32, [_P, _D]),
    "lbm_set_solid": (_I32, [_P, _I32, _D]),
    "lbm_links": (_I32, [_P, _I64, _P, ctypes.POINTER(_I64)]),
    "lbm_time": (_I64, [_P]),
    "lbm_nsolid": (_I32, [_P]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_status_string": (ctypes.c_char_p, [_I32]),
    "lbm_set_graph": (_I32, [_P, _I32]),
    "lbm_set_wait_limit": (_I32, [_P, _I64]),
    "lbm_set_force_overlap": (_I32, [_P, _I32]),
    "lbm_force_overlap": (_I32, [_P]),
    "lbm_state_size": (_I32, [_P, ctypes.POINTER(_I64)]),
    "lbm_save": (_I32, [_P, _P, _I64]),
    "lbm_load": (_I32, [_P, _P, _I64]),
    "lbm_set_timing": (_I32, [_P, _I32]),
    "lbm_get_timing": (_I32, [_P, _D, ctypes.POINTER(_I64)]),
    "lbm_launch_count": (_I64, [_P]),
    "lbm_set_kernel_variant": (_I32, [_P, _I32]),
    "lbm_kernel_variant": (_I32, [_P]),
    "lbm_autotune": (_I32, [_P, _I32, ctypes.POINTER(_I32)]),
    "lbm_batch_create": (_I32, [ctypes.POINTER(lbm_config), _I32, ctypes.POINTER(_P)]),
    "lbm_batch_destroy": (_I32, [_P]),
    "lbm_batch_size": (_I32, [_P]),
    "lbm_batch_case": (_I32, [_P, _I32, ctypes.POINTER(_P)]),
    "lbm_batch_add_solid": (_I32, [_P, _I32, ctypes.POINTER(lbm_disk), ctypes.POINTER(_I32)]),
    "lbm_batch_set_convergence": (_I32, [_P, _I32, ctypes.c_double, _I64]),
    "lbm_batch_set_convergence_window": (_I32, [_P, _I32]),
    "lbm_batch_run": (_I32, [_P, _I64, ctypes.POINTER(_I32)]),
    "lbm_batch_state": (_I32, [_P, _P, _P, _P]),
    "lbm_batch_retire": (_I32, [_P, _P, _I32]),
    "lbm_batch_set_launch": (_I32, [_P, _I32, _I32, _I32, _I32]),
    "lbm_batch_get_launch": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                    ctypes.POINTER(_I32)]),
    "lbm_batch_autotune": (_I32, [_P, _I32, _P]),
    "lbm_batch_set_timing": (_I32, [_P, _I32]),
    "lbm_batch_get_timing": (_I32, [_P, _D, ctypes.POINTER(_I64)]),
    "lbm_batch_launch_count": (_I64, [_P]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_unet_create": (_I32, [ctypes.POINTER(lbm_unet_config), ctypes.POINTER(_P)]),
    "lbm_unet_destroy": (_I32, [_P]),
    "lbm_unet_set_wait_limit": (_I32, [_P, _I64]),
    "lbm_unet_last_error": (ctypes.c_char_p, [_P]),
    "lbm_unet_param_count": (_I64, [_P]),
    "lbm_unet_get_params": (_I32, [_P, _P, _I32]),
    "lbm_unet_set_params": (_I32, [_P, _P, _I32]),
    "lbm_unet_forward": (_I32, [_P, _P, _P, _I32, _I32]),
    "lbm_unet_gradients": (_I32, [_P, _P, _P, _P, _I32, _P, _D, _I32]),
    "lbm_unet_train_step": (_I32, [_P, _P, _P, _P, _I32, ctypes.c_float, _D, _I32]),
    "lbm_unet_input": (_I32, [_P, _P, ctypes.c_double, _P]),
    "lbm_case_input": (_I32, [_P, ctypes.c_double, _P]),
    "lbm_warm_start": (_I32, [_P, _P, ctypes.c_double, ctypes.c_double, _I32]),
}


def header_symbols() -> list[str]:
    """Names of the functions declared in include/lbm.h and include/lbm_nn.h."""
    out = []
    for name in ("lbm.h", "lbm_nn.h"):
        with open(os.path.join(_build.INCLUDE, name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        out += re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)
    return out


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm_gb300.so (building it first if needed); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run the build first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, ctx=None):
    if st != LBM_OK:
        lib = load()
        msg = lib.lbm_last_error(ctx).decode() if lib.lbm_last_error(ctx) else ""
        raise LBMError(st, msg or lib.lbm_status_string(st).decode())


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


# ------------------------------------------------ same-name thin wrappers

def lbm_config_default() -> lbm_config:
    c = lbm_config()
    load().lbm_config_default(ctypes.byref(c))
    return c


def lbm_create(cfg: lbm_config):
    h = _P()
    _check(load().lbm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lbm_destroy(ctx):
    _check(load().lbm_destroy(ctx))


def lbm_add_solid(ctx, disk: lbm_disk) -> int:
    out = _I32()
    _check(load().lbm_add_solid(ctx, ctypes.byref(disk), ctypes.byref(out)), ctx)
    return int(out.value)


def lbm_step(ctx, n: int):
    _check(load().lbm_step(ctx, int(n)), ctx)


def lbm_sync(ctx):
    _check(load().lbm_sync(ctx), ctx)


def lbm_forces(ctx, form: int, first: int, count: int, out, on_device: bool = False):
    _check(load().lbm_forces(ctx, int(form), int(first), int(count), _ptr(out), int(on_device)), ctx)


def lbm_fields(ctx, rho, ux, uy, on_device: bool = False):
    _check(load().lbm_fields(ctx, _ptr(rho), _ptr(ux), _ptr(uy), int(on_device)), ctx)


def lbm_fields_static(ctx, rho, ux, uy):
    """lbm_fields into host arrays without any device allocation (see lbm.h)."""
    _check(load().lbm_fields_static(ctx, _ptr(rho), _ptr(ux), _ptr(uy)), ctx)


LBM_FIELDS_STATIC_MAX_NODES = 524288


def lbm_get_populations(ctx, f, on_device: bool = False):
    _check(load().lbm_get_populations(ctx, _ptr(f), int(on_device)), ctx)


def lbm_set_populations(ctx, f, on_device: bool = False):
    _check(load().lbm_set_populations(ctx, _ptr(f), int(on_device)), ctx)


def lbm_get_owner(ctx, owner, on_device: bool = False):
    _check(load().lbm_get_owner(ctx, _ptr(owner), int(on_device)), ctx)


def lbm_get_solids(ctx, out: np.ndarray):
    _check(load().lbm_get_solids(ctx, out.ctypes.data_as(_D)), ctx)


def lbm_set_solid(ctx, sid: int, state):
    st = np.ascontiguousarray(state, dtype=np.float64)
    _check(load().lbm_set_solid(ctx, int(sid), st.ctypes.data_as(_D)), ctx)


def lbm_links(ctx, cap: int, out) -> int:
    n = _I64()
    _check(load().lbm_links(ctx, int(cap), _ptr(out) if cap else None, ctypes.byref(n)), ctx)
    return int(n.value)


def lbm_time(ctx) -> int:
    return int(load().lbm_time(ctx))


def lbm_nsolid(ctx) -> int:
    return int(load().lbm_nsolid(ctx))


def lbm_last_error(ctx=None) -> str:
    r = load().lbm_last_error(ctx)
    return r.decode() if r else ""


def lbm_status_string(st: int) -> str:
    return load().lbm_status_string(int(st)).decode()


def lbm_set_graph(ctx, steps: int):
    _check(load().lbm_set_graph(ctx, int(steps)), ctx)


def lbm_set_force_overlap(ctx, on: bool):
    _check(load().lbm_set_force_overlap(ctx, int(bool(on))), ctx)


def lbm_force_overlap(ctx) -> int:
    return load().lbm_force_overlap(ctx)


def lbm_set_wait_limit(ctx, polls: int):
    _check(load().lbm_set_wait_limit(ctx, int(polls)), ctx)


def lbm_state_size(ctx) -> int:
    n = _I64()
    _check(load().lbm_state_size(ctx, ctypes.byref(n)), ctx)
    return n.value


def lbm_save(ctx, buf):
    """Save the context's state into buf (a writable host array of uint8)."""
    _check(load().lbm_save(ctx, _ptr(buf), int(buf.nbytes)), ctx)


def lbm_load(ctx, buf):
    _check(load().lbm_load(ctx, _ptr(buf), int(buf.nbytes)), ctx)


def lbm_set_timing(ctx, enable: bool):
    _check(load().lbm_set_timing(ctx, int(bool(enable))), ctx)


def lbm_get_timing(ctx):
    ms = ctypes.c_double()
    n = _I64()
    _check(load().lbm_get_timing(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return float(ms.value), int(n.value)


def lbm_launch_count(ctx) -> int:
    return int(load().lbm_launch_count(ctx))


def lbm_set_kernel_variant(ctx, variant: int):
    _check(load().lbm_set_kernel_variant(ctx, int(variant)), ctx)


def lbm_kernel_variant(ctx) -> int:
    return int(load().lbm_kernel_variant(ctx))


def lbm_autotune(ctx, steps: int = 4) -> int:
    best = _I32()
    _check(load().lbm_autotune(ctx, int(steps), ctypes.byref(best)), ctx)
    return int(best.value)


# ------------------------------------------------------------- batches

LBM_CASE_ACTIVE, LBM_CASE_CONVERGED, LBM_CASE_CAPPED, LBM_CASE_UNSTABLE = range(4)


def _bcheck(st: int, b=None):
    if st != LBM_OK:
        lib = load()
        r = lib.lbm_batch_last_error(b)
        raise LBMError(st, (r.decode() if r else "") or lib.lbm_status_string(st).decode())


def lbm_batch_create(configs) -> ctypes.c_void_p:
    arr = (lbm_config * len(configs))(*configs)
    h = _P()
    _bcheck(load().lbm_batch_create(arr, len(configs), ctypes.byref(h)))
    return h


def lbm_batch_destroy(b):
    _bcheck(load().lbm_batch_destroy(b), b)


def lbm_batch_size(b) -> int:
    return int(load().lbm_batch_size(b))


def lbm_batch_case(b, k: int):
    h = _P()
    _bcheck(load().lbm_batch_case(b, int(k), ctypes.byref(h)), b)
    return h


def lbm_batch_add_solid(b, k: int, disk: lbm_disk) -> int:
    out = _I32()
    _bcheck(load().lbm_batch_add_solid(b, int(k), ctypes.byref(disk), ctypes.byref(out)), b)
    return int(out.value)


def lbm_batch_set_convergence(b, every: int, tol: float, max_steps: int):
    _bcheck(load().lbm_batch_set_convergence(b, int(every), float(tol), int(max_steps)), b)


def lbm_batch_set_convergence_window(b, tests: int):
    _bcheck(load().lbm_batch_set_convergence_window(b, int(tests)), b)


def lbm_batch_run(b, steps: int) -> int:
    na = _I32()
    _bcheck(load().lbm_batch_run(b, int(steps), ctypes.byref(na)), b)
    return int(na.value)


def lbm_batch_state(b, state, steps, drag):
    _bcheck(load().lbm_batch_state(b, _ptr(state), _ptr(steps), _ptr(drag)), b)


def lbm_batch_retire(b, ids):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    _bcheck(load().lbm_batch_retire(b, _ptr(ids) if ids.size else None, int(ids.size)), b)


def lbm_batch_set_launch(b, variant: int, tile_rows: int = 1, persistent: bool = False,
                         graph: bool = True):
    _bcheck(load().lbm_batch_set_launch(b, int(variant), int(tile_rows), int(bool(persistent)),
                                        int(bool(graph))), b)


def lbm_batch_get_launch(b):
    """(variant, tile_rows, persistent)"""
    v, h, p = _I32(), _I32(), _I32()
    _bcheck(load().lbm_batch_get_launch(b, ctypes.byref(v), ctypes.byref(h), ctypes.byref(p)), b)
    return int(v.value), int(h.value), int(p.value)


LBM_BATCH_TUNE_SHAPES = 10


def lbm_batch_autotune(b, steps: int = 4):
    """Fastest (variant, tile_rows, persistent); see lbm.h."""
    best = np.zeros(3, dtype=np.int32)
    _bcheck(load().lbm_batch_autotune(b, int(steps), _ptr(best)), b)
    return int(best[0]), int(best[1]), int(best[2])


def lbm_batch_set_timing(b, enable: bool):
    _bcheck(load().lbm_batch_set_timing(b, int(bool(enable))), b)


def lbm_batch_get_timing(b):
    ms = ctypes.c_double()
    n = _I64()
    _bcheck(load().lbm_batch_get_timing(b, ctypes.byref(ms), ctypes.byref(n)), b)
    return float(ms.value), int(n.value)


def lbm_batch_launch_count(b) -> int:
    return int(load().lbm_batch_launch_count(b))


def lbm_batch_last_error(b=None) -> str:
    r = load().lbm_batch_last_error(b)
    return r.decode() if r else ""


# ------------------------------------------------------ warm-start net

def _ncheck(st: int, net=None):
    if st != LBM_OK:
        lib = load()
        r = lib.lbm_unet_last_error(net)
        raise LBMError(st, (r.decode() if r else "") or lib.lbm_status_string(st).decode())


def lbm_unet_create(cfg: lbm_unet_config):
    h = _P()
    _ncheck(load().lbm_unet_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lbm_unet_destroy(net):
    _ncheck(load().lbm_unet_destroy(net), net)


def lbm_unet_set_wait_limit(net, polls: int):
    _ncheck(load().lbm_unet_set_wait_limit(net, int(polls)), net)


def lbm_unet_param_count(net) -> int:
    return int(load().lbm_unet_param_count(net))


def lbm_unet_get_params(net, out, on_device: bool = False):
    _ncheck(load().lbm_unet_get_params(net, _ptr(out), int(on_device)), net)


def lbm_unet_set_params(net, params, on_device: bool = False):
    _ncheck(load().lbm_unet_set_params(net, _ptr(params), int(on_device)), net)


def lbm_unet_forward(net, x, out, batch: int, on_device: bool = False):
    _ncheck(load().lbm_unet_forward(net, _ptr(x), _ptr(out), int(batch), int(on_device)), net)


def lbm_unet_gradients(net, x, target, fluid, batch: int, grads, on_device: bool = False) -> float:
    loss = ctypes.c_double()
    _ncheck(load().lbm_unet_gradients(net, _ptr(x), _ptr(target), _ptr(fluid), int(batch),
                                      _ptr(grads), ctypes.byref(loss), int(on_device)), net)
    return float(loss.value)


def lbm_unet_train_step(net, x, target, fluid, batch: int, lr: float, on_device: bool = False) -> float:
    loss = ctypes.c_double()
    _ncheck(load().lbm_unet_train_step(net, _ptr(x), _ptr(target), _ptr(fluid), int(batch),
                                       float(lr), ctypes.byref(loss), int(on_device)), net)
    return float(loss.value)


def lbm_case_input(ctx, reynolds: float, in_dev):
    """Network input [8][ny][nx] of the case held by ctx (device tensor)."""
    _check(load().lbm_case_input(ctx, float(reynolds), _ptr(in_dev)), ctx)


def lbm_unet_input(net, owner_dev, reynolds: float, in_dev):
    _ncheck(load().lbm_unet_input(net, _ptr(owner_dev), float(reynolds), _ptr(in_dev)), net)


LBM_WS_BASE, LBM_WS_FLUX = 1, 2


def lbm_warm_start(ctx, prediction_dev, u_scale: float, rho_scale: float, base: bool = False,
                   flux: bool = False):
    flags = (LBM_WS_BASE if base else 0) | (LBM_WS_FLUX if flux else 0)
    _check(load().lbm_warm_start(ctx, _ptr(prediction_dev), float(u_scale), float(rho_scale),
                                 flags), ctx)


class UNet:
    """Owns an lbm_unet (see include/lbm_nn.h)."""

    def __init__(self, height, width, *, levels=4, base=32, max_batch=8, seed=0, device=0,
                 stream=None):
        self.cfg = lbm_unet_config(levels=levels, base=base, height=height, width=width,
                                   max_batch=max_batch, device=device, seed=seed, stream=stream)
        self.levels, self.base, self.H, self.W = levels, base, height, width
        self.max_batch = max_batch
        self._h = lbm_unet_create(self.cfg)

    def close(self):
        if getattr(self, "_h", None):
            lbm_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def nparam(self) -> int:
        return lbm_unet_param_count(self._h)

    def set_wait_limit(self, polls: int):
        lbm_unet_set_wait_limit(self._h, polls)

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        lbm_unet_get_params(self._h, out)
        return out

    def set_params(self, p):
        lbm_unet_set_params(self._h, np.ascontiguousarray(p, dtype=np.float32))

    def forward(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty((x.shape[0], 3, self.H, self.W), dtype=np.float32)
        lbm_unet_forward(self._h, x, out, x.shape[0])
        return out

    def gradients(self, x, target, fluid):
        x = np.ascontiguousarray(x, dtype=np.float32)
        g = np.empty(self.nparam, dtype=np.float32)
        loss = lbm_unet_gradients(self._h, x, np.ascontiguousarray(target, dtype=np.float32),
                                  np.ascontiguousarray(fluid, dtype=np.float32), x.shape[0], g)
        return loss, g

    def train_step(self, x, target, fluid, lr, on_device=False) -> float:
        if not on_device:
            x = np.ascontiguousarray(x, dtype=np.float32)
            target = np.ascontiguousarray(target, dtype=np.float32)
            fluid = np.ascontiguousarray(fluid, dtype=np.float32)
        return lbm_unet_train_step(self._h, x, target, fluid, x.shape[0], lr, on_device)


# ----------------------------------------------------------- convenience

def make_config(nx, ny, tau, *, rho0=1.0, u0=(0.0, 0.0), bc_x=LBM_PERIODIC, bc_y=LBM_PERIODIC,
                wall_ux=(0.0, 0.0), body_force=(0.0, 0.0), inflow_umax=0.0, gravity=(0.0, 0.0),
                lub_range=0.0, precision=LBM_FP64, rho_w_mode=LBM_RHOW_CONST,
                refill=LBM_REFILL_A1, force_ring=256, device=0, stream=None,
                motion_cme=0, relative_changes=0, collision=0, boundary=0) -> lbm_config:
    """An lbm_config (see include/lbm.h for every field).  Model options:
    collision LBM_BGK | LBM_MRT; boundary LBM_HALFWAY | LBM_INTERPOLATED (the
    disks' boundary condition); motion_cme 1 drives free solids by the Eq. 4
    force instead of Eq. 5; relative_changes 1 books covered and fresh nodes
    in the Eq. 5 record as m (u - v)."""
    c = lbm_config_default()
    c.nx, c.ny, c.bc_x, c.bc_y = int(nx), int(ny), int(bc_x), int(bc_y)
    c.tau, c.rho0 = float(tau), float(rho0)
    c.u0[0], c.u0[1] = map(float, u0)
    c.wall_ux[0], c.wall_ux[1] = map(float, wall_ux)
    c.body_force[0], c.body_force[1] = map(float, body_force)
    c.inflow_umax = float(inflow_umax)
    c.gravity[0], c.gravity[1] = map(float, gravity)
    c.lub_range = float(lub_range)
    c.precision = PRECISION_NAMES.get(precision, precision) if isinstance(precision, str) else int(precision)
    c.rho_w_mode, c.refill, c.force_ring = int(rho_w_mode), int(refill), int(force_ring)
    c.device = int(device)
    c.motion_cme = int(motion_cme)
    c.relative_changes = int(relative_changes)
    c.collision = int(collision)
    c.boundary = int(boundary)
    c.stream = stream
    return c


class Lattice:
    """Owns one lbm_ctx.  Results come back as numpy arrays (host) unless a
    torch tensor is passed to the *_into methods."""

    def __init__(self, nx, ny, tau, **kw):
        self.cfg = make_config(nx, ny, tau, **kw)
        self.nx, self.ny = int(nx), int(ny)
        self._h = lbm_create(self.cfg)

    @classmethod
    def from_workload(cls, w: dict, *, precision=LBM_FP64, add_solids=True, **kw):
        """Build from a workload description (see the workloads package)."""
        opts = dict(rho0=w.get("rho0", 1.0), u0=w.get("u0", (0.0, 0.0)), bc_x=w["bc_x"],
                    bc_y=w["bc_y"], wall_ux=w.get("wall_ux", (0.0, 0.0)),
                    body_force=w.get("body_force", (0.0, 0.0)),
                    inflow_umax=w.get("inflow_umax", 0.0), gravity=w.get("gravity", (0.0, 0.0)),
                    lub_range=w.get("lub_range", 0.0), rho_w_mode=w.get("rho_w_mode", 0),
                    refill=w.get("refill", 1), precision=precision,
                    motion_cme=w.get("motion_cme", 0),
                    relative_changes=w.get("relative_changes", 0),
                    collision=w.get("collision", 0), boundary=w.get("boundary", 0))
        opts.update(kw)
        lat = cls(w["nx"], w["ny"], w["tau"], **opts)
        if add_solids:
            for s in w["solids"]:
                lat.add_disk(**s)
        return lat

    def close(self):
        if getattr(self, "_h", None) and not getattr(self, "_borrowed", False):
            lbm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def t(self) -> int:
        return lbm_time(self._h)

    @property
    def nsolid(self) -> int:
        return lbm_nsolid(self._h)

    def add_disk(self, cx, cy, r, vx=0.0, vy=0.0, omega=0.0, rho_s=1.0, motion=LBM_PRESCRIBED):
        d = lbm_disk(cx=cx, cy=cy, r=r, vx=vx, vy=vy, omega=omega, rho_s=rho_s, motion=motion)
        return lbm_add_solid(self._h, d)

    def step(self, n: int = 1):
        lbm_step(self._h, n)

    def sync(self):
        lbm_sync(self._h)

    def forces(self, first: int, count: int) -> np.ndarray:
        """[count][nsolid][2 (Eq. 4, Eq. 5)][Fx, Fy, T] for steps first.. (host)."""
        ns = self.nsolid
        out = np.zeros((2, max(count, 0), ns, 3))
        for form in (LBM_CME, LBM_GME):
            buf = np.zeros((max(count, 0), ns, 3))
            if count and ns:
                lbm_forces(self._h, form, first, count, buf)
            out[form] = buf
        return np.ascontiguousarray(out.transpose(1, 2, 0, 3))

    def step_record(self, n: int) -> np.ndarray:
        t0 = self.t
        self.step(n)
        return self.forces(t0, n)

    def fields(self):
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        lbm_fields(self._h, rho, ux, uy)
        return rho, ux, uy

    def get_f(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.nx))
        lbm_get_populations(self._h, out)
        return out

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        lbm_set_populations(self._h, f)

    def owner(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.int32)
        lbm_get_owner(self._h, out)
        return out

    def solids(self) -> np.ndarray:
        out = np.zeros((max(self.nsolid, 1), 5))
        lbm_get_solids(self._h, out)
        return out[: self.nsolid]

    def set_solid_velocity(self, sid: int, vx: float, vy: float, omega: float):
        st = self.solids()[sid].copy()
        st[2:] = (vx, vy, omega)
        lbm_set_solid(self._h, sid, st)

    def links(self) -> np.ndarray:
        n = lbm_links(self._h, 0, None)
        out = np.zeros((max(n, 1), 4), dtype=np.int32)
        lbm_links(self._h, n, out)
        return out[:n]

    def set_graph(self, steps: int):
        lbm_set_graph(self._h, steps)

    def set_force_overlap(self, on: bool):
        lbm_set_force_overlap(self._h, on)

    def force_overlap(self) -> int:
        return lbm_force_overlap(self._h)

    def set_wait_limit(self, polls: int):
        lbm_set_wait_limit(self._h, polls)

    def save(self) -> np.ndarray:
        """The context's state (lbm_save) as a host array of bytes."""
        buf = np.empty(lbm_state_size(self._h), dtype=np.uint8)
        lbm_save(self._h, buf)
        return buf

    def load(self, state: np.ndarray):
        lbm_load(self._h, np.ascontiguousarray(state, dtype=np.uint8))

    def set_timing(self, enable: bool):
        lbm_set_timing(self._h, enable)

    def timing(self):
        return lbm_get_timing(self._h)

    def launch_count(self) -> int:
        return lbm_launch_count(self._h)

    def set_kernel_variant(self, variant: int):
        lbm_set_kernel_variant(self._h, variant)

    def kernel_variant(self) -> int:
        return lbm_kernel_variant(self._h)

    def autotune(self, steps: int = 4) -> int:
        return lbm_autotune(self._h, steps)


class Batch:
    """Owns an lbm_batch: many independent domains stepped together.  Case k
    is read through ``case(k)``, a Lattice view on the batch's context."""

    def __init__(self, configs):
        self.configs = list(configs)
        self._h = lbm_batch_create(self.configs)
        self._views = {}

    @classmethod
    def from_workloads(cls, ws, *, precision=LBM_FP32_DEV, force_ring=4, **kw):
        cfgs = []
        for w in ws:
            opts = dict(rho0=w.get("rho0", 1.0), u0=w.get("u0", (0.0, 0.0)), bc_x=w["bc_x"],
                        bc_y=w["bc_y"], wall_ux=w.get("wall_ux", (0.0, 0.0)),
                        body_force=w.get("body_force", (0.0, 0.0)),
                        inflow_umax=w.get("inflow_umax", 0.0),
                        rho_w_mode=w.get("rho_w_mode", 0), refill=w.get("refill", 1),
                        precision=precision, force_ring=force_ring)
            opts.update(kw)
            cfgs.append(make_config(w["nx"], w["ny"], w["tau"], **opts))
        b = cls(cfgs)
        for k, w in enumerate(ws):
            for d in w["solids"]:
                b.add_disk(k, d["cx"], d["cy"], d["r"])
        return b

    def close(self):
        if getattr(self, "_h", None):
            lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.configs)

    @property
    def handle(self):
        return self._h

    def add_disk(self, k: int, cx, cy, r) -> int:
        return lbm_batch_add_solid(self._h, k, lbm_disk(cx=cx, cy=cy, r=r))

    def set_convergence(self, every=100, tol=1e-7, max_steps=2_000_000, window=1):
        lbm_batch_set_convergence(self._h, every, tol, max_steps)
        lbm_batch_set_convergence_window(self._h, window)

    def run(self, steps: int) -> int:
        """Advance the active cases by up to ``steps``; returns the active count."""
        return lbm_batch_run(self._h, steps)

    def retire(self, ids):
        lbm_batch_retire(self._h, ids)

    def state(self):
        n = len(self)
        st = np.zeros(n, dtype=np.int32)
        steps = np.zeros(n, dtype=np.int64)
        drag = np.zeros(n)
        lbm_batch_state(self._h, st, steps, drag)
        return st, steps, drag

    def case(self, k: int) -> "Lattice":
        if k not in self._views:
            v = Lattice.__new__(Lattice)
            v.cfg = self.configs[k]
            v.nx, v.ny = int(v.cfg.nx), int(v.cfg.ny)
            v._h = lbm_batch_case(self._h, k)
            v._borrowed = True
            self._views[k] = v
        return self._views[k]

    def set_launch(self, variant: int, tile_rows: int = 1, persistent: bool = False,
                   graph: bool = True):
        lbm_batch_set_launch(self._h, variant, tile_rows, persistent, graph)

    def launch(self):
        return lbm_batch_get_launch(self._h)

    def autotune(self, steps: int = 4, cache: str | None = None):
        """Fastest (variant, tile_rows, persistent) of the fused kernel.
        With ``cache`` (a JSON file), a result stored under the same key (GPU
        name, precision and the batch's size classes) is reused without
        timing, and a new result is stored."""
        key = None
        if cache:
            import json
            key = _tune_key(self.configs)
            try:
                with open(cache) as fh:
                    table = json.load(fh)
            except (OSError, ValueError):
                table = {}
            if key in table:
                v, h, p = table[key]
                self.set_launch(int(v), int(h), bool(p))
                return int(v), int(h), int(p)
        best = lbm_batch_autotune(self._h, steps)
        if cache:
            import json
            try:
                with open(cache) as fh:
                    table = json.load(fh)
            except (OSError, ValueError):
                table = {}
            table[key] = list(best)
            with open(cache, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
        return best

    def set_timing(self, enable: bool):
        lbm_batch_set_timing(self._h, enable)

    def timing(self):
        return lbm_batch_get_timing(self._h)

    def launch_count(self) -> int:
        return lbm_batch_launch_count(self._h)


def _tune_key(configs) -> str:
    """Autotuner cache key: device name, precision, and the number of cases
    per size class (x extent rounded up to a power of two, total nodes to a
    power of four)."""
    import math
    try:
        import torch
        dev = torch.cuda.get_device_name(int(configs[0].device)) if torch.cuda.is_available() else "cpu"
    except Exception:
        dev = "unknown"
    classes = {}
    for c in configs:
        k = f"x{1 << max(0, math.ceil(math.log2(c.nx)))}"
        classes[k] = classes.get(k, 0) + 1
    cells = sum(int(c.nx) * int(c.ny) for c in configs)
    parts = ",".join(f"{k}:{v}" for k, v in sorted(classes.items()))
    return f"{dev}|p{int(configs[0].precision)}|{parts}|n4^{round(math.log(max(cells, 1), 4))}"
