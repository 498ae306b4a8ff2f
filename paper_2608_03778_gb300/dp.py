"""Thin ctypes binding of libdiffpower.so (``include/diffpower.h``).

Argument marshalling only: every function has the C name, forwards to the
library and raises :class:`DPError` on a non-zero status.  Array arguments may
be numpy arrays (host memory, ``on_device=0``) or CUDA torch tensors
(``on_device=1``); ``None`` stands for NULL.  There is no fallback: if the
library cannot be loaded, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_out", "libdiffpower.so")

STATUS = {0: "DP_OK", 1: "DP_EINVAL", 2: "DP_EPARSE", 3: "DP_ECYCLE", 4: "DP_ENOMEM", 5: "DP_ECUDA",
          6: "DP_ETIMEOUT", 7: "DP_ESTATE", 8: "DP_EUNSUPPORTED"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (or python -m "
                      "paper_2608_03778_gb300._build) first")
_lib = ctypes.CDLL(LIB_PATH)


class DPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class dp_config(ctypes.Structure):
    _fields_ = [("vdd", ctypes.c_double), ("fclk", ctypes.c_double), ("beta_min", ctypes.c_float),
                ("beta_max", ctypes.c_float), ("tr_mode", ctypes.c_int32), ("grad_mode", ctypes.c_int32),
                ("sim_words", ctypes.c_int32), ("schedule", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class dp_info(ctypes.Structure):
    _fields_ = [("n_nets", ctypes.c_int64), ("n_start", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("n_edges", ctypes.c_int64), ("n_levels", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("device_bytes", ctypes.c_size_t), ("block_threads", ctypes.c_int32),
                ("cluster_threads", ctypes.c_int32)]


class dp_compiled_view(ctypes.Structure):
    _fields_ = [("lvl_ptr", ctypes.POINTER(ctypes.c_int32)), ("fanin", ctypes.POINTER(ctypes.c_uint32)),
                ("fout_ptr", ctypes.POINTER(ctypes.c_int32)), ("fout_edge", ctypes.POINTER(ctypes.c_int32)),
                ("net_of_user", ctypes.POINTER(ctypes.c_int32)), ("cell_of_user", ctypes.POINTER(ctypes.c_int32)),
                ("base_cap", ctypes.POINTER(ctypes.c_float)), ("pincap", ctypes.POINTER(ctypes.c_float)),
                ("op_arity", ctypes.POINTER(ctypes.c_uint8)), ("op_tt", ctypes.POINTER(ctypes.c_uint16)),
                ("bc_ops", ctypes.POINTER(ctypes.c_uint8)), ("bc_args", ctypes.POINTER(ctypes.c_int8)),
                ("bc_offset", ctypes.POINTER(ctypes.c_int32)), ("bc_length", ctypes.POINTER(ctypes.c_int32)),
                ("n_bc", ctypes.c_int64)]


class dp_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("hbm_budget", ctypes.c_size_t),
                ("plain", ctypes.c_int32), ("analysis", dp_config), ("slots_per_design", ctypes.c_int32)]


class dp_request(ctypes.Structure):
    _fields_ = [("design", ctypes.c_int32), ("sp", ctypes.c_void_p), ("tr", ctypes.c_void_p),
                ("cells", ctypes.c_void_p), ("pincap", ctypes.c_void_p), ("n_delta", ctypes.c_int32),
                ("want_grad", ctypes.c_int32), ("power", ctypes.c_void_p), ("grad_sp", ctypes.c_void_p),
                ("grad_tr", ctypes.c_void_p), ("grad_pincap", ctypes.c_void_p)]


class dp_server_stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("requests", ctypes.c_int64), ("max_batch_seen", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("designs", ctypes.c_int32), ("host_launch_s", ctypes.c_double)]


_P = ctypes.c_void_p
_S = ctypes.c_int


def _sig(name, args, res=_S):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("dp_config_default", [ctypes.POINTER(dp_config)], None)
_sig("dp_last_error", [_P], ctypes.c_char_p)
_sig("dp_compile", [ctypes.c_char_p, ctypes.c_size_t, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(_P),
                    ctypes.c_char_p, ctypes.c_size_t])
_sig("dp_compiled_free", [_P], None)
_sig("dp_compiled_info", [_P, ctypes.POINTER(dp_info)])
_sig("dp_compiled_view_get", [_P, ctypes.POINTER(dp_compiled_view)])
_sig("dp_compile_function", [ctypes.c_char_p, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint16),
                             ctypes.POINTER(ctypes.c_int32)])
_sig("dp_create", [ctypes.c_int, _P, ctypes.POINTER(_P)])
_sig("dp_destroy", [_P], None)
_sig("dp_sync", [_P])
_sig("dp_selftest_wait", [_P, ctypes.c_double])
_sig("dp_selftest_pending_error", [ctypes.c_int, ctypes.POINTER(ctypes.c_int32)])
_sig("dp_probe_latency", [_P, ctypes.c_int32, _P])
_sig("dp_design_load", [_P, ctypes.c_char_p, ctypes.c_size_t, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(_P)])
_sig("dp_design_upload", [_P, _P, ctypes.POINTER(_P)])
_sig("dp_design_free", [_P], None)
_sig("dp_design_info", [_P, ctypes.POINTER(dp_info)])
_sig("dp_set_inputs", [_P, _P, _P, ctypes.c_int32, _S])
_sig("dp_set_pincap", [_P, _P, _P, ctypes.c_int32, _S])
_sig("dp_propagate", [_P, ctypes.POINTER(dp_config)])
_sig("dp_simulate", [_P, ctypes.POINTER(dp_config)])
_sig("dp_total_power", [_P, _S, _P])
_sig("dp_backward", [_P, ctypes.POINTER(dp_config), _P, _P, _P, _P, _S])
_sig("dp_get_nets", [_P, _P, _P, _P, _P, _P, _P, _S])
_sig("dp_step", [_P, ctypes.POINTER(dp_config), _P, _P, _P, _P, _P, _S])
_sig("dp_phase_times", [_P, _P])
_sig("dp_step_kernels", [_P, ctypes.POINTER(ctypes.c_int64)])
_sig("dp_power_noalloc", [ctypes.c_int, _P, _P, _P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _P, _P])
_sig("dp_set_stream", [_P, _P])
_sig("dp_sizing_scores", [_P, ctypes.POINTER(dp_config), ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _S])
_sig("dp_server_config_default", [ctypes.POINTER(dp_server_config)], None)
_sig("dp_server_create", [ctypes.POINTER(dp_server_config), ctypes.POINTER(_P)])
_sig("dp_server_destroy", [_P], None)
_sig("dp_server_last_error", [_P], ctypes.c_char_p)
_sig("dp_server_add_design", [_P, ctypes.c_char_p, ctypes.c_size_t, ctypes.c_char_p, ctypes.c_size_t, _P, _P,
                              ctypes.POINTER(ctypes.c_int32)])
_sig("dp_server_design_info", [_P, ctypes.c_int32, ctypes.POINTER(dp_info)])
_sig("dp_server_submit", [_P, ctypes.POINTER(dp_request), ctypes.POINTER(ctypes.c_uint64)])
_sig("dp_server_submit_many", [_P, ctypes.POINTER(dp_request), ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)])
_sig("dp_server_wait", [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)])
_sig("dp_server_get_stats", [_P, ctypes.POINTER(dp_server_stats)])
_sig("dp_get_power", [_P, _S, _P, _S])
_sig("dp_set_inputs_batch", [_P, _P, _P, ctypes.c_int32, _S])
_sig("dp_batch_tuning", [_P, _P, _P])
_sig("dp_backward_weighted", [_P, ctypes.POINTER(dp_config), _P, ctypes.c_int32, _P, _P, _P, _P, _S])
_sig("dp_ascent_step", [_P, _P, _P, ctypes.c_int64, ctypes.c_float])
_sig("dp_virus_eval", [_P, _P, ctypes.c_int32, _P, _P, _S])

_sig("dp_compiled_save", [_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)])
_sig("dp_compiled_load", [_P, ctypes.c_size_t, ctypes.POINTER(_P), ctypes.c_char_p, ctypes.c_size_t])
_sig("dp_design_load_blob", [_P, _P, ctypes.c_size_t, ctypes.POINTER(_P)])

EXPORTED = ["dp_config_default", "dp_last_error", "dp_compile", "dp_compiled_free", "dp_compiled_info",
            "dp_compiled_save", "dp_compiled_load", "dp_design_load_blob",
            "dp_compiled_view_get", "dp_compile_function", "dp_create", "dp_destroy", "dp_sync", "dp_design_load",
            "dp_design_upload", "dp_design_free", "dp_design_info", "dp_set_inputs", "dp_set_pincap",
            "dp_propagate", "dp_simulate", "dp_total_power", "dp_backward", "dp_get_nets", "dp_step",
            "dp_phase_times", "dp_step_kernels", "dp_power_noalloc", "dp_selftest_wait",
            "dp_selftest_pending_error", "dp_probe_latency", "dp_set_stream",
            "dp_get_power", "dp_set_inputs_batch", "dp_batch_tuning", "dp_backward_weighted", "dp_ascent_step",
            "dp_virus_eval", "dp_sizing_scores", "dp_server_config_default", "dp_server_create", "dp_server_destroy",
            "dp_server_last_error", "dp_server_add_design", "dp_server_design_info", "dp_server_submit",
            "dp_server_submit_many",
            "dp_server_wait", "dp_server_get_stats"]


def _ptr(x):
    """Host or device address of an array argument (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported array argument {type(x)}")


class _Ctx:
    """Holds the context pointer for error messages."""
    current = None


def _check(status: int, ctx=None):
    if status != 0:
        msg = _lib.dp_last_error(ctx).decode() if ctx else ""
        raise DPError(status, msg)


def config(**kw) -> dp_config:
    """dp_config_default() with fields overridden by keyword."""
    c = dp_config()
    _lib.dp_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def dp_compile(netlist: str, library: str):
    nb, lb = netlist.encode(), library.encode()
    out = _P()
    err = ctypes.create_string_buffer(512)
    st = _lib.dp_compile(nb, len(nb), lb, len(lb), ctypes.byref(out), err, 512)
    if st != 0:
        raise DPError(st, err.value.decode())
    return out.value


def dp_compiled_free(c) -> None:
    _lib.dp_compiled_free(c)


def dp_compiled_save(c) -> bytes:
    """The compiled netlist as a blob."""
    n = ctypes.c_size_t(0)
    _check(_lib.dp_compiled_save(c, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.dp_compiled_save(c, buf, n.value, ctypes.byref(n)))
    return buf.raw[:n.value]


def dp_compiled_load(blob: bytes):
    out = _P()
    err = ctypes.create_string_buffer(256)
    st = _lib.dp_compiled_load(blob, len(blob), ctypes.byref(out), err, 256)
    if st != 0:
        raise DPError(st, err.value.decode())
    return out.value


def dp_compiled_info(c) -> dp_info:
    i = dp_info()
    _check(_lib.dp_compiled_info(c, ctypes.byref(i)))
    return i


def dp_compiled_view_get(c) -> dict:
    """Copies of the compiled arrays as numpy arrays."""
    info = dp_compiled_info(c)
    v = dp_compiled_view()
    _check(_lib.dp_compiled_view_get(c, ctypes.byref(v)))
    nn, nc, ne, L = info.n_nets, info.n_cells, info.n_edges, info.n_levels

    def arr(p, n, dt):
        return np.ctypeslib.as_array(p, shape=(n,)).astype(dt, copy=True) if n else np.zeros(0, dt)

    return {
        "lvl_ptr": arr(v.lvl_ptr, L + 1, np.int32), "fanin": arr(v.fanin, 4 * nc, np.uint32),
        "fout_ptr": arr(v.fout_ptr, nn + 1, np.int32), "fout_edge": arr(v.fout_edge, ne, np.int32),
        "net_of_user": arr(v.net_of_user, nn, np.int32), "cell_of_user": arr(v.cell_of_user, nc, np.int32),
        "base_cap": arr(v.base_cap, nn, np.float32), "pincap": arr(v.pincap, nc, np.float32),
        "op_arity": arr(v.op_arity, 256, np.uint8), "op_tt": arr(v.op_tt, 256, np.uint16),
        "bc_ops": arr(v.bc_ops, v.n_bc, np.uint8), "bc_args": arr(v.bc_args, v.n_bc, np.int8),
        "bc_offset": arr(v.bc_offset, 256, np.int32), "bc_length": arr(v.bc_length, 256, np.int32),
        "info": info,
    }


def dp_compile_function(func: str) -> dict:
    ops = (ctypes.c_uint8 * 64)()
    args = (ctypes.c_int8 * 64)()
    ln, nin, lid = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    tt = ctypes.c_uint16()
    st = _lib.dp_compile_function(func.encode(), ctypes.cast(ops, _P), ctypes.cast(args, _P), 64, ctypes.byref(ln),
                                  ctypes.byref(nin), ctypes.byref(tt), ctypes.byref(lid))
    if st != 0:
        raise DPError(st, f"cannot compile {func!r}")
    n = min(ln.value, 64)
    return {"ops": list(ops[:n]), "args": list(args[:n]), "n_inputs": nin.value, "tt": tt.value,
            "logic_id": lid.value}


def dp_create(device: int = 0, stream: int | None = None):
    out = _P()
    _check(_lib.dp_create(device, stream, ctypes.byref(out)))
    return out.value


def dp_destroy(ctx) -> None:
    _lib.dp_destroy(ctx)


def dp_sync(ctx) -> None:
    _check(_lib.dp_sync(ctx), ctx)


def dp_selftest_wait(ctx, seconds: float) -> None:
    _check(_lib.dp_selftest_wait(ctx, seconds), ctx)


def dp_probe_latency(ctx, levels: int = 1000) -> dict:
    """Per-level latency figures of the level-synchronous schedule (microseconds)."""
    out = np.zeros(6, np.float64)
    _check(_lib.dp_probe_latency(ctx, levels, out.ctypes.data), ctx)
    return {"barrier_us_256": float(out[0]), "level_us_256": float(out[1]), "barrier_us_512": float(out[2]),
            "level_us_512": float(out[3]), "l2_load_us": float(out[4]), "grid_blocks": int(out[5])}


def dp_selftest_pending_error(action: int) -> int:
    """0: read the library runtime's pending CUDA error code; 1: plant a host-side launch
    configuration error first; 2: read and clear it."""
    code = ctypes.c_int32(0)
    _check(_lib.dp_selftest_pending_error(action, ctypes.byref(code)))
    return int(code.value)


def dp_design_load(ctx, netlist: str, library: str):
    nb, lb = netlist.encode(), library.encode()
    out = _P()
    _check(_lib.dp_design_load(ctx, nb, len(nb), lb, len(lb), ctypes.byref(out)), ctx)
    return out.value


def dp_design_load_blob(ctx, blob: bytes):
    out = _P()
    _check(_lib.dp_design_load_blob(ctx, blob, len(blob), ctypes.byref(out)), ctx)
    return out.value


def dp_design_upload(ctx, compiled):
    out = _P()
    _check(_lib.dp_design_upload(ctx, compiled, ctypes.byref(out)), ctx)
    return out.value


def dp_design_free(d) -> None:
    _lib.dp_design_free(d)


def dp_design_info(d) -> dp_info:
    i = dp_info()
    _check(_lib.dp_design_info(d, ctypes.byref(i)))
    return i


def dp_set_inputs(ctx, d, sp, tr, n_scen: int = 1, on_device: int = 0) -> None:
    _check(_lib.dp_set_inputs(d, _ptr(sp), _ptr(tr), n_scen, on_device), ctx)


def dp_set_pincap(ctx, d, cells, pincap, on_device: int = 0) -> None:
    _check(_lib.dp_set_pincap(d, _ptr(cells), _ptr(pincap), len(cells), on_device), ctx)


def dp_set_pincap_all(ctx, d, pincap, n_cells: int, on_device: int = 0) -> None:
    """Every cell's input pin cap, in cell-line order (dp_set_pincap with a NULL cell list)."""
    _check(_lib.dp_set_pincap(d, None, _ptr(pincap), n_cells, on_device), ctx)


def dp_propagate(ctx, d, cfg: dp_config) -> None:
    _check(_lib.dp_propagate(d, ctypes.byref(cfg)), ctx)


def dp_simulate(ctx, d, cfg: dp_config) -> None:
    _check(_lib.dp_simulate(d, ctypes.byref(cfg)), ctx)


def dp_total_power(ctx, d, hybrid: int = 0, n_scen: int = 1):
    """Power in watts: a float for one scenario, an array of n_scen values for a batch
    (n_scen must be the batch's size: the library writes that many values)."""
    w = np.zeros(max(int(n_scen), 1), np.float64)
    _check(_lib.dp_total_power(d, hybrid, w.ctypes.data), ctx)
    return float(w[0]) if n_scen == 1 else w


def dp_backward(ctx, d, cfg: dp_config, grad_sp_in=None, grad_tr_in=None, grad_pincap=None, grad_cload=None,
                on_device: int = 0) -> None:
    _check(_lib.dp_backward(d, ctypes.byref(cfg), _ptr(grad_sp_in), _ptr(grad_tr_in), _ptr(grad_pincap),
                            _ptr(grad_cload), on_device), ctx)


def dp_get_nets(ctx, d, sp=None, tr=None, beta=None, tr_hyb=None, toggles=None, ones=None,
                on_device: int = 0) -> None:
    _check(_lib.dp_get_nets(d, _ptr(sp), _ptr(tr), _ptr(beta), _ptr(tr_hyb), _ptr(toggles), _ptr(ones),
                            on_device), ctx)


def dp_step(ctx, d, cfg: dp_config, grad_sp_in=None, grad_tr_in=None, grad_pincap=None, grad_cload=None,
            watts=None, on_device: int = 0) -> None:
    _check(_lib.dp_step(d, ctypes.byref(cfg), _ptr(grad_sp_in), _ptr(grad_tr_in), _ptr(grad_pincap),
                        _ptr(grad_cload), _ptr(watts), on_device), ctx)


def dp_phase_times(ctx, d) -> np.ndarray:
    ms = np.zeros(5, np.float32)
    _check(_lib.dp_phase_times(d, ms.ctypes.data), ctx)
    return ms


def dp_step_kernels(d) -> int:
    k = ctypes.c_int64()
    _check(_lib.dp_step_kernels(d, ctypes.byref(k)))
    return k.value


def dp_power_noalloc(device: int, tr, beta, cload, n: int, vdd: float, fclk: float, watts, stream=None) -> None:
    """Power reduction that allocates no device memory (all arrays are caller-owned device memory)."""
    _check(_lib.dp_power_noalloc(device, _ptr(tr), _ptr(beta), _ptr(cload), n, vdd, fclk, _ptr(watts), stream))


def dp_set_stream(ctx, stream) -> None:
    _check(_lib.dp_set_stream(ctx, stream), ctx)


def dp_get_power(ctx, d, watts, hybrid: int = 0, on_device: int = 0) -> None:
    """Powers into a caller buffer (float64: one value, or n_scen for batched inputs)."""
    _check(_lib.dp_get_power(d, hybrid, _ptr(watts), on_device), ctx)


def dp_set_inputs_batch(ctx, d, sp, tr, n_scen: int, on_device: int = 0) -> None:
    _check(_lib.dp_set_inputs_batch(d, _ptr(sp), _ptr(tr), n_scen, on_device), ctx)


def dp_batch_tuning(d):
    """((fwd_bx, fwd_by, fwd_v), (bwd_bx, bwd_by, bwd_v), (fwd_ms, bwd_ms)) chosen by the autotuner
    (v: scenarios per thread)."""
    sh = np.zeros(6, np.int32)
    ms = np.zeros(2, np.float32)
    _check(_lib.dp_batch_tuning(d, sh.ctypes.data, ms.ctypes.data))
    return (int(sh[0]), int(sh[1]), int(sh[2])), (int(sh[3]), int(sh[4]), int(sh[5])), (float(ms[0]), float(ms[1]))


def dp_backward_weighted(ctx, d, cfg: dp_config, weights=None, cap_reduce: int = 0, grad_sp_in=None,
                         grad_tr_in=None, grad_pincap=None, grad_cload=None, on_device: int = 0) -> None:
    _check(_lib.dp_backward_weighted(d, ctypes.byref(cfg), _ptr(weights), cap_reduce, _ptr(grad_sp_in),
                                     _ptr(grad_tr_in), _ptr(grad_pincap), _ptr(grad_cload), on_device), ctx)


def dp_ascent_step(ctx, x, g, n: int, eta: float) -> None:
    """x <- clip(x + eta g, 0, 1) on device arrays."""
    _check(_lib.dp_ascent_step(ctx, _ptr(x), _ptr(g), n, eta), ctx)


def dp_virus_eval(ctx, d, sp, n_scen: int, p_virus, v0=None, on_device: int = 0) -> None:
    _check(_lib.dp_virus_eval(d, _ptr(sp), n_scen, _ptr(v0), _ptr(p_virus), on_device), ctx)


# ---- request server ----

def _scheck(status: int, srv) -> None:
    if status != 0:
        raise DPError(status, _lib.dp_server_last_error(srv).decode() if srv else "")


def server_config(**kw) -> dp_server_config:
    """dp_server_config_default() with fields overridden by keyword (analysis: a dp_config)."""
    c = dp_server_config()
    _lib.dp_server_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def dp_server_create(cfg: dp_server_config):
    out = _P()
    st = _lib.dp_server_create(ctypes.byref(cfg), ctypes.byref(out))
    if st != 0:
        raise DPError(st, "dp_server_create")
    return out.value


def dp_server_destroy(srv) -> None:
    _lib.dp_server_destroy(srv)


def dp_server_add_design(srv, netlist: str, library: str, ref_sp=None, ref_tr=None) -> int:
    nb, lb = netlist.encode(), library.encode()
    i = ctypes.c_int32()
    _scheck(_lib.dp_server_add_design(srv, nb, len(nb), lb, len(lb), _ptr(ref_sp), _ptr(ref_tr), ctypes.byref(i)),
            srv)
    return i.value


def dp_server_design_info(srv, design: int) -> dp_info:
    info = dp_info()
    _scheck(_lib.dp_server_design_info(srv, design, ctypes.byref(info)), srv)
    return info


def request(design: int, power, sp=None, tr=None, cells=None, pincap=None, want_grad: int = 0, grad_sp=None,
            grad_tr=None, grad_pincap=None) -> dp_request:
    """A dp_request over host arrays (kept alive by the caller until the wait returns)."""
    r = dp_request()
    r.design = design
    r.sp, r.tr = _ptr(sp), _ptr(tr)
    r.cells, r.pincap = _ptr(cells), _ptr(pincap)
    r.n_delta = 0 if cells is None else len(cells)
    r.want_grad = want_grad
    r.power = _ptr(power)
    r.grad_sp, r.grad_tr, r.grad_pincap = _ptr(grad_sp), _ptr(grad_tr), _ptr(grad_pincap)
    return r


def dp_server_submit(srv, req: dp_request) -> int:
    t = ctypes.c_uint64()
    _scheck(_lib.dp_server_submit(srv, ctypes.byref(req), ctypes.byref(t)), srv)
    return t.value


def dp_server_submit_many(srv, reqs) -> list:
    """Queues a list of requests at once; returns their tickets."""
    n = len(reqs)
    arr = (dp_request * n)(*reqs)
    t = (ctypes.c_uint64 * n)()
    _scheck(_lib.dp_server_submit_many(srv, arr, n, t), srv)
    return list(t)


def dp_server_wait(srv, ticket: int, timeout_s: float = 0.0) -> float:
    """Waits for a request; returns its latency (submission to completion) in ms."""
    ms = ctypes.c_double()
    _scheck(_lib.dp_server_wait(srv, ticket, timeout_s, ctypes.byref(ms)), srv)
    return ms.value


def dp_server_get_stats(srv) -> dp_server_stats:
    s = dp_server_stats()
    _scheck(_lib.dp_server_get_stats(srv, ctypes.byref(s)), srv)
    return s


def dp_sizing_scores(ctx, d, cfg: dp_config, mode: int = 0, scores=None, k: int = 0, top_cells=None,
                     top_scores=None, on_device: int = 0) -> None:
    """Eq. 8 scores per cell line and the top-k cells (after dp_backward / dp_step)."""
    _check(_lib.dp_sizing_scores(d, ctypes.byref(cfg), mode, _ptr(scores), k, _ptr(top_cells), _ptr(top_scores),
                                 on_device), ctx)
