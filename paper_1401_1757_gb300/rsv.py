"""ctypes binding of the C ABI in include/rsv.h (argument marshalling only).

Every function keeps its C name.  Arrays go in as NumPy arrays (host) or torch
tensors (device or pinned host); nothing here computes a reserve.  Loading
fails loudly when the CUDA library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librsv.so")

RSV_OK, RSV_E_ARG, RSV_E_NOMEM, RSV_E_CUDA, RSV_E_STATE, RSV_E_TIMEOUT, RSV_E_ASSUMPTION = 0, -1, -2, -3, -4, -5, -6
RSV_E_LIMIT = -7
STATUS_NAMES = {0: "RSV_OK", -1: "RSV_E_ARG", -2: "RSV_E_NOMEM", -3: "RSV_E_CUDA", -4: "RSV_E_STATE",
                -5: "RSV_E_TIMEOUT", -6: "RSV_E_ASSUMPTION", -7: "RSV_E_LIMIT"}
RSV_SL_ANNUITY, RSV_JL_REVERSIONARY, RSV_TERM_ASSURANCE, RSV_ENDOWMENT = 0, 1, 2, 3
RSV_JOINT_ANNUITY, RSV_LAST_SURVIVOR, RSV_JOINT_TERM, RSV_JOINT_ENDOWMENT = 4, 5, 6, 7
RSV_LS_TERM, RSV_LS_ENDOWMENT = 8, 9
RSV_FORM_F64, RSV_FORM_F32, RSV_FORM_F32_COMP, RSV_FORM_F32_DEFLATED = 0, 1, 2, 3
RSV_VARIANT_TIME_SCAN = -2   # the FP64 parallel-in-time scan (see include/rsv.h)
RSV_VARIANT_SUMMATION = -3   # the FP64 O(S^2) summation definition
RSV_PAY_END, RSV_PAY_START, RSV_PAY_FRACTION = 0, 1, 2
FORM_NAMES = {0: "f64", 1: "f32", 2: "f32comp", 3: "f32defl"}
RSV_OUT_V0, RSV_OUT_SCEN_TOTAL, RSV_OUT_PT_MEAN, RSV_OUT_TRAJ = 1, 2, 4, 8


class rsv_policy(C.Structure):
    _fields_ = [("product", C.c_int32), ("age1_m", C.c_int32), ("age2_m", C.c_int32),
                ("term_m", C.c_int32), ("state0", C.c_int32), ("table1", C.c_int32),
                ("table2", C.c_int32), ("reserved", C.c_int32), ("amount", C.c_double),
                ("reversion", C.c_double)]


POLICY_DTYPE = np.dtype([("product", "<i4"), ("age1_m", "<i4"), ("age2_m", "<i4"), ("term_m", "<i4"),
                         ("state0", "<i4"), ("table1", "<i4"), ("table2", "<i4"), ("reserved", "<i4"),
                         ("amount", "<f8"), ("reversion", "<f8")])
assert POLICY_DTYPE.itemsize == C.sizeof(rsv_policy) == 48


class rsv_schedule(C.Structure):
    _fields_ = [("every", C.c_int32), ("first", C.c_int32), ("since", C.c_int32), ("steps_per_year", C.c_int32),
                ("escalation", C.c_double), ("increase", C.c_double)]


SCHEDULE_DTYPE = np.dtype([("every", "<i4"), ("first", "<i4"), ("since", "<i4"), ("steps_per_year", "<i4"),
                           ("escalation", "<f8"), ("increase", "<f8")])
assert SCHEDULE_DTYPE.itemsize == C.sizeof(rsv_schedule) == 32


RSV_MLIFE_ANNUITY, RSV_MLIFE_ASSURANCE = 0, 1

MLIFE_DTYPE = np.dtype([("m", "<i4"), ("kind", "<i4"), ("k", "<i4"), ("term_m", "<i4"), ("age_m", "<i4", (4,)),
                        ("table", "<i4", (4,)), ("dead0", "<i4"), ("reserved", "<i4"), ("amount", "<f8")])
assert MLIFE_DTYPE.itemsize == 64


class rsv_opts(C.Structure):
    _fields_ = [("form", C.c_int32), ("outputs", C.c_int32), ("horizon", C.c_int32),
                ("on_device", C.c_int32), ("variant", C.c_int32), ("payment", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class rsv_out(C.Structure):
    _fields_ = [("V0", C.c_void_p), ("V0d", C.c_void_p), ("scen_total", C.c_void_p),
                ("pt_mean", C.c_void_p), ("traj", C.c_void_p)]


RSV_NESTED_MC, RSV_NESTED_SURROGATE, RSV_NESTED_CURVE = 0, 1, 2


class rsv_nested_spec(C.Structure):
    _fields_ = [("n_outer", C.c_int32), ("n_nodes", C.c_int32), ("node_step_m", C.c_int32),
                ("n_inner", C.c_int32), ("seed", C.c_uint64), ("a", C.c_double), ("b", C.c_double),
                ("sigma", C.c_double), ("r0", C.c_double), ("mode", C.c_int32), ("batch_outer", C.c_int32),
                ("outer_first", C.c_int32)]


class rsv_nested_out(C.Structure):
    _fields_ = [("L_mean", C.c_void_p), ("L_q995", C.c_void_p), ("r_node", C.c_void_p), ("D0", C.c_void_p),
                ("L_all", C.c_void_p), ("n_fallback", C.c_void_p)]


class rsv_surrogate_cfg(C.Structure):
    _fields_ = [("n_train", C.c_int64), ("n_val", C.c_int64), ("epochs", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_double), ("seed", C.c_uint64), ("a", C.c_double), ("b", C.c_double),
                ("sigma", C.c_double), ("r0", C.c_double), ("max_node_m", C.c_int32), ("widen", C.c_double),
                ("tol", C.c_double), ("margin", C.c_double)]


class rsv_surrogate_report(C.Structure):
    _fields_ = [("train_loss", C.c_double), ("val_max_rel", C.c_double), ("val_p99_rel", C.c_double),
                ("val_median_rel", C.c_double), ("val_rms_rel", C.c_double), ("frac_fallback", C.c_double),
                ("combined_max_rel", C.c_double), ("label_ms", C.c_double), ("train_ms", C.c_double),
                ("infer_ms", C.c_double), ("n_label", C.c_int64), ("n_infer", C.c_int64),
                ("n_buckets", C.c_int64), ("n_flagged", C.c_int64), ("y_mean", C.c_double), ("y_std", C.c_double)]


QUERY_DTYPE = np.dtype([("pol", "<i4"), ("m", "<i4"), ("state", "<i4"), ("reserved", "<i4"), ("r", "<f8")])
RSV_QUERY_NETWORK, RSV_QUERY_RECURRENCE, RSV_QUERY_FALLBACK = 0, 1, 2


class RsvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

# Exported symbols of librsv.so that include/rsv.h declares.
EXPORTS = ["rsv_create", "rsv_destroy", "rsv_set_stream", "rsv_load_decrements", "rsv_load_portfolio",
           "rsv_load_decrements_fraction", "rsv_load_scenarios_fraction", "rsv_load_cashflows", "rsv_load_schedules",
           "rsv_clear_cashflows", "rsv_compute_mlife", "rsv_surrogate_save", "rsv_surrogate_load",
           "rsv_selftest_bounded_wait", "rsv_selftest_generator_math",
           "rsv_load_scenarios", "rsv_compute_reserves", "rsv_compute_nested", "rsv_variant_count", "rsv_variant_name",
           "rsv_tune", "rsv_synchronize", "rsv_last_error", "rsv_last_kernel_ms", "rsv_device_sm_count",
           "rsv_reserves_noalloc", "rsv_mlp_param_count", "rsv_mlp_init", "rsv_mlp_set_params",
           "rsv_mlp_get_params", "rsv_mlp_set_backend", "rsv_mlp_forward", "rsv_mlp_gradient", "rsv_surrogate_train",
           "rsv_surrogate_query", "rsv_probe_fma_peak", "rsv_mlp_trace"]


def load_library(path: str = LIB_PATH):
    """Load librsv.so (raises if it is missing: the product has no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                          "(there is no CPU fallback)")
    try:  # share the CUDA runtime that torch already loaded, if any
        import torch  # noqa: F401
    except Exception:
        pass
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "rsv_create": ([C.POINTER(vp), C.c_int, vp], i32),
        "rsv_destroy": ([vp], i32),
        "rsv_set_stream": ([vp, vp], i32),
        "rsv_load_decrements": ([vp, i32, vp, i32], i32),
        "rsv_load_portfolio": ([vp, vp, i64], i32),
        "rsv_load_scenarios": ([vp, vp, i32, i32, i32], i32),
        "rsv_load_decrements_fraction": ([vp, i32, vp, i32], i32),
        "rsv_load_scenarios_fraction": ([vp, vp, i32, i32, i32], i32),
        "rsv_load_cashflows": ([vp, vp, i64, i32], i32),
        "rsv_load_schedules": ([vp, vp, i64, i32], i32),
        "rsv_clear_cashflows": ([vp], i32),
        "rsv_compute_mlife": ([vp, vp, i64, C.POINTER(rsv_opts), C.POINTER(rsv_out)], i32),
        "rsv_surrogate_save": ([vp, C.c_char_p], i32),
        "rsv_selftest_bounded_wait": ([i32, vp, i32], i32),
        "rsv_selftest_generator_math": ([i32, vp, vp, vp, i64, vp], i32),
        "rsv_surrogate_load": ([vp, C.c_char_p], i32),
        "rsv_compute_reserves": ([vp, C.POINTER(rsv_opts), C.POINTER(rsv_out)], i32),
        "rsv_compute_nested": ([vp, C.POINTER(rsv_opts), C.POINTER(rsv_nested_spec), C.POINTER(rsv_nested_out)],
                               i32),
        "rsv_variant_count": ([i32], i32),
        "rsv_variant_name": ([i32, i32], C.c_char_p),
        "rsv_tune": ([vp, C.POINTER(rsv_opts), i32, C.POINTER(i32), C.POINTER(C.c_float)], i32),
        "rsv_synchronize": ([vp], i32),
        "rsv_last_error": ([vp], C.c_char_p),
        "rsv_last_kernel_ms": ([vp], C.c_float),
        "rsv_device_sm_count": ([vp], i32),
        "rsv_reserves_noalloc": ([C.c_int, vp, vp, i32, vp, i32, vp, i32, i32, vp, vp], i32),
        "rsv_mlp_param_count": ([], i64),
        "rsv_mlp_init": ([vp, C.c_uint64], i32),
        "rsv_mlp_set_params": ([vp, vp, i64], i32),
        "rsv_mlp_get_params": ([vp, vp, i64], i32),
        "rsv_mlp_forward": ([vp, vp, i64, vp], i32),
        "rsv_mlp_set_backend": ([vp, i32], i32),
        "rsv_mlp_gradient": ([vp, vp, vp, i64, vp, vp], i32),
        "rsv_surrogate_train": ([vp, C.POINTER(rsv_surrogate_cfg), C.POINTER(rsv_surrogate_report)], i32),
        "rsv_surrogate_query": ([vp, vp, i64, i32, vp], i32),
        "rsv_probe_fma_peak": ([i32, vp, i32, C.POINTER(C.c_double)], i32),
        "rsv_mlp_trace": ([vp, i32, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    _lib = lib
    return lib


def _check(ctx, st):
    if st != RSV_OK:
        msg = _lib.rsv_last_error(ctx).decode() if ctx else ""
        raise RsvError(st, msg)


def _ptr(x):
    """Address of a NumPy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def rsv_create(device: int = 0, stream=None):
    """Returns an opaque context handle.  ``stream``: a torch.cuda.Stream, a raw
    cudaStream_t integer, or None (legacy default stream)."""
    lib = load_library()
    h = C.c_void_p()
    s = getattr(stream, "cuda_stream", stream)
    _check(None, lib.rsv_create(C.byref(h), device, s))
    return h


def rsv_destroy(ctx):
    _check(ctx, load_library().rsv_destroy(ctx))


def rsv_set_stream(ctx, stream):
    _check(ctx, _lib.rsv_set_stream(ctx, getattr(stream, "cuda_stream", stream)))


def rsv_load_decrements(ctx, table_id: int, p_monthly):
    p = np.ascontiguousarray(p_monthly, dtype=np.float64)
    _check(ctx, _lib.rsv_load_decrements(ctx, table_id, p.ctypes.data, len(p)))


def rsv_load_decrements_fraction(ctx, table_id: int, p_f):
    """Survival over the first fraction f of each month (RSV_PAY_FRACTION)."""
    p = np.ascontiguousarray(p_f, dtype=np.float64)
    _check(ctx, _lib.rsv_load_decrements_fraction(ctx, table_id, p.ctypes.data, len(p)))


def policy_records(pol) -> np.ndarray:
    """Policy records in the ABI layout from a dict of arrays (as made by ``synth``)
    or an existing record array."""
    if isinstance(pol, np.ndarray) and pol.dtype == POLICY_DTYPE:
        return np.ascontiguousarray(pol)
    n = len(pol["product"])
    rec = np.zeros(n, POLICY_DTYPE)
    for k in ("product", "age1_m", "age2_m", "term_m", "state0", "table1", "table2", "amount", "reversion"):
        rec[k] = pol[k]
    return rec


def rsv_load_portfolio(ctx, pol):
    rec = policy_records(pol)
    _check(ctx, _lib.rsv_load_portfolio(ctx, rec.ctypes.data if len(rec) else None, len(rec)))


def rsv_load_scenarios(ctx, v, layout: int = 0):
    """v: host FP64 [n_scen, n_steps] (layout 0) or [n_steps, n_scen] (layout 1);
    a NumPy array or a (pinned) CPU torch tensor."""
    if isinstance(v, np.ndarray):
        v = np.ascontiguousarray(v, dtype=np.float64)
        ptr, shape = v.ctypes.data, v.shape
    else:
        assert v.dtype.__str__() == "torch.float64" and v.device.type == "cpu" and v.is_contiguous()
        ptr, shape = v.data_ptr(), tuple(v.shape)
    n_scen, n_steps = (shape[0], shape[1]) if layout == 0 else (shape[1], shape[0])
    _check(ctx, _lib.rsv_load_scenarios(ctx, ptr, n_scen, n_steps, layout))


def rsv_load_scenarios_fraction(ctx, v_f, layout: int = 0):
    """Discount factors over the first fraction f of each step (RSV_PAY_FRACTION),
    shaped as for rsv_load_scenarios."""
    v = np.ascontiguousarray(v_f, dtype=np.float64)
    n_scen, n_steps = (v.shape[0], v.shape[1]) if layout == 0 else (v.shape[1], v.shape[0])
    _check(ctx, _lib.rsv_load_scenarios_fraction(ctx, v.ctypes.data, n_scen, n_steps, layout))


def rsv_load_cashflows(ctx, cf):
    """Cash-flow multipliers c_t / c: host FP64 [n_pol, n_steps]."""
    a = np.ascontiguousarray(cf, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("cf must be [n_pol, n_steps]")
    _check(ctx, _lib.rsv_load_cashflows(ctx, a.ctypes.data, a.shape[0], a.shape[1]))


def schedule_records(sch) -> np.ndarray:
    """Schedule records in the ABI layout from a dict of arrays or a record array."""
    if isinstance(sch, np.ndarray) and sch.dtype == SCHEDULE_DTYPE:
        return np.ascontiguousarray(sch)
    n = len(sch["every"])
    rec = np.zeros(n, SCHEDULE_DTYPE)
    for k in SCHEDULE_DTYPE.names:
        rec[k] = sch[k]
    return rec


def rsv_load_schedules(ctx, sch, n_steps: int):
    """One payment schedule per policy, expanded on the device into rows of n_steps."""
    rec = schedule_records(sch)
    _check(ctx, _lib.rsv_load_schedules(ctx, rec.ctypes.data if len(rec) else None, len(rec), n_steps))


def rsv_clear_cashflows(ctx):
    _check(ctx, _lib.rsv_clear_cashflows(ctx))


def rsv_compute_reserves(ctx, form: int = RSV_FORM_F32_COMP, outputs: int = RSV_OUT_V0, horizon: int = 0,
                         on_device: bool = False, variant: int = -1, V0=None, V0d=None, scen_total=None,
                         pt_mean=None, traj=None, payment: int = 0):
    """Runs the recurrence.  Output buffers (NumPy for on_device=False, CUDA
    torch tensors for on_device=True) are caller-sized; see include/rsv.h."""
    o = rsv_opts(form, outputs, horizon, 1 if on_device else 0, variant, payment)
    out = rsv_out(_ptr(V0), _ptr(V0d), _ptr(scen_total), _ptr(pt_mean), _ptr(traj))
    _check(ctx, _lib.rsv_compute_reserves(ctx, C.byref(o), C.byref(out)))


def mlife_records(pol) -> np.ndarray:
    """m-life records in the ABI layout from a dict of arrays (age_m and table
    [n, 4]) or an existing record array."""
    if isinstance(pol, np.ndarray) and pol.dtype == MLIFE_DTYPE:
        return np.ascontiguousarray(pol)
    n = len(pol["m"])
    rec = np.zeros(n, MLIFE_DTYPE)
    for k in MLIFE_DTYPE.names:
        if k in pol:
            rec[k] = pol[k]
    return rec


def rsv_compute_mlife(ctx, pol, form: int = RSV_FORM_F32_COMP, outputs: int = RSV_OUT_V0, on_device: bool = False,
                      V0=None, V0d=None, scen_total=None):
    """Reserves of m-life policies (see include/rsv.h) under the loaded tables and
    scenarios; outputs [n, n_scen] and [n_scen]."""
    rec = mlife_records(pol)
    o = rsv_opts(form, outputs, 0, 1 if on_device else 0, -1, 0)
    out = rsv_out(_ptr(V0), _ptr(V0d), _ptr(scen_total), None, None)
    _check(ctx, _lib.rsv_compute_mlife(ctx, rec.ctypes.data if len(rec) else None, len(rec), C.byref(o),
                                       C.byref(out)))


def rsv_compute_nested(ctx, form: int = RSV_FORM_F32_COMP, *, n_outer: int, n_nodes: int, node_step_m: int = 12,
                       n_inner: int = 1000, seed: int = 0, a: float = 0.1, b: float = 0.04, sigma: float = 0.01,
                       r0: float = 0.03, mode: int = RSV_NESTED_MC, batch_outer: int = 0, outer_first: int = 0,
                       on_device: bool = False, L_mean=None, L_q995=None, r_node=None, D0=None, L_all=None,
                       n_fallback=None):
    """Nested valuation (see include/rsv.h).  Output buffers are caller-sized
    ([n_outer, n_nodes] and [n_outer, n_nodes, n_inner])."""
    o = rsv_opts(form, 0, 0, 1 if on_device else 0, -1)
    sp = rsv_nested_spec(n_outer, n_nodes, node_step_m, n_inner, seed, a, b, sigma, r0, mode, batch_outer, outer_first)
    out = rsv_nested_out(_ptr(L_mean), _ptr(L_q995), _ptr(r_node), _ptr(D0), _ptr(L_all), _ptr(n_fallback))
    _check(ctx, _lib.rsv_compute_nested(ctx, C.byref(o), C.byref(sp), C.byref(out)))


def rsv_selftest_bounded_wait(device: int = 0, stream=None, never_completes: bool = False) -> int:
    """Run the bounded-wait self-test; returns the status code (RSV_OK or RSV_E_TIMEOUT)."""
    return load_library().rsv_selftest_bounded_wait(device, getattr(stream, "cuda_stream", stream),
                                                    1 if never_completes else 0)


def rsv_selftest_generator_math(w, x, device: int = 0, stream=None):
    """The inner-path generator's ln u, sin 2 pi u, cos 2 pi u (u = (w + 1/2) 2^-32)
    and e^x on the device; returns an (n, 4) float64 array."""
    w = np.ascontiguousarray(w, dtype=np.uint32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if w.shape != x.shape or w.ndim != 1:
        raise ValueError("w and x must be 1-D arrays of the same length")
    out = np.empty((len(w), 4), dtype=np.float64)
    st = load_library().rsv_selftest_generator_math(device, getattr(stream, "cuda_stream", stream), w.ctypes.data,
                                                    x.ctypes.data, len(w), out.ctypes.data)
    if st != RSV_OK:
        raise RsvError(st, f"rsv_selftest_generator_math failed ({st})")
    return out


def rsv_probe_fma_peak(device: int = 0, stream=None, fp64: bool = False) -> float:
    """Measured FP32 (or FP64) FMA throughput of the device in TFLOP/s."""
    lib = load_library()
    out = C.c_double()
    st = lib.rsv_probe_fma_peak(device, getattr(stream, "cuda_stream", stream), 1 if fp64 else 0, C.byref(out))
    if st != RSV_OK:
        raise RsvError(st, f"rsv_probe_fma_peak failed ({st})")
    return out.value


def rsv_variant_count(form: int) -> int:
    return load_library().rsv_variant_count(form)


def rsv_variant_name(form: int, variant: int) -> str:
    return load_library().rsv_variant_name(form, variant).decode()


def rsv_tune(ctx, form: int, horizon: int = 0, reps: int = 3):
    """Times every kernel variant of ``form`` on the loaded data; keeps the fastest
    as the context default.  Returns (best index, [ms per variant])."""
    n = rsv_variant_count(form)
    ms = (C.c_float * n)()
    best = C.c_int32(-1)
    o = rsv_opts(form, RSV_OUT_V0 | RSV_OUT_SCEN_TOTAL, horizon, 1, -1)
    _check(ctx, _lib.rsv_tune(ctx, C.byref(o), reps, C.byref(best), ms))
    return best.value, list(ms)


def rsv_synchronize(ctx):
    _check(ctx, _lib.rsv_synchronize(ctx))


def rsv_last_error(ctx) -> str:
    return _lib.rsv_last_error(ctx).decode()


def rsv_last_kernel_ms(ctx) -> float:
    return float(_lib.rsv_last_kernel_ms(ctx))


def rsv_device_sm_count(ctx) -> int:
    return int(_lib.rsv_device_sm_count(ctx))


def rsv_reserves_noalloc(device: int, stream, pols, p_monthly, v, V0, scen_total=None):
    """The valuation without allocation (see include/rsv.h): every argument is a
    CUDA torch tensor the caller owns -- ``pols`` the 48-byte records as uint8
    [n_pol * 48], ``p_monthly`` float64 [n_ages], ``v`` float64 step-major
    [n_steps, n_scen], ``V0`` float64 [n_pol, n_scen], ``scen_total`` float64
    [n_scen] or None."""
    lib = load_library()
    n_pol = pols.numel() // 48
    n_steps, n_scen = int(v.shape[0]), int(v.shape[1])
    st = lib.rsv_reserves_noalloc(device, getattr(stream, "cuda_stream", stream), _ptr(pols), n_pol,
                                  _ptr(p_monthly), int(p_monthly.numel()), _ptr(v), n_scen, n_steps, _ptr(V0),
                                  _ptr(scen_total))
    if st != RSV_OK:
        raise RsvError(st, "rsv_reserves_noalloc")


def rsv_mlp_param_count() -> int:
    return int(load_library().rsv_mlp_param_count())


def rsv_mlp_init(ctx, seed: int = 0):
    _check(ctx, _lib.rsv_mlp_init(ctx, seed))


def rsv_mlp_set_params(ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, _lib.rsv_mlp_set_params(ctx, p.ctypes.data, p.size))


def rsv_mlp_get_params(ctx):
    p = np.zeros(rsv_mlp_param_count(), np.float32)
    _check(ctx, _lib.rsv_mlp_get_params(ctx, p.ctypes.data, p.size))
    return p


RSV_MLP_MMA_SYNC, RSV_MLP_TCGEN05 = 0, 1


def rsv_mlp_set_backend(ctx, backend: int):
    _check(ctx, _lib.rsv_mlp_set_backend(ctx, backend))


def rsv_mlp_forward(ctx, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.zeros(X.shape[0], np.float32)
    _check(ctx, _lib.rsv_mlp_forward(ctx, X.ctypes.data, X.shape[0], y.ctypes.data))
    return y


def rsv_mlp_gradient(ctx, X, target):
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(target, dtype=np.float32)
    g = np.zeros(rsv_mlp_param_count(), np.float32)
    loss = C.c_float()
    _check(ctx, _lib.rsv_mlp_gradient(ctx, X.ctypes.data, t.ctypes.data, X.shape[0], g.ctypes.data,
                                      C.byref(loss)))
    return g, loss.value


def bf16_bits_to_f64(bits):
    """BF16 values given by their 16-bit patterns, as FP64 (exact)."""
    b = np.ascontiguousarray(bits, dtype=np.uint16)
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def rsv_mlp_trace(ctx, X, backend: int = RSV_MLP_MMA_SYNC, target=None):
    """One pass of the network with every layer's values (see include/rsv.h).
    Returns a dict: Xb [n][64], Z [4][n][256], A [4][n][256] (FP64 of the BF16
    values; the tcgen05 path fills A[0..2] with 2 gelu), y [n]; with a target
    (mma.sync only) also dZ, dZb [4][n][256] and grads."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    L = n * 256
    Xb = np.zeros((n, 64), np.uint16)
    Z = np.zeros((4, n, 256), np.float32)
    A = np.zeros((4, n, 256), np.uint16)
    y = np.zeros(n, np.float32)
    dZ = dZb = grads = t = None
    if target is not None:
        t = np.ascontiguousarray(target, dtype=np.float32)
        dZ = np.zeros((4, n, 256), np.float32)
        dZb = np.zeros((4, n, 256), np.uint16)
        grads = np.zeros(rsv_mlp_param_count(), np.float32)
    _check(ctx, _lib.rsv_mlp_trace(ctx, backend, X.ctypes.data, _ptr(t), n, Xb.ctypes.data, Z.ctypes.data,
                                   A.ctypes.data, y.ctypes.data, _ptr(dZ), _ptr(dZb), _ptr(grads)))
    out = {"Xb": bf16_bits_to_f64(Xb), "Z": Z.astype(np.float64), "A": bf16_bits_to_f64(A).reshape(4, n, 256),
           "y": y.astype(np.float64)}
    if target is not None:
        out.update(dZ=dZ.astype(np.float64), dZb=bf16_bits_to_f64(dZb).reshape(4, n, 256),
                   grads=grads.astype(np.float64))
    return out


def rsv_surrogate_save(ctx, path: str):
    """Write the trained surrogate (network, normalisation, fallback map) to ``path``."""
    _check(ctx, _lib.rsv_surrogate_save(ctx, os.fsencode(path)))


def rsv_surrogate_load(ctx, path: str):
    """Read a surrogate written by rsv_surrogate_save."""
    _check(ctx, _lib.rsv_surrogate_load(ctx, os.fsencode(path)))


def rsv_surrogate_train(ctx, n_train=10_000_000, n_val=1_000_000, epochs=20, batch=8192, lr=2e-3, seed=0,
                        a=0.1, b=0.04, sigma=0.01, r0=0.03, max_node_m=600, widen=1.5, tol=1e-3, margin=0.3) -> dict:
    cfg = rsv_surrogate_cfg(n_train, n_val, epochs, batch, lr, seed, a, b, sigma, r0, max_node_m, widen, tol, margin)
    rep = rsv_surrogate_report()
    _check(ctx, _lib.rsv_surrogate_train(ctx, C.byref(cfg), C.byref(rep)))
    return {k: getattr(rep, k) for k, _ in rsv_surrogate_report._fields_}


def rsv_surrogate_query(ctx, queries, how=RSV_QUERY_FALLBACK):
    """queries: a QUERY_DTYPE record array (pol, m, state, r); returns FP64 reserves."""
    q = np.ascontiguousarray(queries, dtype=QUERY_DTYPE)
    out = np.zeros(len(q))
    _check(ctx, _lib.rsv_surrogate_query(ctx, q.ctypes.data, len(q), how, out.ctypes.data))
    return out
