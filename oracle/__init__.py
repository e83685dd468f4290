"""FP64 CPU oracle for the vector reserve recurrence (Tucker & Bull, arXiv 1401.1757).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library and its
Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``rsv_oracle.c`` (plain C99, FP64, no fused
multiply-add); this module compiles it with gcc on first use and marshals NumPy
arrays through ctypes.  See the C file for what each function computes and
which passage of the paper it follows.  Every function is pinned by the CPU
tests in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "rsv_oracle.c"), os.path.join(_HERE, "rsv_nested_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "librsv_oracle.so")
_lock = threading.Lock()
_lib = None

SL_ANNUITY, JL_REVERSIONARY, TERM_ASSURANCE, ENDOWMENT = 0, 1, 2, 3
JOINT_ANNUITY, LAST_SURVIVOR, JOINT_TERM, JOINT_ENDOWMENT = 4, 5, 6, 7
LS_TERM, LS_ENDOWMENT = 8, 9

CFLAGS = ["-std=gnu99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (idempotent).  Returns its path."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def use_library(path=None):
    """Load the oracle from ``path`` instead of the default build (None: back to the
    default).  Used by the mutation tests, which compile deliberately broken copies
    of the oracle source to show that the pins catch them."""
    global _lib
    with _lock:
        _lib = None
    if path is not None:
        _load(path)


def _load(path=None):
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(path or build())
            i32, i64, dp, ip = C.c_int32, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int32)
            lib.orc_n_states.argtypes = [C.c_int]
            lib.orc_transition.argtypes = [C.c_int, C.c_double, C.c_double, dp]
            lib.orc_cashflow.argtypes = [C.c_int, C.c_double, C.c_double, dp]
            lib.orc_steps.argtypes = [C.c_int] * 6 + [C.c_double, dp]
            lib.orc_chain.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_int, dp, dp, dp, dp, C.c_int, dp, dp, C.c_int, C.c_int, dp]
            lib.orc_reserves_batch.argtypes = [i64, ip, ip, ip, ip, ip, ip, ip, dp, dp,
                                               i32, i32, dp, i32, i32, dp, i32, i32, dp, dp]
            lib.orc_reserves_batch_method.argtypes = [i64, ip, ip, ip, ip, ip, ip, ip, dp, dp,
                                                      i32, i32, dp, i32, i32, dp, i32, i32, i32, dp, dp]
            lib.orc_chain_cf.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_int, dp, dp, dp, dp, C.c_int, dp, dp, dp, C.c_int, C.c_int, dp]
            lib.orc_reserves_batch_cf.argtypes = [i64, ip, ip, ip, ip, ip, ip, ip, dp, dp,
                                                  i32, i32, dp, i32, i32, dp, dp, i32, i32, i32, dp, dp]
            lib.orc_schedule.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                         C.c_double, dp]
            lib.orc_full_state.argtypes = [C.c_int, C.c_int]
            lib.orc_mlife_transition.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_mlife_chain.argtypes = [C.c_int, C.c_int, C.c_int, dp, ip, dp, dp, C.c_int, dp, dp]
            lib.orc_max_threads.restype = C.c_int
            if hasattr(lib, "orc_nested_node"):
                _bind_nested(lib)
            _lib = lib
    return _lib


def _bind_nested(lib):
    dp, ip, u32 = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_uint32
    lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.orc_gauss_pair.argtypes = [C.c_uint64, u32, u32, u32, u32, dp]
    lib.orc_vasicek_path.argtypes = [C.c_uint64, u32, u32, u32, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_int, dp, dp]
    lib.orc_nested_node.argtypes = [C.c_int64, ip, ip, dp, C.c_int32, C.c_int32, dp, C.c_uint64,
                                    C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                    C.c_int32, C.c_int32, ip, dp, dp, dp]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def n_states(product: int) -> int:
    return _load().orc_n_states(product)


def full_state(product: int, state0: int) -> int:
    """Index in the full state vector of a record's reduced valuation state."""
    return _load().orc_full_state(product, state0)


def transition(product: int, px: float, py: float = 0.0) -> np.ndarray:
    """Full-state W (row = state at the start, column = state at the end)."""
    n = n_states(product)
    W = np.zeros(n * n)
    _load().orc_transition(product, px, py, _p(W))
    return W.reshape(n, n)


def cashflow(product: int, amount: float, rho: float = 0.0) -> np.ndarray:
    n = n_states(product)
    c = np.zeros(n)
    _load().orc_cashflow(product, amount, rho, _p(c))
    return c


def steps(product: int, age1: int, age2: int, term: int, n_ages: int, horizon: int = 0,
          amount: float = 1.0):
    """(S, boundary vector r_S) of a policy."""
    rS = np.zeros(9)
    S = _load().orc_steps(product, age1, age2, term, n_ages, horizon, amount, _p(rS))
    return S, rS[: n_states(product)].copy()


def schedule(n_steps: int, every: int = 1, first: int = 0, since: int = 0, steps_per_year: int = 12,
             escalation: float = 0.0, increase: float = 0.0) -> np.ndarray:
    """Cash-flow multipliers c_t of a payment schedule (see ``orc_schedule``)."""
    cf = np.zeros(n_steps)
    st = _load().orc_schedule(n_steps, every, first, since, steps_per_year, escalation, increase, _p(cf))
    if st != 0:
        raise ValueError("bad schedule parameters")
    return cf


def mlife_transition(m: int, model: int, p) -> np.ndarray:
    """W^m of m lives (Section 4.3) for survival probabilities p[0..m-1]."""
    n = model ** m
    W = np.zeros(81 * 81)
    pp = _d(np.asarray(p, float).reshape(-1)) if m > 0 else np.zeros(1)
    if _load().orc_mlife_transition(m, model, _p(pp), _p(W)) != n:
        raise ValueError("bad m-life model")
    return W[: n * n].reshape(n, n)


def mlife_chain(m: int, model: int, tables, ages, c, rS, S: int, v) -> np.ndarray:
    """Reserve vectors r_t, t = 0..S, of an m-life contract: [S+1, model^m]."""
    n = model ** m
    tabs = np.atleast_2d(_d(tables))
    if tabs.shape[0] != m:
        raise ValueError("one table row per life")
    ag = _i(ages)
    cc, rr, vv = _d(c), _d(rS), _d(v)
    if len(cc) != n or len(rr) != n or len(vv) < S:
        raise ValueError("bad sizes")
    out = np.zeros((S + 1) * n)
    if _load().orc_mlife_chain(m, model, tabs.shape[1], _p(tabs), _p(ag, C.c_int32), _p(cc), _p(rr), S,
                               _p(vv), _p(out)) != n:
        raise ValueError("orc_mlife_chain failed")
    return out.reshape(S + 1, n)


def chain(product: int, age1: int, amount: float, table_x, v, *, age2: int = 0, term: int = 0,
          rho: float = 0.0, table_y=None, table_fx=None, table_fy=None, vf=None, cf=None,
          horizon: int = 0, method: str = "recurrence") -> np.ndarray:
    """Reserve vectors r_t, t = 0..S, of one policy under one discount sequence.

    Returns an array [S+1, n] (full state space).  ``table_fx``/``table_fy`` and
    ``vf`` give survival and discounting over the fraction f of a step; they
    default to the one-step ones (f = 1).  ``cf`` (length >= S) scales the
    nominal cash-flow vector of each step (default: level).
    """
    lib = _load()
    tx = _d(table_x)
    ty = _d(table_y) if table_y is not None else tx
    tfx = _d(table_fx) if table_fx is not None else tx
    tfy = _d(table_fy) if table_fy is not None else (ty if table_fx is None else tfx)
    v = _d(v)
    vf = _d(vf) if vf is not None else v
    n = n_states(product)
    out = np.zeros((len(v) + 1) * n)
    m = {"recurrence": 0, "summation": 1}[method]
    cfa = None
    if cf is not None:
        cfa = np.zeros(len(v))
        cfa[: min(len(v), len(cf))] = _d(cf)[: len(v)]
    S = lib.orc_chain_cf(product, age1, age2, term, amount, rho, len(tx), _p(tx), _p(ty), _p(tfx),
                         _p(tfy), len(v), _p(v), _p(vf), _p(cfa) if cfa is not None else None, horizon, m,
                         _p(out))
    if S < 0:
        raise ValueError(f"orc_chain failed with code {S}")
    return out[: (S + 1) * n].reshape(S + 1, n)


def reserves_batch(pol: dict, tables, v, horizon: int = 0, nthreads: int = 0, totals: bool = True,
                   method: str = "recurrence", cf=None):
    """V0[p, s] (FP64) of every policy in every scenario, f = 1, by the recurrence
    (or, with ``method="summation"``, by the summation definition at every step).

    ``pol`` is a dict of arrays as made by ``synth``; ``tables`` is [n_tables,
    n_ages] or [n_ages]; ``v`` is [n_scen, n_steps]; ``cf`` (optional) is
    [n_pol, n_steps] cash-flow multipliers.  Returns (V0, scen_total).
    """
    lib = _load()
    tables = np.atleast_2d(_d(tables))
    v = np.atleast_2d(_d(v))
    n = len(pol["product"])
    V0 = np.zeros((n, v.shape[0]))
    tot = np.zeros(v.shape[0]) if totals else None
    a = {k: _i(pol[k]) for k in ("product", "age1_m", "age2_m", "term_m", "state0", "table1", "table2")}
    amount, rho = _d(pol["amount"]), _d(pol["reversion"])
    m = {"recurrence": 0, "summation": 1}[method]
    cfa = None
    if cf is not None:
        cfa = _d(cf)
        if cfa.shape != (n, v.shape[1]):
            raise ValueError("cf must be [n_pol, n_steps]")
    st = lib.orc_reserves_batch_cf(n, _p(a["product"], C.c_int32), _p(a["age1_m"], C.c_int32),
                                   _p(a["age2_m"], C.c_int32), _p(a["term_m"], C.c_int32),
                                   _p(a["state0"], C.c_int32), _p(a["table1"], C.c_int32),
                                   _p(a["table2"], C.c_int32), _p(amount), _p(rho),
                                   tables.shape[0], tables.shape[1], _p(tables), v.shape[0], v.shape[1],
                                   _p(v), _p(cfa) if cfa is not None else None, horizon, nthreads, m, _p(V0),
                                   _p(tot) if totals else None)
    if st != 0:
        raise ValueError(f"orc_reserves_batch failed with code {st}")
    return V0, tot


def max_threads() -> int:
    return _load().orc_max_threads()


# ------------------------------------------------------------------ nested ----
STREAM_OUTER, STREAM_INNER = 2, 3


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    _load().orc_philox4x32_10(c, k, out)
    return [int(x) for x in out]


def gauss_pairs(seed, k, c1, c2, c3):
    z = np.zeros(4)
    _load().orc_gauss_pair(seed, k, c1, c2, c3, _p(z))
    return z


def vasicek_path(seed, c1, c2, c3, n_steps, r_start, a=0.1, b=0.04, sigma=0.01):
    """(v[0..n_steps), r after n_steps) of one counter-based Vasicek path."""
    v = np.zeros(max(1, n_steps))
    r = C.c_double()
    _load().orc_vasicek_path(seed, c1, c2, c3, a, b, sigma, r_start, n_steps, _p(v), C.byref(r))
    return v[:n_steps], r.value


def outer_path(seed, o, n_steps, r0=0.03, a=0.1, b=0.04, sigma=0.01):
    return vasicek_path(seed, o, 0, STREAM_OUTER << 24, n_steps, r0, a, b, sigma)


def inner_path(seed, o, n, i, n_steps, r_start, a=0.1, b=0.04, sigma=0.01):
    return vasicek_path(seed, i, n, (STREAM_INNER << 24) | o, n_steps, r_start, a, b, sigma)


def nested_node(pol, tables, seed, o, n, idx, node_step=12, a=0.1, b=0.04, sigma=0.01, r0=0.03):
    """Liabilities L_{o,n,i} (FP64) for the inner paths ``idx`` of node n of outer
    path o, and (rate at the node, discount product 0 -> node)."""
    lib = _load()
    tables = np.atleast_2d(_d(tables))
    nn = len(pol["product"])
    ipol = np.ascontiguousarray(np.stack([pol["age1_m"], pol["age2_m"], pol["term_m"], pol["state0"],
                                          pol["table1"], pol["table2"]], axis=1).astype(np.int32))
    dpol = np.ascontiguousarray(np.stack([pol["amount"], pol["reversion"]], axis=1).astype(np.float64))
    prod = _i(pol["product"])
    idx = _i(np.atleast_1d(idx))
    L = np.zeros(len(idx))
    rn, d0 = C.c_double(), C.c_double()
    st = lib.orc_nested_node(nn, _p(prod, C.c_int32), _p(ipol, C.c_int32), _p(dpol), tables.shape[0],
                             tables.shape[1], _p(tables), seed, a, b, sigma, r0, node_step, o, n, len(idx),
                             _p(idx, C.c_int32), _p(L), C.byref(rn), C.byref(d0))
    if st != 0:
        raise ValueError(f"orc_nested_node failed with code {st}")
    return L, rn.value, d0.value
