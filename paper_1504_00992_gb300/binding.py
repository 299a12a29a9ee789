"""Thin ctypes binding of libtebd_gb300.so (include/tebd_gb300.h).

Every function here marshals arguments and calls the C ABI function of the
same name; all arithmetic of the bond update runs in the library's CUDA
kernels.  There is no fallback: if the library is missing, or no CUDA device
is present when a compute call is made, an exception is raised.

Arrays: host complex data are numpy complex128 (interleaved re, im), device
data are passed as raw integer addresses (e.g. torch.Tensor.data_ptr()).
"""
import ctypes
import os

import numpy as np

from . import build as _build

TEBD_OK = 0
TEBD_EINVAL = -1
TEBD_ENOMEM = -2
TEBD_ECUDA = -3
TEBD_ENUMERIC = -4
TEBD_ETIMEOUT = -5
TEBD_ENOTIMPL = -6
TEBD_ESTATE = -7
TEBD_PREC_FP64 = 0
TEBD_PREC_TF32 = 2
TEBD_PREC_BF16 = 3

_CODES = {0: "TEBD_OK", -1: "TEBD_EINVAL", -2: "TEBD_ENOMEM", -3: "TEBD_ECUDA", -4: "TEBD_ENUMERIC",
          -5: "TEBD_ETIMEOUT", -6: "TEBD_ENOTIMPL", -7: "TEBD_ESTATE"}


class TebdError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{_CODES.get(code, code)}: {msg}")


# tebd_alloc_fn / tebd_release_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

TEBD_FAULT_NONE = 0
TEBD_FAULT_ALLOC = 1
TEBD_FAULT_TC_STALL = 2


class TebdDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("d", ctypes.c_int), ("d_site", ctypes.POINTER(ctypes.c_int)),
                ("chi_max", ctypes.c_int), ("chi_bond", ctypes.POINTER(ctypes.c_int)),
                ("p", ctypes.c_int), ("q", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("sv_cutoff", ctypes.c_double), ("chain", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int), ("workspace_budget", ctypes.c_size_t),
                ("alloc", ALLOC_FN), ("release", RELEASE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("fused", ctypes.c_int)]


class TorchAllocator:
    """Device blocks of a TEBD handle from PyTorch's CUDA caching allocator
    (torch.cuda.caching_allocator_alloc / _delete), so that the handle's
    arena, checkpoints and reverse-pass buffers share the caller's memory
    pool.  Keep the object alive as long as a handle uses it; `live` maps the
    blocks it has handed out to their sizes."""

    def __init__(self, device=None, stream=None):
        import torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, ctx):
            try:
                ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:   # out of memory: the library sees NULL
                return None
            self.live[ptr] = int(nbytes)
            return ptr

        def _release(ptr, ctx):
            if ptr:
                self.live.pop(int(ptr), None)
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.release = RELEASE_FN(_release)


_LIB = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_d = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "tebd_create": (_i, [_i, _i, _i, _i, _i, _u64, ctypes.POINTER(_vp)]),
    "tebd_create_ex": (_i, [ctypes.POINTER(TebdDesc), ctypes.POINTER(_vp)]),
    "tebd_create_multi": (_i, [_i, ctypes.POINTER(TebdDesc), ctypes.POINTER(_vp)]),
    "tebd_num_chains": (_i, [_vp, _pi]),
    "tebd_select_chain": (_i, [_vp, _i]),
    "tebd_workspace_info": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t), _pi, _pi]),
    "tebd_wave_info": (_i, [_vp, _i, _i, _pi, _pd]),
    "tebd_plan_query": (_i, [_i, ctypes.POINTER(TebdDesc), ctypes.POINTER(ctypes.c_size_t), _pi, _pi]),
    "tebd_destroy": (_i, [_vp]),
    "tebd_set_stream": (_i, [_vp, _vp]),
    "tebd_set_allocator": (_i, [_vp, ALLOC_FN, RELEASE_FN, _vp]),
    "tebd_set_sweep_count": (_i, [_vp, _i64]),
    "tebd_bond_weights": (_i, [_vp, _pd]),
    "tebd_fault_inject": (_i, [_i]),
    "rrsvd_clear_error": (_i, [_vp]),
    "rrsvd_plan_autotune": (_i, [_vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "rrsvd_plan_tuning": (_i, [_vp, _pi, _pd]),
    "rrsvd_plan_set_tuning": (_i, [_vp, _pi]),
    "tebd_set_product_state": (_i, [_vp, _pd]),
    "tebd_set_mps": (_i, [_vp, ctypes.POINTER(_pd), ctypes.POINTER(_pd), _pi]),
    "tebd_get_mps": (_i, [_vp, ctypes.POINTER(_pd), ctypes.POINTER(_pd), _pi]),
    "tebd_set_gates": (_i, [_vp, _i, _pd]),
    "tebd_step_even": (_i, [_vp]),
    "tebd_step_odd": (_i, [_vp]),
    "tebd_expect": (_i, [_vp, _i, _pd, _pd]),
    "tebd_get_lambda": (_i, [_vp, _i, _pd, _pi]),
    "tebd_discarded_weight": (_i, [_vp, _pd]),
    "tebd_sweep_count": (_i, [_vp, ctypes.POINTER(_i64)]),
    "tebd_backward": (_i, [_vp, _i, _pd, _pd, _pd]),
    "tebd_record": (_i, [_vp, _i]),
    "tebd_last_error": (ctypes.c_char_p, [_vp]),
    "rrsvd_plan_create": (_i, [_i, _i, _i, _i, _i, _i, _i, _u64, ctypes.POINTER(_vp)]),
    "rrsvd_plan_destroy": (_i, [_vp]),
    "rrsvd_plan_create_ex": (_i, [_i, _i, _i, _i, _i, _i, _i, _u64, _i, _d, _i, ctypes.POINTER(_vp)]),
    "rrsvd_plan_widths": (_i, [_vp, _pi]),
    "rrsvd_workspace_size": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "rrsvd_plan_dims": (_i, [_vp, _pi, _pi]),
    "rrsvd_execute": (_i, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "rrsvd_execute_host": (_i, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rrsvd_execute_host_async": (_i, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rrsvd_host_wait": (_i, [_vp]),
    "rrsvd_last_error": (ctypes.c_char_p, [_vp]),
    "rrsvd_execute_noalloc": (_i, [_i, _i, _i, _i, _i, _i, _u64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tebd_philox4x64_10": (_i, [_vp, _i64, _u64, _u64, _vp, _vp]),
    "rrsvd_sketch_omega": (_i, [_i, _i, _u64, _i64, _i64, _i64, _i, _vp, _vp]),
    "tebd_profiler_enable": (_i, [_i]),
    "tebd_profiler_reset": (_i, []),
    "tebd_profiler_read": (_i, [_i, ctypes.c_char_p, _pd, ctypes.POINTER(_i64), _pi]),
}


def header_functions():
    """Names of the functions declared in include/tebd_gb300.h."""
    import re
    path = os.path.join(_build.ROOT, "include", "tebd_gb300.h")
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tebd_\w+|rrsvd_\w+)\s*\(", txt)))


def load(path=None):
    """Load the library (built in-tree by __graft_entry__.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _c128(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _dp(a):
    return a.ctypes.data_as(_pd)


# ------------------------------------------------------------------ TEBD
def _check(h, rc):
    if rc != TEBD_OK:
        msg = load().tebd_last_error(h) if h else b""
        raise TebdError(rc, (msg or b"").decode())


def tebd_create(N, d, chi_max, p, q, seed):
    h = _vp()
    rc = load().tebd_create(N, d, chi_max, p, q, seed, ctypes.byref(h))
    if rc != TEBD_OK:
        raise TebdError(rc, "tebd_create")
    return h


_KEEP = []


def _desc(N, d_site, chi_bond, p, q, seed, precision=TEBD_PREC_FP64, sv_cutoff=0.0, chain=0, use_graph=0,
          autotune=0, workspace_budget=0, allocator=None, fused=0):
    ds = (ctypes.c_int * N)(*[int(x) for x in d_site])
    cb = (ctypes.c_int * (N - 1))(*[int(x) for x in chi_bond])
    _KEEP.append((ds, cb))
    d = TebdDesc(N, int(d_site[0]), ds, int(max(chi_bond)), cb, p, q, seed, precision, sv_cutoff, chain,
                 use_graph, autotune, workspace_budget)
    if allocator is not None:
        d.alloc = allocator.alloc
        d.release = allocator.release
    d.fused = fused
    return d


def tebd_create_ex(N, d_site, chi_bond, p, q, seed, precision=TEBD_PREC_FP64, sv_cutoff=0.0, chain=0, use_graph=0,
                   autotune=0, workspace_budget=0, allocator=None, fused=0):
    desc = _desc(N, d_site, chi_bond, p, q, seed, precision, sv_cutoff, chain, use_graph, autotune,
                 workspace_budget, allocator, fused)
    h = _vp()
    rc = load().tebd_create_ex(ctypes.byref(desc), ctypes.byref(h))
    _KEEP.clear()
    if rc != TEBD_OK:
        raise TebdError(rc, "tebd_create_ex")
    return h


def tebd_create_multi(chains, p, q, seed, precision=TEBD_PREC_FP64, sv_cutoff=0.0, chain=0, use_graph=0,
                      autotune=0, workspace_budget=0, allocator=None, fused=0):
    """chains: list of (N, d_site list, chi_bond list)."""
    arr = (TebdDesc * len(chains))()
    for c, (N, d_site, chi_bond) in enumerate(chains):
        arr[c] = _desc(N, d_site, chi_bond, p, q, seed, precision, sv_cutoff, chain, use_graph, autotune,
                       workspace_budget, allocator if c == 0 else None, fused)
    h = _vp()
    rc = load().tebd_create_multi(len(chains), arr, ctypes.byref(h))
    _KEEP.clear()
    if rc != TEBD_OK:
        raise TebdError(rc, "tebd_create_multi")
    return h


def tebd_plan_query(chains, p, q, seed, precision=TEBD_PREC_FP64, autotune=0, workspace_budget=0):
    """The (arena bytes, waves even, waves odd) that tebd_create_multi would
    plan for these chains, computed on the host without a GPU."""
    arr = (TebdDesc * max(1, len(chains)))()
    for c, (N, d_site, chi_bond) in enumerate(chains):
        arr[c] = _desc(N, d_site, chi_bond, p, q, seed, precision, 0.0, 0, 0, autotune, workspace_budget)
    b, we, wo = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
    rc = load().tebd_plan_query(len(chains), arr, ctypes.byref(b), ctypes.byref(we), ctypes.byref(wo))
    _KEEP.clear()
    if rc != TEBD_OK:
        raise TebdError(rc, "tebd_plan_query")
    return b.value, we.value, wo.value


def tebd_num_chains(h):
    n = ctypes.c_int()
    _check(h, load().tebd_num_chains(h, ctypes.byref(n)))
    return n.value


def tebd_select_chain(h, chain):
    _check(h, load().tebd_select_chain(h, chain))


def tebd_workspace_info(h):
    b, we, wo = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
    _check(h, load().tebd_workspace_info(h, ctypes.byref(b), ctypes.byref(we), ctypes.byref(wo)))
    return b.value, we.value, wo.value


def tebd_wave_info(h, parity, wave):
    """Dict of one wave's plan and tuning (tebd_wave_info)."""
    info = (ctypes.c_int * 20)()
    ms = (ctypes.c_double * 2)()
    _check(h, load().tebd_wave_info(h, parity, wave, info, ms))
    return {"bonds": info[0], "m": info[1], "n": info[2], "k": info[3], "l": info[4], "fused": info[5],
            "tiles": list(info[6:12]), "mixed": {"tc_half": info[12], "qr_threads": info[13], "qrbh": info[14],
                                                 "jacobi": info[15], "products": info[16]},
            "tune_ms": [ms[0], ms[1]]}


def tebd_tuning_table(h):
    """Every wave's plan and tuning, both parities."""
    _, we, wo = tebd_workspace_info(h)
    return {par: [tebd_wave_info(h, par, w) for w in range(n)] for par, n in ((0, we), (1, wo))}


def tebd_destroy(h):
    load().tebd_destroy(h)


def tebd_set_stream(h, stream_ptr):
    _check(h, load().tebd_set_stream(h, _vp(int(stream_ptr))))


def tebd_set_allocator(h, allocator=None):
    """Moves the handle's device memory to `allocator` (an object with ctypes
    callbacks .alloc / .release, e.g. TorchAllocator), or back to cudaMalloc
    when None.  The caller keeps `allocator` alive while the handle uses it."""
    if allocator is None:
        _check(h, load().tebd_set_allocator(h, ALLOC_FN(), RELEASE_FN(), None))
    else:
        _check(h, load().tebd_set_allocator(h, allocator.alloc, allocator.release, None))


def tebd_set_sweep_count(h, count):
    _check(h, load().tebd_set_sweep_count(h, int(count)))


def tebd_bond_weights(h, n_bonds):
    out = np.zeros(n_bonds, dtype=np.float64)
    _check(h, load().tebd_bond_weights(h, _dp(out)))
    return out


def tebd_fault_inject(kind):
    rc = load().tebd_fault_inject(kind)
    if rc != TEBD_OK:
        raise TebdError(rc, "tebd_fault_inject")


def tebd_set_product_state(h, psis):
    flat = _c128(np.concatenate([np.ravel(np.asarray(v, dtype=np.complex128)) for v in psis]))
    _check(h, load().tebd_set_product_state(h, _dp(flat.view(np.float64))))


def tebd_set_mps(h, gammas, lambdas):
    gs = [_c128(g) for g in gammas]
    ls = [np.ascontiguousarray(np.asarray(l, dtype=np.float64)) for l in lambdas]
    chi = (ctypes.c_int * len(ls))(*[len(l) for l in ls])
    gp = (_pd * len(gs))(*[_dp(g.view(np.float64)) for g in gs])
    lp = (_pd * len(ls))(*[_dp(l) for l in ls])
    _check(h, load().tebd_set_mps(h, gp, lp, chi))


def tebd_get_mps(h, dims, caps):
    """dims: local dimensions (N); caps: bond capacities (N-1).  Returns
    (gammas, lambdas) with the current bond dimensions."""
    N = len(dims)
    ext = [1] + list(caps) + [1]
    gbufs = [np.zeros(dims[s] * ext[s] * ext[s + 1], dtype=np.complex128) for s in range(N)]
    lbufs = [np.zeros(c, dtype=np.float64) for c in caps]
    chi = (ctypes.c_int * (N - 1))()
    gp = (_pd * N)(*[_dp(g.view(np.float64)) for g in gbufs])
    lp = (_pd * (N - 1))(*[_dp(l) for l in lbufs])
    _check(h, load().tebd_get_mps(h, gp, lp, chi))
    ce = [1] + list(chi) + [1]
    gammas = [gbufs[s][: dims[s] * ce[s] * ce[s + 1]].reshape(dims[s], ce[s], ce[s + 1]) for s in range(N)]
    lambdas = [lbufs[b][: ce[b + 1]] for b in range(N - 1)]
    return gammas, lambdas


def tebd_set_gates(h, parity, gates):
    flat = _c128(np.concatenate([np.ravel(_c128(g)) for g in gates]))
    _check(h, load().tebd_set_gates(h, parity, _dp(flat.view(np.float64))))


def tebd_step_even(h):
    _check(h, load().tebd_step_even(h))


def tebd_step_odd(h):
    _check(h, load().tebd_step_odd(h))


def tebd_expect(h, site, op):
    o = _c128(op)
    out = np.zeros(2, dtype=np.float64)
    _check(h, load().tebd_expect(h, site, _dp(o.view(np.float64)), _dp(out)))
    return complex(out[0], out[1])


def tebd_get_lambda(h, bond, cap):
    out = np.zeros(cap, dtype=np.float64)
    chi = ctypes.c_int()
    _check(h, load().tebd_get_lambda(h, bond, _dp(out), ctypes.byref(chi)))
    return out[: chi.value].copy()


def tebd_discarded_weight(h):
    out = np.zeros(2, dtype=np.float64)
    _check(h, load().tebd_discarded_weight(h, _dp(out)))
    return float(out[0]), float(out[1])


def tebd_sweep_count(h):
    c = ctypes.c_int64()
    _check(h, load().tebd_sweep_count(h, ctypes.byref(c)))
    return c.value


def tebd_record(h, on=True):
    _check(h, load().tebd_record(h, 1 if on else 0))


def tebd_backward(h, site, op, dims):
    """Gate cotangents of L = Re <op_site>: returns (even, odd), each a list of
    N-1 complex (d_b d_{b+1})^2 matrices (zero for the other parity)."""
    sizes = [(dims[b] * dims[b + 1]) for b in range(len(dims) - 1)]
    tot = sum(x * x for x in sizes)
    ge = np.zeros(tot, dtype=np.complex128)
    go = np.zeros(tot, dtype=np.complex128)
    o = _c128(op)
    _check(h, load().tebd_backward(h, site, _dp(o.view(np.float64)), _dp(ge.view(np.float64)),
                                   _dp(go.view(np.float64))))
    out = []
    for arr in (ge, go):
        mats, off = [], 0
        for x in sizes:
            mats.append(arr[off:off + x * x].reshape(x, x).copy())
            off += x * x
        out.append(mats)
    return out[0], out[1]


def tebd_last_error(h):
    return (load().tebd_last_error(h) or b"").decode()


# ------------------------------------------------------------------ RRSVD
def _pcheck(plan, rc):
    if rc != TEBD_OK:
        msg = load().rrsvd_last_error(plan) if plan else b""
        raise TebdError(rc, (msg or b"").decode())


def rrsvd_plan_create(m, n, k_max, p, q, batch, precision=TEBD_PREC_FP64, seed=0):
    h = _vp()
    rc = load().rrsvd_plan_create(m, n, k_max, p, q, batch, precision, seed, ctypes.byref(h))
    if rc != TEBD_OK:
        raise TebdError(rc, "rrsvd_plan_create")
    return h


def rrsvd_plan_create_ex(m, n, k_max, p, q, batch, precision=TEBD_PREC_FP64, seed=0, check_r=0, check_eps=0.0,
                         l_max=0):
    h = _vp()
    rc = load().rrsvd_plan_create_ex(m, n, k_max, p, q, batch, precision, seed, check_r, check_eps, l_max,
                                     ctypes.byref(h))
    if rc != TEBD_OK:
        raise TebdError(rc, "rrsvd_plan_create_ex")
    return h


def rrsvd_plan_widths(plan, batch):
    out = (ctypes.c_int * batch)()
    _pcheck(plan, load().rrsvd_plan_widths(plan, out))
    return list(out)


def rrsvd_plan_destroy(plan):
    load().rrsvd_plan_destroy(plan)           # finishes pending asynchronous calls first
    _IN_FLIGHT.pop(plan.value, None)


def rrsvd_workspace_size(plan):
    s = ctypes.c_size_t()
    _pcheck(plan, load().rrsvd_workspace_size(plan, ctypes.byref(s)))
    return s.value


def rrsvd_plan_dims(plan):
    k, l = ctypes.c_int(), ctypes.c_int()
    _pcheck(plan, load().rrsvd_plan_dims(plan, ctypes.byref(k), ctypes.byref(l)))
    return k.value, l.value


def rrsvd_execute(plan, theta_ptr, chain0, sigma_ptr, U_ptr, Vh_ptr, w_ptr, rank_ptr, ws_ptr, ws_bytes, stream_ptr=0):
    """Device-pointer call (integers, 0 for NULL)."""
    def vp(x):
        return _vp(int(x)) if x else None
    _pcheck(plan, load().rrsvd_execute(plan, vp(theta_ptr), chain0, vp(sigma_ptr), vp(U_ptr), vp(Vh_ptr), vp(w_ptr),
                                       vp(rank_ptr), vp(ws_ptr), ws_bytes, vp(stream_ptr)))


def _host_buffers(plan, theta, sigma, U, Vh, w, rank):
    """Addresses of a host-buffer call's numpy arrays, after checking what the
    library will read and write through them: theta (batch, m, n) complex128,
    sigma (batch, k) float64, U (batch, m, k) and Vh (batch, k, n) complex128,
    w (batch,) float64, rank (batch,) int32 (k from the plan), each C-ordered
    and the outputs writeable; the optional ones may be None.  The library
    reads and writes exactly these extents, so a mismatch is refused here
    (TEBD_EINVAL) instead of touching memory past a buffer."""
    if theta is None or sigma is None:
        raise TebdError(TEBD_EINVAL, "theta and sigma are required")
    if np.ndim(theta) != 3:
        raise TebdError(TEBD_EINVAL, "theta must be (batch, m, n)")
    k, _ = rrsvd_plan_dims(plan)
    batch, m, n = theta.shape
    want = (("theta", theta, np.complex128, batch * m * n, False), ("sigma", sigma, np.float64, batch * k, True),
            ("U", U, np.complex128, batch * m * k, True), ("Vh", Vh, np.complex128, batch * k * n, True),
            ("w", w, np.float64, batch, True), ("rank", rank, np.int32, batch, True))
    out = []
    for name, a, dt, size, written in want:
        if a is None:
            out.append(None)
            continue
        if not isinstance(a, np.ndarray) or a.dtype != dt or not a.flags.c_contiguous or a.size != size:
            raise TebdError(TEBD_EINVAL, f"{name}: a C-ordered {np.dtype(dt).name} array of {size} elements is "
                                         f"needed")
        if written and not a.flags.writeable:
            raise TebdError(TEBD_EINVAL, f"{name} is read-only")
        out.append(_vp(a.ctypes.data))
    return out


# arrays of rrsvd_execute_host_async calls still in flight, per plan address:
# kept alive here until the plan's next wait
_IN_FLIGHT = {}


def rrsvd_execute_host(plan, theta, chain0, sigma, U=None, Vh=None, w=None, rank=None, stream_ptr=0):
    """Host-buffer call: theta (batch, m, n) complex128 in, results written
    into the given numpy arrays (contiguous; pinned memory recommended).  It
    waits for the plan's pending asynchronous calls first."""
    bufs = _host_buffers(plan, theta, sigma, U, Vh, w, rank)
    try:
        _pcheck(plan, load().rrsvd_execute_host(plan, bufs[0], chain0, *bufs[1:],
                                                _vp(int(stream_ptr)) if stream_ptr else None))
    finally:
        _IN_FLIGHT.pop(plan.value, None)


def rrsvd_execute_host_async(plan, theta, chain0, sigma, U=None, Vh=None, w=None, rank=None, stream_ptr=0):
    """Enqueued host-buffer call (rrsvd_execute_host_async): the outputs are
    valid after rrsvd_host_wait(plan); theta must not change before then.  The
    binding holds the arrays until that wait."""
    bufs = _host_buffers(plan, theta, sigma, U, Vh, w, rank)
    _IN_FLIGHT.setdefault(plan.value, []).append((theta, sigma, U, Vh, w, rank))
    _pcheck(plan, load().rrsvd_execute_host_async(plan, bufs[0], chain0, *bufs[1:],
                                                  _vp(int(stream_ptr)) if stream_ptr else None))


def rrsvd_host_wait(plan):
    try:
        _pcheck(plan, load().rrsvd_host_wait(plan))
    finally:
        _IN_FLIGHT.pop(plan.value, None)


def rrsvd_execute_noalloc(m, n, k_max, p, q, batch, seed, chain0, theta_ptr, sigma_ptr, U_ptr=0, Vh_ptr=0,
                          w_ptr=0, rank_ptr=0, stream_ptr=0):
    """No-allocation truncation on device buffers (integers, 0 for NULL):
    same results as rrsvd_execute with a plan of the same sizes; scratch is a
    fixed 16 MiB array inside the library shared by every call."""
    def vp(x):
        return _vp(int(x)) if x else None
    rc = load().rrsvd_execute_noalloc(m, n, k_max, p, q, batch, seed, chain0, vp(theta_ptr), vp(sigma_ptr),
                                      vp(U_ptr), vp(Vh_ptr), vp(w_ptr), vp(rank_ptr), vp(stream_ptr))
    if rc != TEBD_OK:
        raise TebdError(rc, "rrsvd_execute_noalloc")


def tebd_philox4x64_10(counters_ptr, count, key0, key1, words_ptr, stream_ptr=0):
    """Philox4x64-10 blocks of the library's sketch generator on device
    buffers (integer addresses of 4 * count uint64 each)."""
    rc = load().tebd_philox4x64_10(_vp(int(counters_ptr)) if counters_ptr else None, count, key0 & (2**64 - 1),
                                   key1 & (2**64 - 1), _vp(int(words_ptr)) if words_ptr else None,
                                   _vp(int(stream_ptr)) if stream_ptr else None)
    if rc != TEBD_OK:
        raise TebdError(rc, "tebd_philox4x64_10")


def rrsvd_sketch_omega(n, l, seed, bond, sweep, chain, precision, out_ptr, stream_ptr=0):
    """The n x l sketch matrix (row-major, device buffer: complex128 for the
    FP64 form, complex64 for the mixed form) exactly as the sketch draws it."""
    rc = load().rrsvd_sketch_omega(n, l, seed & (2**64 - 1), bond, sweep, chain, precision,
                                   _vp(int(out_ptr)) if out_ptr else None,
                                   _vp(int(stream_ptr)) if stream_ptr else None)
    if rc != TEBD_OK:
        raise TebdError(rc, "rrsvd_sketch_omega")


def rrsvd_last_error(plan):
    return (load().rrsvd_last_error(plan) or b"").decode()


def rrsvd_clear_error(plan):
    _pcheck(plan, load().rrsvd_clear_error(plan))


def rrsvd_plan_autotune(plan, theta_ptr, ws_ptr, ws_bytes, stream_ptr=0):
    """Time the plan's launch choices on device theta and keep the fastest."""
    def vp(x):
        return _vp(int(x)) if x else None
    _pcheck(plan, load().rrsvd_plan_autotune(plan, vp(theta_ptr), vp(ws_ptr), ws_bytes, vp(stream_ptr)))


def rrsvd_plan_tuning(plan):
    info = (ctypes.c_int * 16)()
    ms = (ctypes.c_double * 2)()
    _pcheck(plan, load().rrsvd_plan_tuning(plan, info, ms))
    return {"tiles": list(info[0:6]), "tc_half": info[6], "qr_threads": info[7], "qrbh": info[8], "jacobi": info[9],
            "tuned": info[10], "products": info[11], "ms_rules": ms[0], "ms_kept": ms[1]}


def rrsvd_plan_set_tuning(plan, choices):
    """Sets a plan's launch choices from a dict laid out as rrsvd_plan_tuning's."""
    info = (ctypes.c_int * 16)()
    info[0:6] = [int(x) for x in choices.get("tiles", [0] * 6)]
    info[6] = int(choices.get("tc_half", 0))
    info[7] = int(choices.get("qr_threads", 0))
    info[8] = int(choices.get("qrbh", 0))
    info[9] = int(choices.get("jacobi", 0))
    info[11] = int(choices.get("products", 0))
    _pcheck(plan, load().rrsvd_plan_set_tuning(plan, info))


# ------------------------------------------------------------------ kernel timing
def tebd_profiler_enable(on=True):
    load().tebd_profiler_enable(1 if on else 0)


def tebd_profiler_reset():
    load().tebd_profiler_reset()


def tebd_profiler_read():
    """{kernel class: (total ms, launches)} accumulated since the last reset."""
    L = load()
    cnt = ctypes.c_int()
    L.tebd_profiler_read(0, None, None, None, ctypes.byref(cnt))
    n = cnt.value
    if n == 0:
        return {}
    names = ctypes.create_string_buffer(64 * n)
    ms = np.zeros(n, dtype=np.float64)
    nl = np.zeros(n, dtype=np.int64)
    L.tebd_profiler_read(n, names, _dp(ms), nl.ctypes.data_as(ctypes.POINTER(_i64)), ctypes.byref(cnt))
    out = {}
    for i in range(n):
        nm = names.raw[64 * i: 64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(nl[i]))
    return out


# ------------------------------------------------------------------ convenience wrappers
class Tebd:
    """Owning wrapper of a tebd_t handle (the calls above, bound to one chain)."""

    def __init__(self, N, d, chi_max, p, q, seed=0, d_site=None, chi_bond=None, sv_cutoff=0.0, chain=0,
                 stream=None, use_graph=0, autotune=0, precision=TEBD_PREC_FP64, workspace_budget=0,
                 allocator=None, fused=0):
        self.N = N
        self.dims = list(d_site) if d_site is not None else [d] * N
        self.chi_bond = list(chi_bond) if chi_bond is not None else [chi_max] * (N - 1)
        self.allocator = allocator
        if d_site is None and chi_bond is None and sv_cutoff == 0.0 and chain == 0 and not use_graph \
                and not autotune and precision == TEBD_PREC_FP64 and not workspace_budget and allocator is None \
                and not fused:
            self.h = tebd_create(N, d, chi_max, p, q, seed)
        else:
            self.h = tebd_create_ex(N, self.dims, self.chi_bond, p, q, seed, precision, sv_cutoff, chain,
                                    use_graph, autotune, workspace_budget, allocator, fused)
        caps = []
        for b in range(N - 1):
            left = int(np.prod([float(x) for x in self.dims[: b + 1]]))
            right = int(np.prod([float(x) for x in self.dims[b + 1:]]))
            caps.append(int(min(self.chi_bond[b], left, right)))
        self.caps = caps
        if stream is not None:
            tebd_set_stream(self.h, stream)

    def close(self):
        if self.h:
            tebd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_product_state(self, psis):
        tebd_set_product_state(self.h, psis)

    def set_mps(self, gammas, lambdas):
        tebd_set_mps(self.h, gammas, lambdas)

    def get_mps(self):
        return tebd_get_mps(self.h, self.dims, self.caps)

    def set_gates(self, parity, gates):
        tebd_set_gates(self.h, parity, gates)

    def step_even(self):
        tebd_step_even(self.h)

    def step_odd(self):
        tebd_step_odd(self.h)

    def expect(self, site, op):
        return tebd_expect(self.h, site, op)

    def get_lambda(self, bond):
        return tebd_get_lambda(self.h, bond, self.caps[bond])

    def discarded_weight(self):
        return tebd_discarded_weight(self.h)

    def sweeps(self):
        return tebd_sweep_count(self.h)

    def set_sweep_count(self, count):
        tebd_set_sweep_count(self.h, count)

    def bond_weights(self):
        return tebd_bond_weights(self.h, self.N - 1)

    def set_allocator(self, allocator):
        tebd_set_allocator(self.h, allocator)
        self.allocator = allocator

    def record(self, on=True):
        tebd_record(self.h, on)

    def backward(self, site, op):
        return tebd_backward(self.h, site, op, self.dims)

    def tuning_table(self):
        return tebd_tuning_table(self.h)


def _caps(dims, chi_bond):
    caps = []
    N = len(dims)
    for b in range(N - 1):
        left = float(np.prod([float(x) for x in dims[: b + 1]]))
        right = float(np.prod([float(x) for x in dims[b + 1:]]))
        caps.append(int(min(chi_bond[b], left, right)))
    return caps


class MultiTebd:
    """Many chains in one handle; per-chain calls take the chain index."""

    def __init__(self, chains, p, q, seed=0, use_graph=0, autotune=0, workspace_budget=0, stream=None,
                 precision=TEBD_PREC_FP64, allocator=None, fused=0):
        self.chains = [(N, list(ds), list(cb)) for N, ds, cb in chains]
        self.allocator = allocator
        self.h = tebd_create_multi(self.chains, p, q, seed, precision=precision, use_graph=use_graph,
                                   autotune=autotune, workspace_budget=workspace_budget, allocator=allocator,
                                   fused=fused)
        self.caps = [_caps(ds, cb) for _, ds, cb in self.chains]
        if stream is not None:
            tebd_set_stream(self.h, stream)

    def close(self):
        if self.h:
            tebd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sel(self, c):
        tebd_select_chain(self.h, c)

    def set_product_state(self, c, psis):
        self._sel(c)
        tebd_set_product_state(self.h, psis)

    def set_gates(self, c, parity, gates):
        self._sel(c)
        tebd_set_gates(self.h, parity, gates)

    def step_even(self):
        tebd_step_even(self.h)

    def step_odd(self):
        tebd_step_odd(self.h)

    def expect(self, c, site, op):
        self._sel(c)
        return tebd_expect(self.h, site, op)

    def get_lambda(self, c, bond):
        self._sel(c)
        return tebd_get_lambda(self.h, bond, self.caps[c][bond])

    def discarded_weight(self, c):
        self._sel(c)
        return tebd_discarded_weight(self.h)

    def bond_weights(self, c):
        self._sel(c)
        return tebd_bond_weights(self.h, self.chains[c][0] - 1)

    def set_mps(self, c, gammas, lambdas):
        self._sel(c)
        tebd_set_mps(self.h, gammas, lambdas)

    def workspace_info(self):
        return tebd_workspace_info(self.h)

    def tuning_table(self):
        return tebd_tuning_table(self.h)
