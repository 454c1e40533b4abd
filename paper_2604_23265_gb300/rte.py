"""Python binding of librte.so (ctypes).  Argument marshalling only: every step of
the solver runs in the library's CUDA kernels; there is no fallback.

Device arrays are torch CUDA tensors (contiguous, on the context's device);
they are passed to the C ABI as raw pointers.  Names follow ``include/rte.h``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librte.so")
_lib = None

RTE_OK, RTE_EINVAL, RTE_ENOMEM, RTE_ECUDA, RTE_ENOTCONV, RTE_ESTALL, RTE_ETIMEOUT, \
    RTE_ESINGULAR, RTE_ECANCELLED, RTE_ENOTSUP = range(10)
RTE_F64, RTE_F32 = 0, 1
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONV", "ESTALL", "ETIMEOUT",
                "ESINGULAR", "ECANCELLED", "ENOTSUP"]


class RteError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 10 else status}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int)]


class Quadrature(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int)]


class CtxInfo(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int), ("M", ctypes.c_int), ("N", ctypes.c_int),
                ("nmat", ctypes.c_int), ("n", ctypes.c_int64), ("device_bytes", ctypes.c_size_t)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("inner_precision", ctypes.c_int), ("use_x0", ctypes.c_int),
                ("stall_ratio", ctypes.c_double), ("timeout_ms", ctypes.c_double),
                ("cancel", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("fell_back", ctypes.c_int), ("relres", ctypes.c_double), ("seconds", ctypes.c_double),
                ("history_len", ctypes.c_int), ("history", ctypes.c_double * 32)]

    def as_dict(self):
        """The fields as a dict, the residual history trimmed to its entries."""
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("history", "history_len")}
        d["history"] = [self.history[i] for i in range(min(self.history_len, 32))]
        return d


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); the C declarations live in include/rte.h
SIGNATURES = {
    "rte_setup": (_I, [ctypes.POINTER(Grid), ctypes.POINTER(Quadrature), _P, _P, _P, _P, _I, _D, _P,
                       _P, ctypes.POINTER(_P)]),
    "rte_setup_ex": (_I, [ctypes.POINTER(Grid), ctypes.POINTER(Quadrature), _P, _P, _P, _P, _I, _D, _P,
                          _P, _I, ctypes.POINTER(_P)]),
    "rte_block_setup_info": (_I, [_P, ctypes.POINTER(_I)]),
    "rte_set_response_path": (_I, [_P, _I]),
    "rte_response_on_tensor_cores": (_I, [_P]),
    "rte_destroy": (None, [_P]),
    "rte_trim_memory": (_I, []),
    "rte_last_error": (ctypes.c_char_p, [_P]),
    "rte_info": (_I, [_P, ctypes.POINTER(CtxInfo)]),
    "rte_rhs": (_I, [_P, _P]),
    "rte_apply": (_I, [_P, _I, _P, _P]),
    "rte_apply_adjoint": (_I, [_P, _I, _P, _P]),
    "rte_block_apply": (_I, [_P, _I, _P, _P]),
    "rte_reconstruct": (_I, [_P, _P, _P]),
    "rte_export_basis": (_I, [_P, _P, _P, _P]),
    "rte_export_blocks": (_I, [_P, _P, _P]),
    "rte_response_apply": (_I, [_P, _P, _P]),
    "rte_cgs2": (_I, [_P, _P, _I, _P, _P]),
    "rte_cgs2_df64": (_I, [_P, _P, _I, _P, _P]),
    "rte_arnoldi_basis_df64": (_I, [_P, _I, _P]),
    "rte_cgs2_noalloc": (_I, [_P, _I, ctypes.c_int64, _P, _P, _P]),
    "rte_arnoldi_basis": (_I, [_P, _I, _P]),
    "rte_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "rte_solve": (_I, [_P, _P, ctypes.POINTER(SolveOpts), _P, ctypes.POINTER(SolveInfo)]),
    "rte_atfps_solve": (_I, [_P, ctypes.POINTER(SolveOpts), _I, _P, ctypes.POINTER(SolveInfo)]),
    "rte_eigenbasis": (_I, [_I, _D, _D, _I, _P, _P]),
    "rte_fp64_fma_rate": (_I, [_P, ctypes.POINTER(_D)]),
    "rte_fp32_fma_rate": (_I, [_P, ctypes.POINTER(_D)]),
    "rte_profile": (_I, [_P, _I]),
    "rte_server_config_default": (None, [_P]),
    "rte_server_create": (_I, [_P, _P, ctypes.POINTER(_P)]),
    "rte_server_create_multi": (_I, [_P, _P, _I, ctypes.POINTER(_P)]),
    "rte_server_submit": (_I, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "rte_server_wait": (_I, [_P, ctypes.c_int64, _D, _P, _P]),
    "rte_server_cancel": (_I, [_P, ctypes.c_int64]),
    "rte_server_stats": (_I, [_P, _P]),
    "rte_server_destroy": (None, [_P]),
    "mgnet_clone": (_I, [_P, _P, ctypes.POINTER(_P)]),
    "mgnet_create": (_I, [_P, _P, ctypes.POINTER(_P)]),
    "mgnet_destroy": (None, [_P]),
    "mgnet_param_count": (ctypes.c_int64, [_P]),
    "mgnet_get_config": (_I, [_P, _P]),
    "mgnet_inject_fault": (_I, [_P, _I]),
    "mgnet_set_precision": (_I, [_P, _I]),
    "rte_solve_group": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "mgnet_set_loss": (_I, [_P, _I]),
    "mgnet_get_loss": (_I, [_P]),
    "rte_atfps_setup": (_I, [_P, _D, ctypes.POINTER(ctypes.c_int64)]),
    "rte_atfps_mask": (_I, [_P, _P]),
    "rte_atfps_apply": (_I, [_P, _P, _P]),
    "rte_atfps_apply_t": (_I, [_P, _P, _P]),
    "mgnet_get_precision": (_I, [_P]),
    "mgnet_kernel_status": (_I, [_I]),
    "mgnet_set_params": (_I, [_P, _P, ctypes.c_int64]),
    "mgnet_get_params": (_I, [_P, _P, ctypes.c_int64]),
    "mgnet_precond": (_I, [_P, _P, _P, _P]),
    "mgnet_apply": (_I, [_P, _P, _P, _P]),
    "mgnet_train_step": (_I, [_P, _P, _P, _I, _D, ctypes.POINTER(_D)]),
    "mgnet_loss_grad": (_I, [_P, _P, _P, _I, ctypes.POINTER(_D), _P]),
    "mgnet_save": (_I, [_P, ctypes.c_char_p]),
    "mgnet_load": (_I, [_P, ctypes.c_char_p]),
    "rte_profile_read": (_I, [_P, ctypes.POINTER(KernelStat), _I]),
}


def load(path: Optional[str] = None):
    """Load librte.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, ctx_ptr=None):
    if st != RTE_OK:
        msg = load().rte_last_error(ctx_ptr)
        raise RteError(st, msg.decode() if msg else "")


def _host(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev(t, dtype, numel):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"expected contiguous {dtype} with >= {numel} elements, got {t.dtype} "
                         f"{tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def trim_memory():
    """Return the unused blocks of the library's device memory pools
    (rte_trim_memory); contexts keep what they hold."""
    _check(load().rte_trim_memory())


def fp64_fma_rate(stream=None):
    """Measured FP64 FMA throughput of the current GPU, GFLOP/s."""
    v = ctypes.c_double()
    _check(load().rte_fp64_fma_rate(_stream_ptr(stream), ctypes.byref(v)))
    return v.value


def fp32_fma_rate(stream=None):
    """Measured FP32 FMA throughput of the current GPU (CUDA cores), GFLOP/s."""
    v = ctypes.c_double()
    _check(load().rte_fp32_fma_rate(_stream_ptr(stream), ctypes.byref(v)))
    return v.value


def eigenbasis(M, g, one_minus_gamma, axis):
    """Host FP64 eigenpairs of the local TFPS problem (rte_eigenbasis); no GPU needed."""
    xi = np.zeros(M)
    L = np.zeros((M, M))
    _check(load().rte_eigenbasis(int(M), float(g), float(one_minus_gamma), int(axis),
                                 xi.ctypes.data_as(_P), L.ctypes.data_as(_P)))
    return xi, L


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_device_bytes", ctypes.c_size_t), ("slots", _I),
                ("inject_alloc_failure_id", ctypes.c_int64), ("grouped", _I)]


class Request(ctypes.Structure):
    _fields_ = [("I", _I), ("M", _I), ("sigma_T", _P), ("sigma_a", _P), ("q", _P), ("eps", _P),
                ("eps_is_scalar", _I), ("g", _D), ("inflow", _P), ("tol", _D), ("max_iter", _I),
                ("restart", _I), ("use_net", _I)]


class Result(ctypes.Structure):
    _fields_ = [("status", _I), ("info", SolveInfo), ("latency_s", _D), ("queue_s", _D),
                ("footprint", ctypes.c_size_t), ("used_net", _I)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("completed", ctypes.c_int64), ("active", _I),
                ("bytes_in_use", ctypes.c_size_t)]


class Server:
    """Continuous-batching solve server (rte_server_*); thread-safe."""

    def __init__(self, slots=4, max_device_bytes=64 << 30, net=None, inject_alloc_failure_id=-1, grouped=False):
        """net: None, one MgNet, or a list of MgNets with distinct M (a request
        with use_net runs on the one for its M whose depth fits its grid)."""
        cfg = ServerConfig()
        load().rte_server_config_default(ctypes.byref(cfg))
        cfg.slots, cfg.max_device_bytes = int(slots), int(max_device_bytes)
        cfg.inject_alloc_failure_id = int(inject_alloc_failure_id)
        cfg.grouped = 1 if grouped else 0
        nets = [] if net is None else (list(net) if isinstance(net, (list, tuple)) else [net])
        arr = (ctypes.c_void_p * max(len(nets), 1))(*[m.ptr for m in nets])
        out = ctypes.c_void_p()
        _check(load().rte_server_create_multi(ctypes.byref(cfg), arr, len(nets), ctypes.byref(out)))
        self.ptr = out
        self._meta = {}

    def submit(self, md, tol=1e-8, use_net=False, max_iter=0, restart=0):
        """Queue a solve of the medium md (rte_server_submit); returns the request id. use_net:
        precondition with the server's network for md.M when one fits the grid."""
        arrs = [np.ascontiguousarray(a, np.float64) for a in
                (md.sigma_T, md.sigma_a, md.q, np.asarray(md.eps).reshape(-1), md.inflow)]
        eps_scalar = int(arrs[3].size == 1)
        req = Request(md.I, md.M, *[a.ctypes.data_as(_P) for a in arrs[:4]], eps_scalar, float(md.g),
                      arrs[4].ctypes.data_as(_P), float(tol), int(max_iter), int(restart), int(use_net))
        rid = ctypes.c_int64()
        _check(load().rte_server_submit(self.ptr, ctypes.byref(req), ctypes.byref(rid)))
        self._meta[rid.value] = (md.M, md.I)
        return rid.value

    def wait(self, rid, timeout_ms=0.0):
        """Block until request rid is done (rte_server_wait); returns (result dict, psi as a host array
        [M * N])."""
        M, I = self._meta[rid]
        res = Result()
        psi = np.zeros(M * I * I)
        _check(load().rte_server_wait(self.ptr, int(rid), float(timeout_ms), ctypes.byref(res),
                                      psi.ctypes.data_as(_P)))
        del self._meta[rid]
        d = {"status": STATUS_NAMES[res.status], "latency_s": res.latency_s, "queue_s": res.queue_s,
             "footprint": res.footprint, "used_net": bool(res.used_net)}
        if res.status != RTE_OK:
            msg = load().rte_last_error(None)
            d["error"] = msg.decode() if msg else ""
        d.update(res.info.as_dict())
        return d, psi

    def cancel(self, rid):
        """Cancel request rid (rte_server_cancel)."""
        _check(load().rte_server_cancel(self.ptr, int(rid)))

    def stats(self):
        """Queue, occupancy and byte counters (rte_server_stats)."""
        st = ServerStats()
        _check(load().rte_server_stats(self.ptr, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        """Stop the server (rte_server_destroy); requests still waiting are cancelled."""
        if getattr(self, "ptr", None):
            load().rte_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_group(ctxs, xs, pcs=None, tol=1e-8, restart=50, max_iter=20000, inner_precision=RTE_F32,
                use_x0=False, stall_ratio=0.9, timeout_ms=0.0):
    """rte_solve_group: the solves of several contexts (one stream) in lockstep
    with their Arnoldi steps in shared launches.  Returns one info dict (with
    its "status") per solve."""
    import torch
    count = len(ctxs)
    o = SolveOpts()
    load().rte_solve_opts_default(ctypes.byref(o))
    o.tol, o.restart, o.max_iter = float(tol), int(restart), int(max_iter)
    o.inner_precision, o.use_x0 = int(inner_precision), int(use_x0)
    o.stall_ratio, o.timeout_ms = float(stall_ratio), float(timeout_ms)
    cp = (_P * count)(*[c.ptr for c in ctxs])
    xp = (_P * count)(*[_dev(x, torch.float64, c.n) for c, x in zip(ctxs, xs)])
    pp = (_P * count)(*[(p.ptr if p is not None else None) for p in (pcs or [None] * count)])
    infos = (SolveInfo * count)()
    sts = (ctypes.c_int * count)()
    _check(load().rte_solve_group(cp, pp, count, ctypes.byref(o), xp, infos, sts))
    out = []
    for i in range(count):
        d = infos[i].as_dict()
        d["status"] = STATUS_NAMES[sts[i]]
        out.append(d)
    return out


class MgNetConfig(ctypes.Structure):
    _fields_ = [("M", _I), ("levels", _I), ("c0", _I), ("cmax", _I), ("cc", _I), ("ccmax", _I),
                ("act", _I)]


class MgNet:
    """The learned preconditioner (mgnet_*); weights as one float32 vector in
    the order of ``workloads.param_shapes``."""

    def __init__(self, shape, stream=None):
        cfg = MgNetConfig(shape.M, shape.levels, shape.c0, shape.cmax, shape.cc, shape.ccmax,
                          1 if getattr(shape, "act", "linear") == "relu" else 0)
        out = ctypes.c_void_p()
        _check(load().mgnet_create(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(out)))
        self.ptr = out
        self.shape = shape
        self.count = int(load().mgnet_param_count(self.ptr))

    FAULT_NONE, FAULT_NAN = 0, 1

    def inject_fault(self, kind):
        """Host-side fault injection (mgnet_inject_fault): FAULT_NAN makes every
        preconditioner output NaN; FAULT_NONE restores normal operation."""
        _check(load().mgnet_inject_fault(self.ptr, int(kind)))

    def config(self):
        """The library's record of the configuration (mgnet_get_config)."""
        c = MgNetConfig()
        _check(load().mgnet_get_config(self.ptr, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in c._fields_}

    def close(self):
        """Free the network (mgnet_destroy)."""
        if getattr(self, "ptr", None):
            load().mgnet_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def flatten(params, shape):
        """Parameter dict -> float32 vector in the library's order (workloads.param_shapes)."""
        from . import workloads
        return np.concatenate([np.asarray(params[name], np.float64).ravel()
                               for name, _ in workloads.param_shapes(shape)]).astype(np.float32)

    @staticmethod
    def unflatten(flat, shape):
        """float32 vector -> parameter dict of float64 arrays."""
        from . import workloads
        out, o = {}, 0
        for name, shp in workloads.param_shapes(shape):
            k = int(np.prod(shp))
            out[name] = np.asarray(flat[o:o + k], np.float64).reshape(shp)
            o += k
        return out

    def set_params(self, params):
        """Set the weights from a dict or a flat vector (mgnet_set_params; resets the Adam state)."""
        flat = params if isinstance(params, np.ndarray) else self.flatten(params, self.shape)
        flat = np.ascontiguousarray(flat, np.float32)
        _check(load().mgnet_set_params(self.ptr, flat.ctypes.data_as(_P), flat.size))

    FP32, BF16 = 0, 1

    @property
    def precision(self):
        """Convolution arithmetic when preconditioning: MgNet.BF16 (tensor
        cores, default) or MgNet.FP32 (CUDA cores)."""
        return int(load().mgnet_get_precision(self.ptr))

    @precision.setter
    def precision(self, value):
        """Set the convolution arithmetic (mgnet_set_precision; RteError for another value)."""
        _check(load().mgnet_set_precision(self.ptr, int(value)))

    PLAIN, FILTERED = 0, 1

    @property
    def loss(self):
        """Training loss: MgNet.PLAIN (Eq. loss) or MgNet.FILTERED (Eq. loss_delta,
        needs Context.atfps_setup on the training contexts)."""
        return int(load().mgnet_get_loss(self.ptr))

    @loss.setter
    def loss(self, value):
        """Set the training loss (mgnet_set_loss; RteError for another value)."""
        _check(load().mgnet_set_loss(self.ptr, int(value)))

    @staticmethod
    def kernel_status(reset=True):
        """1 if a bounded wait of a tensor-core network kernel expired."""
        return int(load().mgnet_kernel_status(1 if reset else 0))

    def get_params(self):
        """The weights as a float32 vector (mgnet_get_params)."""
        flat = np.zeros(self.count, np.float32)
        _check(load().mgnet_get_params(self.ptr, flat.ctypes.data_as(_P), flat.size))
        return flat

    def precond(self, ctx, r, z):
        """z = Net(r) in face-flux space (mgnet_precond): r float64 [n], z float32 [n], device tensors."""
        import torch
        _check(load().mgnet_precond(self.ptr, ctx.ptr, _dev(r, torch.float64, ctx.n),
                                    _dev(z, torch.float32, ctx.n)))
        return z

    def apply(self, ctx, r, z):
        """z = D Net(r) (mgnet_apply): r, z float64 [n], device tensors."""
        import torch
        _check(load().mgnet_apply(self.ptr, ctx.ptr, _dev(r, torch.float64, ctx.n),
                                  _dev(z, torch.float64, ctx.n)))
        return z

    def _ptrs(self, ctx, rs):
        import torch
        arr = (_P * len(rs))(*[_dev(r, torch.float64, ctx.n).value for r in rs])
        return arr

    def train_step(self, ctx, rs, lr):
        """One Adam step on a batch of right-hand sides of ctx (mgnet_train_step); returns the batch
        loss before the step."""
        loss = ctypes.c_double()
        arr = self._ptrs(ctx, rs)
        _check(load().mgnet_train_step(self.ptr, ctx.ptr, ctypes.cast(arr, _P), len(rs), float(lr),
                                       ctypes.byref(loss)))
        return loss.value

    def loss_grad(self, ctx, rs):
        """(loss, gradient as a float32 vector) without updating the weights (mgnet_loss_grad)."""
        loss = ctypes.c_double()
        g = np.zeros(self.count, np.float32)
        arr = self._ptrs(ctx, rs)
        _check(load().mgnet_loss_grad(self.ptr, ctx.ptr, ctypes.cast(arr, _P), len(rs),
                                      ctypes.byref(loss), g.ctypes.data_as(_P)))
        return loss.value, g

    def save(self, path):
        """Checkpoint the weights and the Adam state to path (mgnet_save)."""
        _check(load().mgnet_save(self.ptr, str(path).encode()))

    def load(self, path):
        """Restore a checkpoint from path (mgnet_load)."""
        _check(load().mgnet_load(self.ptr, str(path).encode()))


class Context:
    """One RTE system (rte_setup); see include/rte.h for the layouts."""

    BLOCKS_AUTO, BLOCKS_EXACT, BLOCKS_TABULATED = 0, 1, 2
    RESPONSE_AUTO, RESPONSE_PER_CELL = 0, 1

    def __init__(self, I, M, sigma_T, sigma_a, q, eps, g, inflow=None, stream=None, block_mode=0):
        lib = load()
        N = I * I
        self._keep = []
        sT, psT = _host(np.broadcast_to(sigma_T, (N,)))
        sa, psa = _host(np.broadcast_to(sigma_a, (N,)))
        qq, pq = _host(np.broadcast_to(q, (N,)))
        e = np.asarray(eps, np.float64)
        scalar = int(e.size == 1)
        ee, pe = _host(e.reshape(-1) if not scalar else e.reshape(1))
        if inflow is not None:
            fl, pf = _host(np.asarray(inflow).reshape(4 * I * M))
        else:
            fl, pf = None, None
        out = ctypes.c_void_p()
        st = lib.rte_setup_ex(ctypes.byref(Grid(I)), ctypes.byref(Quadrature(M)), psT, psa, pq, pe,
                              scalar, float(g), pf, _stream_ptr(stream), int(block_mode), ctypes.byref(out))
        _check(st, None)
        self.ptr = out
        self.I, self.M, self.N = I, M, N
        self.n = 2 * M * N

    @classmethod
    def from_medium(cls, md, stream=None, block_mode=0):
        """The context of a workloads.Medium (rte_setup_ex; block_mode: Context.BLOCKS_*)."""
        return cls(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow, stream, block_mode)

    def tabulated_nodes(self):
        """Interpolation nodes of the per-cell blocks (0: inverted cell by cell)."""
        v = ctypes.c_int()
        _check(load().rte_block_setup_info(self.ptr, ctypes.byref(v)), self.ptr)
        return v.value

    def set_response_path(self, path):
        """How the inner operator applies R (rte_set_response_path; Context.RESPONSE_*)."""
        _check(load().rte_set_response_path(self.ptr, int(path)), self.ptr)

    def response_on_tensor_cores(self):
        """True when R z runs on the tensor cores from the node tables."""
        v = load().rte_response_on_tensor_cores(self.ptr)
        if v < 0:
            raise RuntimeError("rte_response_on_tensor_cores: bad context")
        return bool(v)

    def close(self):
        """Free the context (rte_destroy)."""
        if getattr(self, "ptr", None):
            load().rte_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """Sizes, materials and device bytes (rte_ctx_info)."""
        i = CtxInfo()
        _check(load().rte_info(self.ptr, ctypes.byref(i)), self.ptr)
        return {k: getattr(i, k) for k, _ in i._fields_}

    def rhs(self, b):
        """Write b of Eq. 2DTFPS_linear_sys into the float64 device vector b."""
        import torch
        _check(load().rte_rhs(self.ptr, _dev(b, torch.float64, self.n)), self.ptr)
        return b

    def apply(self, x, y, precision=RTE_F64):
        """y = A x (rte_apply), FP64 or FP32 by precision."""
        import torch
        dt = torch.float64 if precision == RTE_F64 else torch.float32
        _check(load().rte_apply(self.ptr, precision, _dev(x, dt, self.n), _dev(y, dt, self.n)), self.ptr)
        return y

    def apply_adjoint(self, y, x, precision=RTE_F64):
        """x = A^T y (rte_apply_adjoint)."""
        import torch
        dt = torch.float64 if precision == RTE_F64 else torch.float32
        _check(load().rte_apply_adjoint(self.ptr, precision, _dev(y, dt, self.n), _dev(x, dt, self.n)),
               self.ptr)
        return x

    def block_apply(self, r, z, transpose=False):
        """z = D r, or D^T r with transpose, with the per-cell inverse blocks (rte_block_apply)."""
        import torch
        _check(load().rte_block_apply(self.ptr, int(transpose), _dev(r, torch.float32, self.n),
                                      _dev(z, torch.float32, self.n)), self.ptr)
        return z

    def reconstruct(self, x, psi):
        """Angular flux at the cell centres, psi float64 [M][N] (rte_reconstruct)."""
        import torch
        _check(load().rte_reconstruct(self.ptr, _dev(x, torch.float64, self.n),
                                      _dev(psi, torch.float64, self.M * self.N)), self.ptr)
        return psi

    def export_basis(self):
        """(xi [nmat][2M], L [nmat][M][2M], material of every cell) (rte_export_basis)."""
        info = self.info()
        nmat, M, N = info["nmat"], self.M, self.N
        xi = np.zeros((nmat, 2 * M))
        L = np.zeros((nmat, M, 2 * M))
        mat = np.zeros(N, np.int32)
        _check(load().rte_export_basis(self.ptr, xi.ctypes.data_as(_P), L.ctypes.data_as(_P),
                                       mat.ctypes.data_as(_P)), self.ptr)
        return xi, L, mat

    def export_blocks(self):
        """(D [N][2M][2M] float64, R [N][2M][2M] float32), row-major per cell."""
        D = np.zeros((self.N, 2 * self.M, 2 * self.M), np.float64)
        R = np.zeros((self.N, 2 * self.M, 2 * self.M), np.float32)
        _check(load().rte_export_blocks(self.ptr, D.ctypes.data_as(_P), R.ctypes.data_as(_P)),
               self.ptr)
        return D, R

    def response_apply(self, v, w):
        """w = A D v = v - P R v (face-flux space), double [n]."""
        import torch
        _check(load().rte_response_apply(self.ptr, _dev(v, torch.float64, self.n),
                                         _dev(w, torch.float64, self.n)), self.ptr)
        return w

    def cgs2(self, V, k, w, h):
        """One classical Gram-Schmidt step with reorthogonalisation of w against k vectors of V
        (rte_cgs2)."""
        import torch
        _check(load().rte_cgs2(self.ptr, _dev(V, torch.float64, k * self.n), int(k),
                               _dev(w, torch.float64, self.n), _dev(h, torch.float64, k + 1)),
               self.ptr)
        return h

    def cgs2_df64(self, V, k, w, h):
        """rte_cgs2 on df64 vectors (float32 tensors: V [k][2][n], w [2][n], hi plane then lo plane;
        h float64 [k + 1]) with the arithmetic of the solver's Arnoldi step (rte_cgs2_df64)."""
        import torch
        _check(load().rte_cgs2_df64(self.ptr, _dev(V, torch.float32, 2 * k * self.n), int(k),
                                    _dev(w, torch.float32, 2 * self.n), _dev(h, torch.float64, k + 1)),
               self.ptr)
        return h

    def arnoldi_basis_df64(self, k, V):
        """k Arnoldi vectors of A D as df64 (float32 tensor [k][2][n]; rte_arnoldi_basis_df64)."""
        import torch
        _check(load().rte_arnoldi_basis_df64(self.ptr, int(k), _dev(V, torch.float32, 2 * k * self.n)), self.ptr)
        return V

    def profile(self, enable=True):
        """Clear the per-kernel counters; enable=True also times every launch."""
        _check(load().rte_profile(self.ptr, int(enable)), self.ptr)

    def profile_read(self):
        """{kernel class: (launches, ms, algorithmic bytes, FP64 flops)}."""
        n = load().rte_profile_read(self.ptr, None, 0)
        arr = (KernelStat * n)()
        got = load().rte_profile_read(self.ptr, arr, n)
        if got < 0:
            _check(RTE_ECUDA, self.ptr)
        return {a.name.decode(): (a.launches, a.ms, a.bytes, a.flops) for a in arr[:got]}

    def atfps_setup(self, delta):
        """ATFPS filter of the loss (Sec. 2.3); returns the number of kept coordinates."""
        rows = ctypes.c_int64()
        _check(load().rte_atfps_setup(self.ptr, float(delta), ctypes.byref(rows)), self.ptr)
        self.atfps_rows = rows.value
        return rows.value

    def atfps_mask(self):
        """Selection [2M][N] (1 = kept) of the current filter."""
        m = np.zeros(2 * self.M * self.I * self.I, np.uint8)
        _check(load().rte_atfps_mask(self.ptr, m.ctypes.data_as(_P)), self.ptr)
        return m.reshape(2 * self.M, self.I * self.I)

    def atfps_apply(self, y, out):
        """out = F y, the kept interface projections (rte_atfps_apply)."""
        import torch
        _check(load().rte_atfps_apply(self.ptr, _dev(y, torch.float64, self.n),
                                      _dev(out, torch.float64, self.atfps_rows)), self.ptr)
        return out

    def atfps_apply_t(self, r, y):
        """y = F^T r (rte_atfps_apply_t)."""
        import torch
        _check(load().rte_atfps_apply_t(self.ptr, _dev(r, torch.float64, self.atfps_rows),
                                        _dev(y, torch.float64, self.n)), self.ptr)
        return y

    def arnoldi_basis(self, k, V):
        """k Arnoldi vectors of the block-Jacobi preconditioned operator from b."""
        import torch
        _check(load().rte_arnoldi_basis(self.ptr, int(k), _dev(V, torch.float64, k * self.n)), self.ptr)
        return V

    def solve(self, x, pc=None, tol=1e-8, restart=50, max_iter=20000, inner_precision=RTE_F32,
              use_x0=False, stall_ratio=0.9, timeout_ms=0.0, raise_on_error=True):
        """FGMRES(restart) solve of A x = b (rte_solve); pc None is block Jacobi. Returns the info dict."""
        import torch
        o = SolveOpts()
        load().rte_solve_opts_default(ctypes.byref(o))
        o.tol, o.restart, o.max_iter = float(tol), int(restart), int(max_iter)
        o.inner_precision, o.use_x0 = int(inner_precision), int(use_x0)
        o.stall_ratio, o.timeout_ms = float(stall_ratio), float(timeout_ms)
        inf = SolveInfo()
        pcp = pc.ptr if pc is not None else None
        st = load().rte_solve(self.ptr, pcp, ctypes.byref(o), _dev(x, torch.float64, self.n),
                              ctypes.byref(inf))
        d = inf.as_dict()
        d["status"] = STATUS_NAMES[st] if 0 <= st < 10 else st
        if raise_on_error and st not in (RTE_OK, RTE_ENOTCONV):
            _check(st, self.ptr)
        return d

    def atfps_solve(self, x, layers=True, tol=1e-8, restart=50, max_iter=20000, use_x0=False, timeout_ms=0.0,
                    raise_on_error=True):
        """Compressed ATFPS solve (rte_atfps_solve) after atfps_setup(delta):
        x (float64 [2M][N] device) receives the kept coefficients and, with
        layers, the reconstructed dropped ones."""
        import torch
        o = SolveOpts()
        load().rte_solve_opts_default(ctypes.byref(o))
        o.tol, o.restart, o.max_iter = float(tol), int(restart), int(max_iter)
        o.use_x0, o.timeout_ms = int(use_x0), float(timeout_ms)
        inf = SolveInfo()
        st = load().rte_atfps_solve(self.ptr, ctypes.byref(o), 1 if layers else 0, _dev(x, torch.float64, self.n),
                                    ctypes.byref(inf))
        d = inf.as_dict()
        d["status"] = STATUS_NAMES[st] if 0 <= st < 10 else st
        if raise_on_error and st not in (RTE_OK, RTE_ENOTCONV):
            _check(st, self.ptr)
        return d
