"""Python binding of libqaoa (include/qaoa.h): argument marshalling only.

Every computation runs in the C++ planner or the CUDA kernels behind the C
ABI; this module converts arguments, checks shapes, passes raw pointers and
the current CUDA stream, and raises :class:`QAOAError` on a negative status.
There is no fallback: if the library has not been built, loading fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqaoa.so")

QAOA_OK = 0
QAOA_E_INVALID = -1
QAOA_E_CONE_TOO_LARGE = -2
QAOA_E_OOM = -3
QAOA_E_CUDA = -4
QAOA_E_DEVICE = -5

ORBITS_OFF = 0
ORBITS = 1
FULL_CONE = 2
SHELL_PLAIN = 4
BIG_GENERAL = 8
CONE_CLASSES = 16
BLOCK_PLAIN = 32


class QAOAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libqaoa error {code}: {msg}")
        self.code = code


class Tuning(C.Structure):
    _fields_ = [("points_per_task", C.c_int32), ("blocks_per_sm", C.c_int32), ("big_scratch_bytes", C.c_int64),
                ("reg_bits_grad", C.c_int32), ("chunk_window", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [
        ("p", C.c_int32), ("n_graphs", C.c_int32), ("n_edges_total", C.c_int64),
        ("n_reps", C.c_int64), ("max_qubits", C.c_int32), ("max_inner", C.c_int32),
        ("max_edges", C.c_int32), ("on_device", C.c_int32), ("n_big", C.c_int64),
        ("amps_per_point", C.c_double), ("t_orbits_s", C.c_double), ("t_cones_s", C.c_double),
        ("orbits_complete", C.c_int32), ("n_big_general_energy", C.c_int64), ("n_big_general_grad", C.c_int64),
        ("depth1_kernel", C.c_int32),
    ]


_lib = None
_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
_F64P = C.POINTER(C.c_double)

_SIGS = {
    "qaoa_plan_graphs": (C.c_int, [C.c_int32, _I32P, _I64P, _I32P, C.c_int32, C.c_uint32, C.c_int32,
                                   C.c_int64, C.POINTER(_P)]),
    "qaoa_plan_graph": (C.c_int, [C.c_int32, C.c_int64, _I32P, C.c_int32, C.c_uint32, C.c_int32,
                                  C.c_int64, C.POINTER(_P)]),
    "qaoa_plan_free": (None, [_P]),
    "qaoa_plan_info": (C.c_int, [_P, C.POINTER(PlanInfo)]),
    "qaoa_plan_orbits": (C.c_int, [_P, C.c_int32, _I32P, _I64P, _F64P, _I32P]),
    "qaoa_plan_cone_classes": (C.c_int, [_P, C.c_int32, _I32P, _I64P]),
    "qaoa_plan_graphs_weighted": (C.c_int, [C.c_int32, _I32P, _I64P, _I32P, _I32P, C.c_int32, C.c_uint32,
                                            C.c_int32, C.c_int64, C.POINTER(_P)]),
    "qaoa_plan_cone_weights": (C.c_int, [_P, C.c_int64, _I32P]),
    "qaoa_plan_reps": (C.c_int, [_P, _I32P, _I64P, _I32P, _I32P, _I32P, _I32P, _I32P]),
    "qaoa_plan_cone": (C.c_int, [_P, C.c_int64, _I32P, _I32P, _I32P]),
    "qaoa_plan_shell": (C.c_int, [_P, C.c_int64, _I32P, _I64P]),
    "qaoa_plan_blocks": (C.c_int, [_P, C.c_int64, _I64P, _I32P, C.POINTER(C.c_uint8), C.POINTER(C.c_double)]),
    "qaoa_edge_orbits": (C.c_int, [C.c_int32, C.c_int64, _I32P, C.c_int64, _I32P, _I64P, _I64P, _F64P, _I32P]),
    "qaoa_plan_upload": (C.c_int, [_P]),
    "qaoa_cut_table": (C.c_int, [_P, C.c_int64, _P, _P]),
    "qaoa_energy": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    "qaoa_norms": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "qaoa_energy_grad": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P]),
    "qaoa_energy_noalloc": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    "qaoa_device_status": (C.c_int, [_P, _I32P]),
    "qaoa_plan_timing": (C.c_int, [_P, C.c_int32]),
    "qaoa_plan_set_tuning": (C.c_int, [_P, C.POINTER(Tuning)]),
    "qaoa_plan_get_tuning": (C.c_int, [_P, C.POINTER(Tuning)]),
    "qaoa_graph_create": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, C.POINTER(_P)]),
    "qaoa_graph_launch": (C.c_int, [_P, _P]),
    "qaoa_graph_free": (None, [_P]),
    "qaoa_kernel_time": (C.c_int, [_P, _F64P, _I64P, _I64P]),
    "qaoa_inject_fault": (C.c_int, [C.c_int32, C.c_int32]),
    "qaoa_last_error": (C.c_char_p, []),
    "qaoa_version": (C.c_char_p, []),
}


def lib():
    """The loaded libqaoa (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2101_10296_gb300.build.build()")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def _check(code):
    if code != QAOA_OK:
        raise QAOAError(code, lib().qaoa_last_error().decode())


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def edge_orbits(n, edges, budget=0):
    """Host-only orbit finder: (orbit_id[m], n_orbits, n_generators, log10|Aut|, complete)."""
    e = _i32(np.asarray(edges).reshape(-1, 2))
    m = e.shape[0]
    oid = np.zeros(m, dtype=np.int32)
    norb, ngen = C.c_int64(), C.c_int64()
    l10 = C.c_double()
    comp = C.c_int32()
    _check(lib().qaoa_edge_orbits(n, m, _ptr(e, C.c_int32), budget, _ptr(oid, C.c_int32), C.byref(norb),
                                  C.byref(ngen), C.byref(l10), C.byref(comp)))
    return oid, norb.value, ngen.value, l10.value, bool(comp.value)


FAULT_NONE, FAULT_GENERATOR, FAULT_DEVICE_ALLOC = 0, 1, 2


def inject_fault(kind, count=1):
    """Make the next ``count`` events of ``kind`` fail on the host (testing only)."""
    _check(lib().qaoa_inject_fault(kind, count))


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Plan:
    """A planned batch of graphs (orbits + cones), owning its device copy."""

    def __init__(self, graphs, p, orbits=True, full_cone=False, max_cone_qubits=0, search_budget=0,
                 shell_plain=False, big_general=False, cone_classes=False, weights=None, block_plain=False):
        """graphs: (n, edges) or a list of them; weights: None (MaxCut) or one
        integer array per graph (edge weights / colours, see
        qaoa_plan_graphs_weighted)."""
        if isinstance(graphs, tuple):
            graphs = [graphs]
            if weights is not None and np.ndim(weights[0]) == 0:
                weights = [weights]
        nv = _i32([g[0] for g in graphs])
        offs = [0]
        rows = []
        for n, e in graphs:
            e = np.asarray(e, dtype=np.int64).reshape(-1, 2)
            rows.append(e)
            offs.append(offs[-1] + e.shape[0])
        edges = _i32(np.concatenate(rows) if rows else np.zeros((0, 2)))
        offs = np.asarray(offs, dtype=np.int64)
        flags = (ORBITS if orbits else ORBITS_OFF) | (FULL_CONE if full_cone else 0) | (SHELL_PLAIN if shell_plain else 0)
        flags |= (BIG_GENERAL if big_general else 0) | (CONE_CLASSES if cone_classes else 0)
        flags |= BLOCK_PLAIN if block_plain else 0
        h = C.c_void_p()
        if weights is None:
            _check(lib().qaoa_plan_graphs(len(graphs), _ptr(nv, C.c_int32), _ptr(offs, C.c_int64),
                                          _ptr(edges, C.c_int32) if edges.size else None, p, flags,
                                          max_cone_qubits, search_budget, C.byref(h)))
        else:
            w = _i32(np.concatenate([np.asarray(x).reshape(-1) for x in weights]) if len(weights) else [])
            if w.size != edges.shape[0]:
                raise ValueError("one weight per edge is needed")
            _check(lib().qaoa_plan_graphs_weighted(len(graphs), _ptr(nv, C.c_int32), _ptr(offs, C.c_int64),
                                                   _ptr(edges, C.c_int32) if edges.size else None,
                                                   _ptr(w, C.c_int32) if w.size else None, p, flags,
                                                   max_cone_qubits, search_budget, C.byref(h)))
        self._h = h
        self.p = p
        self.n_graphs = len(graphs)
        self.n_edges = [int(r.shape[0]) for r in rows]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().qaoa_plan_free(self._h)
            self._h = C.c_void_p()

    __del__ = close

    @property
    def handle(self):
        return self._h

    def info(self):
        i = PlanInfo()
        _check(lib().qaoa_plan_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in PlanInfo._fields_}

    def orbits(self, graph=0):
        oid = np.zeros(self.n_edges[graph], dtype=np.int32)
        norb = C.c_int64()
        l10 = C.c_double()
        comp = C.c_int32()
        _check(lib().qaoa_plan_orbits(self._h, graph, _ptr(oid, C.c_int32), C.byref(norb), C.byref(l10),
                                      C.byref(comp)))
        return oid, norb.value, l10.value, bool(comp.value)

    def cone_classes(self, graph=0):
        """(class id per edge = smallest edge of its cone class, number of classes)."""
        cid = np.zeros(self.n_edges[graph], dtype=np.int32)
        ncls = C.c_int64()
        _check(lib().qaoa_plan_cone_classes(self._h, graph, _ptr(cid, C.c_int32), C.byref(ncls)))
        return cid, ncls.value

    def reps(self):
        r = self.info()["n_reps"]
        out = {k: np.zeros(r, dtype=np.int32) for k in ("graph", "weight", "n_qubits", "n_inner", "n_cone_edges")}
        edge = np.zeros(r, dtype=np.int64)
        mix = np.zeros((r, self.p), dtype=np.int32)
        _check(lib().qaoa_plan_reps(self._h, _ptr(out["graph"], C.c_int32), _ptr(edge, C.c_int64),
                                    _ptr(out["weight"], C.c_int32), _ptr(out["n_qubits"], C.c_int32),
                                    _ptr(out["n_inner"], C.c_int32), _ptr(out["n_cone_edges"], C.c_int32),
                                    _ptr(mix, C.c_int32)))
        out["edge"] = edge
        out["mix_qubits"] = mix
        return out

    def cone(self, rep):
        reps = self.reps()
        nq = int(reps["n_qubits"][rep])
        ne = int(reps["n_cone_edges"][rep])
        verts = np.zeros(nq, dtype=np.int32)
        dist = np.zeros(nq, dtype=np.int32)
        ce = np.zeros((max(ne, 1), 2), dtype=np.int32)
        _check(lib().qaoa_plan_cone(self._h, rep, _ptr(verts, C.c_int32), _ptr(dist, C.c_int32),
                                    _ptr(ce, C.c_int32)))
        return verts, dist, ce[:ne]

    def cone_weights(self, rep):
        """Weights of the cone's edges (order of :meth:`cone`)."""
        ne = int(self.reps()["n_cone_edges"][rep])
        w = np.zeros(max(ne, 1), dtype=np.int32)
        _check(lib().qaoa_plan_cone_weights(self._h, rep, _ptr(w, C.c_int32)))
        return w[:ne]

    def shell(self, rep):
        """(class index per cone qubit, -1 for inner; number of shell blocks)."""
        nq = int(self.reps()["n_qubits"][rep])
        cls = np.zeros(nq, dtype=np.int32)
        nb = C.c_int64()
        _check(lib().qaoa_plan_shell(self._h, rep, _ptr(cls, C.c_int32), C.byref(nb)))
        return cls, nb.value

    def blocks(self, rep):
        """(counts [n_blocks, n_classes] uint8, weight [n_blocks] float64): the
        shell blocks the cone is evolved for (see qaoa_plan_blocks)."""
        nb, nc = C.c_int64(), C.c_int32()
        _check(lib().qaoa_plan_blocks(self._h, rep, C.byref(nb), C.byref(nc), None, None))
        counts = np.zeros((nb.value, nc.value), dtype=np.uint8)
        w = np.zeros(nb.value, dtype=np.float64)
        _check(lib().qaoa_plan_blocks(self._h, rep, None, None, _ptr(counts, C.c_uint8) if counts.size else None,
                                      _ptr(w, C.c_double)))
        return counts, w

    def shell_blocks(self):
        """Number of shell blocks of every representative (plan order)."""
        r = self.info()["n_reps"]
        out = np.zeros(r, dtype=np.int64)
        nb = C.c_int64()
        for i in range(r):
            _check(lib().qaoa_plan_shell(self._h, i, None, C.byref(nb)))
            out[i] = nb.value
        return out

    def upload(self):
        _check(lib().qaoa_plan_upload(self._h))

    def cut_table(self, rep, stream=None):
        import torch
        nq = int(self.reps()["n_qubits"][rep])
        out = torch.empty(1 << nq, dtype=torch.uint8, device="cuda")
        _check(lib().qaoa_cut_table(self._h, rep, C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def _params(self, params):
        import torch
        if not (isinstance(params, torch.Tensor) and params.is_cuda and params.dtype == torch.float64):
            raise TypeError("params must be a CUDA float64 tensor")
        # device pointers must be on the current device (the library checks that the
        # plan is there too); outputs are allocated next to params
        if params.device.index != torch.cuda.current_device():
            raise ValueError(f"params are on {params.device}, the current device is "
                             f"cuda:{torch.cuda.current_device()}")
        if params.dim() == 2:
            params = params.unsqueeze(0)
        if params.dim() != 3 or params.shape[0] != self.n_graphs or params.shape[2] != 2 * self.p:
            raise ValueError(f"params must have shape [{self.n_graphs}, P, {2 * self.p}]")
        return params.contiguous()

    def energy(self, params, terms=False, stream=None):
        """E[g, j] for params [G, P, 2p] (CUDA float64); optionally <ZZ> per rep."""
        import torch
        params = self._params(params)
        G, P = params.shape[0], params.shape[1]
        e = torch.empty(G, P, dtype=torch.float64, device=params.device)
        t = torch.empty(self.info()["n_reps"], P, dtype=torch.float64, device=params.device) if terms else None
        _check(lib().qaoa_energy(self._h, P, C.c_void_p(params.data_ptr()), C.c_void_p(e.data_ptr()),
                                 C.c_void_p(t.data_ptr()) if terms else None, _stream_handle(stream)))
        return (e, t) if terms else e

    def norms(self, params, stream=None):
        """sum_z |psi_z|^2 of every representative's cone state at every point,
        [n_reps, P] (1 up to the FP32 state's rounding; a diagnostic)."""
        import torch
        params = self._params(params)
        P = params.shape[1]
        out = torch.empty(self.info()["n_reps"], P, dtype=torch.float64, device=params.device)
        _check(lib().qaoa_norms(self._h, P, C.c_void_p(params.data_ptr()), C.c_void_p(out.data_ptr()),
                                _stream_handle(stream)))
        return out

    def energy_noalloc(self, params, out=None, terms=None, stream=None):
        """E[g, j] through qaoa_energy_noalloc, into caller-provided tensors.

        The library allocates nothing during the call; ``out`` (and ``terms``)
        are allocated here by torch only when not given.  The plan must have
        been uploaded (``upload()``).
        """
        import torch
        params = self._params(params)
        G, P = params.shape[0], params.shape[1]
        if out is None:
            out = torch.empty(G, P, dtype=torch.float64, device=params.device)

        def _need(t, shape, name):
            # the library writes float64 values through the raw pointer: anything
            # else would be written past the end of the caller's buffer
            if not isinstance(t, torch.Tensor):
                raise TypeError(f"{name} must be a torch tensor")
            if t.dtype != torch.float64 or not t.is_cuda or t.device != params.device:
                raise ValueError(f"{name} must be a float64 tensor on {params.device}")
            if tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous tensor of shape {list(shape)}")

        _need(out, (G, P), "out")
        if terms is not None:
            _need(terms, (self.info()["n_reps"], P), "terms")
        _check(lib().qaoa_energy_noalloc(self._h, P, C.c_void_p(params.data_ptr()), C.c_void_p(out.data_ptr()),
                                         C.c_void_p(terms.data_ptr()) if terms is not None else None,
                                         _stream_handle(stream)))
        return out

    def energy_grad(self, params, terms=False, stream=None):
        """(E[g, j], dE/dtheta[g, j, 2p]) by the adjoint kernels."""
        import torch
        params = self._params(params)
        G, P = params.shape[0], params.shape[1]
        e = torch.empty(G, P, dtype=torch.float64, device=params.device)
        g = torch.empty(G, P, 2 * self.p, dtype=torch.float64, device=params.device)
        t = torch.empty(self.info()["n_reps"], P, dtype=torch.float64, device=params.device) if terms else None
        _check(lib().qaoa_energy_grad(self._h, P, C.c_void_p(params.data_ptr()), C.c_void_p(e.data_ptr()),
                                      C.c_void_p(g.data_ptr()), C.c_void_p(t.data_ptr()) if terms else None,
                                      _stream_handle(stream)))
        return (e, g, t) if terms else (e, g)

    def set_tuning(self, points_per_task=0, blocks_per_sm=0, big_scratch_bytes=0, reg_bits_grad=0, chunk_window=0):
        """Launch tuning for later calls (0 = default); see qaoa_tuning_t."""
        t = Tuning(points_per_task, blocks_per_sm, big_scratch_bytes, reg_bits_grad, chunk_window)
        _check(lib().qaoa_plan_set_tuning(self._h, C.byref(t)))

    def get_tuning(self):
        t = Tuning()
        _check(lib().qaoa_plan_get_tuning(self._h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def graph(self, params, grad=True, terms=False):
        """A captured CUDA graph of one evaluation with fixed buffers (see PlanGraph)."""
        return PlanGraph(self, params, grad=grad, terms=terms)

    def set_timing(self, enable=True):
        """Record CUDA events around every later call's cone kernel(s)."""
        _check(lib().qaoa_plan_timing(self._h, 1 if enable else 0))

    def kernel_time(self):
        """(summed cone-kernel ms, cone-kernel launches, all launches) since the last read."""
        ms = C.c_double()
        n = C.c_int64()
        a = C.c_int64()
        _check(lib().qaoa_kernel_time(self._h, C.byref(ms), C.byref(n), C.byref(a)))
        return ms.value, n.value, a.value

    def device_status(self):
        s = C.c_int32()
        _check(lib().qaoa_device_status(self._h, C.byref(s)))
        return s.value


class PlanGraph:
    """One energy (or energy + gradient) evaluation captured as a CUDA graph.

    ``params`` is copied into a buffer the graph owns a pointer to; call
    :meth:`run` with new parameters (same shape) to replay the graph; the
    outputs ``energy``, ``grad`` and ``terms`` are overwritten in place.
    """

    def __init__(self, plan, params, grad=True, terms=False):
        import torch
        params = plan._params(params)
        G, P = params.shape[0], params.shape[1]
        self.plan = plan
        self.params = params.clone()
        dev = params.device
        self.energy = torch.empty(G, P, dtype=torch.float64, device=dev)
        self.grad = torch.empty(G, P, 2 * plan.p, dtype=torch.float64, device=dev) if grad else None
        self.terms = torch.empty(plan.info()["n_reps"], P, dtype=torch.float64, device=dev) if terms else None
        h = C.c_void_p()
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        _check(lib().qaoa_graph_create(plan.handle, P, ptr(self.params), ptr(self.energy), ptr(self.grad),
                                       ptr(self.terms), C.byref(h)))
        self._h = h

    def run(self, params=None, stream=None):
        """Replays the graph; ``params`` (optional) is copied into its buffer
        first: a CUDA float64 tensor, or a host float64 tensor of the same
        shape (pinned, for an asynchronous copy)."""
        if params is not None:
            import torch
            if isinstance(params, torch.Tensor) and not params.is_cuda:
                if params.dtype != torch.float64 or params.numel() != self.params.numel():
                    raise ValueError(f"params must be float64 with {self.params.numel()} elements")
                self.params.copy_(params.reshape(self.params.shape), non_blocking=True)
            else:
                self.params.copy_(self.plan._params(params))
        _check(lib().qaoa_graph_launch(self._h, _stream_handle(stream)))
        return (self.energy, self.grad) if self.grad is not None else self.energy

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().qaoa_graph_free(self._h)
            self._h = C.c_void_p()

    __del__ = close


def _autograd_cls():
    import torch

    class QAOAEnergy(torch.autograd.Function):
        """E(theta) with dE/dtheta from the adjoint kernels (one launch does both)."""

        @staticmethod
        def forward(ctx, params, plan):
            ctx.shape = params.shape
            if params.requires_grad:
                e, g = plan.energy_grad(params.detach())
                ctx.save_for_backward(g)
            else:
                e = plan.energy(params.detach())
            return e

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return (grad_out.reshape(g.shape[:-1]).unsqueeze(-1) * g).reshape(ctx.shape), None

    return QAOAEnergy


_QAOAEnergy = None


def qaoa_energy(params, plan):
    """Differentiable E(params) for ``plan`` (params: CUDA float64 [G, P, 2p])."""
    global _QAOAEnergy
    if _QAOAEnergy is None:
        _QAOAEnergy = _autograd_cls()
    return _QAOAEnergy.apply(params, plan)
