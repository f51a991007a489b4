"""paper_1404_4797_gb300 -- size-constrained label propagation (SCLaP), cluster
contraction, projection and the multilevel partitioner of Meyerhenke, Sanders
and Schulz (2014) on one GB300 GPU.

This module is a thin ctypes binding over the C ABI in include/sclap.h (the
library _build/libsclap.so, built by ``build.py``).  It only marshals arguments:
every step runs in the library's CUDA kernels.  There is no CPU fallback; if the
library is missing every call raises.

Graphs are dicts of tensors: xadj int64 [n+1], adjncy int32 [nnz], adjwgt int32
[nnz], vwgt int32 [n] (see ``inputs``).  Device entry points want CUDA tensors;
``partition_multilevel`` also accepts CPU (ideally pinned) tensors and then
copies them to the GPU inside the call.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsclap.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EGRAPH, EOVERFLOW, ENOMEM, ECUDA, ETIMEOUT, ENOTIMPL = range(8)
MAX_LEVELS = 64


class SclapError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} (code {code})")
        self.code = code


class Graph(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("xadj", C.c_void_p),
                ("adjncy", C.c_void_p), ("adjwgt", C.c_void_p), ("vwgt", C.c_void_p)]


class GraphOwned(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("xadj", C.c_void_p),
                ("adjncy", C.c_void_p), ("adjwgt", C.c_void_p), ("vwgt", C.c_void_p)]


class Batch(C.Structure):
    _fields_ = [("ngraphs", C.c_int32), ("graphs", C.POINTER(Graph))]


class MLParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("eps", C.c_double), ("U", C.c_int64),
                ("cluster_rounds", C.c_int32), ("refine_rounds", C.c_int32),
                ("subrounds", C.c_int32), ("n_stop", C.c_int64), ("max_levels", C.c_int32),
                ("init_seeds", C.c_int32), ("init_rounds", C.c_int32), ("seed", C.c_uint64),
                ("degree_order", C.c_int32)]


class MLStats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n", C.c_int64 * MAX_LEVELS),
                ("nnz", C.c_int64 * MAX_LEVELS),
                ("cluster_rounds_done", C.c_int32 * MAX_LEVELS),
                ("refine_rounds_done", C.c_int32 * MAX_LEVELS),
                ("U", C.c_int64), ("lmax", C.c_int64), ("init_best", C.c_int32),
                ("init_cut", C.c_int64), ("init_maxbw", C.c_int64), ("cut", C.c_int64),
                ("maxbw", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("small_max", C.c_int32), ("med_max", C.c_int32), ("mid_max", C.c_int32),
                ("seg_smem", C.c_int32)]


class Prof(C.Structure):
    _fields_ = [("propose_launches", C.c_int64), ("propose_ms", C.c_double),
                ("propose_bytes", C.c_double), ("entries_scanned", C.c_int64),
                ("nodes_visited", C.c_int64), ("kernel_launches", C.c_int64),
                ("graph_launches", C.c_int64)]


_P64 = C.POINTER(C.c_int64)
_P32 = C.POINTER(C.c_int32)
_VP = C.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "sclap_strerror": (C.c_char_p, [C.c_int]),
    "sclap_set_validation": (C.c_int, [C.c_int]),
    "sclap_set_launch_mode": (C.c_int, [C.c_int]),
    "sclap_set_tuning": (C.c_int, [C.POINTER(Tuning)]),
    "sclap_get_tuning": (None, [C.POINTER(Tuning)]),
    "sclap_ml_defaults": (None, [C.POINTER(MLParams), C.c_int32, C.c_double, C.c_uint64]),
    "sclap_cluster": (C.c_int, [C.POINTER(Graph), C.c_int64, C.c_int32, C.c_int32, C.c_uint64,
                                _VP, _VP, _P32, _VP]),
    "sclap_cluster_degree_ordered": (C.c_int, [C.POINTER(Graph), C.c_int64, C.c_int32, C.c_int32,
                                               C.c_uint64, _VP, _VP, _P32, _VP]),
    "sclap_refine": (C.c_int, [C.POINTER(Graph), C.c_int32, C.c_double, C.c_int32, C.c_int32,
                               C.c_uint64, _VP, _P64, _P64, _P32, _VP]),
    "sclap_refine_bound": (C.c_int, [C.POINTER(Graph), C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                     C.c_uint64, _VP, _P32, _VP]),
    "contract_graph": (C.c_int, [C.POINTER(Graph), _VP, C.POINTER(GraphOwned), _VP, _VP]),
    "project_partition": (C.c_int, [C.c_int64, _VP, _VP, _VP, _VP]),
    "sclap_cut": (C.c_int, [C.POINTER(Graph), _VP, C.c_int32, _P64, _P64, _VP]),
    "sclap_cut_noalloc": (C.c_int, [C.POINTER(Graph), _VP, C.c_int32, _P64, _P64, _VP]),
    "sclap_initial_partition": (C.c_int, [C.POINTER(Graph), C.c_int32, C.c_int64, C.c_int32,
                                          C.c_int32, C.c_int32, C.c_uint64, _VP, _P64, _P64,
                                          _P32, _VP]),
    "sclap_refine_batched": (C.c_int, [C.POINTER(Batch), C.c_int32, C.c_double, C.c_int32,
                                       C.c_int32, C.c_int32, _P32, C.POINTER(C.c_uint64), _VP,
                                       _P64, _P64, _VP]),
    "partition_multilevel": (C.c_int, [C.POINTER(Graph), C.POINTER(MLParams), _VP,
                                       C.POINTER(MLStats), _VP]),
    "sclap_vcycle": (C.c_int, [C.POINTER(Graph), C.POINTER(MLParams), _VP, C.POINTER(MLStats),
                               _VP]),
    "sclap_graph_copy_out": (C.c_int, [C.POINTER(GraphOwned), _VP, _VP, _VP, _VP, _VP]),
    "sclap_graph_free": (None, [C.POINTER(GraphOwned)]),
    "sclap_refine_learned": (C.c_int, [C.POINTER(Graph), C.c_int32, C.c_double, C.c_int32,
                                       C.c_int32, C.c_uint64, _VP, C.c_float, C.c_int32, _VP,
                                       _P64, _P64, _P32, _P64, _VP, _VP, _VP]),
    "sclap_mlp_score": (C.c_int, [_VP, C.c_int64, _VP, _VP, _VP]),
    "sclap_mlp_loss_grad": (C.c_int, [_VP, _VP, C.c_int64, _VP, C.c_int32, _VP,
                                      C.POINTER(C.c_double), _VP]),
    "sclap_mlp_train": (C.c_int, [_VP, _VP, C.c_int64, _VP, C.c_int32, C.c_int32, C.c_float,
                                  C.c_uint64, C.POINTER(C.c_double), _VP]),
    "sclap_mlp_pack_bf16": (C.c_int, [_VP, _VP, _VP]),
    "sclap_wait_selftest": (C.c_int, [C.c_int64]),
    "sclap_inject_alloc_failure": (C.c_int, [C.c_int64]),
    "sclap_prof_enable": (None, [C.c_int]),
    "sclap_prof_reset": (None, []),
    "sclap_prof_read": (C.c_int, [C.POINTER(Prof)]),
}

EXPORTS = tuple(_SIGS)


def lib():
    """Loads libsclap.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsclap.so not built ({LIB_PATH}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().sclap_strerror(code).decode()
    except Exception:  # library missing
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != OK:
        raise SclapError(rc, what)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _graph(g: dict) -> Graph:
    for key, dt in (("xadj", torch.int64), ("adjncy", torch.int32), ("adjwgt", torch.int32),
                    ("vwgt", torch.int32)):
        t = g[key]
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"graph[{key!r}] must be a contiguous {dt} tensor")
    return Graph(g["vwgt"].numel(), g["adjncy"].numel(), g["xadj"].data_ptr(),
                 g["adjncy"].data_ptr(), g["adjwgt"].data_ptr(), g["vwgt"].data_ptr())


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise TypeError("this entry point takes CUDA tensors")


def set_validation(on: bool) -> bool:
    return bool(lib().sclap_set_validation(1 if on else 0))


def set_launch_mode(mode: int) -> int:
    """How a call's SCLaP rounds are launched (0 one round at a time, 1 all
    enqueued ahead, 2 captured in a CUDA graph, -1 the default: 2 for batched
    runs, 0 otherwise; results do not depend on it).  Returns the previous
    mode."""
    return int(lib().sclap_set_launch_mode(int(mode)))


def get_tuning() -> dict:
    """The degree-bin and segment thresholds later calls use."""
    t = Tuning()
    lib().sclap_get_tuning(C.byref(t))
    return {name: getattr(t, name) for name, _ in Tuning._fields_}


def set_tuning(small_max: int, med_max: int, mid_max: int, seg_smem: int):
    """Sets the thresholds (results do not depend on them; see sclap.h)."""
    _check(lib().sclap_set_tuning(C.byref(Tuning(small_max, med_max, mid_max, seg_smem))),
           "sclap_set_tuning")


def sclap_cluster(g: dict, U: int, rounds: int, subrounds: int = 4, seed: int = 1,
                  constraint_part: torch.Tensor | None = None, stream=None,
                  degree_ordered: bool = False):
    """Size-constrained clustering (Sec. III.A), by hash-coloured or (with
    degree_ordered) degree-ordered sub-rounds.  Returns (labels, rounds_done)."""
    _require_cuda(g["xadj"], constraint_part)
    n = g["vwgt"].numel()
    labels = torch.empty(n, dtype=torch.int32, device=g["xadj"].device)
    rd = C.c_int32(0)
    gg = _graph(g)
    fn = lib().sclap_cluster_degree_ordered if degree_ordered else lib().sclap_cluster
    _check(fn(C.byref(gg), U, rounds, subrounds, seed & (2**64 - 1), _ptr(constraint_part),
              _ptr(labels), C.byref(rd), _stream(stream)), "sclap_cluster")
    return labels, rd.value


def sclap_refine(g: dict, k: int, eps: float, rounds: int, subrounds: int, seed: int,
                 part: torch.Tensor, stream=None):
    """SCLaP refinement (Sec. III.A).  Refines a copy of `part`; returns
    (part, cut, block_weights[k] (CPU int64 tensor), rounds_done)."""
    _require_cuda(g["xadj"], part)
    p = part.to(torch.int32).clone()
    cut = C.c_int64(0)
    bw = torch.zeros(k, dtype=torch.int64)
    rd = C.c_int32(0)
    gg = _graph(g)
    _check(lib().sclap_refine(C.byref(gg), k, eps, rounds, subrounds, seed & (2**64 - 1), _ptr(p),
                              C.byref(cut), C.cast(bw.data_ptr(), _P64), C.byref(rd),
                              _stream(stream)), "sclap_refine")
    return p, cut.value, bw, rd.value


MLP_PARAMS = 1313


def sclap_refine_learned(g: dict, k: int, eps: float, rounds: int, subrounds: int, seed: int,
                         part: torch.Tensor, net: torch.Tensor | None = None, z_min: float = 0.0,
                         full_every: int = 3, trace: bool = False, stream=None):
    """Refinement with the learned gate (see include/sclap.h).  `net`: device
    int16/uint16-bit bf16 parameters [1313] or None.  Returns (part, cut,
    block_weights, rounds_done, visited, trace_x [r, n, 6] or None,
    trace_y [r, n] or None)."""
    _require_cuda(g["xadj"], part)
    n = g["vwgt"].numel()
    p = part.to(torch.int32).clone()
    cut = C.c_int64(0)
    bw = torch.zeros(k, dtype=torch.int64)
    rd = C.c_int32(0)
    vis = C.c_int64(0)
    if net is not None and (net.numel() != MLP_PARAMS or net.element_size() != 2):
        raise TypeError("net must hold 1313 bf16 bit patterns (16-bit elements)")
    tx = torch.zeros((max(rounds, 1), n, 6), dtype=torch.float32, device=p.device) if trace else None
    ty = torch.zeros((max(rounds, 1), n), dtype=torch.uint8, device=p.device) if trace else None
    gg = _graph(g)
    _check(lib().sclap_refine_learned(C.byref(gg), k, eps, rounds, subrounds, seed & (2**64 - 1),
                                      _ptr(net), z_min, full_every, _ptr(p), C.byref(cut),
                                      C.cast(bw.data_ptr(), _P64), C.byref(rd), C.byref(vis),
                                      _ptr(tx), _ptr(ty), _stream(stream)),
           "sclap_refine_learned")
    r = rd.value
    return (p, cut.value, bw, r, vis.value, None if tx is None else tx[:r],
            None if ty is None else ty[:r])


def sclap_mlp_score(x: torch.Tensor, net: torch.Tensor, stream=None) -> torch.Tensor:
    """Logits of the bf16 network on feature rows x (device float32 [N, 6])."""
    _require_cuda(x, net)
    x = x.to(torch.float32).contiguous()
    z = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().sclap_mlp_score(_ptr(x), x.shape[0], _ptr(net), _ptr(z), _stream(stream)),
           "sclap_mlp_score")
    return z


def sclap_mlp_loss_grad(x: torch.Tensor, y: torch.Tensor, params: torch.Tensor,
                        bf16_in: bool = False, stream=None):
    """Mean logistic loss and gradient (device float32 [1313]) of float params
    (bf16_in: of the bf16 network inference runs, straight-through gradient)."""
    _require_cuda(x, y, params)
    x = x.to(torch.float32).contiguous()
    y = y.to(torch.uint8).contiguous()
    params = params.to(torch.float32).contiguous()
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = C.c_double(0)
    _check(lib().sclap_mlp_loss_grad(_ptr(x), _ptr(y), x.shape[0], _ptr(params),
                                     1 if bf16_in else 0, _ptr(grad), C.byref(loss),
                                     _stream(stream)), "sclap_mlp_loss_grad")
    return loss.value, grad


def sclap_mlp_train(x: torch.Tensor, y: torch.Tensor, params: torch.Tensor, epochs: int,
                    batch: int, lr: float, seed: int, stream=None):
    """Minibatch SGD on the scorer; trains a copy of params.  Returns (params, loss)."""
    _require_cuda(x, y, params)
    x = x.to(torch.float32).contiguous()
    y = y.to(torch.uint8).contiguous()
    prm = params.to(torch.float32).clone().contiguous()
    loss = C.c_double(0)
    _check(lib().sclap_mlp_train(_ptr(x), _ptr(y), x.shape[0], _ptr(prm), epochs, batch, lr,
                                 seed & (2**64 - 1), C.byref(loss), _stream(stream)),
           "sclap_mlp_train")
    return prm, loss.value


def bf16_bits(params: torch.Tensor, stream=None) -> torch.Tensor:
    """The bf16 network (int16 bit patterns, nearest-even rounding) of float
    scorer parameters, computed by the library (sclap_mlp_pack_bf16)."""
    _require_cuda(params)
    prm = params.to(torch.float32).contiguous()
    if prm.numel() != MLP_PARAMS:
        raise TypeError("params must hold 1313 floats")
    net = torch.empty(MLP_PARAMS, dtype=torch.int16, device=prm.device)
    _check(lib().sclap_mlp_pack_bf16(_ptr(prm), _ptr(net), _stream(stream)), "sclap_mlp_pack_bf16")
    return net


def sclap_refine_bound(g: dict, nblocks: int, B: int, rounds: int, subrounds: int, seed: int,
                       part: torch.Tensor, stream=None):
    """Refinement with an explicit bound B on each of `nblocks` blocks.  Returns
    (part, rounds_done)."""
    _require_cuda(g["xadj"], part)
    p = part.to(torch.int32).clone()
    rd = C.c_int32(0)
    gg = _graph(g)
    _check(lib().sclap_refine_bound(C.byref(gg), nblocks, B, rounds, subrounds,
                                    seed & (2**64 - 1), _ptr(p), C.byref(rd), _stream(stream)),
           "sclap_refine_bound")
    return p, rd.value


def contract_graph(g: dict, labels: torch.Tensor, stream=None):
    """Cluster contraction (Sec. III, Sec. IV.C).  Returns (coarse graph, f2c)."""
    _require_cuda(g["xadj"], labels)
    dev = g["xadj"].device
    n = g["vwgt"].numel()
    f2c = torch.empty(n, dtype=torch.int32, device=dev)
    out = GraphOwned()
    gg = _graph(g)
    st = _stream(stream)
    _check(lib().contract_graph(C.byref(gg), _ptr(labels.to(torch.int32)), C.byref(out),
                                _ptr(f2c), st), "contract_graph")
    try:
        cg = {"xadj": torch.empty(out.n + 1, dtype=torch.int64, device=dev),
              "adjncy": torch.empty(out.nnz, dtype=torch.int32, device=dev),
              "adjwgt": torch.empty(out.nnz, dtype=torch.int32, device=dev),
              "vwgt": torch.empty(out.n, dtype=torch.int32, device=dev)}
        _check(lib().sclap_graph_copy_out(C.byref(out), _ptr(cg["xadj"]), _ptr(cg["adjncy"]),
                                          _ptr(cg["adjwgt"]), _ptr(cg["vwgt"]), st),
               "sclap_graph_copy_out")
    finally:
        lib().sclap_graph_free(C.byref(out))
    return cg, f2c


def project_partition(f2c: torch.Tensor, coarse_part: torch.Tensor, stream=None):
    """Uncoarsening (Sec. IV.C): fine_part[v] = coarse_part[f2c[v]]."""
    _require_cuda(f2c, coarse_part)
    out = torch.empty_like(f2c, dtype=torch.int32)
    _check(lib().project_partition(f2c.numel(), _ptr(f2c), _ptr(coarse_part), _ptr(out),
                                   _stream(stream)), "project_partition")
    return out


def sclap_cut(g: dict, part: torch.Tensor, k: int, stream=None):
    """Returns (cut, block_weights[k] as a CPU int64 tensor)."""
    _require_cuda(g["xadj"], part)
    cut = C.c_int64(0)
    bw = torch.zeros(k, dtype=torch.int64)
    gg = _graph(g)
    _check(lib().sclap_cut(C.byref(gg), _ptr(part), k, C.byref(cut), C.cast(bw.data_ptr(), _P64),
                           _stream(stream)), "sclap_cut")
    return cut.value, bw


def sclap_cut_noalloc(g: dict, part: torch.Tensor, k: int, stream=None):
    """Like sclap_cut, but the library allocates nothing (its accumulators are a
    fixed device array; k <= 65536).  Returns (cut, block_weights[k] on the CPU)."""
    _require_cuda(g["xadj"], part)
    cut = C.c_int64(0)
    bw = torch.zeros(k, dtype=torch.int64)
    gg = _graph(g)
    _check(lib().sclap_cut_noalloc(C.byref(gg), _ptr(part), k, C.byref(cut),
                                   C.cast(bw.data_ptr(), _P64), _stream(stream)),
           "sclap_cut_noalloc")
    return cut.value, bw


def sclap_initial_partition(g: dict, k: int, B: int, P: int, rounds: int, subrounds: int,
                            seed: int, stream=None):
    """Initial partition (stand-in for the evolutionary partitioner).  Returns
    (part, cuts[P], maxbw[P], best)."""
    _require_cuda(g["xadj"])
    part = torch.empty(g["vwgt"].numel(), dtype=torch.int32, device=g["xadj"].device)
    cuts = torch.zeros(P, dtype=torch.int64)
    mx = torch.zeros(P, dtype=torch.int64)
    best = C.c_int32(0)
    gg = _graph(g)
    _check(lib().sclap_initial_partition(C.byref(gg), k, B, P, rounds, subrounds,
                                         seed & (2**64 - 1), _ptr(part),
                                         C.cast(cuts.data_ptr(), _P64),
                                         C.cast(mx.data_ptr(), _P64), C.byref(best),
                                         _stream(stream)), "sclap_initial_partition")
    return part, cuts, mx, best.value


def sclap_refine_batched(graphs: list, k: int, eps: float, rounds: int, subrounds: int,
                         seeds, run_graph, stream=None):
    """Batched SCLaP runs over uneven graphs (the population stand-in): run r
    on graph run_graph[r] with seed seeds[r].  Returns (list of per-run
    partitions (CUDA int32), cuts[nruns], maxbw[nruns])."""
    for g in graphs:
        _require_cuda(g["xadj"])
    views = (Graph * len(graphs))(*[_graph(g) for g in graphs])
    b = Batch(len(graphs), views)
    rg = torch.as_tensor(list(run_graph), dtype=torch.int32)
    sd = (C.c_uint64 * len(rg))(*[int(x) & (2**64 - 1) for x in seeds])
    if len(sd) != len(rg):
        raise ValueError("one seed per run")
    ns = [graphs[i]["vwgt"].numel() for i in rg.tolist()]
    parts = torch.empty(max(sum(ns), 1), dtype=torch.int32, device=graphs[0]["xadj"].device)
    cuts = torch.zeros(len(ns), dtype=torch.int64)
    mx = torch.zeros(len(ns), dtype=torch.int64)
    _check(lib().sclap_refine_batched(C.byref(b), k, eps, rounds, subrounds, len(ns),
                                      C.cast(rg.data_ptr(), _P32), sd, _ptr(parts),
                                      C.cast(cuts.data_ptr(), _P64), C.cast(mx.data_ptr(), _P64),
                                      _stream(stream)), "sclap_refine_batched")
    out, off = [], 0
    for n in ns:
        out.append(parts[off:off + n])
        off += n
    return out, cuts, mx


def default_params(k: int, eps: float = 0.03, seed: int = 1, **kw) -> dict:
    p = MLParams()
    lib().sclap_ml_defaults(C.byref(p), k, eps, seed & (2**64 - 1))
    d = {name: getattr(p, name) for name, _ in MLParams._fields_}
    d.update(kw)
    return d


def partition_multilevel(g: dict, params: dict, part_out: torch.Tensor | None = None,
                         stream=None):
    """The multilevel partitioner (Sec. IV.E).  Graph tensors may live on the GPU
    or on the host; `part_out` (int32 [n]) may be either too (default: same
    device as the graph).  Returns (part, stats dict)."""
    n = g["vwgt"].numel()
    if part_out is None:
        part_out = torch.empty(n, dtype=torch.int32, device=g["xadj"].device)
    mp = MLParams(**params)
    st = MLStats()
    gg = _graph(g)
    _check(lib().partition_multilevel(C.byref(gg), C.byref(mp), _ptr(part_out), C.byref(st),
                                      _stream(stream)), "partition_multilevel")
    L = st.levels
    stats = dict(levels=L, n=list(st.n[:L]), nnz=list(st.nnz[:L]),
                 cluster_rounds_done=list(st.cluster_rounds_done[:L]),
                 refine_rounds_done=list(st.refine_rounds_done[:L]), U=st.U, lmax=st.lmax,
                 init_best=st.init_best, init_cut=st.init_cut, init_maxbw=st.init_maxbw,
                 cut=st.cut, maxbw=st.maxbw)
    return part_out, stats


def sclap_vcycle(g: dict, params: dict, part: torch.Tensor, stream=None):
    """One iterated V-cycle seeded by `part` (Sec. IV.E); works on a copy.
    Returns (part, stats dict)."""
    p = part.to(torch.int32).clone()
    mp = MLParams(**params)
    st = MLStats()
    gg = _graph(g)
    _check(lib().sclap_vcycle(C.byref(gg), C.byref(mp), _ptr(p), C.byref(st), _stream(stream)),
           "sclap_vcycle")
    L = st.levels
    stats = dict(levels=L, n=list(st.n[:L]), nnz=list(st.nnz[:L]),
                 cluster_rounds_done=list(st.cluster_rounds_done[:L]),
                 refine_rounds_done=list(st.refine_rounds_done[:L]), U=st.U, lmax=st.lmax,
                 init_best=st.init_best, init_cut=st.init_cut, init_maxbw=st.init_maxbw,
                 cut=st.cut, maxbw=st.maxbw)
    return p, stats


def inject_alloc_failure(after: int):
    """Makes the library's scratch allocation number `after` (counted from
    now) fail as out of memory; -1 turns the injection off (a test hook)."""
    _check(lib().sclap_inject_alloc_failure(int(after)), "sclap_inject_alloc_failure")


def wait_selftest(limit_cycles: int) -> int:
    """Runs the arbitration barrier with one CTA absent (see sclap_wait_selftest);
    returns the status code (ETIMEOUT is the expected one)."""
    return int(lib().sclap_wait_selftest(int(limit_cycles)))


def prof_enable(on: bool = True):
    lib().sclap_prof_enable(1 if on else 0)


def prof_reset():
    lib().sclap_prof_reset()


def prof_read() -> dict:
    p = Prof()
    _check(lib().sclap_prof_read(C.byref(p)), "sclap_prof_read")
    return {name: getattr(p, name) for name, _ in Prof._fields_}
