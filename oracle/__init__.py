"""CPU oracle for SCLaP, contraction, projection and the multilevel driver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library; the two only see the same seeded inputs.

The arithmetic lives in ``sclap_oracle.c`` (plain C, one thread); this module
compiles it with gcc on first use and wraps it with ctypes.  Function names
and argument order follow the C file, which cites the paper section each
routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sclap_oracle.c")
_HDR = os.path.join(_HERE, "sclap_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libsclap_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EGRAPH, EOVERFLOW, ENOMEM = 0, 1, 2, 3, 4
MAX_LEVELS = 64


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc -O2, plain C99)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(p) > os.path.getmtime(_SO) for p in (_SRC, _HDR))
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o",
                               tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class MLParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("eps", C.c_double), ("U", C.c_int64),
                ("cluster_rounds", C.c_int32), ("refine_rounds", C.c_int32),
                ("subrounds", C.c_int32), ("n_stop", C.c_int64),
                ("max_levels", C.c_int32), ("init_seeds", C.c_int32),
                ("init_rounds", C.c_int32), ("seed", C.c_uint64), ("degree_order", C.c_int32)]


class MLStats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n", C.c_int64 * MAX_LEVELS),
                ("nnz", C.c_int64 * MAX_LEVELS),
                ("cluster_rounds_done", C.c_int32 * MAX_LEVELS),
                ("refine_rounds_done", C.c_int32 * MAX_LEVELS),
                ("U", C.c_int64), ("lmax", C.c_int64), ("init_best", C.c_int32),
                ("init_cut", C.c_int64), ("init_maxbw", C.c_int64),
                ("cut", C.c_int64), ("maxbw", C.c_int64)]


_P64 = C.POINTER(C.c_int64)
_P32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # SCLAP_ORACLE_LIB: a prebuilt variant (the mutation tests plant
            # deliberate mistakes in a copy of the C source and load it here)
            L = C.CDLL(os.environ.get("SCLAP_ORACLE_LIB") or build())
            L.or_mix64.restype = C.c_uint64
            L.or_mix64.argtypes = [C.c_uint64]
            L.or_colour.restype = C.c_uint32
            L.or_colour.argtypes = [C.c_uint64, C.c_int32, C.c_int64, C.c_int32]
            L.or_tie.restype = C.c_uint32
            L.or_tie.argtypes = [C.c_uint64, C.c_int32, C.c_int64, C.c_int64]
            L.or_lmax.restype = C.c_int64
            L.or_lmax.argtypes = [C.c_int64, C.c_int32, C.c_double]
            g = [C.c_int64, _P64, _P32, _P32, _P32]
            L.or_validate.argtypes = g
            L.or_cluster.argtypes = g + [C.c_int64, C.c_int32, C.c_int32, C.c_uint64, _P32,
                                         _P32, _P32, _P64]
            L.or_cluster_degree_ordered.argtypes = L.or_cluster.argtypes
            L.or_degree_colours.argtypes = [C.c_int64, _P64, C.c_uint64, C.c_int32, C.c_int32,
                                            _P32]
            L.or_refine_bound.argtypes = g + [C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                              C.c_uint64, _P32, _P32, _P64]
            L.or_refine.argtypes = g + [C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                        C.c_uint64, _P32, _P64, _P64, _P32, _P64]
            L.or_contract.argtypes = g + [_P32, _P64, _P64, C.POINTER(_P64), C.POINTER(_P32),
                                          C.POINTER(_P32), C.POINTER(_P32), _P32]
            L.or_free.argtypes = [C.c_void_p]
            L.or_project.argtypes = [C.c_int64, _P32, _P32, _P32]
            L.or_cut.restype = C.c_int64
            L.or_cut.argtypes = [C.c_int64, _P64, _P32, _P32, _P32]
            L.or_block_weights.argtypes = [C.c_int64, _P32, _P32, C.c_int32, _P64]
            L.or_initial_partition.argtypes = g + [C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                                   C.c_int32, C.c_uint64, _P32, _P64, _P64, _P32]
            L.or_multilevel.argtypes = g + [C.POINTER(MLParams), _P32, C.POINTER(MLStats)]
            L.or_vcycle.argtypes = g + [C.POINTER(MLParams), _P32, C.POINTER(MLStats)]
            _PP64 = C.POINTER(_P64)
            _PP32 = C.POINTER(_P32)
            _PU64 = C.POINTER(C.c_uint64)
            L.or_refine_batched.argtypes = [C.c_int32, _P64, _PP64, _PP32, _PP32, _PP32,
                                            C.c_int32, _P64, C.c_int32, C.c_int32, _PU64,
                                            C.c_int32, _P32, _P32, _P64, _P64]
            L.or_lpt_start.argtypes = [C.c_int64, _P32, C.c_int32, C.c_uint64, _P32]
            _PF = C.POINTER(C.c_float)
            _PU8 = C.POINTER(C.c_uint8)
            _PU16 = C.POINTER(C.c_uint16)
            L.or_set_threads.argtypes = [C.c_int]
            L.or_get_threads.restype = C.c_int
            L.or_bf16.restype = C.c_float
            L.or_bf16.argtypes = [C.c_float]
            L.or_log2_feature.restype = C.c_float
            L.or_log2_feature.argtypes = [C.c_int64]
            L.or_features.argtypes = [C.c_int64, _P64, _P32, _P32, _P32, _P64, C.c_int64, _PU8,
                                      _P64, _P64, _PF]
            L.or_mlp_score.argtypes = [C.c_int64, _PF, _PU16, _PF]
            L.or_refine_learned.argtypes = g + [C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                                C.c_uint64, _PU16, C.c_float, C.c_int32, _P32,
                                                _P32, _P64, _P64, _PF, _PU8]
            L.or_mlp_loss_grad.restype = C.c_double
            L.or_mlp_loss_grad.argtypes = [_PF, _PU8, C.c_int64, _PF, C.POINTER(C.c_double)]
            L.or_mlp_loss_grad_bf16.restype = C.c_double
            L.or_mlp_loss_grad_bf16.argtypes = [_PF, _PU8, C.c_int64, _PF,
                                                C.POINTER(C.c_double)]
            _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(_P64)


def _p32(a):
    return a.ctypes.data_as(_P32)


def _graph_args(g):
    xadj = np.ascontiguousarray(g["xadj"], dtype=np.int64)
    adjncy = np.ascontiguousarray(g["adjncy"], dtype=np.int32)
    adjwgt = np.ascontiguousarray(g["adjwgt"], dtype=np.int32)
    vwgt = np.ascontiguousarray(g["vwgt"], dtype=np.int32)
    n = len(xadj) - 1
    keep = (xadj, adjncy, adjwgt, vwgt)
    return keep, [n, _p64(xadj), _p32(adjncy), _p32(adjwgt), _p32(vwgt)]


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


def set_threads(t: int) -> None:
    """Threads of the oracle's per-node propose loop (results do not depend on it)."""
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return int(lib().or_get_threads())


def mix64(z: int) -> int:
    return int(lib().or_mix64(z & (2**64 - 1)))


def colour(seed: int, rnd: int, v: int, S: int) -> int:
    return int(lib().or_colour(seed, rnd, v, S))


def tie(seed: int, rnd: int, v: int, L: int) -> int:
    return int(lib().or_tie(seed, rnd, v, L))


def lmax(cV: int, k: int, eps: float) -> int:
    return int(lib().or_lmax(cV, k, eps))


def validate(g) -> int:
    keep, a = _graph_args(g)
    return int(lib().or_validate(*a))


def cluster(g, U, rounds, subrounds, seed, constraint_part=None, return_moves=False,
            degree_ordered=False):
    keep, a = _graph_args(g)
    n = a[0]
    lab = np.empty(n, np.int32)
    rd = C.c_int32(0)
    mv = np.zeros(max(rounds, 1), np.int64)
    cp = None if constraint_part is None else np.ascontiguousarray(constraint_part, np.int32)
    fn = lib().or_cluster_degree_ordered if degree_ordered else lib().or_cluster
    rc = fn(*a, U, rounds, subrounds, seed, None if cp is None else _p32(cp),
            _p32(lab), C.byref(rd), _p64(mv))
    _check(rc, "cluster")
    if return_moves:
        return lab, rd.value, mv[:rd.value].copy()
    return lab, rd.value


def degree_colours(g, seed, rnd, S):
    """Sub-round of every node in round rnd under degree-ordered colours."""
    xadj = np.ascontiguousarray(g["xadj"], dtype=np.int64)
    n = xadj.size - 1
    out = np.empty(n, np.int32)
    _check(lib().or_degree_colours(n, _p64(xadj), seed, rnd, S, _p32(out)), "degree_colours")
    return out


def refine_bound(g, nblocks, B, rounds, subrounds, seed, part, return_moves=False):
    keep, a = _graph_args(g)
    p = np.array(part, dtype=np.int32, copy=True)
    rd = C.c_int32(0)
    mv = np.zeros(max(rounds, 1), np.int64)
    rc = lib().or_refine_bound(*a, nblocks, B, rounds, subrounds, seed, _p32(p), C.byref(rd),
                               _p64(mv))
    _check(rc, "refine_bound")
    if return_moves:
        return p, rd.value, mv[:rd.value].copy()
    return p, rd.value


def refine(g, k, eps, rounds, subrounds, seed, part):
    """Returns (part, cut, block_weights, rounds_done)."""
    keep, a = _graph_args(g)
    p = np.array(part, dtype=np.int32, copy=True)
    cut = C.c_int64(0)
    bw = np.zeros(k, np.int64)
    rd = C.c_int32(0)
    rc = lib().or_refine(*a, k, eps, rounds, subrounds, seed, _p32(p), C.byref(cut), _p64(bw),
                         C.byref(rd), None)
    _check(rc, "refine")
    return p, cut.value, bw, rd.value


def contract(g, labels):
    """Returns (coarse graph dict, f2c)."""
    keep, a = _graph_args(g)
    n = a[0]
    lab = np.ascontiguousarray(labels, np.int32)
    f2c = np.empty(n, np.int32)
    cn, cnnz = C.c_int64(0), C.c_int64(0)
    px, pa, pw, pv = _P64(), _P32(), _P32(), _P32()
    rc = lib().or_contract(*a, _p32(lab), C.byref(cn), C.byref(cnnz), C.byref(px), C.byref(pa),
                           C.byref(pw), C.byref(pv), _p32(f2c))
    _check(rc, "contract")
    n2, m2 = cn.value, cnnz.value
    out = {
        "xadj": np.ctypeslib.as_array(px, shape=(n2 + 1,)).copy(),
        "adjncy": np.ctypeslib.as_array(pa, shape=(max(m2, 1),))[:m2].copy(),
        "adjwgt": np.ctypeslib.as_array(pw, shape=(max(m2, 1),))[:m2].copy(),
        "vwgt": np.ctypeslib.as_array(pv, shape=(max(n2, 1),))[:n2].copy(),
    }
    for p in (px, pa, pw, pv):
        lib().or_free(C.cast(p, C.c_void_p))
    return out, f2c


def project(f2c, coarse_part):
    f2c = np.ascontiguousarray(f2c, np.int32)
    cp = np.ascontiguousarray(coarse_part, np.int32)
    out = np.empty(len(f2c), np.int32)
    lib().or_project(len(f2c), _p32(f2c), _p32(cp), _p32(out))
    return out


def cut(g, part) -> int:
    keep, a = _graph_args(g)
    p = np.ascontiguousarray(part, np.int32)
    return int(lib().or_cut(a[0], a[1], a[2], a[3], _p32(p)))


def block_weights(g, part, k):
    vw = np.ascontiguousarray(g["vwgt"], np.int32)
    p = np.ascontiguousarray(part, np.int32)
    bw = np.zeros(k, np.int64)
    lib().or_block_weights(len(vw), _p32(vw), _p32(p), k, _p64(bw))
    return bw


def initial_partition(g, k, B, P, rounds, subrounds, seed):
    """Returns (part, cuts[P], maxbw[P], best)."""
    keep, a = _graph_args(g)
    part = np.empty(a[0], np.int32)
    cuts = np.zeros(P, np.int64)
    mx = np.zeros(P, np.int64)
    best = C.c_int32(0)
    rc = lib().or_initial_partition(*a, k, B, P, rounds, subrounds, seed, _p32(part),
                                    _p64(cuts), _p64(mx), C.byref(best))
    _check(rc, "initial_partition")
    return part, cuts, mx, best.value


def lpt_start(g, k, seed):
    """The LPT start of one run (see or_lpt_start): block per node."""
    vw = np.ascontiguousarray(g["vwgt"], np.int32)
    part = np.empty(len(vw), np.int32)
    _check(lib().or_lpt_start(len(vw), _p32(vw), k, seed & (2**64 - 1), _p32(part)), "lpt_start")
    return part


def refine_batched(graphs, k, eps, rounds, subrounds, seeds, run_graph):
    """Batched runs, run r on graph run_graph[r] with seed seeds[r] (see
    or_refine_batched).  Returns (list of per-run partitions, cuts[nruns],
    maxbw[nruns])."""
    keeps = [_graph_args(g) for g in graphs]
    ng = len(graphs)
    ns = np.array([a[0] for _, a in keeps], np.int64)
    xs = (_P64 * ng)(*[a[1] for _, a in keeps])
    As = (_P32 * ng)(*[a[2] for _, a in keeps])
    Ws = (_P32 * ng)(*[a[3] for _, a in keeps])
    Cs = (_P32 * ng)(*[a[4] for _, a in keeps])
    Bg = np.array([lmax(int(np.asarray(g["vwgt"], np.int64).sum()), k, eps) for g in graphs],
                  np.int64)
    rg = np.ascontiguousarray(run_graph, np.int32)
    nr = len(rg)
    sd = np.ascontiguousarray([int(x) & (2**64 - 1) for x in seeds], np.uint64)
    if len(sd) != nr:
        raise ValueError("one seed per run")
    tot = int(sum(ns[g] for g in rg))
    parts = np.empty(max(tot, 1), np.int32)
    cuts = np.zeros(nr, np.int64)
    mx = np.zeros(nr, np.int64)
    rc = lib().or_refine_batched(ng, _p64(ns), xs, As, Ws, Cs, k, _p64(Bg), rounds, subrounds,
                                 sd.ctypes.data_as(C.POINTER(C.c_uint64)), nr, _p32(rg),
                                 _p32(parts), _p64(cuts), _p64(mx))
    _check(rc, "refine_batched")
    out, off = [], 0
    for g in rg:
        out.append(parts[off:off + ns[g]].copy())
        off += ns[g]
    return out, cuts, mx


def default_params(k, eps=0.03, seed=1, **kw):
    p = dict(k=k, eps=eps, U=0, cluster_rounds=3, refine_rounds=6, subrounds=4, n_stop=2000,
             max_levels=32, init_seeds=8, init_rounds=6, seed=seed, degree_order=0)
    p.update(kw)
    return p


def _ml_stats(st):
    L = st.levels
    return dict(levels=L, n=list(st.n[:L]), nnz=list(st.nnz[:L]),
                cluster_rounds_done=list(st.cluster_rounds_done[:L]),
                refine_rounds_done=list(st.refine_rounds_done[:L]), U=st.U, lmax=st.lmax,
                init_best=st.init_best, init_cut=st.init_cut, init_maxbw=st.init_maxbw,
                cut=st.cut, maxbw=st.maxbw)


def vcycle(g, params: dict, part):
    """One V-cycle seeded by `part`.  Returns (part, stats dict)."""
    keep, a = _graph_args(g)
    p = np.array(part, dtype=np.int32, copy=True)
    mp = MLParams(**params)
    st = MLStats()
    rc = lib().or_vcycle(*a, C.byref(mp), _p32(p), C.byref(st))
    _check(rc, "vcycle")
    return p, _ml_stats(st)


def multilevel(g, params: dict):
    """Returns (part, stats dict)."""
    keep, a = _graph_args(g)
    part = np.empty(a[0], np.int32)
    mp = MLParams(**params)
    st = MLStats()
    rc = lib().or_multilevel(*a, C.byref(mp), _p32(part), C.byref(st))
    _check(rc, "multilevel")
    L = st.levels
    stats = dict(levels=L, n=list(st.n[:L]), nnz=list(st.nnz[:L]),
                 cluster_rounds_done=list(st.cluster_rounds_done[:L]),
                 refine_rounds_done=list(st.refine_rounds_done[:L]), U=st.U, lmax=st.lmax,
                 init_best=st.init_best, init_cut=st.init_cut, init_maxbw=st.init_maxbw,
                 cut=st.cut, maxbw=st.maxbw)
    return part, stats


# ---------------------------------------------------------------- learned gate

MLP_NPARAM = 1313
MLP_LAYOUT = {"W1": (0, (32, 6)), "b1": (192, (32,)), "W2": (224, (32, 32)),
              "b2": (1248, (32,)), "W3": (1280, (32,)), "b3": (1312, (1,))}


def _pf(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _pu8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _pu16(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint16))


def bf16(x: float) -> float:
    """bfloat16 rounding (nearest, ties to even) of a float32."""
    return float(lib().or_bf16(C.c_float(x)))


def log2_feature(x: int) -> float:
    return float(lib().or_log2_feature(x))


def features(g, lab, W, lmax, moved=None, vis_best=None, vis_own=None):
    """Six bf16-rounded features per node, float32 [n, 6] (see or_features)."""
    keep, a = _graph_args(g)
    n = a[0]
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    W = np.ascontiguousarray(W, dtype=np.int64)
    mv = None if moved is None else np.ascontiguousarray(moved, dtype=np.uint8)
    vb = None if vis_best is None else np.ascontiguousarray(vis_best, dtype=np.int64)
    vo = None if vis_own is None else np.ascontiguousarray(vis_own, dtype=np.int64)
    x = np.zeros((n, 6), np.float32)
    lib().or_features(n, a[1], a[2], a[3], _p32(lab), _p64(W), lmax,
                      None if mv is None else _pu8(mv), None if vb is None else _p64(vb),
                      None if vo is None else _p64(vo), _pf(x))
    return x


def mlp_score(X, net_bf16):
    """Logits of the bf16 network (uint16 [1313]) on feature rows X [N, 6]."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    net = np.ascontiguousarray(net_bf16, dtype=np.uint16)
    z = np.zeros(X.shape[0], np.float32)
    lib().or_mlp_score(X.shape[0], _pf(X), _pu16(net), _pf(z))
    return z


def refine_learned(g, k, eps, rounds, subrounds, seed, part, net_bf16=None, z_min=0.0,
                   full_every=3, trace=False):
    """Returns (part, moves per round, visited, trace_x or None, trace_y or None)."""
    keep, a = _graph_args(g)
    n = a[0]
    p = np.array(part, dtype=np.int32, copy=True)
    rd = C.c_int32(0)
    moves = np.zeros(max(rounds, 1), np.int64)
    visited = C.c_int64(0)
    net = None if net_bf16 is None else np.ascontiguousarray(net_bf16, dtype=np.uint16)
    tx = np.zeros((rounds, n, 6), np.float32) if trace else None
    ty = np.zeros((rounds, n), np.uint8) if trace else None
    rc = lib().or_refine_learned(*a, k, eps, rounds, subrounds, seed,
                                 None if net is None else _pu16(net), z_min, full_every,
                                 _p32(p), C.byref(rd), _p64(moves), C.byref(visited),
                                 None if tx is None else _pf(tx), None if ty is None else _pu8(ty))
    _check(rc, "refine_learned")
    r = rd.value
    return (p, moves[:r].copy(), visited.value, None if tx is None else tx[:r],
            None if ty is None else ty[:r])


def mlp_loss_grad(X, y, params, bf16_in=False):
    """Mean logistic loss and its gradient (float64 [1313]) of float32
    parameters: of the float network, or with bf16_in of the network inference
    runs (bf16 parameters and hidden outputs, straight-through gradient)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    prm = np.ascontiguousarray(params, dtype=np.float32)
    grad = np.zeros(MLP_NPARAM, np.float64)
    fn = lib().or_mlp_loss_grad_bf16 if bf16_in else lib().or_mlp_loss_grad
    loss = fn(_pf(X), _pu8(y), X.shape[0], _pf(prm), grad.ctypes.data_as(C.POINTER(C.c_double)))
    return float(loss), grad
