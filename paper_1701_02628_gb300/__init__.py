"""GB300 (sm_103a) bipartite-graph partial coloring and distance-2 coloring.

Thin Python binding of the C ABI declared in ``include/bgpc.h``: argument
marshalling only.  Every step of the coloring runs in the CUDA kernels of
``libbgpc_gb300.so``; there is no CPU fallback, and importing the functions
below raises if the library has not been built (``build.build()``).

PyTorch is used for device memory and streams: graph arrays are int32 CUDA
tensors, colors come back as an int32 CUDA tensor, and every call runs on the
current torch stream unless one is given.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

BGPC_OK, BGPC_STOPPED = 0, 1
BGPC_EINVAL, BGPC_ENOMEM, BGPC_ECUDA, BGPC_EROUNDS = -1, -2, -3, -4
BGPC_ETIMEOUT, BGPC_EUNSORTED, BGPC_EINTERNAL = -5, -6, -7
BGPC_FF, BGPC_B1, BGPC_B2, BGPC_B2X = 0, 1, 2, 3
BGPC_DETECT_AUTO, BGPC_DETECT_NETS, BGPC_DETECT_PAIRS = 0, 1, 2
BGPC_GATHER_AUTO, BGPC_GATHER_CTA = 0, 1
BGPC_BATCH_PERSISTENT, BGPC_BATCH_STREAMS = 0, 1
BGPC_BATCH_MAPPINGS = 12
BGPC_MAX_REPORT = 64
NO_BIG = (1 << 31) - 1

_c_i32p = ctypes.POINTER(ctypes.c_int32)


class bgpc_graph_t(ctypes.Structure):
    _fields_ = [("n_a", ctypes.c_int32), ("n_b", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("a_ptr", ctypes.c_void_p), ("a_idx", ctypes.c_void_p),
                ("b_ptr", ctypes.c_void_p), ("b_idx", ctypes.c_void_p)]


class bgpc_ugraph_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("ptr", ctypes.c_void_p), ("idx", ctypes.c_void_p)]


class bgpc_opts_t(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("waves", ctypes.c_int32), ("big_net", ctypes.c_int32),
                ("rank", ctypes.c_void_p), ("max_rounds", ctypes.c_int32),
                ("validate", ctypes.c_int32), ("stop_after_waves", ctypes.c_int64),
                ("W_out", ctypes.c_void_p), ("want_balance", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("stop_before_removal", ctypes.c_int32),
                ("batch_streams", ctypes.c_int32), ("detect", ctypes.c_int32),
                ("gather", ctypes.c_int32), ("net_rounds", ctypes.c_int32),
                ("timeout_us", ctypes.c_int64), ("batch_engine", ctypes.c_int32),
                ("batch_mapping", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class bgpc_stats_t(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("colors", ctypes.c_int32),
                ("w_per_round", ctypes.c_int64 * BGPC_MAX_REPORT),
                ("trav_per_round", ctypes.c_int64 * BGPC_MAX_REPORT),
                ("trav_total", ctypes.c_int64),
                ("stopped_m", ctypes.c_int32), ("stopped_wave", ctypes.c_int32),
                ("n_sets", ctypes.c_int32), ("max_card", ctypes.c_int32),
                ("mean_card", ctypes.c_double), ("std_card", ctypes.c_double),
                ("incid_total", ctypes.c_int64), ("w_total", ctypes.c_int64),
                ("trav_large", ctypes.c_int64), ("incid_large", ctypes.c_int64),
                ("w_large", ctypes.c_int64), ("pieces_total", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("color_launches", ctypes.c_int64),
                ("ms_setup", ctypes.c_double), ("ms_color", ctypes.c_double),
                ("ms_publish", ctypes.c_double), ("ms_detect", ctypes.c_double),
                ("ms_gather", ctypes.c_double), ("trav_hub", ctypes.c_int64),
                ("hub_pairs", ctypes.c_int64), ("hub_words", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("hub_threshold", ctypes.c_int32),
                ("hubs", ctypes.c_int32)]


EXPORTS = ["bgpc_opts_default", "bgpc_ctx_create", "bgpc_ctx_destroy", "bgpc_color",
           "bgpc_color_batched", "d2gc_color", "bgpc_validate", "bgpc_color_sets", "bgpc_color_sets_noalloc",
           "bgpc_features", "bgpc_mlp_sync", "bgpc_mlp_forward", "bgpc_mlp_grad",
           "bgpc_mlp_adam", "bgpc_mlp_train_step", "bgpc_rank_from_scores", "bgpc_strerror",
           "bgpc_rank_smallest_last"]
MLP_IN, MLP_HIDDEN, MLP_PARAMS = 8, 64, 4801


class bgpc_mlp_t(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("w_bf16", ctypes.c_void_p),
                ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("step", ctypes.c_int64)]
BGPC_NOALLOC_MAX_COLORS = 1 << 20

_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libbgpc_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libbgpc_gb300.so is not built: run "
                           "paper_1701_02628_gb300.build.build() (or __graft_entry__.build())")
    lib = ctypes.CDLL(_build.LIB)
    vp = ctypes.c_void_p
    lib.bgpc_opts_default.argtypes = [ctypes.POINTER(bgpc_opts_t)]
    lib.bgpc_opts_default.restype = None
    lib.bgpc_ctx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.bgpc_ctx_destroy.argtypes = [vp]
    lib.bgpc_color.argtypes = [vp, ctypes.POINTER(bgpc_graph_t), ctypes.POINTER(bgpc_opts_t),
                               vp, ctypes.POINTER(bgpc_stats_t), vp]
    lib.d2gc_color.argtypes = [vp, ctypes.POINTER(bgpc_ugraph_t), ctypes.POINTER(bgpc_opts_t),
                               vp, ctypes.POINTER(bgpc_stats_t), vp]
    lib.bgpc_validate.argtypes = [vp, ctypes.POINTER(bgpc_graph_t), vp,
                                  ctypes.POINTER(ctypes.c_int64), vp]
    lib.bgpc_color_sets.argtypes = [vp, vp, ctypes.c_int32, vp, ctypes.c_int32, _c_i32p, _c_i32p,
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.bgpc_color_sets_noalloc.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, _c_i32p, _c_i32p,
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), vp]
    lib.bgpc_color_sets_noalloc.restype = ctypes.c_int
    lib.bgpc_color_batched.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(bgpc_graph_t),
                                       ctypes.POINTER(bgpc_opts_t), ctypes.POINTER(vp),
                                       ctypes.POINTER(bgpc_stats_t), _c_i32p, _c_i32p, vp]
    lib.bgpc_color_batched.restype = ctypes.c_int
    M = ctypes.POINTER(bgpc_mlp_t)
    fp = ctypes.POINTER(ctypes.c_float)
    lib.bgpc_features.argtypes = [vp, ctypes.POINTER(bgpc_graph_t), ctypes.c_int32, vp, vp]
    lib.bgpc_mlp_sync.argtypes = [vp, M, vp]
    lib.bgpc_mlp_forward.argtypes = [vp, M, vp, ctypes.c_int32, vp, vp]
    lib.bgpc_mlp_grad.argtypes = [vp, M, vp, vp, ctypes.c_int32, vp, fp, vp]
    lib.bgpc_mlp_adam.argtypes = [vp, M, vp, ctypes.c_float, vp]
    lib.bgpc_mlp_train_step.argtypes = [vp, M, vp, vp, ctypes.c_int32, ctypes.c_float, fp, vp]
    lib.bgpc_rank_from_scores.argtypes = [vp, vp, ctypes.c_int32, vp, vp]
    lib.bgpc_rank_smallest_last.argtypes = [vp, ctypes.POINTER(bgpc_graph_t), ctypes.c_int64,
                                            vp, _c_i32p, vp]
    lib.bgpc_rank_smallest_last.restype = ctypes.c_int
    for name in ("bgpc_features", "bgpc_mlp_sync", "bgpc_mlp_forward", "bgpc_mlp_grad",
                 "bgpc_mlp_adam", "bgpc_mlp_train_step", "bgpc_rank_from_scores"):
        getattr(lib, name).restype = ctypes.c_int
    lib.bgpc_strerror.argtypes = [ctypes.c_int]
    lib.bgpc_strerror.restype = ctypes.c_char_p
    for name in ("bgpc_ctx_create", "bgpc_ctx_destroy", "bgpc_color", "d2gc_color",
                 "bgpc_validate", "bgpc_color_sets"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class BgpcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {bgpc_strerror(status)} ({status})")


def bgpc_strerror(status: int) -> str:
    return load().bgpc_strerror(status).decode()


def _check(status: int, where: str) -> int:
    if status < 0:
        raise BgpcError(status, where)
    return status


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype=torch.int32):
    if t is None:
        return None
    if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check_n(t):
    """Element counts travel as int32 through the C ABI: refuse larger ones
    instead of letting ctypes wrap them."""
    if t.numel() > (1 << 31) - 1:
        raise ValueError(f"{t.numel()} elements exceed the C ABI's int32 sizes")


def _fptr(t):
    return _ptr(t, torch.float32)


class Context:
    """A library context (device scratch memory) on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.bgpc_ctx_create(ctypes.byref(h), device), "bgpc_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load().bgpc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class DeviceGraph:
    """Bipartite graph with int32 CUDA tensors (see bgpc_graph_t)."""
    n_a: int
    n_b: int
    a_ptr: torch.Tensor
    a_idx: torch.Tensor
    b_ptr: torch.Tensor
    b_idx: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.a_idx.numel())

    @staticmethod
    def from_host(g, device="cuda") -> "DeviceGraph":
        t = lambda a: torch.as_tensor(a, dtype=torch.int32).to(device).contiguous()
        return DeviceGraph(int(g.n_a), int(g.n_b), t(g.a_ptr), t(g.a_idx), t(g.b_ptr), t(g.b_idx))

    def c_struct(self) -> bgpc_graph_t:
        return bgpc_graph_t(self.n_a, self.n_b, self.nnz, _ptr(self.a_ptr), _ptr(self.a_idx),
                            _ptr(self.b_ptr), _ptr(self.b_idx))


@dataclass
class DeviceUGraph:
    """Undirected graph with int32 CUDA tensors (see bgpc_ugraph_t)."""
    n: int
    ptr: torch.Tensor
    idx: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.idx.numel())

    @staticmethod
    def from_host(g, device="cuda") -> "DeviceUGraph":
        t = lambda a: torch.as_tensor(a, dtype=torch.int32).to(device).contiguous()
        return DeviceUGraph(int(g.n), t(g.ptr), t(g.idx))

    def c_struct(self) -> bgpc_ugraph_t:
        return bgpc_ugraph_t(self.n, self.nnz, _ptr(self.ptr), _ptr(self.idx))


def bgpc_opts_default() -> bgpc_opts_t:
    o = bgpc_opts_t()
    load().bgpc_opts_default(ctypes.byref(o))
    return o


def make_opts(policy=BGPC_FF, chunk=64, waves=16, big_net=64, rank=None, max_rounds=1000,
              validate=False, stop_after_waves=0, W_out=None, want_balance=False,
              profile=False, stop_before_removal=False, batch_streams=0,
              detect=BGPC_DETECT_AUTO, gather=BGPC_GATHER_AUTO, net_rounds=0,
              timeout_us=0, batch_engine=0, batch_mapping=0) -> bgpc_opts_t:
    o = bgpc_opts_default()
    o.policy, o.chunk, o.waves, o.big_net = policy, chunk, waves, big_net
    o.rank = _ptr(rank)
    o.max_rounds = max_rounds
    o.validate = int(bool(validate))
    o.stop_after_waves = stop_after_waves
    o.W_out = _ptr(W_out)
    o.want_balance = int(bool(want_balance))
    o.profile = int(bool(profile))
    o.stop_before_removal = int(bool(stop_before_removal))
    o.batch_streams = batch_streams
    o.detect = detect
    o.gather = gather
    o.net_rounds = net_rounds
    o.timeout_us = timeout_us
    o.batch_engine = batch_engine
    o.batch_mapping = batch_mapping
    return o


def stats_dict(st: bgpc_stats_t) -> dict:
    r = min(st.rounds, BGPC_MAX_REPORT)
    return dict(rounds=st.rounds, colors=st.colors,
                w_per_round=list(st.w_per_round[:r]), trav_per_round=list(st.trav_per_round[:r]),
                trav_total=st.trav_total, stopped_m=st.stopped_m, stopped_wave=st.stopped_wave,
                n_sets=st.n_sets, max_card=st.max_card, mean_card=st.mean_card,
                std_card=st.std_card, incid_total=st.incid_total, w_total=st.w_total,
                trav_large=st.trav_large, incid_large=st.incid_large, w_large=st.w_large,
                pieces_total=st.pieces_total,
                kernel_launches=st.kernel_launches,
                color_launches=st.color_launches, ms_setup=st.ms_setup, ms_color=st.ms_color,
                ms_publish=st.ms_publish, ms_detect=st.ms_detect, ms_gather=st.ms_gather,
                trav_hub=st.trav_hub, hub_pairs=st.hub_pairs, hub_words=st.hub_words,
                ms_total=st.ms_total, hub_threshold=st.hub_threshold, hubs=st.hubs)


def bgpc_color(ctx: Context, g: DeviceGraph, colors: torch.Tensor = None, stream=None, **opts):
    """Color V_A (bgpc_color).  Returns (colors, stats dict, status)."""
    if colors is None:
        colors = torch.empty(g.n_a, dtype=torch.int32, device=g.a_ptr.device)
    o = make_opts(**opts)
    gs = g.c_struct()
    st = bgpc_stats_t()
    rc = load().bgpc_color(ctx.handle, ctypes.byref(gs), ctypes.byref(o), _ptr(colors),
                           ctypes.byref(st), _stream(stream))
    _check(rc, "bgpc_color")
    return colors, stats_dict(st), rc


def bgpc_color_batched(ctx: Context, graphs, colors=None, stream=None, **opts):
    """Color a batch of independent graphs with one call (bgpc_color_batched).
    Returns (list of color tensors, batch stats dict, rounds per graph,
    number of colors per graph)."""
    G = len(graphs)
    if colors is None:
        colors = [torch.empty(max(gr.n_a, 1), dtype=torch.int32, device=gr.a_ptr.device)
                  for gr in graphs]
    o = make_opts(**opts)
    gs = (bgpc_graph_t * G)(*[gr.c_struct() for gr in graphs])
    cp = (ctypes.c_void_p * G)(*[c.data_ptr() for c in colors])
    rounds = (ctypes.c_int32 * G)()
    ncol = (ctypes.c_int32 * G)()
    st = bgpc_stats_t()
    _check(load().bgpc_color_batched(ctx.handle, G, gs, ctypes.byref(o), cp, ctypes.byref(st),
                                     rounds, ncol, _stream(stream)), "bgpc_color_batched")
    return ([c[:gr.n_a] for c, gr in zip(colors, graphs)], stats_dict(st), list(rounds),
            list(ncol))


def d2gc_color(ctx: Context, g: DeviceUGraph, colors: torch.Tensor = None, stream=None, **opts):
    """Distance-2 coloring (d2gc_color).  Returns (colors, stats dict, status)."""
    if colors is None:
        colors = torch.empty(g.n, dtype=torch.int32, device=g.ptr.device)
    o = make_opts(**opts)
    gs = g.c_struct()
    st = bgpc_stats_t()
    rc = load().d2gc_color(ctx.handle, ctypes.byref(gs), ctypes.byref(o), _ptr(colors),
                           ctypes.byref(st), _stream(stream))
    _check(rc, "d2gc_color")
    return colors, stats_dict(st), rc


def bgpc_validate(ctx: Context, g: DeviceGraph, colors: torch.Tensor, stream=None) -> int:
    """Number of V_A vertices uncolored or in conflict (bgpc_validate)."""
    n = ctypes.c_int64(0)
    gs = g.c_struct()
    _check(load().bgpc_validate(ctx.handle, ctypes.byref(gs), _ptr(colors), ctypes.byref(n),
                                _stream(stream)), "bgpc_validate")
    return n.value


def bgpc_color_sets(ctx: Context, colors: torch.Tensor, max_colors: int, stream=None):
    """Color-set cardinalities and statistics (bgpc_color_sets)."""
    _check_n(colors)
    card = torch.zeros(max(max_colors, 1), dtype=torch.int64, device=colors.device)
    ns, mx = ctypes.c_int32(0), ctypes.c_int32(0)
    mean, std = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().bgpc_color_sets(ctx.handle, _ptr(colors), colors.numel(),
                                  ctypes.c_void_p(card.data_ptr()), max(max_colors, 1),
                                  ctypes.byref(ns), ctypes.byref(mx), ctypes.byref(mean),
                                  ctypes.byref(std), _stream(stream)), "bgpc_color_sets")
    return card, dict(n_sets=ns.value, max_card=mx.value, mean_card=mean.value,
                      std_card=std.value)


def bgpc_color_sets_noalloc(colors: torch.Tensor, max_colors: int, stream=None) -> dict:
    """Color-set statistics without any device allocation
    (bgpc_color_sets_noalloc): for callers that cannot allocate, e.g. under
    an allocator that owns the whole memory budget or in loops that must not
    enter the driver's allocator.  Runs on the device that holds ``colors``
    (and, unless given, that device's current stream).  Calls that overlap on
    the GPU race (they share one fixed scratch array)."""
    _check_n(colors)
    ns, mx = ctypes.c_int32(0), ctypes.c_int32(0)
    mean, std = ctypes.c_double(0), ctypes.c_double(0)
    with torch.cuda.device(colors.device):
        st = _stream(stream) if stream is not None else \
            ctypes.c_void_p(torch.cuda.current_stream(colors.device).cuda_stream)
        _check(load().bgpc_color_sets_noalloc(_ptr(colors), colors.numel(), max_colors,
                                              ctypes.byref(ns), ctypes.byref(mx),
                                              ctypes.byref(mean), ctypes.byref(std), st),
               "bgpc_color_sets_noalloc")
    return dict(n_sets=ns.value, max_card=mx.value, mean_card=mean.value, std_card=std.value)


# ------------------------------------------------------------ learned order

class MLP:
    """Parameters of the order model (bgpc_mlp_t): float32 master weights w,
    their bfloat16 values (as int16 storage), Adam moments and step count,
    all on one CUDA device.  ``params`` is the packed float32 vector [4801]
    (W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3)."""

    def __init__(self, ctx: "Context", params: torch.Tensor, stream=None):
        if params.numel() != MLP_PARAMS:
            raise ValueError("expected 4801 parameters")
        dev = params.device if params.is_cuda else torch.device("cuda", ctx.device)
        self.w = params.detach().to(dev, torch.float32).contiguous().clone()
        self.w_bf16 = torch.empty(MLP_PARAMS, dtype=torch.int16, device=dev)
        self.adam_m = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
        self.adam_v = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
        self.step = 0
        self.sync(ctx, stream)

    def c_struct(self) -> bgpc_mlp_t:
        return bgpc_mlp_t(self.w.data_ptr(), self.w_bf16.data_ptr(), self.adam_m.data_ptr(),
                          self.adam_v.data_ptr(), self.step)

    def sync(self, ctx: "Context", stream=None):
        """Refresh the bfloat16 copy after writing ``w`` (bgpc_mlp_sync)."""
        m = self.c_struct()
        _check(load().bgpc_mlp_sync(ctx.handle, ctypes.byref(m), _stream(stream)),
               "bgpc_mlp_sync")

    def bf16_values(self) -> torch.Tensor:
        """The weights the forward pass uses, as float32 values."""
        return (self.w_bf16.to(torch.int32) << 16).view(torch.float32)


def features(ctx: Context, g: DeviceGraph, big_net: int = 64, out=None, stream=None):
    """Per-vertex features X [n_a, 8] (bgpc_features)."""
    X = out if out is not None else torch.empty((g.n_a, MLP_IN), dtype=torch.float32,
                                                device=g.a_ptr.device)
    gs = g.c_struct()
    _check(load().bgpc_features(ctx.handle, ctypes.byref(gs), big_net,
                                _fptr(X) if g.n_a else None, _stream(stream)), "bgpc_features")
    return X


def mlp_forward(ctx: Context, mlp: MLP, X: torch.Tensor, out=None, stream=None):
    """Scores [n] of the rows of X (bgpc_mlp_forward)."""
    n = X.shape[0]
    s = out if out is not None else torch.empty(n, dtype=torch.float32, device=X.device)
    m = mlp.c_struct()
    _check(load().bgpc_mlp_forward(ctx.handle, ctypes.byref(m), _fptr(X) if n else None, n,
                                   _fptr(s) if n else None, _stream(stream)), "bgpc_mlp_forward")
    return s


def mlp_grad(ctx: Context, mlp: MLP, X: torch.Tensor, y: torch.Tensor, stream=None):
    """(gradient [4801], loss) of the mean squared error (bgpc_mlp_grad)."""
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
    loss = ctypes.c_float(0)
    m = mlp.c_struct()
    _check(load().bgpc_mlp_grad(ctx.handle, ctypes.byref(m), _fptr(X), _fptr(y), X.shape[0],
                                _fptr(g), ctypes.byref(loss), _stream(stream)), "bgpc_mlp_grad")
    return g, loss.value


def mlp_adam(ctx: Context, mlp: MLP, grad: torch.Tensor, lr: float, stream=None):
    """One Adam step with the given gradient (bgpc_mlp_adam)."""
    m = mlp.c_struct()
    _check(load().bgpc_mlp_adam(ctx.handle, ctypes.byref(m), _fptr(grad), lr, _stream(stream)),
           "bgpc_mlp_adam")
    mlp.step = m.step


def mlp_train_step(ctx: Context, mlp: MLP, X: torch.Tensor, y: torch.Tensor, lr: float,
                   stream=None) -> float:
    """Gradient and Adam step (bgpc_mlp_train_step); returns the loss before the step."""
    loss = ctypes.c_float(0)
    m = mlp.c_struct()
    _check(load().bgpc_mlp_train_step(ctx.handle, ctypes.byref(m), _fptr(X), _fptr(y),
                                      X.shape[0], lr, ctypes.byref(loss), _stream(stream)),
           "bgpc_mlp_train_step")
    mlp.step = m.step
    return loss.value


def rank_from_scores(ctx: Context, score: torch.Tensor, out=None, stream=None):
    """rank [n] int32: position in the order of decreasing score, ties by index
    (bgpc_rank_from_scores)."""
    n = score.numel()
    r = out if out is not None else torch.empty(n, dtype=torch.int32, device=score.device)
    _check(load().bgpc_rank_from_scores(ctx.handle, _fptr(score) if n else None, n,
                                        _ptr(r) if n else None, _stream(stream)),
           "bgpc_rank_from_scores")
    return r


def sl_rank(ctx: Context, g: DeviceGraph, max_pairs: int = 1 << 31, stream=None):
    """Smallest-last rank (bgpc_rank_smallest_last): (rank tensor, degeneracy)."""
    rank = torch.empty(max(g.n_a, 1), dtype=torch.int32, device=g.a_ptr.device)
    dg = ctypes.c_int32(0)
    gs = g.c_struct()
    _check(load().bgpc_rank_smallest_last(ctx.handle, ctypes.byref(gs), max_pairs,
                                          _ptr(rank), ctypes.byref(dg), _stream(stream)),
           "bgpc_rank_smallest_last")
    return rank[:g.n_a], dg.value


def learned_rank(ctx: Context, g: DeviceGraph, mlp: MLP, big_net: int = 64, stream=None):
    """features -> MLP score -> rank, ready for bgpc_color(..., rank=...)."""
    X = features(ctx, g, big_net, stream=stream)
    return rank_from_scores(ctx, mlp_forward(ctx, mlp, X, stream=stream), stream=stream)


def order_target(ctx: Context, g: DeviceGraph, stream=None, **opts) -> torch.Tensor:
    """Training target of the order model for graph g: the color every vertex
    gets from a plain first-fit coloring in id order, divided by the number
    of colors (vertices that end up in high colors are the hard ones, and the
    learned order colors them first)."""
    c, st, _ = bgpc_color(ctx, g, stream=stream, **opts)
    return c.to(torch.float32) / float(max(st["colors"], 1))


def train_order(ctx: Context, graphs, params: torch.Tensor, steps: int = 200,
                lr: float = 3e-3, big_net: int = 64, stream=None):
    """Fit the order model on the given graphs: features and targets of every
    graph, concatenated, then ``steps`` full-batch Adam steps (every step is
    bgpc_mlp_train_step).  Returns (MLP, list of losses)."""
    Xs, ys = [], []
    for g in graphs:
        Xs.append(features(ctx, g, big_net, stream=stream))
        ys.append(order_target(ctx, g, stream=stream))
    X = torch.cat(Xs).contiguous()
    y = torch.cat(ys).contiguous()
    mlp = MLP(ctx, params, stream)
    losses = [mlp_train_step(ctx, mlp, X, y, lr, stream) for _ in range(steps)]
    return mlp, losses
