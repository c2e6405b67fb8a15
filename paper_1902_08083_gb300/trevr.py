"""Python binding of libtrevr (include/trevr.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module passes
device pointers of torch tensors and the current CUDA stream through ctypes.
There is no CPU fallback: if libtrevr.so is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtrevr.so")

TREVR_OK = 0
ERRORS = {
    1: "TREVR_ERR_INVALID_ARGUMENT",
    2: "TREVR_ERR_OUT_OF_DOMAIN",
    3: "TREVR_ERR_STACK_OVERFLOW",
    4: "TREVR_ERR_ITERATION_LIMIT",
    5: "TREVR_ERR_CUDA",
    6: "TREVR_ERR_OUT_OF_MEMORY",
}

# names of every entry point declared in include/trevr.h
EXPORTS = (
    "trevr_build_tree", "trevr_compute_flux", "trevr_compute_flux_backward",
    "trevr_compute_flux_moments", "trevr_check",
    "trevr_tree_info",
    "trevr_tree_export", "trevr_tree_free", "trevr_status_string", "trevr_kernel_launches",
    "trevr_morton_sort_noalloc", "trevr_batch_create", "trevr_compute_flux_batched",
    "trevr_batch_check", "trevr_batch_free", "trevr_build_tree_bands", "trevr_compute_flux_bands",
    "trevr_tree_set_smoothing",
)
NOALLOC_MAX_N = 1 << 20


class TrevrError(RuntimeError):
    def __init__(self, code, where=""):
        name = ERRORS.get(code, f"code {code}")
        super().__init__(f"{where}: {name}" if where else name)
        self.code = code


class Domain(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("side", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("theta_open", ctypes.c_float), ("tau_ref", ctypes.c_float),
                ("bucket", ctypes.c_int), ("sinks_per_warp", ctypes.c_int),
                ("block_size", ctypes.c_int), ("stack_depth", ctypes.c_int),
                ("walk_variant", ctypes.c_int), ("bg_radius", ctypes.c_float),
                ("tau_stop", ctypes.c_float), ("sub_bucket", ctypes.c_int),
                ("ray_walk", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("interactions", ctypes.c_longlong), ("segments", ctypes.c_longlong),
                ("src_nodes_visited", ctypes.c_longlong),
                ("refine_expansions", ctypes.c_longlong), ("cells_clipped", ctypes.c_longlong),
                ("build_ms", ctypes.c_float),
                ("walk_ms", ctypes.c_float), ("rays_terminated", ctypes.c_longlong),
                ("sub_bucket_segments", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtrevr.so and declare its signatures (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is not built; run paper_1902_08083_gb300._build.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        ll = ctypes.c_longlong
        lib.trevr_build_tree.argtypes = [P, P, P, ll, P, P, ll, ctypes.POINTER(Domain),
                                         ctypes.POINTER(Params), P, ctypes.POINTER(P)]
        lib.trevr_build_tree.restype = ctypes.c_int
        lib.trevr_compute_flux.argtypes = [P, P, ll, ctypes.POINTER(Params), P, P,
                                           ctypes.POINTER(Stats), P]
        lib.trevr_compute_flux.restype = ctypes.c_int
        lib.trevr_build_tree_bands.argtypes = [P, P, P, ll, P, P, ll, ctypes.c_int,
                                               ctypes.POINTER(Domain), ctypes.POINTER(Params), P,
                                               ctypes.POINTER(P)]
        lib.trevr_build_tree_bands.restype = ctypes.c_int
        lib.trevr_compute_flux_bands.argtypes = [P, P, ll, ctypes.POINTER(Params), P, P,
                                                 ctypes.POINTER(Stats), P]
        lib.trevr_compute_flux_bands.restype = ctypes.c_int
        lib.trevr_tree_set_smoothing.argtypes = [P, P, P]
        lib.trevr_tree_set_smoothing.restype = ctypes.c_int
        lib.trevr_compute_flux_backward.argtypes = [P, P, ll, ctypes.POINTER(Params), P, P, P,
                                                    P]
        lib.trevr_compute_flux_backward.restype = ctypes.c_int
        lib.trevr_batch_create.argtypes = [P, ctypes.c_int, ctypes.POINTER(P)]
        lib.trevr_batch_create.restype = ctypes.c_int
        lib.trevr_compute_flux_batched.argtypes = [P, ctypes.POINTER(Params), P,
                                                   ctypes.POINTER(Stats), P]
        lib.trevr_compute_flux_batched.restype = ctypes.c_int
        lib.trevr_batch_check.argtypes = [P, P]
        lib.trevr_batch_check.restype = ctypes.c_int
        lib.trevr_batch_free.argtypes = [P]
        lib.trevr_batch_free.restype = None
        lib.trevr_compute_flux_moments.argtypes = [P, P, ll, ctypes.POINTER(Params), P, P, P, P]
        lib.trevr_compute_flux_moments.restype = ctypes.c_int
        lib.trevr_check.argtypes = [P, P]
        lib.trevr_check.restype = ctypes.c_int
        lib.trevr_tree_info.argtypes = [P, ctypes.POINTER(ll), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ll), ctypes.POINTER(ll)]
        lib.trevr_tree_info.restype = ctypes.c_int
        lib.trevr_tree_export.argtypes = [P] * 20
        lib.trevr_tree_export.restype = ctypes.c_int
        lib.trevr_tree_free.argtypes = [P]
        lib.trevr_tree_free.restype = None
        lib.trevr_morton_sort_noalloc.argtypes = [P, ll, ctypes.POINTER(Domain), P, P, P]
        lib.trevr_morton_sort_noalloc.restype = ctypes.c_int
        lib.trevr_kernel_launches.argtypes = []
        lib.trevr_kernel_launches.restype = ctypes.c_ulonglong
        lib.trevr_status_string.argtypes = [ctypes.c_int]
        lib.trevr_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _dev_ptr(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(theta=0.75, tau_ref=0.1, bucket=8, sinks_per_warp=0, block_size=0,
                stack_depth=0, walk_variant=0, bg_radius=0.0, tau_stop=0.0, sub_bucket=0,
                ray_walk=0):
    """trevr_params; ray_walk = 1 selects the top-down ray walk (0: the paper's)."""
    return Params(float(theta), float(tau_ref), int(bucket), int(sinks_per_warp),
                  int(block_size), int(stack_depth), int(walk_variant), float(bg_radius),
                  float(tau_stop), int(sub_bucket), int(ray_walk))


class Tree:
    """A radiation tree built on the GPU (trevr_build_tree); owns the C handle.

    alpha (N,) and src_lum (S,); or, for several bands (trevr_build_tree_bands),
    alpha (B, N) and src_lum (B, S)."""

    def __init__(self, gas_xyz, alpha, src_xyz, src_lum, weight=None, lo=(0.0, 0.0, 0.0),
                 side=1.0, bucket=8, stream=None):
        lib = load_library()
        self._lib = lib
        self._h = None
        gas_xyz = gas_xyz.contiguous()
        src_xyz = src_xyz.contiguous()
        if gas_xyz.dim() != 2 or gas_xyz.shape[0] != 3:
            raise ValueError("gas_xyz must have shape (3, N)")
        if src_xyz.dim() != 2 or src_xyz.shape[0] != 3:
            raise ValueError("src_xyz must have shape (3, S)")
        self.n_gas = int(gas_xyz.shape[1])
        self.n_src = int(src_xyz.shape[1])
        self.device = gas_xyz.device
        dom = Domain((ctypes.c_float * 3)(*[float(v) for v in lo]), float(side))
        prm = make_params(bucket=bucket)
        h = ctypes.c_void_p()
        self.n_bands = 0
        if alpha.dim() == 2:
            self.n_bands = int(alpha.shape[0])
            if alpha.shape[1] != self.n_gas or (self.n_src and
                                                tuple(src_lum.shape) != (self.n_bands, self.n_src)):
                raise ValueError("alpha (B, N) and src_lum (B, S) must have the same B")
            alpha_c = alpha.contiguous()  # kept alive until the call has returned
            lum_c = src_lum.contiguous() if self.n_src else None
            rc = lib.trevr_build_tree_bands(
                _dev_ptr(gas_xyz, torch.float32, "gas_xyz"),
                _dev_ptr(alpha_c, torch.float32, "alpha"),
                _dev_ptr(weight, torch.float32, "weight"), self.n_gas,
                _dev_ptr(src_xyz, torch.float32, "src_xyz") if self.n_src else None,
                _dev_ptr(lum_c, torch.float32, "src_lum") if self.n_src else None,
                self.n_src, self.n_bands, ctypes.byref(dom), ctypes.byref(prm),
                _stream_ptr(stream), ctypes.byref(h))
            where = "trevr_build_tree_bands"
        else:
            rc = lib.trevr_build_tree(
                _dev_ptr(gas_xyz, torch.float32, "gas_xyz"),
                _dev_ptr(alpha, torch.float32, "alpha"),
                _dev_ptr(weight, torch.float32, "weight"), self.n_gas,
                _dev_ptr(src_xyz, torch.float32, "src_xyz") if self.n_src else None,
                _dev_ptr(src_lum, torch.float32, "src_lum") if self.n_src else None, self.n_src,
                ctypes.byref(dom), ctypes.byref(prm), _stream_ptr(stream), ctypes.byref(h))
            where = "trevr_build_tree"
        if rc != TREVR_OK:
            raise TrevrError(rc, where)
        self._h = h
        self.bucket = bucket
        self.side = float(side)
        nn = ctypes.c_longlong()
        md = ctypes.c_int()
        lib.trevr_tree_info(h, ctypes.byref(nn), ctypes.byref(md), None, None)
        self.n_nodes = nn.value
        self.max_depth = md.value

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            self._lib.trevr_tree_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_smoothing(self, hsml, stream=None):
        """Smoothing lengths (N,) fp32 on the device, caller order, for the sub-bucket
        particle trace (trevr_tree_set_smoothing); then pass sub_bucket=1."""
        hsml = hsml.contiguous()
        if hsml.numel() != self.n_gas:
            raise ValueError(f"hsml has {hsml.numel()} elements, expected {self.n_gas}")
        rc = self._lib.trevr_tree_set_smoothing(self._h, _dev_ptr(hsml, torch.float32, "hsml"),
                                                _stream_ptr(stream))
        if rc != TREVR_OK:
            raise TrevrError(rc, "trevr_tree_set_smoothing")

    def export(self, stream=None):
        """Copy the tree into torch tensors on the tree's device (see trevr_tree_export)."""
        dev = self.device
        n, nc, ns = self.n_gas, self.n_nodes + 1, self.n_src
        i32 = dict(dtype=torch.int32, device=dev)
        f32 = dict(dtype=torch.float32, device=dev)
        out = dict(key=torch.empty(n, dtype=torch.int64, device=dev),
                   perm=torch.empty(n, **i32), leaf_of=torch.empty(n, **i32),
                   first=torch.empty(nc, **i32), count=torch.empty(nc, **i32),
                   child=torch.empty(nc, **i32), parent=torch.empty(nc, **i32),
                   depth=torch.empty(nc, **i32), glo=torch.empty(nc, 3, **i32),
                   ghi=torch.empty(nc, 3, **i32), abar=torch.empty(nc, **f32),
                   dalpha=torch.empty(nc, **f32), lum=torch.empty(nc, **f32),
                   cen=torch.empty(nc, 3, **f32), l2=torch.empty(nc, **f32),
                   src_first=torch.empty(nc, **i32), src_count=torch.empty(nc, **i32),
                   src_order=torch.empty(max(ns, 1), **i32))
        order = ("key", "perm", "leaf_of", "first", "count", "child", "parent", "depth", "glo",
                 "ghi", "abar", "dalpha", "lum", "cen", "l2", "src_first", "src_count",
                 "src_order")
        rc = self._lib.trevr_tree_export(self._h, *(ctypes.c_void_p(out[k].data_ptr())
                                                     for k in order), _stream_ptr(stream))
        if rc != TREVR_OK:
            raise TrevrError(rc, "trevr_tree_export")
        out["src_order"] = out["src_order"][:ns]
        return out


def build_tree(gas_xyz, alpha, src_xyz, src_lum, weight=None, lo=(0.0, 0.0, 0.0), side=1.0,
               bucket=8, stream=None) -> Tree:
    return Tree(gas_xyz, alpha, src_xyz, src_lum, weight, lo, side, bucket, stream)


def compute_flux(tree: Tree, theta=0.75, tau_ref=0.1, sink_idx=None, out=None, counters=False,
                 stats=False, stream=None, **tuning):
    """Flux at the sinks (trevr_compute_flux). Returns flux, plus the per-sink counters
    (n, 4) int32 and/or a stats dict when asked. `tuning` holds the other fields of
    trevr_params (launch shape, walk_variant, bg_radius, tau_stop, sub_bucket,
    ray_walk)."""
    lib = tree._lib
    n = tree.n_gas if sink_idx is None else int(sink_idx.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=tree.device)
    elif out.numel() != n:
        raise ValueError(f"out has {out.numel()} elements, expected {n}")
    cnt = torch.empty(n, 4, dtype=torch.int32, device=tree.device) if counters else None
    st = Stats() if stats else None
    prm = make_params(theta, tau_ref, tree.bucket, **tuning)
    rc = lib.trevr_compute_flux(tree.handle, _dev_ptr(sink_idx, torch.int64, "sink_idx"), n,
                                ctypes.byref(prm), _dev_ptr(out, torch.float32, "out"),
                                _dev_ptr(cnt, torch.int32, "counters"),
                                ctypes.byref(st) if st is not None else None, _stream_ptr(stream))
    if rc != TREVR_OK:
        raise TrevrError(rc, "trevr_compute_flux")
    res = [out]
    if counters:
        res.append(cnt)
    if stats:
        res.append(st.as_dict())
    return res[0] if len(res) == 1 else tuple(res)


def compute_flux_bands(tree: Tree, theta=0.75, tau_ref=0.1, sink_idx=None, out=None,
                       counters=False, stats=False, stream=None, **tuning):
    """Flux of every band (trevr_compute_flux_bands) for a tree built with alpha (B, N):
    returns (B, n) fp32, plus counters / stats as compute_flux."""
    lib = tree._lib
    n = tree.n_gas if sink_idx is None else int(sink_idx.shape[0])
    nb = max(tree.n_bands, 1)
    if out is None:
        out = torch.empty(nb, n, dtype=torch.float32, device=tree.device)
    elif tuple(out.shape) != (nb, n):
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {(nb, n)}")
    cnt = torch.empty(n, 4, dtype=torch.int32, device=tree.device) if counters else None
    st = Stats() if stats else None
    prm = make_params(theta, tau_ref, tree.bucket, **tuning)
    rc = lib.trevr_compute_flux_bands(tree.handle, _dev_ptr(sink_idx, torch.int64, "sink_idx"),
                                      n, ctypes.byref(prm), _dev_ptr(out, torch.float32, "out"),
                                      _dev_ptr(cnt, torch.int32, "counters"),
                                      ctypes.byref(st) if st is not None else None,
                                      _stream_ptr(stream))
    if rc != TREVR_OK:
        raise TrevrError(rc, "trevr_compute_flux_bands")
    res = [out]
    if counters:
        res.append(cnt)
    if stats:
        res.append(st.as_dict())
    return res[0] if len(res) == 1 else tuple(res)


def morton_sort_noalloc(gas_xyz, lo=(0.0, 0.0, 0.0), side=1.0, keys_out=None, perm_out=None,
                        stream=None):
    """Morton keys and stable sort of the particles (trevr_morton_sort_noalloc): the
    library allocates nothing; the output tensors are allocated here unless given.

    gas_xyz is (3, N) fp32; keys_out (int64) and perm_out (int32) must hold at least
    N elements. Every tensor must sit on one CUDA device, which is made current for
    the call (the C side looks up its scratch array on the current device and
    launches there); `stream`, if given, must belong to that device."""
    # shapes, sizes and devices first (no GPU needed to reject them), then CUDA
    if not isinstance(gas_xyz, torch.Tensor):
        raise TypeError("gas_xyz must be a CUDA tensor")
    if gas_xyz.dim() != 2 or gas_xyz.shape[0] != 3:
        raise ValueError(f"gas_xyz must have shape (3, N), got {tuple(gas_xyz.shape)}")
    dev = gas_xyz.device
    n = int(gas_xyz.shape[1])
    for name, t in (("keys_out", keys_out), ("perm_out", perm_out)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or t.device != dev:
            raise ValueError(f"{name} must be a tensor on {dev}")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} elements, fewer than the {n} particles")
    if stream is not None and stream.device != dev:
        raise ValueError(f"stream belongs to {stream.device}, the tensors to {dev}")
    if not gas_xyz.is_cuda:
        raise TypeError("gas_xyz must be a CUDA tensor")
    lib = load_library()
    with torch.cuda.device(dev):
        if keys_out is None:
            keys_out = torch.empty(n, dtype=torch.int64, device=dev)
        if perm_out is None:
            perm_out = torch.empty(n, dtype=torch.int32, device=dev)
        xyz = gas_xyz.contiguous()  # kept alive until the call has returned
        dom = Domain((ctypes.c_float * 3)(*[float(v) for v in lo]), float(side))
        rc = lib.trevr_morton_sort_noalloc(_dev_ptr(xyz, torch.float32, "gas_xyz"),
                                           n, ctypes.byref(dom),
                                           _dev_ptr(keys_out, torch.int64, "keys_out"),
                                           _dev_ptr(perm_out, torch.int32, "perm_out"),
                                           _stream_ptr(stream))
        del xyz
    if rc != TREVR_OK:
        raise TrevrError(rc, "trevr_morton_sort_noalloc")
    return keys_out, perm_out


def compute_flux_moments(tree: Tree, theta=0.75, tau_ref=0.1, sink_idx=None, pressure=True,
                         stream=None, **tuning):
    """(flux[n], flux vector[3, n], pressure[6, n] or None) at the sinks
    (trevr_compute_flux_moments): sum f, sum f n, sum f n n^T (xx yy zz xy xz yz)."""
    lib = tree._lib
    n = tree.n_gas if sink_idx is None else int(sink_idx.shape[0])
    dev = tree.device
    flux = torch.empty(n, dtype=torch.float32, device=dev)
    fvec = torch.empty(3, n, dtype=torch.float32, device=dev)
    press = torch.empty(6, n, dtype=torch.float32, device=dev) if pressure else None
    prm = make_params(theta, tau_ref, tree.bucket, **tuning)
    rc = lib.trevr_compute_flux_moments(tree.handle, _dev_ptr(sink_idx, torch.int64, "sink_idx"),
                                        n, ctypes.byref(prm), _dev_ptr(flux, torch.float32, "f"),
                                        _dev_ptr(fvec, torch.float32, "fvec"),
                                        _dev_ptr(press, torch.float32, "press"),
                                        _stream_ptr(stream))
    if rc != TREVR_OK:
        raise TrevrError(rc, "trevr_compute_flux_moments")
    return flux, fvec, press


def compute_flux_backward(tree: Tree, grad_flux, theta=0.75, tau_ref=0.1, sink_idx=None,
                          stream=None, **tuning):
    """Adjoint of compute_flux with the forward decisions frozen (trevr_compute_flux_backward).
    Returns (grad_lum[n_src], grad_alpha[n_gas]) in the caller's order."""
    lib = tree._lib
    n = tree.n_gas if sink_idx is None else int(sink_idx.shape[0])
    grad_flux = grad_flux.contiguous().to(torch.float32)
    if grad_flux.numel() != n:
        raise ValueError(f"grad_flux has {grad_flux.numel()} elements, expected {n}")
    gl = torch.empty(tree.n_src, dtype=torch.float32, device=tree.device)
    ga = torch.empty(tree.n_gas, dtype=torch.float32, device=tree.device)
    prm = make_params(theta, tau_ref, tree.bucket, **tuning)
    rc = lib.trevr_compute_flux_backward(
        tree.handle, _dev_ptr(sink_idx, torch.int64, "sink_idx"), n, ctypes.byref(prm),
        _dev_ptr(grad_flux, torch.float32, "grad_flux"),
        _dev_ptr(gl, torch.float32, "grad_lum") if tree.n_src else None,
        _dev_ptr(ga, torch.float32, "grad_alpha"), _stream_ptr(stream))
    if rc != TREVR_OK:
        raise TrevrError(rc, "trevr_compute_flux_backward")
    return gl, ga


class TrevrFlux(torch.autograd.Function):
    """Flux at every gas particle as a differentiable function of the absorption
    coefficients alpha and the source luminosities (positions are not differentiated).
    The backward pass is the library's adjoint with the forward decisions frozen."""

    @staticmethod
    def forward(ctx, gas_xyz, alpha, src_xyz, src_lum, theta, tau_ref, bucket, lo, side, weight):
        tree = build_tree(gas_xyz.detach(), alpha.detach().contiguous(), src_xyz.detach(),
                          src_lum.detach().contiguous(),
                          None if weight is None else weight.detach(), lo, side, bucket)
        flux = compute_flux(tree, theta, tau_ref)
        ctx.tree = tree
        ctx.theta, ctx.tau_ref = theta, tau_ref
        return flux

    @staticmethod
    def backward(ctx, grad_flux):
        gl, ga = compute_flux_backward(ctx.tree, grad_flux, ctx.theta, ctx.tau_ref)
        ctx.tree.free()
        return None, ga, None, gl, None, None, None, None, None, None


def trevr_flux(gas_xyz, alpha, src_xyz, src_lum, theta=0.75, tau_ref=0.1, bucket=8,
               lo=(0.0, 0.0, 0.0), side=1.0, weight=None):
    """Differentiable flux (see TrevrFlux)."""
    return TrevrFlux.apply(gas_xyz, alpha, src_xyz, src_lum, theta, tau_ref, bucket, lo, side,
                           weight)


class Batch:
    """Independent trees processed by one persistent launch (trevr_batch_create).

    Owns one fp32 flux tensor per tree (caller order) and the device array of their
    pointers, so a call only enqueues device work and can be captured in a CUDA graph."""

    def __init__(self, trees):
        lib = load_library()
        self._lib = lib
        self._h = None
        self.trees = list(trees)
        arr = (ctypes.c_void_p * len(self.trees))(*[t.handle.value for t in self.trees])
        h = ctypes.c_void_p()
        rc = lib.trevr_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.trees),
                                    ctypes.byref(h))
        if rc != TREVR_OK:
            raise TrevrError(rc, "trevr_batch_create")
        self._h = h
        dev = self.trees[0].device
        self.flux = [torch.empty(t.n_gas, dtype=torch.float32, device=dev) for t in self.trees]
        self._ptrs = torch.tensor([f.data_ptr() for f in self.flux], dtype=torch.int64,
                                  device=dev)
        self.n_sinks = sum(t.n_gas for t in self.trees)
        self.graph = None

    def run(self, theta=0.75, tau_ref=0.1, stats=False, stream=None, **tuning):
        """Enqueue the batched flux (results in self.flux); stats=True synchronises."""
        prm = make_params(theta, tau_ref, self.trees[0].bucket, **tuning)
        st = Stats() if stats else None
        rc = self._lib.trevr_compute_flux_batched(self._h, ctypes.byref(prm),
                                                  ctypes.c_void_p(self._ptrs.data_ptr()),
                                                  ctypes.byref(st) if st is not None else None,
                                                  _stream_ptr(stream))
        if rc != TREVR_OK:
            raise TrevrError(rc, "trevr_compute_flux_batched")
        return st.as_dict() if stats else None

    def capture(self, theta=0.75, tau_ref=0.1, **tuning):
        """Capture one batched call in a CUDA graph (after a first call with the same
        tuning has built the work items); replay with self.replay()."""
        self.run(theta, tau_ref, **tuning)  # builds the work items outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(theta, tau_ref, stream=s, **tuning)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def check(self, stream=None):
        rc = self._lib.trevr_batch_check(self._h, _stream_ptr(stream))
        if rc != TREVR_OK:
            raise TrevrError(rc, "trevr_batch_check")

    def free(self):
        if self._h is not None and self._h.value:
            self._lib.trevr_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels launched by libtrevr so far in this process."""
    return int(load_library().trevr_kernel_launches())


def check(tree: Tree, stream=None):
    rc = tree._lib.trevr_check(tree.handle, _stream_ptr(stream))
    if rc != TREVR_OK:
        raise TrevrError(rc, "trevr_check")
