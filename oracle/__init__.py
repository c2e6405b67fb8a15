"""FP64 CPU oracle for the TREVR hot path (Grond et al. 2019, arXiv:1902.08083).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline
leg of the benchmark use it. The CUDA library never imports or calls it.

The arithmetic lives in ``trevr_oracle.c`` (plain C, OpenMP over sinks); this
module compiles it with gcc and marshals numpy arrays through ctypes.

Every oracle function has a pin in ``tests/test_oracle_*.py`` (brute force,
closed form, hand-worked example or invariant); see the header of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trevr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtrevr_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ERR_INVALID_ARGUMENT = 1
ORC_ERR_OUT_OF_DOMAIN = 2
ORC_ERR_NO_MEMORY = 6


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        f32 = ctypes.c_float
        lib.orc_build.argtypes = [P, P, P, P, P, i64, P, P, P, P, i64, P, f32, ctypes.c_int,
                                  ctypes.POINTER(P)]
        lib.orc_build.restype = ctypes.c_int
        lib.orc_tree_free.argtypes = [P]
        lib.orc_tree_free.restype = None
        lib.orc_n_nodes.argtypes = [P]
        lib.orc_n_nodes.restype = i64
        lib.orc_morton_keys.argtypes = [P, P, P, i64, P, f32, P]
        lib.orc_morton_keys.restype = ctypes.c_int
        lib.orc_export_nodes.argtypes = [P] * 19
        lib.orc_export_nodes.restype = None
        lib.orc_export_nodes32.argtypes = [P] * 8
        lib.orc_export_nodes32.restype = None
        lib.orc_export_directional.argtypes = [P] * 3
        lib.orc_export_directional.restype = None
        lib.orc_export_particles.argtypes = [P] * 4
        lib.orc_export_particles.restype = None
        lib.orc_export_sources.argtypes = [P] * 3
        lib.orc_export_sources.restype = None
        lib.orc_flux.argtypes = [P, P, i64, f32, f32, P, P, P, ctypes.c_int]
        lib.orc_flux.restype = ctypes.c_int
        lib.orc_flux_moments.argtypes = [P, P, i64, f32, f32, P, P, P, ctypes.c_int]
        lib.orc_flux_moments.restype = ctypes.c_int
        lib.orc_flux_background.argtypes = [P, P, i64, f32, f32, f32, P, P, ctypes.c_int]
        lib.orc_flux_background.restype = ctypes.c_int
        lib.orc_flux_terminated.argtypes = [P, P, i64, f32, f32, f32, f32, P, P, ctypes.c_int]
        lib.orc_flux_terminated.restype = ctypes.c_int
        lib.orc_build_bands.argtypes = [P, P, P, P, P, i64, P, P, P, P, i64, ctypes.c_int, P,
                                        f32, ctypes.c_int, ctypes.POINTER(P)]
        lib.orc_build_bands.restype = ctypes.c_int
        lib.orc_flux_bands.argtypes = [P, P, i64, f32, f32, P, P, ctypes.c_int]
        lib.orc_flux_bands.restype = ctypes.c_int
        lib.orc_set_smoothing.argtypes = [P, P]
        lib.orc_set_smoothing.restype = ctypes.c_int
        lib.orc_flux_sub.argtypes = [P, P, i64, f32, f32, P, P, ctypes.c_int]
        lib.orc_flux_sub.restype = ctypes.c_int
        lib.orc_sink_interactions.argtypes = [P, i64, f32, f32, f32, i64] + [P] * 8
        lib.orc_sink_interactions.restype = i64
        lib.orc_ray_tau.argtypes = [P, i64, i64, P, f32, P, P]
        lib.orc_ray_tau.restype = ctypes.c_double
        lib.orc_ray_tau_walk.argtypes = [P, i64, i64, P, f32, ctypes.c_int, P, P]
        lib.orc_ray_tau_walk.restype = ctypes.c_double
        lib.orc_flux_topdown.argtypes = [P, P, i64, f32, f32, P, P, ctypes.c_int]
        lib.orc_flux_topdown.restype = ctypes.c_int
        lib.orc_adjoint.argtypes = [P, P, i64, P, f32, f32, P, P, ctypes.c_int]
        lib.orc_adjoint.restype = ctypes.c_int
        lib.orc_replay_record.argtypes = [P, P, i64, f32, f32, ctypes.POINTER(P)]
        lib.orc_replay_record.restype = ctypes.c_int
        lib.orc_replay_free.argtypes = [P]
        lib.orc_replay_free.restype = None
        lib.orc_replay_loss.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_double]
        lib.orc_replay_loss.restype = ctypes.c_double
        lib.orc_replay_loss_planes.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_double,
                                               ctypes.c_int]
        lib.orc_replay_loss_planes.restype = ctypes.c_double
        lib.orc_replay_kinks.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_double]
        lib.orc_replay_kinks.restype = i64
        lib.orc_leaf_of_point.argtypes = [P, f32, f32, f32]
        lib.orc_leaf_of_point.restype = i64
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


def morton_keys(xyz, lo, side):
    """63-bit Morton keys of the points xyz (3, N) in the cubic domain (Sec. 2.3)."""
    lib = _load()
    xyz = _f32(xyz)
    n = xyz.shape[1]
    x, y, z = (np.ascontiguousarray(xyz[d]) for d in range(3))
    keys = np.zeros(n, dtype=np.uint64)
    lo32 = _f32(lo)
    rc = lib.orc_morton_keys(_ptr(x), _ptr(y), _ptr(z), n, _ptr(lo32), float(side), _ptr(keys))
    if rc != ORC_OK:
        raise OracleError(rc)
    return keys


class OracleTree:
    """The oracle's radiation tree over gas particles, with sources deposited in its leaves."""

    def __init__(self, gas_xyz, alpha, src_xyz, src_lum, lo=(0.0, 0.0, 0.0), side=1.0,
                 bucket=8, weight=None):
        """alpha (N,) and src_lum (S,); or, for several bands, alpha (B, N) and
        src_lum (B, S) (orc_build_bands: the walk uses the band-summed luminosity and
        refines where any band asks)."""
        lib = _load()
        self._lib = lib
        gas_xyz = _f32(gas_xyz)
        src_xyz = _f32(src_xyz).reshape(3, -1)
        self.n_gas = gas_xyz.shape[1]
        self.n_src = src_xyz.shape[1]
        gx, gy, gz = (np.ascontiguousarray(gas_xyz[d]) for d in range(3))
        sx, sy, sz = (np.ascontiguousarray(src_xyz[d]) for d in range(3))
        self._keep = (gx, gy, gz, sx, sy, sz)
        a = _f32(alpha)
        w = None if weight is None else _f32(weight)
        lum = _f32(src_lum)
        lo32 = _f32(lo)
        h = ctypes.c_void_p()
        self.n_bands = 0
        if a.ndim == 2:
            self.n_bands = a.shape[0]
            if lum.shape != (self.n_bands, self.n_src) or a.shape[1] != self.n_gas:
                raise ValueError("alpha (B, N) and src_lum (B, S) must have the same B")
            self._keep = self._keep + (a, lum)
            rc = lib.orc_build_bands(_ptr(gx), _ptr(gy), _ptr(gz), _ptr(a), _ptr(w), self.n_gas,
                                     _ptr(sx), _ptr(sy), _ptr(sz), _ptr(lum), self.n_src,
                                     self.n_bands, _ptr(lo32), float(side), int(bucket),
                                     ctypes.byref(h))
        else:
            rc = lib.orc_build(_ptr(gx), _ptr(gy), _ptr(gz), _ptr(a), _ptr(w), self.n_gas,
                               _ptr(sx), _ptr(sy), _ptr(sz), _ptr(lum), self.n_src, _ptr(lo32),
                               float(side), int(bucket), ctypes.byref(h))
        if rc != ORC_OK:
            raise OracleError(rc)
        self._h = h
        self.lo = np.asarray(lo, dtype=np.float64)
        self.side = float(side)
        self.bucket = int(bucket)
        self.n_nodes = int(lib.orc_n_nodes(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_tree_free(h)
            self._h = None

    # ---- exports -------------------------------------------------------
    def nodes(self):
        n = self.n_nodes
        out = dict(
            first=np.zeros(n, np.int64), count=np.zeros(n, np.int64),
            parent=np.zeros(n, np.int64), lower=np.zeros(n, np.int64),
            upper=np.zeros(n, np.int64), split_bit=np.zeros(n, np.int32),
            depth=np.zeros(n, np.int32), glo=np.zeros((n, 3), np.int32),
            ghi=np.zeros((n, 3), np.int32), W=np.zeros(n), abar=np.zeros(n),
            amin=np.zeros(n), amax=np.zeros(n), L=np.zeros(n), cen=np.zeros((n, 3)),
            lrad=np.zeros(n), src_first=np.zeros(n, np.int64), src_count=np.zeros(n, np.int64))
        self._lib.orc_export_nodes(
            self._h, *(_ptr(out[k]) for k in (
                "first", "count", "parent", "lower", "upper", "split_bit", "depth", "glo", "ghi",
                "W", "abar", "amin", "amax", "L", "cen", "lrad", "src_first", "src_count")))
        return out

    def nodes32(self):
        n = self.n_nodes
        out = dict(abar=np.zeros(n, np.float32), dalpha=np.zeros(n, np.float32),
                   L=np.zeros(n, np.float32), cen=np.zeros((n, 3), np.float32),
                   l2=np.zeros(n, np.float32), blo=np.zeros((n, 3), np.float32),
                   bhi=np.zeros((n, 3), np.float32))
        self._lib.orc_export_nodes32(self._h, *(_ptr(out[k]) for k in (
            "abar", "dalpha", "L", "cen", "l2", "blo", "bhi")))
        return out

    def directional(self):
        """Directional (x, y, z) alpha_min and alpha_max of every node, shape (n, 3)."""
        amin = np.zeros((self.n_nodes, 3))
        amax = np.zeros((self.n_nodes, 3))
        self._lib.orc_export_directional(self._h, _ptr(amin), _ptr(amax))
        return amin, amax

    def particles(self):
        n = self.n_gas
        key = np.zeros(n, np.uint64)
        perm = np.zeros(n, np.int64)
        leaf = np.zeros(n, np.int64)
        self._lib.orc_export_particles(self._h, _ptr(key), _ptr(perm), _ptr(leaf))
        return dict(key=key, perm=perm, leaf_of=leaf)

    def sources(self):
        n = self.n_src
        order = np.zeros(n, np.int64)
        leaf = np.zeros(n, np.int64)
        self._lib.orc_export_sources(self._h, _ptr(order), _ptr(leaf))
        return dict(order=order, leaf=leaf)

    # ---- the method ----------------------------------------------------
    def flux(self, theta, tau_ref, sinks=None, nthreads=0, with_counters=False):
        """FP64 flux at the given sinks (caller indices; None = every gas particle).

        Returns flux, or (flux, counters[n,4], margin[n]) with with_counters.
        counters columns: interactions, segments, visited source nodes, refinements.
        """
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros(n)
        cnt = np.zeros((n, 4), np.int64) if with_counters else None
        mar = np.zeros(n) if with_counters else None
        rc = self._lib.orc_flux(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                _ptr(flux), _ptr(cnt), _ptr(mar), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return (flux, cnt, mar) if with_counters else flux

    def flux_background(self, theta, tau_ref, radius, sinks=None, nthreads=0,
                        with_counters=False):
        """Flux with all sources treated as background sources on the sphere of `radius`
        around the domain centre: merged centroids are moved onto the sphere (Sec. 2.2.4)."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros(n)
        cnt = np.zeros((n, 4), np.int64) if with_counters else None
        rc = self._lib.orc_flux_background(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                           float(radius), _ptr(flux), _ptr(cnt), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return (flux, cnt) if with_counters else flux

    def set_smoothing(self, h):
        """Smoothing lengths (N,) for the sub-bucket particle trace."""
        h = _f32(h)
        self._keep = self._keep + (h,)
        rc = self._lib.orc_set_smoothing(self._h, _ptr(h))
        if rc != ORC_OK:
            raise OracleError(rc)

    def flux_sub(self, theta, tau_ref, sinks=None, nthreads=0, with_counters=False):
        """Flux with the sub-bucket particle trace: a bucket whose alpha spread times the
        chord exceeds tau_ref (every bucket if tau_ref <= 0) integrates the SPH field
        of the particles along the chord, leaving out the receiving particle. counters
        columns: those of flux(), then the sub-bucket segments."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros(n)
        cnt = np.zeros((n, 5), np.int64) if with_counters else None
        rc = self._lib.orc_flux_sub(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                    _ptr(flux), _ptr(cnt), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return (flux, cnt) if with_counters else flux

    def flux_bands(self, theta, tau_ref, sinks=None, nthreads=0, with_counters=False):
        """Flux of every band (tree built with alpha (B, N)), shape (B, n); counters as
        in flux()."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros((max(self.n_bands, 1), n))
        cnt = np.zeros((n, 4), np.int64) if with_counters else None
        rc = self._lib.orc_flux_bands(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                      _ptr(flux), _ptr(cnt), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return (flux, cnt) if with_counters else flux

    def flux_terminated(self, theta, tau_ref, tau_stop, sinks=None, nthreads=0,
                        with_counters=False, bg_radius=0.0):
        """Flux with early ray termination (Sec. 4): a ray whose optical depth passes
        tau_stop > 0 adds nothing (bg_radius > 0: with the background sources of
        flux_background). counters columns: interactions, segments, visited source nodes,
        refinements (of the complete rays), terminated rays."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros(n)
        cnt = np.zeros((n, 5), np.int64) if with_counters else None
        rc = self._lib.orc_flux_terminated(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                           float(tau_stop), float(bg_radius), _ptr(flux),
                                           _ptr(cnt), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return (flux, cnt) if with_counters else flux

    def flux_moments(self, theta, tau_ref, sinks=None, nthreads=0):
        """(flux[n], flux vector[n,3] = sum f n, pressure[n,6] = sum f n n^T (xx,yy,zz,xy,xz,yz)),
        n the unit vector from each pseudo-source to the sink (Eq. simpflux)."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros(n)
        fvec = np.zeros((n, 3))
        press = np.zeros((n, 6))
        rc = self._lib.orc_flux_moments(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                        _ptr(flux), _ptr(fvec), _ptr(press), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return flux, fvec, press

    def interactions(self, sink, theta, tau_ref, cap=1 << 16, bg_radius=0.0):
        """Interaction list of one sink: node C, q, L, tau, summed length, flux, nseg, src."""
        out = dict(node=np.zeros(cap, np.int64), q=np.zeros((cap, 3)), L=np.zeros(cap),
                   tau=np.zeros(cap), len_sum=np.zeros(cap), flux=np.zeros(cap),
                   nseg=np.zeros(cap, np.int64), src=np.zeros(cap, np.int64))
        n = self._lib.orc_sink_interactions(
            self._h, int(sink), float(theta), float(tau_ref), float(bg_radius), cap,
            *(_ptr(out[k]) for k in ("node", "q", "L", "tau", "len_sum", "flux", "nseg", "src")))
        if n < 0 or n > cap:
            raise OracleError(ORC_ERR_NO_MEMORY)
        return {k: v[:n] for k, v in out.items()}

    def ray_tau(self, sink, node, q, tau_ref, topdown=False):
        """Optical depth (tau, summed segment length, segment count) of the method's ray
        from sink (caller index) to point q inside node; topdown selects the top-down
        ray walk instead of the paper's bottom-up one."""
        q = _f32(q)
        ls = ctypes.c_double()
        ns = ctypes.c_int64()
        t = self._lib.orc_ray_tau_walk(self._h, int(sink), int(node), _ptr(q), float(tau_ref),
                                       int(bool(topdown)), ctypes.byref(ls), ctypes.byref(ns))
        return t, ls.value, ns.value

    def flux_topdown(self, theta, tau_ref, sinks=None, nthreads=0, with_counters=False):
        """FP64 flux with the top-down ray walk (the ray starts as one segment in the
        lowest common ancestor of the sink's bucket and the source cell, and only the
        refinement criterion splits it). Returns flux, or (flux, counters[n,4]) with
        with_counters (interactions, segments, visited source nodes, refinements)."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        n = sinks.shape[0]
        flux = np.zeros(n)
        cnt = np.zeros((n, 4), np.int64) if with_counters else None
        rc = self._lib.orc_flux_topdown(self._h, _ptr(sinks), n, float(theta), float(tau_ref),
                                        _ptr(flux), _ptr(cnt), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return (flux, cnt) if with_counters else flux

    def adjoint(self, theta, tau_ref, grad_flux, sinks=None, nthreads=0):
        """FP64 gradients (grad_lum[n_src], grad_alpha[n_gas], caller order) of a loss with
        dLoss/dF = grad_flux at the sinks, decisions frozen."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        g = np.ascontiguousarray(grad_flux, dtype=np.float64)
        gl = np.zeros(self.n_src)
        ga = np.zeros(self.n_gas)
        rc = self._lib.orc_adjoint(self._h, _ptr(sinks), len(sinks), _ptr(g), float(theta),
                                   float(tau_ref), _ptr(gl), _ptr(ga), int(nthreads))
        if rc != ORC_OK:
            raise OracleError(rc)
        return gl, ga

    def replay(self, theta, tau_ref, sinks=None):
        """Record the decisions of the forward pass for `sinks`; returns a Replay."""
        if sinks is None:
            sinks = np.arange(self.n_gas, dtype=np.int64)
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = self._lib.orc_replay_record(self._h, _ptr(sinks), len(sinks), float(theta),
                                         float(tau_ref), ctypes.byref(h))
        if rc != ORC_OK:
            raise OracleError(rc)
        return Replay(self, h, len(sinks))

    def leaf_of_point(self, x, y, z):
        return int(self._lib.orc_leaf_of_point(self._h, float(x), float(y), float(z)))


class Replay:
    """Frozen decisions of one forward pass; evaluates sum_k w_k log F_k under a single
    perturbed luminosity (kind 0) or absorption coefficient (kind 1)."""

    def __init__(self, tree, handle, n_sink):
        self.tree = tree
        self._h = handle
        self.n_sink = n_sink

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.tree._lib.orc_replay_free(self._h)
            self._h = None

    def loss(self, w, kind=-1, index=0, h=0.0, frozen_planes=False):
        """frozen_planes: every segment keeps the bounding slab planes of the
        unperturbed ray, which makes the loss analytic in h (the function the
        adjoint differentiates); otherwise lengths are re-clipped (kinks where a
        bounding plane switches)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.shape[0] == self.n_sink
        return float(self.tree._lib.orc_replay_loss_planes(self.tree._h, self._h, _ptr(w),
                                                           int(kind), int(index), float(h),
                                                           int(bool(frozen_planes))))

    def kinks(self, kind, index, h):
        """Recorded segments whose bounding planes differ between -h and +h."""
        return int(self.tree._lib.orc_replay_kinks(self.tree._h, self._h, int(kind),
                                                   int(index), float(h)))
