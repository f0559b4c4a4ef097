"""ctypes binding of the C-ABI in include/xrl.h (argument marshalling only).

Every computation runs in libxrl.so; this module converts NumPy arrays and
torch CUDA tensors into pointers and sizes, and turns error codes into
exceptions.  There is no CPU fallback: if the library is missing, loading it
raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

STATUS = {0: "XRL_OK", 1: "XRL_EINVAL", 2: "XRL_ETOPO", 3: "XRL_ENOMEM", 4: "XRL_ECUDA",
          5: "XRL_ENOCONV", 6: "XRL_ETIMEOUT", 7: "XRL_ESTATE"}


class XRLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("fmm_order", ctypes.c_int32), ("leaf_target", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("inner_iters", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("device", ctypes.c_int32), ("separation", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
                ("mac_theta", ctypes.c_double), ("mg_cycles", ctypes.c_int32), ("rhs_chunk", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_panels", ctypes.c_int32), ("n_live", ctypes.c_int32), ("n_branches", ctypes.c_int32),
                ("n_loops", ctypes.c_int32), ("n_ports", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("n_boxes", ctypes.c_int32), ("near_nnz", ctypes.c_int64),
                ("n_vertex_loops", ctypes.c_int32), ("n_global_loops", ctypes.c_int32),
                ("total_iters", ctypes.c_int32), ("total_inner", ctypes.c_int32), ("n_mvm", ctypes.c_int32),
                ("max_rel_res", ctypes.c_double), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("mvm_ms", ctypes.c_double), ("peak_device_bytes", ctypes.c_int64),
                ("near_nnz_padded", ctypes.c_int64), ("precond_setup_ms", ctypes.c_double),
                ("tc_targets_per_cta", ctypes.c_int32), ("setup_phase_ms", ctypes.c_double * 6),
                ("mg_levels", ctypes.c_int32), ("mg_coarse_n", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("cached_device_bytes", ctypes.c_int64)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["setup_phase_ms"] = list(self.setup_phase_ms)
        return out


def library_path():
    return os.path.join(_HERE, "libxrl.so")


# exported symbols and their signatures (must match include/xrl.h)
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "xrl_default_options": (None, [ctypes.POINTER(Options)]),
    "xrl_create": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "xrl_set_mesh": (ctypes.c_int, [_P, ctypes.c_int64, _D, ctypes.c_int64, _I, _I]),
    "xrl_set_mesh_panels": (ctypes.c_int, [_P, ctypes.c_int64, _D, ctypes.c_int64, _I, _I]),
    "xrl_set_conductors": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D]),
    "xrl_add_port": (ctypes.c_int, [_P, ctypes.c_int64, _I, ctypes.c_int64, _I, _I]),
    "xrl_setup": (ctypes.c_int, [_P]),
    "xrl_fmm_mvm": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D]),
    "xrl_fmm_mvm_device": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "xrl_fmm_mvm_device_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "xrl_direct_mvm_device": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "xrl_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "xrl_fmm_mvm32_device": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "xrl_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _I, _I, _D, _D]),
    "xrl_solve": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D, _D]),
    "xrl_apply_operator": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D, _D]),
    "xrl_apply_precond_matrix": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D, _D]),
    "xrl_apply_precond_inverse": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D, _D]),
    "xrl_export_tree": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), _I, _I]),
    "xrl_export_branches": (ctypes.c_int, [_P, _I, _I]),
    "xrl_export_loops": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), _I, ctypes.POINTER(ctypes.c_int8)]),
    "xrl_export_lists": (ctypes.c_int, [_P, ctypes.c_int32, _I, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_int64), _I, ctypes.POINTER(ctypes.c_int64), _I]),
    "xrl_set_profiling": (ctypes.c_int, [_P, ctypes.c_int32]),
    "xrl_get_profile": (ctypes.c_int, [_P, ctypes.c_int32, _D, ctypes.POINTER(ctypes.c_int64), _D, _D]),
    "xrl_reset_profile": (ctypes.c_int, [_P]),
    "xrl_kernel_launches": (ctypes.c_int64, [_P]),
    "xrl_get_stream": (ctypes.c_void_p, [_P]),
    "xrl_get_panel_currents": (ctypes.c_int, [_P, ctypes.c_int32, _D]),
    "xrl_panel_features": (ctypes.c_int, [_P, ctypes.c_int32, _D, ctypes.c_double, _P, _P, _D, _P]),
    "xrl_solve_guess": (ctypes.c_int, [_P, ctypes.c_int32, _D, _P, _D, _D, _I, _D]),
    "xrl_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(_P)]),
    "xrl_mlp_num_params": (ctypes.c_int64, [_P]),
    "xrl_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
    "xrl_mlp_train_step": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_float, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_double), _P]),
    "xrl_mlp_gradients": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_double)]),
    "xrl_mlp_get_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "xrl_mlp_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "xrl_mlp_last_error": (ctypes.c_char_p, [_P]),
    "xrl_mlp_destroy": (None, [_P]),
    "xrl_last_error": (ctypes.c_char_p, [_P]),
    "xrl_destroy": (None, [_P]),
}


def lib():
    """Load libxrl.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libxrl.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


class XRL:
    """One library context: a mesh, its setup products and solves."""

    def __init__(self, **opts):
        L = lib()
        o = Options()
        L.xrl_default_options(ctypes.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        h = _P()
        self._check(L.xrl_create(ctypes.byref(o), ctypes.byref(h)), None)
        self.h = h
        self.opts = o
        self.n_tri = 0
        self._last_nsys = 0

    def _check(self, code, h):
        if code != 0:
            msg = lib().xrl_last_error(h).decode() if h else ""
            raise XRLError(code, msg)

    def close(self):
        if getattr(self, "h", None):
            lib().xrl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- problem definition -------------------------------------------------
    def set_mesh(self, xyz, tri, cond=None):
        """tri: [n, 3] triangles, or [n, 4] hybrid panels (-1 in the 4th slot of a triangle)."""
        xyz = np.ascontiguousarray(xyz, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        c = None if cond is None else np.ascontiguousarray(cond, np.int32)
        self.n_tri = tri.shape[0]
        fn = lib().xrl_set_mesh_panels if tri.shape[1] == 4 else lib().xrl_set_mesh
        self._check(fn(self.h, xyz.shape[0], _dp(xyz), tri.shape[0], _ip(tri),
                       None if c is None else _ip(c)), self.h)

    def set_conductors(self, sigma, thickness):
        s = np.ascontiguousarray(sigma, np.float64)
        t = np.ascontiguousarray(thickness, np.float64)
        self._check(lib().xrl_set_conductors(self.h, s.shape[0], _dp(s), _dp(t)), self.h)

    def add_port(self, src, sink):
        s = np.ascontiguousarray(src, np.int32)
        k = np.ascontiguousarray(sink, np.int32)
        pid = ctypes.c_int32()
        self._check(lib().xrl_add_port(self.h, s.shape[0], _ip(s), k.shape[0], _ip(k), ctypes.byref(pid)), self.h)
        return pid.value

    def setup(self):
        self._check(lib().xrl_setup(self.h), self.h)

    @classmethod
    def from_mesh(cls, mesh, **opts):
        """Context for a mesh object with xyz, tri, cond, term, ports, sigma, thickness."""
        x = cls(**opts)
        x.set_mesh(mesh.xyz, mesh.tri, mesh.cond)
        x.set_conductors(mesh.sigma, mesh.thickness)
        term = np.asarray(mesh.term)
        for s, k in mesh.ports:
            x.add_port(np.flatnonzero(term == s), np.flatnonzero(term == k))
        x.setup()
        return x

    # ---- products --------------------------------------------------------------
    def fmm_mvm(self, x):
        """y = P x with host arrays; x is [N] or [n_cols][N]."""
        x = np.ascontiguousarray(x, np.float64)
        one = x.ndim == 1
        xx = x[None] if one else x
        y = np.empty_like(xx)
        self._check(lib().xrl_fmm_mvm(self.h, xx.shape[0], _dp(xx), _dp(y)), self.h)
        return y[0] if one else y

    def fmm_mvm_device(self, x, y, stream=None):
        """y = P x on torch CUDA tensors [n_cols][N] (float64, contiguous)."""
        assert x.is_cuda and x.dtype.is_floating_point and x.is_contiguous() and y.is_contiguous()
        nc = 1 if x.dim() == 1 else x.shape[0]
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(lib().xrl_fmm_mvm_device(self.h, nc, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(y.data_ptr()), s), self.h)

    def fmm_mvm32_device(self, x, y, stream=None):
        """y = P x in the FP32 inner-iteration product on torch CUDA float32 tensors [n_cols][N]."""
        assert x.is_cuda and x.is_contiguous() and y.is_contiguous()
        nc = 1 if x.dim() == 1 else x.shape[0]
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(lib().xrl_fmm_mvm32_device(self.h, nc, ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), s), self.h)

    def direct_mvm_device(self, x, y, stream=None):
        assert x.is_cuda and x.is_contiguous() and y.is_contiguous()
        nc = 1 if x.dim() == 1 else x.shape[0]
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(lib().xrl_direct_mvm_device(self.h, nc, ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(y.data_ptr()), s), self.h)

    def solve(self, freqs):
        f = np.ascontiguousarray(freqs, np.float64)
        npt = self.stats()["n_ports"]
        R = np.empty((f.shape[0], npt, npt))
        L = np.empty_like(R)
        code = lib().xrl_solve(self.h, f.shape[0], _dp(f), _dp(R), _dp(L))
        self._check(code, self.h)
        self._last_nsys = f.shape[0] * npt
        return R, L

    def apply_operator(self, freqs, v, precond_matrix=False, precond_inverse=False):
        """w_s = Z(f_s) v_s (or Q(f_s) v_s, or Q(f_s)^-1 v_s); v complex [n_sys][n_loops]."""
        f = np.ascontiguousarray(freqs, np.float64)
        v = np.ascontiguousarray(v, np.complex128)
        w = np.empty_like(v)
        fn = lib().xrl_apply_operator
        if precond_matrix:
            fn = lib().xrl_apply_precond_matrix
        if precond_inverse:
            fn = lib().xrl_apply_precond_inverse
        self._check(fn(self.h, f.shape[0], _dp(f), v.ctypes.data_as(_D), w.ctypes.data_as(_D)), self.h)
        return w

    def autotune(self, n_cols, mvm_tol=1e-6, precision=1):
        """Pick leaf_target and fmm_order (see xrl_autotune); returns (leaf, order, ms, err)."""
        leaf = ctypes.c_int32()
        order = ctypes.c_int32()
        ms = ctypes.c_double()
        err = ctypes.c_double()
        self._check(lib().xrl_autotune(self.h, n_cols, mvm_tol, precision, ctypes.byref(leaf), ctypes.byref(order),
                                       ctypes.byref(ms), ctypes.byref(err)), self.h)
        self.opts.leaf_target = leaf.value
        self.opts.fmm_order = order.value
        return leaf.value, order.value, ms.value, err.value

    # ---- learned initial guess -------------------------------------------------------
    def panel_currents(self, normalize=True):
        """[n_sys][n_panels][6] panel currents of the last solve (per unit port current if normalize)."""
        st = self.stats()
        n = st["n_panels"]
        # n_sys of the last solve is inferred from the buffer the library fills
        nsys = self._last_nsys
        out = np.empty((nsys, n, 6))
        self._check(lib().xrl_get_panel_currents(self.h, 1 if normalize else 0, _dp(out)), self.h)
        return out

    def features(self, freqs, f0, ip0):
        """ip0: torch CUDA float64 [n_ports][n_panels][6] -> (torch float32 [n_f*n_p][n_panels][24],
        per-port reference scale [n_ports])."""
        import torch
        f = np.ascontiguousarray(freqs, np.float64)
        npt = self.stats()["n_ports"]
        feat = torch.empty((f.shape[0] * npt, self.n_tri, 24), device=ip0.device, dtype=torch.float32)
        scale = np.empty(npt)
        self._check(lib().xrl_panel_features(self.h, f.shape[0], _dp(f), float(f0),
                                             ctypes.c_void_p(ip0.data_ptr()), ctypes.c_void_p(feat.data_ptr()),
                                             _dp(scale), None), self.h)
        return feat, scale

    def solve_guess(self, freqs, shape):
        """xrl_solve from predicted current shapes (torch CUDA float32 [n_sys][n_panels][6])."""
        f = np.ascontiguousarray(freqs, np.float64)
        npt = self.stats()["n_ports"]
        nsys = f.shape[0] * npt
        R = np.empty((f.shape[0], npt, npt))
        L = np.empty_like(R)
        acc = np.zeros(nsys, np.int32)
        gr = np.zeros(nsys)
        self._check(lib().xrl_solve_guess(self.h, f.shape[0], _dp(f), ctypes.c_void_p(shape.data_ptr()), _dp(R),
                                          _dp(L), _ip(acc), _dp(gr)), self.h)
        self._last_nsys = nsys
        return R, L, acc, gr

    # ---- profiling ---------------------------------------------------------------
    PHASES = ["p2p", "p2m", "m2m", "m2l", "l2l", "l2p", "operator", "precond", "krylov", "p2p64", "m2l64"]

    def set_profiling(self, on=True):
        self._check(lib().xrl_set_profiling(self.h, 1 if on else 0), self.h)

    def reset_profile(self):
        self._check(lib().xrl_reset_profile(self.h), self.h)

    def profile(self):
        """{phase: dict(ms, launches, flops, bytes)} since the last reset."""
        out = {}
        for i, name in enumerate(self.PHASES):
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            fl = ctypes.c_double()
            by = ctypes.c_double()
            self._check(lib().xrl_get_profile(self.h, i, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                              ctypes.byref(by)), self.h)
            out[name] = {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}
        return out

    def stream_handle(self):
        """The library's own cudaStream_t as an int (for torch.cuda.ExternalStream)."""
        return int(lib().xrl_get_stream(self.h) or 0)

    def kernel_launches(self):
        return int(lib().xrl_kernel_launches(self.h))

    # ---- introspection ---------------------------------------------------------
    def stats(self):
        s = Stats()
        self._check(lib().xrl_get_stats(self.h, ctypes.byref(s)), self.h)
        return s.as_dict()

    def export_tree(self):
        n = self.n_tri
        keys = np.empty(n, np.uint64)
        perm = np.empty(n, np.int32)
        leaf = np.empty(n, np.int32)
        self._check(lib().xrl_export_tree(self.h, keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                          _ip(perm), _ip(leaf)), self.h)
        return keys, perm, leaf

    def export_branches(self):
        nb = self.stats()["n_branches"]
        t = np.empty(nb, np.int32)
        h = np.empty(nb, np.int32)
        self._check(lib().xrl_export_branches(self.h, _ip(t), _ip(h)), self.h)
        return t, h

    def export_loops(self):
        nl = self.stats()["n_loops"]
        ptr = np.empty(nl + 1, np.int64)
        P64 = ctypes.POINTER(ctypes.c_int64)
        self._check(lib().xrl_export_loops(self.h, ptr.ctypes.data_as(P64), None, None), self.h)
        col = np.empty(ptr[-1], np.int32)
        val = np.empty(ptr[-1], np.int8)
        self._check(lib().xrl_export_loops(self.h, ptr.ctypes.data_as(P64), _ip(col),
                                           val.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))), self.h)
        return ptr, col, val

    def export_lists(self, level):
        nb = ctypes.c_int32()
        self._check(lib().xrl_export_lists(self.h, level, ctypes.byref(nb), None, None, None, None, None), self.h)
        n = nb.value
        keys = np.empty(n, np.uint64)
        vptr = np.empty(n + 1, np.int64)
        P64 = ctypes.POINTER(ctypes.c_int64)
        self._check(lib().xrl_export_lists(self.h, level, ctypes.byref(nb),
                                           keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                           vptr.ctypes.data_as(P64), None, None, None), self.h)
        vsrc = np.empty(vptr[-1], np.int32)
        st = self.stats()
        is_leaf = level == st["n_levels"] - 1
        uptr = np.empty(n + 1, np.int64) if is_leaf else None
        self._check(lib().xrl_export_lists(self.h, level, ctypes.byref(nb),
                                           keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                           vptr.ctypes.data_as(P64), _ip(vsrc),
                                           uptr.ctypes.data_as(P64) if is_leaf else None, None), self.h)
        usrc = None
        if is_leaf:
            usrc = np.empty(uptr[-1], np.int32)
            self._check(lib().xrl_export_lists(self.h, level, ctypes.byref(nb), None, None, None,
                                               uptr.ctypes.data_as(P64), _ip(usrc)), self.h)
        return keys, vptr, vsrc, uptr, usrc


class MLP:
    """Per-panel network of the library (BF16 weights, FP32 accumulation)."""

    def __init__(self, n_in=24, width=128, n_hidden=3, n_out=6, seed=0, device=0):
        h = _P()
        code = lib().xrl_mlp_create(n_in, width, n_hidden, n_out, seed, device, ctypes.byref(h))
        if code != 0:
            raise XRLError(code, "xrl_mlp_create")
        self.h = h
        self.n_in, self.n_out = n_in, n_out

    def _check(self, code):
        if code != 0:
            raise XRLError(code, lib().xrl_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().xrl_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_params(self):
        return int(lib().xrl_mlp_num_params(self.h))

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], self.n_out), device=x.device, dtype=torch.float32)
        self._check(lib().xrl_mlp_forward(self.h, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr()), None))
        return y

    def train_step(self, x, t, lr=1e-3, weight_decay=1e-4):
        loss = ctypes.c_double()
        self._check(lib().xrl_mlp_train_step(self.h, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(t.data_ptr()), lr, weight_decay, ctypes.byref(loss),
                                             None))
        return loss.value

    def gradients(self, x, t):
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_double()
        self._check(lib().xrl_mlp_gradients(self.h, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(t.data_ptr()),
                                            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
        return g, loss.value

    def get_params(self):
        p = np.empty(self.n_params, np.float32)
        self._check(lib().xrl_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._check(lib().xrl_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
