"""Thin ctypes binding of libfe2 (the C ABI declared in include/fe2.h).

Argument marshalling only: every step of the RVE block runs in the CUDA
kernels of libfe2.  PyTorch provides device memory and the stream.  There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.

Module-level functions carry the C names (``fe2_create``, ``fe2_rve_solve``
...); :class:`Fe2Context` wraps them for tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfe2.so")

FE2_OK, FE2_ERR_ARG, FE2_ERR_CUDA, FE2_ERR_BUDGET = 0, 1, 2, 3
FE2_ERR_NOT_PD, FE2_ERR_NAN, FE2_ERR_NO_CONV, FE2_ERR_TIMEOUT = 4, 5, 6, 7
FE2_ELEM_Q4, FE2_ELEM_HEX8 = 0, 1
FE2_PREC_FP64, FE2_PREC_MIXED = 0, 1
FE2_FACTOR_AUTO, FE2_FACTOR_CUDA_CORE, FE2_FACTOR_TENSOR_CORE, FE2_FACTOR_CUDA_CORE_PIPELINED = 0, 1, 2, 3
FACTOR_KERNELS = {"auto": FE2_FACTOR_AUTO, "cuda_core": FE2_FACTOR_CUDA_CORE, "tensor_core": FE2_FACTOR_TENSOR_CORE,
                  "cuda_core_pipelined": FE2_FACTOR_CUDA_CORE_PIPELINED}
FE2_BASIS_DIRAC, FE2_BASIS_CONST = 0, 1
MACRO_BASES = {"dirac": FE2_BASIS_DIRAC, "const": FE2_BASIS_CONST}
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_BUDGET", 4: "NOT_PD", 5: "NAN",
                6: "NO_CONV", 7: "TIMEOUT"}


class fe2_config(C.Structure):
    _fields_ = [("dim", C.c_int), ("elem", C.c_int), ("precision", C.c_int),
                ("hbm_budget_bytes", C.c_size_t), ("cuda_stream", C.c_void_p),
                ("refine_tol", C.c_double), ("max_refine", C.c_int),
                ("factor_kernel", C.c_int), ("macro_basis", C.c_int)]


class Fe2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = C.c_void_p
_I = C.c_int
_IP = C.POINTER(C.c_int)
_DP = C.POINTER(C.c_double)

_SIGS = {
    "fe2_create": (_I, [C.POINTER(fe2_config), C.POINTER(_P)]),
    "fe2_destroy": (None, [_P]),
    "fe2_last_error": (C.c_char_p, [_P]),
    "fe2_sync": (_I, [_P]),
    "fe2_rve_bytes": (C.c_size_t, [_P, _I]),
    "fe2_rve_register": (_I, [_P, _I, _IP, C.POINTER(C.c_uint8), _I, _DP, _IP]),
    "fe2_rve_release": (_I, [_P, _I, _IP]),
    "fe2_rve_define": (_I, [_P, _I, _IP, C.POINTER(C.c_uint8), _I, _DP, _IP]),
    "fe2_rve_admit": (_I, [_P, _I, _IP]),
    "fe2_rve_evict": (_I, [_P, _I, _IP]),
    "fe2_rve_resident": (_I, [_P, _I]),
    "fe2_micro_assemble": (_I, [_P, _I, _IP, _P]),
    "fe2_nullspace_reduce": (_I, [_P, _I, _IP]),
    "fe2_condense": (_I, [_P, _I, _IP, _P, _P, _P, _P]),
    "fe2_rve_solve": (_I, [_P, _I, _IP, _P, _P, _P, _P, _P]),
    "fe2_macro_step": (_I, [_P, _I, _IP, _P]),
    "fe2_macro_setup": (_I, [_P, _I, _DP, _I, _IP, C.POINTER(C.c_uint8)]),
    "fe2_macro_set_positions": (_I, [_P, _DP, C.POINTER(C.c_uint8)]),
    "fe2_macro_get_positions": (_I, [_P, _DP]),
    "fe2_macro_set_load": (_I, [_P, _DP]),
    "fe2_macro_set_edge_load": (_I, [_P, _I, _IP, _DP, C.c_double]),
    "fe2_rve_set_quad_weights": (_I, [_P, _I, _IP, _DP]),
    "fe2_macro_gradients": (_I, [_P, _P, _P]),
    "fe2_macro_residual": (_I, [_P, _P, _P]),
    "fe2_macro_solve": (_I, [_P, _P, _P, _P, _P, _P]),
    "fe2_macro_system_size": (_I, [_P, _IP, _IP]),
    "fe2_macro_assemble": (_I, [_P, _P, _P, _P, _P]),
    "fe2_macro_norm": (_I, [_P, _P, _P]),
    "fe2_macro_solve_assembled": (_I, [_P, _P, _P, _P, _P, _P]),
    "fe2_rve_average_stress": (_I, [_P, _I, _IP, _P]),
    "fe2_rve_residual_norm": (_I, [_P, _I, _IP, _P]),
    "fe2_rve_export": (_I, [_P, _I, _I, _DP]),
    "fe2_rve_set_w": (_I, [_P, _I, _DP]),
    "fe2_rve_w_copy": (_I, [_P, _I, _IP, _P, _I, _I]),
    "fe2_launch_count": (C.c_longlong, [_P]),
    "fe2_rve_solve_noalloc": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fe2_noalloc_last_error": (C.c_char_p, []),
    "fe2_server_create": (_I, [_P, _I, _I, C.POINTER(_P)]),
    "fe2_server_destroy": (None, [_P]),
    "fe2_server_submit": (_I, [_P, _I, _IP, _DP, C.POINTER(C.c_longlong)]),
    "fe2_server_pump": (_I, [_P, _IP]),
    "fe2_server_take": (_I, [_P, _I, C.POINTER(C.c_longlong), _DP, _DP, _IP, _DP]),
    "fe2_server_pending": (_I, [_P]),
    "fe2_server_use_graphs": (_I, [_P, _I]),
    "fe2_server_graph_stats": (_I, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "fe2_server_bucket": (_I, [_P, _I]),
    "fe2_server_mixed_sizes": (_I, [_P, _I]),
    "fe2_server_memory_stats": (_I, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                     C.POINTER(C.c_longlong), C.POINTER(C.c_size_t)]),
    "fe2_selftest_wait_timeout": (_I, [_P, _P]),
    "fe2_profile": (_I, [_P, _I]),
    "fe2_profile_read": (_I, [_P, _I, C.c_char_p, _DP, C.POINTER(C.c_longlong)]),
}


def load(path: str = LIB_PATH):
    """Load libfe2 (built by ``paper_2312_12771_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfe2 not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


# C-named thin wrappers --------------------------------------------------------
def _call(name, *args):
    return getattr(load(), name)(*args)


def fe2_create(cfg):
    h = C.c_void_p()
    st = _call("fe2_create", C.byref(cfg), C.byref(h))
    if st != FE2_OK:
        raise Fe2Error(st, "fe2_create failed")
    return h


def fe2_destroy(h):
    _call("fe2_destroy", h)


def fe2_last_error(h):
    return _call("fe2_last_error", h).decode()


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _ids(ids):
    a = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
    return a, a.ctypes.data_as(_IP)


def rve_solve_noalloc(N, phase, mat, Fbar, out, stream=None):
    """Call fe2_rve_solve_noalloc: the fused mixed-precision RVE solve with all
    intermediate data in the library's fixed device scratch array (no device
    allocation by the library).  phase [n, N*N] uint8, mat [n, nphase, 4] f64,
    Fbar [n, 2, 2] f64 and the outputs out = (sigma [n,4], Cbar [n,4,4],
    status [n] int32, err [n] f64 or None) are caller-owned CUDA tensors on the
    current device; a wrong device, dtype, shape or layout raises ValueError
    before the library is called."""
    import torch
    if Fbar.dim() != 3 or tuple(Fbar.shape[1:]) != (2, 2):
        raise ValueError(f"Fbar must be [n, 2, 2], got {tuple(Fbar.shape)}")
    n = Fbar.shape[0]
    if mat.dim() != 3 or mat.shape[0] != n or mat.shape[2] != 4:
        raise ValueError(f"mat must be [n, nphase, 4], got {tuple(mat.shape)}")
    nphase = mat.shape[1]
    sig, Cb, st, err = out
    dev = torch.device("cuda", torch.cuda.current_device())
    want = [("phase", phase, torch.uint8, (n, N * N)), ("mat", mat, torch.float64, (n, nphase, 4)),
            ("Fbar", Fbar, torch.float64, (n, 2, 2)), ("sigma", sig, torch.float64, (n, 4)),
            ("Cbar", Cb, torch.float64, (n, 4, 4)), ("status", st, torch.int32, (n,))]
    if err is not None:
        want.append(("err", err, torch.float64, (n,)))
    for name, t, dt, shape in want:
        if not isinstance(t, torch.Tensor) or t.device != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device {dev}")
        if t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt} tensor of shape {shape}, got {t.dtype} "
                             f"{tuple(t.shape)}{'' if t.is_contiguous() else ' (not contiguous)'}")
    s = stream if stream is not None else torch.cuda.current_stream()
    code = load().fe2_rve_solve_noalloc(int(N), int(n), int(nphase), _ptr(phase), _ptr(mat), _ptr(Fbar),
                                        _ptr(sig), _ptr(Cb), _ptr(st), _ptr(err), C.c_void_p(s.cuda_stream))
    if code != FE2_OK:
        why = load().fe2_noalloc_last_error().decode()
        raise Fe2Error(code, f"fe2_rve_solve_noalloc(N={N}, n={n}) failed: {why}")
    return out


class Fe2Context:
    """A libfe2 context on the current CUDA device and stream."""

    def __init__(self, dim=2, precision="mixed", hbm_budget_bytes=0, refine_tol=1e-10, max_refine=2,
                 stream=None, factor="auto", basis="dirac"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libfe2 needs a CUDA GPU (GB300, sm_103a)")
        self.torch = torch
        self.dim = dim
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.precision = precision
        cfg = fe2_config(dim, FE2_ELEM_Q4 if dim == 2 else FE2_ELEM_HEX8,
                         FE2_PREC_MIXED if precision == "mixed" else FE2_PREC_FP64,
                         int(hbm_budget_bytes), C.c_void_p(self.stream.cuda_stream), float(refine_tol),
                         int(max_refine), FACTOR_KERNELS[factor], MACRO_BASES[basis])
        self.basis = basis
        self.nq = 4 if basis == "const" else 1
        self.cfg = cfg
        self.h = fe2_create(cfg)
        self.lib = load()

    def close(self):
        if getattr(self, "h", None) is not None:
            fe2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != FE2_OK:
            raise Fe2Error(st, f"{what}: {fe2_last_error(self.h)}")

    # -- registry ---------------------------------------------------------------
    def register(self, N, phase_concat, mat):
        N = np.ascontiguousarray(np.asarray(N, dtype=np.int32))
        ph = np.ascontiguousarray(np.asarray(phase_concat, dtype=np.uint8))
        mat = np.ascontiguousarray(np.asarray(mat, dtype=np.float64))
        nphase = mat.shape[1]
        out = np.zeros(len(N), dtype=np.int32)
        st = self.lib.fe2_rve_register(self.h, len(N), N.ctypes.data_as(_IP),
                                       ph.ctypes.data_as(C.POINTER(C.c_uint8)), nphase,
                                       mat.ctypes.data_as(_DP), out.ctypes.data_as(_IP))
        self._check(st, "fe2_rve_register")
        return out

    def register_batch(self, batch):
        return self.register(batch.N, batch.phase_concat(), batch.mat)

    def define(self, N, phase_concat, mat):
        """fe2_rve_define: RVE definitions without device state (admitted on use)."""
        N = np.ascontiguousarray(np.asarray(N, dtype=np.int32))
        ph = np.ascontiguousarray(np.asarray(phase_concat, dtype=np.uint8))
        mat = np.ascontiguousarray(np.asarray(mat, dtype=np.float64))
        out = np.zeros(len(N), dtype=np.int32)
        st = self.lib.fe2_rve_define(self.h, len(N), N.ctypes.data_as(_IP), ph.ctypes.data_as(C.POINTER(C.c_uint8)),
                                     mat.shape[1], mat.ctypes.data_as(_DP), out.ctypes.data_as(_IP))
        self._check(st, "fe2_rve_define")
        return out

    def define_batch(self, batch):
        return self.define(batch.N, batch.phase_concat(), batch.mat)

    def admit(self, ids):
        a, p = _ids(ids)
        self._check(self.lib.fe2_rve_admit(self.h, len(a), p), "fe2_rve_admit")

    def evict(self, ids):
        a, p = _ids(ids)
        self._check(self.lib.fe2_rve_evict(self.h, len(a), p), "fe2_rve_evict")

    def resident(self, rve_id):
        return int(self.lib.fe2_rve_resident(self.h, int(rve_id)))

    def release(self, ids):
        a, p = _ids(ids)
        self._check(self.lib.fe2_rve_release(self.h, len(a), p), "fe2_rve_release")

    def rve_bytes(self, N):
        return int(self.lib.fe2_rve_bytes(self.h, int(N)))

    # -- the hot path ------------------------------------------------------------
    def _outs(self, n):
        """(sigma_eff [n, nq*d*d], Cbar [n, nq*d*d, nq*d*d], status [n], err [n])."""
        t = self.torch
        dd = self.dim * self.dim * self.nq
        dev = "cuda"
        return (t.empty((n, dd), dtype=t.float64, device=dev), t.empty((n, dd, dd), dtype=t.float64, device=dev),
                t.empty(n, dtype=t.int32, device=dev), t.empty(n, dtype=t.float64, device=dev))

    def rve_solve(self, ids, Fbar, out=None):
        """Fused S1-S6: returns (sigma_eff [n,d*d], Cbar [n,d*d,d*d], status [n], err [n])."""
        a, p = _ids(ids)
        Fbar = Fbar.contiguous()
        assert Fbar.is_cuda and Fbar.dtype == self.torch.float64
        sig, Cb, st, err = out if out is not None else self._outs(len(a))
        self._check(self.lib.fe2_rve_solve(self.h, len(a), p, _ptr(Fbar), _ptr(sig), _ptr(Cb), _ptr(st), _ptr(err)),
                    "fe2_rve_solve")
        return sig, Cb, st, err

    def micro_assemble(self, ids, Fbar):
        a, p = _ids(ids)
        Fbar = Fbar.contiguous()
        self._check(self.lib.fe2_micro_assemble(self.h, len(a), p, _ptr(Fbar)), "fe2_micro_assemble")

    def nullspace_reduce(self, ids):
        a, p = _ids(ids)
        self._check(self.lib.fe2_nullspace_reduce(self.h, len(a), p), "fe2_nullspace_reduce")

    def condense(self, ids, out=None):
        a, p = _ids(ids)
        sig, Cb, st, err = out if out is not None else self._outs(len(a))
        self._check(self.lib.fe2_condense(self.h, len(a), p, _ptr(sig), _ptr(Cb), _ptr(st), _ptr(err)),
                    "fe2_condense")
        return sig, Cb, st, err

    def macro_step(self, ids, dFbar):
        a, p = _ids(ids)
        dFbar = dFbar.contiguous()
        self._check(self.lib.fe2_macro_step(self.h, len(a), p, _ptr(dFbar)), "fe2_macro_step")

    # -- macro problem (S7) --------------------------------------------------------
    def macro_setup(self, X, conn, fixed):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        conn = np.ascontiguousarray(np.asarray(conn, dtype=np.int32))
        fixed = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
        self._check(self.lib.fe2_macro_setup(self.h, len(X), X.ctypes.data_as(_DP), len(conn),
                                             conn.ctypes.data_as(_IP), fixed.ctypes.data_as(C.POINTER(C.c_uint8))),
                    "fe2_macro_setup")
        self.macro_nnode, self.macro_ngp = len(X), (1 << self.dim) * len(conn)

    def macro_set_positions(self, q, which=None):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        w = None if which is None else np.ascontiguousarray(np.asarray(which, dtype=np.uint8))
        self._check(self.lib.fe2_macro_set_positions(self.h, q.ctypes.data_as(_DP),
                                                     None if w is None else w.ctypes.data_as(C.POINTER(C.c_uint8))),
                    "fe2_macro_set_positions")

    def macro_get_positions(self):
        q = np.zeros((self.macro_nnode, self.dim))
        self._check(self.lib.fe2_macro_get_positions(self.h, q.ctypes.data_as(_DP)), "fe2_macro_get_positions")
        return q

    def rve_set_quad_weights(self, ids, wq):
        """Element RVEs: normalised weights [n][nq] of their macro Gauss points."""
        a, p = _ids(ids)
        w = np.ascontiguousarray(np.asarray(wq, dtype=np.float64).reshape(len(a), self.nq))
        self._check(self.lib.fe2_rve_set_quad_weights(self.h, len(a), p, w.ctypes.data_as(_DP)),
                    "fe2_rve_set_quad_weights")

    def macro_set_load(self, fext):
        """Nodal external forces [nnode][d] of the current load (None = no load)."""
        if fext is None:
            self._check(self.lib.fe2_macro_set_load(self.h, None), "fe2_macro_set_load")
            return
        f = np.ascontiguousarray(np.asarray(fext, dtype=np.float64).reshape(self.macro_nnode, self.dim))
        self._check(self.lib.fe2_macro_set_load(self.h, f.ctypes.data_as(_DP)), "fe2_macro_set_load")

    def macro_set_edge_load(self, nodes, T, scale=1.0):
        """Surface load of a constant traction T on the boundary polyline `nodes`
        (consistent nodal forces computed by the library), times `scale`."""
        a, p = _ids(nodes)
        t = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(2))
        self._check(self.lib.fe2_macro_set_edge_load(self.h, len(a), p, t.ctypes.data_as(_DP), float(scale)),
                    "fe2_macro_set_edge_load")

    def macro_gradients(self, Fbar, eta=None):
        """Fbar_b of every macro Gauss point; eta (optional) receives the weights."""
        self._check(self.lib.fe2_macro_gradients(self.h, _ptr(Fbar), None if eta is None else _ptr(eta)),
                    "fe2_macro_gradients")

    def macro_residual(self, stress, rnorm):
        self._check(self.lib.fe2_macro_residual(self.h, _ptr(stress), _ptr(rnorm)), "fe2_macro_residual")

    def macro_solve(self, sigma, Cbar, dFbar, rnorm, status=None):
        self._check(self.lib.fe2_macro_solve(self.h, _ptr(sigma), _ptr(Cbar), _ptr(dFbar), _ptr(rnorm),
                                             _ptr(status)), "fe2_macro_solve")

    def macro_system_size(self):
        """(free macro DOFs, half bandwidth) of the assembled macro system."""
        nf, kd = C.c_int(0), C.c_int(0)
        self._check(self.lib.fe2_macro_system_size(self.h, C.byref(nf), C.byref(kd)), "fe2_macro_system_size")
        return nf.value, kd.value

    def macro_assemble(self, sigma, Cbar, K, R):
        """Assemble K (None with Cbar None: R only) and R into caller-owned buffers."""
        self._check(self.lib.fe2_macro_assemble(self.h, _ptr(sigma), _ptr(Cbar), _ptr(K), _ptr(R)),
                    "fe2_macro_assemble")

    def macro_norm(self, R, rnorm):
        self._check(self.lib.fe2_macro_norm(self.h, _ptr(R), _ptr(rnorm)), "fe2_macro_norm")

    def macro_solve_assembled(self, K, R, dFbar, rnorm, status=None):
        self._check(self.lib.fe2_macro_solve_assembled(self.h, _ptr(K), _ptr(R), _ptr(dFbar), _ptr(rnorm),
                                                       _ptr(status)), "fe2_macro_solve_assembled")

    def rve_average_stress(self, ids, Pbar):
        a, p = _ids(ids)
        self._check(self.lib.fe2_rve_average_stress(self.h, len(a), p, _ptr(Pbar)), "fe2_rve_average_stress")

    def rve_residual_norm(self, ids, out):
        a, p = _ids(ids)
        self._check(self.lib.fe2_rve_residual_norm(self.h, len(a), p, _ptr(out)), "fe2_rve_residual_norm")

    def sync(self):
        self._check(self.lib.fe2_sync(self.h), "fe2_sync")

    def launch_count(self):
        return int(self.lib.fe2_launch_count(self.h))

    def profile(self, enable=True):
        self._check(self.lib.fe2_profile(self.h, 1 if enable else 0), "fe2_profile")

    def profile_read(self):
        """{kernel name: (total ms, launches)} since profiling was enabled."""
        n = self.lib.fe2_profile_read(self.h, 0, None, None, None)
        names = C.create_string_buffer(48 * max(n, 1))
        ms = np.zeros(max(n, 1))
        cnt = np.zeros(max(n, 1), dtype=np.int64)
        n = self.lib.fe2_profile_read(self.h, n, names, ms.ctypes.data_as(_DP),
                                      cnt.ctypes.data_as(C.POINTER(C.c_longlong)))
        out = {}
        for k in range(n):
            nm = names.raw[48 * k:48 * (k + 1)].split(b"\0")[0].decode()
            out[nm] = (float(ms[k]), int(cnt[k]))
        return out

    # -- diagnostics ---------------------------------------------------------------
    def export(self, rve_id, what, N):
        d = self.dim
        nm = d * (N ** d - 1)
        size = {0: nm * nm, 1: nm, 2: nm * d * d, 3: nm, 4: d ** 4 + d * d}[what]
        out = np.zeros(size)
        self._check(self.lib.fe2_rve_export(self.h, int(rve_id), int(what), out.ctypes.data_as(_DP)),
                    "fe2_rve_export")
        if what == 0:
            return out.reshape(nm, nm)
        if what == 2:
            return out.reshape(nm, d * d)
        return out

    def w_copy(self, ids, buf, to_buf):
        """Snapshot (to_buf) or restore w~ of the RVEs through buf [n, ld] (CUDA, f64)."""
        a, p = _ids(ids)
        self._check(self.lib.fe2_rve_w_copy(self.h, len(a), p, _ptr(buf), int(buf.shape[1]), 1 if to_buf else 0),
                    "fe2_rve_w_copy")

    def set_w(self, rve_id, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        self._check(self.lib.fe2_rve_set_w(self.h, int(rve_id), w.ctypes.data_as(_DP)), "fe2_rve_set_w")
