"""ctypes binding of libwdb (include/wdb.h). Argument marshalling only: every step of the
computation runs in the library's CUDA kernels.

Device buffers are torch tensors (float32, contiguous, on the current CUDA device); the
stream is torch's current stream. The library must have been built
(``python -m paper_1512_08401_gb300.build`` or ``__graft_entry__.build()``); there is no
fallback, and a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwdb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "wdb.h")

PRECOND = {"none": 0, "jacobi": 1, "spai": 2}
RULE = {"weighted": 0, "naive": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "NaN or Inf",
          5: "timeout", 6: "diverged", 7: "unsupported", 8: "I/O error", 9: "tile plan invariant broken"}


class WdbError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"libwdb: {STATUS.get(status, status)}: {detail}")
        self.status = status


class PlanSummary(C.Structure):
    _fields_ = [("items", C.c_int), ("pairs", C.c_int), ("batches", C.c_int), ("split_tiles", C.c_int),
                ("super_subbands", C.c_int), ("smem_bytes", C.c_int), ("macs", C.c_longlong), ("groups", C.c_int)]


class ThetaInfo(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_cols", C.c_int), ("levels", C.c_int), ("n_subbands", C.c_int),
                ("wavelet_taps", C.c_int), ("rule", C.c_int), ("K_requested", C.c_longlong),
                ("K_eff", C.c_longlong), ("n_taps", C.c_longlong), ("n_candidates", C.c_longlong),
                ("theta_max_abs", C.c_double), ("phase_table_len", C.c_int), ("build_ms", C.c_double),
                ("plan_tuned", C.c_int), ("plan_items", C.c_int * 2), ("plan_split_tiles", C.c_int * 2),
                ("plan_super_subbands", C.c_int * 2), ("plan_groups", C.c_int * 2),
                ("plan_smem_bytes", C.c_int * 2), ("plan_grid", C.c_int * 2)]


class VThetaInfo(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_cols", C.c_int), ("levels", C.c_int), ("n_subbands", C.c_int),
                ("rule", C.c_int), ("K_requested", C.c_longlong), ("K_eff", C.c_longlong), ("n_taps", C.c_longlong),
                ("n_candidates", C.c_longlong), ("candidate_slots", C.c_longlong), ("n_probes", C.c_int),
                ("n_classes", C.c_int), ("n_plan_rows", C.c_int), ("plan_taps", C.c_longlong * 2),
                ("theta_max_abs", C.c_double), ("build_ms", C.c_double)]


class SolveParams(C.Structure):
    _fields_ = [("lam", C.c_double), ("w_subband_host", C.POINTER(C.c_double)), ("max_iters", C.c_int),
                ("tol", C.c_double), ("precond", C.c_int), ("jacobi_eps", C.c_double),
                ("check_every", C.c_int), ("x_init_dev", C.c_void_p), ("no_graph", C.c_int),
                ("target_objective", C.c_double), ("time_kernels", C.c_int), ("kkt_check", C.c_int),
                ("ista", C.c_int), ("fused", C.c_int), ("spin_limit", C.c_longlong)]


class SolveResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("objective", C.c_double), ("primal", C.c_double), ("gap", C.c_double),
                ("rel_gap", C.c_double), ("support", C.c_longlong), ("tau", C.c_double),
                ("L_hat", C.c_double), ("solve_ms", C.c_double), ("ms_k1", C.c_double), ("ms_k2", C.c_double),
                ("timed_chunks", C.c_int), ("first_primal_below", C.c_int), ("status", C.c_int),
                ("kkt_off", C.c_double), ("kkt_on", C.c_double), ("gap64", C.c_double), ("rel_gap64", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KktResult(C.Structure):
    _fields_ = [("objective", C.c_double), ("gap", C.c_double), ("rel_gap", C.c_double), ("kkt_off", C.c_double),
                ("kkt_on", C.c_double), ("gmax", C.c_double), ("support", C.c_longlong)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_longlong, C.c_double
pd = C.POINTER(C.c_double)
pi = C.POINTER(C.c_int)

_SIGS = {
    "wdb_build_theta": (i32, [pd, i32, i32, i32, i32, C.c_char_p, i32, i64, i32, vp, C.POINTER(vp)]),
    "wdb_theta_from_taps": (i32, [i32, i32, C.c_char_p, i32, i64, pi, pi, pi, pi, pd, vp, C.POINTER(vp)]),
    "wdb_theta_info_get": (i32, [vp, C.POINTER(ThetaInfo)]),
    "wdb_theta_export_taps": (i32, [vp, i64, pi, pi, pi, pi, pd]),
    "wdb_theta_precond": (i32, [vp, i32, f64, vp, pd, pd, pd, pd, pd]),
    "wdb_theta_set_precond": (i32, [vp, i32, pd, f64]),
    "wdb_theta_save": (i32, [vp, C.c_char_p]),
    "wdb_theta_load": (i32, [C.c_char_p, vp, C.POINTER(vp)]),
    "wdb_theta_free": (None, [vp]),
    "wdb_theta_apply": (i32, [vp, vp, vp, i32, vp]),
    "wdb_theta_replan": (i32, [vp, i32, f64, f64, i32, vp]),
    "wdb_tile_plan_check": (i32, [i32, i32, i32, i64, pi, pi, pi, pi, pd, i32, i32, i32, f64, f64, i32, i32,
                                  C.POINTER(PlanSummary)]),
    "wdb_solve": (i32, [vp, vp, vp, C.POINTER(SolveParams), vp, C.POINTER(SolveResult)]),
    "wdb_solve_coeffs": (i32, [vp, vp, vp, C.POINTER(SolveParams), vp, C.POINTER(SolveResult)]),
    "wdb_theta_objective": (i32, [vp, vp, vp, f64, pd, vp, pd]),
    "wdb_theta_kkt": (i32, [vp, vp, vp, f64, pd, vp, C.POINTER(KktResult)]),
    "wdb_solve_batch": (i32, [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(SolveParams), vp,
                              C.POINTER(SolveResult)]),
    "wdb_fftop_create": (i32, [pd, i32, i32, i32, i32, C.c_char_p, i32, vp, C.POINTER(vp)]),
    "wdb_fftop_free": (None, [vp]),
    "wdb_fftop_objective": (i32, [vp, vp, vp, f64, pd, vp, pd]),
    "wdb_fftop_precond": (i32, [vp, i32, f64, vp, pd, pd, pd]),
    "wdb_fftop_set_precond": (i32, [vp, i32, pd, f64]),
    "wdb_solve_fft": (i32, [vp, vp, vp, C.POINTER(SolveParams), vp, C.POINTER(SolveResult)]),
    "wdb_vtheta_build": (i32, [pd, i32, i32, i32, i32, C.c_char_p, i32, i64, i32, vp, C.POINTER(vp)]),
    "wdb_vtheta_from_taps": (i32, [i32, i32, C.c_char_p, i32, i64, pi, pi, pi, pi, pi, pd, vp, C.POINTER(vp)]),
    "wdb_vtheta_info_get": (i32, [vp, C.POINTER(VThetaInfo)]),
    "wdb_vtheta_export_taps": (i32, [vp, i64, pi, pi, pi, pi, pi, pd]),
    "wdb_vtheta_apply": (i32, [vp, vp, vp, i32, vp]),
    "wdb_vtheta_precond": (i32, [vp, i32, f64, vp, pd, pd, pd, pd, pd]),
    "wdb_vtheta_set_precond": (i32, [vp, i32, pd, f64]),
    "wdb_vtheta_solve": (i32, [vp, vp, vp, C.POINTER(SolveParams), vp, C.POINTER(SolveResult)]),
    "wdb_vtheta_solve_coeffs": (i32, [vp, vp, vp, C.POINTER(SolveParams), vp, C.POINTER(SolveResult)]),
    "wdb_vtheta_objective": (i32, [vp, vp, vp, f64, pd, vp, pd]),
    "wdb_vtheta_free": (None, [vp]),
    "wdb_vtheta_plan_check": (i32, [i32, i32, C.c_char_p, i32, i64, pi, pi, pi, pi, pi, pd, i32, pd, pd]),
    "wdb_dwt": (i32, [vp, vp, i32, i32, C.c_char_p, i32, vp]),
    "wdb_idwt": (i32, [vp, vp, i32, i32, C.c_char_p, i32, vp]),
    "wdb_dwt_noalloc": (i32, [vp, vp, i32, i32, C.c_char_p, i32, vp]),
    "wdb_wavelet_filters": (i32, [C.c_char_p, i32, pd, pd, pi]),
    "wdb_cnn_create": (i32, [i32, i32, i32, i32, i32, C.c_ulonglong, vp, C.POINTER(vp)]),
    "wdb_cnn_free": (None, [vp]),
    "wdb_cnn_num_params": (i64, [vp]),
    "wdb_cnn_set_params": (i32, [vp, C.POINTER(C.c_float), i64, vp]),
    "wdb_cnn_get_params": (i32, [vp, C.POINTER(C.c_float), i64]),
    "wdb_cnn_forward": (i32, [vp, vp, vp, i32, vp]),
    "wdb_cnn_loss_grad": (i32, [vp, vp, vp, i32, vp, pd, C.POINTER(C.c_float)]),
    "wdb_cnn_train_step": (i32, [vp, vp, vp, i32, f64, vp, pd]),
    "wdb_cnn_save": (i32, [vp, C.c_char_p]),
    "wdb_cnn_load": (i32, [C.c_char_p, vp, C.POINTER(vp)]),
    "wdb_solve_warm": (i32, [vp, vp, vp, vp, C.POINTER(SolveParams), vp, C.POINTER(SolveResult), pi]),
    "wdb_status_str": (C.c_char_p, [i32]),
    "wdb_last_error": (C.c_char_p, []),
    "wdb_kernel_launches": (i64, [i32]),
}


def header_functions() -> list[str]:
    """Names of the functions declared in include/wdb.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(wdb_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """Load libwdb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_1512_08401_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise WdbError(status, lib().wdb_last_error().decode())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dev(t, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(pd)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(pi)


def kernel_launches(reset: bool = False) -> int:
    return int(lib().wdb_kernel_launches(1 if reset else 0))


def wavelet_filters(name: str = "db4"):
    h = np.zeros(32)
    g = np.zeros(32)
    n = C.c_int()
    _check(lib().wdb_wavelet_filters(name.encode(), 32, h.ctypes.data_as(pd), g.ctypes.data_as(pd), C.byref(n)))
    return h[:n.value].copy(), g[:n.value].copy()


def make_params(lam=1e-3, max_iters=200, tol=0.0, precond="spai", jacobi_eps=0.0, check_every=10, x_init=None,
                w_subband=None, no_graph=False, target_objective=0.0, time_kernels=False, kkt_check=False,
                ista=False, fused=False, spin_limit=0):
    p = SolveParams()
    p.lam = float(lam)
    keep = None
    if w_subband is not None:
        keep = np.ascontiguousarray(w_subband, dtype=np.float64)
        p.w_subband_host = keep.ctypes.data_as(pd)
    p.max_iters = int(max_iters)
    p.tol = float(tol)
    p.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
    p.jacobi_eps = float(jacobi_eps)
    p.check_every = int(check_every)
    p.x_init_dev = None if x_init is None else _dev(x_init).value
    p.no_graph = 1 if no_graph else 0
    p.target_objective = float(target_objective)
    p.time_kernels = 1 if time_kernels else 0
    p.kkt_check = 1 if kkt_check else 0
    p.ista = 1 if ista else 0
    p.fused = 1 if fused else 0
    p.spin_limit = int(spin_limit)
    return p, keep


class Theta:
    """Theta_K handle (library-owned device memory)."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)
        self.info = self._info()

    @classmethod
    def build(cls, psf, n_rows, n_cols, wavelet="db4", levels=4, K=None, rule="weighted", stream=None):
        psf, pp = _f64(psf)
        kh, kw = psf.shape
        K = n_rows * n_cols * 30 if K is None else int(K)
        out = C.c_void_p()
        _check(lib().wdb_build_theta(pp, kh, kw, n_rows, n_cols, wavelet.encode(), levels, K,
                                     RULE[rule] if isinstance(rule, str) else int(rule), _stream(stream),
                                     C.byref(out)))
        return cls(out.value)

    @classmethod
    def from_taps(cls, n_rows, n_cols, wavelet, levels, a, b, oy, ox, v, stream=None):
        a, pa = _i32(a)
        b, pb = _i32(b)
        oy, py = _i32(oy)
        ox, px = _i32(ox)
        v, pv = _f64(v)
        out = C.c_void_p()
        _check(lib().wdb_theta_from_taps(n_rows, n_cols, wavelet.encode(), levels, len(v), pa, pb, py, px, pv,
                                         _stream(stream), C.byref(out)))
        return cls(out.value)

    @classmethod
    def load(cls, path, stream=None):
        out = C.c_void_p()
        _check(lib().wdb_theta_load(path.encode(), _stream(stream), C.byref(out)))
        return cls(out.value)

    def _info(self) -> ThetaInfo:
        i = ThetaInfo()
        _check(lib().wdb_theta_info_get(self._h, C.byref(i)))
        return i

    @property
    def N(self) -> int:
        return self.info.n_rows * self.info.n_cols

    def export_taps(self):
        n = self.info.n_taps
        a, b, oy, ox = (np.zeros(n, np.int32) for _ in range(4))
        v = np.zeros(n)
        _check(lib().wdb_theta_export_taps(self._h, n, a.ctypes.data_as(pi), b.ctypes.data_as(pi),
                                           oy.ctypes.data_as(pi), ox.ctypes.data_as(pi), v.ctypes.data_as(pd)))
        return a, b, oy, ox, v

    def precond(self, kind="spai", jacobi_eps=0.0, stream=None):
        n = self.info.phase_table_len
        P, Md, M2d = np.zeros(n), np.zeros(n), np.zeros(n)
        tau, L = C.c_double(), C.c_double()
        _check(lib().wdb_theta_precond(self._h, PRECOND[kind], jacobi_eps, _stream(stream), P.ctypes.data_as(pd),
                                       Md.ctypes.data_as(pd), M2d.ctypes.data_as(pd), C.byref(tau), C.byref(L)))
        return {"P": P, "Md": Md, "M2d": M2d, "tau": tau.value, "L_hat": L.value}

    def set_precond(self, kind, P, tau):
        P, pp = _f64(P)
        _check(lib().wdb_theta_set_precond(self._h, PRECOND[kind], pp, float(tau)))

    def save(self, path):
        _check(lib().wdb_theta_save(self._h, path.encode()))

    def replan(self, smem_budget=0, cap_share=0.0, split_share=0.0, super_tiles=False, grouped=False, stream=None):
        """Planner plans for the FP32 kernels in place of the autotuned ones (wdb_theta_replan);
        super_tiles: 2 x 2 super tiles where they fit; grouped: items over every subband of a level."""
        mode = 2 if grouped else (1 if super_tiles else 0)
        _check(lib().wdb_theta_replan(self._h, int(smem_budget), float(cap_share), float(split_share), mode,
                                      _stream(stream)))
        self.info = self._info()

    def apply(self, x, out, transpose=False, stream=None):
        _check(lib().wdb_theta_apply(self._h, _dev(x, self.N), _dev(out, self.N), 1 if transpose else 0,
                                     _stream(stream)))
        return out

    def solve(self, u, x, stream=None, **kw):
        p, _keep = make_params(**kw)
        r = SolveResult()
        _check(lib().wdb_solve(self._h, _dev(u, self.N), _dev(x, self.N), C.byref(p), _stream(stream), C.byref(r)))
        return r.as_dict()

    def solve_coeffs(self, x0, x, stream=None, **kw):
        p, _keep = make_params(**kw)
        r = SolveResult()
        _check(lib().wdb_solve_coeffs(self._h, _dev(x0, self.N), _dev(x, self.N), C.byref(p), _stream(stream),
                                      C.byref(r)))
        return r.as_dict()

    def objective(self, x, x0, lam=1e-3, w_subband=None, stream=None):
        E = C.c_double()
        w = None
        pw = None
        if w_subband is not None:
            w, pw = _f64(w_subband)
        _check(lib().wdb_theta_objective(self._h, _dev(x, self.N), _dev(x0, self.N), float(lam), pw,
                                         _stream(stream), C.byref(E)))
        return E.value

    def kkt(self, x, x0, lam=1e-3, w_subband=None, stream=None):
        """FP64 optimality check of x (wdb_theta_kkt): objective, gap, KKT residuals."""
        out = KktResult()
        pw = None
        if w_subband is not None:
            w, pw = _f64(w_subband)
        _check(lib().wdb_theta_kkt(self._h, _dev(x, self.N), _dev(x0, self.N), float(lam), pw, _stream(stream),
                                   C.byref(out)))
        return out.as_dict()

    def free(self):
        if self._h:
            lib().wdb_theta_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class VTheta:
    """Theta_K of a row-varying blur (wdb_vtheta_*): psfs[i] is the PSF of image row i."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)
        self.info = self._info()

    @classmethod
    def build(cls, psfs, n_rows, n_cols, wavelet="db4", levels=4, K=None, rule="weighted", stream=None):
        psfs, pp = _f64(psfs)
        if psfs.ndim != 3 or psfs.shape[0] != n_rows:
            raise ValueError("psfs must be [n_rows, kh, kw]")
        _, kh, kw = psfs.shape
        K = n_rows * n_cols * 30 if K is None else int(K)
        out = C.c_void_p()
        _check(lib().wdb_vtheta_build(pp, kh, kw, n_rows, n_cols, wavelet.encode(), levels, K,
                                      RULE[rule] if isinstance(rule, str) else int(rule), _stream(stream),
                                      C.byref(out)))
        return cls(out.value)

    @classmethod
    def from_taps(cls, n_rows, n_cols, wavelet, levels, a, py, b, qy, ox, v, stream=None):
        arrs = [_i32(z) for z in (a, py, b, qy, ox)]
        v, pv = _f64(v)
        out = C.c_void_p()
        _check(lib().wdb_vtheta_from_taps(n_rows, n_cols, wavelet.encode(), levels, len(v), *[p for _, p in arrs],
                                          pv, _stream(stream), C.byref(out)))
        return cls(out.value)

    def _info(self) -> VThetaInfo:
        i = VThetaInfo()
        _check(lib().wdb_vtheta_info_get(self._h, C.byref(i)))
        return i

    @property
    def N(self) -> int:
        return self.info.n_rows * self.info.n_cols

    def export_taps(self):
        n = self.info.n_taps
        a, py, b, qy, ox = (np.zeros(n, np.int32) for _ in range(5))
        v = np.zeros(n)
        _check(lib().wdb_vtheta_export_taps(self._h, n, *[z.ctypes.data_as(pi) for z in (a, py, b, qy, ox)],
                                            v.ctypes.data_as(pd)))
        return a, py, b, qy, ox, v

    def precond(self, kind="spai", jacobi_eps=0.0, stream=None):
        n = self.info.n_classes
        P, Md, M2d = np.zeros(n), np.zeros(n), np.zeros(n)
        tau, L = C.c_double(), C.c_double()
        _check(lib().wdb_vtheta_precond(self._h, PRECOND[kind], jacobi_eps, _stream(stream), P.ctypes.data_as(pd),
                                        Md.ctypes.data_as(pd), M2d.ctypes.data_as(pd), C.byref(tau), C.byref(L)))
        return {"P": P, "Md": Md, "M2d": M2d, "tau": tau.value, "L_hat": L.value}

    def set_precond(self, kind, P, tau):
        P, pp = _f64(P)
        _check(lib().wdb_vtheta_set_precond(self._h, PRECOND[kind], pp, float(tau)))

    def apply(self, x, out, transpose=False, stream=None):
        _check(lib().wdb_vtheta_apply(self._h, _dev(x, self.N), _dev(out, self.N), 1 if transpose else 0,
                                      _stream(stream)))
        return out

    def solve(self, u, x, stream=None, **kw):
        p, _keep = make_params(**kw)
        r = SolveResult()
        _check(lib().wdb_vtheta_solve(self._h, _dev(u, self.N), _dev(x, self.N), C.byref(p), _stream(stream),
                                      C.byref(r)))
        return r.as_dict()

    def solve_coeffs(self, x0, x, stream=None, **kw):
        p, _keep = make_params(**kw)
        r = SolveResult()
        _check(lib().wdb_vtheta_solve_coeffs(self._h, _dev(x0, self.N), _dev(x, self.N), C.byref(p),
                                             _stream(stream), C.byref(r)))
        return r.as_dict()

    def objective(self, x, x0, lam=1e-3, w_subband=None, stream=None):
        E = C.c_double()
        pw = None
        if w_subband is not None:
            w, pw = _f64(w_subband)
        _check(lib().wdb_vtheta_objective(self._h, _dev(x, self.N), _dev(x0, self.N), float(lam), pw,
                                          _stream(stream), C.byref(E)))
        return E.value

    def free(self):
        if self._h:
            lib().wdb_vtheta_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class FFTOp:
    """Exact operator H Psi for the FFT path."""

    def __init__(self, psf, n_rows, n_cols, wavelet="db4", levels=4, stream=None):
        psf, pp = _f64(psf)
        kh, kw = psf.shape
        out = C.c_void_p()
        _check(lib().wdb_fftop_create(pp, kh, kw, n_rows, n_cols, wavelet.encode(), levels, _stream(stream),
                                      C.byref(out)))
        self._h = out
        self.N = n_rows * n_cols
        self.n_subbands = 3 * levels + 1

    def precond(self, kind="spai", jacobi_eps=0.0, stream=None):
        P = np.zeros(self.n_subbands)
        tau, L = C.c_double(), C.c_double()
        _check(lib().wdb_fftop_precond(self._h, PRECOND[kind], jacobi_eps, _stream(stream), P.ctypes.data_as(pd),
                                       C.byref(tau), C.byref(L)))
        return {"P": P, "tau": tau.value, "L_hat": L.value}

    def set_precond(self, kind, P, tau):
        P, pp = _f64(P)
        _check(lib().wdb_fftop_set_precond(self._h, PRECOND[kind], pp, float(tau)))

    def objective(self, u, x, lam=1e-3, w_subband=None, stream=None):
        """Exact objective of the iterate x for the image u (wdb_fftop_objective)."""
        E = C.c_double()
        pw = None
        if w_subband is not None:
            w, pw = _f64(w_subband)
        _check(lib().wdb_fftop_objective(self._h, _dev(u, self.N), _dev(x, self.N), float(lam), pw, _stream(stream),
                                         C.byref(E)))
        return E.value

    def solve(self, u, x, stream=None, **kw):
        p, _keep = make_params(**kw)
        r = SolveResult()
        _check(lib().wdb_solve_fft(self._h, _dev(u, self.N), _dev(x, self.N), C.byref(p), _stream(stream),
                                   C.byref(r)))
        return r.as_dict()

    def free(self):
        if self._h:
            lib().wdb_fftop_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tile_plan_check(n_rows, n_cols, levels, a, b, oy, ox, v, transpose=False, esize=4, smem_budget=0,
                    cap_share=0.0, split_share=0.0, super_tiles=False, ctas=0, grouped=False):
    """Build one operator's tile plan for a tap list on the host and check its invariants
    (wdb_tile_plan_check); returns the plan summary as a dict, raises WdbError on a fault."""
    a, pa = _i32(a)
    b, pb = _i32(b)
    oy, py = _i32(oy)
    ox, px = _i32(ox)
    v, pv = _f64(v)
    sm = PlanSummary()
    _check(lib().wdb_tile_plan_check(n_rows, n_cols, levels, len(v), pa, pb, py, px, pv, 1 if transpose else 0,
                                      esize, smem_budget, cap_share, split_share,
                                      2 if grouped else (1 if super_tiles else 0), ctas, C.byref(sm)))
    return {f: getattr(sm, f) for f, _ in PlanSummary._fields_}


def vtheta_plan_check(n_rows, n_cols, wavelet, levels, a, py, b, qy, ox, v, x, transpose=False):
    """Host emulation of one row-plan application (wdb_vtheta_plan_check): returns y (FP64)."""
    arrs = [_i32(z) for z in (a, py, b, qy, ox)]
    v, pv = _f64(v)
    x, px = _f64(x)
    y = np.zeros(n_rows * n_cols)
    _check(lib().wdb_vtheta_plan_check(n_rows, n_cols, wavelet.encode(), levels, len(v), *[p for _, p in arrs], pv,
                                       1 if transpose else 0, px, y.ctypes.data_as(pd)))
    return y


def dwt(img, coef, n_rows, n_cols, wavelet="db4", levels=4, stream=None):
    _check(lib().wdb_dwt(_dev(img, n_rows * n_cols), _dev(coef, n_rows * n_cols), n_rows, n_cols,
                         wavelet.encode(), levels, _stream(stream)))
    return coef


def idwt(coef, img, n_rows, n_cols, wavelet="db4", levels=4, stream=None):
    _check(lib().wdb_idwt(_dev(coef, n_rows * n_cols), _dev(img, n_rows * n_cols), n_rows, n_cols,
                          wavelet.encode(), levels, _stream(stream)))
    return img


def dwt_noalloc(img, coef, n_rows, n_cols, wavelet="db4", levels=4, stream=None):
    """Forward transform without any device allocation (scratch in a static device array)."""
    _check(lib().wdb_dwt_noalloc(_dev(img, n_rows * n_cols), _dev(coef, n_rows * n_cols), n_rows, n_cols,
                                 wavelet.encode(), levels, _stream(stream)))
    return coef


def solve_batch(thetas, us, xs, params_list, stream=None):
    """Solve many problems together (one Theta handle per problem). params_list: dicts of
    make_params keyword arguments. Returns one result dict per problem."""
    B = len(thetas)
    TH = (C.c_void_p * B)(*[t._h.value for t in thetas])
    U = (C.c_void_p * B)(*[_dev(u, t.N).value for u, t in zip(us, thetas)])
    X = (C.c_void_p * B)(*[_dev(x, t.N).value for x, t in zip(xs, thetas)])
    keep = []
    P = (SolveParams * B)()
    for i, kw in enumerate(params_list):
        p, k = make_params(**kw)
        keep.append(k)
        P[i] = p
    R = (SolveResult * B)()
    _check(lib().wdb_solve_batch(B, TH, U, X, P, _stream(stream), R))
    return [R[i].as_dict() for i in range(B)]


class WarmStartNet:
    """The warm-start U-Net (wdb_cnn_*): images are [B, H, W] float32 CUDA tensors."""

    def __init__(self, levels=4, channels=32, height=128, width=128, max_batch=16, seed=0, stream=None,
                 _handle=None):
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            _check(lib().wdb_cnn_create(levels, channels, height, width, max_batch, seed, _stream(stream),
                                        C.byref(self._h)))
        self.levels, self.channels, self.height, self.width, self.max_batch = levels, channels, height, width, max_batch

    @classmethod
    def load(cls, path, stream=None):
        h = C.c_void_p()
        _check(lib().wdb_cnn_load(path.encode(), _stream(stream), C.byref(h)))
        with open(path, "rb") as f:
            hdr = np.frombuffer(f.read(8 + 7 * 8)[8:], dtype=np.int64)
        return cls(int(hdr[0]), int(hdr[1]), int(hdr[2]), int(hdr[3]), int(hdr[4]), _handle=h)

    @property
    def num_params(self) -> int:
        return int(lib().wdb_cnn_num_params(self._h))

    def set_params(self, flat, stream=None):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib().wdb_cnn_set_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size, _stream(stream)))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.num_params, dtype=np.float32)
        _check(lib().wdb_cnn_get_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))
        return a

    def _img(self, t):
        B = t.shape[0] if t.dim() == 3 else 1
        return _dev(t, B * self.height * self.width), B

    def forward(self, u, v, stream=None):
        pu, B = self._img(u)
        pv, _ = self._img(v)
        _check(lib().wdb_cnn_forward(self._h, pu, pv, B, _stream(stream)))
        return v

    def loss_grad(self, u, target, want_grad=True, stream=None):
        pu, B = self._img(u)
        pt, _ = self._img(target)
        loss = C.c_double()
        g = np.empty(self.num_params, dtype=np.float32) if want_grad else None
        gp = g.ctypes.data_as(C.POINTER(C.c_float)) if want_grad else None
        _check(lib().wdb_cnn_loss_grad(self._h, pu, pt, B, _stream(stream), C.byref(loss), gp))
        return loss.value, g

    def train_step(self, u, target, lr, stream=None):
        pu, B = self._img(u)
        pt, _ = self._img(target)
        loss = C.c_double()
        _check(lib().wdb_cnn_train_step(self._h, pu, pt, B, lr, _stream(stream), C.byref(loss)))
        return loss.value

    def solve_warm(self, theta, u, x, stream=None, **kw):
        """wdb_solve_warm: returns (result dict, start used: 1 network, 0 cold start x = 0)."""
        p, _keep = make_params(**kw)
        r = SolveResult()
        used = C.c_int()
        _check(lib().wdb_solve_warm(theta._h, self._h, _dev(u, theta.N), _dev(x, theta.N), C.byref(p),
                                    _stream(stream), C.byref(r), C.byref(used)))
        return r.as_dict(), int(used.value)

    def save(self, path):
        _check(lib().wdb_cnn_save(self._h, path.encode()))

    def free(self):
        if self._h:
            lib().wdb_cnn_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
