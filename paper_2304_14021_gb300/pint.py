"""Thin ctypes binding of libpint (include/pint.h): argument marshalling only.

Every step of the solve runs in the CUDA kernels of libpint.  Tensors are
torch CUDA tensors (FP64, contiguous, layout [n][y][x]); PyTorch only provides
device memory and the stream.  There is no CPU fallback: if the shared library
is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libpint.so")

PINT_OK, PINT_EINVAL, PINT_ENOMEM, PINT_ECUDA, PINT_ENOCONV, PINT_EDIVERGED = 0, -1, -2, -3, -4, -5
BIHARMONIC, LINEAR_CH, CAHN_HILLIARD = 0, 1, 2
BC_SIMPLY_SUPPORTED, BC_NEUMANN = 0, 1
FP64, MIXED, MIXED_FF = 0, 1, 2
HIST_MAX = 256

EQUATIONS = {"biharmonic": BIHARMONIC, "linear_ch": LINEAR_CH, "cahn_hilliard": CAHN_HILLIARD,
             "cahn_hilliard_eyre": 3}
BCS = {"ss": BC_SIMPLY_SUPPORTED, "neumann": BC_NEUMANN, "neumann_v": 2}
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "mixed_ff": MIXED_FF}
PRECISION_NAMES = {v: k for k, v in PRECISIONS.items()}


class Problem(C.Structure):
    _fields_ = [("equation", C.c_int), ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("bc", C.c_int),
                ("eps", C.c_double), ("beta", C.c_double), ("T", C.c_double), ("nt", C.c_int),
                ("n_windows", C.c_int), ("theta", C.c_double), ("alpha", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int), ("precision", C.c_int), ("init_guess", C.c_int), ("tol_update", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("windows", C.c_int), ("iters_last", C.c_int),
                ("rel_residual", C.c_double), ("contraction", C.c_double), ("jbar", C.c_double),
                ("hist", C.c_double * HIST_MAX), ("segments", C.c_int), ("nt_min", C.c_int),
                ("retries", C.c_int), ("update_norm", C.c_double), ("precision", C.c_int), ("time_gemm", C.c_int),
                ("fused_spatial", C.c_int), ("tune_cached", C.c_int)]

    def as_dict(self) -> dict:
        return {"status": self.status, "iters": self.iters, "windows": self.windows,
                "iters_last": self.iters_last, "rel_residual": self.rel_residual,
                "contraction": self.contraction, "jbar": self.jbar, "segments": self.segments,
                "nt_min": self.nt_min, "retries": self.retries, "update_norm": self.update_norm,
                "precision": PRECISION_NAMES.get(self.precision, self.precision), "time_gemm": self.time_gemm,
                "fused_spatial": self.fused_spatial, "tune_cached": self.tune_cached,
                "hist": [self.hist[i] for i in range(min(self.iters_last + 1, HIST_MAX))]}


class TuneEntry(C.Structure):
    _fields_ = [("time_fwd_gemm", C.c_int), ("time_inv_gemm", C.c_int), ("fused_spatial", C.c_int),
                ("ms", C.c_float)]


NPHASE = 8
PHASES = ["residual", "check", "time_fwd", "spatial0", "spatial1", "spatial2", "time_inv", "setup"]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * NPHASE), ("launches", C.c_longlong * NPHASE)]


class PintError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def lib() -> C.CDLL:
    """Load libpint.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libpint.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.pint_create.argtypes = [C.POINTER(Problem), vp, C.POINTER(vp)]
        L.pint_create.restype = C.c_int
        L.pint_invariants.argtypes = [vp, dp, dp, C.c_longlong]
        L.pint_invariants.restype = C.c_int
        L.pint_footprint.argtypes = [C.POINTER(Problem)]
        L.pint_footprint.restype = C.c_longlong
        L.pint_solve.argtypes = [vp, vp, vp, C.POINTER(Stats)]
        L.pint_solve.restype = C.c_int
        L.pint_solve_host.argtypes = [vp, vp, vp, C.POINTER(Stats)]
        L.pint_solve_host.restype = C.c_int
        L.pint_residual.argtypes = [vp, vp, vp, vp, dp]
        L.pint_residual.restype = C.c_int
        L.pint_precond_apply.argtypes = [vp, C.c_double, vp, vp]
        L.pint_precond_apply.restype = C.c_int
        L.pint_profile_enable.argtypes = [vp, C.c_int]
        L.pint_profile_enable.restype = C.c_int
        L.pint_profile_read.argtypes = [vp, C.POINTER(Profile), C.c_int]
        L.pint_profile_read.restype = C.c_int
        L.pint_set_option.argtypes = [vp, C.c_int, C.c_longlong]
        L.pint_set_option.restype = C.c_int
        L.pint_residual_static.argtypes = [C.POINTER(Problem), vp, vp, vp, vp, vp]
        L.pint_residual_static.restype = C.c_int
        L.pint_solve_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(Stats),
                                       C.POINTER(C.c_int)]
        L.pint_solve_batch.restype = C.c_int
        L.pint_tune_lookup.argtypes = [C.POINTER(Problem), C.POINTER(TuneEntry)]
        L.pint_tune_lookup.restype = C.c_int
        L.pint_tune_load.argtypes = [C.c_char_p]
        L.pint_tune_load.restype = C.c_int
        L.pint_tune_save.argtypes = [C.c_char_p]
        L.pint_tune_save.restype = C.c_int
        L.pint_tune_clear.argtypes = []
        L.pint_tune_clear.restype = None
        L.pint_destroy.argtypes = [vp]
        L.pint_destroy.restype = None
        L.pint_strerror.argtypes = [C.c_int]
        L.pint_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().pint_strerror(code).decode()
    except OSError:
        return f"pint error {code}"


def make_problem(equation="biharmonic", dim=1, nx=64, ny=1, bc="ss", eps=1.0, beta=0.0, T=0.01, nt=32,
                 n_windows=1, theta=1.0, alpha=1e-2, tol=1e-10, max_iter=100, precision="fp64",
                 init_guess=0, tol_update=0.0) -> Problem:
    eq = EQUATIONS.get(equation, equation)
    b = BCS.get(bc, bc)
    pr = PRECISIONS.get(precision, precision)
    return Problem(int(eq), int(dim), int(nx), int(ny if dim == 2 else 1), int(b), float(eps), float(beta),
                   float(T), int(nt), int(n_windows), float(theta), float(alpha), float(tol), int(max_iter),
                   int(pr), int(init_guess), float(tol_update))


def footprint(**kw) -> int:
    p = make_problem(**kw)
    return int(lib().pint_footprint(C.byref(p)))


def tune_lookup(**kw):
    """The autotuner's entry for this problem's shape, or None (pint_tune_lookup)."""
    p = make_problem(**kw)
    e = TuneEntry()
    rc = lib().pint_tune_lookup(C.byref(p), C.byref(e))
    if rc < 0:
        raise PintError(rc, "pint_tune_lookup")
    if rc == 0:
        return None
    return {"time_fwd_gemm": e.time_fwd_gemm, "time_inv_gemm": e.time_inv_gemm, "fused_spatial": e.fused_spatial,
            "ms": e.ms}


def tune_load(path: str) -> int:
    rc = lib().pint_tune_load(str(path).encode())
    if rc < 0:
        raise PintError(rc, "pint_tune_load")
    return rc


def tune_save(path: str) -> int:
    rc = lib().pint_tune_save(str(path).encode())
    if rc < 0:
        raise PintError(rc, "pint_tune_save")
    return rc


def tune_clear() -> None:
    lib().pint_tune_clear()


STATIC_SCRATCH_BYTES = 278528


def residual_static(u0, U, rel_res, r=None, stream=None, **problem) -> None:
    """pint_residual_static: residual and ||r||/||b|| without a handle and without
    allocating (scratch in a static device array).  rel_res: a float64 CUDA
    tensor with one element that receives the norm; asynchronous on `stream`."""
    import torch
    p = make_problem(**problem)
    if stream is None:
        stream = torch.cuda.current_stream()
    rc = lib().pint_residual_static(C.byref(p), C.c_void_p(stream.cuda_stream), C.c_void_p(_ptr(u0)),
                                    C.c_void_p(_ptr(U)), C.c_void_p(_ptr(r)) if r is not None else None,
                                    C.c_void_p(_ptr(rel_res)))
    if rc != PINT_OK:
        raise PintError(rc, "pint_residual_static")


def _ptr(t) -> int:
    if t is None:
        return None
    if not t.is_cuda or str(t.dtype) != "torch.float64" or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def solve_batch(solvers, u0s, Us) -> list[dict]:
    """pint_solve_batch over independent Solvers (give each its own stream to
    overlap them on the GPU).  Returns the per-instance stats (with "rc")."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s._h.value for s in solvers])
    a0 = (C.c_void_p * n)(*[_ptr(u) for u in u0s])
    aU = (C.c_void_p * n)(*[_ptr(U) for U in Us])
    st = (Stats * n)()
    rcs = (C.c_int * n)()
    lib().pint_solve_batch(hs, n, a0, aU, st, rcs)
    out = []
    for i in range(n):
        d = st[i].as_dict()
        d["rc"] = rcs[i]
        out.append(d)
    return out


class Solver:
    """One pint handle: pint_create / pint_solve / pint_residual /
    pint_precond_apply / pint_destroy."""

    def __init__(self, stream=None, **problem):
        import torch
        self.problem = make_problem(**problem)
        self.kw = dict(problem)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        rc = lib().pint_create(C.byref(self.problem), C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != PINT_OK:
            raise PintError(rc, "pint_create")
        self._h = h

    @property
    def nt(self) -> int:
        return self.problem.nt

    @property
    def nspace(self) -> int:
        return self.problem.nx * (self.problem.ny if self.problem.dim == 2 else 1)

    def solve(self, u0, U, check: bool = True) -> dict:
        st = Stats()
        rc = lib().pint_solve(self._h, C.c_void_p(_ptr(u0)), C.c_void_p(_ptr(U)), C.byref(st))
        if check and rc not in (PINT_OK,):
            raise PintError(rc, "pint_solve")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def solve_host(self, u0, U, check: bool = True) -> dict:
        """u0, U: numpy float64 arrays (C-contiguous) in host memory."""
        st = Stats()
        rc = lib().pint_solve_host(self._h, C.c_void_p(u0.ctypes.data), C.c_void_p(U.ctypes.data), C.byref(st))
        if check and rc != PINT_OK:
            raise PintError(rc, "pint_solve_host")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def residual(self, u0, U, r=None) -> float:
        rel = C.c_double(0.0)
        rc = lib().pint_residual(self._h, C.c_void_p(_ptr(u0)), C.c_void_p(_ptr(U)),
                                 C.c_void_p(_ptr(r)) if r is not None else None, C.byref(rel))
        if rc != PINT_OK:
            raise PintError(rc, "pint_residual")
        return rel.value

    def precond_apply(self, r, delta, jbar: float = 0.0) -> None:
        rc = lib().pint_precond_apply(self._h, C.c_double(jbar), C.c_void_p(_ptr(r)), C.c_void_p(_ptr(delta)))
        if rc != PINT_OK:
            raise PintError(rc, "pint_precond_apply")

    def set_graphs(self, on: bool = True) -> None:
        rc = lib().pint_set_option(self._h, 1, 1 if on else 0)
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def set_fused_spatial(self, on: bool = True) -> None:
        rc = lib().pint_set_option(self._h, 3, 1 if on else 0)
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def set_varying_jacobian(self, inner: int) -> None:
        """Space-varying averaged Jacobian in Step 2 (Cahn-Hilliard), inner GMRES length; 0 turns it off."""
        rc = lib().pint_set_option(self._h, 5, int(inner))
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def set_krylov(self, restart: int) -> None:
        """Outer flexible GMRES(restart) around the preconditioner (linear equations); 0 turns it off."""
        rc = lib().pint_set_option(self._h, 4, int(restart))
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def set_time_gemm(self, mode: int) -> None:
        """Steps 1 and 3 as tensor-core DFT products: -1 chosen by measurement, 0 FFT, 1 matrix products."""
        rc = lib().pint_set_option(self._h, 8, int(mode))
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def set_fx_residual(self, on: bool = True) -> None:
        """PINT_MIXED, linear equations: block fixed-point residual on the integer pipes (on) or FP64 kernel."""
        rc = lib().pint_set_option(self._h, 6, 1 if on else 0)
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def set_log_invariants(self, on: bool = True) -> None:
        """Record each time level's mass and discrete energy during pint_solve (read with invariants())."""
        rc = lib().pint_set_option(self._h, 7, 1 if on else 0)
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def invariants(self):
        """(mass, energy) numpy arrays over all time levels of the last solve (pint_invariants)."""
        import numpy as np
        n = lib().pint_invariants(self._h, None, None, 0)
        if n < 0:
            raise PintError(n, "pint_invariants")
        m, e = np.zeros(n), np.zeros(n)
        rc = lib().pint_invariants(self._h, m.ctypes.data_as(C.POINTER(C.c_double)),
                                   e.ctypes.data_as(C.POINTER(C.c_double)), n)
        if rc < 0:
            raise PintError(rc, "pint_invariants")
        return m, e

    def set_adaptive_windows(self, on: bool = True) -> None:
        rc = lib().pint_set_option(self._h, 2, 1 if on else 0)
        if rc != PINT_OK:
            raise PintError(rc, "pint_set_option")

    def profile_enable(self, on=True) -> None:
        """on: False/0 off, True/1 every phase, 2 coarse (residual + check, whole Steps 1-3)."""
        mode = 2 if on == 2 else (1 if on else 0)
        rc = lib().pint_profile_enable(self._h, mode)
        if rc != PINT_OK:
            raise PintError(rc, "pint_profile_enable")

    def profile_read(self, reset: bool = False) -> dict:
        pr = Profile()
        rc = lib().pint_profile_read(self._h, C.byref(pr), 1 if reset else 0)
        if rc != PINT_OK:
            raise PintError(rc, "pint_profile_read")
        return {name: {"ms": pr.ms[i], "launches": int(pr.launches[i])} for i, name in enumerate(PHASES)}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().pint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
