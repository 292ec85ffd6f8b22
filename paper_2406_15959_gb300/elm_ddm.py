"""Python binding of libelmddm (include/elm_ddm.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; PyTorch provides device
memory and the stream.  If the library cannot be loaded this module raises; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

(OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_OOM, ERR_NONFINITE, ERR_RANK, ERR_NOT_SPD, ERR_CAPACITY,
 ERR_NOCONV, ERR_TIMEOUT) = range(11)
ERROR_NAMES = {ERR_ARG: "ERR_ARG", ERR_STATE: "ERR_STATE", ERR_CUDA: "ERR_CUDA",
               ERR_OOM: "ERR_OOM", ERR_NONFINITE: "ERR_NONFINITE", ERR_RANK: "ERR_RANK",
               ERR_NOT_SPD: "ERR_NOT_SPD", ERR_CAPACITY: "ERR_CAPACITY", ERR_NOCONV: "ERR_NOCONV",
               ERR_TIMEOUT: "ERR_TIMEOUT"}

# Every symbol the header declares.
SYMBOLS = ("elm_ddm_setup", "elm_ddm_setup_flux", "elm_ddm_assemble", "elm_ddm_schur", "elm_ddm_solve",
           "elm_ddm_eval", "elm_ddm_export", "elm_ddm_check", "elm_ddm_get_info",
           "elm_ddm_profile", "elm_ddm_profile_report", "elm_ddm_destroy",
           "elm_ddm_last_error", "elm_ddm_chol_solve_noalloc", "elm_ddm_interface_order",
           "elm_ddm_profile_only", "elm_ddm_solve_cg", "elm_ddm_set_coefficient",
           "elm_ddm_solve_pcg", "elm_ddm_get_points", "elm_ddm_set_wait_limit",
           "elm_ddm_fp64_gemm", "elm_ddm_fp64_gemm_workspace", "elm_ddm_set_tuning", "elm_ddm_set_ridge",
           "elm_ddm_selftest")
SELFTEST_PIVOT_RCP = 0
TUNE_PANEL_CTAS, TUNE_UPD_GRID = 0, 1
GEMM_TILE32, GEMM_TILE64, GEMM_PERSISTENT, GEMM_FUSED_SPLIT, GEMM_FUSED_SPLIT_B, GEMM_PERSISTENT_WIDE = range(6)
BUF_K, BUF_A, BUF_D, BUF_M, BUF_L = range(5)
PTS_INTERIOR, PTS_BOUNDARY, PTS_INTERFACE, PTS_NORMALS = range(4)


class ElmDdmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int32), ("n_neurons", ctypes.c_int32),
                ("m_max", ctypes.c_int32), ("n_gamma", ctypes.c_int32),
                ("op", ctypes.c_int32), ("max_rhs", ctypes.c_int32), ("flags", ctypes.c_int32)]


class FluxRowsDesc(ctypes.Structure):
    """elm_ddm_flux_rows: explicit rows of A^s (cross points)."""
    _fields_ = [("n_flux", ctypes.c_int32), ("f_max", ctypes.c_int32), ("count", ctypes.c_void_p),
                ("row", ctypes.c_void_p), ("nrm", ctypes.c_void_p), ("fdof", ctypes.c_void_p)]


FLAG_FP64_SIMT = 1
FLAG_SCHUR_CG = 2
FLAG_DIRECT_ASSEMBLY = 4
FLAG_MIXED = 8
FLAG_NEURONS_PER_SUB = 16
FLAG_RIDGE = 32
FLAG_BLOCK_JACOBI = 64
OP_POISSON, OP_VARCOEF = 0, 1


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libelmddm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libelmddm.so not found at {path}")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.elm_ddm_setup.argtypes = [ctypes.POINTER(Desc), P, P, P, P, P, ctypes.POINTER(P)]
    lib.elm_ddm_setup_flux.argtypes = [ctypes.POINTER(Desc), P, P, P, P, ctypes.POINTER(FluxRowsDesc), P,
                                       ctypes.POINTER(P)]
    lib.elm_ddm_assemble.argtypes = [P, P, P]
    lib.elm_ddm_schur.argtypes = [P]
    lib.elm_ddm_solve.argtypes = [P, P, I, P, P]
    lib.elm_ddm_eval.argtypes = [P, I, P, P, P, P, P]
    lib.elm_ddm_export.argtypes = [P, I, I, P, I]
    lib.elm_ddm_check.argtypes = [P]
    lib.elm_ddm_interface_order.argtypes = [P, P]
    lib.elm_ddm_profile.argtypes = [P, I]
    lib.elm_ddm_set_coefficient.argtypes = [P, P]
    lib.elm_ddm_solve_cg.argtypes = [P, P, I, ctypes.c_double, I, P, P, ctypes.POINTER(I)]
    lib.elm_ddm_solve_pcg.argtypes = [P, P, I, P, I, ctypes.c_double, I, P, P, ctypes.POINTER(I)]
    lib.elm_ddm_profile_only.argtypes = [P, ctypes.c_char_p]
    lib.elm_ddm_profile_report.argtypes = [P, ctypes.c_char_p, I]
    lib.elm_ddm_get_info.argtypes = [P, I, D]
    lib.elm_ddm_get_points.argtypes = [P, I, P, P]
    lib.elm_ddm_set_wait_limit.argtypes = [P, ctypes.c_double, I]
    lib.elm_ddm_set_tuning.argtypes = [P, I, I]
    lib.elm_ddm_set_ridge.argtypes = [P, ctypes.c_double]
    LL = ctypes.c_longlong
    lib.elm_ddm_fp64_gemm_workspace.argtypes = [I, I, I, I]
    lib.elm_ddm_fp64_gemm_workspace.restype = ctypes.c_size_t
    lib.elm_ddm_fp64_gemm.argtypes = [I, I, I, I, ctypes.c_double, P, LL, LL, P, LL, LL, ctypes.c_double,
                                      P, LL, LL, P, ctypes.c_size_t, P]
    lib.elm_ddm_selftest.argtypes = [I, P, P, I, P]
    lib.elm_ddm_destroy.argtypes = [P]
    lib.elm_ddm_last_error.argtypes = [P]
    lib.elm_ddm_last_error.restype = ctypes.c_char_p
    for name in SYMBOLS:
        if name not in ("elm_ddm_last_error", "elm_ddm_fp64_gemm_workspace"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(t) -> int:
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


@dataclass
class GeometryArrays:
    counts: np.ndarray   # int32 [N, 3]
    xy: np.ndarray       # float64 [N, m_max, 2]
    nrm: np.ndarray      # float64 [N, m_max, 2]
    dof: np.ndarray      # int32 [N, m_max]
    n_gamma: int
    flux: object = None  # workload.FluxRows (explicit A-rows at cross points) or None

    @classmethod
    def from_geometry(cls, g):
        f = getattr(g, "flux", None)
        if f is not None:
            f = type(f)(int(f.n_flux), np.ascontiguousarray(f.count, np.int32), np.ascontiguousarray(f.row, np.int32),
                        np.ascontiguousarray(f.nrm, np.float64), np.ascontiguousarray(f.fdof, np.int32))
        return cls(np.ascontiguousarray(g.counts, np.int32), np.ascontiguousarray(g.xy, np.float64),
                   np.ascontiguousarray(g.nrm, np.float64), np.ascontiguousarray(g.dof, np.int32),
                   int(g.n_gamma), f)


class Solver:
    """One decomposition on one GPU: setup -> assemble(theta) -> schur() -> solve(rhs)."""

    def __init__(self, geom, n_neurons: int, max_rhs: int = 1, stream=None, fp64_simt: bool = False,
                 schur_cg: bool = False, op: int = OP_POISSON, direct_assembly: bool = False,
                 mixed: bool = False, neurons=None, ridge: float | None = None,
                 block_jacobi: bool = False):
        """neurons: None (n_neurons in every subdomain) or int [N] per-subdomain counts <= n_neurons
        (ELM_DDM_FLAG_NEURONS_PER_SUB).  ridge: None, or alpha of ELM_DDM_FLAG_RIDGE.
        block_jacobi: ELM_DDM_FLAG_BLOCK_JACOBI (the per-edge block preconditioner of solve_cg)."""
        import torch
        self.lib = load()
        ga = geom if isinstance(geom, GeometryArrays) else GeometryArrays.from_geometry(geom)
        N, m_max = ga.xy.shape[0], ga.xy.shape[1]
        self.N, self.n, self.m_max, self.n_gamma = N, int(n_neurons), m_max, ga.n_gamma
        self.max_rhs = max_rhs
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        flags = ((FLAG_FP64_SIMT if fp64_simt else 0) | (FLAG_SCHUR_CG if schur_cg else 0) |
                 (FLAG_DIRECT_ASSEMBLY if direct_assembly else 0) | (FLAG_MIXED if mixed else 0) |
                 (FLAG_NEURONS_PER_SUB if neurons is not None else 0) |
                 (FLAG_RIDGE if ridge is not None else 0) | (FLAG_BLOCK_JACOBI if block_jacobi else 0))
        desc = Desc(N, self.n, m_max, ga.n_gamma, op, max_rhs, flags)
        h = ctypes.c_void_p()
        self._keep = ga
        counts = ga.counts
        if neurons is not None:
            counts = np.ascontiguousarray(np.concatenate([ga.counts, np.asarray(neurons, np.int32)[:, None]], 1),
                                          np.int32)
        self._counts_arg = counts
        if ga.flux is None:
            rc = self.lib.elm_ddm_setup(ctypes.byref(desc), counts.ctypes.data, ga.xy.ctypes.data,
                                        ga.nrm.ctypes.data, ga.dof.ctypes.data,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        else:
            f = ga.flux
            fd = FluxRowsDesc(int(f.n_flux), int(f.row.shape[1]), f.count.ctypes.data, f.row.ctypes.data,
                              f.nrm.ctypes.data, f.fdof.ctypes.data)
            rc = self.lib.elm_ddm_setup_flux(ctypes.byref(desc), counts.ctypes.data, ga.xy.ctypes.data,
                                             ga.nrm.ctypes.data, ga.dof.ctypes.data, ctypes.byref(fd),
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != OK:
            raise ElmDdmError(rc, self.lib.elm_ddm_last_error(None).decode())
        self.h = h
        self.ridge = ridge
        if ridge is not None:
            self._check_rc(self.lib.elm_ddm_set_ridge(self.h, float(ridge)))

    # -- helpers
    def _check_rc(self, rc):
        if rc != OK:
            raise ElmDdmError(rc, self.lib.elm_ddm_last_error(self.h).decode())

    def info(self, key: int) -> float:
        v = ctypes.c_double()
        self._check_rc(self.lib.elm_ddm_get_info(self.h, key, ctypes.byref(v)))
        return v.value

    @property
    def launches(self) -> int:
        return int(self.info(2))

    @property
    def kernels_launched(self) -> int:
        """CUDA kernels the library has launched in this process."""
        return int(self.info(7))

    @property
    def workspace_bytes(self) -> int:
        return int(self.info(1))

    # -- Algorithm 1
    def assemble(self, W, b):
        self._check_rc(self.lib.elm_ddm_assemble(self.h, _ptr(W), _ptr(b)))

    def set_coefficient(self, coef_rows):
        """ELM_DDM_OP_VARCOEF: (rho, d rho/dx, d rho/dy) per row, CUDA float64 [N, m_max, 3]."""
        self._check_rc(self.lib.elm_ddm_set_coefficient(self.h, _ptr(coef_rows.contiguous())))

    def schur(self):
        self._check_rc(self.lib.elm_ddm_schur(self.h))

    def solve(self, rhs, u_gamma=None, c=None):
        """rhs: CUDA float64 [nrhs, N, m_max] or [N, m_max].  Returns (u_gamma, c)."""
        import torch
        squeeze = rhs.dim() == 2
        r = rhs.unsqueeze(0) if squeeze else rhs
        nrhs = r.shape[0]
        if c is None:
            c = torch.empty((nrhs, self.N, self.n), dtype=torch.float64, device=rhs.device)
        if u_gamma is None and self.n_gamma > 0:
            u_gamma = torch.empty((nrhs, self.n_gamma), dtype=torch.float64, device=rhs.device)
        self._check_rc(self.lib.elm_ddm_solve(self.h, _ptr(r.contiguous()), nrhs,
                                              _ptr(u_gamma) if self.n_gamma > 0 else None, _ptr(c)))
        if squeeze:
            return (u_gamma[0] if u_gamma is not None else None), c[0]
        return u_gamma, c

    def solve_cg(self, rhs, tol: float = 1e-9, maxit: int = 10000, u_gamma=None, c=None,
                 require_convergence: bool = True, x0=None, jacobi=False):
        """As solve(), with the interface system solved by CG to relative residual tol
        (from x0 [nrhs, n_gamma] if given; jacobi: False / True (diagonal) / "block" (the
        per-edge blocks, needs block_jacobi=True at construction)).
        Returns (u_gamma, c, iterations)."""
        import torch
        squeeze = rhs.dim() == 2
        r = rhs.unsqueeze(0) if squeeze else rhs
        nrhs = r.shape[0]
        if c is None:
            c = torch.empty((nrhs, self.N, self.n), dtype=torch.float64, device=rhs.device)
        if u_gamma is None and self.n_gamma > 0:
            u_gamma = torch.empty((nrhs, self.n_gamma), dtype=torch.float64, device=rhs.device)
        it = ctypes.c_int(0)
        x0p = None
        if x0 is not None:
            x0 = (x0.unsqueeze(0) if x0.dim() == 1 else x0).contiguous()
            x0p = _ptr(x0)
        ugp = _ptr(u_gamma) if self.n_gamma > 0 else None
        if x0p is None and not jacobi:  # the paper's plain CG from zero
            rc = self.lib.elm_ddm_solve_cg(self.h, _ptr(r.contiguous()), nrhs, float(tol), int(maxit), ugp,
                                           _ptr(c), ctypes.byref(it))
        else:
            prec = 2 if jacobi == "block" else int(bool(jacobi))
            rc = self.lib.elm_ddm_solve_pcg(self.h, _ptr(r.contiguous()), nrhs, x0p, prec,
                                            float(tol), int(maxit), ugp, _ptr(c), ctypes.byref(it))
        if rc != ERR_NOCONV or require_convergence:
            self._check_rc(rc)
        if squeeze:
            return (u_gamma[0] if u_gamma is not None else None), c[0], it.value
        return u_gamma, c, it.value

    def eval(self, xy, owner, c, u=None, grad=None):
        import torch
        npts = xy.shape[0]
        if u is None:
            u = torch.empty(npts, dtype=torch.float64, device=xy.device)
        if grad is None:
            grad = torch.empty((npts, 2), dtype=torch.float64, device=xy.device)
        self._check_rc(self.lib.elm_ddm_eval(self.h, npts, _ptr(xy), _ptr(owner), _ptr(c), _ptr(u),
                                             _ptr(grad)))
        return u, grad

    def export(self, what: int, s: int = 0):
        """Copy of an internal matrix (BUF_*) as a CUDA tensor [rows, cols] (column-major
        data, returned transposed into row-major indexing)."""
        import torch
        rows, cols = self._export_shape(what, s)
        out = torch.empty((max(cols, 1), max(rows, 1)), dtype=torch.float64, device="cuda")
        self._check_rc(self.lib.elm_ddm_export(self.h, what, s, _ptr(out), max(rows, 1)))
        return out.t()[:rows, :cols]

    def _export_shape(self, what, s):
        mi, mb, mg = (int(v) for v in self._keep.counts[s])
        ns = int(self._counts_arg[s, 3]) if self._counts_arg.shape[1] == 4 else self.n
        pad = self.n - ns + (ns if self.ridge is not None else 0)
        if what == BUF_K:
            return mi + mb + mg + pad, self.n + mg
        mf = mg if self._keep.flux is None else int(self._keep.flux.count[s])   # rows of A^s
        if what == BUF_A:
            return mf, self.n
        if what == BUF_D:
            return mg, mg
        if what == BUF_M:
            return mf, mg
        if what == BUF_L:
            return self.n_gamma, self.n_gamma
        raise ValueError(what)

    def get_points(self, kind: int):
        """Points of one kind (PTS_*) as held by the handle: (CUDA float64 [N, kmax, 2],
        int32 counts [N])."""
        import torch
        counts = np.zeros(self.N, np.int32)
        self._check_rc(self.lib.elm_ddm_get_points(self.h, kind, None, counts.ctypes.data))
        kmax = int(counts.max()) if self.N else 0
        out = torch.empty((self.N, max(kmax, 1), 2), dtype=torch.float64, device="cuda")
        self._check_rc(self.lib.elm_ddm_get_points(self.h, kind, _ptr(out), None))
        return out[:, :kmax], counts

    def set_wait_limit(self, seconds: float = 2.0, hold_release: bool = False):
        """Limit of the device-side waits of the triangular solves (hold_release: test hook
        that makes them run out)."""
        self._check_rc(self.lib.elm_ddm_set_wait_limit(self.h, float(seconds), int(hold_release)))

    def set_tuning(self, panel_ctas: int | None = None, upd_grid: int | None = None):
        """Tile choices (elm_ddm_set_tuning): panel CTAs per subdomain (0, 4, 8) and the grid cap
        of the persistent products (0 = one CTA per SM)."""
        if panel_ctas is not None:
            self._check_rc(self.lib.elm_ddm_set_tuning(self.h, TUNE_PANEL_CTAS, int(panel_ctas)))
        if upd_grid is not None:
            self._check_rc(self.lib.elm_ddm_set_tuning(self.h, TUNE_UPD_GRID, int(upd_grid)))

    @property
    def refinement(self) -> dict:
        """Mixed-precision mode: steps, fallback and last relative correction of the last solve."""
        return {"steps": int(self.info(10)), "fell_back": bool(self.info(11)), "eta": self.info(12),
                "low_precision_factor": bool(self.info(13))}

    @property
    def cooperative_solves(self) -> bool:
        return self.info(9) == 1.0

    def interface_order(self) -> np.ndarray:
        """Internal index of every interface unknown (the order of BUF_L's rows)."""
        order = np.zeros(max(self.n_gamma, 1), np.int32)
        self._check_rc(self.lib.elm_ddm_interface_order(self.h, order.ctypes.data))
        return order[:self.n_gamma]

    def profile(self, enable: bool = True, only: str | None = None):
        """Per-launch event timing on (optionally of one kernel class only) or off."""
        self._check_rc(self.lib.elm_ddm_profile_only(self.h, only.encode() if only else None))
        self._check_rc(self.lib.elm_ddm_profile(self.h, int(enable)))

    def profile_report(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check_rc(self.lib.elm_ddm_profile_report(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def check(self):
        self._check_rc(self.lib.elm_ddm_check(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.elm_ddm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fp64_gemm(A, B, C, alpha: float = 1.0, beta: float = 0.0, kernel: int = GEMM_TILE32, stream=None):
    """C = alpha A B^T + beta C with the library's FP64-accurate tensor-core product
    (elm_ddm_fp64_gemm); A [M, K], B [N, K], C [M, N] CUDA float64 tensors of any strides.
    Returns C."""
    import torch
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    ws_bytes = lib.elm_ddm_fp64_gemm_workspace(kernel, M, N, K)
    if ws_bytes == 0:
        raise ElmDdmError(ERR_ARG, f"unsupported shape {M}x{N}x{K} for kernel {kernel}")
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device=A.device)
    base = (ws.data_ptr() + 255) // 256 * 256
    st = (stream or torch.cuda.current_stream(A.device)).cuda_stream
    rc = lib.elm_ddm_fp64_gemm(kernel, M, N, K, float(alpha), A.data_ptr(), A.stride(0), A.stride(1),
                               B.data_ptr(), B.stride(0), B.stride(1), float(beta), C.data_ptr(),
                               C.stride(0), C.stride(1), base, ws_bytes, st)
    if rc != OK:
        raise ElmDdmError(rc, "elm_ddm_fp64_gemm")
    return C


def selftest(which: int, x, stream=None):
    """y = f(x) elementwise for the device routine `which` (elm_ddm_selftest); x a CUDA
    float64 tensor.  Returns y."""
    import torch
    lib = load()
    x = x.contiguous()
    y = torch.empty_like(x)
    st = (stream or torch.cuda.current_stream(x.device)).cuda_stream
    rc = lib.elm_ddm_selftest(which, x.data_ptr(), y.data_ptr(), x.numel(), st)
    if rc != OK:
        raise ElmDdmError(rc, "elm_ddm_selftest")
    return y


def run_workload(w, device="cuda", max_rhs=1):
    """Convenience: full solve of a :class:`workload.Workload` on the GPU.
    Returns dict with u_gamma, c, u and grad at the test points (torch CUDA tensors)."""
    import torch
    dev = torch.device(device)
    coef = getattr(w, "coef_rows", None)
    s = Solver(w.geom, w.n_neurons, max_rhs=max_rhs, op=OP_VARCOEF if coef is not None else OP_POISSON)
    if coef is not None:
        s.set_coefficient(torch.as_tensor(coef, device=dev))
    W = torch.as_tensor(w.W, device=dev).contiguous()
    b = torch.as_tensor(w.b, device=dev).contiguous()
    rhs = torch.as_tensor(w.rhs, device=dev).contiguous()
    txy = torch.as_tensor(w.test_xy, device=dev).contiguous()
    own = torch.as_tensor(w.test_owner, device=dev).contiguous()
    s.assemble(W, b)
    s.schur()
    ug, c = s.solve(rhs)
    u, g = s.eval(txy, own, c)
    s.check()
    out = {"u_gamma": ug, "c": c, "u": u, "grad": g, "solver": s}
    return out


def _main(argv=None):
    """python -m paper_2406_15959_gb300.elm_ddm WORKLOAD [SOLVES] [--fp64-simt]

    Runs SOLVES full solves (setup once, then assemble + schur + solve + eval) of a named
    workload from workload.WORKLOADS on cuda:0 and prints the time of the last one."""
    import sys
    import time
    import torch
    from . import workload as wl
    args = list(sys.argv[1:] if argv is None else argv)
    simt = "--fp64-simt" in args
    args = [a for a in args if a != "--fp64-simt"]
    name = args[0] if args else "poisson_2x2_n200"
    count = int(args[1]) if len(args) > 1 else 1
    w = wl.WORKLOADS[name]()
    dev = torch.device("cuda:0")
    coef = getattr(w, "coef_rows", None)
    s = Solver(w.geom, w.n_neurons, fp64_simt=simt, op=OP_VARCOEF if coef is not None else OP_POISSON)
    if coef is not None:
        s.set_coefficient(torch.as_tensor(coef, device=dev))
    W = torch.as_tensor(w.W, device=dev)
    b = torch.as_tensor(w.b, device=dev)
    rhs = torch.as_tensor(w.rhs, device=dev)
    txy = torch.as_tensor(w.test_xy, device=dev)
    own = torch.as_tensor(w.test_owner, device=dev, dtype=torch.int32)
    for _ in range(count):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s.assemble(W, b)
        s.schur()
        _, c = s.solve(rhs)
        u, _ = s.eval(txy, own, c)
        s.check()
        dt = time.perf_counter() - t0
    print(f"{name}: {count} solve(s), last {1e3 * dt:.2f} ms, u[0] = {float(u[0]):.12e}")
    s.close()


if __name__ == "__main__":
    _main()
