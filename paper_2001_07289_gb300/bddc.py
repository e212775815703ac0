"""Thin Python binding of the BDDC-SO C ABI (include/bddc_so.h).

Argument marshalling only: every step of setup, apply, PCG and gradient runs
in the CUDA library.  Vectors are torch float64 CUDA tensors in the node-grid
layout; the library is loaded from the in-tree build and importing this
module fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbddc_so.so")

BDDC_OK, BDDC_ERR_ARG, BDDC_ERR_NOT_SPD, BDDC_ERR_NOCONV = 0, -1, -2, -3
BDDC_ERR_BREAKDOWN, BDDC_ERR_CUDA, BDDC_ERR_OOM, BDDC_ERR_TIMEOUT, BDDC_ERR_UNSUPPORTED = -4, -5, -6, -7, -8
BDDC_FP64, BDDC_MIXED = 0, 1
BDDC_W_CARD, BDDC_W_RHO = 0, 1
BDDC_SEL_VEF, BDDC_SEL_VE, BDDC_SEL_VF, BDDC_SEL_V, BDDC_SEL_F, BDDC_SEL_EF = 0, 1, 2, 3, 4, 5
BDDC_DEBUG_CLEAR, BDDC_DEBUG_NEGATE_NEUMANN_PIVOT, BDDC_DEBUG_NEGATE_DIRICHLET_PIVOT, BDDC_DEBUG_WAIT_TRIES = 0, 1, 2, 3
SELECTIONS = {"vef": BDDC_SEL_VEF, "ve": BDDC_SEL_VE, "vf": BDDC_SEL_VF, "v": BDDC_SEL_V, "f": BDDC_SEL_F,
              "ef": BDDC_SEL_EF}
BDDC_BETA_STANDARD, BDDC_BETA_FLEXIBLE = 0, 1
BETA_RULES = {"standard": BDDC_BETA_STANDARD, "flexible": BDDC_BETA_FLEXIBLE}


class BddcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double)]


class Partition(C.Structure):
    _fields_ = [("ncut", C.c_int * 3), ("cut", C.POINTER(C.c_int) * 3), ("piece", C.POINTER(C.c_int))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("weights", C.c_int), ("L_elems", C.c_int),
                ("selection", C.c_int), ("use_graph", C.c_int), ("maxit", C.c_int), ("beta_rule", C.c_int),
                ("ml_block", C.c_int), ("ml_sub", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("r0_norm", C.c_double),
                ("r_norm", C.c_double), ("alphas", C.POINTER(C.c_double)),
                ("betas", C.POINTER(C.c_double)), ("capacity", C.c_int), ("solve_ms", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("n_coarse", C.c_int), ("n_vertices", C.c_int),
                ("max_local_coarse", C.c_int), ("n_free", C.c_longlong), ("bytes", C.c_longlong),
                ("factor_bytes", C.c_longlong), ("setup_ms", C.c_double), ("phase_ms", C.c_double * 6),
                ("launches", C.c_longlong), ("coarse_fma", C.c_double), ("local_factor_fma", C.c_double),
                ("apply_bytes", C.c_longlong), ("apply_cluster", C.c_int), ("local_band_flops", C.c_double),
                ("factor_kernel", C.c_int), ("factor_tc_subdomains", C.c_int), ("pinned_subdomains", C.c_int),
                ("n_buckets", C.c_int), ("bucket_subdomains", C.c_int * 2),
                ("bucket_ring", C.c_int * 2), ("bucket_ctas", C.c_int * 2), ("ml_blocks", C.c_int),
                ("ml_coarse2", C.c_int)]


class Analysis(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("n_coarse", C.c_int), ("n_vertices", C.c_int), ("n_edges", C.c_int),
                ("n_faces", C.c_int), ("max_local_coarse", C.c_int), ("n_fronts", C.c_int),
                ("n_levels", C.c_int), ("max_front", C.c_int), ("front_entries", C.c_longlong),
                ("coarse_fma", C.c_double), ("ml_blocks", C.c_int), ("ml_coarse2", C.c_int),
                ("ml_fronts2", C.c_int)]


class Paths(C.Structure):
    _fields_ = [("n_pieces", C.c_longlong), ("n_pairs", C.c_longlong), ("n_direct", C.c_longlong),
                ("n_without_path", C.c_longlong), ("min_ratio", C.c_double), ("worst_pair", C.c_longlong * 2)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"BDDC-SO CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    lib.bddc_setup.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), C.POINTER(Options), vp, vp,
                               C.POINTER(vp)]
    lib.bddc_apply.argtypes = [vp, vp, vp, vp]
    lib.bddc_apply_noalloc.argtypes = [vp, vp, vp, vp]
    lib.bddc_operator.argtypes = [vp, vp, vp, vp]
    lib.pcg_solve.argtypes = [vp, vp, vp, C.c_double, C.POINTER(Stats), vp]
    lib.bddc_gradient.argtypes = [vp, vp, vp, vp, vp]
    lib.bddc_solve_host.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), C.POINTER(Options), dp, dp, dp,
                                    C.c_double, C.POINTER(Stats)]
    lib.bddc_get_info.argtypes = [vp, C.POINTER(Info)]
    lib.bddc_set_apply_schedule.argtypes = [vp, C.c_int]
    lib.bddc_set_bucket_schedule.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    lib.bddc_analyze.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), C.POINTER(Options), C.POINTER(Analysis)]
    lib.bddc_acceptable_paths.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), C.POINTER(Options), dp,
                                          C.POINTER(Paths)]
    lib.bddc_get_coarse_basis.argtypes = [vp, ip, dp, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                          C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.bddc_get_coarse_matrix.argtypes = [vp, dp]
    lib.bddc_destroy.argtypes = [vp]
    lib.bddc_debug_inject.argtypes = [C.c_int, C.c_longlong]
    lib.bddc_last_error.argtypes = [vp]
    lib.bddc_last_error.restype = C.c_char_p
    for f in ("bddc_setup", "bddc_analyze", "bddc_acceptable_paths", "bddc_apply", "bddc_apply_noalloc", "bddc_operator", "pcg_solve", "bddc_gradient", "bddc_solve_host",
              "bddc_get_info", "bddc_get_coarse_basis", "bddc_get_coarse_matrix", "bddc_destroy",
              "bddc_set_apply_schedule", "bddc_set_bucket_schedule", "bddc_debug_inject"):
        getattr(lib, f).restype = C.c_int
    return lib


lib = _load()

EXPORTS = ("bddc_setup", "bddc_analyze", "bddc_acceptable_paths", "bddc_apply", "bddc_apply_noalloc", "bddc_operator", "pcg_solve", "bddc_gradient", "bddc_solve_host",
           "bddc_get_info", "bddc_get_coarse_basis", "bddc_get_coarse_matrix", "bddc_destroy",
           "bddc_last_error", "bddc_set_apply_schedule", "bddc_set_bucket_schedule", "bddc_debug_inject")


def _check(code: int, handle=None):
    if code != BDDC_OK:
        msg = lib.bddc_last_error(handle)
        raise BddcError(code, msg.decode() if msg else "")


def _ptr(t: torch.Tensor) -> C.c_void_p:
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _vptr(t: torch.Tensor, n: int) -> C.c_void_p:
    """_ptr for a vector the library reads or writes n entries of."""
    if t.numel() != n:
        raise ValueError(f"expected {n} entries, got {t.numel()}")
    return _ptr(t)


def debug_inject(what: int, value: int = 0):
    """bddc_debug_inject: process-wide test hooks (negated pivot at the next
    setups, lowered report limit of the bounded device waits, or clear)."""
    _check(lib.bddc_debug_inject(int(what), int(value)), None)


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _structs(nx, ny, nz, h, cuts, L, precision, weights, maxit, use_graph, selection="vef", beta="standard",
             piece=None, ml_block=0, ml_sub=0):
    mesh = Mesh(nx, ny, nz, h)
    part = Partition()
    keep = []
    for d in range(3):
        arr = (C.c_int * max(1, len(cuts[d])))(*cuts[d])
        keep.append(arr)
        part.ncut[d] = len(cuts[d])
        part.cut[d] = C.cast(arr, C.POINTER(C.c_int))
    if piece is not None:
        lab = np.ascontiguousarray(np.asarray(piece).reshape(-1), dtype=np.int32)
        if lab.size != nx * ny * nz:
            raise ValueError(f"piece has {lab.size} labels, the mesh {nx * ny * nz} elements")
        keep.append(lab)
        part.piece = lab.ctypes.data_as(C.POINTER(C.c_int))
    prec = {"fp64": BDDC_FP64, "mixed": BDDC_MIXED}[precision] if isinstance(precision, str) else precision
    wts = {"card": BDDC_W_CARD, "rho": BDDC_W_RHO}[weights] if isinstance(weights, str) else weights
    sel = SELECTIONS[selection] if isinstance(selection, str) else selection
    opt = Options(prec, wts, L, sel, int(use_graph), maxit, BETA_RULES[beta] if isinstance(beta, str) else beta,
                  int(ml_block), int(ml_sub))
    return mesh, part, opt, keep


def analyze(nx: int, ny: int, nz: int, cuts: Sequence[Sequence[int]], L: int, h: float = 0.0,
            precision="fp64", weights="card", selection="vef", piece=None, ml_block: int = 0,
            ml_sub: int = 0) -> dict:
    """bddc_analyze: host-only counts of objects and of the coarse elimination
    plan; piece: optional per-element sub-subdomain labels (else boxes of L);
    ml_block / ml_sub: the level-2 sizes of the multilevel coarse level."""
    mesh, part, opt, keep = _structs(nx, ny, nz, h if h > 0 else 1.0 / nx, cuts, L, precision, weights, 2000, False,
                                     selection, piece=piece, ml_block=ml_block, ml_sub=ml_sub)
    out = Analysis()
    _check(lib.bddc_analyze(C.byref(mesh), C.byref(part), C.byref(opt), C.byref(out)), None)
    return {k: getattr(out, k) for k, _ in Analysis._fields_}


def acceptable_paths(nx: int, ny: int, nz: int, cuts: Sequence[Sequence[int]], L: int, alpha=None,
                     selection="vef", piece=None) -> dict:
    """bddc_acceptable_paths: host-only acceptable-path check of a selection;
    alpha (nx*ny*nz element coefficients, x fastest) or None for alpha = 1;
    piece: optional per-element sub-subdomain labels (else boxes of L)."""
    mesh, part, opt, keep = _structs(nx, ny, nz, 1.0 / nx, cuts, L, "fp64", "card", 2000, False, selection,
                                     piece=piece)
    a = None
    if alpha is not None:
        a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
        if a.size != nx * ny * nz:
            raise ValueError(f"alpha has {a.size} entries, the mesh {nx * ny * nz} elements")
    out = Paths()
    _check(lib.bddc_acceptable_paths(C.byref(mesh), C.byref(part), C.byref(opt),
                                     None if a is None else a.ctypes.data_as(C.POINTER(C.c_double)),
                                     C.byref(out)), None)
    d = {k: getattr(out, k) for k, _ in Paths._fields_}
    d["worst_pair"] = list(d["worst_pair"])
    return d


class BDDC:
    """A set-up BDDC-SO preconditioner (bddc_setup) and its operations."""

    def __init__(self, nx: int, ny: int, nz: int, cuts: Sequence[Sequence[int]], L: int,
                 alpha: torch.Tensor, h: float = 0.0, precision="fp64", weights="card",
                 maxit: int = 2000, use_graph: bool = False, selection="vef", beta="standard", piece=None,
                 ml_block: int = 0, ml_sub: int = 0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = h if h > 0 else 1.0 / nx
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
        self.maxit = maxit
        mesh, part, opt, keep = _structs(nx, ny, nz, self.h, cuts, L, precision, weights, maxit, use_graph,
                                         selection, beta, piece=piece, ml_block=ml_block, ml_sub=ml_sub)
        self._handle = C.c_void_p()
        _check(lib.bddc_setup(C.byref(mesh), C.byref(part), C.byref(opt), _vptr(alpha, nx * ny * nz), _stream(),
                              C.byref(self._handle)), None)

    @classmethod
    def from_problem(cls, p, alpha: Optional[torch.Tensor] = None, **kw):
        a = alpha if alpha is not None else torch.from_numpy(p.alpha).cuda()
        kw.setdefault("precision", p.precision)
        kw.setdefault("weights", p.weights)
        kw.setdefault("selection", p.selection)
        kw.setdefault("piece", getattr(p, "piece", None))
        return cls(p.nx, p.ny, p.nz, p.cuts, p.L, a, h=p.h, **kw)

    def _vec(self):
        return torch.empty(self.n_nodes, dtype=torch.float64, device="cuda")

    def apply(self, r: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        z = out if out is not None else self._vec()
        _check(lib.bddc_apply(self._handle, _vptr(r, self.n_nodes), _vptr(z, self.n_nodes), _stream()), self._handle)
        return z

    def apply_noalloc(self, r: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """bddc_apply_noalloc: the same z = B r with the library's fixed device
        array as work space (no device allocation inside the call)."""
        z = out if out is not None else self._vec()
        _check(lib.bddc_apply_noalloc(self._handle, _vptr(r, self.n_nodes), _vptr(z, self.n_nodes), _stream()), self._handle)
        return z

    def operator(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        y = out if out is not None else self._vec()
        _check(lib.bddc_operator(self._handle, _vptr(x, self.n_nodes), _vptr(y, self.n_nodes), _stream()), self._handle)
        return y

    def solve(self, b: torch.Tensor, rtol: float, out: Optional[torch.Tensor] = None, raise_on_noconv=True):
        x = out if out is not None else self._vec()
        cap = self.maxit
        al = (C.c_double * cap)()
        be = (C.c_double * cap)()
        st = Stats(0, 0, 0.0, 0.0, C.cast(al, C.POINTER(C.c_double)), C.cast(be, C.POINTER(C.c_double)), cap, 0.0)
        code = lib.pcg_solve(self._handle, _vptr(b, self.n_nodes), _vptr(x, self.n_nodes), rtol, C.byref(st),
                             _stream())
        if code != BDDC_OK and (raise_on_noconv or code != BDDC_ERR_NOCONV):
            _check(code, self._handle)
        it = st.iterations
        stats = dict(iterations=it, converged=bool(st.converged), r0_norm=st.r0_norm, r_norm=st.r_norm,
                     alphas=np.array(al[:it]), betas=np.array(be[:max(it - 1, 0)]), solve_ms=st.solve_ms,
                     status=code)
        return x, stats

    def gradient(self, u: torch.Tensor, lam: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        g = out if out is not None else torch.empty(self.nx * self.ny * self.nz, dtype=torch.float64,
                                                   device="cuda")
        _check(lib.bddc_gradient(self._handle, _vptr(u, self.n_nodes), _vptr(lam, self.n_nodes),
                                 _vptr(g, self.nx * self.ny * self.nz), _stream()), self._handle)
        return g

    def set_apply_schedule(self, ctas_per_subdomain: int):
        """bddc_set_apply_schedule: 1, 2 or 4 CTAs per subdomain in the apply's local solves."""
        _check(lib.bddc_set_apply_schedule(self._handle, int(ctas_per_subdomain)), self._handle)

    def set_bucket_schedule(self, bucket: int, ring_depth: int, ctas_per_subdomain: int):
        """bddc_set_bucket_schedule: ring depth (6 or 4) and CTAs per subdomain of one size bucket."""
        _check(lib.bddc_set_bucket_schedule(self._handle, int(bucket), int(ring_depth), int(ctas_per_subdomain)),
               self._handle)

    def info(self) -> dict:
        i = Info()
        _check(lib.bddc_get_info(self._handle, C.byref(i)), self._handle)
        out = {k: getattr(i, k) for k, _ in Info._fields_}
        for k in ("phase_ms", "bucket_subdomains", "bucket_ring", "bucket_ctas"):
            out[k] = list(out[k])
        return out

    def coarse_basis(self, sub: int):
        nb, nc = C.c_int(), C.c_int()
        _check(lib.bddc_get_coarse_basis(self._handle, sub, None, None, None, C.byref(nb), C.byref(nc)),
               self._handle)
        phi = np.zeros((nb.value, nc.value))
        gid = np.zeros(nc.value, dtype=np.int32)
        node = np.zeros(nb.value, dtype=np.int64)
        _check(lib.bddc_get_coarse_basis(self._handle, sub, phi.ctypes.data_as(C.POINTER(C.c_double)),
                                         gid.ctypes.data_as(C.POINTER(C.c_int)),
                                         node.ctypes.data_as(C.POINTER(C.c_longlong)), None, None),
               self._handle)
        return phi, gid, node

    def coarse_matrix(self) -> np.ndarray:
        n = self.info()["n_coarse"]
        a = np.zeros((n, n))
        _check(lib.bddc_get_coarse_matrix(self._handle, a.ctypes.data_as(C.POINTER(C.c_double))), self._handle)
        return a

    def close(self):
        if self._handle:
            lib.bddc_destroy(self._handle)
            self._handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_host(nx, ny, nz, cuts, L, alpha: np.ndarray, b: np.ndarray, rtol: float, h: float = 0.0,
               precision="fp64", weights="card", maxit: int = 2000, use_graph: bool = False,
               selection="vef", piece=None, ml_block: int = 0, ml_sub: int = 0):
    """bddc_solve_host: setup + PCG from host arrays, result in a host array."""
    h = h if h > 0 else 1.0 / nx
    mesh, part, opt, keep = _structs(nx, ny, nz, h, cuts, L, precision, weights, maxit, use_graph, selection,
                                     piece=piece, ml_block=ml_block, ml_sub=ml_sub)
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    if a.size != nx * ny * nz or bb.size != (nx + 1) * (ny + 1) * (nz + 1):
        raise ValueError("alpha needs nx*ny*nz entries and b (nx+1)(ny+1)(nz+1)")
    x = np.zeros_like(bb)
    st = Stats(0, 0, 0.0, 0.0, None, None, 0, 0.0)
    code = lib.bddc_solve_host(C.byref(mesh), C.byref(part), C.byref(opt),
                               a.ctypes.data_as(C.POINTER(C.c_double)), bb.ctypes.data_as(C.POINTER(C.c_double)),
                               x.ctypes.data_as(C.POINTER(C.c_double)), rtol, C.byref(st))
    _check(code, None)
    return x, dict(iterations=st.iterations, converged=bool(st.converged), r_norm=st.r_norm,
                   r0_norm=st.r0_norm, solve_ms=st.solve_ms)


class BddcSolve(torch.autograd.Function):
    """u = A(alpha)^{-1} b by BDDC-SO PCG.  Backward: the adjoint solve
    A lambda = dJ/du with the same set-up preconditioner (A is symmetric),
    dJ/dalpha_e = -h lambda_e^T K u_e (bddc_gradient) and dJ/db = lambda.
    Only u is kept from the forward pass."""

    @staticmethod
    def forward(ctx, alpha, b, problem, rtol):
        pre = BDDC.from_problem(problem, alpha=alpha.detach().contiguous())
        u, stats = pre.solve(b.detach().contiguous(), rtol)
        ctx.pre, ctx.rtol = pre, rtol
        ctx.save_for_backward(u)
        ctx.stats = stats
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        lam, _ = ctx.pre.solve(grad_u.contiguous(), ctx.rtol, raise_on_noconv=False)
        g = ctx.pre.gradient(u, lam)
        ctx.pre.close()
        return g, lam, None, None
