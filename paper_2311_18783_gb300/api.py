"""ctypes binding of include/geneo.h.  Device buffers are torch CUDA tensors
(float64, contiguous); streams are torch streams.  Every entry point has the
same name as its C function without the ``geneo_`` prefix."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgeneo.so")

PREC_FP64, PREC_FP32, PREC_BF16 = 0, 1, 2
COARSE_NONE, COARSE_SNK, COARSE_NK = 0, 1, 2
TAU_RECIPROCAL, TAU_PAPER = 0, 1
PENCIL_FILTERED, PENCIL_CLASSICAL = 0, 1
NOT_CONVERGED = 1


class GeneoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"geneo status {status}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("active", C.POINTER(C.c_uint8)), ("mu_inv", C.POINTER(C.c_double)),
                ("eps", C.POINTER(C.c_double)), ("gamma", C.c_double),
                ("px", C.c_int32), ("py", C.c_int32), ("pz", C.c_int32),
                ("overlap", C.c_int32), ("tau", C.c_double),
                ("cell_part", C.POINTER(C.c_int32)),
                ("natural_faces", C.POINTER(C.c_uint8))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("coarse", C.c_int32), ("geneo", C.c_int32),
                ("tau_convention", C.c_int32), ("lobpcg_block", C.c_int32),
                ("lobpcg_maxit", C.c_int32), ("lobpcg_tol", C.c_double), ("seed", C.c_uint64),
                ("coarse_dense", C.c_int32), ("coarse_leaf", C.c_int32),
                ("use_graph", C.c_int32), ("gradient_shift", C.c_int32),
                ("keep_eigvecs", C.c_int32), ("warm_start", C.c_void_p),
                ("lobpcg_neumann", C.c_int32), ("balanced", C.c_int32),
                ("geneo_pencil", C.c_int32), ("autotune", C.c_int32),
                ("autotune_cache", C.c_char_p)]


class Sizes(C.Structure):
    _fields_ = [("nverts", C.c_int64), ("ncells", C.c_int64), ("ntets", C.c_int64),
                ("nedges", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
                ("nsub", C.c_int32), ("k0", C.c_int32), ("k1", C.c_int32),
                ("sum_ni", C.c_int64), ("max_ni", C.c_int64), ("n0", C.c_int64),
                ("n0_snk", C.c_int64), ("n0_geneo", C.c_int64),
                ("local_factor_bytes", C.c_int64), ("coarse_factor_bytes", C.c_int64),
                ("setup_seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("relres", C.c_double), ("seconds", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("local_symv_launches", C.c_int64),
                ("local_symv_ms", C.c_double), ("coarse_symv_launches", C.c_int64),
                ("coarse_symv_ms", C.c_double), ("local_symv_bytes", C.c_int64),
                ("local_symv_flops", C.c_int64), ("coarse_solve_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None

# exported C functions and their argument types
_SIGS = {
    "geneo_default_options": (None, [C.POINTER(Options)]),
    "geneo_setup": (C.c_int, [C.POINTER(Problem), C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "geneo_setup_topology": (C.c_int, [C.POINTER(Problem), C.POINTER(Options),
                                       C.POINTER(C.c_void_p)]),
    "geneo_destroy": (None, [C.c_void_p]),
    "geneo_query": (C.c_int, [C.c_void_p, C.POINTER(Sizes)]),
    "geneo_assemble_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_local_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_coarse_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_apply_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                              C.POINTER(SolveInfo), C.c_void_p]),
    "geneo_solve_refined": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                      C.c_int32, C.c_int32, C.POINTER(SolveInfo), C.c_void_p]),
    "geneo_use_balanced": (C.c_int, [C.c_void_p, C.c_int32]),
    "geneo_use_persistent_coarse": (C.c_int, [C.c_void_p, C.c_int32]),
    "geneo_use_gradient_precision": (C.c_int, [C.c_void_p, C.c_int32]),
    "geneo_symv_config_count": (C.c_int, [C.c_int32]),
    "geneo_use_symv_config": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "geneo_solve_gmres": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                                    C.c_int32, C.POINTER(SolveInfo), C.c_void_p]),
    "geneo_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                                   C.POINTER(SolveInfo), C.c_void_p]),
    "geneo_solve_segments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_int32, C.POINTER(SolveInfo), C.c_void_p]),
    "geneo_compose_size": (C.c_int, [C.c_int32, C.POINTER(Problem), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]),
    "geneo_compose": (C.c_int, [C.c_int32, C.POINTER(Problem), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_compose_field": (C.c_int, [C.c_int32, C.POINTER(Problem), C.POINTER(C.c_void_p),
                                      C.c_int32, C.c_void_p]),
    "geneo_setup_batch": (C.c_int, [C.c_int32, C.POINTER(Problem), C.POINTER(Options),
                                    C.POINTER(C.c_void_p)]),
    "geneo_apply_preconditioner_block": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p,
                                                   C.c_int32, C.c_void_p]),
    "geneo_solve_block": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                    C.c_int32, C.POINTER(SolveInfo), C.c_void_p]),
    "geneo_export": (C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p, C.c_int64,
                               C.POINTER(C.c_int64)]),
    "geneo_use_precision": (C.c_int, [C.c_void_p, C.c_int32]),
    "geneo_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "geneo_profile_read": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "geneo_symv_packed_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
    "geneo_mlp_create": (C.c_int, [C.c_uint64, C.POINTER(C.c_void_p)]),
    "geneo_mlp_destroy": (None, [C.c_void_p]),
    "geneo_mlp_param_count": (C.c_int64, []),
    "geneo_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "geneo_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "geneo_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                      C.c_void_p, C.c_void_p]),
    "geneo_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                  C.c_void_p]),
    "geneo_mlp_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "geneo_last_error": (C.c_char_p, []),
    "geneo_strerror": (C.c_char_p, [C.c_int]),
}

_EXPORT_DTYPES = {
    "edges": np.int32, "dir_edge": np.uint8, "dof_edge": np.int32, "dof_vert": np.int32,
    "A_rowptr": np.int32, "A_col": np.int32, "A_val": np.float64, "N_off": np.int64,
    "N_idx": np.int32, "owner": np.int32, "snk_sub": np.int32, "snk_vert": np.int32,
    "geneo_sub": np.int32, "geneo_lambda": np.float64, "geneo_found": np.int32,
    "Zcol_ptr": np.int64, "Zcol_row": np.int32, "Zcol_val": np.float64, "k0k1": np.int32,
    "loc_f32": np.float32, "loc_nt": np.int32, "loc_toff": np.int64, "loc_voff": np.int64,
    "loc_vlen": np.int64, "mlp_features": np.float32, "eig_V": np.float64, "eig_nq": np.int32,
    "lobpcg_iters": np.int32, "lobpcg_iters_first": np.int32, "seg_off": np.int64,
    "xv_off": np.int64, "xv_vert": np.int32, "setup_stages": np.float64, "autotune": np.float64, "coarse_steps": np.float64,
}


def load_library(path=LIB_PATH):
    """Load libgeneo.so; raises OSError if it is missing (build it with
    ``__graft_entry__.build()`` or ``python paper_2311_18783_gb300/build.py``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: the CUDA library must be built first")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(status):
    if status < 0:
        msg = _LIB.geneo_last_error().decode()
        raise GeneoError(status, msg)
    return status


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def default_options(**kw):
    lib = load_library()
    o = Options()
    lib.geneo_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "autotune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def _problem_array(workloads, keep):
    """ctypes array of Problem structs for workload-like objects (nx, ny, nz,
    hx, hy, hz, active, mu_inv, eps, gamma, parts, overlap, tau and an
    optional cell_part); the NumPy arrays they point to are appended to keep."""
    arr = (Problem * len(workloads))()
    for q, w in enumerate(workloads):
        nc = w.nx * w.ny * w.nz
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(w.active, dtype=np.uint8), (nc,)))
        mu = np.ascontiguousarray(np.broadcast_to(np.asarray(w.mu_inv, dtype=np.float64), (nc,)))
        ep = np.ascontiguousarray(np.broadcast_to(np.asarray(w.eps, dtype=np.float64), (nc,)))
        keep += [a, mu, ep]
        cp = nat = None
        if getattr(w, "cell_part", None) is not None:
            keep.append(np.ascontiguousarray(w.cell_part, dtype=np.int32))
            cp = keep[-1].ctypes.data_as(C.POINTER(C.c_int32))
        if getattr(w, "natural", None) is not None:
            keep.append(np.ascontiguousarray(w.natural, dtype=np.uint8))
            nat = keep[-1].ctypes.data_as(C.POINTER(C.c_uint8))
        arr[q] = Problem(w.nx, w.ny, w.nz, w.hx, w.hy, w.hz,
                         a.ctypes.data_as(C.POINTER(C.c_uint8)),
                         mu.ctypes.data_as(C.POINTER(C.c_double)),
                         ep.ctypes.data_as(C.POINTER(C.c_double)),
                         w.gamma, w.parts[0], w.parts[1], w.parts[2], w.overlap, w.tau, cp, nat)
    return arr


def shard_problems(workloads, rank, world):
    """Indices of the independent problems rank `rank` of `world` sets up:
    largest-first assignment by active cell count to the least loaded rank
    (ties to the lower rank), so every problem goes to exactly one rank and
    the loads differ by at most one problem.  Independent problems need no
    exchange between ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    size = [int(np.count_nonzero(np.broadcast_to(w.active, (w.nx * w.ny * w.nz,))))
            for w in workloads]
    order = sorted(range(len(workloads)), key=lambda i: (-size[i], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += size[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def compose(workloads):
    """Independent problems composed into one grid by the library (host
    only, no GPU needed); see geneo_compose in include/geneo.h.  Returns a
    dict with nx, ny, nz, h, active, mu_inv, eps, cell_part, zoff and, when
    every workload has f_slot [nrhs, nverts, 7, 3], the composed f_slot."""
    lib = load_library()
    keep = []
    probs = _problem_array(workloads, keep)
    np_ = len(workloads)
    dims = (C.c_int32 * 3)()
    h = C.c_double()
    _check(lib.geneo_compose_size(np_, probs, dims, C.byref(h)))
    nx, ny, nz = dims
    nc = nx * ny * nz
    out = {"nx": nx, "ny": ny, "nz": nz, "h": h.value,
           "active": np.empty(nc, np.uint8), "mu_inv": np.empty(nc), "eps": np.empty(nc),
           "cell_part": np.empty(nc, np.int32), "zoff": np.empty(np_, np.int32)}
    _check(lib.geneo_compose(np_, probs, *(out[k].ctypes.data_as(C.c_void_p) for k in
                                           ("active", "mu_inv", "eps", "cell_part", "zoff"))))
    if all(getattr(w, "f_slot", None) is not None for w in workloads):
        fs = [np.ascontiguousarray(w.f_slot, dtype=np.float64) for w in workloads]
        nrhs = fs[0].shape[0]
        ptrs = (C.c_void_p * np_)(*(f.ctypes.data for f in fs))
        f = np.empty((nrhs, (nx + 1) * (ny + 1) * (nz + 1), 7, 3))
        _check(lib.geneo_compose_field(np_, probs, ptrs, nrhs, f.ctypes.data_as(C.c_void_p)))
        out["f_slot"] = f
    return out


class Solver:
    """One set-up problem on the current CUDA device."""

    def __init__(self, nx, ny, nz, h, active, mu_inv, eps, gamma, parts, overlap, tau,
                 options=None, cell_part=None, natural=None, **opt_kw):
        lib = load_library()
        self._keep = [np.ascontiguousarray(active, dtype=np.uint8),
                      np.ascontiguousarray(mu_inv, dtype=np.float64),
                      np.ascontiguousarray(eps, dtype=np.float64)]
        cp = nat = None
        if cell_part is not None:
            self._keep.append(np.ascontiguousarray(cell_part, dtype=np.int32))
            cp = self._keep[-1].ctypes.data_as(C.POINTER(C.c_int32))
        if natural is not None:
            self._keep.append(np.ascontiguousarray(natural, dtype=np.uint8))
            nat = self._keep[-1].ctypes.data_as(C.POINTER(C.c_uint8))
        hx, hy, hz = (h, h, h) if np.isscalar(h) else h
        p = Problem(nx, ny, nz, hx, hy, hz,
                    self._keep[0].ctypes.data_as(C.POINTER(C.c_uint8)),
                    self._keep[1].ctypes.data_as(C.POINTER(C.c_double)),
                    self._keep[2].ctypes.data_as(C.POINTER(C.c_double)),
                    gamma, parts[0], parts[1], parts[2], overlap, tau, cp, nat)
        o = options if options is not None else default_options(**opt_kw)
        ctx = C.c_void_p()
        _check(lib.geneo_setup(C.byref(p), C.byref(o), C.byref(ctx)))
        self._ctx = ctx
        self.options = o
        self.sizes = self.query()
        self.n = self.sizes["n"]

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active, w.mu_inv, w.eps, w.gamma,
                   w.parts, w.overlap, w.tau, cell_part=getattr(w, "cell_part", None),
                   natural=getattr(w, "natural", None), **kw)

    @classmethod
    def topology(cls, w, options=None, **opt_kw):
        """Host-only context of a workload (geneo_setup_topology, no GPU
        needed): query() and the integer names of export() only."""
        lib = load_library()
        self = cls.__new__(cls)
        self._keep = []
        probs = _problem_array([w], self._keep)
        o = options if options is not None else default_options(**opt_kw)
        ctx = C.c_void_p()
        _check(lib.geneo_setup_topology(probs, C.byref(o), C.byref(ctx)))
        self._ctx = ctx
        self.options = o
        self.sizes = self.query()
        self.n = self.sizes["n"]
        return self

    @classmethod
    def batch(cls, workloads, options=None, **opt_kw):
        """Independent problems in one context (geneo_setup_batch); solve with
        solve_segments, one PCG per problem in the given order.  The composed
        load of every problem's f_slot comes from compose(workloads)."""
        lib = load_library()
        self = cls.__new__(cls)
        self._keep = []
        probs = _problem_array(workloads, self._keep)
        o = options if options is not None else default_options(**opt_kw)
        ctx = C.c_void_p()
        _check(lib.geneo_setup_batch(len(workloads), probs, C.byref(o), C.byref(ctx)))
        self._ctx = ctx
        self.options = o
        self.sizes = self.query()
        self.n = self.sizes["n"]
        return self

    def close(self):
        if getattr(self, "_ctx", None):
            _LIB.geneo_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self):
        s = Sizes()
        _check(_LIB.geneo_query(self._ctx, C.byref(s)))
        return s.as_dict()

    def assemble_rhs(self, f_slot, b, stream=None):
        """f_slot: host float64 [nverts, 7, 3]; b: CUDA tensor [n]."""
        f = np.ascontiguousarray(f_slot, dtype=np.float64)
        _check(_LIB.geneo_assemble_rhs(self._ctx, f.ctypes.data_as(C.c_void_p), _ptr(b),
                                       _stream(stream)))
        return b

    def spmv(self, x, y, stream=None):
        _check(_LIB.geneo_spmv(self._ctx, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def local_solve(self, r, w, stream=None):
        _check(_LIB.geneo_local_solve(self._ctx, _ptr(r), _ptr(w), _stream(stream)))
        return w

    def coarse_solve(self, r, y, stream=None):
        _check(_LIB.geneo_coarse_solve(self._ctx, _ptr(r), _ptr(y), _stream(stream)))
        return y

    def apply_preconditioner(self, r, z, stream=None):
        _check(_LIB.geneo_apply_preconditioner(self._ctx, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def solve(self, b, x, tol=1e-8, maxit=1000, stream=None):
        info = SolveInfo()
        st = _check(_LIB.geneo_solve(self._ctx, _ptr(b), _ptr(x), tol, maxit, C.byref(info),
                                     _stream(stream)))
        return {"status": st, "iters": info.iters, "relres": info.relres,
                "seconds": info.seconds}

    def solve_refined(self, b, x, tol=1e-8, maxit=1000, nref=1, stream=None):
        """PCG plus nref refinement steps with accurate residuals; relres is
        the accurate ||b - A x|| / ||b|| of the returned x."""
        info = SolveInfo()
        st = _check(_LIB.geneo_solve_refined(self._ctx, _ptr(b), _ptr(x), tol, maxit, nref,
                                             C.byref(info), _stream(stream)))
        return {"status": st, "iters": info.iters, "relres": info.relres,
                "seconds": info.seconds}

    def solve_gmres(self, b, x, tol=1e-6, maxit=1000, restart=100, stream=None):
        """Right-preconditioned GMRES(restart) from x = 0; relres is the true
        relative residual."""
        info = SolveInfo()
        st = _check(_LIB.geneo_solve_gmres(self._ctx, _ptr(b), _ptr(x), tol, maxit, restart,
                                           C.byref(info), _stream(stream)))
        return {"status": st, "iters": info.iters, "relres": info.relres,
                "seconds": info.seconds}

    def use_symv_config(self, precision, index):
        _check(_LIB.geneo_use_symv_config(self._ctx, precision, index))

    @staticmethod
    def symv_config_count(precision):
        return _check(load_library().geneo_symv_config_count(precision))

    def use_gradient_precision(self, precision):
        _check(_LIB.geneo_use_gradient_precision(self._ctx, precision))

    def use_balanced(self, on=True):
        _check(_LIB.geneo_use_balanced(self._ctx, 1 if on else 0))

    def use_persistent_coarse(self, on=True):
        """The coarse solve as one cooperative launch (True, default) or one
        launch per level and phase (False); identical results."""
        _check(_LIB.geneo_use_persistent_coarse(self._ctx, 1 if on else 0))

    def apply_preconditioner_block(self, R, Z, stream=None):
        """R, Z: CUDA float64 tensors [nrhs, n] (contiguous)."""
        _check(_LIB.geneo_apply_preconditioner_block(self._ctx, _ptr(R), _ptr(Z), R.shape[0],
                                                     _stream(stream)))
        return Z

    def solve_block(self, B, X, tol=1e-8, maxit=1000, stream=None):
        """B, X: CUDA float64 tensors [nrhs, n]; returns the status and one
        info dict per column."""
        k = B.shape[0]
        info = (SolveInfo * k)()
        st = _check(_LIB.geneo_solve_block(self._ctx, _ptr(B), _ptr(X), k, tol, maxit, info,
                                           _stream(stream)))
        return st, [{"iters": i.iters, "relres": i.relres, "seconds": i.seconds} for i in info]

    def solve_segments(self, b, x, tol=1e-8, maxit=1000, stream=None):
        """One PCG per independent component; returns the status and one info
        dict per component (unknown ranges: export("seg_off"))."""
        k = len(self.export("seg_off")) - 1
        info = (SolveInfo * max(k, 1))()
        st = _check(_LIB.geneo_solve_segments(self._ctx, _ptr(b), _ptr(x), tol, maxit, info,
                                              _stream(stream)))
        return st, [{"iters": i.iters, "relres": i.relres, "seconds": i.seconds}
                    for i in info[:k]]

    def solve_host(self, b, tol=1e-8, maxit=1000, stream=None, out=None):
        """b: host float64 array [n] (pinned tensors are fastest).  Returns x."""
        import torch
        bh = b if isinstance(b, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(b))
        xh = out if out is not None else torch.empty_like(bh)
        info = SolveInfo()
        st = _check(_LIB.geneo_solve_host(self._ctx, C.c_void_p(bh.data_ptr()),
                                          C.c_void_p(xh.data_ptr()), tol, maxit, C.byref(info),
                                          _stream(stream)))
        return xh, {"status": st, "iters": info.iters, "relres": info.relres,
                    "seconds": info.seconds}

    def use_precision(self, precision):
        _check(_LIB.geneo_use_precision(self._ctx, precision))

    def profile(self, on=True):
        _check(_LIB.geneo_profile_enable(self._ctx, 1 if on else 0))

    def profile_read(self):
        p = Profile()
        _check(_LIB.geneo_profile_read(self._ctx, C.byref(p)))
        return p.as_dict()

    def export(self, name):
        size = C.c_int64(0)
        _check(_LIB.geneo_export(self._ctx, name.encode(), None, 0, C.byref(size)))
        dt = np.dtype(_EXPORT_DTYPES[name])
        out = np.empty(size.value // dt.itemsize, dtype=dt)
        _check(_LIB.geneo_export(self._ctx, name.encode(), out.ctypes.data_as(C.c_void_p),
                                 size.value, C.byref(size)))
        return out


class Mlp:
    """Warm-start network of the local eigensolves (5 -> 128 -> 128 -> 8),
    on the current CUDA device."""

    def __init__(self, seed=0):
        lib = load_library()
        h = C.c_void_p()
        _check(lib.geneo_mlp_create(seed, C.byref(h)))
        self._h = h
        self.nparam = lib.geneo_mlp_param_count()

    @property
    def handle(self):
        return self._h.value

    def params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _check(_LIB.geneo_mlp_get_params(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparam
        _check(_LIB.geneo_mlp_set_params(self._h, p.ctypes.data_as(C.c_void_p)))

    def loss_grad(self, solver, stream=None):
        loss = C.c_double()
        g = np.empty(self.nparam, dtype=np.float32)
        _check(_LIB.geneo_mlp_loss_grad(self._h, solver._ctx, C.byref(loss),
                                        g.ctypes.data_as(C.c_void_p), _stream(stream)))
        return loss.value, g

    def train(self, solver, steps, lr=1e-3, stream=None):
        losses = np.empty(steps, dtype=np.float64)
        _check(_LIB.geneo_mlp_train(self._h, solver._ctx, steps, lr,
                                    losses.ctypes.data_as(C.c_void_p), _stream(stream)))
        return losses

    def infer(self, solver, X, stream=None):
        """X: CUDA float64 tensor of 8 * loc_vlen (padded local rows)."""
        _check(_LIB.geneo_mlp_infer(self._h, solver._ctx, _ptr(X), _stream(stream)))
        return X

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _LIB.geneo_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
