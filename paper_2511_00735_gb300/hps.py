"""ctypes binding of libhps.so (the C ABI declared in include/hps.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Device buffers are torch CUDA tensors (complex128, contiguous); host buffers are
numpy arrays.  There is no CPU fallback: without the built library or a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhps.so")

HPS_OK = 0
HPS_ENOTCONV = -4
HPS_ENUMERIC = -9
HPS_FP64 = 0
HPS_MIXED = 1
OUTER_DEFAULT = -1  # outer FGMRES arithmetic (hps_set_outer_arith)
OUTER_FP64 = 0
OUTER_DF64 = 1
SWEEP_DEFAULT = -1  # sweep-product arithmetic of an HPS_MIXED tree (hps_set_sweep_arith)
SWEEP_FP32 = 0
SWEEP_BF16X3 = 1
MV_DEFAULT = -1  # double-float Arnoldi matvec method (hps_set_arnoldi_matvec)
MV_SIMT = 0
MV_TENSOR = 1
TUNE_OFF = 0
TUNE_ON = 1
TUNE_FORCE = 16  # + i: candidate i of every launch configuration list

_STATUS = {0: "HPS_OK", -1: "HPS_EINVAL", -2: "HPS_ENOMEM", -3: "HPS_ENOTBUILT", -4: "HPS_ENOTCONV",
           -5: "HPS_ETIMEOUT", -6: "HPS_ECUDA", -7: "HPS_ENODEV", -8: "HPS_EUNSUPPORTED", -9: "HPS_ENUMERIC"}

# every entry point of include/hps.h
EXPORTS = ["hps_create", "hps_destroy", "hps_set_allocator", "hps_last_error", "hps_strerror", "hps_mesh",
           "hps_sizes", "hps_node_coords", "hps_boundary_points", "hps_index_maps", "hps_set_coeff",
           "hps_build_leaves", "hps_leaf_T", "hps_merge_levels", "hps_stage_T", "hps_rhs", "hps_skel_matvec",
           "hps_precond_apply", "hps_gmres_solve", "hps_kernel_launches", "hps_profile", "hps_profile_read",
           "hps_leaf_maps_noalloc", "hps_build_leaves_batch", "hps_release_workspace",
           "hps_set_outer_arith", "hps_set_gamma", "hps_volume_solution", "hps_set_sweep_arith",
           "hps_set_arnoldi_matvec", "hps_skel_matvec_mixed", "hps_profile_kernels", "hps_profile_kernels_read",
           "hps_set_autotune", "hps_autotune_table", "hps_autotune_clear"]

PHASES = ["leaf", "merge", "rhs", "matvec", "precond", "ortho", "other"]
KERNEL_CLASSES = ["sweep", "merge_gemm"]


class HPSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class HPSInfo(C.Structure):
    _fields_ = [("outer_iterations", C.c_int), ("converged", C.c_int), ("max_rel_residual", C.c_double),
                ("iterations", C.POINTER(C.c_int)), ("rel_residual", C.POINTER(C.c_double)),
                ("ms_rhs", C.c_double), ("ms_solve", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhps.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "hps_create": (i, [C.POINTER(vp), i, vp]),
        "hps_destroy": (i, [vp]),
        "hps_set_allocator": (i, [vp, ALLOC_FN, FREE_FN, vp]),
        "hps_last_error": (C.c_char_p, [vp]),
        "hps_strerror": (C.c_char_p, [i]),
        "hps_mesh": (i, [vp, i, i, i]),
        "hps_sizes": (i, [vp, C.POINTER(ll), C.POINTER(ll), C.POINTER(i), C.POINTER(ll)]),
        "hps_node_coords": (i, [vp, vp, vp]),
        "hps_boundary_points": (i, [vp, vp, vp, vp, vp]),
        "hps_index_maps": (i, [vp, vp, vp, vp]),
        "hps_set_coeff": (i, [vp, d, d, vp]),
        "hps_build_leaves": (i, [vp, i]),
        "hps_leaf_T": (i, [vp, i, i, vp]),
        "hps_merge_levels": (i, [vp, i, i]),
        "hps_stage_T": (i, [vp, i, i, vp]),
        "hps_rhs": (i, [vp, vp, vp, i]),
        "hps_skel_matvec": (i, [vp, vp, vp, i]),
        "hps_precond_apply": (i, [vp, vp, vp, i, i]),
        "hps_gmres_solve": (i, [vp, vp, vp, i, d, i, i, i, vp, C.POINTER(HPSInfo)]),
        "hps_kernel_launches": (ll, []),
        "hps_profile": (i, [vp, i]),
        "hps_profile_read": (i, [vp, vp, vp, vp]),
        "hps_leaf_maps_noalloc": (i, [i, vp, i, d, d, vp, i, vp]),
        "hps_build_leaves_batch": (i, [C.POINTER(vp), i, i]),
        "hps_release_workspace": (i, [vp]),
        "hps_set_outer_arith": (i, [vp, i]),
        "hps_set_gamma": (i, [vp, i]),
        "hps_set_sweep_arith": (i, [vp, i]),
        "hps_set_arnoldi_matvec": (i, [vp, i]),
        "hps_skel_matvec_mixed": (i, [vp, vp, vp, i]),
        "hps_volume_solution": (i, [vp, vp, vp, vp, i, vp]),
        "hps_profile_kernels": (i, [vp, i]),
        "hps_profile_kernels_read": (i, [vp, vp, vp, vp, vp]),
        "hps_set_autotune": (i, [vp, i]),
        "hps_autotune_table": (i, [C.c_char_p, i]),
        "hps_autotune_clear": (None, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> int:
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(type(x))


class Solver:
    """One libhps context on one CUDA device and stream.

    torch_alloc=True routes the library's device allocations through the torch
    caching allocator (PyTorch supplies device memory and the stream)."""

    def __init__(self, device: int = 0, stream=None, torch_alloc: bool = True):
        import torch

        self.torch = torch
        self.lib = load_library()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        self._check(self.lib.hps_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)), None)
        self.h = h
        self._held = {}
        if torch_alloc:
            dev = torch.device("cuda", device)

            def _alloc(nbytes, user):
                # allocate on this context's stream whatever thread calls, so the caching
                # allocator only reuses the block in that stream's order
                try:
                    with torch.cuda.stream(self.stream):
                        t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
                except RuntimeError:
                    return None
                p = t.data_ptr()
                self._held[p] = t
                return p

            def _free(p, user):
                self._held.pop(p, None)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            self._check(self.lib.hps_set_allocator(self.h, self._alloc_cb, self._free_cb, None))
        self.nx = self.N = None

    # -- helpers -------------------------------------------------------------
    def _check(self, status, h="self"):
        if status not in (HPS_OK,):
            msg = self.lib.hps_last_error(self.h if h == "self" else None) if h == "self" else b""
            raise HPSError(status, (msg or b"").decode())
        return status

    def close(self):
        if getattr(self, "h", None):
            self.lib.hps_destroy(self.h)
            self.h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cplx(self, shape):
        return self.torch.empty(shape, dtype=self.torch.complex128, device=f"cuda:{self.device}")

    # -- mesh ----------------------------------------------------------------
    def mesh(self, nx: int, N: int):
        self._check(self.lib.hps_mesh(self.h, nx, nx, N))
        self.nx, self.N = nx, N
        self.n_skel, self.n_bdry, self.levels, _ = self.sizes()
        self.E = nx * nx
        self.q = N - 1

    def sizes(self):
        a, b, held = C.c_longlong(), C.c_longlong(), C.c_longlong()
        lv = C.c_int()
        self._check(self.lib.hps_sizes(self.h, C.byref(a), C.byref(b), C.byref(lv), C.byref(held)))
        return a.value, b.value, lv.value, held.value

    def bytes_held(self) -> int:
        return self.sizes()[3]

    def release_workspace(self):
        """Free the per-solve buffers, keep the leaf maps and the merge tree."""
        self._check(self.lib.hps_release_workspace(self.h))

    def set_outer_arith(self, mode: int):
        """Outer FGMRES arithmetic: OUTER_FP64, OUTER_DF64 (mixed leaves only) or OUTER_DEFAULT."""
        self._check(self.lib.hps_set_outer_arith(self.h, mode))

    def set_sweep_arith(self, mode: int):
        """Sweep-product arithmetic of HPS_MIXED trees built after this call: SWEEP_FP32,
        SWEEP_BF16X3 or SWEEP_DEFAULT (bf16x3)."""
        self._check(self.lib.hps_set_sweep_arith(self.h, mode))

    def set_arnoldi_matvec(self, method: int):
        """Double-float Arnoldi matvec of later HPS_OUTER_DF64 solves: MV_TENSOR (exact splitting
        on the tensor cores), MV_SIMT or MV_DEFAULT (tensor)."""
        self._check(self.lib.hps_set_arnoldi_matvec(self.h, method))

    def set_gamma(self, gamma: int):
        """Coarse calls per level of the preconditioner: 1 = V-cycle, gamma > 1 = gamma-cycle."""
        self._check(self.lib.hps_set_gamma(self.h, int(gamma)))

    def node_coords(self):
        n = self.E * (self.N + 1) ** 2
        x, y = np.empty(n), np.empty(n)
        self._check(self.lib.hps_node_coords(self.h, _ptr(x), _ptr(y)))
        return x.reshape(self.E, -1), y.reshape(self.E, -1)

    def boundary_points(self):
        x, y, nx, ny = (np.empty(self.n_bdry) for _ in range(4))
        self._check(self.lib.hps_boundary_points(self.h, _ptr(x), _ptr(y), _ptr(nx), _ptr(ny)))
        return x, y, nx, ny

    def index_maps(self):
        n = self.E * 4 * self.q
        a, b, c = (np.empty(n, dtype=np.int32) for _ in range(3))
        self._check(self.lib.hps_index_maps(self.h, _ptr(a), _ptr(b), _ptr(c)))
        return a, b, c

    # -- build ---------------------------------------------------------------
    def set_coeff(self, kappa: float, b, eta: float | None = None):
        eta = kappa if eta is None else eta
        if hasattr(b, "data_ptr"):
            b = b.to(self.torch.float64).contiguous()
        else:
            b = np.ascontiguousarray(b, dtype=np.float64)
        self._b_keep = b
        self._check(self.lib.hps_set_coeff(self.h, float(kappa), float(eta), C.c_void_p(_ptr(b))))

    def build_leaves(self, precision: int = HPS_FP64):
        self._check(self.lib.hps_build_leaves(self.h, precision))

    def leaf_T(self, e0: int, count: int = 1):
        nb = 4 * self.q
        out = np.empty((count, nb, nb), dtype=np.complex128)
        self._check(self.lib.hps_leaf_T(self.h, e0, count, _ptr(out)))
        return out

    def merge_levels(self, L_exact: int, exact_coarse: bool = False):
        self._check(self.lib.hps_merge_levels(self.h, L_exact, int(bool(exact_coarse))))

    def stage_T(self, stage: int, sub: int):
        a = 1 << ((stage + 1) // 2)
        b = 1 << (stage // 2)
        n = 2 * (a + b) * self.q
        out = np.empty((n, n), dtype=np.complex128)
        self._check(self.lib.hps_stage_T(self.h, stage, sub, _ptr(out)))
        return out

    # -- profiling -------------------------------------------------------------
    def profile(self, enable: bool = True):
        self._check(self.lib.hps_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """{phase: (device ms, kernel launches, phase instances)} since profile(True)."""
        n = len(PHASES)
        ms = np.zeros(n)
        la = np.zeros(n, dtype=np.int64)
        ca = np.zeros(n, dtype=np.int64)
        self._check(self.lib.hps_profile_read(self.h, _ptr(ms), _ptr(la), _ptr(ca)))
        return {ph: (float(ms[i]), int(la[i]), int(ca[i])) for i, ph in enumerate(PHASES)}

    def profile_kernels(self, enable: bool = True):
        """Bracket every launch of the kernel classes (KERNEL_CLASSES) with CUDA events."""
        self._check(self.lib.hps_profile_kernels(self.h, int(bool(enable))))

    def profile_kernels_read(self):
        """{class: (device ms, launches, algorithmic bytes, algorithmic flops)} since profile_kernels(True)."""
        n = len(KERNEL_CLASSES)
        ms, by, fl = np.zeros(n), np.zeros(n), np.zeros(n)
        la = np.zeros(n, dtype=np.int64)
        self._check(self.lib.hps_profile_kernels_read(self.h, _ptr(ms), _ptr(la), _ptr(by), _ptr(fl)))
        return {k: (float(ms[i]), int(la[i]), float(by[i]), float(fl[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def set_autotune(self, mode: int):
        """Tile autotuner of the tensor-core GEMMs: TUNE_OFF, TUNE_ON or TUNE_FORCE + i."""
        self._check(self.lib.hps_set_autotune(self.h, int(mode)))

    # -- skeleton operators (device tensors [nrhs][n]) ------------------------
    def rhs(self, t):
        nrhs = t.shape[0]
        out = self._cplx((nrhs, self.n_skel))
        self._check(self.lib.hps_rhs(self.h, _ptr(t), _ptr(out), nrhs))
        return out

    def matvec(self, x):
        nrhs = x.shape[0]
        out = self._cplx((nrhs, self.n_skel))
        self._check(self.lib.hps_skel_matvec(self.h, _ptr(x), _ptr(out), nrhs))
        return out

    def matvec_mixed(self, x):
        """The Arnoldi matvec of the mixed path: Pi M x with x rounded to FP32, result in FP64."""
        nrhs = x.shape[0]
        out = self._cplx((nrhs, self.n_skel))
        self._check(self.lib.hps_skel_matvec_mixed(self.h, _ptr(x), _ptr(out), nrhs))
        return out

    def precond_apply(self, r, inner_iters: int = 5):
        nrhs = r.shape[0]
        out = self._cplx((nrhs, self.n_skel))
        self._check(self.lib.hps_precond_apply(self.h, _ptr(r), _ptr(out), nrhs, inner_iters))
        return out

    def gmres_solve(self, t, tol: float = 1e-10, inner_iters: int = 5, restart: int = 60, max_outer: int = 20,
                    out=None, raise_on_notconv: bool = True, s=None):
        """Solve M g = RHS(t, s); t is [nrhs][n_bdry] complex128 (torch CUDA tensor or numpy array),
        s (optional) the sources [nrhs][E][(N+1)^2] complex128.
        Returns (g, info dict); g has the same kind (device/host) as t unless `out` is given."""
        nrhs = t.shape[0]
        if out is None:
            out = self._cplx((nrhs, self.n_skel)) if hasattr(t, "data_ptr") else np.empty(
                (nrhs, self.n_skel), dtype=np.complex128)
        its = (C.c_int * nrhs)()
        res = (C.c_double * nrhs)()
        info = HPSInfo(0, 0, 0.0, C.cast(its, C.POINTER(C.c_int)), C.cast(res, C.POINTER(C.c_double)), 0.0, 0.0)
        sp = None if s is None else C.c_void_p(_ptr(s))
        st = self.lib.hps_gmres_solve(self.h, C.c_void_p(_ptr(t)), sp, nrhs, float(tol), int(inner_iters),
                                      int(restart), int(max_outer), C.c_void_p(_ptr(out)), C.byref(info))
        if st != HPS_OK and not (st == HPS_ENOTCONV and not raise_on_notconv):
            self._check(st)
        d = {"status": st, "outer_iterations": info.outer_iterations, "converged": info.converged,
             "max_rel_residual": info.max_rel_residual, "iterations": list(its), "rel_residual": list(res),
             "ms_rhs": info.ms_rhs, "ms_solve": info.ms_solve}
        return out, d


    def volume_solution(self, g, t=None, s=None, out=None):
        """Element fields u [nrhs][E][(N+1)^2] from the skeleton solution g (and t, s)."""
        nrhs = g.shape[0]
        n1 = self.N + 1
        if out is None:
            out = self._cplx((nrhs, self.E, n1 * n1)) if hasattr(g, "data_ptr") else np.empty(
                (nrhs, self.E, n1 * n1), dtype=np.complex128)
        tp = None if t is None else C.c_void_p(_ptr(t))
        sp = None if s is None else C.c_void_p(_ptr(s))
        self._check(self.lib.hps_volume_solution(self.h, tp, sp, C.c_void_p(_ptr(g)), nrhs, C.c_void_p(_ptr(out))))
        return out


def build_leaves_batch(solvers, precision: int = HPS_FP64):
    """hps_build_leaves for several Solver contexts at once (one leaf launch per GLL order)."""
    lib = load_library()
    arr = (C.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    st = lib.hps_build_leaves_batch(arr, len(solvers), precision)
    if st != HPS_OK:
        raise HPSError(st, (lib.hps_last_error(solvers[0].h) or b"").decode())


def kernel_launches() -> int:
    """Kernels launched by libhps in this process so far."""
    return int(load_library().hps_kernel_launches())


def exported_symbols(path: str = LIB_PATH):
    """Names of the hps_* entry points the shared library exports (no CUDA call)."""
    lib = C.CDLL(path)
    return [n for n in EXPORTS if hasattr(lib, n)]


def setup(solver: Solver, prob, precision: int = HPS_FP64, build: bool = True):
    """Mesh + coefficient (+ leaves) for a seeded problem from paper_2511_00735_gb300.inputs.
    b is sampled at the library's node coordinates; returns the plane-wave impedance data
    t [nrhs][n_bdry] (numpy complex128) at the library's boundary points."""
    from . import inputs

    solver.mesh(prob.nx, prob.N)
    X, Y = solver.node_coords()
    solver.set_coeff(prob.kappa, inputs.eval_b(prob.bumps, X, Y), prob.eta)
    if build:
        solver.build_leaves(precision)
    bx, by, bnx, bny = solver.boundary_points()
    t = np.stack([inputs.plane_wave_impedance(th, prob.kappa, prob.eta, bx, by, bnx, bny)
                  for th in prob.thetas])
    return np.ascontiguousarray(t)


def autotune_table() -> str:
    """The process-wide tile-autotuner table as text (one line per tuned GEMM shape)."""
    lib = load_library()
    n = lib.hps_autotune_table(None, 0)
    buf = C.create_string_buffer(256 * (n + 1))
    lib.hps_autotune_table(buf, len(buf))
    return buf.value.decode()


def autotune_clear():
    """Empty the process-wide tile-autotuner table."""
    load_library().hps_autotune_clear()
