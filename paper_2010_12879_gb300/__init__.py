"""GB300 SPFD Poisson solver -- Python binding of ``libspfd.so``.

The binding only marshals arguments: it passes device pointers, sizes and the
CUDA stream of PyTorch tensors to the C ABI declared in ``include/spfd.h``;
every step of the computation runs in the library's CUDA kernels.  There is
no fallback: if ``libspfd.so`` is missing or no GPU is present, the calls
raise.

Functions mirror the C entry points (``spfd_build``, ``spfd_solve``,
``spfd_solve_host``, ``spfd_efield``, ``spfd_efield_complex``, ``spfd_get_info``,
``spfd_destroy``,
``spfd_last_error``, ``spfd_opts_default``); :class:`Solver` wraps them for
``torch.float64`` tensors.
"""

from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB as LIB_PATH

SPFD_OK, SPFD_EINVAL, SPFD_ENOMEM, SPFD_ECUDA, SPFD_ENOTCONVERGED, SPFD_EINTERNAL = range(6)
STATUS_NAMES = {0: "SPFD_OK", 1: "SPFD_EINVAL", 2: "SPFD_ENOMEM", 3: "SPFD_ECUDA",
                4: "SPFD_ENOTCONVERGED", 5: "SPFD_EINTERNAL"}
SPFD_SMOOTHER_JACOBI, SPFD_SMOOTHER_CHEBYSHEV = 0, 1
SPFD_FP64, SPFD_MIXED = 0, 1

# Names declared in include/spfd.h (checked against the library by the tests).
EXPORTS = ("spfd_opts_default", "spfd_build", "spfd_solve", "spfd_solve_host",
           "spfd_efield", "spfd_efield_complex", "spfd_get_info", "spfd_kernel_stats", "spfd_destroy",
           "spfd_last_error", "spfd_residual_noalloc", "spfd_release_cached_memory",
           "spfd_energy_grad", "spfd_solve_batch", "spfd_percentile",
           "spfd_group_create", "spfd_group_solve", "spfd_group_destroy",
           "spfd_autotune_report", "spfd_tree_cotree", "spfd_pipeline_host",
           "spfd_fp64_fma_rate")


class SpfdOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("smoother", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("precision", ctypes.c_int), ("coarse_max", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("verbose", ctypes.c_int),
                ("profile", ctypes.c_int), ("autotune", ctypes.c_int)]


class SpfdInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_res_true", ctypes.c_double),
                ("ms_build", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("n_dof", ctypes.c_int64), ("n_comp", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("n_bricks", ctypes.c_int64),
                ("bytes_device", ctypes.c_int64), ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SpfdKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double)]


class SpfdTuneEntry(ctypes.Structure):
    _fields_ = [("family", ctypes.c_char_p), ("level", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("order", ctypes.c_int), ("ms_order0", ctypes.c_double),
                ("ms_order1", ctypes.c_double), ("ms_order2", ctypes.c_double)]


class SpfdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib():
    """Load libspfd.so (built by ``paper_2010_12879_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            vp, dp = ctypes.c_void_p, ctypes.c_double
            L.spfd_opts_default.argtypes = [ctypes.POINTER(SpfdOpts)]
            L.spfd_opts_default.restype = None
            L.spfd_build.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                     ctypes.POINTER(SpfdOpts), vp, ctypes.POINTER(vp)]
            L.spfd_build.restype = ctypes.c_int
            L.spfd_solve.argtypes = [vp, vp, dp, vp, ctypes.POINTER(SpfdInfo)]
            L.spfd_solve.restype = ctypes.c_int
            L.spfd_solve_batch.argtypes = [vp, ctypes.c_int, vp, dp, vp,
                                           ctypes.POINTER(SpfdInfo)]
            L.spfd_solve_batch.restype = ctypes.c_int
            L.spfd_solve_host.argtypes = [vp, vp, dp, vp, ctypes.POINTER(SpfdInfo)]
            L.spfd_solve_host.restype = ctypes.c_int
            L.spfd_efield.argtypes = [vp, vp, vp, dp, vp]
            L.spfd_efield.restype = ctypes.c_int
            L.spfd_efield_complex.argtypes = [vp, vp, vp, vp, vp, dp, vp]
            L.spfd_efield_complex.restype = ctypes.c_int
            L.spfd_get_info.argtypes = [vp, ctypes.POINTER(SpfdInfo)]
            L.spfd_get_info.restype = ctypes.c_int
            L.spfd_kernel_stats.argtypes = [vp, ctypes.POINTER(SpfdKernelStat), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_int]
            L.spfd_kernel_stats.restype = ctypes.c_int
            L.spfd_destroy.argtypes = [vp]
            L.spfd_destroy.restype = None
            L.spfd_last_error.argtypes = []
            L.spfd_last_error.restype = ctypes.c_char_p
            L.spfd_residual_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, dp, vp, ctypes.POINTER(dp)]
            L.spfd_residual_noalloc.restype = ctypes.c_int
            L.spfd_tree_cotree.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, vp, vp]
            L.spfd_tree_cotree.restype = ctypes.c_int
            L.spfd_pipeline_host.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             dp, dp, dp, ctypes.POINTER(SpfdOpts), vp, vp, vp,
                                             ctypes.POINTER(SpfdInfo)]
            L.spfd_pipeline_host.restype = ctypes.c_int
            L.spfd_fp64_fma_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]
            L.spfd_fp64_fma_rate.restype = ctypes.c_int
            L.spfd_energy_grad.argtypes = [vp, vp, vp, dp, dp, ctypes.POINTER(dp), vp, vp,
                                           ctypes.POINTER(SpfdInfo)]
            L.spfd_energy_grad.restype = ctypes.c_int
            L.spfd_percentile.argtypes = [vp, vp, vp, ctypes.c_int, dp, ctypes.POINTER(dp),
                                          ctypes.POINTER(ctypes.c_int64)]
            L.spfd_percentile.restype = ctypes.c_int
            L.spfd_group_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp,
                                            ctypes.POINTER(vp)]
            L.spfd_group_create.restype = ctypes.c_int
            L.spfd_group_solve.argtypes = [vp, ctypes.POINTER(vp), dp, ctypes.POINTER(vp),
                                           ctypes.POINTER(SpfdInfo)]
            L.spfd_group_solve.restype = ctypes.c_int
            L.spfd_group_destroy.argtypes = [vp]
            L.spfd_group_destroy.restype = None
            L.spfd_autotune_report.argtypes = [vp, ctypes.POINTER(SpfdTuneEntry), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]
            L.spfd_autotune_report.restype = ctypes.c_int
            L.spfd_release_cached_memory.argtypes = [ctypes.POINTER(ctypes.c_size_t)]
            L.spfd_release_cached_memory.restype = ctypes.c_int
            _lib = L
    return _lib


def spfd_last_error() -> str:
    return lib().spfd_last_error().decode(errors="replace")


def _check(status: int, allow=(SPFD_OK,)):
    if status not in allow:
        raise SpfdError(status, spfd_last_error())
    return status


def spfd_opts_default() -> SpfdOpts:
    o = SpfdOpts()
    lib().spfd_opts_default(ctypes.byref(o))
    return o


def spfd_build(sigma_ptr: int, nx: int, ny: int, nz: int, h: float,
               opts: SpfdOpts | None = None, stream: int = 0) -> int:
    """Raw entry point: returns the context handle (an int)."""
    out = ctypes.c_void_p()
    st = lib().spfd_build(ctypes.c_void_p(sigma_ptr), nx, ny, nz, float(h),
                          ctypes.byref(opts) if opts is not None else None,
                          ctypes.c_void_p(stream), ctypes.byref(out))
    _check(st)
    return out.value


def spfd_solve(ctx: int, a_ptr: int, tol: float, psi_ptr: int):
    info = SpfdInfo()
    st = lib().spfd_solve(ctypes.c_void_p(ctx), ctypes.c_void_p(a_ptr), float(tol),
                          ctypes.c_void_p(psi_ptr), ctypes.byref(info))
    _check(st, allow=(SPFD_OK, SPFD_ENOTCONVERGED))
    return st, info


def spfd_solve_batch(ctx: int, nrhs: int, a_ptr: int, tol: float, psi_ptr: int):
    infos = (SpfdInfo * max(nrhs, 1))()
    st = lib().spfd_solve_batch(ctypes.c_void_p(ctx), int(nrhs), ctypes.c_void_p(a_ptr),
                                float(tol), ctypes.c_void_p(psi_ptr), infos)
    _check(st, allow=(SPFD_OK, SPFD_ENOTCONVERGED))
    return st, [infos[j] for j in range(nrhs)]


def spfd_solve_host(ctx: int, a_ptr: int, tol: float, psi_ptr: int):
    info = SpfdInfo()
    st = lib().spfd_solve_host(ctypes.c_void_p(ctx), ctypes.c_void_p(a_ptr),
                               float(tol), ctypes.c_void_p(psi_ptr), ctypes.byref(info))
    _check(st, allow=(SPFD_OK, SPFD_ENOTCONVERGED))
    return st, info


def spfd_efield(ctx: int, a_ptr: int, psi_ptr: int, omega: float, E_ptr: int):
    _check(lib().spfd_efield(ctypes.c_void_p(ctx), ctypes.c_void_p(a_ptr),
                             ctypes.c_void_p(psi_ptr), float(omega),
                             ctypes.c_void_p(E_ptr)))


def spfd_efield_complex(ctx: int, a_re_ptr: int, psi_re_ptr: int, a_im_ptr: int,
                        psi_im_ptr: int, omega: float, E_ptr: int):
    _check(lib().spfd_efield_complex(ctypes.c_void_p(ctx), ctypes.c_void_p(a_re_ptr),
                                     ctypes.c_void_p(psi_re_ptr), ctypes.c_void_p(a_im_ptr),
                                     ctypes.c_void_p(psi_im_ptr), float(omega),
                                     ctypes.c_void_p(E_ptr)))


def spfd_get_info(ctx: int) -> SpfdInfo:
    info = SpfdInfo()
    _check(lib().spfd_get_info(ctypes.c_void_p(ctx), ctypes.byref(info)))
    return info


def spfd_kernel_stats(ctx: int, reset: bool = False) -> list:
    """Per-kernel-family timing of a context built with ``profile=1``."""
    n = ctypes.c_int(0)
    _check(lib().spfd_kernel_stats(ctypes.c_void_p(ctx), None, 0, ctypes.byref(n), 0))
    arr = (SpfdKernelStat * max(n.value, 1))()
    _check(lib().spfd_kernel_stats(ctypes.c_void_p(ctx), arr, n.value, ctypes.byref(n),
                                   1 if reset else 0))
    return [{"name": s.name.decode(), "launches": s.launches, "ms": s.ms,
             "bytes": s.bytes, "flops": s.flops} for s in arr[:n.value]]


def spfd_destroy(ctx: int):
    lib().spfd_destroy(ctypes.c_void_p(ctx))


def spfd_energy_grad(ctx: int, a_ptr: int, psi_ptr: int, omega: float, tol: float,
                     dJda_ptr: int, dJds_ptr: int):
    """J and its gradients into the given device arrays; returns
    (status, J, SpfdInfo of the adjoint solve)."""
    J = ctypes.c_double(0.0)
    info = SpfdInfo()
    st = _check(lib().spfd_energy_grad(ctypes.c_void_p(ctx), ctypes.c_void_p(a_ptr),
                                       ctypes.c_void_p(psi_ptr), float(omega), float(tol),
                                       ctypes.byref(J), ctypes.c_void_p(dJda_ptr),
                                       ctypes.c_void_p(dJds_ptr), ctypes.byref(info)),
                allow=(SPFD_OK, SPFD_ENOTCONVERGED))
    return st, J.value, info


def spfd_percentile(ctx: int, E_ptr: int, labels_ptr: int, n_labels: int, p: float):
    """Nearest-rank p-quantile of |E| per tissue label and over the whole
    body (step 6); returns (values, counts), lists of n_labels + 1."""
    vals = (ctypes.c_double * (n_labels + 1))()
    cnts = (ctypes.c_int64 * (n_labels + 1))()
    _check(lib().spfd_percentile(ctypes.c_void_p(ctx), ctypes.c_void_p(E_ptr),
                                 ctypes.c_void_p(labels_ptr), int(n_labels), float(p),
                                 vals, cnts))
    return list(vals), list(cnts)


def spfd_autotune_report(ctx: int) -> list:
    """The autotuner's block-order decisions for batched solves (dicts)."""
    n = ctypes.c_int(0)
    _check(lib().spfd_autotune_report(ctypes.c_void_p(ctx), None, 0, ctypes.byref(n)))
    arr = (SpfdTuneEntry * max(n.value, 1))()
    _check(lib().spfd_autotune_report(ctypes.c_void_p(ctx), arr, n.value, ctypes.byref(n)))
    return [{"family": e.family.decode(), "level": e.level, "nrhs": e.nrhs, "order": e.order,
             "ms_order0": e.ms_order0, "ms_order1": e.ms_order1, "ms_order2": e.ms_order2}
            for e in arr[:n.value]]


def spfd_release_cached_memory() -> int:
    """Give the library's cached idle device blocks back to the driver;
    returns the bytes released."""
    out = ctypes.c_size_t(0)
    _check(lib().spfd_release_cached_memory(ctypes.byref(out)))
    return out.value


def spfd_residual_noalloc(sigma_ptr: int, a_ptr: int, psi_ptr: int, nx: int,
                          ny: int, nz: int, h: float, stream: int = 0) -> float:
    """Relative residual of psi computed without a context and without
    allocating device memory, for callers whose device memory is reserved by
    another allocator or that must stay out of the allocator.  The call
    synchronises ``stream``, which therefore must not be capturing into a
    CUDA graph."""
    out = ctypes.c_double(0.0)
    _check(lib().spfd_residual_noalloc(ctypes.c_void_p(sigma_ptr), ctypes.c_void_p(a_ptr),
                                       ctypes.c_void_p(psi_ptr), nx, ny, nz, float(h),
                                       ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def spfd_tree_cotree(b_ptr: int, nx: int, ny: int, nz: int, j0: int, k0: int,
                     stream: int, a_ptr: int) -> None:
    """Step 3 (Sec. II-A): edge potentials from facet fluxes by tree-cotree
    gauging on the comb tree of root line (j0, k0) (device pointers)."""
    _check(lib().spfd_tree_cotree(ctypes.c_void_p(b_ptr), nx, ny, nz, j0, k0,
                                  ctypes.c_void_p(stream), ctypes.c_void_p(a_ptr)))


def tree_cotree(b, j0: int | None = None, k0: int | None = None, out=None):
    """``torch.float64`` CUDA tensor b [3][nz+1][ny+1][nx+1] of facet fluxes
    -> edge potentials a of the same shape (new tensor, or ``out``), on the
    current stream; the root line defaults to the grid's centre."""
    import torch
    if not (b.is_cuda and b.dtype == torch.float64 and b.is_contiguous() and b.dim() == 4
            and b.shape[0] == 3):
        raise ValueError("b must be a contiguous float64 CUDA tensor [3][nz+1][ny+1][nx+1]")
    nz, ny, nx = (int(v) - 1 for v in b.shape[1:])
    j0 = ny // 2 if j0 is None else int(j0)
    k0 = nz // 2 if k0 is None else int(k0)
    a = torch.empty_like(b) if out is None else out
    if not (a.shape == b.shape and a.dtype == torch.float64 and a.is_cuda and a.is_contiguous()):
        raise ValueError("out must match b")
    spfd_tree_cotree(b.data_ptr(), nx, ny, nz, j0, k0,
                     torch.cuda.current_stream(b.device).cuda_stream, a.data_ptr())
    return a


def pipeline_host(sigma, a, h: float, tol: float, omega: float, psi_out, E_out,
                  opts=None, stream: int = 0):
    """Steps 4 and 5 (Sec. II-A) with host arrays: ``sigma`` [nz][ny][nx] and
    ``a`` [3][nz+1][ny+1][nx+1] (float64, C-contiguous CPU tensors or numpy
    arrays; pinned tensors give the fastest copies) in, Psi and |E| written
    to ``psi_out`` / ``E_out`` (host, same kinds).  Returns (status, info)."""
    def ptr(x):
        return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
    nz, ny, nx = (int(v) for v in sigma.shape)
    info = SpfdInfo()
    st = _check(lib().spfd_pipeline_host(
        ctypes.c_void_p(ptr(sigma)), ctypes.c_void_p(ptr(a)), nx, ny, nz, float(h), float(tol),
        float(omega), ctypes.byref(opts) if opts is not None else None,
        ctypes.c_void_p(stream), ctypes.c_void_p(ptr(psi_out)), ctypes.c_void_p(ptr(E_out)),
        ctypes.byref(info)), allow=(SPFD_OK, SPFD_ENOTCONVERGED))
    return st, info.as_dict()


def spfd_fp64_fma_rate(stream: int = 0):
    """This GPU's FP64 FMA rate: (TFLOP/s, ms of the timed kernel)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().spfd_fp64_fma_rate(ctypes.c_void_p(stream), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def spfd_group_create(ctxs, stream: int = 0) -> int:
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    out = ctypes.c_void_p()
    _check(lib().spfd_group_create(arr, len(ctxs), ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def spfd_group_solve(group: int, a_ptrs, tol: float, psi_ptrs):
    """Returns (status, list of SpfdInfo)."""
    n = len(a_ptrs)
    a = (ctypes.c_void_p * n)(*a_ptrs)
    p = (ctypes.c_void_p * n)(*psi_ptrs)
    infos = (SpfdInfo * n)()
    st = _check(lib().spfd_group_solve(ctypes.c_void_p(group), a, float(tol), p, infos),
                allow=(SPFD_OK, SPFD_ENOTCONVERGED))
    return st, list(infos)


def spfd_group_destroy(group: int):
    lib().spfd_group_destroy(ctypes.c_void_p(group))


class Group:
    """Several Solver contexts (bodies of different sizes) solved together
    by one launch of a captured CUDA graph (``spfd_group_*`` in
    ``include/spfd.h``).  Close the group before its solvers."""

    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.device(dev):
            self.handle = spfd_group_create([s.ctx for s in self.solvers],
                                            self.stream.cuda_stream)

    def solve(self, a_list, tol: float = 0.0, psi_list=None):
        """Psi of every body; returns (list of psi, list of info dicts, status)."""
        import torch
        if len(a_list) != len(self.solvers):
            raise ValueError("one source field per solver")
        for S, a in zip(self.solvers, a_list):
            S._check_edges(a)
        if psi_list is None:
            psi_list = [torch.empty(S.node_shape, dtype=torch.float64, device=a.device)
                        for S, a in zip(self.solvers, a_list)]
        st, infos = spfd_group_solve(self.handle, [a.data_ptr() for a in a_list], tol,
                                     [p.data_ptr() for p in psi_list])
        return psi_list, [i.as_dict() for i in infos], st

    def close(self):
        if getattr(self, "handle", None):
            spfd_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Solver:
    """Context bound to one conductivity model.

    ``sigma`` is a contiguous ``torch.float64`` CUDA tensor of shape
    ``(nz, ny, nx)``; arrays follow the layouts documented in
    ``include/spfd.h``.  Work is ordered on ``stream`` (default: the current
    PyTorch stream at construction).
    """

    def __init__(self, sigma, h: float, opts: SpfdOpts | None = None,
                 stream=None, **kw):
        import torch
        if not (sigma.is_cuda and sigma.dtype == torch.float64 and sigma.dim() == 3
                and sigma.is_contiguous()):
            raise ValueError("sigma must be a contiguous float64 CUDA tensor (nz, ny, nx)")
        if opts is None:
            opts = spfd_opts_default()
        for k, v in kw.items():
            setattr(opts, k, v)
        self.opts = opts
        self.stream = stream if stream is not None else torch.cuda.current_stream(sigma.device)
        self.device = sigma.device
        nz, ny, nx = sigma.shape
        self.dims = (nx, ny, nz)
        self.h = float(h)
        with torch.cuda.device(sigma.device):
            self.ctx = spfd_build(sigma.data_ptr(), nx, ny, nz, h, opts,
                                  self.stream.cuda_stream)

    @property
    def node_shape(self):
        nx, ny, nz = self.dims
        return (nz + 1, ny + 1, nx + 1)

    def _check_edges(self, a):
        import torch
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                and tuple(a.shape) == (3,) + self.node_shape):
            raise ValueError(f"a must be a contiguous float64 CUDA tensor of shape {(3,) + self.node_shape}")

    def solve(self, a, tol: float = 0.0, psi=None):
        """Psi for edge potentials ``a``; returns (psi, info dict, status)."""
        import torch
        self._check_edges(a)
        if psi is None:
            psi = torch.empty(self.node_shape, dtype=torch.float64, device=a.device)
        st, info = spfd_solve(self.ctx, a.data_ptr(), tol, psi.data_ptr())
        return psi, info.as_dict(), st

    def solve_batch(self, a, tol: float = 0.0, psi=None):
        """Psi for each of the source fields ``a`` (contiguous float64 CUDA,
        ``(k, 3) + node_shape``) in one batched solve; returns (psi of shape
        ``(k,) + node_shape``, list of k info dicts, status)."""
        import torch
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                and a.dim() == 5 and tuple(a.shape[1:]) == (3,) + self.node_shape):
            raise ValueError(f"a must be a contiguous float64 CUDA tensor of shape "
                             f"(k, 3) + {self.node_shape}")
        k = a.shape[0]
        if psi is None:
            psi = torch.empty((k,) + self.node_shape, dtype=torch.float64, device=a.device)
        st, infos = spfd_solve_batch(self.ctx, k, a.data_ptr(), tol, psi.data_ptr())
        return psi, [i.as_dict() for i in infos], st

    def solve_host(self, a_host, psi_host, tol: float = 0.0):
        """Host-array variant (``a_host``/``psi_host``: contiguous CPU float64
        tensors, ideally pinned); returns (info dict, status)."""
        st, info = spfd_solve_host(self.ctx, a_host.data_ptr(), tol, psi_host.data_ptr())
        return info.as_dict(), st

    def efield(self, a, psi, omega: float, E=None):
        import torch
        self._check_edges(a)
        nx, ny, nz = self.dims
        if E is None:
            E = torch.empty((nz, ny, nx), dtype=torch.float64, device=a.device)
        spfd_efield(self.ctx, a.data_ptr(), psi.data_ptr(), omega, E.data_ptr())
        return E

    def efield_complex(self, a_re, psi_re, a_im, psi_im, omega: float, E=None):
        """|E| of the complex source a_re + j a_im from the solutions of its
        two parts (include/spfd.h, spfd_efield_complex)."""
        import torch
        self._check_edges(a_re)
        self._check_edges(a_im)
        nx, ny, nz = self.dims
        if E is None:
            E = torch.empty((nz, ny, nx), dtype=torch.float64, device=a_re.device)
        spfd_efield_complex(self.ctx, a_re.data_ptr(), psi_re.data_ptr(), a_im.data_ptr(),
                            psi_im.data_ptr(), omega, E.data_ptr())
        return E

    def energy_grad(self, a, psi, omega: float, tol: float = 0.0):
        """J = mean over conducting voxels of |E|^2 and its gradients with
        respect to ``a`` (edges) and the voxel conductivities (adjoint solve,
        include/spfd.h).  Returns (J, dJda, dJdsigma, info dict, status)."""
        import torch
        self._check_edges(a)
        nx, ny, nz = self.dims
        dJda = torch.empty_like(a)
        dJds = torch.empty((nz, ny, nx), dtype=torch.float64, device=a.device)
        st, J, info = spfd_energy_grad(self.ctx, a.data_ptr(), psi.data_ptr(), omega, tol,
                                       dJda.data_ptr(), dJds.data_ptr())
        return J, dJda, dJds, info.as_dict(), st

    def percentile(self, E, labels=None, n_labels: int = 0, p: float = 0.99):
        """Nearest-rank p-quantile of ``E`` (contiguous float64 CUDA, voxel
        shape) over the conducting voxels of each label 0..n_labels-1 of
        ``labels`` (contiguous int32 CUDA, voxel shape) and, last, over the
        whole body.  Returns (values, counts), lists of n_labels + 1."""
        import torch
        nx, ny, nz = self.dims
        if not (E.is_cuda and E.dtype == torch.float64 and E.is_contiguous()
                and tuple(E.shape) == (nz, ny, nx)):
            raise ValueError("E must be a contiguous float64 CUDA tensor (nz, ny, nx)")
        lp = 0
        if n_labels > 0:
            if labels is None or not (labels.is_cuda and labels.dtype == torch.int32
                                      and labels.is_contiguous()
                                      and tuple(labels.shape) == (nz, ny, nx)):
                raise ValueError("labels must be a contiguous int32 CUDA tensor (nz, ny, nx)")
            lp = labels.data_ptr()
        return spfd_percentile(self.ctx, E.data_ptr(), lp, n_labels, p)

    def autotune_report(self) -> list:
        return spfd_autotune_report(self.ctx)

    def info(self) -> dict:
        return spfd_get_info(self.ctx).as_dict()

    def kernel_stats(self, reset: bool = False) -> list:
        return spfd_kernel_stats(self.ctx, reset)

    def close(self):
        if getattr(self, "ctx", None):
            spfd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
