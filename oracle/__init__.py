"""CPU FP64 oracle for the SPFD Poisson solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_2010_12879_gb300``) never imports, links or runs it, and the two share
no code; the only common module is ``spfd_inputs`` (seeded input generators,
which hold none of the method's arithmetic).

The arithmetic lives in ``spfd_oracle.c`` (plain C, FP64, OpenMP loops), which
this wrapper compiles with gcc on first use and calls through ctypes.  Every
function cites the paper passage it follows:

* ``conductances``  -- the diagonal M_k of Eq. 3 (Sec. II), reading R1;
* ``assemble``      -- CSR of G^T M_k G over the conducting nodes (Eq. 3,
  Sec. III-A), readings R1, R3;
* ``rhs``           -- -G^T M_k a (Eq. 3);
* ``components`` / ``project`` -- the per-component constant nullspace (R4);
* ``pcg``           -- Jacobi-preconditioned CG to a recomputed relative
  residual (Sec. II-A premise of 1e-12; the oracle defaults to 1e-13), R5;
* ``efield``        -- |E| from Eq. 1, voxel averaged (Sec. III-E), R6;
* ``efield_complex`` -- the same for a complex (phasor) source, whose real
  and imaginary parts are solved separately (the operator is real): the
  magnitude of the complex field, reading R7;
* ``energy`` / ``div`` / ``energy_gradient`` -- the adjoint gradient of
  J = mean over conducting voxels of |E|^2 with respect to a and sigma: one
  extra Eq. 3 solve A lambda = G^T dJ/du (same operator), then
  dJ/da = dJ/du - M G lambda and dJ/dsigma from dJ/dg = -(G lambda) u (R1);
* ``nearest_rank`` / ``percentile`` -- step 6 of the pipeline (Sec. II-A,
  Sec. III-E): the 99th percentile of the voxel-averaged |E| per tissue and
  over the whole body, nearest-rank (reading R14);
* ``curl`` -- Eq. 2, b = C a: facet fluxes as the discrete curl of the edge
  potentials (reading R15);
* ``comb_tree`` / ``bfs_tree`` / ``tree_cotree`` -- step 3 of the pipeline
  (Sec. II-A, Eq. 2): the edge potentials a with a = 0 on the edges of a
  spanning tree of the node grid and C a = b, found from that definition by a
  sparse least-squares solve over the cotree edges (reading R16; small grids
  only).

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(closed forms, brute force on tiny grids, invariants); none is unpinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spfd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

i64 = ctypes.c_int64
dp = ctypes.POINTER(ctypes.c_double)
lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``spfd_oracle.c`` into ``oracle/_build/liboracle.so``.

    FMA contraction is disabled so that x86-64 and aarch64 hosts round alike.
    """
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (force or not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
            "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_conductances.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
            L.orc_index_nodes.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, lp]
            L.orc_index_nodes.restype = i64
            L.orc_assemble.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, lp, lp, lp, dp]
            L.orc_assemble.restype = i64
            L.orc_rhs.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            L.orc_matvec.argtypes = [i64, lp, lp, dp, dp, dp]
            L.orc_components.argtypes = [i64, lp, lp, lp]
            L.orc_components.restype = i64
            L.orc_project.argtypes = [i64, lp, i64, dp]
            L.orc_project.restype = ctypes.c_int
            L.orc_pcg.argtypes = [i64, lp, lp, dp, dp, ctypes.c_double, i64, dp, dp]
            L.orc_pcg.restype = ctypes.c_int
            L.orc_efield.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, dp]
            L.orc_energy.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, dp]
            L.orc_energy.restype = ctypes.c_double
            L.orc_div.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            L.orc_energy_grads.argtypes = [dp, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_nearest_rank.argtypes = [ctypes.c_double, i64]
            L.orc_nearest_rank.restype = i64
            L.orc_percentile.argtypes = [dp, dp, ctypes.POINTER(ctypes.c_int32), i64,
                                         ctypes.c_int, ctypes.c_double, dp, lp]
            L.orc_percentile.restype = ctypes.c_int
            L.orc_curl.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later parallel loops (timing only)."""
    lib().orc_set_num_threads(int(n))


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(dp)


def _l(a):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(lp)


def _dims(sigma):
    nz, ny, nx = sigma.shape
    return nx, ny, nz


def conductances(sigma: np.ndarray, h: float) -> np.ndarray:
    """Edge conductances g, shape (3, nz+1, ny+1, nx+1) (Eq. 3's M_k, R1)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    nx, ny, nz = _dims(sigma)
    g = np.zeros((3, nz + 1, ny + 1, nx + 1))
    lib().orc_conductances(_d(sigma), nx, ny, nz, float(h), _d(g))
    return g


@dataclass
class System:
    """The assembled Eq. 3 operator over the conducting nodes."""

    dims: tuple              # (nx, ny, nz) voxels
    h: float
    g: np.ndarray            # (3, nz+1, ny+1, nx+1)
    dof: np.ndarray          # int64 node-grid map -> compact index or -1
    nodes: np.ndarray        # int64 compact index -> flat node id
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    comp: np.ndarray         # int64 component id per compact unknown
    ncomp: int

    @property
    def n(self) -> int:
        return int(self.nodes.size)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def gather(self, full: np.ndarray) -> np.ndarray:
        return np.ascontiguousarray(full.reshape(-1)[self.nodes])

    def scatter(self, x: np.ndarray) -> np.ndarray:
        nx, ny, nz = self.dims
        out = np.zeros((nz + 1) * (ny + 1) * (nx + 1))
        out[self.nodes] = x
        return out.reshape(nz + 1, ny + 1, nx + 1)


def assemble(sigma: np.ndarray, h: float) -> System:
    """Assemble G^T M_k G on the conducting nodes and label its components."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    nx, ny, nz = _dims(sigma)
    L = lib()
    g = conductances(sigma, h)
    dof = np.empty((nz + 1) * (ny + 1) * (nx + 1), dtype=np.int64)
    n = int(L.orc_index_nodes(_d(g), nx, ny, nz, _l(dof)))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(7 * n, 1), dtype=np.int64)
    val = np.zeros(max(7 * n, 1))
    nnz = int(L.orc_assemble(_d(g), nx, ny, nz, _l(dof), _l(rowptr), _l(col), _d(val)))
    col, val = col[:nnz].copy(), val[:nnz].copy()
    comp = np.empty(max(n, 1), dtype=np.int64)
    ncomp = int(L.orc_components(n, _l(rowptr), _l(col), _l(comp)))
    if ncomp < 0:
        raise MemoryError("oracle component labelling")
    nodes = np.flatnonzero(dof >= 0).astype(np.int64)
    return System((nx, ny, nz), float(h), g, dof, nodes, rowptr, col, val,
                  comp[:n].copy(), ncomp)


def rhs_full(g: np.ndarray, a: np.ndarray) -> np.ndarray:
    """b = -G^T M_k a on the whole node grid (Eq. 3)."""
    _, nzp, nyp, nxp = g.shape
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == g.shape
    b = np.zeros((nzp, nyp, nxp))
    lib().orc_rhs(_d(np.ascontiguousarray(g)), _d(a), nxp - 1, nyp - 1, nzp - 1, _d(b))
    return b


def rhs(sys: System, a: np.ndarray) -> np.ndarray:
    """b restricted to the unknowns (not yet projected)."""
    return sys.gather(rhs_full(sys.g, a))


def matvec(sys: System, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(sys.n)
    lib().orc_matvec(sys.n, _l(sys.rowptr), _l(sys.col), _d(sys.val), _d(x), _d(y))
    return y


def project(sys: System, x: np.ndarray) -> np.ndarray:
    """Remove each component's unweighted mean (R4); returns a new array."""
    y = np.array(x, dtype=np.float64, copy=True)
    if sys.n and lib().orc_project(sys.n, _l(sys.comp), sys.ncomp, _d(y)) != 0:
        raise MemoryError("oracle projection")
    return y


def pcg(sys: System, b: np.ndarray, tol: float = 1e-13, maxit: int = 1_000_000):
    """Jacobi-PCG from x = 0 (R5).  Returns (x, info dict)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(max(sys.n, 1))
    info = np.zeros(3)
    rc = lib().orc_pcg(sys.n, _l(sys.rowptr), _l(sys.col), _d(sys.val), _d(b),
                       float(tol), int(maxit), _d(x), _d(info))
    if rc != 0:
        raise MemoryError("oracle pcg")
    return x[:sys.n], {"iters": int(info[0]), "rel_res": float(info[1]),
                       "converged": bool(info[2])}


def solve(sigma: np.ndarray, h: float, a: np.ndarray, tol: float = 1e-13,
          maxit: int = 1_000_000, sys: System | None = None):
    """Psi on the node grid (zero at removed nodes, zero mean per component)
    solving Eq. 3, plus the solver report.  Returns (psi, info, sys)."""
    if sys is None:
        sys = assemble(sigma, h)
    b = project(sys, rhs(sys, a))
    x, info = pcg(sys, b, tol, maxit)
    x = project(sys, x)
    return sys.scatter(x), info, sys


def efield(sigma: np.ndarray, a: np.ndarray, psi: np.ndarray, h: float,
           omega: float) -> np.ndarray:
    """Voxel-averaged |E| (Eq. 1, Sec. III-E, R6), shape (nz, ny, nx)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    nx, ny, nz = _dims(sigma)
    assert a.shape == (3, nz + 1, ny + 1, nx + 1) and psi.shape == (nz + 1, ny + 1, nx + 1)
    E = np.zeros((nz, ny, nx))
    lib().orc_efield(_d(sigma), _d(a), _d(psi), nx, ny, nz, float(h), float(omega), _d(E))
    return E


def efield_complex(sigma: np.ndarray, a_re: np.ndarray, psi_re: np.ndarray,
                   a_im: np.ndarray, psi_im: np.ndarray, h: float,
                   omega: float) -> np.ndarray:
    """|E| of a complex source (Eq. 1 for a phasor a = a_re + j a_im, R7):
    the operator of Eq. 3 is real, so Psi = psi_re + j psi_im comes from two
    real solves, and the voxel-averaged complex field E_re + j E_im has the
    magnitude sqrt(|E_re|^2 + |E_im|^2) (a peak-phasor magnitude).  Evaluated
    as that definition reads: each part's |E| by ``efield``, squared, added,
    square root."""
    e_re = efield(sigma, a_re, psi_re, h, omega)
    e_im = efield(sigma, a_im, psi_im, h, omega)
    return np.sqrt(e_re * e_re + e_im * e_im)


def energy(sigma: np.ndarray, a: np.ndarray, psi: np.ndarray, h: float,
           omega: float):
    """J = mean over conducting voxels of |E|^2 (Eq. 1, R6) and its gradient
    gJ = dJ/du on the edges (u = a + G Psi).  Returns (J, gJ)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    nx, ny, nz = _dims(sigma)
    gJ = np.zeros((3, nz + 1, ny + 1, nx + 1))
    J = float(lib().orc_energy(_d(sigma), _d(a), _d(psi), nx, ny, nz, float(h),
                               float(omega), _d(gJ)))
    return J, gJ


def div(v: np.ndarray) -> np.ndarray:
    """G^T v on the node grid for an edge field v of shape (3, nz+1, ny+1, nx+1)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    _, nzp, nyp, nxp = v.shape
    out = np.zeros((nzp, nyp, nxp))
    lib().orc_div(_d(v), nxp - 1, nyp - 1, nzp - 1, _d(out))
    return out


def energy_gradient(sigma: np.ndarray, h: float, a: np.ndarray, omega: float,
                    tol: float = 1e-13, sys: System | None = None):
    """J and its gradients by the adjoint method (module docstring).

    Returns a dict with J, dJda (edges), dJdsigma (voxels, zero in air),
    psi and lam (node grids) and the two solver reports."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    psi, info, sys = solve(sigma, h, a, tol, sys=sys)
    J, gJ = energy(sigma, a, psi, h, omega)
    badj = project(sys, sys.gather(div(gJ)))
    lam, info_adj = pcg(sys, badj, tol)
    lam_full = sys.scatter(project(sys, lam))
    nx, ny, nz = _dims(sigma)
    dJda = np.zeros_like(a)
    dJds = np.zeros_like(sigma)
    lib().orc_energy_grads(_d(sigma), _d(a), _d(psi), _d(lam_full), _d(gJ),
                           _d(np.ascontiguousarray(sys.g)), nx, ny, nz, float(h),
                           _d(dJda), _d(dJds))
    return {"J": J, "dJda": dJda, "dJdsigma": dJds, "psi": psi, "lam": lam_full,
            "info": info, "info_adj": info_adj}


def nearest_rank(p: float, n: int) -> int:
    """Least integer k >= p * n (exact), k >= 1; 0 when n = 0 (R14)."""
    return int(lib().orc_nearest_rank(float(p), int(n)))


def percentile(sigma: np.ndarray, E: np.ndarray, labels: np.ndarray, n_labels: int,
               p: float = 0.99):
    """Nearest-rank p-quantile of |E| over the conducting voxels of each
    tissue label 0..n_labels-1 and, last, over the whole body (step 6 of
    Sec. II-A, Sec. III-E, R14).  Returns (values, counts), each of length
    n_labels + 1; a group without voxels gets NaN and count 0."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    assert sigma.shape == E.shape == lab.shape
    out = np.zeros(n_labels + 1)
    cnt = np.zeros(n_labels + 1, dtype=np.int64)
    rc = lib().orc_percentile(_d(sigma), _d(E), lab.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              sigma.size, int(n_labels), float(p), _d(out), _l(cnt))
    if rc != 0:
        raise MemoryError("oracle percentile")
    return out, cnt


# ------------------------------------------------------------ Eq. 2, step 3

def curl(a: np.ndarray) -> np.ndarray:
    """b = C a (Eq. 2): the flux through facet d at node (i, j, k), the
    square spanned by the +d1 and +d2 edges of that node (d1, d2 the cyclic
    successors of d), circulated right-handed about +d (R15).  Layout of a;
    slots of facets that would leave the grid are 0."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    _, nzp, nyp, nxp = a.shape
    b = np.empty_like(a)
    lib().orc_curl(_d(a), nxp - 1, nyp - 1, nzp - 1, _d(b))
    return b


def _edge_exists(shape_nodes):
    """[3][nz+1][ny+1][nx+1] mask of the slots that hold an edge."""
    nzp, nyp, nxp = shape_nodes
    m = np.zeros((3, nzp, nyp, nxp), dtype=bool)
    m[0, :, :, :nxp - 1] = True
    m[1, :, :nyp - 1, :] = True
    m[2, :nzp - 1, :, :] = True
    return m


def _facet_exists(shape_nodes):
    """[3][nz+1][ny+1][nx+1] mask of the slots that hold a facet: facet d at
    a node exists when both of its spanning edges exist there."""
    nzp, nyp, nxp = shape_nodes
    m = np.zeros((3, nzp, nyp, nxp), dtype=bool)
    m[0, :nzp - 1, :nyp - 1, :] = True   # spanned by y and z edges
    m[1, :nzp - 1, :, :nxp - 1] = True   # spanned by z and x edges
    m[2, :, :nyp - 1, :nxp - 1] = True   # spanned by x and y edges
    return m


def comb_tree(dims, j0: int, k0: int) -> np.ndarray:
    """Edge mask [3][nz+1][ny+1][nx+1] of the comb spanning tree of the node
    grid on the root line (j, k) = (j0, k0): every z edge, the y edges of the
    plane k = k0 and the x edges of the root line.  Every node reaches the
    root line through its z column, then the plane's y line; the tree has
    (nodes - 1) edges (R16)."""
    nx, ny, nz = dims
    t = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=bool)
    t[2, :nz, :, :] = True
    t[1, k0, :ny, :] = True
    t[0, k0, j0, :nx] = True
    return t


def bfs_tree(dims, root) -> np.ndarray:
    """Edge mask of the breadth-first spanning tree of the node grid from
    node root = (i0, j0, k0) (scipy's breadth-first order over the grid
    graph; each node is joined to the node it was discovered from)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    nx, ny, nz = dims
    shp = (nz + 1, ny + 1, nx + 1)
    nn = int(np.prod(shp))
    ex = _edge_exists(shp)
    ids = np.arange(nn).reshape(shp)
    step = (1, nx + 1, (nx + 1) * (ny + 1))
    rows, cols = [], []
    for d in range(3):
        tail = ids[ex[d]]
        rows.append(tail)
        cols.append(tail + step[d])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    graph = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(nn, nn)).tocsr()
    i0, j0, k0 = root
    _, pred = breadth_first_order(graph, int(ids[k0, j0, i0]), directed=False,
                                  return_predecessors=True)
    t = np.zeros((3,) + shp, dtype=bool)
    for v in range(nn):
        u = int(pred[v])
        if u < 0:
            continue
        lo, hi = min(u, v), max(u, v)
        d = step.index(hi - lo)
        kk, jj, ii = np.unravel_index(lo, shp)
        t[d, kk, jj, ii] = True
    return t


def curl_matrix(shape_nodes):
    """Sparse C of Eq. 2 over every slot: row d*NN + n is facet d at node n
    (zero rows where no facet exists), column d*NN + n the d edge of node n
    (R15)."""
    import scipy.sparse as sp
    nzp, nyp, nxp = shape_nodes
    nn = nxp * nyp * nzp
    step = (1, nxp, nxp * nyp)
    fx = _facet_exists(shape_nodes)
    ids = np.arange(nn).reshape(shape_nodes)
    rows, cols, vals = [], [], []
    for d in range(3):
        d1, d2 = (d + 1) % 3, (d + 2) % 3
        n = ids[fx[d]]
        row = d * nn + n
        for col, v in ((d1 * nn + n, 1.0), (d2 * nn + n + step[d1], 1.0),
                       (d1 * nn + n + step[d2], -1.0), (d2 * nn + n, -1.0)):
            rows.append(row)
            cols.append(col)
            vals.append(np.full(n.size, v))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * nn, 3 * nn)).tocsr()


def tree_cotree(b: np.ndarray, tree: np.ndarray) -> np.ndarray:
    """Step 3 (Sec. II-A), tree-cotree gauging of Eq. 2: the edge potentials
    a with a = 0 on the tree edges and C a = b.  For a spanning tree the
    cotree columns of C are independent (a gradient that vanishes on a
    spanning tree vanishes everywhere), so for a divergence-free b this is
    the unique solution of the overdetermined system, found here by a sparse
    direct solve of its normal equations (R16).  Small grids only."""
    import scipy.sparse.linalg as spla
    b = np.ascontiguousarray(b, dtype=np.float64)
    shp = b.shape[1:]
    C = curl_matrix(shp)
    ex = _edge_exists(shp).reshape(-1)
    cot = np.flatnonzero(ex & ~tree.reshape(-1))
    fx = np.flatnonzero(_facet_exists(shp).reshape(-1))
    Cc = C[fx][:, cot]
    rhs = b.reshape(-1)[fx]
    N = (Cc.T @ Cc).tocsc()
    x = spla.spsolve(N, Cc.T @ rhs)
    a = np.zeros(b.size)
    a[cot] = x
    return a.reshape(b.shape)
