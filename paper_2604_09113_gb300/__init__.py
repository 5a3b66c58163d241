"""Python binding of libromb (include/romb.h): argument marshalling only.

Every numerical step runs in the CUDA kernels of ``libromb.so``; this module
converts numpy arrays / torch tensors to plain pointers and checks statuses.
Importing it fails loudly when the shared library has not been built
(``python -m paper_2604_09113_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libromb.so")

ROMB_FP64, ROMB_FP32_SPLIT, ROMB_BF16_SPLIT = 0, 1, 2
ROMB_MEM_HOST, ROMB_MEM_DEVICE = 0, 1
ROMB_LOADS_QUADRATURE, ROMB_LOADS_REDUCED = 0, 1
ROMB_PRECOND_AUTO, ROMB_PRECOND_FP64, ROMB_PRECOND_FP32 = -1, 0, 1
FIELDS = {"chat": 0, "theta": 1, "K": 2, "S": 3, "psi": 4, "sc_local": 5, "D": 6, "fine": 7, "flags": 8, "loads": 9}
STATUS = {0: "ROMB_OK", -1: "ROMB_E_ARG", -2: "ROMB_E_CUDA", -3: "ROMB_E_OOM", -4: "ROMB_E_OUT_OF_BOX",
          -5: "ROMB_E_BAD_MAP", -6: "ROMB_E_NOT_SPD", -7: "ROMB_E_NOT_CONVERGED", -8: "ROMB_E_NAN",
          -9: "ROMB_E_FORMAT", -10: "ROMB_E_STATE", -11: "ROMB_E_SCRATCH"}


class RombError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class RombTrainSpec(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("basis", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("r", ctypes.c_int), ("n_r", ctypes.c_int), ("n_threads", ctypes.c_int),
                ("lo", ctypes.c_double), ("hi", ctypes.c_double), ("body", ctypes.c_int)]


class RombLattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("p", ctypes.c_int), ("map_order", ctypes.c_int),
                ("basis", ctypes.c_int), ("mem", ctypes.c_int),
                ("ctrl", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("family", ctypes.c_void_p),
                ("E", ctypes.c_double), ("nu", ctypes.c_double), ("rho", ctypes.c_double),
                ("dirichlet_mask", ctypes.c_uint), ("traction", ctypes.c_void_p),
                ("cell_present", ctypes.c_void_p), ("edge_clamped", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2604_09113_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "romb_create": ([ctypes.POINTER(P), I, S, P], I),
        "romb_destroy": ([P], None),
        "romb_strerror": ([I], ctypes.c_char_p),
        "romb_train_load": ([P, ctypes.c_char_p, ctypes.POINTER(I)], I),
        "romb_assemble": ([P, ctypes.POINTER(RombLattice), I], I),
        "romb_assemble_host_K": ([P, ctypes.POINTER(RombLattice), P], I),
        "romb_factor": ([P], I),
        "romb_bddc_solve": ([P, I, P, D, I, P, P, P], I),
        "romb_stats": ([P, P, P], I),
        "romb_field_bytes": ([P, I], S),
        "romb_read": ([P, I, P, S], I),
        "romb_train": ([ctypes.POINTER(RombTrainSpec), P, I, ctypes.c_char_p], I),
        "romb_launch_count": ([P], ctypes.c_longlong),
        "romb_compliance_grad": ([P, P, P, P, P], I),
        "romb_compliance_grad_noalloc": ([P, P, P, P, P], I),
        "romb_train_snapshot": ([ctypes.POINTER(RombTrainSpec), P, P], I),
        "romb_fma_probe": ([I, I, I, I, P, P, ctypes.POINTER(D)], I),
        "romb_train_gpu": ([I, ctypes.POINTER(RombTrainSpec), P, I, ctypes.c_char_p], I),
        "romb_train_snapshots_gpu": ([I, ctypes.POINTER(RombTrainSpec), P, I, P], I),
        "romb_set_load_form": ([P, I], I),
        "romb_set_body_force": ([P, D, D], I),
        "romb_set_precond_precision": ([P, I], I),
        "romb_set_exact_fallback": ([P, I], I),
        "romb_train_gpu_clustered": ([I, ctypes.POINTER(RombTrainSpec), I, P, I, ctypes.c_char_p], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def _check(status: int, what: str):
    if status != 0:
        raise RombError(status, f"{what}: {_lib.romb_strerror(status).decode()}")


def _ptr(a, keep: list):
    """Host numpy array (made contiguous) or device tensor -> (pointer, is_device)."""
    if a is None:
        return None, False
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        keep.append(a)
        return ctypes.c_void_p(a.data_ptr()), True
    arr = np.ascontiguousarray(a)
    keep.append(arr)
    return ctypes.c_void_p(arr.ctypes.data), False


def make_lattice(lat, keep: list, device_arrays: dict | None = None) -> RombLattice:
    """Marshal a lattice description (an object with the fields of
    ``romb_lattice``) into the C struct.  ``device_arrays`` may map 'ctrl',
    'mu', 'family', 'traction' (and 'present', 'edge_clamped', uint8) to CUDA
    tensors that are passed in place; ``lat.present`` / ``lat.edge_clamped``
    (None: every cell, no clamped cell edge) give the layout."""
    dev = device_arrays or {}
    ctrl, d1 = _ptr(dev.get("ctrl", np.asarray(lat.ctrl, dtype=np.float64)), keep)
    mu, d2 = _ptr(dev.get("mu", np.asarray(lat.mu, dtype=np.float64)), keep)
    fam, d3 = _ptr(dev.get("family", np.asarray(lat.family, dtype=np.int32)), keep)
    tr, d4 = _ptr(dev.get("traction", np.asarray(lat.traction, dtype=np.float64).reshape(8)), keep)
    if len({d1, d2, d3, d4}) != 1:
        raise ValueError("lattice arrays must all be host arrays or all device tensors")
    # layout arrays (absent cells, clamped cell edges): uint8, in the same memory
    ptrs = []
    for name in ("present", "edge_clamped"):
        a = getattr(lat, name, None)
        if name in dev:
            a = dev[name]
        elif a is not None:
            a = np.asarray(a).astype(np.uint8).reshape(-1)
            if d1:
                import torch
                a = torch.from_numpy(a).to(dev["ctrl"].device)
        q, dq = _ptr(a, keep)
        if q is not None and dq != d1:
            raise ValueError("layout arrays must live where the other lattice arrays do")
        ptrs.append(q)
    L = RombLattice(lat.nx, lat.ny, lat.p, lat.m, lat.basis, ROMB_MEM_DEVICE if d1 else ROMB_MEM_HOST,
                    ctrl, mu, fam, float(lat.E), float(lat.nu), float(lat.rho), int(lat.dirichlet_mask), tr,
                    ptrs[0], ptrs[1])
    return L


def romb_create(device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int | None = None):
    h = ctypes.c_void_p()
    _check(_lib.romb_create(ctypes.byref(h), device, mem_budget_bytes, cuda_stream), "romb_create")
    return h


def romb_destroy(ctx) -> None:
    _lib.romb_destroy(ctx)


def romb_train_load(ctx, path: str) -> int:
    fam = ctypes.c_int()
    _check(_lib.romb_train_load(ctx, path.encode(), ctypes.byref(fam)), "romb_train_load")
    return fam.value


def romb_assemble(ctx, lat, precision: int = ROMB_FP64, device_arrays=None) -> None:
    keep = []
    L = make_lattice(lat, keep, device_arrays)
    _check(_lib.romb_assemble(ctx, ctypes.byref(L), precision), "romb_assemble")


def romb_assemble_host_K(ctx, lat, K) -> None:
    keep = []
    L = make_lattice(lat, keep)
    Kp, _ = _ptr(np.asarray(K, dtype=np.float64), keep)
    _check(_lib.romb_assemble_host_K(ctx, ctypes.byref(L), Kp), "romb_assemble_host_K")


def romb_factor(ctx) -> None:
    _check(_lib.romb_factor(ctx), "romb_factor")


def romb_bddc_solve(ctx, nodes: int, nrhs: int = 1, traction_sets=None, rtol: float = 1e-8, maxit: int = 500,
                    out=None, allow_not_converged: bool = False):
    """Returns (u [nrhs, nodes, 2], iterations [nrhs], relative residuals [nrhs]).
    ``out`` may be a CUDA tensor of that shape, and ``traction_sets`` a CUDA
    tensor [nrhs, 8] (device memory, when the lattice was passed as device
    tensors)."""
    keep = []
    if out is None:
        out = np.zeros((nrhs, nodes, 2))
    up, _ = _ptr(out, keep)
    if traction_sets is not None and not getattr(traction_sets, "is_cuda", False):
        traction_sets = np.asarray(traction_sets, dtype=np.float64)
    tp, _ = _ptr(traction_sets, keep)
    its = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs)
    st = _lib.romb_bddc_solve(ctx, nrhs, tp, rtol, maxit, up, its.ctypes.data, rel.ctypes.data)
    if not (allow_not_converged and st == -7):
        _check(st, "romb_bddc_solve")
    return out, its, rel


def romb_set_load_form(ctx, form: int) -> None:
    """ROMB_LOADS_QUADRATURE (edge quadrature) or ROMB_LOADS_REDUCED (the
    reduced model of the force integrals of version-2 model files)."""
    _check(_lib.romb_set_load_form(ctx, form), "romb_set_load_form")


def romb_set_precond_precision(ctx, mode: int) -> None:
    """ROMB_PRECOND_AUTO (FP32 after a split-precision assembly), ROMB_PRECOND_FP64
    or ROMB_PRECOND_FP32: the precision of the preconditioner's operators from
    the next romb_factor on."""
    _check(_lib.romb_set_precond_precision(ctx, int(mode)), "romb_set_precond_precision")


def romb_set_exact_fallback(ctx, max_cells: int) -> None:
    """Cells (at most max_cells; 0: off) whose reduced-model stiffness is not
    positive definite are assembled from their exact tensors and factorised
    again (per-cell flag 16)."""
    _check(_lib.romb_set_exact_fallback(ctx, int(max_cells)), "romb_set_exact_fallback")


def romb_set_body_force(ctx, bx: float, by: float) -> None:
    """A constant body force per unit area (needs ROMB_LOADS_REDUCED and force
    models with a volume part; (0, 0) switches it off)."""
    _check(_lib.romb_set_body_force(ctx, bx, by), "romb_set_body_force")


def romb_stats(ctx, ncells: int | None = None):
    ms = np.zeros(8)
    flags = np.zeros(ncells, dtype=np.int32) if ncells else None
    _check(_lib.romb_stats(ctx, ms.ctypes.data, None if flags is None else flags.ctypes.data), "romb_stats")
    return ms, flags


def romb_compliance_grad(ctx, n_ctrl: int, ncells: int):
    """Returns (compliance, dc/dctrl [n_ctrl, 2], dc/dR [cells], dc/dmu [cells, 4]) of the last solve."""
    c = ctypes.c_double()
    dx = np.zeros((n_ctrl, 2))
    dR = np.zeros(ncells)
    dmu = np.zeros((ncells, 4))
    _check(_lib.romb_compliance_grad(ctx, ctypes.byref(c), dx.ctypes.data, dR.ctypes.data, dmu.ctypes.data),
           "romb_compliance_grad")
    return c.value, dx, dR, dmu


def romb_compliance_grad_noalloc(ctx, n_ctrl: int, ncells: int):
    """romb_compliance_grad computed in the library's fixed static scratch
    (no device allocation in the call); same results."""
    c = ctypes.c_double()
    dx = np.zeros((n_ctrl, 2))
    dR = np.zeros(ncells)
    dmu = np.zeros((ncells, 4))
    _check(_lib.romb_compliance_grad_noalloc(ctx, ctypes.byref(c), dx.ctypes.data, dR.ctypes.data,
                                             dmu.ctypes.data), "romb_compliance_grad_noalloc")
    return c.value, dx, dR, dmu


def romb_fma_probe(precision: int, blocks: int, threads: int, iters: int, cuda_stream, out) -> float:
    """Enqueue the FMA-rate probe (precision 0 FP64, 1 FP32) on a stream;
    ``out`` is a CUDA tensor of blocks * threads elements.  Returns the
    launch's floating-point operations (the caller times the launch)."""
    fl = ctypes.c_double()
    _check(_lib.romb_fma_probe(precision, blocks, threads, iters, cuda_stream, ctypes.c_void_p(out.data_ptr()),
                               ctypes.byref(fl)), "romb_fma_probe")
    return fl.value


def romb_launch_count(ctx) -> int:
    return int(_lib.romb_launch_count(ctx))


def romb_read(ctx, field: str) -> np.ndarray:
    f = FIELDS[field]
    nbytes = _lib.romb_field_bytes(ctx, f)
    if nbytes == 0:
        raise RombError(-10, f"field {field} not available")
    out = np.zeros(nbytes // 4, dtype=np.int32) if field == "flags" else np.zeros(nbytes // 8)
    _check(_lib.romb_read(ctx, f, out.ctypes.data, nbytes), "romb_read")
    return out


class Context:
    """Owns one romb context (RAII wrapper over romb_create / romb_destroy)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, cuda_stream=None):
        self.h = romb_create(device, mem_budget_bytes, cuda_stream)

    def close(self):
        if self.h:
            romb_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def romb_train(family: int, basis: int, p: int, r: int, n_r: int, lo: float, hi: float, samples, path: str,
               q: int = 2, n_threads: int = 0, body: bool = False) -> None:
    """Offline training on the host CPU (see include/romb.h); body: the force
    model also reduces the body-force volume integrals."""
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    spec = RombTrainSpec(family, basis, p, q, r, n_r, n_threads, lo, hi, int(body))
    _check(_lib.romb_train(ctypes.byref(spec), smp.ctypes.data, len(smp), path.encode()), "romb_train")


def romb_train_gpu(family: int, basis: int, p: int, r: int, n_r: int, lo: float, hi: float, samples, path: str,
                   q: int = 2, device: int = 0, body: bool = False) -> None:
    """Offline training on the GPU (see include/romb.h); same model file format."""
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    spec = RombTrainSpec(family, basis, p, q, r, n_r, 0, lo, hi, int(body))
    _check(_lib.romb_train_gpu(device, ctypes.byref(spec), smp.ctypes.data, len(smp), path.encode()),
           "romb_train_gpu")


def romb_train_gpu_clustered(family: int, basis: int, p: int, r: int, n_r: int, lo: float, hi: float, n_k: int,
                             samples, path: str, q: int = 2, device: int = 0, body: bool = False) -> None:
    """Clustered offline training on the GPU (Sec. 4.2.1): samples [n_k^4, n_s, 4],
    block k in cluster k's box (see include/romb.h)."""
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    if smp.ndim != 3 or smp.shape[0] != n_k ** 4 or smp.shape[2] != 4:
        raise ValueError("samples must be [n_k^4, n_s, 4]")
    spec = RombTrainSpec(family, basis, p, q, r, n_r, 0, lo, hi, int(body))
    _check(_lib.romb_train_gpu_clustered(device, ctypes.byref(spec), n_k, smp.ctypes.data, smp.shape[1],
                                         path.encode()), "romb_train_gpu_clustered")


def romb_train_snapshots_gpu(family: int, basis: int, p: int, mus, q: int = 2, device: int = 0) -> np.ndarray:
    """Snapshots I(mu) of Eq. (MDEIM I) at the rows of mus [n, 4], computed on the GPU: [n, n_i]."""
    mu = np.ascontiguousarray(mus, dtype=np.float64).reshape(-1, 4)
    spec = RombTrainSpec(family, basis, p, q, 1, 1, 0, 0.0, 1.0)
    out = np.zeros((len(mu), (p + 1) ** 4 * (q + 1) ** 2 * 4))
    _check(_lib.romb_train_snapshots_gpu(device, ctypes.byref(spec), mu.ctypes.data, len(mu), out.ctypes.data),
           "romb_train_snapshots_gpu")
    return out


def romb_train_snapshot(family: int, basis: int, p: int, mu4, q: int = 2) -> np.ndarray:
    spec = RombTrainSpec(family, basis, p, q, 1, 1, 1, 0.0, 1.0)
    mu = np.ascontiguousarray(mu4, dtype=np.float64)
    out = np.zeros((p + 1) ** 4 * (q + 1) ** 2 * 4)
    _check(_lib.romb_train_snapshot(ctypes.byref(spec), mu.ctypes.data, out.ctypes.data), "romb_train_snapshot")
    return out
