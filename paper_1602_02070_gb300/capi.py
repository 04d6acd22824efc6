"""Thin ctypes binding of libcpca.so (include/cpca.h).

Argument marshalling only: every function here validates Python-side types,
allocates outputs and workspaces as torch CUDA tensors, and calls the C entry
point of the same name on the current torch stream. Every step of the
computation runs in the library's CUDA kernels; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpca.so")

CPCA_OK = 0
CPCA_ERR_INVALID_ARG = 1
CPCA_ERR_CUDA = 2
CPCA_ERR_WORKSPACE = 3
CPCA_ERR_SINGULAR = 4
CPCA_ERR_NOT_CONVERGED = 5
CPCA_ERR_TIMEOUT = 6
CPCA_ERR_CAPACITY = 7
CPCA_ERR_NONFINITE = 8
LAP_NORMALIZED = 0
LAP_COMBINATORIAL = 1

_STATUS = {1: "INVALID_ARG", 2: "CUDA", 3: "WORKSPACE", 4: "SINGULAR", 5: "NOT_CONVERGED",
           6: "TIMEOUT", 7: "CAPACITY", 8: "NONFINITE"}


class CpcaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"CPCA_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class cpca_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class cpca_frpcag_params(C.Structure):
    _fields_ = [("gamma_r", C.c_double), ("gamma_c", C.c_double), ("step", C.c_double),
                ("max_iter", C.c_int32), ("eps", C.c_double),
                ("power_iters", C.c_int32), ("power_seed", C.c_uint64), ("blocks", C.c_int32),
                ("start_iter", C.c_int32), ("start_prev", C.c_void_p), ("prev_out", C.c_void_p)]


class cpca_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("step", C.c_double), ("norm_r", C.c_double),
                ("norm_c", C.c_double), ("rel_change", C.c_double), ("objective", C.c_double)]


class cpca_problem(C.Structure):
    _fields_ = [("Yt", C.c_void_p), ("rr", C.c_int32), ("rc", C.c_int32), ("ldyt", C.c_int64),
                ("Lr", cpca_csr), ("Lc", cpca_csr), ("gamma_r", C.c_double),
                ("gamma_c", C.c_double), ("step", C.c_double), ("X", C.c_void_p),
                ("ldx", C.c_int64)]


class cpca_frpcag_grad_info(C.Structure):
    _fields_ = [("dgamma_r", C.c_double), ("dgamma_c", C.c_double), ("dlambda", C.c_double),
                ("dnorm_r", C.c_double), ("dnorm_c", C.c_double), ("lambda_", C.c_double),
                ("norm_r", C.c_double), ("norm_c", C.c_double)]


class cpca_decode_params(C.Structure):
    _fields_ = [("rank_ratio", C.c_double), ("k_override", C.c_int32), ("kmax", C.c_int32),
                ("delta", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("svd_iters", C.c_int32), ("svd_seed", C.c_uint64)]


class cpca_decode_info(C.Structure):
    _fields_ = [("k", C.c_int32), ("cg_iters_u", C.c_int32), ("cg_iters_v", C.c_int32),
                ("cg_res_u", C.c_double), ("cg_res_v", C.c_double),
                ("s_tilde", C.c_double * 64), ("b", C.c_int32)]


class cpca_cluster_params(C.Structure):
    _fields_ = [("k", C.c_int32), ("kmeans_iters", C.c_int32), ("seed", C.c_uint64), ("cg_tol", C.c_double),
                ("cg_max_iter", C.c_int32)]


class cpca_cluster_info(C.Structure):
    _fields_ = [("kmeans_steps", C.c_int32), ("cg_iters", C.c_int32), ("cg_res", C.c_double)]


class cpca_alt_params(C.Structure):
    _fields_ = [("gamma_r", C.c_double), ("gamma_c", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("blocks", C.c_int32)]


class cpca_alt_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("rel_res", C.c_double)]


class cpca_kron_info(C.Structure):
    _fields_ = [("chunks", C.c_int32), ("cg_iters", C.c_int32), ("cg_res", C.c_double)]


_lib = None

# (name, restype, argtypes) of every exported entry point in include/cpca.h
_SIGS = [
    ("cpca_last_error", C.c_char_p, []),
    ("cpca_version", C.c_int32, []),
    ("cpca_launch_count", C.c_uint64, []),
    ("cpca_profile_enable", C.c_int32, [C.c_int32, C.c_char_p]),
    ("cpca_profile_read", C.c_int32, [C.c_int32, C.c_char_p, C.c_int32, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int32)]),
    ("cpca_knn_graph_workspace_size", C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    ("cpca_knn_last_bruteforce", C.c_int32, []),
    ("cpca_knn_last_uncertified", C.c_int32, []),
    ("cpca_knn_last_err_rel", C.c_double, []),
    ("cpca_knn_graph", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double,
      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
      C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_sample", C.c_int32,
     [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    ("cpca_frpcag_workspace_size", C.c_size_t, [C.c_int32, C.c_int32]),
    ("cpca_frpcag_solve", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.POINTER(cpca_csr), C.POINTER(cpca_csr),
      C.POINTER(cpca_frpcag_params), C.c_void_p, C.c_int64, C.POINTER(cpca_solve_info),
      C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_frpcag_solve_noalloc", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.POINTER(cpca_csr), C.POINTER(cpca_csr),
      C.POINTER(cpca_frpcag_params), C.c_void_p, C.c_int64, C.POINTER(cpca_solve_info),
      C.c_void_p]),
    ("cpca_frpcag_status", C.c_int32, [C.c_void_p, C.c_void_p]),
    ("cpca_debug_set_barrier_spin_limit", C.c_int32, [C.c_int64]),
    ("cpca_frpcag_batched_workspace_size", C.c_size_t, [C.c_void_p, C.c_int32]),
    ("cpca_frpcag_solve_batched", C.c_int32,
     [C.c_void_p, C.c_int32, C.POINTER(cpca_frpcag_params), C.c_void_p, C.c_void_p, C.c_size_t,
      C.c_void_p]),
    ("cpca_frpcag_tune_batched", C.c_int32,
     [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_float), C.c_void_p, C.c_size_t,
      C.c_void_p]),
    ("cpca_frpcag_backward_workspace_size", C.c_size_t, [C.c_int32] * 5 + [C.c_int64] * 2),
    ("cpca_frpcag_forward_tape", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.POINTER(cpca_csr), C.POINTER(cpca_csr),
      C.POINTER(cpca_frpcag_params), C.c_int32, C.c_void_p, C.c_int64,
      C.POINTER(cpca_frpcag_grad_info), C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_frpcag_backward", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.POINTER(cpca_csr), C.POINTER(cpca_csr),
      C.POINTER(cpca_frpcag_params), C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
      C.POINTER(cpca_frpcag_grad_info), C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_laplacian_workspace_size", C.c_size_t, [C.c_int32]),
    ("cpca_laplacian_values", C.c_int32,
     [C.POINTER(cpca_csr), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_laplacian_weight_grad", C.c_int32,
     [C.POINTER(cpca_csr), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t,
      C.c_void_p]),
    ("cpca_decode_entries", C.c_int32,
     [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
      C.c_void_p, C.c_void_p]),
    ("cpca_decode_workspace_size", C.c_size_t, [C.c_int32] * 5 + [C.c_int64] * 2),
    ("cpca_decode_backward_workspace_size", C.c_size_t, [C.c_int32] * 5 + [C.c_int64] * 2),
    ("cpca_decode_backward", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
      C.POINTER(cpca_csr), C.POINTER(cpca_csr), C.POINTER(cpca_decode_params), C.c_int32,
      C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
      C.c_size_t, C.c_void_p]),
    ("cpca_decode", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
      C.POINTER(cpca_csr), C.POINTER(cpca_csr), C.POINTER(cpca_decode_params), C.c_void_p,
      C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32),
      C.POINTER(cpca_decode_info), C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_cluster_decode_workspace_size", C.c_size_t, [C.c_int32] * 4 + [C.c_int64]),
    ("cpca_cluster_decode", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_int32, C.POINTER(cpca_csr),
      C.POINTER(cpca_cluster_params), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(cpca_cluster_info),
      C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_subspace_project_workspace_size", C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    ("cpca_subspace_project", C.c_int32,
     [C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
      C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_alternate_decode_workspace_size", C.c_size_t, [C.c_int32, C.c_int32]),
    ("cpca_alternate_decode", C.c_int32,
     [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
      C.POINTER(cpca_csr), C.POINTER(cpca_csr), C.POINTER(cpca_alt_params), C.c_void_p, C.c_int64,
      C.POINTER(cpca_alt_info), C.c_void_p, C.c_size_t, C.c_void_p]),
    ("cpca_kron_reduce_workspace_size", C.c_size_t, [C.c_int32, C.c_int32, C.c_int64]),
    ("cpca_kron_reduce", C.c_int32,
     [C.POINTER(cpca_csr), C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
      C.c_void_p, C.c_void_p, C.POINTER(cpca_kron_info), C.c_void_p, C.c_size_t, C.c_void_p]),
]


def exported_names():
    return [s[0] for s in _SIGS]


def lib():
    """Load libcpca.so (building it first if it is missing). Raises if the
    CUDA library cannot be loaded: there is no CPU path."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b
            _b.build()
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != CPCA_OK:
        raise CpcaError(status, lib().cpca_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _require_cuda(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")


def _require_matrix(t, rows: int, cols: int, name: str, like: torch.Tensor | None = None,
                    host_ok: bool = False):
    """A float32 CUDA matrix of exactly rows x cols with unit column stride
    (row-major rows, any leading dimension), on the device of ``like``
    (with ``host_ok``, a page-locked host matrix is accepted too: a kernel
    writes it over the CPU-GPU link). Checked before any launch: a smaller
    buffer would be written past its end."""
    if host_ok and isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned() or t.dtype != torch.float32:
            raise ValueError(f"{name} must be a float32 CUDA tensor or page-locked (pinned) host tensor")
        if t.dim() != 2 or tuple(t.shape) != (rows, cols):
            raise ValueError(f"{name} must be {rows} x {cols}, got {tuple(t.shape)}")
        if t.stride(1) != 1 or t.stride(0) < cols:
            raise ValueError(f"{name} must be row-major with unit column stride")
        return
    _require_cuda(t, torch.float32, name)
    if t.dim() != 2 or tuple(t.shape) != (rows, cols):
        raise ValueError(f"{name} must be {rows} x {cols}, got {tuple(t.shape)}")
    if t.stride(1) != 1 or t.stride(0) < cols:
        raise ValueError(f"{name} must be row-major with unit column stride")
    if like is not None and t.device != like.device:
        raise ValueError(f"{name} is on {t.device}, expected {like.device}")


def _workspace(nbytes: int, device) -> torch.Tensor:
    """Scratch for one call. CPCA_FAULT=alloc (host-side fault injection)
    makes this fail as a real allocation failure would, before any launch."""
    if os.environ.get("CPCA_FAULT") == "alloc":
        raise CpcaError(CPCA_ERR_WORKSPACE, "injected workspace allocation failure (CPCA_FAULT=alloc)")
    try:
        return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    except torch.cuda.OutOfMemoryError as e:
        raise CpcaError(CPCA_ERR_WORKSPACE, f"workspace of {int(nbytes)} bytes: {e}") from e


def knn_last_bruteforce() -> int:
    """Queries of the last cpca_knn_graph call (this thread) that fell back
    to exact brute force because their candidates were not certified."""
    return int(lib().cpca_knn_last_bruteforce())


def knn_last_uncertified() -> int:
    """Queries of the last cpca_knn_graph call (this thread) left with the
    exact nearest of their tensor-core candidates, uncertified, because the
    brute-force budget was exceeded."""
    return int(lib().cpca_knn_last_uncertified())


def knn_last_err_rel() -> float:
    """Relative error bound (times |q|^2 + |b|^2) of the candidate ranking
    that the last cpca_knn_graph call (this thread) certified against."""
    return float(lib().cpca_knn_last_err_rel())


def launch_count() -> int:
    return int(lib().cpca_launch_count())


def profile_enable(on: bool = True, prefix: str = "") -> None:
    lib().cpca_profile_enable(int(on), prefix.encode())


def profile_read(max_names: int = 64) -> dict:
    """{kernel name: (total ms, launches)} of the launches recorded since
    profile_enable (waits for their events)."""
    nl = 64
    names = C.create_string_buffer(max_names * nl)
    ms = (C.c_double * max_names)()
    cnt = (C.c_int32 * max_names)()
    n = lib().cpca_profile_read(max_names, names, nl, ms, cnt)
    out = {}
    for i in range(min(n, max_names)):
        nm = names.raw[i * nl:(i + 1) * nl].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out


@dataclass
class Csr:
    """Device CSR Laplacian (and optional edge weights on the same pattern)."""
    rowptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    weight: torch.Tensor | None = None
    sigma2: float = 0.0

    @property
    def n(self) -> int:
        return self.rowptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.col.numel()

    def c(self) -> cpca_csr:
        return cpca_csr(self.n, self.nnz, self.rowptr.data_ptr(), self.col.data_ptr(),
                        self.val.data_ptr() if self.val is not None else None)

    @staticmethod
    def from_scipy(L, device="cuda", weight=None) -> "Csr":
        """From a scipy Laplacian; ``weight`` (a scipy matrix W) is read on
        L's pattern (0 where W has no entry, e.g. the diagonal)."""
        L = L.tocsr()
        L.sort_indices()
        w = None
        if weight is not None:
            rows = L.indptr.searchsorted(range(L.nnz), side="right") - 1
            w = torch.as_tensor(weight.tocsr()[rows, L.indices].A1.astype("float32"), device=device)
        return Csr(torch.as_tensor(L.indptr.astype("int64"), device=device),
                   torch.as_tensor(L.indices.astype("int32"), device=device),
                   torch.as_tensor(L.data.astype("float32"), device=device), w)

    def pattern_scipy(self, values):
        """A scipy CSR matrix with this pattern and the given per-entry values."""
        import scipy.sparse as sp
        v = values.double().cpu().numpy() if isinstance(values, torch.Tensor) else values
        return sp.csr_matrix((v, self.col.cpu().numpy(), self.rowptr.cpu().numpy()),
                             shape=(self.n, self.n))

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.double().cpu().numpy(), self.col.cpu().numpy(),
                              self.rowptr.cpu().numpy()), shape=(self.n, self.n))


def cpca_knn_graph(pts: torch.Tensor, K: int, lap_type: int = LAP_NORMALIZED,
                   sigma2: float = -1.0, transposed: bool = False, want_knn: bool = False):
    """kNN graph + Laplacian of the rows of ``pts`` (or of its columns if
    ``transposed``). Returns (Csr, knn_idx, knn_d2) with the kNN lists None
    unless ``want_knn``."""
    _require_cuda(pts, torch.float32, "pts")
    if pts.dim() != 2 or pts.stride(1) != 1:
        raise ValueError("pts must be a 2-D row-major tensor")
    rows, cols = pts.shape
    npts, dim = (cols, rows) if transposed else (rows, cols)
    dev = pts.device
    cap = npts * (2 * K + 1)
    rowptr = torch.empty(npts + 1, dtype=torch.int64, device=dev)
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    val = torch.empty(cap, dtype=torch.float32, device=dev)
    weight = torch.empty(cap, dtype=torch.float32, device=dev)
    kidx = torch.empty(npts, K, dtype=torch.int32, device=dev) if want_knn else None
    kd2 = torch.empty(npts, K, dtype=torch.float32, device=dev) if want_knn else None
    ws = _workspace(lib().cpca_knn_graph_workspace_size(npts, dim, K, int(transposed)), dev)
    nnz = C.c_int64(0)
    s2 = C.c_double(0)
    _check(lib().cpca_knn_graph(_ptr(pts), npts, dim, pts.stride(0), int(transposed), K, lap_type,
                                sigma2, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(weight), cap,
                                _ptr(kidx), _ptr(kd2), C.byref(nnz), C.byref(s2), _ptr(ws),
                                ws.numel(), _stream()))
    n = nnz.value
    return Csr(rowptr, col[:n], val[:n], weight[:n], s2.value), kidx, kd2


def cpca_sample(seed: int, p: int, n: int, rho_r: int, rho_c: int, Y: torch.Tensor | None = None,
                device="cuda"):
    """Omega_r, Omega_c (ascending int32) and, if Y is given, Y~ = Y[Omega_r][:, Omega_c]."""
    if Y is not None:
        _require_cuda(Y, torch.float32, "Y")
        device = Y.device
    om_r = torch.empty(rho_r, dtype=torch.int32, device=device)
    om_c = torch.empty(rho_c, dtype=torch.int32, device=device)
    # rows padded to a multiple of 4 floats: 16-byte row stride for TMA and vector loads
    ldyt = (rho_c + 3) // 4 * 4
    Yt = (torch.empty(rho_r, ldyt, dtype=torch.float32, device=device)[:, :rho_c]
          if Y is not None else None)
    _check(lib().cpca_sample(seed & (2 ** 64 - 1), p, n, rho_r, rho_c, _ptr(Y),
                             Y.stride(0) if Y is not None else 0, _ptr(om_r), _ptr(om_c),
                             _ptr(Yt), ldyt, _stream()))
    return om_r, om_c, Yt


def frpcag_params(gamma_r=1.0, gamma_c=1.0, step=-1.0, max_iter=300, eps=0.0,
                  power_iters=200, power_seed=0, blocks=0, start_iter=0, start_prev=None,
                  prev_out=None) -> cpca_frpcag_params:
    """Parameters of cpca_frpcag_solve; start_prev / prev_out are device
    tensors (rr x rc, the leading dimension of the solve's output) or None:
    the caller keeps them alive for the call."""
    for name, t in (("start_prev", start_prev), ("prev_out", prev_out)):
        if t is not None:
            _require_cuda(t, torch.float32, name)
    return cpca_frpcag_params(gamma_r, gamma_c, step, max_iter, eps, power_iters, power_seed,
                              blocks, start_iter, None if start_prev is None else start_prev.data_ptr(),
                              None if prev_out is None else prev_out.data_ptr())


def cpca_frpcag_solve(Yt: torch.Tensor, Lr: Csr, Lc: Csr, params: cpca_frpcag_params | None = None,
                      want_info: bool = True, out: torch.Tensor | None = None, ws=None, **kw):
    """FISTA for FRPCAG on Y~ (rr x rc). Returns (X, info or None)."""
    _require_cuda(Yt, torch.float32, "Yt")
    rr, rc = Yt.shape if Yt.dim() == 2 else (0, 0)
    _require_matrix(Yt, rr, rc, "Yt")
    prm = params if params is not None else frpcag_params(**kw)
    X = out if out is not None else torch.empty(rr, rc, dtype=torch.float32, device=Yt.device)
    _require_matrix(X, rr, rc, "out", Yt)
    if ws is None:
        ws = _workspace(lib().cpca_frpcag_workspace_size(rr, rc), Yt.device)
    info = cpca_solve_info() if want_info else None
    lr, lc = Lr.c(), Lc.c()
    _check(lib().cpca_frpcag_solve(_ptr(Yt), rr, rc, Yt.stride(0), C.byref(lr), C.byref(lc),
                                   C.byref(prm), _ptr(X), X.stride(0),
                                   C.byref(info) if info is not None else None, _ptr(ws),
                                   ws.numel(), _stream()))
    return X, info


def cpca_frpcag_solve_noalloc(Yt: torch.Tensor, Lr: Csr, Lc: Csr,
                              params: cpca_frpcag_params | None = None, want_info: bool = True,
                              out: torch.Tensor | None = None, **kw):
    """cpca_frpcag_solve with the library's built-in scratch instead of a
    workspace (for callers that cannot allocate device memory; problems up to
    the built-in scratch size). Returns (X, info or None)."""
    _require_cuda(Yt, torch.float32, "Yt")
    rr, rc = Yt.shape if Yt.dim() == 2 else (0, 0)
    _require_matrix(Yt, rr, rc, "Yt")
    prm = params if params is not None else frpcag_params(**kw)
    X = out if out is not None else torch.empty(rr, rc, dtype=torch.float32, device=Yt.device)
    _require_matrix(X, rr, rc, "out", Yt)
    info = cpca_solve_info() if want_info else None
    lr, lc = Lr.c(), Lc.c()
    _check(lib().cpca_frpcag_solve_noalloc(_ptr(Yt), rr, rc, Yt.stride(0), C.byref(lr), C.byref(lc),
                                           C.byref(prm), _ptr(X), X.stride(0),
                                           C.byref(info) if info is not None else None,
                                           _stream()))
    return X, info


def cpca_frpcag_status(ws: torch.Tensor | None = None) -> None:
    """Raises CpcaError(CPCA_ERR_TIMEOUT) if a grid barrier of the last
    FISTA solve on ``ws`` (None: the built-in no-allocation scratch) gave
    up. Synchronises the current stream. Info-less solves are asynchronous,
    so this is where their timeouts surface."""
    _check(lib().cpca_frpcag_status(_ptr(ws), _stream()))


def debug_set_barrier_spin_limit(polls: int) -> None:
    """Test hook: polls before a grid-barrier wait of a new launch gives up
    (0 restores the default)."""
    lib().cpca_debug_set_barrier_spin_limit(int(polls))


def frpcag_tape_workspace(Yt: torch.Tensor, Lr: Csr, Lc: Csr, params: cpca_frpcag_params,
                          ckpt_every: int = 20) -> torch.Tensor:
    rr, rc = Yt.shape
    T = 0 if params.step > 0 else params.power_iters
    return _workspace(lib().cpca_frpcag_backward_workspace_size(rr, rc, params.max_iter, ckpt_every, T,
                                                                Lr.nnz, Lc.nnz), Yt.device)


def cpca_frpcag_forward_tape(Yt: torch.Tensor, Lr: Csr, Lc: Csr, params: cpca_frpcag_params,
                             ckpt_every: int = 20, ws=None):
    """Forward FISTA solve that records the tape for cpca_frpcag_backward
    (resume=True). Returns (X, ws, info)."""
    _require_cuda(Yt, torch.float32, "Yt")
    rr, rc = Yt.shape
    if ws is None:
        ws = frpcag_tape_workspace(Yt, Lr, Lc, params, ckpt_every)
    X = torch.empty(rr, rc, dtype=torch.float32, device=Yt.device)
    info = cpca_frpcag_grad_info()
    lr, lc = Lr.c(), Lc.c()
    _check(lib().cpca_frpcag_forward_tape(_ptr(Yt), rr, rc, Yt.stride(0), C.byref(lr), C.byref(lc),
                                          C.byref(params), ckpt_every, _ptr(X), X.stride(0),
                                          C.byref(info), _ptr(ws), ws.numel(), _stream()))
    return X, ws, info


def cpca_frpcag_backward(Yt: torch.Tensor, Lr: Csr, Lc: Csr, dX: torch.Tensor,
                         params: cpca_frpcag_params | None = None, ckpt_every: int = 20,
                         want_dL: bool = True, want_dw: bool = False,
                         lap_type: int = LAP_NORMALIZED, ws=None, resume: bool = False, **kw):
    """Reverse-mode derivative of cpca_frpcag_solve for dloss/dX = dX.
    Returns dict: dYt (rr x rc), dLr, dLc (FP64 per CSR entry, or None),
    dwr, dwc (FP32 per CSR entry, needs Lr.weight / Lc.weight, or None),
    info (cpca_frpcag_grad_info). resume=True reuses the tape that
    cpca_frpcag_forward_tape left in ``ws``."""
    _require_cuda(Yt, torch.float32, "Yt")
    _require_cuda(dX, torch.float32, "dX")
    prm = params if params is not None else frpcag_params(**kw)
    rr, rc = Yt.shape
    dev = Yt.device
    if resume and ws is None:
        raise ValueError("resume needs the forward tape workspace")
    if ws is None:
        ws = frpcag_tape_workspace(Yt, Lr, Lc, prm, ckpt_every)
    dY = torch.empty(rr, rc, dtype=torch.float32, device=dev)
    dLr = torch.empty(Lr.nnz, dtype=torch.float64, device=dev) if want_dL else None
    dLc = torch.empty(Lc.nnz, dtype=torch.float64, device=dev) if want_dL else None
    dwr = dwc = None
    if want_dw:
        if Lr.weight is None or Lc.weight is None:
            raise ValueError("want_dw needs Lr.weight and Lc.weight")
        dwr = torch.empty(Lr.nnz, dtype=torch.float32, device=dev)
        dwc = torch.empty(Lc.nnz, dtype=torch.float32, device=dev)
    info = cpca_frpcag_grad_info()
    lr, lc = Lr.c(), Lc.c()
    _check(lib().cpca_frpcag_backward(
        _ptr(Yt), rr, rc, Yt.stride(0), C.byref(lr), C.byref(lc), C.byref(prm), ckpt_every,
        int(resume), _ptr(dX), dX.stride(0), _ptr(dY), dY.stride(0), _ptr(dLr), _ptr(dLc),
        _ptr(Lr.weight) if want_dw else None, _ptr(Lc.weight) if want_dw else None, lap_type,
        _ptr(dwr), _ptr(dwc), C.byref(info), _ptr(ws), ws.numel(), _stream()))
    return {"dYt": dY, "dLr": dLr, "dLc": dLc, "dwr": dwr, "dwc": dwc, "info": info}


class Batch:
    """A fixed set of FRPCAG problems for cpca_frpcag_solve_batched: holds
    the C problem table, the outputs X_i and one workspace, so repeated
    solves (or a CUDA-graph capture of one) reuse the same buffers."""

    def __init__(self, problems):
        # problems: list of dicts with Yt (CUDA tensor), Lr, Lc (Csr), gamma_r,
        # gamma_c and optional step
        n = len(problems)
        self.keep = []
        self.X = []
        self.table = (cpca_problem * n)()
        for i, q in enumerate(problems):
            Yt = q["Yt"]
            _require_cuda(Yt, torch.float32, "Yt")
            X = torch.empty(Yt.shape[0], Yt.shape[1], dtype=torch.float32, device=Yt.device)
            self.X.append(X)
            self.keep += [Yt, q["Lr"], q["Lc"]]
            self.table[i] = cpca_problem(Yt.data_ptr(), Yt.shape[0], Yt.shape[1], Yt.stride(0),
                                         q["Lr"].c(), q["Lc"].c(), q["gamma_r"], q["gamma_c"],
                                         q.get("step", -1.0), X.data_ptr(), X.stride(0))
        self.n = n
        nbytes = lib().cpca_frpcag_batched_workspace_size(self.table, n)
        if nbytes == 0:
            raise CpcaError(CPCA_ERR_INVALID_ARG, "bad batch")
        self.ws = _workspace(nbytes, problems[0]["Yt"].device)

    def solve(self, params: cpca_frpcag_params, want_info: bool = False):
        infos = (cpca_solve_info * self.n)() if want_info else None
        _check(lib().cpca_frpcag_solve_batched(self.table, self.n, C.byref(params), infos,
                                               _ptr(self.ws), self.ws.numel(), _stream()))
        return self.X, (list(infos) if want_info else None)

    def tune(self):
        """Run the autotuner; returns (blocks, ms per 10 iterations)."""
        b = C.c_int32(0)
        ms = C.c_float(0)
        _check(lib().cpca_frpcag_tune_batched(self.table, self.n, C.byref(b), C.byref(ms),
                                              _ptr(self.ws), self.ws.numel(), _stream()))
        return b.value, ms.value


def decode_params(rank_ratio=0.1, k_override=0, kmax=24, delta=0.0, cg_tol=1e-6, cg_max_iter=0,
                  svd_iters=6, svd_seed=0) -> cpca_decode_params:
    return cpca_decode_params(rank_ratio, k_override, kmax, delta, cg_tol, cg_max_iter, svd_iters,
                              svd_seed)


def cpca_decode(Xt: torch.Tensor, omega_r: torch.Tensor, omega_c: torch.Tensor, p: int, n: int,
                Lr: Csr, Lc: Csr, params: cpca_decode_params | None = None, want_X: bool = True,
                out: torch.Tensor | None = None, ws=None, check_status: bool = True, **kw):
    """Approximate decoder (Algorithm 2). Returns dict X, U, V, sigma, k, info, status."""
    _require_cuda(Xt, torch.float32, "Xt")
    rr, rc = Xt.shape if Xt.dim() == 2 else (0, 0)
    _require_matrix(Xt, rr, rc, "Xt")
    prm = params if params is not None else decode_params(**kw)
    dev = Xt.device
    kmax = prm.kmax
    X = (out if out is not None else torch.empty(p, n, dtype=torch.float32, device=dev)) if want_X else None
    if X is not None:
        _require_matrix(X, p, n, "out", Xt, host_ok=True)  # device, or pinned host (written in place)
    U = torch.empty(p, kmax, dtype=torch.float32, device=dev)
    V = torch.empty(n, kmax, dtype=torch.float32, device=dev)
    sig = torch.empty(kmax, dtype=torch.float64, device=dev)
    if ws is None:
        ws = _workspace(lib().cpca_decode_workspace_size(p, n, rr, rc, kmax, Lr.nnz, Lc.nnz), dev)
    k = C.c_int32(0)
    info = cpca_decode_info()
    lr, lc = Lr.c(), Lc.c()
    st = lib().cpca_decode(_ptr(Xt), rr, rc, Xt.stride(0), _ptr(omega_r), _ptr(omega_c), p, n,
                           C.byref(lr), C.byref(lc), C.byref(prm), _ptr(X),
                           X.stride(0) if X is not None else n, _ptr(U), _ptr(V), _ptr(sig),
                           C.byref(k), C.byref(info), _ptr(ws), ws.numel(), _stream())
    if check_status:
        _check(st)
    kk = k.value
    return {"X": X, "U": U[:, :kk], "V": V[:, :kk], "sigma": sig[:kk], "k": kk, "info": info,
            "status": st}


def cpca_cluster_decode(Xt: torch.Tensor, omega_c: torch.Tensor, n: int, Lc: Csr, k: int,
                        kmeans_iters: int = 100, seed: int = 0, cg_tol: float = 1e-6, cg_max_iter: int = 0,
                        want_C: bool = False, ws=None, check_status: bool = True):
    """Clustering decoder (Algorithm 3). Returns dict labels (n), labels_t
    (the k-means labels of Xt's columns), C (n x k or None), info, status."""
    _require_cuda(Xt, torch.float32, "Xt")
    rr, rc = Xt.shape
    dev = Xt.device
    prm = cpca_cluster_params(k, kmeans_iters, seed, cg_tol, cg_max_iter)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    labels_t = torch.empty(rc, dtype=torch.int32, device=dev)
    Cm = torch.empty(n, k, dtype=torch.float32, device=dev) if want_C else None
    if ws is None:
        ws = _workspace(lib().cpca_cluster_decode_workspace_size(rr, rc, n, k, Lc.nnz), dev)
    info = cpca_cluster_info()
    lc = Lc.c()
    st = lib().cpca_cluster_decode(_ptr(Xt), rr, rc, Xt.stride(0), _ptr(omega_c), n, C.byref(lc), C.byref(prm),
                                   _ptr(labels), _ptr(labels_t), _ptr(Cm), C.byref(info), _ptr(ws), ws.numel(),
                                   _stream())
    if check_status:
        _check(st)
    return {"labels": labels, "labels_t": labels_t, "C": Cm, "info": info, "status": st}


def cpca_subspace_project(side: int, basis: torch.Tensor, k: int, Y: torch.Tensor,
                          out: torch.Tensor | None = None, ws=None) -> torch.Tensor:
    """Approximate decoder 2 (side 0: X = U U^T Y, basis U p x ldb) or 3
    (side 1: X = Y V V^T, basis V n x ldb), first k basis columns."""
    _require_cuda(Y, torch.float32, "Y")
    _require_cuda(basis, torch.float32, "basis")
    p, n = Y.shape if Y.dim() == 2 else (0, 0)
    _require_matrix(Y, p, n, "Y")
    if basis.dim() != 2 or basis.stride(1) != 1 or basis.shape[0] != (p if side == 0 else n) \
            or basis.shape[1] < k:
        raise ValueError("basis must be row-major, (p or n) x (>= k)")
    ldb = basis.stride(0)
    X = out if out is not None else torch.empty(p, n, dtype=torch.float32, device=Y.device)
    _require_matrix(X, p, n, "out", Y)
    if ws is None:
        ws = _workspace(lib().cpca_subspace_project_workspace_size(p, n, ldb), Y.device)
    _check(lib().cpca_subspace_project(side, _ptr(basis), ldb, k, _ptr(Y), Y.stride(0), p, n, _ptr(X),
                                       X.stride(0), _ptr(ws), ws.numel(), _stream()))
    return X


def alt_params(gamma_r=1.0, gamma_c=1.0, tol=1e-6, max_iter=2000, blocks=0) -> cpca_alt_params:
    return cpca_alt_params(gamma_r, gamma_c, tol, max_iter, blocks)


def cpca_alternate_decode(Xt: torch.Tensor, omega_r: torch.Tensor, omega_c: torch.Tensor, p: int,
                          n: int, Lr: Csr, Lc: Csr, params: cpca_alt_params | None = None,
                          out: torch.Tensor | None = None, ws=None, check_status: bool = True, **kw):
    """Alternate decoder (Eq. alternatedecoder) by PCG on the full p x n
    matrix. Returns (X, info, status)."""
    _require_cuda(Xt, torch.float32, "Xt")
    rr, rc = Xt.shape if Xt.dim() == 2 else (0, 0)
    _require_matrix(Xt, rr, rc, "Xt")
    prm = params if params is not None else alt_params(**kw)
    X = out if out is not None else torch.empty(p, n, dtype=torch.float32, device=Xt.device)
    _require_matrix(X, p, n, "out", Xt)
    if ws is None:
        ws = _workspace(lib().cpca_alternate_decode_workspace_size(p, n), Xt.device)
    info = cpca_alt_info()
    lr, lc = Lr.c(), Lc.c()
    st = lib().cpca_alternate_decode(_ptr(Xt), rr, rc, Xt.stride(0), _ptr(omega_r), _ptr(omega_c), p, n,
                                     C.byref(lr), C.byref(lc), C.byref(prm), _ptr(X), X.stride(0),
                                     C.byref(info), _ptr(ws), ws.numel(), _stream())
    if check_status:
        _check(st)
    return X, info, st


def cpca_kron_reduce(L: Csr, omega: torch.Tensor, tol: float = 1e-6, max_iter: int = 0, want_csr: bool = True,
                     ws=None, check_status: bool = True):
    """Kron reduction of L onto the sampled nodes omega (Sec. IV-A).
    Returns dict Lt (rho x rho dense), csr (Csr with every entry stored, or
    None), info, status."""
    _require_cuda(L.val, torch.float32, "L.val")
    rho = omega.numel()
    dev = L.val.device
    Lt = torch.empty(rho, rho, dtype=torch.float32, device=dev)
    rp = col = val = None
    if want_csr:
        rp = torch.empty(rho + 1, dtype=torch.int64, device=dev)
        col = torch.empty(rho * rho, dtype=torch.int32, device=dev)
        val = torch.empty(rho * rho, dtype=torch.float32, device=dev)
    if ws is None:
        ws = _workspace(lib().cpca_kron_reduce_workspace_size(L.n, rho, L.nnz), dev)
    info = cpca_kron_info()
    lc = L.c()
    st = lib().cpca_kron_reduce(C.byref(lc), _ptr(omega), rho, tol, max_iter, _ptr(Lt), Lt.stride(0), _ptr(rp),
                                _ptr(col), _ptr(val), C.byref(info), _ptr(ws), ws.numel(), _stream())
    if check_status:
        _check(st)
    return {"Lt": Lt, "csr": Csr(rp, col, val) if want_csr else None, "info": info, "status": st}


def decode_backward_workspace(Xt: torch.Tensor, p: int, n: int, Lr: Csr, Lc: Csr,
                              params: cpca_decode_params) -> torch.Tensor:
    rr, rc = Xt.shape
    return _workspace(lib().cpca_decode_backward_workspace_size(p, n, rr, rc, params.kmax, Lr.nnz,
                                                                Lc.nnz), Xt.device)


def cpca_decode_backward(Xt: torch.Tensor, omega_r: torch.Tensor, omega_c: torch.Tensor, p: int,
                         n: int, Lr: Csr, Lc: Csr, k: int, h_row: torch.Tensor,
                         h_col: torch.Tensor, h_grad: torch.Tensor,
                         params: cpca_decode_params | None = None, want_dL: bool = True,
                         want_dw: bool = False, lap_type: int = LAP_NORMALIZED, ws=None,
                         resume: bool = False, **kw):
    """Reverse-mode derivative of cpca_decode (rank k fixed) for a loss of X
    at entries (h_row, h_col) with gradient h_grad there. Returns dict:
    dXt (rr x rc), dLr, dLc (FP64 per CSR entry or None), dwr, dwc (FP32 per
    CSR entry, needs Lr.weight / Lc.weight, or None). resume=True reuses the
    factors a cpca_decode call left in ``ws`` (decode_backward_workspace)."""
    _require_cuda(Xt, torch.float32, "Xt")
    _require_cuda(h_grad, torch.float32, "h_grad")
    prm = params if params is not None else decode_params(**kw)
    rr, rc = Xt.shape
    dev = Xt.device
    if resume and ws is None:
        raise ValueError("resume needs the forward's workspace")
    if ws is None:
        ws = decode_backward_workspace(Xt, p, n, Lr, Lc, prm)
    dXt = torch.empty(rr, rc, dtype=torch.float32, device=dev)
    dLr = torch.empty(Lr.nnz, dtype=torch.float64, device=dev) if want_dL else None
    dLc = torch.empty(Lc.nnz, dtype=torch.float64, device=dev) if want_dL else None
    dwr = dwc = None
    if want_dw:
        if Lr.weight is None or Lc.weight is None:
            raise ValueError("want_dw needs Lr.weight and Lc.weight")
        dwr = torch.empty(Lr.nnz, dtype=torch.float32, device=dev)
        dwc = torch.empty(Lc.nnz, dtype=torch.float32, device=dev)
    lr, lc = Lr.c(), Lc.c()
    nh = h_grad.numel()
    _check(lib().cpca_decode_backward(
        _ptr(Xt), rr, rc, Xt.stride(0), _ptr(omega_r), _ptr(omega_c), p, n, C.byref(lr),
        C.byref(lc), C.byref(prm), k, int(resume), nh, _ptr(h_row), _ptr(h_col), _ptr(h_grad), _ptr(dXt),
        dXt.stride(0), _ptr(dLr), _ptr(dLc), _ptr(Lr.weight) if want_dw else None,
        _ptr(Lc.weight) if want_dw else None, lap_type, _ptr(dwr), _ptr(dwc), _ptr(ws), ws.numel(),
        _stream()))
    return {"dXt": dXt, "dLr": dLr, "dLc": dLc, "dwr": dwr, "dwc": dwc}


def laplacian_values(pattern: Csr, w: torch.Tensor, lap_type: int = LAP_NORMALIZED) -> torch.Tensor:
    """Laplacian values (Sec. I) on ``pattern`` from edge weights w (per CSR
    entry, 0 on the diagonal)."""
    _require_cuda(w, torch.float32, "w")
    val = torch.empty(pattern.nnz, dtype=torch.float32, device=w.device)
    ws = _workspace(lib().cpca_laplacian_workspace_size(pattern.n), w.device)
    c = cpca_csr(pattern.n, pattern.nnz, pattern.rowptr.data_ptr(), pattern.col.data_ptr(), None)
    _check(lib().cpca_laplacian_values(C.byref(c), _ptr(w), lap_type, _ptr(val), _ptr(ws), ws.numel(),
                                       _stream()))
    return val


def laplacian_weight_grad(L: Csr, w: torch.Tensor, dL: torch.Tensor,
                          lap_type: int = LAP_NORMALIZED) -> torch.Tensor:
    """dloss/dw per CSR entry from dloss/dL (FP64 per entry) through the
    Laplacian-of-weights map of Sec. I."""
    _require_cuda(w, torch.float32, "w")
    _require_cuda(dL, torch.float64, "dL")
    dw = torch.empty(L.nnz, dtype=torch.float32, device=w.device)
    ws = _workspace(lib().cpca_laplacian_workspace_size(L.n), w.device)
    c = L.c()
    _check(lib().cpca_laplacian_weight_grad(C.byref(c), _ptr(w), _ptr(dL), lap_type, _ptr(dw), _ptr(ws),
                                            ws.numel(), _stream()))
    return dw


def decode_entries(U: torch.Tensor, V: torch.Tensor, sigma: torch.Tensor, k: int,
                   h_row: torch.Tensor, h_col: torch.Tensor) -> torch.Tensor:
    """X at the entries (h_row, h_col) from cpca_decode's U, V (row stride =
    kmax), sigma."""
    out = torch.empty(h_row.numel(), dtype=torch.float32, device=U.device)
    _check(lib().cpca_decode_entries(_ptr(U), _ptr(V), U.stride(0), _ptr(sigma), k, h_row.numel(),
                                     _ptr(h_row), _ptr(h_col), _ptr(out), _stream()))
    return out
