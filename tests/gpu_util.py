"""Helpers shared by the GPU tests: host <-> device layout conversions only."""
import numpy as np


def torch():
    import torch as _t
    return _t


def dev_matrix(X: np.ndarray, dtype="f32", ld=None):
    """n x d host array -> row-major CUDA tensor (optionally with a padded leading dimension)."""
    t = torch()
    n, d = X.shape
    ld = d if ld is None else ld
    tdt = {"f32": t.float32, "bf16": t.bfloat16}[dtype]
    buf = t.zeros((n, ld), dtype=tdt, device="cuda")
    buf[:, :d] = t.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to("cuda").to(tdt)
    return buf[:, :d] if ld != d else buf


def stored_f64(Xdev):
    """The exact stored values of a device matrix as float64 on the host."""
    t = torch()
    return Xdev.to(t.float32).cpu().numpy().astype(np.float64)


def dev_basis(V: np.ndarray):
    """d x m host basis -> (m, d) contiguous float32 CUDA tensor (d x m column-major)."""
    t = torch()
    return t.from_numpy(np.ascontiguousarray(V.T, dtype=np.float32)).to("cuda")


def host_basis(Vt) -> np.ndarray:
    """(m, d) CUDA tensor -> d x m float64 host array."""
    return Vt.double().cpu().numpy().T.copy()


def empty_basis(d, m):
    t = torch()
    return t.empty((m, d), dtype=t.float32, device="cuda")


def normwise(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
