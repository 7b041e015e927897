"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_bf16_f64(x: np.ndarray) -> np.ndarray:
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).to(
        torch.float64).numpy()


DTYPES = {0: "float32", 1: "bfloat16", 2: "float64"}


def dev_tensor(x: np.ndarray, prec: int):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    return t.to(getattr(torch, DTYPES[prec])).cuda()


def host_values(t) -> np.ndarray:
    return t.detach().to("cpu").to(dtype=__import__("torch").float64).numpy()


def max_rel(a, b) -> float:
    """Largest element error relative to the largest reference element."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mb = float(np.max(np.abs(b))) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (mb if mb > 0 else 1.0)) if b.size else 0.0


def assert_close(got, ref, tol, elem=None):
    """Relative L2 error within `tol`, and every element within `elem` of
    the largest reference magnitude (default: tol for the FP32/FP64
    tolerances; 2^-6 for the bf16 ones, one bf16 unit of the largest element
    plus rounding), so that an error confined to a few elements (a ragged
    tile tail, one detector edge) cannot hide in the norm."""
    if elem is None:
        elem = tol if tol <= 1e-5 else 2.0 ** -6
    e2, em = rel(got, ref), max_rel(got, ref)
    assert e2 <= tol and em <= elem, "rel L2 %.3e (tol %.1e), max elem %.3e (tol %.1e)" % (e2, tol, em, elem)
