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
