"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import torch


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def max_order_rel(X, ref) -> float:
    """max over batch and order of ||X_k - ref_k||_F / ||ref_k||_F."""
    X = np.asarray(X)
    ref = np.asarray(ref)
    num = np.sqrt(np.sum(np.abs(X - ref) ** 2, axis=(-1, -2)))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-1, -2)))
    return float(np.max(num / np.where(den == 0, 1.0, den)))
