"""Helpers for the GPU tests: move column-major numpy inputs to the device and adapt the CUDA
path to the ``compress(X, tol, d_max, start, mode)`` interface the pins use."""
import numpy as np
import torch


def to_device(X: np.ndarray, dtype=torch.float64, device="cuda:0") -> torch.Tensor:
    """Column-major (m x n) numpy array -> column-major CUDA tensor."""
    X = np.asarray(X)
    if X.ndim == 1:
        X = X[:, None]
    t = torch.from_numpy(np.ascontiguousarray(X.T)).to(device=device, dtype=dtype)
    return t.t()


def to_numpy(t: torch.Tensor) -> np.ndarray:
    return np.asfortranarray(t.detach().to("cpu", torch.float64).numpy())


def gpu_compress(X, tol, d_max, start=0, mode="maxcol_abs", dtype=torch.float64, weights=None):
    import paper_1503_05947_gb300 as rbd

    w = None
    if weights is not None:
        w = torch.as_tensor(np.ascontiguousarray(weights, dtype=np.float64), device="cuda:0")
    r = rbd.compress(to_device(X, dtype), tol, d_max, start=start, tol_mode=mode, weights=w)
    return {"Y": to_numpy(r.Y), "T": to_numpy(r.T), "pivots": r.pivots.cpu().numpy(),
            "err": r.err.cpu().numpy(), "nu": r.nu.cpu().numpy(), "d": r.d, "next_pivot": r.next_pivot,
            "fro": None, "result": r}
