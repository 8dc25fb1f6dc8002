"""Helpers shared by the GPU parity tests (host <-> device marshalling only)."""
import numpy as np


def to_dev(Xh, dtype=None):
    """Host column-major numpy matrix -> column-major (m, n) CUDA tensor view."""
    import torch

    Xh = np.asarray(Xh)
    if Xh.ndim == 1:
        Xh = Xh.reshape(-1, 1)
    t = torch.from_numpy(np.ascontiguousarray(Xh.T))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().T


def to_host(R):
    import torch

    torch.cuda.synchronize()
    return R.detach().cpu().numpy()


def info_of(info):
    import torch

    torch.cuda.synchronize()
    return [int(v) for v in info.cpu().tolist()]
