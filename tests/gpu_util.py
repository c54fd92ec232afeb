"""Helpers of the GPU tests: build once, move arrays to the device, compare with the oracle."""
import numpy as np

from paper_2106_03583_gb300 import build, snac

_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        _built = True


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().double().numpy()


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def plan(blocks, **kw):
    ensure_built()
    return snac.Plan(blocks, **kw)


def modes_from_planes(P):
    """Oracle planes (n_z, n_xy) -> the library's mode-space layout [q][cell] (identical order)."""
    return np.ascontiguousarray(P).ravel()
