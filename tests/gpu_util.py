"""Helpers of the GPU parity tests: build contexts, move arrays, call the oracle."""
import numpy as np

from oracle.lattice import to_grid


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def fields(arr, dims, nc):
    V = int(np.prod(dims))
    return [to_grid(np.asarray(a).reshape(V, nc), dims) for a in arr]


def ext(fields_list):
    """list of (T,Z,Y,X,nc) -> external [n][V][nc]"""
    return np.ascontiguousarray(np.stack([f.reshape(-1, f.shape[-1]) for f in fields_list]))
