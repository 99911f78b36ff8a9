"""Helpers for GPU parity tests: move uint64 arrays to/from torch int64 tensors."""
import numpy as np
import torch


def dev(a):
    """numpy uint64/int64 array -> CUDA int64 tensor with the same bits."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a.copy()).cuda()


def host(t):
    """CUDA int64 tensor -> numpy uint64 array with the same bits."""
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().view(np.uint64)


def dev_f64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def unpack_bits(words, n):
    """[P][ceil(n/64)] packed words -> [P][n] uint64 of 0/1."""
    w = np.asarray(words, dtype=np.uint64)
    P = w.shape[0]
    idx = np.arange(n)
    return ((w[:, idx // 64] >> (idx % 64).astype(np.uint64)) & np.uint64(1)).reshape(P, n)
