"""Shared helpers of the GPU tests: device datasets and numpy views of tensors."""
import numpy as np


def ctx():
    from paper_2311_06952_gb300 import deoct
    return deoct.Context(0)


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def u16(t):
    return t.cpu().numpy().view(np.uint16)


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_dataset(c, X, y, K, rank_bytes):
    from paper_2311_06952_gb300 import deoct
    return deoct.encode_dataset(c, to_dev(np.ascontiguousarray(X, np.float32)), to_dev(y.astype(np.uint8)),
                                K, rank_bytes)


def ranks_np(ds):
    """[F][n] uint32 view of a device dataset's ranks (padding columns dropped)."""
    r = u16(ds.ranks) if ds.rank_bytes == 2 else u32(ds.ranks)
    return r[:, : ds.n].astype(np.uint32)
