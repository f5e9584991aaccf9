"""Helpers shared by the GPU tests: device tensors and mask packing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def stream():
    return torch.cuda.current_stream().cuda_stream


def pack_masks(masks):
    """bool [B, n] -> uint32 [B, ceil(n/32)] with bit i%32 of word i/32 = node i."""
    masks = np.atleast_2d(masks)
    B, n = masks.shape
    nw = (n + 31) // 32
    bits = np.zeros((B, nw * 32), dtype=np.uint8)
    bits[:, :n] = masks
    return np.packbits(bits, axis=1, bitorder="little").view("<u4").reshape(B, nw)


def unpack_masks(words, n):
    words = np.ascontiguousarray(np.atleast_2d(words).astype("<u4"))
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :n].astype(bool)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()
