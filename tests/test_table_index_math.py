"""The hub-cost table fill of the allocation kernels finds the row k = e / hst
of table entry e (hst = p | 1, the odd row stride) without an integer
division: k from the float32 product (e + 0.5) * RN(1 / hst), then one
correction step either way.  This checks, for every p the library accepts
(1..255) and every entry of its table, that the product is never off by more
than one row, so the single correction always lands on e // hst -- the same
float32 operations in the same order, emulated with NumPy."""
import numpy as np


def _hstride(p):
    return p | 1


def _cstride(p):
    return (p * _hstride(p) + 3) // 4 * 4


def test_row_of_every_table_entry_is_exact_for_every_p():
    for p in range(1, 256):
        hst, cst = _hstride(p), _cstride(p)
        e = np.arange(cst, dtype=np.int64)
        inv = np.float32(1.0) / np.float32(hst)
        prod = (e.astype(np.float32) + np.float32(0.5)) * inv          # two float32 roundings
        k = prod.astype(np.int64)                                      # truncation, prod >= 0
        exact = e // hst
        assert np.abs(k - exact).max() <= 1, p
        # the kernel's correction step
        l = e - k * hst
        k = np.where(l < 0, k - 1, np.where(l >= hst, k + 1, k))
        l = e - k * hst
        assert (k == exact).all() and (l >= 0).all() and (l < hst).all(), p
