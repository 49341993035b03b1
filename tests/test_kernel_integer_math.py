"""Integer identities the DAS kernels rely on, checked exhaustively on the host (no GPU).

* The staging conversion numbers a stage's (trace row, 8-sample segment) pairs row-major and
  recovers the row of pair i as (i * ceil(2^16 / n)) >> 16 for a window of n segments
  (n <= 64: a staged window holds at most 512 samples).
* The reverse kernel's window flush recovers the row of cell i as (i * ceil(2^20 / n)) >> 20
  for rows of n <= 129 four-sample cells.
* int16 samples become floats exactly by the exponent-bias add: the bits 0x4B400000 + v
  are 1.5 * 2^23 + v for |v| < 2^22, so subtracting 1.5 * 2^23 leaves v.
"""
import numpy as np


def test_row_of_segment_pair_by_multiply_shift():
    for n in range(1, 65):
        m = -(-65536 // n)
        i = np.arange(8 * n + 256, dtype=np.int64)
        assert np.array_equal((i * m) >> 16, i // n), n
        assert int(i[-1]) * m < 2**32          # the 32-bit product cannot wrap


def test_row_of_flush_cell_by_multiply_shift():
    for n in range(1, 140):
        m = -(-(1 << 20) // n)
        i = np.arange(8 * n + 8, dtype=np.int64)
        assert np.array_equal((i * m) >> 20, i // n), n
        assert int(i[-1]) * m < 2**32


def test_int16_exponent_bias_conversion_is_exact():
    v = np.arange(-32768, 32768, dtype=np.int32)
    f = (np.int32(0x4B400000) + v).view(np.float32)
    assert np.array_equal(f - np.float32(12582912.0), v.astype(np.float32))
