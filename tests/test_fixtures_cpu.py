"""The per-block field check used by the GPU build tests (no GPU): single-precision rounding of
an oracle field passes it, and an error planted in a block much smaller than its node fails it
although the node-wide relative error stays below the single-precision bound."""
import numpy as np

from tests import _fixtures as X


def test_block_check_passes_rounding_and_catches_a_small_wrong_block():
    ref = X.room_field_oracle(True)
    nz = X.fro(ref.reshape(-1, 60, 6)) > 0
    ref = ref[nz]
    rounded = X.unpack_field(X.pack_field(ref))
    assert X.block_ratio(rounded, ref, X.TAU_F32).max() <= 1.0
    # the smallest block (relative to its node) of the node where it is smallest
    bk = X.fro(ref)                                            # [N, 10]
    rel = bk / np.sqrt((bk ** 2).sum(axis=1, keepdims=True))
    n, k = np.unravel_index(np.argmin(np.where(rel > 0, rel, np.inf)), rel.shape)
    assert rel[n, k] < 0.05
    bad = rounded.copy()
    bad[n, k] *= 1.0 + 1e-4          # 10x the bound inside the block
    assert X.rel_fro(bad.reshape(-1, 60, 6), ref.reshape(-1, 60, 6))[n] <= X.TAU_F32
    assert X.block_ratio(bad, ref, X.TAU_F32)[n, k] > 1.0


def test_record_layouts_round_trip():
    """float32 records: entry e of C_k at 21 k + e (stride 216); bfloat16 records: at 22 k + e with
    zeros at 22 k + 21 and 220..223 (stride 224)."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5, 10, 6, 6))
    A = A + A.transpose(0, 1, 3, 2)
    for stride, blk in ((216, 21), (224, 22)):
        buf = X.pack_field(A, stride)
        assert buf.shape == (5, stride)
        np.testing.assert_array_equal(X.unpack_field(buf), A.astype(np.float32).astype(np.float64))
        k, e = 3, 7                                     # entry 7 = (row 1, col 2)
        assert buf[2, blk * k + e] == np.float32(A[2, k, 1, 2])
        assert not buf[:, 10 * blk:].any()
        if blk == 22:
            assert not buf[:, 21:220:22].any()
