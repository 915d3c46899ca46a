"""md_philox_static: the allocation-free variant of md_philox, whose device
staging buffers are a static array inside the library.  Collected last, so it
also runs after every other test has used the device.

Philox blocks are integers: the bar is bit-exact agreement with md_philox.
"""
import numpy as np
import pytest


def counters(n, seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= (1 << 30) - 1      # within the counter range the cuRAND mapping reaches
    return ctr


def test_size_beyond_static_scratch_is_rejected_on_the_host():
    """n > MD_PHILOX_STATIC_MAX fails with MD_ETOOLARGE before any CUDA call."""
    from paper_2205_14121_gb300 import build as B
    B.build()
    import paper_2205_14121_gb300._binding as Bd
    with pytest.raises(Bd.MdError) as e:
        Bd.md_philox_static(np.zeros((Bd.MD_PHILOX_STATIC_MAX + 1, 4), np.uint32), [1, 2])
    assert e.value.code == -8 and "static scratch" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("use_library", [False, True])
def test_static_scratch_matches_allocating_entry_point(use_library):
    """Two calls in a row (the second shorter, so the first call's contents stay
    in the array beyond its n), then the largest size; each bit-exact with
    md_philox on the same counters."""
    from paper_2205_14121_gb300._binding import MD_PHILOX_STATIC_MAX, md_philox, md_philox_static
    key = np.array([0x9E3779B9, 0x1234ABCD], np.uint32)
    for n, seed in ((5000, 1), (3001, 2), (MD_PHILOX_STATIC_MAX, 3)):
        ctr = counters(n, seed)
        ref = md_philox(ctr, key, use_library=use_library)
        got = md_philox_static(ctr, key, use_library=use_library)
        assert np.array_equal(got, ref), f"n={n}: {np.argwhere(got != ref)[:4]}"
