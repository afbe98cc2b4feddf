"""The oracle against what the paper and the mathematics fix (CPU only)."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    err, tol = pin(orc)
    assert err <= tol, f"{pin.__name__}: error {err:.3e} > {tol:.1e}"


def test_batch_matches_single(orc):
    """The threaded batch driver returns exactly the single-translation results."""
    import numpy as np
    from paper_2202_02847_gb300 import workloads as W
    g = W.rng(5)
    C = W.random_solids(g, 37, 6)
    sh = W.shifts(g, 37)
    out, used = orc.batch("m2l", 6, 7, C, sh, nthreads=3)
    assert used >= 1
    for i in (0, 17, 36):
        assert np.array_equal(out[i], orc.translate("m2l", 6, 7, C[i], sh[i]))
    acc = np.ones_like(out)
    orc.batch("m2l", 6, 7, C, sh, out=acc, accumulate=True)
    assert np.allclose(acc - 1.0, out, rtol=0, atol=1e-15 * np.abs(out).max())
