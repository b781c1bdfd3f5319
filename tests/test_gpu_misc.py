"""mra_scale (the constant factors of the bound-state Helmholtz iteration, Sec. 3.2) and the FP64
throughput probe behind the FP64 apply's roofline."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


def test_scale_multiplies_every_coefficient(mra):
    import torch
    keys, coeffs = W.random_tree_coeffs(120, 6, 3, seed=21)
    t = mra.Tree.from_host(keys, coeffs, 8.0)
    ref = t.coeffs[: t.n].clone() * (-1.0 / (2.0 * 3.141592653589793))
    mra.scale(t, -1.0 / (2.0 * 3.141592653589793))
    torch.testing.assert_close(t.coeffs[: t.n], ref, rtol=0.0, atol=0.0)
    empty = mra.Tree.empty(2, 6, 8.0)
    mra.scale(empty, 3.0)  # no boxes: nothing to do
    with pytest.raises(mra.MraError):
        mra.scale(t, float("nan"))


def test_fp64_probe_rates_are_plausible(mra):
    """Both probes report a positive rate below the nominal FP64 figures of this part by far
    (a probe whose arithmetic was optimised away would report an absurd rate)."""
    dfma, dmma = mra.measure_fp64_peak(0.8)
    assert 0.05 < dfma < 10.0
    assert 0.05 < dmma < 100.0
