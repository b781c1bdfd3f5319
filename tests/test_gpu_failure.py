"""The failure path of the tensor-core apply, made to run on the GPU without a fault.

Every wait of the split kernel is bounded (about two seconds of SM clock) and gives up when the
other warpgroup has aborted; the CTA then waits (bounded) for its own copies and MMAs, frees its
tensor memory and sets an error word that the host turns into MRA_ERR_TIMEOUT.  The test hook
mra_debug_inject_stall makes the first CTA of the next split apply skip the block copies of its
first term, so that those waits run out; the call must report MRA_ERR_TIMEOUT and the next apply
must give the normal result on the same context.
"""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    import torch
    assert torch.cuda.is_available()
    from paper_1507_01888_gb300 import mra as m
    m.load()
    return m


@pytest.mark.parametrize("kern,tile_variant", [(0, 0), (1, 0), (1, 2)])
def test_split_wait_runs_out_and_the_context_survives(mra, kern, tile_variant):
    """Both kernels: the source-stationary one (k = 6 here) and the destination-stationary one's
    four-tile and one-tile shapes."""
    f = W.gaussian_sum(2, 1.0, 20.0, seed=41, centre_box=3.0)
    keys, coeffs, _ = O.project(f, 6, 8.0, uniform_level=2)
    op = mra.Operator(mra.POISSON, 8, 6, 8.0, 2, 2, max_disp=1, fit_eps=1e-4)
    opts = mra.make_opts(precision=mra.PREC_SPLIT_BF16, stencil=mra.STENCIL_NEAREST, tile_variant=tile_variant,
                         split_kernel=kern)
    tree = mra.Tree.from_host(keys, coeffs, 8.0)
    ref, _ = mra.apply(op, tree, opts)
    mra.debug_inject_stall()
    t0 = time.perf_counter()
    with pytest.raises(mra.MraError) as e:
        mra.apply(op, tree, opts)
    assert e.value.code == mra.MRA_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    out, _ = mra.apply(op, tree, opts)  # the same context, no injection: the normal result
    assert (out.host()[0] == ref.host()[0]).all()
    assert np.array_equal(out.host()[1], ref.host()[1])
