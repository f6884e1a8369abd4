"""zolo_solve_noalloc -- the block solve for callers that must not allocate device memory
on repeated calls (hosts whose device memory belongs to another component, allocation-free
loops) -- gives the same result as
zolo_solve, on two calls in a row with different right-hand sides.  Kept in a file that
pytest collects last."""
import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from gpu_common import case, colrel, dev, host, need_gpu
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["cplx3d_9", "real2d_40"])
def test_noalloc_solve_matches_solve(name):
    need_gpu()
    import torch
    pen, leaf, gaps, lam = case(name)
    fac = Z.Factor(pen.A, pen.B, Z.Filter(*gaps, 2, 2), opts=Z.default_opts(grid=pen.dims, leaf_max=leaf))
    k = 12
    B1 = dev(synth.random_block(pen.n, k, 31))
    B2 = dev(synth.random_block(pen.n, k, 32))
    for pole in range(2):
        for herm in (False, True):
            ref1 = host(fac.solve(pole, B1, herm=herm))          # set-up call: builds the schedule for k
            ref2 = host(fac.solve(pole, B2, herm=herm))
            out = torch.empty_like(B1)
            got1 = host(fac.solve_noalloc(pole, B1, out, herm=herm))
            got2 = host(fac.solve_noalloc(pole, B2, out, herm=herm))
            assert colrel(got1, ref1) < 1e-12
            assert colrel(got2, ref2) < 1e-12


def test_noalloc_rejects_what_it_cannot_do():
    need_gpu()
    import torch
    pen, leaf, gaps, lam = case("cplx3d_9")
    fac = Z.Factor(pen.A, pen.B, Z.Filter(*gaps, 2, 2), opts=Z.default_opts(grid=pen.dims, leaf_max=leaf))
    B = dev(synth.random_block(pen.n, 5, 1))
    with pytest.raises(Z.ZoloError) as e:                    # no schedule for k = 5 yet
        fac.solve_noalloc(0, B, torch.empty_like(B))
    assert e.value.status == Z.EINVAL
    mixed = Z.Factor(pen.A, pen.B, Z.Filter(*gaps, 2, 2),
                     opts=Z.default_opts(grid=pen.dims, leaf_max=leaf, precision=Z.PREC_MIXED))
    mixed.solve(0, B)
    with pytest.raises(Z.ZoloError) as e:
        mixed.solve_noalloc(0, B, torch.empty_like(B))
    assert e.value.status == Z.EINVAL
    big = dev(synth.random_block(pen.n, 4000, 2))            # workspace beyond the fixed array
    fac.solve(0, big)
    with pytest.raises(Z.ZoloError) as e:
        fac.solve_noalloc(0, big, torch.empty_like(big))
    assert e.value.status == Z.EINVAL
