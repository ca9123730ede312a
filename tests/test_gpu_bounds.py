"""The certificate's binary32 bounds (Thm proofRoots needs upper bounds of
|z| and |p'| along the disk orbit; Thm diskArithmetic's radii are upper
bounds): the square-root bound sqrt.approx.f32 x (1 + 2^-19), rounded
upward, is checked against the exact square root over every normal
binary32 on the GPU at hand."""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as m
    m.load()
    return m


def test_sqrt_upper_bound_holds_for_every_binary32(mt):
    n_fail, max_rel = mt.check_sqrt_up()
    assert n_fail == 0
    # the approximation's own error leaves the 2^-19 factor a wide margin
    assert 0.0 < max_rel < 2.0 ** -21, max_rel
