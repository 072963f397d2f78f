"""GPU parity of the synthetic divergent kernels (both forms) against the
oracle, bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("pattern", ["SB1", "SB2", "SB3", "SB4", "SB1-R", "SB2-R", "SB3-R",
                                     "SB4-R"])
@pytest.mark.parametrize("iters,rounds", [(0, 3), (1, 1), (3, 5), (7, 16)])
def test_matches_oracle(darm, pattern, variant, iters, rounds):
    import torch
    data = synth.uniform_u32(900 + iters * 17 + rounds, 1024 * 37)
    expect = oracle.sb_run(pattern, data, iters, rounds)
    d = to_dev(data)
    darm.sb_run(pattern, d, iters, rounds, variant=variant)
    torch.cuda.synchronize()
    assert_equal(f"{pattern} {variant}", d.cpu().numpy(), expect)


def test_bad_arguments(darm):
    d = to_dev(np.zeros(1024, np.uint32))
    with pytest.raises(KeyError):
        darm.sb_run("SB9", d, 1, 1)
    with pytest.raises(darm.DarmError):
        darm.sb_run("SB1", d, -1, 1)
