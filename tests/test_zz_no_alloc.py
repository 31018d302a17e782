"""The allocation-free matching entry point agrees with amg_setup's own first
matching sweep.

amg_match_noalloc exists for callers that may not allocate device memory
when they need a matching (during CUDA-graph stream capture, or under an
external memory pool or budget); it works in a fixed scratch array inside the
library. Matchings are compared bit for bit, like every matching test here.
The calls are made back to back on different inputs and then repeated, so a
stale counter or list left in the shared scratch array by the previous call
would show up as a mismatch. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import dev, setup

pytestmark = pytest.mark.gpu


def _reference_mate(A, w):
    from paper_2006_16147_gb300 import amg
    h = setup(A, w, keep_sweeps=1, max_coarse=1, match_kernel=1)
    m = amg.amg_export_sweep(h, 0, 0)["mate"]
    rounds = amg.amg_hierarchy_info(h)["rounds"][0][0]
    h.close()
    return m, rounds


def _noalloc_mate(A, w):
    import torch
    from paper_2006_16147_gb300 import amg
    mate = torch.full((A.n,), 7, dtype=torch.int32, device="cuda:0")
    rounds = amg.amg_match_noalloc(dev(A.row_ptr), dev(A.col), dev(A.val), dev(w), mate)
    torch.cuda.synchronize()
    return mate.cpu().numpy(), rounds


def test_noalloc_matching_equals_setup_sweep_on_consecutive_calls():
    rng = np.random.default_rng(11)
    inputs = [
        (W.poisson3d(32), np.ones(32 ** 3)),
        (W.random_spd(3000, 0.003, 5), None),
        (W.varcoef3d(20, seed=4), np.ones(20 ** 3)),
    ]
    inputs[1] = (inputs[1][0], rng.uniform(0.5, 2.0, 3000) * rng.choice([-1.0, 1.0], 3000))
    refs = [_reference_mate(A, w) for A, w in inputs]
    # two passes over the inputs: every call follows a call on a different matrix
    for _ in range(2):
        for (A, w), (ref, ref_rounds) in zip(inputs, refs):
            got, rounds = _noalloc_mate(A, w)
            assert np.array_equal(got, ref)
            assert rounds == ref_rounds


def test_noalloc_rejects_sizes_beyond_the_limit():
    from paper_2006_16147_gb300 import amg
    A = W.poisson3d(41)                      # n = 68921 > 65536
    assert A.n > amg.NOALLOC_MAX_N
    import torch
    mate = torch.empty(A.n, dtype=torch.int32, device="cuda:0")
    with pytest.raises(amg.AmgError) as e:
        amg.amg_match_noalloc(dev(A.row_ptr), dev(A.col), dev(A.val), dev(np.ones(A.n)), mate)
    assert e.value.status == -8
