"""The allocation-free matching entry point (amg_match_noalloc) against the
oracle's greedy matching and against amg_setup's own first matching sweep.

amg_match_noalloc exists for callers that may not allocate device memory
when they need a matching: applications that reserve all device memory at
start-up for their own pool or budget, and hosts that forbid allocation after
start-up (cudaMalloc can synchronise the device). It works in a fixed scratch
array inside the library. Matchings are compared bit for bit, like every
matching test here. The calls are made back to back on different inputs and
then repeated, so a stale counter or list left in the shared scratch array by
the previous call would show up as a mismatch. The device's default memory
pool (where the library's stream-ordered allocations come from) and torch's
allocator are read before and after the calls: neither may grow. This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import dev, setup

pytestmark = pytest.mark.gpu

_RESERVED_CURRENT, _USED_CURRENT, _USED_HIGH = 0x5, 0x7, 0x8   # cudaMemPoolAttr values (driver_types.h)


def _cudart():
    for line in open("/proc/self/maps"):
        path = line.split()[-1]
        if "libcudart.so" in path:
            return ctypes.CDLL(path)
    return ctypes.CDLL("libcudart.so")


class _DefaultPool:
    """Reads the attributes of the current device's default memory pool."""

    def __init__(self):
        import torch
        self.rt = _cudart()
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), torch.cuda.current_device()) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, _USED_HIGH, ctypes.byref(z)) == 0


def _reference_mate(A, w):
    from paper_2006_16147_gb300 import amg
    h = setup(A, w, keep_sweeps=1, max_coarse=1, match_kernel=1)
    m = amg.amg_export_sweep(h, 0, 0)["mate"]
    rounds = amg.amg_hierarchy_info(h)["rounds"][0][0]
    h.close()
    return m, rounds


def _inputs():
    rng = np.random.default_rng(11)
    A1 = W.random_spd(3000, 0.003, 5)
    w1 = rng.uniform(0.5, 2.0, 3000) * rng.choice([-1.0, 1.0], 3000)
    return [(W.poisson3d(32), np.ones(32 ** 3)), (A1, w1), (W.varcoef3d(20, seed=4), np.ones(20 ** 3))]


def test_noalloc_matching_equals_oracle_and_setup_sweep_without_allocating(orc):
    import torch
    from paper_2006_16147_gb300 import amg
    inputs = _inputs()
    oracle_mates = [orc.match_greedy(A, w) for A, w in inputs]
    refs = [_reference_mate(A, w) for A, w in inputs]
    # device copies of every input and output before any measurement
    args = [(dev(A.row_ptr), dev(A.col), dev(A.val), dev(w)) for A, w in inputs]
    mates = [torch.full((A.n,), 7, dtype=torch.int32, device="cuda:0") for A, _ in inputs]
    amg.amg_match_noalloc(*args[0], mates[0])        # first call on this device: looks up the array
    torch.cuda.synchronize()
    pool = _DefaultPool()
    used0, reserved0 = pool.get(_USED_CURRENT), pool.get(_RESERVED_CURRENT)
    torch_alloc0 = torch.cuda.memory_allocated()
    pool.reset_high()
    # two passes over the inputs: every call follows a call on a different matrix
    for _ in range(2):
        for a, m, om, (ref, ref_rounds) in zip(args, mates, oracle_mates, refs):
            m.fill_(7)
            rounds = amg.amg_match_noalloc(*a, m)
            torch.cuda.synchronize()
            got = m.cpu().numpy()
            assert np.array_equal(got, np.where(om >= 0, om, -1))
            assert np.array_equal(got, ref)
            assert rounds == ref_rounds
    torch.cuda.synchronize()
    assert pool.get(_USED_CURRENT) == used0
    assert pool.get(_RESERVED_CURRENT) == reserved0
    assert pool.get(_USED_HIGH) <= used0
    assert torch.cuda.memory_allocated() == torch_alloc0


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    from paper_2006_16147_gb300 import amg
    A = W.poisson3d(41)                      # n = 68921 > 65536
    assert A.n > amg.NOALLOC_MAX_N
    mate = torch.empty(A.n, dtype=torch.int32, device="cuda:0")
    with pytest.raises(amg.AmgError) as e:
        amg.amg_match_noalloc(dev(A.row_ptr), dev(A.col), dev(A.val), dev(np.ones(A.n)), mate)
    assert e.value.status == -8
