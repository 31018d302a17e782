"""Helpers shared by the GPU tests: move generated inputs to the device and
run the library through its C ABI."""
import numpy as np


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def setup(A, w=None, **opts):
    from paper_2006_16147_gb300 import amg
    w = np.ones(A.n) if w is None else w
    return amg.amg_setup(dev(A.row_ptr), dev(A.col), dev(A.val), dev(w), **opts)


def solve(h, b, x0=None, rtol=1e-6, maxit=1000):
    import torch
    from paper_2006_16147_gb300 import amg
    x = dev(np.zeros_like(b) if x0 is None else x0)
    info = amg.amg_solve(h, dev(b), x, rtol=rtol, maxit=maxit)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


def vcycle(h, r):
    import torch
    from paper_2006_16147_gb300 import amg
    z = torch.empty(len(r), dtype=torch.float64, device="cuda:0")
    amg.amg_vcycle(h, dev(r), z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


def assert_same_solution(H, b, xg, ig, xo, io, flexible=False, tol=1e-10):
    """The GPU solution equals the oracle's to `tol` relative, whatever the
    iteration counts. When the counts differ (by one, near the stop test),
    the oracle is run again for exactly the GPU's number of iterations
    (rtol = 0 never stops it earlier), so the same iterate is compared."""
    ref = xo
    if ig["iterations"] != io["iterations"]:
        ref, _ = H.pcg(b, rtol=0.0, maxit=ig["iterations"], flexible=flexible)
    assert np.linalg.norm(xg - ref) <= tol * np.linalg.norm(ref), (ig["iterations"], io["iterations"])
