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
