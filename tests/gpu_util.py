"""Helpers shared by the GPU tests: run the CUDA path through the C ABI."""
import numpy as np

import paper_2105_12764_gb300 as mgr


def rel_linf(a, b):
    """Normwise relative L-infinity error max|a-b| / max|b| (coefficients can be ~0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def torch_dtype(dtype):
    import torch

    return torch.float64 if dtype == mgr.MGR_F64 else torch.float32


def np_dtype(dtype):
    return np.float64 if dtype == mgr.MGR_F64 else np.float32


class Runner:
    """Plan + device buffers for one (shape, coords, levels, dtype, prec)."""

    def __init__(self, ctx, shape, coords=None, levels=-1, dtype=mgr.MGR_F64, prec=mgr.MGR_PREC_NATIVE):
        import torch

        self.plan = mgr.Plan(ctx, shape, coords, levels, dtype, prec)
        self.shape = tuple(shape)
        self.td = torch_dtype(dtype)
        self.nd = np_dtype(dtype)
        self.ws = torch.empty(max(self.plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
        self.a = torch.empty(self.shape, dtype=self.td, device="cuda")
        self.b = torch.empty(self.shape, dtype=self.td, device="cuda")

    def decompose(self, u, inplace=False):
        import torch

        self.a.copy_(torch.from_numpy(np.ascontiguousarray(u, dtype=self.nd)))
        dst = self.a if inplace else self.b
        self.plan.decompose(self.a, dst, self.ws)
        torch.cuda.synchronize()
        return dst.cpu().numpy()

    def recompose(self, c, inplace=False):
        import torch

        self.a.copy_(torch.from_numpy(np.ascontiguousarray(c, dtype=self.nd)))
        dst = self.a if inplace else self.b
        self.plan.recompose(self.a, dst, self.ws)
        torch.cuda.synchronize()
        return dst.cpu().numpy()

    def close(self):
        self.plan.close()
