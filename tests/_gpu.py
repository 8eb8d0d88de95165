"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import torch

TOL = {"fp64": 1e-10, "mixed": 1e-5}       # relative tolerances of the FP64 and mixed forms
NP_DT = {"fp64": np.complex128, "mixed": np.complex64}


def to_dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x.astype(NP_DT[prec]))).cuda()


def to_host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


class Gathered:
    """Read-only view of a device state that fetches only the indexed entries,
    so the oracle's row-definition product can run on sampled rows of a state
    too large for host memory."""

    def __init__(self, t):
        self.t = t

    def __getitem__(self, idx):
        i = torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(self.t.device)
        return self.t[i].cpu().numpy().astype(np.complex128)


def seeded_device_state(L, seed, prec):
    """Seeded complex Gaussian state drawn on the device (for sizes whose host
    copy would be too large), normalised."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    re = torch.randn(1 << L, generator=g, device="cuda", dtype=dt)
    im = torch.randn(1 << L, generator=g, device="cuda", dtype=dt)
    z = torch.complex(re, im)
    z /= torch.linalg.vector_norm(z)
    return z
