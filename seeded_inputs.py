"""Seeded synthetic inputs shared by the FP64 oracle and the GPU path.

This module holds no arithmetic of the method (no Hamiltonian, no Krylov
step, no measurement).  It only draws seeded random numbers and names the
workload parameters, so both sides of a parity test receive the *same data*
without sharing code that computes anything the paper defines.

Conventions (state layout of the rank-L tensor view, Sec. IV "row-major"
ordering of the paper):
  * basis index b in [0, 2^L); site k (1-based) is bit L-k, so site 1 is the
    most significant bit.
  * bit value 0 = spin up (sigma^z = +1).  The all-up product state is b = 0.
  * Neel state: site 1 up, site 2 down, ... (bits of the even sites set).
"""
from __future__ import annotations

import numpy as np


def neel_index(L: int) -> int:
    """Basis index of the Neel product state (site 1 up, alternating)."""
    b = 0
    for k in range(2, L + 1, 2):
        b |= 1 << (L - k)
    return b


def all_up_index(L: int) -> int:
    """Basis index of the all-up product state."""
    return 0


def gaussian_state(L: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded complex Gaussian vector of length 2^L, normalised to 1.

    Re and Im parts are iid N(0,1) draws from numpy's Philox-4x32-10
    counter-based generator, so the draw depends only on (L, seed).  The
    normalised vector is Haar-distributed on the unit sphere, which is also
    the random state used for Page-value checks.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    D = 1 << L
    v = rng.standard_normal(2 * D).view(np.complex128)
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def basis_state(L: int, b: int, dtype=np.complex128) -> np.ndarray:
    """Product state |b> as a dense vector."""
    v = np.zeros(1 << L, dtype=dtype)
    v[b] = 1.0
    return v


def ghz_state(L: int, dtype=np.complex128) -> np.ndarray:
    """(|0...0> + |1...1>)/sqrt(2)."""
    v = np.zeros(1 << L, dtype=dtype)
    v[0] = v[-1] = 1.0 / np.sqrt(2.0)
    return v


def batched_instances(n: int = 512, seed: int = 3, lmin: int = 14, lmax: int = 20):
    """Seeded parameters of the batched ground-state workload.

    Returns a list of (L, alpha, h) with L ~ U{lmin..lmax}, alpha ~ U[0.5, 3],
    h ~ U[0.2, 2.0].
    """
    rng = np.random.Generator(np.random.Philox(seed))
    Ls = rng.integers(lmin, lmax + 1, size=n)
    alphas = rng.uniform(0.5, 3.0, size=n)
    hs = rng.uniform(0.2, 2.0, size=n)
    return [(int(a), float(b), float(c)) for a, b, c in zip(Ls, alphas, hs)]


def batch_start_states(Ls, seed: int = 3, dtype=np.complex128):
    """Seeded complex Gaussian start vectors of a batch, one Philox stream per chain.

    Chain k draws from the Philox-4x32-10 generator with key ``seed`` jumped k
    times (disjoint streams); Re and Im iid N(0,1), normalised to 1.
    """
    base = np.random.Philox(seed)
    out = []
    for k, L in enumerate(Ls):
        rng = np.random.Generator(base.jumped(k))
        v = rng.standard_normal(2 << int(L)).view(np.complex128)
        v /= np.linalg.norm(v)
        out.append(v.astype(dtype))
    return out


def field_schedule(nsteps: int = 200, seed: int = 4, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """Seeded piecewise-constant field values h_k ~ U[lo, hi], one per time step."""
    rng = np.random.Generator(np.random.Philox(seed))
    return rng.uniform(lo, hi, size=nsteps)


# Named workloads (chain length, coupling exponent, field, Krylov settings).
# alpha = None means nearest-neighbour couplings only.
WORKLOADS = {
    "nn_ground_L12": dict(L=12, J=1.0, alpha=None, h=1.0, tol=1e-12, seed=1),
    "lrqi_quench_L24": dict(L=24, J=1.0, alpha=1.5, h=0.8, m=20, dt=0.01, t_end=5.0, measure_every=0.1),
    "lrqi_quench_L28": dict(L=28, J=1.0, alpha=1.5, h=0.8, m=20, dt=0.01),
    "lrqi_neel_L30": dict(L=30, J=1.0, alpha=1.0, h=1.2, m=12, dt=0.02, t_end=2.0),
}
