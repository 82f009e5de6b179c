"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws numbers: it holds none of the transform's arithmetic and
imports neither the GPU library nor the oracle.  Every generator is
deterministic in its seed.

Input kinds (the workloads of the QFT->FFT evaluation, Sec. 4):
  gaussian  re/im iid N(0,1), optionally normalised to unit L2
  tones     sum of 1-8 pure tones (integer bins, amplitude U[0.1,1], phase
            U[0,2pi)) plus complex noise with standard deviation 1e-3 per
            component
  basis     computational basis state |j>
  single_tone  one complex exponential at bin k0 (Sec. 4 correctness check),
            unit L2 norm; ``sign`` is the transform's exponent sign, and the
            tone is chosen so that this transform peaks at bin k0

Host arrays are numpy complex128 (numpy PCG64).  ``to_torch`` copies to a
torch tensor of the requested complex dtype/device; ``device_gaussian`` draws
directly on a CUDA device with a seeded ``torch.Generator`` (for sizes where a
host copy is not wanted).
"""
from __future__ import annotations

import numpy as np

KINDS = ("gaussian", "tones", "basis")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian(n: int, seed: int, normalise: bool = True) -> np.ndarray:
    rng = _rng(seed)
    N = 1 << n
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    if normalise:
        x /= np.sqrt(np.sum(np.abs(x) ** 2))
    return x.astype(np.complex128)


def tones(n: int, seed: int, count: int | None = None, noise_std: float = 1e-3) -> np.ndarray:
    rng = _rng(seed)
    N = 1 << n
    if count is None:
        count = int(rng.integers(1, 9))
    x = np.zeros(N, dtype=np.complex128)
    for _ in range(count):
        f = int(rng.integers(0, N))
        a = float(rng.uniform(0.1, 1.0))
        ph = float(rng.uniform(0.0, 2.0 * np.pi))
        # exponent reduced exactly in integers before forming the angle
        x += a * np.exp(1j * (2.0 * np.pi * ((f * np.arange(N, dtype=np.int64)) % N) / N + ph))
    x += noise_std * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    return x


def basis(n: int, j: int) -> np.ndarray:
    x = np.zeros(1 << n, dtype=np.complex128)
    x[j] = 1.0
    return x


def single_tone(n: int, k0: int = 2, sign: int = -1) -> np.ndarray:
    N = 1 << n
    m = (k0 * np.arange(N, dtype=np.int64)) % N
    x = np.exp(-sign * 2j * np.pi * m / N) / np.sqrt(N)
    return x.astype(np.complex128)


def make(kind: str, n: int, seed: int) -> np.ndarray:
    """One input of the named kind (basis index drawn from the seed)."""
    if kind == "gaussian":
        return gaussian(n, seed)
    if kind == "tones":
        return tones(n, seed)
    if kind == "basis":
        return basis(n, int(_rng(seed).integers(0, 1 << n)))
    raise ValueError(kind)


def to_torch(x: np.ndarray, dtype: str = "c64", device: str = "cpu"):
    import torch

    td = torch.complex64 if dtype == "c64" else torch.complex128
    return torch.from_numpy(np.ascontiguousarray(x)).to(device=device, dtype=td)


def device_gaussian(n: int, seed: int, dtype: str = "c64", device: str = "cuda", out=None):
    """re/im iid N(0,1) drawn on the device (not normalised), as a complex tensor."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    N = 1 << n
    if out is None:
        out = torch.empty(N, dtype=torch.complex64 if dtype == "c64" else torch.complex128, device=device)
    v = torch.view_as_real(out)
    # fill in chunks to bound temporary memory
    chunk = 1 << 26
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        v[s:e].normal_(0.0, 1.0, generator=g)
    return out
