"""Seeded synthetic inputs for the sparse FFT (shared by the tests, the benchmark and the oracle checks).

This module only draws inputs: supports, coefficient values, noise and the time signal obtained from
them by an inverse DFT.  It holds none of the sparse-FFT arithmetic, and it imports neither the
GPU binding nor the oracle.

Recipes (the paper measures on no dataset; every workload is synthetic):

* exactly k-sparse (Alg. 1 workloads): k distinct frequencies uniform in [0, n), |X_f| = 1, phase
  uniform in [0, 2 pi); x = IDFT(X) = (1/n) sum_f X_f e^{+2 pi i f t / n} formed in FP64 and
  rounded once to the requested dtype.  The ground truth X stays in FP64.
* general (Alg. 2 workloads): k heavy frequencies with |X_f| = 10^{U[0,1]} (log-uniform in [1, 10])
  and uniform phase, plus i.i.d. circular complex Gaussian noise on every time sample with
  E|eta_t|^2 = P / 10^{snr_db/10}, P = sum_t |x_t|^2 / n of the sparse part.
* Sec. 5 reduction: a k-point signal s repeated n/k times, y_t = s_{t mod k}, whose spectrum lives on
  the multiples of n/k.

Random numbers come from numpy's Philox bit generator keyed by the seed, so every input is
reproducible bit for bit on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 0x5EED0000


def seed_for(config: int, instance: int) -> int:
    """Seed of instance ``instance`` of workload ``config``: 0x5EED0000 + 1000 config + instance."""
    return SEED_BASE + 1000 * int(config) + int(instance)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1)))


@dataclass
class SparseSignal:
    x: np.ndarray            # time signal, requested dtype
    support: np.ndarray      # sorted frequencies of the planted coefficients (int64)
    values: np.ndarray       # planted X at ``support`` (complex128)
    noise_power: float = 0.0  # per-sample noise variance (general workloads)

    def spectrum(self) -> np.ndarray:
        """The planted sparse spectrum as a dense complex128 vector."""
        X = np.zeros(self.x.shape[-1], dtype=np.complex128)
        X[self.support] = self.values
        return X


def draw_support(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    return np.sort(rng.choice(n, size=k, replace=False).astype(np.int64))


def exact_sparse(n: int, k: int, seed: int, dtype=np.complex64) -> SparseSignal:
    rng = _rng(seed)
    support = draw_support(rng, n, k)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=k)
    values = np.exp(1j * phase)
    X = np.zeros(n, dtype=np.complex128)
    X[support] = values
    x = np.fft.ifft(X)
    return SparseSignal(x=x.astype(dtype), support=support, values=values)


def general_noisy(n: int, k: int, seed: int, snr_db: float = 20.0, dtype=np.complex64) -> SparseSignal:
    rng = _rng(seed)
    support = draw_support(rng, n, k)
    mag = 10.0 ** rng.uniform(0.0, 1.0, size=k)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=k)
    values = mag * np.exp(1j * phase)
    X = np.zeros(n, dtype=np.complex128)
    X[support] = values
    x = np.fft.ifft(X)
    power = float(np.sum(np.abs(values) ** 2)) / float(n) ** 2  # sum_t |x_t|^2 / n by Parseval
    noise_var = power / 10.0 ** (snr_db / 10.0)
    noise = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.sqrt(noise_var / 2.0)
    x = x + noise
    return SparseSignal(x=x.astype(dtype), support=support, values=values, noise_power=noise_var)


def integer_sparse(n: int, k: int, L: int, seed: int, noise_std: float = 0.0, dtype=np.complex128) -> SparseSignal:
    """Exactly k-sparse spectrum with integer coefficients, the input model of Sec. 3 (X_f uniform on
    {-L, ..., L} without 0, support uniform without replacement); x = IDFT(X) in FP64, plus, when
    noise_std > 0, circular complex Gaussian noise of that standard deviation per time sample."""
    rng = _rng(seed)
    support = draw_support(rng, n, k)
    mag = rng.integers(1, L + 1, size=k)
    sign = np.where(rng.integers(0, 2, size=k) == 1, 1, -1)
    values = (mag * sign).astype(np.complex128)
    X = np.zeros(n, dtype=np.complex128)
    X[support] = values
    x = np.fft.ifft(X)
    if noise_std > 0.0:
        x = x + (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * (noise_std / np.sqrt(2.0))
    return SparseSignal(x=x.astype(dtype), support=support, values=values, noise_power=noise_std ** 2)


def periodic_extension(n: int, kdim: int, seed: int, dtype=np.complex128):
    """Sec. 5 reduction input: s in C^kdim with unit-magnitude DFT, y_t = s_{t mod kdim}.

    Returns (y, S) with S = DFT_kdim(s) (so that DFT_n(y) = (n/kdim) S on the multiples of n/kdim).
    """
    rng = _rng(seed)
    S = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=kdim))
    s = np.fft.ifft(S)
    y = np.tile(s, n // kdim)
    return y.astype(dtype), S


def exact_sparse_batch_spectra(n: int, k: int, seeds) -> tuple[np.ndarray, np.ndarray]:
    """Supports (int64 [N, k]) and values (complex128 [N, k]) of a batch of exactly k-sparse spectra.

    The i-th row equals ``exact_sparse(n, k, seeds[i])``'s support and values.
    """
    sup = np.zeros((len(seeds), k), dtype=np.int64)
    val = np.zeros((len(seeds), k), dtype=np.complex128)
    for r, s in enumerate(seeds):
        rng = _rng(s)
        sup[r] = draw_support(rng, n, k)
        val[r] = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=k))
    return sup, val


def exact_sparse_batch_device(n: int, k: int, seeds, device, chunk: int = 16, dtype=None):
    """A batch of exactly k-sparse signals built on a torch device (shape [N, n], complex64 unless
    `dtype` says otherwise).

    The spectra are those of ``exact_sparse_batch_spectra``; the inverse DFT runs in complex128 on
    the device (input synthesis only) and is rounded once to the output type.  Returns (x, supports,
    values).
    """
    import torch

    sup, val = exact_sparse_batch_spectra(n, k, seeds)
    N = len(seeds)
    out = torch.empty((N, n), dtype=dtype or torch.complex64, device=device)
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        X = torch.zeros((c1 - c0, n), dtype=torch.complex128, device=device)
        rows = torch.arange(c1 - c0, device=device).unsqueeze(1).expand(-1, k)
        X[rows, torch.as_tensor(sup[c0:c1], device=device)] = torch.as_tensor(val[c0:c1], device=device)
        out[c0:c1] = torch.fft.ifft(X, dim=-1).to(out.dtype)
        del X
    return out, sup, val


def exact_sparse_channels_device(n: int, k: int, seeds, device, chunk: int = 16):
    """C = len(seeds) exactly k-sparse signals as one interleaved multi-channel array [n, C] complex64
    on a torch device (row m holds sample m of every channel); channel c is ``exact_sparse_batch_device``'s
    row c.  Returns (x, supports, values)."""
    import torch

    x, sup, val = exact_sparse_batch_device(n, k, seeds, device, chunk=chunk)
    xt = x.t().contiguous()
    del x
    return xt, sup, val


def sparse_signal_device(n: int, k: int, seed: int, device, snr_db=None):
    """One signal built on a torch device (complex64 [n]): the spectrum of ``exact_sparse`` (snr_db
    None) or of ``general_noisy`` (heavy coefficients; complex Gaussian time noise at snr_db, drawn on
    the device from a torch generator seeded with `seed`, so the noise differs from the numpy
    generator's).  Returns (x, support, values)."""
    import torch

    rng = _rng(seed)
    support = draw_support(rng, n, k)
    mag = np.ones(k) if snr_db is None else 10.0 ** rng.uniform(0.0, 1.0, size=k)
    values = mag * np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=k))
    X = torch.zeros(n, dtype=torch.complex128, device=device)
    X[torch.as_tensor(support, device=device)] = torch.as_tensor(values, device=device)
    x = torch.fft.ifft(X)
    del X
    if snr_db is not None:
        power = float(np.sum(np.abs(values) ** 2)) / float(n) ** 2
        sd = float(np.sqrt(power / 10.0 ** (snr_db / 10.0) / 2.0))
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) & ((1 << 63) - 1))
        noise = torch.randn((n, 2), dtype=torch.float64, device=device, generator=g) * sd
        x = x + torch.view_as_complex(noise)
    return x.to(torch.complex64), support, values
