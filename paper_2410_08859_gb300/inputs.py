"""Seeded synthetic marginals for the unbalanced domain-decomposition workloads.

This module only synthesises input measures (positive densities on an N x N
pixel grid); it holds none of the transport arithmetic, so both the CUDA path
and the FP64 CPU oracle draw their inputs from here.

The paper evaluates on Gaussian-mixture images (Section 5.3, "Test data") that
are not distributed with it; the generators below stand in for them:

* ``mixture_small``  -- 32 x 32, three isotropic Gaussians, 1e-3 floor,
  masses 1.0 / 1.3 (the small FP64 parity workload).
* ``mixture_blobs``  -- 5..20 Gaussian blobs with random weights, floor 1e-6
  of the maximum, mass ratio drawn from U[0.7, 1.5] (the 256 x 256 workload).
* ``lognormal_field`` -- exp of a Gaussian random field with correlation
  length 0.05 (the 1024 x 1024 workload).

Every generator takes an explicit ``seed``; the convention used by the tests
and the benchmark is ``seed = 1000 * workload_id + instance``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["mixture_small", "mixture_blobs", "lognormal_field", "workload",
           "WORKLOADS"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _grid(N: int):
    t = np.arange(N, dtype=np.float64) / N
    return np.meshgrid(t, t, indexing="ij")


def _gaussians(N, rng, n_blobs, sig_lo, sig_hi, w_lo, w_hi, c_lo, c_hi):
    I, J = _grid(N)
    img = np.zeros((N, N))
    for _ in range(n_blobs):
        c = rng.uniform(c_lo, c_hi, size=2)
        sig = rng.uniform(sig_lo, sig_hi)
        w = rng.uniform(w_lo, w_hi)
        img += w * np.exp(-((I - c[0]) ** 2 + (J - c[1]) ** 2) / (2 * sig * sig))
    return img


def mixture_small(N: int = 32, seed: int = 1000, masses=(1.0, 1.3)):
    """Two 3-Gaussian mixtures (sigma in [0.05, 0.2], weights in [0.5, 1.5],
    centres in [0.15, 0.85]^2), normalised to maximum 1, plus a 1e-3 floor,
    scaled to the given total masses.  Returns (mu, nu) as (N, N) float64."""
    rng = _rng(seed)
    out = []
    for m in masses:
        img = _gaussians(N, rng, 3, 0.05, 0.2, 0.5, 1.5, 0.15, 0.85)
        img = img / img.max() + 1e-3
        out.append(img * (m / img.sum()))
    return out[0], out[1]


def mixture_blobs(N: int = 256, seed: int = 2000, mass_ratio=None):
    """5..20 Gaussian blobs (sigma in [0.02, 0.2], weights in [0, 1], centres
    in [0, 1]^2), floor 1e-6 of the maximum; mu has mass 1 and nu has mass
    r ~ U[0.7, 1.5] unless ``mass_ratio`` is given."""
    rng = _rng(seed)
    r = rng.uniform(0.7, 1.5) if mass_ratio is None else float(mass_ratio)
    out = []
    for m in (1.0, r):
        nb = int(rng.integers(5, 21))
        img = _gaussians(N, rng, nb, 0.02, 0.2, 0.0, 1.0, 0.0, 1.0)
        img = img + 1e-6 * img.max()
        out.append(img * (m / img.sum()))
    return out[0], out[1]


def lognormal_field(N: int = 1024, seed: int = 3000, masses=(1.0, 1.2),
                    corr_len: float = 0.05, sigma_log: float = 1.0):
    """exp(g) with g a standardised Gaussian random field: white noise
    smoothed by a periodic Gaussian filter of width ``corr_len`` (FFT),
    times ``sigma_log``; scaled to the given masses."""
    rng = _rng(seed)
    k = np.fft.fftfreq(N) * N  # integer wave numbers
    K1, K2 = np.meshgrid(k, k, indexing="ij")
    filt = np.exp(-0.5 * (2 * np.pi * corr_len) ** 2 * (K1 ** 2 + K2 ** 2))
    out = []
    for m in masses:
        noise = rng.standard_normal((N, N))
        g = np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))
        g = (g - g.mean()) / g.std()
        img = np.exp(sigma_log * g)
        out.append(img * (m / img.sum()))
    return out[0], out[1]


# name -> (generator, default keyword arguments, solver parameters)
WORKLOADS = {
    "mix32": dict(gen=mixture_small, N=32, s=4, eps=(1.0 / 32) ** 2, lam=1.0),
    "blobs256": dict(gen=mixture_blobs, N=256, s=8, eps=(1.0 / 256) ** 2, lam=1.0),
    "lognormal1024": dict(gen=lognormal_field, N=1024, s=16,
                          eps=(2.0 / 1024) ** 2, lam=1.0),
}


def batch_instances(n_inst: int = 64, seed: int = 4000, sides=(64, 128, 256, 512)):
    """Many independent problems: side n ~ U(sides), eps = (2/n)^2,
    lam ~ U{0.5, 1, 5}, blob mixtures of unequal mass (mass ratio in
    [0.7, 1.5]).  Returns a list of dicts (mu, nu, N, eps, lam)."""
    rng = _rng(seed)
    out = []
    for k in range(n_inst):
        N = int(rng.choice(sides))
        lam = float(rng.choice([0.5, 1.0, 5.0]))
        mu, nu = mixture_blobs(N=N, seed=seed + 1 + k)
        out.append(dict(mu=mu, nu=nu, N=N, eps=(2.0 / N) ** 2, lam=lam))
    return out


def workload(name: str, instance: int = 0, N: int | None = None):
    """Return (mu, nu, params) for a named workload; ``N`` overrides the size
    (used for small parity cases of the same distribution)."""
    wid = {"mix32": 1, "blobs256": 2, "lognormal1024": 3}[name]
    spec = dict(WORKLOADS[name])
    gen = spec.pop("gen")
    if N is not None:
        spec["N"] = N
    mu, nu = gen(N=spec["N"], seed=1000 * wid + instance)
    return mu, nu, spec
