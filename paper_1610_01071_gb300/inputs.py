"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers and
names the workloads (sizes, amplitudes, seeds). Both the GPU path and the CPU
oracle consume what it returns.

Workloads (synthetic stand-ins for the paper's ion-acoustic and expansion runs,
Section 4; normalised units lambda_D = omega_pi = c_s = 1, ion q/m = 1):

* ``iaw_small``  — periodic L=64, 128 cells, 2^17 ions, sine amplitude 0.1,
  v_th=1, dt=0.1, K=20, M=10, Haar coarse level 16.
* ``iaw_large``  — ion-wave steepening at scale: periodic 4096 cells (dx=0.5,
  L=2048), 2^24 ions, amplitude 0.5 on the longest mode, v_th=1, K=20, M=10,
  50 macro-steps, 256 coarse coefficients per moment.
* ``slab``       — slab expansion into vacuum (Section 4.2's test, uniform-slab
  variant): bounded grid of 8192 cells (dx=0.5, absorbing walls), n = 1 on the
  central eighth and vacuum elsewhere, 2^25 equal-weight ions (none in the vacuum
  cells), v_th=1, dt=0.1, K=30, M=8, 40 macro-steps, 512 coarse coefficients per
  moment.
* ``iaw_kinetic`` — the paper's two-species ion-acoustic setting (Section 4.1, Runs 5-8
  shape): periodic 1024 cells at dx = 0.28125 (L = 288, about the paper's L = 8 at
  h = 0.28 Debye lengths), 2^23 ions and 2^23 electrons (8192 per cell and species),
  amplitude 0.2, ion v_th = 0.22, electrons q/m = -1800 with v_th = sqrt(1800), dt =
  0.25 / omega_pe, bursts of K = 30 fine steps per macro step of 150 dt (the paper's
  Delta t / delta t), 325 macro steps (T = 287, the paper's t = 8 in ion plasma periods
  of its units), 256 coarse x-bins by 64 velocity cells over [-2.5, 2.5).
"""
from __future__ import annotations

import numpy as np

WORKLOADS = {
    "iaw_small": dict(ncell=128, L=64.0, N=1 << 17, amplitude=0.1, v_th=1.0, dt=0.1, K=20, M=10,
                      n_coarse=16, macro_steps=5, wavelet="haar"),
    "iaw_large": dict(ncell=4096, L=2048.0, N=1 << 24, amplitude=0.5, v_th=1.0, dt=0.1, K=20, M=10,
                      n_coarse=256, macro_steps=50, wavelet="haar"),
    "slab": dict(ncell=8192, L=4096.0, N=1 << 25, amplitude=0.0, v_th=1.0, dt=0.1, K=30, M=8,
                 n_coarse=512, macro_steps=40, wavelet="haar", boundary="absorbing"),
    "iaw_kinetic": dict(ncell=1024, L=288.0, N=1 << 23, amplitude=0.2, v_th=0.22, dt=0.25 / np.sqrt(1800.0),
                        K=30, M=5, n_coarse=256, macro_steps=325, wavelet="haar", electrons="kinetic",
                        qm_e=-1800.0, n_v=64, v_max=2.5),
}


def workload(name: str) -> dict:
    cfg = dict(WORKLOADS[name])
    cfg["dT"] = cfg["M"] * cfg["K"] * cfg["dt"]  # macro step = M bursts of K fine steps
    cfg["qm"] = 1.0
    return cfg


def random_particles(N: int, ncell: int, seed: int, v_th: float = 1.0, sort: bool = True,
                     w_lo: float = 0.5, w_hi: float = 1.5):
    """Random FP32 particle state (cell int32, theta f32 in [0,1), v f32, w f32).

    Weights are uniform in [w_lo, w_hi) * ncell/N so that the mean density is ~1.
    With ``sort`` the cells are non-decreasing (the layout lifting produces)."""
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, ncell, N, dtype=np.int64).astype(np.int32)
    if sort:
        cell.sort()
    theta = rng.random(N, dtype=np.float32)
    v = (rng.standard_normal(N) * v_th).astype(np.float32)
    w = ((w_lo + (w_hi - w_lo) * rng.random(N)) * (ncell / N)).astype(np.float32)
    return cell, theta, v, w


def random_field(ncell: int, seed: int, amp: float = 0.1):
    """Smooth random periodic nodal field (a few low Fourier modes), float64."""
    rng = np.random.default_rng(seed)
    x = np.arange(ncell) / ncell
    f = np.zeros(ncell)
    for m in range(1, 5):
        f += amp / m * (rng.standard_normal() * np.cos(2 * np.pi * m * x) + rng.standard_normal() * np.sin(2 * np.pi * m * x))
    return f


def random_density(ncell: int, seed: int, amp: float = 0.3):
    """Positive periodic nodal density around 1 (float64)."""
    return 1.0 + random_field(ncell, seed, amp)


def random_mlp_params(dims, seed: int, scale: float = 1.0):
    """Random FP32 parameter vector of a dense network with widths dims (flat W_1 [d1][d0],
    b_1, W_2, ...): weights N(0, scale^2 / d_in), biases N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(dims) - 1):
        parts.append(rng.standard_normal(dims[l + 1] * dims[l]) * (scale / np.sqrt(dims[l])))
        parts.append(0.1 * rng.standard_normal(dims[l + 1]))
    return np.concatenate(parts).astype(np.float32)


def regression_set(n: int, d_in: int, d_out: int, seed: int):
    """Smooth synthetic regression pairs: X ~ N(0, 1) + offsets, Y = tanh(X A) B + 0.1 X C,
    FP32, for checking that training reduces a loss."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d_in)) + rng.standard_normal(d_in)
    A = rng.standard_normal((d_in, 64)) / np.sqrt(d_in)
    B = rng.standard_normal((64, d_out)) / 8.0
    C = rng.standard_normal((d_in, d_out)) / np.sqrt(d_in)
    Y = np.tanh(X @ A) @ B + 0.1 * X @ C + 3.0
    return X.astype(np.float32), Y.astype(np.float32)
