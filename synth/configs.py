"""The workload configurations: shapes, spectra, primer parameters, tolerances.

Each entry describes one synthetic workload shaped like the paper's (the
paper's own data sets are not available, these stand in for them).  Plain data,
no arithmetic of the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def spectrum(kind: str, d: int, **kw) -> np.ndarray:
    """Population eigenvalues lambda_1..lambda_d (1-based index i)."""
    i = np.arange(1, d + 1, dtype=np.float64)
    if kind == "geometric":          # lambda_i = rho^i
        return kw["rho"] ** i
    if kind == "harmonic":           # lambda_i = 1 / i
        return 1.0 / i
    if kind == "exp":                # lambda_i = exp(-i / tau)
        return np.exp(-i / kw["tau"])
    if kind == "power_floor":        # lambda_i = i^-alpha + floor
        return i ** (-kw["alpha"]) + kw["floor"]
    if kind == "paper_exp":          # 1000 -> 1 exponentially over d dims (Section 5.1)
        return 1000.0 * (1e-3) ** ((i - 1) / (d - 1))
    if kind == "paper_lin":          # 1000 -> 1 linearly over d dims (Section 5.1)
        return 1000.0 - (999.0) * (i - 1) / (d - 1)
    raise ValueError(kind)


@dataclass(frozen=True)
class Config:
    name: str
    n: int
    d: int
    k: int
    l: int
    spectrum: tuple
    dtype: str = "f32"
    seed: int = 1234
    primers: dict = field(default_factory=dict)
    eig_rtol: float = 1e-5
    angle_tol: float = 1e-4

    @property
    def m(self) -> int:
        return self.k + self.l

    def lam(self) -> np.ndarray:
        kind, kw = self.spectrum[0], dict(self.spectrum[1:]) if len(self.spectrum) > 1 else {}
        return spectrum(kind, self.d, **kw)


CONFIGS = {
    # Plain pPCA, FP32; block power k=8, l=8, T=10 then finalize to k=8.
    "power_fp32_4096x256": Config(
        name="power_fp32_4096x256", n=4096, d=256, k=8, l=8,
        spectrum=("geometric", ("rho", 0.9)), dtype="f32", seed=101,
        primers={"power": {"T": 10}}),
    # Three primers compared, FP32, lambda_i = 1/i, k = l = 32.
    "primers_fp32_100000x1024": Config(
        name="primers_fp32_100000x1024", n=100000, d=1024, k=32, l=32,
        spectrum=("harmonic",), dtype="f32", seed=202,
        primers={"power": {"T": 20},
                 "oja": {"batch": 256, "epochs": 1, "lr0": 1.0, "lr_offset": 100.0},
                 # lr from the paper's grid protocol (Section 5): the least summed angle error over
                 # the top k among {1, 1e-1, ..., 1e-6} (bench.py --tune-eg-lr on this workload)
                 "eigengame": {"steps": 200, "batch": 1024, "lr": 0.1, "momentum": 0.9}}),
    # Precision: image-like, BF16 / FP8 storage, k = l = 64, power T=15, split-precision finalize.
    "precision_bf16_1000000x4096": Config(
        name="precision_bf16_1000000x4096", n=1000000, d=4096, k=64, l=64,
        spectrum=("exp", ("tau", 50.0)), dtype="bf16", seed=303,
        primers={"power": {"T": 15}}, eig_rtol=1e-4, angle_tol=1e-3),
    # Batching: 512 ragged instances (drawn by synth.batch_instances).
    "batch512_fp32": Config(
        name="batch512_fp32", n=0, d=0, k=0, l=0, spectrum=("geometric", ("rho", 0.9)),
        dtype="f32", seed=404, primers={"power": {"T": 10}}),
    # Large-d streaming: EigenGame 500 steps, b = 4096, BF16.
    "largeD_bf16_50000x262144": Config(
        name="largeD_bf16_50000x262144", n=50000, d=262144, k=32, l=32,
        spectrum=("power_floor", ("alpha", 1.5), ("floor", 1e-4)), dtype="bf16", seed=505,
        # lr from the paper's grid protocol (Section 5), as for the 1e5 x 1024 workload
        primers={"eigengame": {"steps": 500, "batch": 4096, "lr": 0.1, "momentum": 0.9}},
        eig_rtol=1e-3, angle_tol=1e-2),
}
