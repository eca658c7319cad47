"""Seeded synthetic traffic tensors (inputs only).

This module is the one place that both the FP64 oracle and the CUDA path
take their inputs from.  It holds none of the completion method's
arithmetic: it draws random numbers, builds a low-tubal-rank ground truth by
the definition of the t-product (a circular convolution of frontal slices
along mode 3, Definition "t-product" in Sec. 2.2), scales it and masks it.

Shapes follow the traffic datasets of Sec. 5 (OD pairs x time slots x days);
the real Abilene / GEANT traces are not available, so these tensors stand in
for them:

* ``T = A * B`` with ``A`` of size n1 x r x n3 and ``B`` of size r x n2 x n3,
  entries ``|N(0,1)|``  -> tubal rank <= r (Proposition "tubrank").
* ``T(i,j,k) <- s_i * p(j) * T(i,j,k)`` with a lognormal(0, 0.5) scale per OD
  pair (mode 1) and a daily profile ``p(j) = 1 + amp*sin(2 pi j / period)``
  (mode 2).  Diagonal scalings of modes 1 and 2 keep the tubal rank <= r.
* ``M = T + noise * rms(T) * N(0,1)`` (the "full" traffic tensor).
* ``mask ~ Bernoulli(observed)`` (iid, random-missing protocol of Sec. 5).
* ``Y0 ~ N(0,1)`` of size r x n2 x n3, the initial factor (spatial domain).

Arrays are numpy arrays indexed ``[i1, i2, i3]``.  ``to_colmajor`` gives the
flat buffer order of the C ABI (i1 fastest, then i2, then i3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2005_09838


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n1: int
    n2: int
    n3: int
    r: int
    period: int
    observed: float
    iters: int
    seed: int

    @property
    def N(self) -> int:
        return self.n1 * self.n2 * self.n3

    @property
    def S(self) -> int:
        return self.n3 // 2 + 1


def config_seed(config: int, observed: float) -> int:
    return SEED_BASE + 100 * config + int(round(100 * observed))


# The named workloads.  C1 and C2 are the plain-method configurations (FP64
# and FP32); C3-C5 belong to the precision / differentiation / batched forms.
def c1(observed: float = 0.5) -> Workload:
    return Workload("C1 16x48x7 r=2 (OD x 30-min slots x days)", 16, 48, 7, 2, 48,
                    observed, 200, config_seed(1, observed))


def c2(observed: float = 0.2) -> Workload:
    return Workload("C2 144x288x168 r=8 (OD x 5-min slots x days)", 144, 288, 168, 8, 288,
                    observed, 100, config_seed(2, observed))


def c3(observed: float = 0.3) -> Workload:
    return Workload("C3 529x96x112 r=32 (OD x 15-min slots x days)", 529, 96, 112, 32, 96,
                    observed, 30, config_seed(3, observed))


def c4(observed: float = 0.2) -> Workload:
    return Workload("C4 529x288x168 r=16 (OD x 5-min slots x days)", 529, 288, 168, 16, 288,
                    observed, 20, config_seed(4, observed))


def custom(n1, n2, n3, r, observed, seed, period=None, iters=10, name=None) -> Workload:
    period = period if period is not None else n2
    return Workload(name or f"{n1}x{n2}x{n3} r={r}", n1, n2, n3, r, period, observed, iters, seed)


def _circular_tproduct(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Ground truth A*B by the t-product definition: slice k of the result is
    sum_l A(:,:,l) B(:,:,(k-l) mod n3) (block-circulant times block vector)."""
    n1, r, n3 = A.shape
    _, n2, _ = B.shape
    T = np.zeros((n1, n2, n3))
    for l in range(n3):
        Bl = np.roll(B, l, axis=2)  # Bl[:,:,k] = B[:,:,(k-l) mod n3]
        T += np.tensordot(A[:, :, l], Bl, axes=([1], [0]))
    return T


def generate(w: Workload, noise: float = 0.01, amp: float = 0.5) -> dict:
    """Draw one seeded instance.  Returns float64 arrays M, T, G (= M on the
    mask, 0 elsewhere), Y0 and the boolean mask."""
    rng = np.random.default_rng(w.seed)
    A = np.abs(rng.standard_normal((w.n1, w.r, w.n3)))
    B = np.abs(rng.standard_normal((w.r, w.n2, w.n3)))
    T = _circular_tproduct(A, B)
    s = np.exp(0.5 * rng.standard_normal(w.n1))
    p = 1.0 + amp * np.sin(2.0 * math.pi * np.arange(w.n2) / w.period)
    T = T * s[:, None, None] * p[None, :, None]
    rms = math.sqrt(float(np.mean(T * T)))
    M = T + noise * rms * rng.standard_normal(T.shape)
    mask = rng.random(T.shape) < w.observed
    Y0 = rng.standard_normal((w.r, w.n2, w.n3))
    G = np.where(mask, M, 0.0)
    return {"M": M, "T": T, "G": G, "mask": mask, "Y0": Y0}


def as_precision(inst: dict, dtype) -> dict:
    """Round the real inputs to ``dtype`` and back to float64, so that an FP32
    run and the FP64 oracle start from bit-identical inputs."""
    out = dict(inst)
    for key in ("M", "T", "G", "Y0"):
        out[key] = inst[key].astype(dtype).astype(np.float64)
    return out


def to_colmajor(a: np.ndarray, dtype=None) -> np.ndarray:
    """Flat buffer with i1 fastest (the C ABI's element order)."""
    a = np.asarray(a)
    if dtype is not None:
        a = a.astype(dtype)
    return np.ascontiguousarray(a.transpose(2, 1, 0)).reshape(-1)


def from_colmajor(flat: np.ndarray, shape) -> np.ndarray:
    n1, n2, n3 = shape
    return np.asarray(flat).reshape(n3, n2, n1).transpose(2, 1, 0)


def nmse(M: np.ndarray, W: np.ndarray, mask: np.ndarray) -> float:
    """Recovery error on the missing entries: sum (M-W)^2 / sum M^2 over the
    complement of the mask."""
    miss = ~mask
    d = (M - W)[miss]
    return float(np.sum(d * d) / np.sum(M[miss] ** 2))


def nmae(M: np.ndarray, W: np.ndarray, mask: np.ndarray) -> float:
    """NMAE of Sec. 5: sum |M-W| / sum |M| over the missing entries."""
    miss = ~mask
    return float(np.sum(np.abs(M - W)[miss]) / np.sum(np.abs(M[miss])))
