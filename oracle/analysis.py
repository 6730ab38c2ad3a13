"""Oracle: structure and kinetics analyses (numpy).

TEST INFRASTRUCTURE (see the package docstring).

Paper, Results: the pair correlation function g(r) of the bodies' centres of
mass, the mean square displacement (MSD) of the centres and the mean square
rotation (MSR).  SI Sec. 5 defines the orientational distance between two
unit quaternions as d(q1, q2) = 1 - <q1, q2>^2 (with the 4-D inner product)
and the MSR as its average over the bodies, taken between a starting
orientation and the orientation at a later time, like the MSD.

g(r) bin decisions follow the CUDA path's stated FP32 recipe: every
operation below is one IEEE single-precision operation with
round-to-nearest (numpy float32), in the stated order, so the integer counts
can be compared exactly.
"""
from __future__ import annotations

import numpy as np


def gr_counts(pos, box, r_max: float, n_bins: int, chunk: int = 2048) -> np.ndarray:
    """Counts of body pairs i < j by minimum-image centre distance, all in
    FP32: d = p_j - p_i; d -= L rint(d invL); r2 = (dx dx + dy dy) + dz dz;
    bin = trunc(sqrt(r2) * (n_bins / r_max)) for r2 < r_max^2, clamped to the
    last bin.  Brute force over all pairs (no pair list)."""
    f = np.float32
    p = np.asarray(pos, dtype=np.float32)[:, :3]
    L = np.asarray(box, dtype=np.float32).reshape(3)
    invL = (f(1.0) / L).astype(np.float32)
    rmax = f(r_max)
    rmax2 = f(rmax * rmax)
    scale = f(f(n_bins) / rmax)
    counts = np.zeros(n_bins, dtype=np.int64)
    N = len(p)
    for i0 in range(0, N, chunk):
        a = p[i0:i0 + chunk]
        d = (p[None, :, :] - a[:, None, :]).astype(np.float32)
        d = (d - (L * np.rint((d * invL).astype(np.float32))).astype(np.float32)).astype(np.float32)
        r2 = ((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]).astype(np.float32)
        ii = np.arange(i0, i0 + len(a))[:, None]
        jj = np.arange(N)[None, :]
        m = (jj > ii) & (r2 < rmax2)
        r = np.sqrt(r2[m]).astype(np.float32)
        k = (r * scale).astype(np.float32).astype(np.int64)
        np.minimum(k, n_bins - 1, out=k)
        counts += np.bincount(k, minlength=n_bins)
    return counts


def gr_normalise(counts, r_max: float, n_frames: int, n_bodies: int, volume: float) -> np.ndarray:
    """g(r_k) = counts_k / (n_frames x ideal-gas count of pairs in shell k):
    N (N - 1)/2 pairs, each in [r_k, r_k+1) with probability
    (4 pi / 3)(r_k+1^3 - r_k^3) / V."""
    n_bins = len(counts)
    edges = np.arange(n_bins + 1) * (float(r_max) / n_bins)
    shell = 4.0 * np.pi / 3.0 * (edges[1:] ** 3 - edges[:-1] ** 3)
    ideal = 0.5 * n_bodies * (n_bodies - 1) * shell / volume
    return np.asarray(counts, dtype=np.float64) / (n_frames * ideal)


def unwrapped(pos, image, box) -> np.ndarray:
    """Unwrapped centres: pos + image x box (FP64)."""
    return (np.asarray(pos, dtype=np.float64)[:, :3]
            + np.asarray(image, dtype=np.float64)[:, :3] * np.asarray(box, dtype=np.float64))


def msd(pos, image, ref_pos, ref_image, box) -> float:
    """Mean square displacement of the unwrapped centres from the reference."""
    d = unwrapped(pos, image, box) - unwrapped(ref_pos, ref_image, box)
    return float(np.mean(np.sum(d * d, axis=1)))


def orientational_distance(q1, q2) -> np.ndarray:
    """SI Sec. 5: d(q1, q2) = 1 - <q1, q2>^2 for unit quaternions."""
    c = np.sum(np.asarray(q1, dtype=np.float64) * np.asarray(q2, dtype=np.float64), axis=-1)
    return 1.0 - c * c


def msr(quat, ref_quat) -> float:
    """Mean square rotation: the orientational distance averaged over bodies."""
    return float(np.mean(orientational_distance(ref_quat, quat)))
