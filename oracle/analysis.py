"""Oracle: structure and kinetics analyses (numpy).

TEST INFRASTRUCTURE (see the package docstring).

Paper, Results: the pair correlation function g(r) of the bodies' centres of
mass, the mean square displacement (MSD) of the centres and the mean square
rotation (MSR).  SI Sec. 5 defines the orientational distance between two
unit quaternions as d(q1, q2) = 1 - <q1, q2>^2 (with the 4-D inner product)
and the MSR as its average over the bodies, taken between a starting
orientation and the orientation at a later time, like the MSD.

g(r) is taken from its plain definition in FP64: the minimum-image
distance r of every pair of centres i < j, counted in bin
k = floor(r n_bins / r_max) when r < r_max.  A single-precision evaluation
can put a pair whose distance lies within its rounding error of a bin edge
into the neighbouring bin; gr_edge_counts gives, per edge, how many pairs lie
that close, so a comparison can allow exactly those moves.
"""
from __future__ import annotations

import numpy as np


def gr_distances(pos, box, r_max: float, chunk: int = 2048) -> np.ndarray:
    """Minimum-image centre distances (FP64) of all pairs i < j with
    r < r_max, by brute force over all pairs (no pair list)."""
    p = np.asarray(pos, dtype=np.float64)[:, :3]
    L = np.asarray(box, dtype=np.float64).reshape(3)
    N = len(p)
    out = []
    for i0 in range(0, N, chunk):
        a = p[i0:i0 + chunk]
        d = p[None, :, :] - a[:, None, :]
        d -= L * np.rint(d / L)
        r = np.sqrt(np.sum(d * d, axis=-1))
        ii = np.arange(i0, i0 + len(a))[:, None]
        jj = np.arange(N)[None, :]
        out.append(r[(jj > ii) & (r < r_max)])
    return np.concatenate(out) if out else np.zeros(0)


def gr_counts(pos, box, r_max: float, n_bins: int, chunk: int = 2048) -> np.ndarray:
    """Counts of pairs i < j in the bins [k dr, (k + 1) dr), dr = r_max / n_bins,
    of their minimum-image centre distance (FP64)."""
    r = gr_distances(pos, box, r_max, chunk)
    k = np.floor(r * (n_bins / float(r_max))).astype(np.int64)
    # r < r_max, so k <= n_bins - 1 in exact arithmetic; the FP64 product can
    # round up to n_bins for r within an ulp of r_max
    np.minimum(k, n_bins - 1, out=k)
    return np.bincount(k, minlength=n_bins)


def gr_edge_counts(pos, box, r_max: float, n_bins: int, tol: float,
                   chunk: int = 2048) -> np.ndarray:
    """Per bin edge e = 0..n_bins (at r = e dr, the last one r_max): the number
    of pairs i < j whose FP64 distance lies within `tol` of that edge,
    including pairs just beyond r_max."""
    r = gr_distances(pos, box, float(r_max) + tol, chunk)
    dr = float(r_max) / n_bins
    e = np.rint(r / dr).astype(np.int64)
    near = (np.abs(r - e * dr) < tol) & (e <= n_bins)
    return np.bincount(e[near], minlength=n_bins + 1)


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
