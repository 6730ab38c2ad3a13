"""Independent FP64 CPU oracle for the rigid-body force/torque path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never calls it, and it never calls the product
library: the two share no code.

Layout:
  bead_sum.c   bead-bead double sum (Lennard-Jones or the half-power
               half-cosine of Eq. 1), brute-force body-pair search, minimum
               bead distance (plain C, FP64, single thread)
  bodies.py    bead templates, mass, inertia, quaternion algebra (numpy FP64)
  nn.py        pair MLP energy, features, forces/torques as exact gradients
               (PyTorch CPU FP64 with autograd), force-matching loss gradient
  md.py        rigid-body velocity Verlet with the NO_SQUISH free-rotor split,
               kinetic energies (numpy FP64)
  sampler.py   training-pair sampler with contact bisection

Every function cites the passage of the paper it follows.  Functions whose
result is not pinned by a closed form, invariant or brute force in
``tests/test_oracle_pins.py`` say "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "bead_sum.c")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (IEEE FP64: no fast-math and
    no FMA contraction, so x86 and Arm hosts give the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp] + _SRC + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            L.orc_lj.argtypes = [ctypes.c_double] * 4 + [dp, dp]
            L.orc_lj.restype = ctypes.c_int
            L.orc_bead_pair.argtypes = [dp, dp, dp, dp, dp, ctypes.c_int64, dp, ctypes.c_int64,
                                        dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.orc_bead_pair.restype = None
            L.orc_pairs_bruteforce.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, i64p,
                                               ctypes.c_int64]
            L.orc_pairs_bruteforce.restype = ctypes.c_int64
            L.orc_forces_beads.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int64, dp,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int64, i64p, dp, dp, dp, dp, dp]
            L.orc_forces_beads.restype = None
            L.orc_min_bead_distance.argtypes = [dp, dp, dp, dp, dp, ctypes.c_int64, dp,
                                                ctypes.c_int64, dp]
            L.orc_min_bead_distance.restype = ctypes.c_double
            L.orc_hphc.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, dp, dp]
            L.orc_hphc.restype = ctypes.c_int
            L.orc_hphc_cutoff.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.orc_hphc_cutoff.restype = ctypes.c_double
            L.orc_pot_cutoff.argtypes = [dp]
            L.orc_pot_cutoff.restype = ctypes.c_double
            L.orc_bead_pair_pot.argtypes = [dp, dp, dp, dp, dp, ctypes.c_int64, dp,
                                            ctypes.c_int64, dp, dp, dp]
            L.orc_bead_pair_pot.restype = None
            L.orc_forces_beads_pot.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int64, dp, dp,
                                               ctypes.c_int64, i64p, dp, dp, dp, dp, dp]
            L.orc_forces_beads_pot.restype = None
            _lib = L
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def lj(r: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5):
    """Bead potential u(r) and -u'(r)/r (energy-shifted, force-truncated LJ)."""
    u = ctypes.c_double()
    f = ctypes.c_double()
    lib().orc_lj(float(r) ** 2, eps, sigma, rc, ctypes.byref(u), ctypes.byref(f))
    return u.value, f.value


def hphc(r: float, A: float, b: float, c: float, p: float, printed: bool = False):
    """Half-power half-cosine bead potential (paper, Eq. 1): u(r) and -u'(r)/r.

    printed=False: the continuous reading (half cosine -A (1 + cos c(r - b))
    from -2A at r = b to 0 at b + pi/c); printed=True: the printed cosine
    -A cos c(r - b), cut at its first zero b + pi/(2c), with the jump at b."""
    u = ctypes.c_double()
    f = ctypes.c_double()
    lib().orc_hphc(float(r) ** 2, A, b, c, p, int(bool(printed)), ctypes.byref(u), ctypes.byref(f))
    return u.value, f.value


def hphc_cutoff(b: float, c: float, printed: bool = False) -> float:
    return float(lib().orc_hphc_cutoff(b, c, int(bool(printed))))


def pot_lj(eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5) -> np.ndarray:
    """Potential descriptor of the Lennard-Jones bead potential."""
    return np.array([0.0, eps, sigma, rc, 0.0])


def pot_hphc(A: float, b: float, c: float, p: float, printed: bool = False) -> np.ndarray:
    """Potential descriptor of the half-power half-cosine bead potential."""
    return np.array([2.0 if printed else 1.0, A, b, c, p])


def pot_cutoff(pot) -> float:
    return float(lib().orc_pot_cutoff(_p(_d(pot))))


def bead_pair(p_i, q_i, p_j, q_j, box, tmpl_i, tmpl_j=None, eps=1.0, sigma=1.0, rc=2.5,
              pot=None):
    """Bead double sum for one body pair (paper, Methods: U = sum_i sum_j u_bead).

    The bead potential is Lennard-Jones (eps, sigma, rc) unless a descriptor
    `pot` (pot_lj / pot_hphc) is given.  Returns dict with E, F_i, F_j,
    tau_i, tau_j (space frame), the bead-level virial (3x3) and the number of
    bead pairs inside the cutoff."""
    tmpl_i = _d(tmpl_i)
    tmpl_j = tmpl_i if tmpl_j is None else _d(tmpl_j)
    out = np.zeros(23)
    if pot is None:
        pot = pot_lj(eps, sigma, rc)
    lib().orc_bead_pair_pot(_p(_d(p_i)), _p(_d(q_i)), _p(_d(p_j)), _p(_d(q_j)), _p(_d(box)),
                            len(tmpl_i), _p(tmpl_i), len(tmpl_j), _p(tmpl_j), _p(_d(pot)),
                            _p(out))
    return {"E": out[0], "F_i": out[1:4].copy(), "F_j": out[4:7].copy(),
            "tau_i": out[7:10].copy(), "tau_j": out[10:13].copy(),
            "virial": out[13:22].reshape(3, 3).copy(), "n_in": int(out[22])}


def pairs_bruteforce(pos, box, Rc) -> np.ndarray:
    """All body pairs i < j with minimum-image |R_ij| < Rc, as an (M, 2) int64 array."""
    pos = _d(pos)
    N = len(pos)
    cap = 1 << 16
    while True:
        out = np.zeros((cap, 2), dtype=np.int64)
        m = lib().orc_pairs_bruteforce(N, _p(pos), _p(_d(box)), float(Rc), _pi(out), cap)
        if m <= cap:
            return out[:m].copy()
        cap = int(m)


def forces_beads(pos, quat, box, tmpl, pairs, eps=1.0, sigma=1.0, rc=2.5, per_pair=False,
                 pot=None):
    """Per-body bead-sum forces and torques over the given body pairs, with the
    Lennard-Jones bead potential (eps, sigma, rc) or the descriptor `pot`.

    Returns (F [N,3], tau [N,3], E, virial9 (COM virial sum R_ij (x) F_j)
    [, per-pair array (M, 23)])."""
    pos = _d(pos)
    quat = _d(quat)
    tmpl = _d(tmpl)
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
    N = len(pos)
    F = np.zeros((N, 3))
    tau = np.zeros((N, 3))
    E = np.zeros(1)
    vir = np.zeros(9)
    pp = np.zeros((len(pairs), 23)) if per_pair else None
    if pot is None:
        pot = pot_lj(eps, sigma, rc)
    lib().orc_forces_beads_pot(N, _p(pos), _p(quat), _p(_d(box)), len(tmpl), _p(tmpl),
                               _p(_d(pot)), len(pairs), _pi(pairs), _p(F), _p(tau), _p(E),
                               _p(vir), _p(pp) if pp is not None else None)
    if per_pair:
        return F, tau, float(E[0]), vir.reshape(3, 3), pp
    return F, tau, float(E[0]), vir.reshape(3, 3)


def min_bead_distance(p_i, q_i, p_j, q_j, box, tmpl) -> float:
    tmpl = _d(tmpl)
    return float(lib().orc_min_bead_distance(_p(_d(p_i)), _p(_d(q_i)), _p(_d(p_j)),
                                             _p(_d(q_j)), _p(_d(box)), len(tmpl), _p(tmpl),
                                             len(tmpl), _p(tmpl)))
