"""Thin Python binding of the C ABI (argument marshalling only).

Device arrays are torch CUDA tensors (float32, contiguous); host arrays are
numpy.  Every computation runs inside librb.so; nothing here computes.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (RB_BF16, RB_DESC_FEATURES10, RB_DESC_PAPER6, RB_F16X3, RB_FP32, RB_PATH_BEADS,
                   RB_PATH_NN, RB_SHAPE_CUBE, RB_SHAPE_CUSTOM, RB_SHAPE_CYLINDER, RBError, check,
                   load)

SHAPES = {"cube": RB_SHAPE_CUBE, "cylinder": RB_SHAPE_CYLINDER, "custom": RB_SHAPE_CUSTOM}
POTENTIALS = {"lj": _lib.RB_POT_LJ, "hphc": _lib.RB_POT_HPHC,
              "hphc_printed": _lib.RB_POT_HPHC_PRINTED}
# "f16x3": FP32 accuracy on the tensor cores (split FP16 operands)
PRECISION = {"fp32": RB_FP32, "bf16": RB_BF16, "f16x3": RB_F16X3, RB_FP32: RB_FP32,
             RB_BF16: RB_BF16, RB_F16X3: RB_F16X3}

__all__ = ["System", "MLP", "FNet", "FNetTrainer", "RBError", "RB_PATH_BEADS", "RB_PATH_NN",
           "RB_FP32", "RB_BF16", "RB_F16X3"]


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t: torch.Tensor, cols: int) -> int:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and t.shape[-1] == cols):
        raise ValueError(f"expected a contiguous float32 CUDA tensor with {cols} columns")
    return t.data_ptr()


def _ptr(x, cols: int):
    """(pointer, is_host) for a torch CUDA tensor or a host numpy array."""
    if x is None:
        return None, 0
    if isinstance(x, torch.Tensor):
        if x.is_cuda:
            return _dev(x, cols), 0
        x = x.numpy()
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.shape[-1] != cols:
        raise ValueError(f"expected {cols} columns")
    return a, 1


class System:
    """rb_create_system / rb_destroy_system and the per-system calls."""

    def __init__(self, n_bodies: int, box, shape: str = "cube", eps: float = 1.0,
                 sigma: float = 1.0, rcut: float = 2.5, max_neighbors: int = 0,
                 template=None, bead_mass: float = 1.0, stream=None, skin: float = 0.0,
                 potential: str = "lj", hphc=None):
        """potential: "lj" (eps, sigma, rcut), "hphc" (the continuous reading
        of Eq. 1) or "hphc_printed"; hphc = dict(A=, b=, c=, p=) for the two
        half-power half-cosine kinds."""
        L = load()
        d = _lib.rb_system_desc()
        d.body.shape = SHAPES[shape]
        self._tmpl_keep = None
        if shape == "custom":
            t = np.ascontiguousarray(template, dtype=np.float32)
            self._tmpl_keep = t
            d.body.n_beads = len(t)
            d.body.bead_xyz_host = t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        d.body.bead_mass = bead_mass
        d.pot.kind = POTENTIALS[potential]
        d.pot.eps, d.pot.sigma, d.pot.rcut = eps, sigma, rcut
        if potential != "lj":
            d.pot.A, d.pot.b, d.pot.c, d.pot.p = (float(hphc[k]) for k in ("A", "b", "c", "p"))
        box = np.broadcast_to(np.asarray(box, dtype=np.float32), (3,))
        for a in range(3):
            d.box[a] = float(box[a])
        d.n_bodies = int(n_bodies)
        d.max_neighbors = int(max_neighbors)
        d.skin = float(skin)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(L.rb_create_system(ctypes.byref(d), _stream_handle(self.stream), ctypes.byref(h)))
        self._h = h
        self.N = int(n_bodies)
        self.box = np.array(box, dtype=np.float32)
        m, r, rc = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        I = (ctypes.c_float * 3)()
        nb = ctypes.c_int32()
        check(L.rb_body_info(h, ctypes.byref(m), I, ctypes.byref(r), ctypes.byref(rc),
                             ctypes.byref(nb)))
        self.mass, self.inertia = m.value, np.array(list(I), dtype=np.float32)
        self.r_circ, self.pair_cutoff, self.n_beads = r.value, rc.value, nb.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().rb_destroy_system(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def template(self) -> np.ndarray:
        out = np.zeros((self.n_beads, 3), dtype=np.float32)
        check(load().rb_body_template(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_state(self, pos=None, quat=None, vel=None, angmom=None):
        arrs = [_ptr(x, 4) for x in (pos, quat, vel, angmom)]
        hosts = {h for (_, h) in arrs if _ is not None}
        if len(hosts) > 1:
            raise ValueError("pass all host arrays or all device tensors")
        host = hosts.pop() if hosts else 0
        ptrs = [(a.ctypes.data if host else a) if a is not None else None for a, _ in arrs]
        check(load().rb_set_state(self._h, *ptrs, host))

    def get_state(self, to_host: bool = False, out: dict = None, sync: bool = True):
        """rb_get_state.  `out`: preallocated tensors (page-locked host tensors
        with to_host) to fill; with to_host and sync=False the copies are only
        queued on the system's stream (rb_get_state's to_host = 2)."""
        keys = ("pos", "quat", "vel", "angmom")
        if out is not None:
            ptrs = [out[k].data_ptr() for k in keys]
        elif to_host:
            out = {k: np.zeros((self.N, 4), dtype=np.float32) for k in keys}
            ptrs = [out[k].ctypes.data for k in keys]
        else:
            out = {k: torch.empty((self.N, 4), dtype=torch.float32, device="cuda") for k in keys}
            ptrs = [out[k].data_ptr() for k in keys]
        mode = (1 if sync else 2) if to_host else 0
        check(load().rb_get_state(self._h, *ptrs, mode))
        return out

    def get_forces(self, to_host: bool = False, out=None, sync: bool = True):
        """rb_get_forces: (force, torque) rows of the last evaluation.  `out`:
        two preallocated tensors (page-locked host tensors with to_host); with
        to_host and sync=False the copies are only queued (to_host = 2)."""
        if out is not None:
            F, T = out
        elif to_host:
            F = torch.empty((self.N, 4), dtype=torch.float32).pin_memory()
            T = torch.empty((self.N, 4), dtype=torch.float32).pin_memory()
        else:
            F = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
            T = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        mode = (1 if sync else 2) if to_host else 0
        check(load().rb_get_forces(self._h, F.data_ptr(), T.data_ptr(), mode))
        return F, T

    def step_host_state(self, block: torch.Tensor, n_steps: int, dt: float,
                        path: int = RB_PATH_BEADS, mlp: "MLP" = None, precision="fp32",
                        sync: bool = True, copies: bool = False):
        """rb_step_host_state: `block` is a page-locked (6, N, 4) FP32 host tensor
        (pos, quat, vel, angmom, force, torque), updated in place.  copies: the
        copy form even where the direct form applies."""
        if block.is_cuda or block.dtype != torch.float32 or tuple(block.shape) != (6, self.N, 4) \
                or not block.is_contiguous():
            raise ValueError("block must be a contiguous (6, N, 4) float32 host tensor")
        check(load().rb_step_host_state(self._h, path, mlp.handle if mlp is not None else None,
                                        PRECISION[precision], int(n_steps), float(dt),
                                        block.data_ptr(), (1 if sync else 0) | (2 if copies else 0)))

    def set_forces(self, force, torque, path: int = RB_PATH_BEADS, mlp: "MLP" = None,
                   precision="fp32"):
        """rb_set_forces: give back the forces of the current state on `path`
        (device tensors, or host tensors: both the same kind)."""
        host = not force.is_cuda
        if torque.is_cuda == host:
            raise ValueError("force and torque must both be host or both device tensors")
        check(load().rb_set_forces(self._h, path, mlp.handle if mlp is not None else None,
                                   PRECISION[precision], force.data_ptr(), torque.data_ptr(),
                                   1 if host else 0))

    def build_pairs(self) -> int:
        n = ctypes.c_int64()
        check(load().rb_build_pairs(self._h, ctypes.byref(n)))
        return n.value

    def pairs(self) -> np.ndarray:
        n = ctypes.c_int64()
        check(load().rb_get_pairs(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        check(load().rb_get_pairs(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  n.value, ctypes.byref(n)))
        return out[: n.value]

    def _finish(self, st, F, T, e, v, energy, virial):
        check(st)
        res = {"force": F, "torque": T}
        if energy:
            res["energy"] = e.value
        if virial:
            res["virial"] = np.array(list(v)).reshape(3, 3)
        return res

    def forces_beads(self, energy: bool = False, virial: bool = False):
        F = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        T = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        e = ctypes.c_double()
        v = (ctypes.c_double * 9)()
        st = load().rb_forces_beads(self._h, F.data_ptr(), T.data_ptr(),
                                    ctypes.byref(e) if energy else None, v if virial else None)
        return self._finish(st, F, T, e, v, energy, virial)

    def forces_nn(self, mlp: "MLP", precision="fp32", energy: bool = False, virial: bool = False):
        F = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        T = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        e = ctypes.c_double()
        v = (ctypes.c_double * 9)()
        st = load().rb_forces_nn(self._h, mlp.handle, PRECISION[precision], F.data_ptr(),
                                 T.data_ptr(), ctypes.byref(e) if energy else None,
                                 v if virial else None)
        return self._finish(st, F, T, e, v, energy, virial)

    def step(self, n_steps: int, dt: float, path: int = RB_PATH_BEADS, mlp: "MLP" = None,
             precision="fp32"):
        check(load().rb_step(self._h, path, mlp.handle if mlp is not None else None,
                             PRECISION[precision], int(n_steps), float(dt)))

    def forces_fnet(self, fnet: "FNet", virial: bool = False):
        F = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        T = torch.empty((self.N, 4), dtype=torch.float32, device="cuda")
        v = (ctypes.c_double * 9)()
        st = load().rb_forces_fnet(self._h, fnet.handle, F.data_ptr(), T.data_ptr(),
                                   v if virial else None)
        return self._finish(st, F, T, None, v, False, virial)

    def step_fnet(self, fnet: "FNet", n_steps: int, dt: float):
        check(load().rb_step_fnet(self._h, fnet.handle, int(n_steps), float(dt)))

    def eval_pairs(self, path: int = RB_PATH_BEADS, mlp: "MLP" = None, precision="fp32"):
        check(load().rb_eval_pairs(self._h, path, mlp.handle if mlp is not None else None,
                                   PRECISION[precision]))

    def checkpoint(self, path: str):
        check(load().rb_checkpoint(self._h, str(path).encode()))

    def restore(self, path: str):
        check(load().rb_restore(self._h, str(path).encode()))

    @property
    def step_count(self) -> int:
        n = ctypes.c_int64()
        check(load().rb_get_step(self._h, ctypes.byref(n)))
        return n.value

    def set_skin(self, skin: float):
        check(load().rb_set_skin(self._h, float(skin)))

    def set_nn_fallback(self, rho_min: float):
        check(load().rb_set_nn_fallback(self._h, float(rho_min)))

    def nn_fallback_count(self) -> int:
        n = ctypes.c_int64()
        check(load().rb_nn_fallback_count(self._h, ctypes.byref(n)))
        return n.value

    def energy(self):
        e, kt, kr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(load().rb_energy(self._h, ctypes.byref(e), ctypes.byref(kt), ctypes.byref(kr)))
        return e.value, kt.value, kr.value

    def sync(self):
        check(load().rb_sync(self._h))

    def set_thermostat(self, kT: float, tau: float):
        """Nose-Hoover NVT for step() (tau <= 0: off, NVE)."""
        check(load().rb_set_thermostat(self._h, float(kT), float(tau)))

    def thermostat(self) -> dict:
        out = (ctypes.c_double * 4)()
        check(load().rb_get_thermostat(self._h, out))
        return {"xi": out[0], "eta": out[1], "Q": out[2], "g_kT": out[3]}

    def set_reference(self):
        check(load().rb_set_reference(self._h))

    def msd_msr(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        check(load().rb_msd_msr(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def images(self) -> np.ndarray:
        out = np.zeros((self.N, 4), dtype=np.int32)
        check(load().rb_get_images(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def gr_counts(self, r_max: float, n_bins: int, counts: torch.Tensor = None) -> torch.Tensor:
        """Adds this frame's pair-distance counts into `counts` (device int32
        tensor of n_bins, zero-initialised when None)."""
        if counts is None:
            counts = torch.zeros(n_bins, dtype=torch.int32, device="cuda")
        check(load().rb_gr_counts(self._h, float(r_max), int(n_bins), counts.data_ptr()))
        return counts

    def gr_normalise(self, counts, r_max: float, n_frames: int) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(counts, dtype=np.uint32))
        g = np.zeros(len(c))
        check(load().rb_gr_normalise(self._h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                     len(c), float(r_max), int(n_frames),
                                     g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return g


class MLP:
    """rb_mlp_create / rb_mlp_destroy and the network calls."""

    def __init__(self, width: int, depth: int = 3, stream=None):
        L = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(L.rb_mlp_create(int(width), int(depth), _stream_handle(self.stream), ctypes.byref(h)))
        self._h = h
        self.width, self.depth = int(width), int(depth)
        self.n_params = int(L.rb_mlp_n_params(int(width), int(depth)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().rb_mlp_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def set_params(self, flat):
        if isinstance(flat, torch.Tensor) and flat.is_cuda:
            t = flat.contiguous().float()
            check(load().rb_mlp_set_params(self._h, t.data_ptr(), t.numel(), 0))
            self._keep = t
        else:
            a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32).ravel())
            check(load().rb_mlp_set_params(self._h, a.ctypes.data, a.size, 1))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        check(load().rb_mlp_get_params(self._h, a.ctypes.data, a.size, 1))
        return a

    def set_symmetry(self, quats, inversion: bool):
        """rb_mlp_set_symmetry: evaluate on canonical configurations under this
        point group ((n, 4) unit quaternions as template_symmetry returns them;
        n = 0 detaches)."""
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        check(load().rb_mlp_set_symmetry(self._h, q.ctypes.data if len(q) else None, len(q),
                                         int(bool(inversion))))

    def set_cutoff(self, r_on: float, r_off: float):
        """rb_mlp_set_cutoff: energy times a smooth switch from 1 at r_on to 0 at
        r_off (r_off = 0 removes it)."""
        check(load().rb_mlp_set_cutoff(self._h, float(r_on), float(r_off)))

    def set_descriptor(self, kind: str = "paper6"):
        """rb_mlp_set_descriptor: "paper6" (the paper's six numbers of a cube
        pair; the cube's point group must be attached) or "features10"."""
        k = {"features10": RB_DESC_FEATURES10, "paper6": RB_DESC_PAPER6}[kind]
        check(load().rb_mlp_set_descriptor(self._h, k))

    def features(self, cfg: torch.Tensor) -> torch.Tensor:
        """rb_nn_features: (n, 10) raw network inputs of (n, 8) configurations."""
        _dev(cfg, 8)
        x = torch.empty((cfg.shape[0], 10), dtype=torch.float32, device="cuda")
        check(load().rb_nn_features(self._h, cfg.shape[0], cfg.data_ptr(), x.data_ptr()))
        check(load().rb_mlp_sync(self._h))
        return x

    def set_pair_symmetrised(self, on: bool = True):
        """rb_mlp_set_pair_symmetrised: system-level evaluations use the energy
        averaged over both choices of reference body of every pair."""
        check(load().rb_mlp_set_pair_symmetrised(self._h, int(bool(on))))

    def canonical(self, cfg: torch.Tensor, labels: torch.Tensor = None):
        """rb_nn_canonical in place on (n, 8) configurations [and (n, 12) labels]."""
        _dev(cfg, 8)
        if labels is not None:
            _dev(labels, 12)
        check(load().rb_nn_canonical(self._h, cfg.shape[0], cfg.data_ptr(),
                                     labels.data_ptr() if labels is not None else None))
        check(load().rb_mlp_sync(self._h))

    def pairs(self, cfg: torch.Tensor, precision="fp32", grad: bool = False):
        """rb_nn_pairs on (n, 8) configurations; returns (n, 12) [and (n, 8)]."""
        n = cfg.shape[0]
        _dev(cfg, 8)
        out = torch.empty((n, 12), dtype=torch.float32, device="cuda")
        g = torch.empty((n, 8), dtype=torch.float32, device="cuda") if grad else None
        check(load().rb_nn_pairs(self._h, PRECISION[precision], n, cfg.data_ptr(),
                                 out.data_ptr(), g.data_ptr() if grad else None))
        check(load().rb_mlp_sync(self._h))
        return (out, g) if grad else out


def template_symmetry(xyz):
    """rb_template_symmetry: (quats (n, 4) float32, inversion bool) of the point
    group of a bead template (n_beads, 3); host only."""
    t = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    q = np.zeros((24, 4), dtype=np.float32)
    n, inv = ctypes.c_int32(), ctypes.c_int32()
    check(load().rb_template_symmetry(t.ctypes.data, len(t), q.ctypes.data, ctypes.byref(n),
                                      ctypes.byref(inv)))
    return q[:n.value].copy(), bool(inv.value)


def peak_probe(kind: str, blocks_per_sm: int, iters: int, stream=None) -> float:
    """rb_peak_probe (asynchronous on the stream): one launch of the named
    probe ("ffma", "ffma2", "ex2", "rcp", "tanh"); returns the operations it
    issues (FMAs for the FMA probes)."""
    k = {"ffma": 0, "ffma2": 1, "ex2": 2, "rcp": 3, "tanh": 4}[kind]
    ops = ctypes.c_double()
    check(load().rb_peak_probe(k, int(blocks_per_sm), int(iters), _stream_handle(stream),
                               ctypes.byref(ops)))
    return ops.value


def tc_gemm_check(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """rb_tc_gemm_check: D = A B^T on one tensor-core tile (diagnostic)."""
    K = A.shape[1]
    N = B.shape[0]
    A = A.contiguous().float()
    B = B.contiguous().float()
    D = torch.empty((A.shape[0], N), dtype=torch.float32, device="cuda")
    check(load().rb_tc_gemm_check(N, K, A.data_ptr(), B.data_ptr(), D.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream))
    return D


def gemm_f32(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None, alpha: float = 1.0,
             beta: float = 0.0, split_k: bool = True) -> torch.Tensor:
    """rb_gemm_f32: C = alpha A B + beta C at FP32 accuracy on the tensor cores.
    A (M x K) and B (K x N) are FP32 CUDA tensors with any strides (in
    elements); C (M x N) row-major with unit column stride."""
    M, K = A.shape
    K2, N = B.shape
    if K2 != K:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    if C.stride(1) != 1 or C.shape != (M, N):
        raise ValueError("C must be M x N with unit column stride")
    ws = torch.empty(32 * M * N if split_k else 0, dtype=torch.float32, device="cuda")
    check(load().rb_gemm_f32(M, N, K, A.data_ptr(), A.stride(0), A.stride(1), B.data_ptr(),
                             B.stride(0), B.stride(1), C.data_ptr(), C.stride(0), float(alpha),
                             float(beta), ws.data_ptr() if split_k else None, ws.numel(),
                             torch.cuda.current_stream().cuda_stream))
    return C


class FNet:
    """rb_fnet_*: the five per-component force/torque networks of cylinders."""

    def __init__(self, width: int, depth: int = 3, stream=None):
        L = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(L.rb_fnet_create(int(width), int(depth), _stream_handle(self.stream), ctypes.byref(h)))
        self._h = h
        self.width, self.depth = int(width), int(depth)
        self.n_params = int(L.rb_fnet_n_params(int(width), int(depth)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().rb_fnet_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def set_params(self, flat):
        if isinstance(flat, torch.Tensor) and flat.is_cuda:
            t = flat.contiguous().float()
            check(load().rb_fnet_set_params(self._h, t.data_ptr(), t.numel(), 0))
            self._keep = t
        else:
            a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32).ravel())
            check(load().rb_fnet_set_params(self._h, a.ctypes.data, a.size, 1))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        check(load().rb_fnet_get_params(self._h, a.ctypes.data, a.size, 1))
        return a

    def pairs(self, cfg: torch.Tensor) -> torch.Tensor:
        """rb_fnet_pairs: cfg (n x 8: s, 0, q_rel) -> (n x 12: F_j, 0, tau_i, 0, tau_j, 0)."""
        _dev(cfg, 8)
        out = torch.empty((cfg.shape[0], 12), dtype=torch.float32, device="cuda")
        check(load().rb_fnet_pairs(self._h, cfg.shape[0], cfg.data_ptr(), out.data_ptr()))
        return out


class FNetTrainer:
    """rb_fnet_trainer_*: regression of the five components on bead labels."""

    def __init__(self, fnet: FNet, max_batch: int, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        h = ctypes.c_void_p()
        check(load().rb_fnet_trainer_create(fnet.handle, int(max_batch), lr, beta1, beta2, eps,
                                            ctypes.byref(h)))
        self._h = h
        self.fnet = fnet

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().rb_fnet_trainer_destroy(h)
            except Exception:
                pass
            self._h = None

    def set_lr(self, lr: float):
        check(load().rb_fnet_trainer_set_lr(self._h, float(lr)))

    def set_cap(self, cap: float, f_scale: float = 0.0):
        check(load().rb_fnet_trainer_set_cap(self._h, float(cap), float(f_scale)))

    def grad(self, cfg: torch.Tensor, labels: torch.Tensor):
        _dev(cfg, 8)
        _dev(labels, 12)
        g = torch.empty(self.fnet.n_params, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        check(load().rb_fnet_train_grad(self._h, cfg.shape[0], cfg.data_ptr(), labels.data_ptr(),
                                        g.data_ptr(), ctypes.byref(loss)))
        return loss.value, g

    def step(self, cfg: torch.Tensor, labels: torch.Tensor, loss: bool = False):
        _dev(cfg, 8)
        _dev(labels, 12)
        out = ctypes.c_double()
        check(load().rb_fnet_train_step(self._h, cfg.shape[0], cfg.data_ptr(), labels.data_ptr(),
                                        ctypes.byref(out) if loss else None))
        return out.value if loss else None


class Trainer:
    """rb_trainer_create / rb_train_grad / rb_train_step / rb_nn_weight_vjp."""

    def __init__(self, mlp: MLP, max_batch: int, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        h = ctypes.c_void_p()
        check(load().rb_trainer_create(mlp.handle, int(max_batch), lr, beta1, beta2, eps,
                                       ctypes.byref(h)))
        self._h = h
        self.mlp = mlp
        self.max_batch = int(max_batch)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().rb_trainer_destroy(h)
            except Exception:
                pass
            self._h = None

    def set_lr(self, lr: float):
        check(load().rb_trainer_set_lr(self._h, float(lr)))

    def grad(self, cfg: torch.Tensor, labels: torch.Tensor, lam_tau: float = 1.0,
             lam_E: float = 0.0, f_scale: float = 0.0, kT_w: float = 0.0):
        _dev(cfg, 8)
        _dev(labels, 12)
        g = torch.empty(self.mlp.n_params, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        check(load().rb_train_grad(self._h, cfg.shape[0], cfg.data_ptr(), labels.data_ptr(),
                                   lam_tau, lam_E, f_scale, kT_w, g.data_ptr(),
                                   ctypes.byref(loss)))
        return loss.value, g

    def step(self, cfg: torch.Tensor, labels: torch.Tensor, lam_tau: float = 1.0,
             lam_E: float = 0.0, want_loss: bool = True, f_scale: float = 0.0,
             kT_w: float = 0.0):
        _dev(cfg, 8)
        _dev(labels, 12)
        loss = ctypes.c_double()
        check(load().rb_train_step(self._h, cfg.shape[0], cfg.data_ptr(), labels.data_ptr(),
                                   lam_tau, lam_E, f_scale, kT_w,
                                   ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def weight_vjp(self, cfg: torch.Tensor, u_cfg: torch.Tensor, c: torch.Tensor):
        _dev(cfg, 8)
        _dev(u_cfg, 8)
        c = c.contiguous().float()
        g = torch.empty(self.mlp.n_params, dtype=torch.float32, device="cuda")
        check(load().rb_nn_weight_vjp(self._h, cfg.shape[0], cfg.data_ptr(), u_cfg.data_ptr(),
                                      c.data_ptr(), g.data_ptr()))
        return g


def sample_pairs(system: System, uniforms: torch.Tensor, contact: float = None):
    """rb_sample_pairs (rb_sample_pairs_at when `contact` is given): (cfg n x 8,
    labels n x 12, rho_contact n) on the device."""
    _dev(uniforms, 6)
    n = uniforms.shape[0]
    cfg = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    lab = torch.empty((n, 12), dtype=torch.float32, device="cuda")
    rc = torch.empty((n,), dtype=torch.float32, device="cuda")
    if contact is None:
        check(load().rb_sample_pairs(system.handle, n, uniforms.data_ptr(), cfg.data_ptr(),
                                     lab.data_ptr(), rc.data_ptr()))
    else:
        check(load().rb_sample_pairs_at(system.handle, n, uniforms.data_ptr(), float(contact),
                                        cfg.data_ptr(), lab.data_ptr(), rc.data_ptr()))
    return cfg, lab, rc


def pairs_swap_reference(cfg: torch.Tensor, labels: torch.Tensor = None, stream=None):
    """rb_pairs_swap_reference in place on (n, 8) configurations [and (n, 12)
    labels]: the same pairs described from the other body."""
    _dev(cfg, 8)
    if labels is not None:
        _dev(labels, 12)
    check(load().rb_pairs_swap_reference(cfg.shape[0], cfg.data_ptr(),
                                         labels.data_ptr() if labels is not None else None,
                                         _stream_handle(stream)))


def _desc(n_bodies: int, box, shape: str = "cube", eps=1.0, sigma=1.0, rcut=2.5,
          max_neighbors: int = 0, skin: float = 0.0):
    d = _lib.rb_system_desc()
    d.body.shape = SHAPES[shape]
    d.body.bead_mass = 1.0
    d.pot.kind = 0
    d.pot.eps, d.pot.sigma, d.pot.rcut = eps, sigma, rcut
    box = np.broadcast_to(np.asarray(box, dtype=np.float32), (3,))
    for a in range(3):
        d.box[a] = float(box[a])
    d.n_bodies = int(n_bodies)
    d.max_neighbors = int(max_neighbors)
    d.skin = float(skin)
    return d


def footprint(n_bodies: int, box, shape: str = "cube") -> int:
    """rb_system_footprint: device bytes of one system."""
    d = _desc(n_bodies, box, shape)
    return int(load().rb_system_footprint(ctypes.byref(d)))


def _result_dict(r) -> dict:
    return {f: getattr(r, f) for f, _ in r._fields_}


class Server:
    """rb_server_create / rb_submit / rb_poll / rb_wait / rb_fetch_state."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, mlp: MLP = None,
                 steps_per_tick: int = 8, lanes: int = None):
        h = ctypes.c_void_p()
        check(load().rb_server_create(int(hbm_budget_bytes), int(max_slots),
                                      mlp.handle if mlp is not None else None,
                                      int(steps_per_tick), ctypes.byref(h)))
        self._h = h
        self.mlp = mlp
        self._n = {}
        if lanes is not None:
            self.set_lanes(lanes)

    def set_network(self, shape: str, mlp: "MLP" = None, rho_min: float = 0.0):
        """rb_server_set_network: the network of network-path requests of bodies
        of this shape ("cube", "cylinder" or "custom"; None: the server's own)
        and its bead-fallback radius (0: none)."""
        check(load().rb_server_set_network(self._h, SHAPES[shape],
                                           mlp.handle if mlp is not None else None, float(rho_min)))
        if mlp is not None:
            self._nets = getattr(self, "_nets", {})
            self._nets[shape] = mlp  # keep it alive while the server may use it

    def set_lanes(self, lanes: int):
        """rb_server_set_lanes: lanes the replicas admitted from now on are spread over."""
        check(load().rb_server_set_lanes(self._h, int(lanes)))

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().rb_server_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, state: dict, box, shape: str = "cube", path: int = RB_PATH_BEADS,
               precision="fp32", n_steps: int = 100, dt: float = 0.002, skin: float = 0.0) -> int:
        n = len(state["pos"])
        d = _desc(n, box, shape, skin=skin)
        arrs = [np.ascontiguousarray(state[k], dtype=np.float32) for k in ("pos", "quat", "vel", "angmom")]
        t = ctypes.c_uint64()
        check(load().rb_submit(self._h, ctypes.byref(d), *[a.ctypes.data for a in arrs], path,
                               PRECISION[precision], int(n_steps), float(dt), ctypes.byref(t)))
        self._n[t.value] = n
        return t.value

    def poll(self, ticket: int):
        r = _lib.rb_result()
        st = load().rb_poll(self._h, ticket, ctypes.byref(r))
        if st == _lib.RB_ENOT_READY:
            return None
        check(st)
        return _result_dict(r)

    def wait(self, ticket: int, timeout_ms: int = 600000):
        r = _lib.rb_result()
        check(load().rb_wait(self._h, ticket, int(timeout_ms), ctypes.byref(r)))
        return _result_dict(r)

    def fetch_state(self, ticket: int) -> dict:
        n = self._n[ticket]
        out = {k: np.zeros((n, 4), dtype=np.float32) for k in ("pos", "quat", "vel", "angmom")}
        check(load().rb_fetch_state(self._h, ticket, *[out[k].ctypes.data for k in
                                                       ("pos", "quat", "vel", "angmom")]))
        return out

    def stats(self) -> dict:
        s = _lib.rb_server_stats_t()
        check(load().rb_server_stats(self._h, ctypes.byref(s)))
        return _result_dict(s)
