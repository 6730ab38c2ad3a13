"""Fit the pair energy network to bead-sum forces and torques on the device.

Every numerical step runs in the library: rb_sample_pairs draws and labels the
training pairs (bead sum), rb_train_step computes the force-matching loss
gradient and applies Adam, rb_nn_pairs evaluates held-out pairs.  This module
only sequences those calls (and picks the energy scale from label statistics
read back once).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import api, inputs


def train_network(shape: str = "cube", width: int = 128, depth: int = 3, n_samples: int = 200_000,
                  steps: int = 3000, batch: int = 4096, lr: float = 1e-3, lam_tau: float = 1.0,
                  lam_E: float = 0.0, seed: int = 2, time_limit_s: float | None = None,
                  log_every: int = 0, f_scale: float = 0.0, kT_w: float = 0.0,
                  symmetric: bool = True, contact: float = 1.0, cutoff_width: float = 0.0,
                  potential: str = "lj", hphc=None, swap_augment: bool = False,
                  descriptor: str = "features10"):
    """Returns (mlp, report).  With `symmetric` the body's point group is
    attached to the network (rb_mlp_set_symmetry), so it learns one copy of
    every class of symmetry-related configurations, and the feature
    normalisation is the mean and spread of the features of the canonical
    training configurations; otherwise it spans the separations contact..Rc
    isotropically.  e_scale and e_shift come from the label energies.
    `contact`: smallest bead-bead distance (sigma units) that defines contact
    for the sampled separations (rb_sample_pairs_at).  `cutoff_width` > 0:
    the energy is switched smoothly to zero between Rc - cutoff_width and Rc
    (rb_mlp_set_cutoff) during training and afterwards.  `potential`, `hphc`:
    the bead potential that labels the samples (as api.System).  `swap_augment`:
    the training set is doubled with every sample described from its other
    body (rb_pairs_swap_reference; the bead labels of two identical bodies
    are symmetric, so the swapped samples are exact)."""
    box = 60.0 if shape == "cube" else 70.0
    sysobj = api.System(8, [box] * 3, shape, potential=potential, hphc=hphc)
    Rc = sysobj.pair_cutoff
    u = torch.from_numpy(inputs.sampler_uniforms(n_samples + 10000, seed)).cuda()
    t0 = time.perf_counter()
    cfg, lab, rho_c = api.sample_pairs(sysobj, u, contact)
    torch.cuda.synchronize()
    t_sample = time.perf_counter() - t0
    cfg_tr, lab_tr = cfg[:n_samples], lab[:n_samples]
    cfg_te, lab_te = cfg[n_samples:], lab[n_samples:]
    if swap_augment:
        cfg_sw, lab_sw = cfg_tr.clone(), lab_tr.clone()
        api.pairs_swap_reference(cfg_sw, lab_sw)
        cfg_tr, lab_tr = torch.cat([cfg_tr, cfg_sw]), torch.cat([lab_tr, lab_sw])
    E = lab_tr[:, 3].double().cpu().numpy()
    rmin = float(rho_c.min().item())
    mu, isd = inputs.feature_normalisation(rmin, Rc)
    group = api.template_symmetry(sysobj.template()) if symmetric else None
    if descriptor == "paper6" and (group is None or shape != "cube"):
        raise ValueError("the paper's six numbers describe cube pairs under the cube's group")
    if group is not None:
        probe = api.MLP(width, depth)
        probe.set_params(inputs.mlp_params(width, depth, seed))
        probe.set_symmetry(*group)
        if descriptor == "paper6":
            probe.set_descriptor("paper6")
            x = probe.features(cfg_tr[:50000].contiguous()).double()
            mu = np.zeros(10)
            isd = np.zeros(10)
            mu[:6] = x[:, :6].mean(0).cpu().numpy()
            isd[:6] = 1.0 / np.maximum(x[:, :6].std(0).cpu().numpy(), 1e-3)
        else:
            cc = cfg_tr[:50000].clone()
            probe.canonical(cc)
            mu, isd = _feature_stats(cc)
    e_scale = float(np.std(np.clip(E, np.percentile(E, 1), np.percentile(E, 99)))) or 1.0
    e_shift = float(np.median(E))
    flat = inputs.mlp_params(width, depth, seed + 1, mu=mu, inv_sd=isd, e_scale=e_scale,
                             e_shift=e_shift)
    mlp = api.MLP(width, depth)
    mlp.set_params(flat)
    if group is not None:
        mlp.set_symmetry(*group)
        if descriptor == "paper6":
            mlp.set_descriptor("paper6")
    if cutoff_width > 0.0:
        mlp.set_cutoff(Rc - cutoff_width, Rc)
    tr = api.Trainer(mlp, batch, lr=lr)
    g = torch.Generator(device="cuda").manual_seed(seed)
    t0 = time.perf_counter()
    losses = []
    k = 0
    for k in range(steps):
        # cosine learning-rate decay to lr / 20
        tr.set_lr(lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps)))))
        idx = torch.randint(0, cfg_tr.shape[0], (batch,), device="cuda", generator=g)
        want = log_every and (k % log_every == 0)
        loss = tr.step(cfg_tr[idx].contiguous(), lab_tr[idx].contiguous(), lam_tau, lam_E,
                       want_loss=bool(want), f_scale=f_scale, kT_w=kT_w)
        if want:
            losses.append((k, loss))
        if time_limit_s is not None and time.perf_counter() - t0 > time_limit_s:
            break
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = mlp.pairs(cfg_te.contiguous(), "fp32")
    err = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    report = {"shape": shape, "width": width, "depth": depth, "samples": n_samples,
              "descriptor": descriptor,
              "swap_augment": swap_augment,
              "symmetry": (f"{len(group[0])} rotations" + (" + inversion" if group[1] else ""))
              if group is not None else None,
              "cutoff": [Rc - cutoff_width, Rc] if cutoff_width > 0.0 else None,
              "steps": k + 1, "batch": batch, "lr": lr, "f_scale": f_scale, "kT_w": kT_w, "t_sample_s": t_sample,
              "t_train_s": t_train, "rho_contact_min": rmin, "Rc": Rc,
              "heldout_e_F": err(out[:, 0:3], lab_te[:, 0:3]),
              "heldout_e_tau_i": err(out[:, 4:7], lab_te[:, 4:7]),
              "heldout_e_tau_j": err(out[:, 8:11], lab_te[:, 8:11]),
              "losses": losses}
    return mlp, report


def _feature_stats(cfg):
    """Mean and inverse spread of the network's 10 input features over
    configurations (n, 8): s, q_rel with a non-negative scalar part, rho,
    1/rho, rho^2."""
    s = cfg[:, :3].double()
    q = cfg[:, 4:8].double()
    q = torch.where(q[:, :1] < 0, -q, q)
    rho = torch.linalg.norm(s, dim=1, keepdim=True)
    x = torch.cat([s, q, rho, 1.0 / rho, rho * rho], 1)
    mu = x.mean(0).cpu().numpy()
    sd = x.std(0).cpu().numpy()
    return mu, 1.0 / np.maximum(sd, 1e-3)


def _err(a, b):
    return float(torch.linalg.norm(a[:, :3] - b[:, :3]) / torch.linalg.norm(b[:, :3]))


def _max_err(a, b):
    """max_i |a_i - b_i| / rms_i |b_i| over the bodies (the worst body's error
    in units of the typical force or torque)."""
    d = torch.linalg.norm(a[:, :3] - b[:, :3], dim=1)
    rms = torch.sqrt(torch.mean(torch.sum(b[:, :3].double() ** 2, dim=1)))
    return float(d.max() / rms)


def force_error(system: api.System, mlp: api.MLP, precision: str = "bf16"):
    """NN-versus-bead error of whole-system forces and torques (model error):
    e_F, e_tau (relative L2 over bodies) and the worst body's error over the
    rms (max_F_over_rms, max_tau_over_rms)."""
    ref = system.forces_beads()
    r = system.forces_nn(mlp, precision)
    system.sync()
    return {"e_F": _err(r["force"], ref["force"]), "e_tau": _err(r["torque"], ref["torque"]),
            "max_F_over_rms": _max_err(r["force"], ref["force"]),
            "max_tau_over_rms": _max_err(r["torque"], ref["torque"])}


def fnet_init(width: int, depth: int, Rc: float, cap: float, seed: int = 0) -> np.ndarray:
    """Initial parameters of the five per-component networks: weights
    N(0, 1/fan_in), zero biases, input normalisation from the ranges of the
    four numbers (p_r, p_z in [0, Rc], theta in [0, pi/2], phi in [-pi, pi]),
    output scale cap / 4 (targets are capped to [-cap, cap])."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(5):
        p = [np.array([Rc / 2, Rc / 2, np.pi / 4, 0.0]), np.array([2 / Rc, 2 / Rc, 4 / np.pi, 1 / np.pi])]
        fan = 4
        for _l in range(depth):
            p.append(rng.standard_normal(width * fan) / np.sqrt(fan))
            p.append(np.zeros(width))
            fan = width
        p.append(rng.standard_normal(width) / np.sqrt(width))
        p.append(np.array([0.0, cap / 4.0, 0.0]))
        parts.append(np.concatenate(p))
    return np.concatenate(parts).astype(np.float32)


def train_fnet(shape: str, width: int, depth: int, n_samples: int, steps: int, batch: int,
               lr: float, cap: float, contact: float = 1.0, seed: int = 0, f_scale: float = 0.0):
    """Per-component networks (rb_fnet) trained on the device: n_samples pairs
    drawn and labelled by the bead sum, capped regression, Adam with cosine
    decay.  Returns (fnet, report)."""
    s = api.System(8, [80.0] * 3, shape)
    u = torch.from_numpy(inputs.sampler_uniforms(n_samples, seed + 101)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cfg, lab, _ = api.sample_pairs(s, u, contact)
    torch.cuda.synchronize()
    t_sample = time.perf_counter() - t0
    f = api.FNet(width, depth)
    f.set_params(fnet_init(width, depth, s.pair_cutoff, cap, seed))
    tr = api.FNetTrainer(f, batch, lr=lr)
    tr.set_cap(cap, f_scale)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    t0 = time.perf_counter()
    first = None
    for k in range(steps):
        idx = torch.randint(0, n_samples, (batch,), device="cuda", generator=g)
        tr.set_lr(lr * 0.5 * (1.0 + np.cos(np.pi * k / max(1, steps))))
        loss = tr.step(cfg[idx].contiguous(), lab[idx].contiguous(), loss=(k == 0))
        if k == 0:
            first = loss
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    last = tr.grad(cfg[:batch].contiguous(), lab[:batch].contiguous())[0]
    return f, {"samples": n_samples, "steps": steps, "batch": batch, "cap": cap, "f_scale": f_scale,
               "contact": contact,
               "t_sample_s": t_sample, "t_train_s": t_train, "loss_first": first, "loss_last": last}


def fnet_force_error(system: api.System, f: api.FNet):
    """Per-component-network-versus-bead error of whole-system forces and torques."""
    ref = system.forces_beads()
    r = system.forces_fnet(f)
    system.sync()
    return {"e_F": _err(r["force"], ref["force"]), "e_tau": _err(r["torque"], ref["torque"]),
            "max_F_over_rms": _max_err(r["force"], ref["force"]),
            "max_tau_over_rms": _max_err(r["torque"], ref["torque"])}
