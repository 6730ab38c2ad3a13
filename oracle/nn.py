"""Oracle: the pair energy network and forces/torques as its gradients.

TEST INFRASTRUCTURE (see the package docstring).  PyTorch CPU, FP64.

The paper replaces the bead double sum by a network g_NN_U that maps the pair
configuration (centre-of-mass separation in the frame of body 1, and the
relative orientation) to the pair energy (Methods, U = g(x, Omega) ~ g_NN_U),
a plain fully connected feed-forward net (Methods, last paragraph; SI Sec. 1),
and takes forces and torques as gradients of that energy (SI Sec. 6:
f_i = -dE/dx_i, tau_eta = -dE/dtheta_eta).  The paper differentiates by
central finite differences; here the gradients are exact (reverse-mode
automatic differentiation of the plain forward definition), and the tests pin
them against central differences.

Readings (the paper leaves these open; the workload fixes some of them):
  * features x (10): s = R(q_i)^T R_ij (3), q_rel = q_i^* (x) q_j made
    canonical with a non-negative scalar part (4), then rho, 1/rho, rho^2
    with rho = |s|; a zero scalar part keeps the sign that makes the first
    non-zero vector component positive;
  * x_hat = (x - mu) * inv_sd with mu, inv_sd stored with the weights;
  * hidden layers z_l = W_l h_{l-1} + b_l, h_l = SiLU(z_l) = z_l sigmoid(z_l);
  * E = e_scale * (w_o . h_D + b_o) + e_shift;
  * torque = minus the derivative of E with respect to a small space-frame
    rotation theta applied as q -> (1, theta/2) (x) q (SI Sec. 6 defines the
    torque about an axis as -dE/dtheta about that axis).

Flat parameter layout (the library uses the same layout, FP32):
  mu[n_in], inv_sd[n_in], W1[w, n_in], b1[w], (W_l[w, w], b_l[w]) for
  l = 2..D, w_o[w], b_o, e_scale, e_shift.
"""
from __future__ import annotations

import numpy as np
import torch

N_IN = 10
DT = torch.float64


def n_params(width: int, depth: int = 3, n_in: int = N_IN) -> int:
    return 2 * n_in + width * n_in + width + (depth - 1) * (width * width + width) + width + 3


def unpack(flat, width: int, depth: int = 3, n_in: int = N_IN, sym=None, cutoff=None,
           desc=None) -> dict:
    """Split the flat parameter vector into named FP64 tensors (views).
    sym: optional point group (symmetry.point_group) -- the network then sees
    every pair configuration in its canonical form (symmetry.py).
    cutoff: optional (r_on, r_off) -- the energy is multiplied by switch().
    desc: None for the 10 features, "paper6" for the paper's six numbers of a
    cube pair (descriptor.py) in the first six inputs, the other four zero."""
    t = flat if isinstance(flat, torch.Tensor) else torch.as_tensor(np.asarray(flat))
    t = t.to(DT)
    assert t.numel() == n_params(width, depth, n_in), (t.numel(), n_params(width, depth, n_in))
    o = 0

    def take(*shape):
        nonlocal o
        n = int(np.prod(shape))
        v = t[o:o + n].reshape(shape)
        o += n
        return v

    p = {"mu": take(n_in), "inv_sd": take(n_in), "W": [], "b": []}
    p["W"].append(take(width, n_in))
    p["b"].append(take(width))
    for _ in range(depth - 1):
        p["W"].append(take(width, width))
        p["b"].append(take(width))
    p["w_o"] = take(width)
    p["b_o"] = take(1)[0]
    p["e_scale"] = take(1)[0]
    p["e_shift"] = take(1)[0]
    assert o == t.numel()
    p["sym"] = sym
    p["cutoff"] = cutoff
    p["desc"] = desc
    assert desc in (None, "paper6")
    return p


def _qmul(a, b):
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([aw * bw - ax * bx - ay * by - az * bz,
                        aw * bx + ax * bw + ay * bz - az * by,
                        aw * by - ax * bz + ay * bw + az * bx,
                        aw * bz + ax * by - ay * bx + az * bw], dim=-1)


def _qconj(q):
    return q * torch.tensor([1.0, -1.0, -1.0, -1.0], dtype=q.dtype)


def _to_body(q, v):
    """R(q)^T v = q^* v q (vector part)."""
    vq = torch.cat([torch.zeros_like(v[..., :1]), v], dim=-1)
    return _qmul(_qmul(_qconj(q), vq), q)[..., 1:]


def canonical_sign(q):
    """+1 or -1 per row so that sign * q has a non-negative scalar part; a
    zero scalar part makes the first non-zero vector component positive."""
    qd = q.detach()
    sgn = torch.where(qd[..., 0] < 0, -1.0, 1.0).to(q.dtype)
    tie = qd[..., 0] == 0
    if bool(tie.any()):
        for r in torch.nonzero(tie).flatten().tolist():
            for c in (1, 2, 3):
                if qd[r, c] != 0:
                    sgn[r] = 1.0 if qd[r, c] > 0 else -1.0
                    break
    return sgn


def features(s, q_rel):
    """x = [s, canonical q_rel, rho, 1/rho, rho^2] with rho = |s|."""
    qc = q_rel * canonical_sign(q_rel).unsqueeze(-1)
    rho = torch.sqrt((s * s).sum(-1, keepdim=True))
    return torch.cat([s, qc, rho, 1.0 / rho, rho * rho], dim=-1)


def mlp_energy(p: dict, x):
    """E(x) of the SiLU network on raw features x (normalised inside)."""
    h = (x - p["mu"]) * p["inv_sd"]
    for W, b in zip(p["W"], p["b"]):
        z = h @ W.T + b
        h = z * torch.sigmoid(z)
    e_hat = h @ p["w_o"] + p["b_o"]
    return p["e_scale"] * e_hat + p["e_shift"]


def switch(rho, r_on: float, r_off: float):
    """Smooth cutoff factor of the network energy (reading: the paper leaves the
    network energy at the pair cutoff open; the bead potential itself is
    shifted to zero at r_c).  1 for rho <= r_on, 0 for rho >= r_off, and in
    between the quintic 1 - t^3 (10 - 15 t + 6 t^2), t = (rho - r_on) /
    (r_off - r_on), whose first and second derivatives vanish at both ends."""
    t = torch.clamp((rho - r_on) / (r_off - r_on), 0.0, 1.0)
    return 1.0 - t ** 3 * (10.0 - 15.0 * t + 6.0 * t * t)


def config_energy(p: dict, s, q_rel):
    """Pair energy from the pair configuration in the frame of body i (in its
    canonical form under the point group when the network has one; times the
    smooth cutoff factor when the network has one)."""
    rho = torch.sqrt((s * s).sum(-1))
    if p.get("desc") == "paper6":
        from . import descriptor

        d = descriptor.describe(s, q_rel).reshape(s.shape[:-1] + (6,))
        x = torch.cat([d, torch.zeros(d.shape[:-1] + (N_IN - 6,), dtype=d.dtype)], -1)
    else:
        if p.get("sym") is not None:
            from . import symmetry

            s, q_rel = symmetry.canonical_torch(s, q_rel, p["sym"])
        x = features(s, q_rel)
    E = mlp_energy(p, x)
    if p.get("cutoff") is not None:
        E = E * switch(rho, *p["cutoff"])
    return E


def pair_forces(p: dict, R_ij, q_i, q_j):
    """Energy, forces and torques (space frame) of NN-evaluated body pairs.

    R_ij = p_j - p_i (minimum image), q_i, q_j unit quaternions; arrays of
    shape (B, 3), (B, 4), (B, 4).  Returns numpy FP64 arrays.
    """
    R = torch.as_tensor(np.asarray(R_ij, dtype=np.float64)).clone().requires_grad_(True)
    qi = torch.as_tensor(np.asarray(q_i, dtype=np.float64))
    qj = torch.as_tensor(np.asarray(q_j, dtype=np.float64))
    th_i = torch.zeros_like(R, requires_grad=True)
    th_j = torch.zeros_like(R, requires_grad=True)
    half = lambda th: torch.cat([torch.zeros_like(th[..., :1]), 0.5 * th], dim=-1)
    qi_t = qi + _qmul(half(th_i), qi)
    qj_t = qj + _qmul(half(th_j), qj)
    s = _to_body(qi_t, R)
    q_rel = _qmul(_qconj(qi_t), qj_t)
    E = config_energy(p, s, q_rel)
    gR, gi, gj = torch.autograd.grad(E.sum(), [R, th_i, th_j])
    return {"E": E.detach().numpy(), "F_i": gR.numpy(), "F_j": -gR.numpy(),
            "tau_i": -gi.numpy(), "tau_j": -gj.numpy()}


def forces_nn(p: dict, pos, quat, box, pairs):
    """Per-body NN forces/torques: each unordered listed pair (i, j), i < j,
    evaluated once with i as the reference body.  Returns F, tau, E_total,
    per-pair energies."""
    pos = np.asarray(pos, dtype=np.float64)
    quat = np.asarray(quat, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    N = len(pos)
    F = np.zeros((N, 3))
    tau = np.zeros((N, 3))
    if len(pairs) == 0:
        return F, tau, 0.0, np.zeros(0)
    i, j = pairs[:, 0], pairs[:, 1]
    d = pos[j] - pos[i]
    d = d - box * np.rint(d / box)
    r = pair_forces(p, d, quat[i], quat[j])
    np.add.at(F, i, r["F_i"])
    np.add.at(F, j, r["F_j"])
    np.add.at(tau, i, r["tau_i"])
    np.add.at(tau, j, r["tau_j"])
    return F, tau, float(r["E"].sum()), r["E"]


def forces_nn_symmetrised(p: dict, pos, quat, box, pairs):
    """Pair energy averaged over both choices of reference body,
    E_s(i, j) = (E(x_ij) + E(x_ji)) / 2, so that it does not depend on how
    the bodies are labelled; forces and torques are its gradients, i.e. the
    mean of forces_nn over the listed pairs and over the same pairs with the
    roles swapped.  Returns F, tau, E_total, per-pair E_s."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    F1, T1, E1, e1 = forces_nn(p, pos, quat, box, pairs)
    F2, T2, E2, e2 = forces_nn(p, pos, quat, box, pairs[:, ::-1])
    return 0.5 * (F1 + F2), 0.5 * (T1 + T2), 0.5 * (E1 + E2), 0.5 * (e1 + e2)


# ------------------------------------------------------------------ training

def predict_labels(p: dict, s, q_rel, create_graph: bool = False):
    """(E, F_j, tau_i, tau_j) in the frame of body i (q_i = identity) for pair
    configurations (s, q_rel); differentiable in the weights if create_graph."""
    s = s.clone().requires_grad_(True)
    th_i = torch.zeros_like(s, requires_grad=True)
    th_j = torch.zeros_like(s, requires_grad=True)
    ident = torch.zeros(s.shape[:-1] + (4,), dtype=s.dtype)
    ident[..., 0] = 1.0
    half = lambda th: torch.cat([torch.zeros_like(th[..., :1]), 0.5 * th], dim=-1)
    qi_t = ident + half(th_i)
    qj_t = q_rel + _qmul(half(th_j), q_rel)
    s_t = _to_body(qi_t, s)
    qr_t = _qmul(_qconj(qi_t), qj_t)
    E = config_energy(p, s_t, qr_t)
    gR, gi, gj = torch.autograd.grad(E.sum(), [s, th_i, th_j], create_graph=create_graph)
    return E, -gR, -gi, -gj


def force_matching_loss(flat, width, depth, pair_cfg, labels, lam_tau, lam_E, f_scale=None,
                        kT_w=None, sym=None, cutoff=None, desc=None):
    """L = mean_b w_b ( |F_j - F_j*|^2 + lam_tau (|tau_i - tau_i*|^2 + |tau_j - tau_j*|^2)
    + lam_E (E - E*)^2 ) with w_b = min(1, exp(-E*/kT_w)) / (1 + (|F_j*|^2 +
    lam_tau (|tau_i*|^2 + |tau_j*|^2)) / f_scale^2); each factor is 1 when its
    parameter is None.  (The paper's training pairs are Boltzmann-distributed,
    coming from simulations at T = 0.2 - 2.0, and it caps large force/torque
    targets, SI Sec. 6: these weights are their counterparts for uniformly drawn
    pairs.)
    pair_cfg: (B, 7) = s, q_rel; labels: (B, 10) =
    E, F_j, tau_i, tau_j (frame of body i).  Returns the loss and dL/dflat
    (zero for mu, inv_sd, e_scale, e_shift, which are not trained).

    parity unpinned for the loss definition itself: the paper trains on
    energies (and, for cylinders, separate force/torque nets) without giving
    the loss; the force-matching form is the workload's.  Its gradient is
    pinned by central differences in the tests.
    """
    flat_t = torch.as_tensor(np.asarray(flat, dtype=np.float64)).clone().requires_grad_(True)
    p = unpack(flat_t, width, depth, sym=sym, cutoff=cutoff, desc=desc)
    cfg = torch.as_tensor(np.asarray(pair_cfg, dtype=np.float64))
    lab = torch.as_tensor(np.asarray(labels, dtype=np.float64))
    E, Fj, ti, tj = predict_labels(p, cfg[:, :3], cfg[:, 3:7], create_graph=True)
    L = ((Fj - lab[:, 1:4]) ** 2).sum(-1) \
        + lam_tau * (((ti - lab[:, 4:7]) ** 2).sum(-1) + ((tj - lab[:, 7:10]) ** 2).sum(-1)) \
        + lam_E * (E - lab[:, 0]) ** 2
    if f_scale:
        mag2 = (lab[:, 1:4] ** 2).sum(-1) + lam_tau * ((lab[:, 4:7] ** 2).sum(-1)
                                                      + (lab[:, 7:10] ** 2).sum(-1))
        L = L / (1.0 + mag2 / f_scale ** 2)
    if kT_w:
        L = L * torch.exp(-torch.clamp(lab[:, 0], min=0.0) / kT_w)
    L = L.mean()
    (g,) = torch.autograd.grad(L, [flat_t])
    g = g.detach().numpy().copy()
    n_in = N_IN
    g[:2 * n_in] = 0.0
    g[-2:] = 0.0
    return float(L.detach()), g


def adam_update(flat, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on the trainable entries; returns new
    (flat, m, v).  The paper does not name its optimiser; Adam with these
    constants is the reading used."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    mask = np.ones_like(flat)
    mask[:2 * N_IN] = 0.0
    mask[-2:] = 0.0
    return flat - mask * lr * mh / (np.sqrt(vh) + eps), m, v
