"""FP64 reference for the soft-alignment tuning loss and its gradients
(test infrastructure only).

Not in the paper: the paper tunes the acceptance threshold and the gap
penalty by random search against human alignments (Section 5.2).  Here the
same two parameters, plus the classifier's four weights and bias, are tuned
by gradient descent on a smoothed alignment:

  f    = [ms/ls, mt/lt, |ls-lt|/max, min/max]          (overlap features)
  s    = sigmoid(w . f + b)                            (sentence similarity)
  V    = soft Needleman-Wunsch value: every max of the fill replaced by
         gamma * log-sum-exp(. / gamma), same borders -i p and -j p
  E    = dV / ds                                       (expected alignment)
  G    = sigmoid((s - thr) / tau)                      (soft acceptance gate)
  P    = clamp(E * G, eps, 1 - eps)
  loss = mean over all cells of all pairs of BCE(P, gold)

Plain PyTorch CPU ops in float64: the value is a cell-by-cell loop written
from the definition, E comes from autograd with create_graph=True and the
parameter gradients from a second autograd pass (derivative of the
derivative).  Slow; for small pairs only.
"""
from __future__ import annotations

import numpy as np
import torch

T = torch.float64


def soft_value(s: torch.Tensor, p: torch.Tensor, gamma: float) -> torch.Tensor:
    """V(N, M) for an N x M similarity tensor (cell loop, definition order)."""
    N, M = s.shape
    V = [[None] * (M + 1) for _ in range(N + 1)]
    V[0][0] = torch.zeros((), dtype=T)
    for i in range(1, N + 1):
        V[i][0] = V[i - 1][0] - p
    for j in range(1, M + 1):
        V[0][j] = V[0][j - 1] - p
    for i in range(1, N + 1):
        for j in range(1, M + 1):
            c = torch.stack([V[i - 1][j - 1] + s[i - 1, j - 1], V[i - 1][j] - p, V[i][j - 1] - p])
            V[i][j] = gamma * torch.logsumexp(c / gamma, 0)
    return V[N][M]


def features(ms, mt, ls, lt) -> torch.Tensor:
    """N x M x 4 feature tensor from integer counts and sentence lengths."""
    ms = torch.as_tensor(np.asarray(ms), dtype=T)
    mt = torch.as_tensor(np.asarray(mt), dtype=T)
    a = torch.as_tensor(np.asarray(ls), dtype=T)[:, None].expand_as(ms)
    b = torch.as_tensor(np.asarray(lt), dtype=T)[None, :].expand_as(ms)
    mx, mn = torch.maximum(a, b), torch.minimum(a, b)
    return torch.stack([ms / a, mt / b, (a - b).abs() / mx, mn / mx], dim=-1)


def loss(pairs, theta: torch.Tensor, gamma: float, tau: float, eps: float = 1e-7,
         create_graph: bool = True) -> torch.Tensor:
    """pairs: list of (ms, mt, ls, lt, gold) with ms/mt/gold N x M arrays.
    theta = [w1, w2, w3, w4, b, gap, thr] (float64 tensor)."""
    w, b, gap, thr = theta[:4], theta[4], theta[5], theta[6]
    tot = torch.zeros((), dtype=T)
    cells = 0
    for ms, mt, ls, lt, gold in pairs:
        f = features(ms, mt, ls, lt)
        s = torch.sigmoid(f @ w + b)
        N, M = s.shape
        cells += N * M
        if N == 0 or M == 0:
            continue
        if not s.requires_grad:  # loss value only: E still needs dV/ds
            s = s.detach().requires_grad_(True)
        V = soft_value(s, gap, gamma)
        (E,) = torch.autograd.grad(V, s, create_graph=create_graph)
        G = torch.sigmoid((s - thr) / tau)
        P = torch.clamp(E * G, eps, 1.0 - eps)
        g = torch.as_tensor(np.asarray(gold), dtype=T)
        tot = tot - (g * torch.log(P) + (1 - g) * torch.log(1 - P)).sum()
    return tot / max(cells, 1)


def loss_and_grad(pairs, theta, gamma, tau, eps=1e-7):
    """(loss, d loss / d theta) as NumPy float64."""
    th = torch.as_tensor(np.asarray(theta, np.float64), dtype=T).clone().requires_grad_(True)
    L = loss(pairs, th, gamma, tau, eps)
    (g,) = torch.autograd.grad(L, th)
    return float(L.detach()), g.numpy()


def loss_value(pairs, theta, gamma, tau, eps=1e-7) -> float:
    """Loss only (still differentiates V once, to get E)."""
    th = torch.as_tensor(np.asarray(theta, np.float64), dtype=T)
    return float(loss(pairs, th, gamma, tau, eps, create_graph=False))


def hvp_cells(ms, mt, ls, lt, gold, theta, gamma, tau, n_cells_total, eps=1e-7):
    """For one pair: (E, u, H u) with u = dL/dE at fixed s (loss normalised by
    n_cells_total), H the Hessian of V in s; all float64 numpy arrays."""
    th = torch.as_tensor(np.asarray(theta, np.float64), dtype=T)
    w, b, gap, thr = th[:4], th[4], th[5], th[6]
    f = features(ms, mt, ls, lt)
    s = torch.sigmoid(f @ w + b).detach().requires_grad_(True)
    V = soft_value(s, gap, gamma)
    (E,) = torch.autograd.grad(V, s, create_graph=True)
    Ed = E.detach().requires_grad_(True)
    G = torch.sigmoid((s.detach() - thr) / tau)
    P = torch.clamp(Ed * G, eps, 1.0 - eps)
    g = torch.as_tensor(np.asarray(gold), dtype=T)
    L = -(g * torch.log(P) + (1 - g) * torch.log(1 - P)).sum() / n_cells_total
    (u,) = torch.autograd.grad(L, Ed)
    (hu,) = torch.autograd.grad(E, s, grad_outputs=u)
    return E.detach().numpy(), u.numpy(), hu.numpy()
