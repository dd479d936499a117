"""An independent FP64 restatement of the forward estimator in plain torch
ops, differentiated by torch.autograd. Test helper only: it pins the
oracle's hand-written reverse sweep (back-propagation, Sec. IV-C of arXiv
2002.02481) against a general-purpose AD engine.

It shares no code with the oracle; the only thing it takes from the oracle
is the array of normals (pinned on its own against cuRAND).
"""
import math

import numpy as np
import torch


def forward_price(spot, time, sigma, S0, r, K, T, n_steps, phi, Z, interp=0, scheme=0):
    """Mean discounted payoff of Euler paths driven by Z [P, N] under the
    bilinear local-vol grid (spot [I], time [J], sigma [I, J]): on ln S
    (scheme 0) or on S (scheme 1), with the spot weight linear in S
    (interp 0) or in ln S (interp 1).

    The cell convention is the largest node index at or below the point,
    clamped so that the cell has a right neighbour; weights are clamped to
    [0, 1] (flat outside the grid)."""
    I, J = spot.shape[0], time.shape[0]
    P = Z.shape[0]
    r = torch.as_tensor(r, dtype=torch.float64)
    T = torch.as_tensor(T, dtype=torch.float64)
    dt = T / n_steps
    sqdt = torch.sqrt(dt)
    state = (torch.log(S0) if scheme == 0 else S0) * torch.ones(P, dtype=torch.float64)
    for n in range(n_steps):
        t = n * dt
        S = torch.exp(state) if scheme == 0 else state
        i = torch.clamp(torch.searchsorted(spot, S.detach(), right=True) - 1, 0, I - 2)
        if interp == 0:
            u = torch.clamp((S - spot[i]) / (spot[i + 1] - spot[i]), 0.0, 1.0)
        else:
            u = torch.clamp((torch.log(S) - torch.log(spot[i])) / (torch.log(spot[i + 1]) - torch.log(spot[i])),
                            0.0, 1.0)
        if J > 1:
            tt = t.detach().reshape(1)
            j = int(torch.clamp(torch.searchsorted(time, tt, right=True) - 1, 0, J - 2).item())
            if float(tt) >= float(time[J - 1]):
                v = torch.tensor(1.0, dtype=torch.float64)      # flat in t beyond the last node
            else:
                v = torch.clamp((t - time[j]) / (time[j + 1] - time[j]), 0.0, 1.0)
            lo = sigma[i, j] * (1 - u) + sigma[i + 1, j] * u
            hi = sigma[i, j + 1] * (1 - u) + sigma[i + 1, j + 1] * u
            sig = lo * (1 - v) + hi * v
        else:
            sig = sigma[i, 0] * (1 - u) + sigma[i + 1, 0] * u
        if scheme == 0:
            state = state + (r - 0.5 * sig * sig) * dt + sig * sqdt * Z[:, n]
        else:
            state = state + r * state * dt + sig * state * sqdt * Z[:, n]
    SN = torch.exp(state) if scheme == 0 else state
    V = torch.exp(-r * T) * torch.relu(phi * (SN - K))
    return V.mean(), SN


def autograd_greeks(spot, time, sigma, S0, r, K, T, n_steps, phi, Z, interp=0, scheme=0):
    """(price, delta, vega [I, J], S_N [P]) by torch.autograd, all FP64."""
    sp = torch.tensor(spot, dtype=torch.float64)
    tm = torch.tensor(time, dtype=torch.float64)
    sg = torch.tensor(sigma, dtype=torch.float64, requires_grad=True)
    s0 = torch.tensor(float(S0), dtype=torch.float64, requires_grad=True)
    z = torch.tensor(Z, dtype=torch.float64)
    price, SN = forward_price(sp, tm, sg, s0, r, K, T, n_steps, phi, z, interp, scheme)
    d_s0, d_sig = torch.autograd.grad(price, [s0, sg])
    return float(price.detach()), float(d_s0), d_sig.numpy(), SN.detach().numpy()


def autograd_all(spot, time, sigma, S0, r, K, T, n_steps, phi, Z, interp=0, scheme=0):
    """Price and its derivatives in S0, every sigma_ij, r and T (n_steps
    fixed) by torch.autograd, all FP64, as a dict."""
    sp = torch.tensor(spot, dtype=torch.float64)
    tm = torch.tensor(time, dtype=torch.float64)
    sg = torch.tensor(sigma, dtype=torch.float64, requires_grad=True)
    s0 = torch.tensor(float(S0), dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(float(r), dtype=torch.float64, requires_grad=True)
    Tt = torch.tensor(float(T), dtype=torch.float64, requires_grad=True)
    z = torch.tensor(Z, dtype=torch.float64)
    price, _ = forward_price(sp, tm, sg, s0, rt, K, Tt, n_steps, phi, z, interp, scheme)
    d_s0, d_sig, d_r, d_T = torch.autograd.grad(price, [s0, sg, rt, Tt])
    return dict(price=float(price.detach()), delta=float(d_s0), vega=d_sig.numpy(), rho=float(d_r),
                dVdT=float(d_T))


def vanna_at_fixed_path(spot, time, sigma, S0, r, K, T, phi, x, cells):
    """Second-order buckets of one fixed Euler path on ln S: the gradient in
    sigma of the path's pathwise delta at the fixed path, plus that delta
    times the gradient of the path's log density (each step Gaussian with
    mean x_n + (r - sigma_n^2/2) dt and standard deviation sigma_n sqrt(dt)),
    both by torch.autograd, FP64.

    x: [N + 1] ln S_0 .. ln S_N; cells: per step (i, j, u, v, inside), the
    bilinear cell and weights at (S_n, t_n), fixed with the path. Returns
    [I, J]."""
    sp = [float(a) for a in spot]
    I, J = len(sp), len(time)
    sg = torch.tensor(sigma, dtype=torch.float64, requires_grad=True)
    N = len(x) - 1
    dt = T / N
    D = torch.ones((), dtype=torch.float64)
    logp = torch.zeros((), dtype=torch.float64)
    for n in range(N):
        i, j, u, v, inside = cells[n]
        S = math.exp(x[n])
        if J > 1:
            lo = sg[i, j] * (1 - u) + sg[i + 1, j] * u
            hi = sg[i, j + 1] * (1 - u) + sg[i + 1, j + 1] * u
            sig = lo * (1 - v) + hi * v
            slope = (1 - v) * (sg[i + 1, j] - sg[i, j]) + v * (sg[i + 1, j + 1] - sg[i, j + 1])
        else:
            sig = sg[i, 0] * (1 - u) + sg[i + 1, 0] * u
            slope = sg[i + 1, 0] - sg[i, 0]
        kappa = S * slope / (sp[i + 1] - sp[i]) if inside else torch.zeros((), dtype=torch.float64)
        dx = x[n + 1] - x[n]
        h = (dx - r * dt) / sig - sig * dt / 2            # d x_{n+1} / d sigma_n along the path
        D = D * (1 + h * kappa)
        e = dx - (r - sig * sig / 2) * dt
        logp = logp - e * e / (2 * sig * sig * dt) - torch.log(sig)
    SN = math.exp(x[N])
    if not phi * (SN - K) > 0:
        return np.zeros((I, J))
    delta = math.exp(-r * T) * phi * SN * D / S0
    (g_delta,) = torch.autograd.grad(delta, [sg], retain_graph=True)
    (g_logp,) = torch.autograd.grad(logp, [sg])
    return (g_delta + delta.detach() * g_logp).numpy()
