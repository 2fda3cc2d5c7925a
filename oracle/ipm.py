"""Oracle of the interior-point outer loop (TEST INFRASTRUCTURE: only the test
suite, the smoke check and the benchmark's CPU baseline use it).

The loop the linear solver sits in (Sec. II: Newton's method on the barrier
problem with continuation mu -> 0, one KKT system K_k per iteration, Eq. 11),
written out plainly in NumPy / SciPy, FP64, in the order of its steps:

  problem   min F(x) = sum c2 Pg^2 + rho theta_ref^2  s.t.  c_E(x) = 0 (power balance),
            c_I(x) + s = u (|S|^2 at both line ends, u = Smax^2), s >= 0,
            xL <= x <= xU on V, Pg, Qg (Eqs. 1-4; slacks as in Eqs. 5-7);
            every term but rho theta_ref^2 depends on angle differences only,
            so that term fixes the reference angle (theta_ref = 0 at the
            optimum) without changing the optimal cost: it removes the
            uniform angle shift, a null direction of K held otherwise only
            by dw
  barrier   log terms on the bounds and on s (Sec. II, the barrier problem)
  Newton    with Sigma_x = zL/(x - xL) + zU/(xU - x) and Sigma_s = w/s, the
            multipliers of the bounds and the slacks eliminated:
              [H + Sigma_x + dw I   J_E^T   J_I^T            ] [dx  ]   [-(grad F + J^T lam - mu/(x-xL) + mu/(xU-x))]
              [J_E                  -dc I   0                ] [dlE ] = [-c_E                                      ]
              [J_I                  0       -(dc + s/w) I    ] [dlI ]   [-(c_I + s - u) - (mu/s - lam_I) s/w       ]
            then ds = (mu/s - lam_I - dlI) s/w, dzL = mu/(x-xL) - zL - Sigma_L dx,
            dzU = mu/(xU-x) - zU + Sigma_U dx, dw = mu/s - w - Sigma_s ds
  step      fraction to the boundary, tau = max(tau_min, 1 - mu): the largest
            alpha <= 1 keeping x - xL, xU - x, s above (1 - tau) times their
            values (primal: x, s, lam), likewise zL, zU, w (dual)
  barrier   mu <- max(tol / 10, min(kappa_mu mu, mu^theta_mu)) whenever the
  update    barrier error E_mu <= kappa_eps mu; stop when E_0 <= tol, where
            E_mu = max(||grad F + J^T lam - zL + zU||, ||c_E||, ||c_I + s - u||,
                       ||lam_I - w||, ||(x - xL) zL - mu||, ||(xU - x) zU - mu||,
                       ||s w - mu||)  (infinity norms)
  start     x0 pushed into [xL + p (xU - xL), xU - p (xU - xL)] (p = push),
            s0 = max(u - c_I(x0), p u), lam0 = 0, zL = mu0/(x - xL),
            zU = mu0/(xU - x), w = mu0/s0

Regularization: dc = 1e-8 on the balance rows' (2,2) diagonal (the
loop's reading; the graded benchmark matrices keep the literal 1e-10): with
1e-10, the elimination of those rows grows the factors by ~1e10 and the
library's static-pivot factorization loses ~10 digits on these matrices
(FGMRES(30) then stalls near 1e-8), while 1e-8 keeps every Newton solve
within a few FGMRES iterations; the step stays an inexact Newton step on
exactly evaluated residuals, so the optimum is unchanged.

The Newton matrix is assembled by the generator (kktgen: the model's exact
derivatives, with the slack term s/w on the flow rows' (2,2) diagonal) and
solved by scipy.sparse.linalg.spsolve. The library's own loop
(kkt_ipm_solve) takes the same steps with its GPU model evaluation and its
refactorization, so both reach the same optimum.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse.linalg as spla

from kktgen import KKTPoint, line_terms


@dataclass
class IPMOptions:
    tol: float = 1e-7
    max_iter: int = 200
    mu0: float = 0.1
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    delta_w: float = 1e-8
    delta_c: float = 1e-8
    push: float = 1e-2
    angle_ref: int = 0          # bus whose angle the pin term holds at 0
    angle_pin: float = 1.0      # rho


@dataclass
class IPMResult:
    x: np.ndarray
    lam: np.ndarray
    zL: np.ndarray
    zU: np.ndarray
    s: np.ndarray
    w: np.ndarray
    iters: int
    objective: float
    err: float
    mu: float
    history: list = field(default_factory=list)


def split(pat, x):
    g = pat.grid
    B, G = g.n_bus, g.n_gen
    return x[:B], x[B:2 * B], x[2 * B:2 * B + G], x[2 * B + G:]


def constraints(pat, data, x):
    """c_E (P then Q balance per bus) and c_I (|S|^2 at the from ends, then the to ends)."""
    g = pat.grid
    V, th, Pg, Qg = split(pat, x)
    (Pf, Qf, *_), (Pt, Qt, *_) = line_terms(g, V, th)
    Pb = -data.Pd.copy()
    Qb = -data.Qd.copy()
    np.add.at(Pb, g.gen_bus, Pg)
    np.add.at(Qb, g.gen_bus, Qg)
    np.add.at(Pb, g.f, -Pf)
    np.add.at(Pb, g.t, -Pt)
    np.add.at(Qb, g.f, -Qf)
    np.add.at(Qb, g.t, -Qt)
    cI = np.concatenate([Pf * Pf + Qf * Qf, Pt * Pt + Qt * Qt]) if pat.flow_limits else np.zeros(0)
    return np.concatenate([Pb, Qb]), cI


def objective(pat, x, opt=IPMOptions()):
    th = split(pat, x)[1][opt.angle_ref]
    return float(np.sum(pat.grid.c2 * split(pat, x)[2] ** 2) + opt.angle_pin * th * th)


def gradient(pat, x, opt=IPMOptions()):
    g = pat.grid
    out = np.zeros(x.size)
    out[2 * g.n_bus:2 * g.n_bus + g.n_gen] = 2.0 * g.c2 * split(pat, x)[2]
    out[g.n_bus + opt.angle_ref] = 2.0 * opt.angle_pin * x[g.n_bus + opt.angle_ref]
    return out


def jacobian(pat, x):
    """J (m x n) read off the assembled K at lam = 0, Sigma = 0, no regularization."""
    V, th, _, _ = split(pat, x)
    n = pat.n_primal
    K = pat.to_scipy(pat.values(KKTPoint(V, th, np.zeros(pat.n_dual), np.zeros(n), 0.0, 0.0, 0.0)))
    return K[n:, :n].tocsr()


def solve(pat, data, x0, opt: IPMOptions = IPMOptions()) -> IPMResult:
    g = pat.grid
    n, m = pat.n_primal, pat.n_dual
    mE = 2 * g.n_bus
    lo, hi = data.bounds(g)
    bl, bu = np.isfinite(lo), np.isfinite(hi)
    u = data.Smax ** 2
    uI = np.concatenate([u, u]) if pat.flow_limits else np.zeros(0)
    # start
    span = np.where(bl & bu, hi - lo, 1.0)
    x = np.array(x0, dtype=np.float64)
    x = np.where(bl, np.maximum(x, lo + opt.push * span), x)
    x = np.where(bu, np.minimum(x, hi - opt.push * span), x)
    _, cI = constraints(pat, data, x)
    s = np.maximum(uI - cI, opt.push * uI)
    lam = np.zeros(m)
    mu = opt.mu0
    dl = np.where(bl, x - lo, 1.0)
    du = np.where(bu, hi - x, 1.0)
    zL = np.where(bl, mu / dl, 0.0)
    zU = np.where(bu, mu / du, 0.0)
    w = mu / s
    hist = []
    err0 = np.inf
    it = 0
    for it in range(opt.max_iter + 1):
        cE, cI = constraints(pat, data, x)
        J = jacobian(pat, x)
        grad = gradient(pat, x, opt)
        dl = np.where(bl, x - lo, 1.0)
        du = np.where(bu, hi - x, 1.0)
        dual = grad + J.T @ lam - zL + zU
        rI = cI + s - uI
        lamI = lam[mE:]
        prods = np.concatenate([(dl * zL)[bl], (du * zU)[bu], s * w])

        def err(mu_):
            return max(np.max(np.abs(dual)), np.max(np.abs(cE)), np.max(np.abs(rI), initial=0.0),
                       np.max(np.abs(lamI - w), initial=0.0), np.max(np.abs(prods - mu_)))

        err0 = err(0.0)
        hist.append((it, objective(pat, x, opt), err0, mu))
        if err0 <= opt.tol or it == opt.max_iter:
            break
        while err(mu) <= opt.kappa_eps * mu and mu > opt.tol / 10:
            mu = max(opt.tol / 10, min(opt.kappa_mu * mu, mu ** opt.theta_mu))
        # Newton system
        sigma = np.where(bl, zL / dl, 0.0) + np.where(bu, zU / du, 0.0)
        sigma[g.n_bus + opt.angle_ref] += 2.0 * opt.angle_pin          # the pin term's Hessian
        D = s / w
        slack = np.concatenate([np.zeros(mE), D])
        V, th, _, _ = split(pat, x)
        K = pat.to_scipy(pat.values(KKTPoint(V, th, lam, sigma, mu, opt.delta_w, opt.delta_c, slack)))
        rx = grad + J.T @ lam - np.where(bl, mu / dl, 0.0) + np.where(bu, mu / du, 0.0)
        rhs = np.concatenate([-rx, -cE, -rI - (mu / s - lamI) * D])
        d = spla.spsolve(K.tocsc(), rhs)
        dx, dlam = d[:n], d[n:]
        dlI = dlam[mE:]
        ds = (mu / s - lamI - dlI) * D
        dzL = np.where(bl, mu / dl - zL - (zL / dl) * dx, 0.0)
        dzU = np.where(bu, mu / du - zU + (zU / du) * dx, 0.0)
        dw = mu / s - w - (w / s) * ds
        # fraction to the boundary
        tau = max(opt.tau_min, 1.0 - mu)

        def max_step(v, dv, mask):
            neg = mask & (dv < 0)
            return float(np.min(-tau * v[neg] / dv[neg])) if np.any(neg) else np.inf

        ap = min(1.0, max_step(dl, dx, bl), max_step(du, -dx, bu), max_step(s, ds, np.ones(s.size, bool)))
        ad = min(1.0, max_step(zL, dzL, bl), max_step(zU, dzU, bu), max_step(w, dw, np.ones(w.size, bool)))
        x = x + ap * dx
        s = s + ap * ds
        lam = lam + ap * dlam
        zL = zL + ad * dzL
        zU = zU + ad * dzU
        w = w + ad * dw
    return IPMResult(x=x, lam=lam, zL=zL, zU=zU, s=s, w=w, iters=it, objective=objective(pat, x, opt), err=float(err0),
                     mu=mu, history=hist)
