"""Stochastic search of the transmission parameters (Sec. 4).

Sec. 4 optimises the Robin / second-order transmission coefficients with the
Covariance Matrix Adaptation Evolution Strategy: each generation samples
lambda points from N(m, sigma^2 C), ranks them by cost, moves the mean to a
weighted average of the mu best, and adapts the step size sigma and the
covariance C, using evolution paths to carry information from previous
generations.  The paper uses a population of 25 and stops after 7200
iterations or below a tolerance of 5e-11 (Sec. 6).

Two costs are provided:

* ``fourier_rate`` / ``fourier_cost``: the maximum over a frequency band of the
  Fourier convergence factor of the two-subdomain Schwarz iteration (Sec. 3),
  |prod_s (p_s + q_s k^2 - k) / (p_s + q_s k^2 + k)|, with the operator
  A = p + q d2/dtau2 entering as the symbol p + q k^2 (the reading that
  reproduces Table 1).
* ``schwarz_iterations_cost``: the measured Schwarz iteration count of a
  gravimetry problem, evaluated for a whole generation at once by the
  batched GPU solve (``Solver.sample_p``).

The CMA-ES here is written from the algorithm's published description
(Hansen, "The CMA Evolution Strategy: A Tutorial", 2016): weighted
recombination, cumulative step-size adaptation, rank-one and rank-mu
covariance updates.  Only host-side arithmetic on a few coordinates lives
here; every cost evaluation of the Schwarz kind runs in the CUDA kernels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ------------------------------------------------------------ Fourier cost --

def fourier_rate(k, p1, q1=0.0, p2=None, q2=None):
    """Convergence factor of the two-subdomain iteration at frequency k."""
    if p2 is None:
        p2 = p1
    if q2 is None:
        q2 = q1
    k = np.asarray(k, dtype=np.float64)
    a1, a2 = p1 + q1 * k * k, p2 + q2 * k * k
    return np.abs((a1 - k) * (a2 - k) / ((a1 + k) * (a2 + k)))


def fourier_cost(params, kmin=0.0174, kmax=1.915, nk=4000, kind="oo0_sym"):
    """max_k rate over a log-spaced band; params in log space:
    oo0_sym (log p), oo0_unsym (log p1, log p2), oo2_sym (log p, log q),
    oo2_unsym (log p1, log q1, log p2, log q2)."""
    x = np.exp(np.asarray(params, dtype=np.float64))
    k = np.geomspace(kmin, kmax, nk)
    if kind == "oo0_sym":
        r = fourier_rate(k, x[0])
    elif kind == "oo0_unsym":
        r = fourier_rate(k, x[0], 0.0, x[1], 0.0)
    elif kind == "oo2_sym":
        r = fourier_rate(k, x[0], x[1])
    elif kind == "oo2_unsym":
        r = fourier_rate(k, x[0], x[1], x[2], x[3])
    else:
        raise ValueError(kind)
    return float(r.max())


# ------------------------------------------------------------------ CMA-ES --

@dataclass
class CMAResult:
    x: np.ndarray          # best point found
    f: float               # its cost
    mean: np.ndarray       # final distribution mean
    iterations: int
    evaluations: int
    stop: str


def cma_es(cost_batch, x0, sigma0, popsize=25, max_iter=7200, tol=5e-11, seed=0):
    """Minimise a cost over R^n.

    cost_batch(X) takes an array of candidates (lambda x n) and returns their
    costs (one batched evaluation per generation).  Stops after max_iter
    generations, when the spread of the generation's costs and the step
    size both fall below tol, or when sigma collapses numerically.
    """
    rng = np.random.default_rng(seed)
    m = np.asarray(x0, dtype=np.float64).copy()
    n = m.size
    lam = int(popsize)
    mu = lam // 2
    w = math.log(mu + 0.5) - np.log(np.arange(1, mu + 1))
    w = w / w.sum()
    mueff = 1.0 / np.sum(w * w)
    # adaptation rates
    cc = (4.0 + mueff / n) / (n + 4.0 + 2.0 * mueff / n)
    cs = (mueff + 2.0) / (n + mueff + 5.0)
    c1 = 2.0 / ((n + 1.3) ** 2 + mueff)
    cmu = min(1.0 - c1, 2.0 * (mueff - 2.0 + 1.0 / mueff) / ((n + 2.0) ** 2 + mueff))
    damps = 1.0 + 2.0 * max(0.0, math.sqrt((mueff - 1.0) / (n + 1.0)) - 1.0) + cs
    chi_n = math.sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n))
    sigma = float(sigma0)
    C = np.eye(n)
    pc = np.zeros(n)
    ps = np.zeros(n)
    best_x, best_f = m.copy(), math.inf
    evals = 0
    stop = "max_iter"
    it = 0
    for it in range(1, max_iter + 1):
        # C = B diag(D^2) B^T
        Cs = 0.5 * (C + C.T)
        evals_c, B = np.linalg.eigh(Cs)
        D = np.sqrt(np.maximum(evals_c, 1e-300))
        z = rng.standard_normal((lam, n))
        y = (z * D) @ B.T
        X = m + sigma * y
        f = np.asarray(cost_batch(X), dtype=np.float64)
        evals += lam
        order = np.argsort(f, kind="stable")
        if f[order[0]] < best_f:
            best_f, best_x = float(f[order[0]]), X[order[0]].copy()
        y_sel = y[order[:mu]]
        y_w = w @ y_sel
        m = m + sigma * y_w
        # step-size path (uses C^-1/2 y_w)
        c_inv_half_yw = B @ ((B.T @ y_w) / D)
        ps = (1.0 - cs) * ps + math.sqrt(cs * (2.0 - cs) * mueff) * c_inv_half_yw
        hsig = np.linalg.norm(ps) / math.sqrt(1.0 - (1.0 - cs) ** (2 * it)) / chi_n < 1.4 + 2.0 / (n + 1.0)
        pc = (1.0 - cc) * pc + (math.sqrt(cc * (2.0 - cc) * mueff) * y_w if hsig else 0.0)
        rank_mu = (y_sel.T * w) @ y_sel
        C = ((1.0 - c1 - cmu) * C + c1 * (np.outer(pc, pc) + (0.0 if hsig else cc * (2.0 - cc)) * C)
             + cmu * rank_mu)
        sigma *= math.exp((cs / damps) * (np.linalg.norm(ps) / chi_n - 1.0))
        spread = float(f[order[-1]] - f[order[0]])
        if spread < tol and sigma * float(D.max()) < tol:
            stop = "tol"
            break
        if sigma * float(D.max()) < 1e-14 * max(1.0, float(np.abs(m).max())):
            stop = "sigma"
            break
    return CMAResult(best_x, best_f, m, it, evals, stop)


def optimise_fourier(kind="oo0_sym", kmin=0.0174, kmax=1.915, seed=0, max_iter=7200, tol=5e-11):
    """CMA-ES on the Fourier cost (population 25, Sec. 4 / Sec. 6); returns
    (coefficients, rho_max)."""
    dim = {"oo0_sym": 1, "oo0_unsym": 2, "oo2_sym": 2, "oo2_unsym": 4}[kind]

    def batch(X):
        return [fourier_cost(x, kmin, kmax, kind=kind) for x in X]

    res = cma_es(batch, np.zeros(dim), 1.0, popsize=25, max_iter=max_iter, tol=tol, seed=seed)
    return np.exp(res.x), res.f, res


def interface_band(extent_a, extent_b, h):
    """Frequency band of an interface face with tangential extents a x b and
    smallest tangential element size h: from the lowest Dirichlet mode,
    pi sqrt(1/a^2 + 1/b^2), to pi over the Q2 node spacing h/2."""
    return math.pi * math.hypot(1.0 / extent_a, 1.0 / extent_b), math.pi / (0.5 * h)


def coefficients(kind, x):
    """(p_lo, q_lo, p_hi, q_hi) for osm_set_transmission from optimised
    parameters: the lower side of a face plays Omega^(1) of Sec. 3."""
    x = [float(v) for v in x]
    if kind == "oo0_sym":
        return (x[0], 0.0, x[0], 0.0)
    if kind == "oo0_unsym":
        return (x[0], 0.0, x[1], 0.0)
    if kind == "oo2_sym":
        return (x[0], x[1], x[0], x[1])
    if kind == "oo2_unsym":
        return (x[0], x[1], x[2], x[3])
    raise ValueError(kind)


def transmission_for_faces(extent_a, extent_b, h, kind="oo2_unsym", seed=0, max_iter=2000):
    """Sec. 4's procedure for a given mesh: CMA-ES on the Fourier rate over
    the faces' band.  Returns (p_lo, q_lo, p_hi, q_hi), rho_max, band."""
    kmin, kmax = interface_band(extent_a, extent_b, h)
    c, rho, _ = optimise_fourier(kind, kmin, kmax, seed=seed, max_iter=max_iter)
    return coefficients(kind, c), rho, (kmin, kmax)


# ------------------------------------------------- Schwarz iteration cost --

def schwarz_iterations_cost(solver, rtol=1e-8, max_outer=400, race=True):
    """Cost of log p: Schwarz iterations to rtol, one batched GPU run per
    generation.  A converged candidate costs its count plus its residual
    (a tie-break below half an iteration); one that was stopped before
    converging (at the cap, or, with race, when the generation's first
    candidate converged) costs its count plus 1/2 plus log10 of how far its
    residual still is from rtol, so the ranking among those follows the
    residual they reached."""

    def batch(X):
        ps = np.exp(np.asarray(X, dtype=np.float64)[:, 0])
        iters, rel, _ = solver.sample_p(ps, rtol=rtol, max_outer=max_outer, race=race)
        conv = rel <= rtol
        cost = iters.astype(np.float64) + 0.5 * np.where(conv, rel / rtol, 1.0)
        return cost + np.where(conv, 0.0, np.log10(np.maximum(rel / rtol, 1.0)))
    return batch


def search_p(solver, p0=10.0, sigma0=1.0, popsize=25, generations=10, rtol=1e-8, max_outer=400, seed=0,
             race=True):
    """CMA-ES over log p with the measured Schwarz iteration count as cost."""
    res = cma_es(schwarz_iterations_cost(solver, rtol, max_outer, race), np.array([math.log(p0)]), sigma0,
                 popsize=popsize, max_iter=generations, tol=0.5, seed=seed)
    return float(np.exp(res.x[0])), res
