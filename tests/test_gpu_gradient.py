"""Adjoint gradient of the surface-gravity misfit (GPU, through the C ABI)
against the oracle's monolithic gradient and against finite differences.

J(drho) = 1/2 ||B phi(drho) - g_obs||^2 is exactly quadratic in drho, so the
central difference of J equals the directional derivative for any step; with
phi linear in drho it can be evaluated without cancellation as
r . (B phi(d)) (r = B phi - g_obs, phi(d) the solve with density d), which
checks the adjoint solve against independent forward solves.
Tolerances: solves to a relative residual of 1e-12; gradients compared in the
normalised form |a - b| <= tol ||b|| (tol 1e-7 against the oracle, 1e-5 for
the finite differences, the target of the gradient check).
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm(cuda_ok):
    from paper_2112_03851_gb300 import build
    build.build()
    import paper_2112_03851_gb300 as pkg
    pkg.load()
    return pkg


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def small_case(n=12, s=3, m=16):
    prob = gen.layered_problem(n, s, p=8.0, seed=2, n_spheres=6)
    st = gen.surface_stations(m)
    rng = np.random.default_rng(4)
    perturbed = prob.drho + rng.normal(0.0, 20.0, prob.drho.size)
    return prob, st, perturbed


def test_device_load_equals_host_load(osm):
    prob, _, _ = small_case()
    a = osm.Solver.from_problem(prob, inner_rtol=1e-13, max_outer=2000)
    b = osm.Solver.from_problem(prob, inner_rtol=1e-13, max_outer=2000)
    b.set_density(np.zeros_like(prob.drho))
    b.set_density_dev(_t(prob.drho))
    pa, na, ra = a.solve(1e-12)
    pb, nb, rb = b.solve(1e-12)
    assert na == nb
    assert float((pa - pb).norm() / pa.norm()) <= 1e-12


def test_gravity_operator_matches_oracle(osm):
    prob, st, _ = small_case()
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-13, max_outer=2000)
    sol.set_stations(st)
    phi, _, _ = sol.solve(1e-12)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    B = oracle.station_matrix(G, st)
    g_ref = B @ phi.cpu().numpy()[G.gnode]
    g = sol.gravity(phi).cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-13 * np.abs(g_ref).max()


def test_potential_vjp_matches_oracle(osm):
    prob, _, _ = small_case()
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-13, max_outer=2000)
    M = oracle.Misfit(prob.xc, prob.yc, prob.zc, gen.surface_stations(4))
    rng = np.random.default_rng(8)
    v = np.zeros(sol.info["n_nodes"])
    v[M.G.gnode] = rng.standard_normal(M.G.n)
    grad = sol.potential_vjp(_t(v), rtol=1e-12).cpu().numpy()
    w, _, _ = M.G.solve(v[M.G.gnode], tol=1e-14)
    ref = M.F.T @ w
    assert np.linalg.norm(grad - ref) <= 1e-7 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_misfit_gradient_matches_oracle(osm, prec):
    prob, st, perturbed = small_case()
    M = oracle.Misfit(prob.xc, prob.yc, prob.zc, st)
    g_obs = M.gravity(perturbed)                         # observations from the oracle
    J_ref, grad_ref = M.value_and_grad(prob.drho, g_obs)
    sol = osm.Solver.from_problem(prob, prec=prec, inner_rtol=1e-13, max_outer=2000)
    sol.set_stations(st)
    sol.set_density_dev(_t(prob.drho))
    rtol, tol = (1e-12, 1e-7) if prec == "fp64" else (1e-10, 1e-6)
    J, grad, dJdp = sol.grad(_t(g_obs), rtol=rtol)
    grad = grad.cpu().numpy()
    assert abs(J - J_ref) <= 10 * tol * J_ref
    assert np.linalg.norm(grad - grad_ref) <= tol * np.linalg.norm(grad_ref)
    assert dJdp == 0.0


def test_autograd_functions(osm):
    import torch
    prob, st, perturbed = small_case()
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-13, max_outer=2000)
    sol.set_stations(st)
    M = oracle.Misfit(prob.xc, prob.yc, prob.zc, st)
    g_obs = _t(M.gravity(perturbed))
    drho = _t(prob.drho).requires_grad_(True)
    J = osm.gravity_misfit(drho, g_obs, sol, rtol=1e-12)
    (gJ,) = torch.autograd.grad(J, drho)
    _, grad, _ = sol.grad(g_obs, rtol=1e-12)
    assert torch.equal(gJ, grad)
    # the potential: d/d drho of sum(c * phi) equals the VJP with v = c
    c = torch.randn(sol.info["n_nodes"], dtype=torch.float64, device="cuda")
    phi = osm.gravity_potential(drho, sol, rtol=1e-12)
    (gphi,) = torch.autograd.grad((c * phi).sum(), drho)
    ref = sol.potential_vjp(c, rtol=1e-12)
    assert float((gphi - ref).norm() / ref.norm()) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gradient_against_finite_differences_full_size(osm, prec):
    """48^3 Q2, 3x3x3 subdomains, 64x64 surface stations, g_obs from a
    density perturbed by N(0, 20^2): 50 seeded unit element directions, in
    FP64 (solves to 1e-12) and in the mixed form (FP32 subdomain CG at the
    bench's inner tolerance 0.4, forward and adjoint solves to 1e-10)."""
    prob = gen.workload("layered48")
    st = gen.surface_stations(64)
    rng = np.random.default_rng(0)
    rt = 1e-12 if prec == "fp64" else 1e-10
    sol = osm.Solver.from_problem(prob, p=10.0, prec=prec, mixed_inner_rtol=0.4, inner_rtol=1e-13, max_outer=3000)
    sol.set_stations(st)
    sol.set_density_dev(_t(prob.drho + rng.normal(0.0, 20.0, prob.drho.size)))
    phi_obs, _, _ = sol.solve(rt)
    g_obs = sol.gravity(phi_obs)
    sol.set_density_dev(_t(prob.drho))
    J, grad, _ = sol.grad(g_obs, rtol=rt)
    phi, _, _ = sol.solve(rt)
    r = (sol.gravity(phi) - g_obs).cpu().numpy()
    grad = grad.cpu().numpy()
    gnorm = np.linalg.norm(grad)
    worst = 0.0
    for _ in range(50):
        d = rng.standard_normal(prob.drho.size)
        d /= np.linalg.norm(d)
        sol.set_density_dev(_t(d))
        phi_d, _, _ = sol.solve(rt)
        fd = float(r @ sol.gravity(phi_d).cpu().numpy())   # (J(+h) - J(-h)) / 2h, exactly
        worst = max(worst, abs(fd - grad @ d) / gnorm)
    assert worst <= 1e-5, worst
    if prec != "fp64":
        return
    # one plain central difference with the absolute step h = 1e-6: at solve
    # accuracy 1e-12 its cancellation noise is ~1e-2 ||grad||, so it is only
    # a coarse check; the linearity form above is the exact one
    d = rng.standard_normal(prob.drho.size)
    d /= np.linalg.norm(d)
    Js = []
    for sgn in (1.0, -1.0):
        sol.set_density_dev(_t(prob.drho + sgn * 1e-6 * d))
        ph, _, _ = sol.solve(1e-12)
        Js.append(0.5 * float(((sol.gravity(ph) - g_obs) ** 2).sum()))
    fd = (Js[0] - Js[1]) / 2e-6
    assert abs(fd - grad @ d) <= 0.1 * gnorm


def test_truncated_schwarz_p_gradient(osm):
    """dJ_N/dp of the misfit after exactly N Schwarz iterations, by reverse-
    mode Schwarz on the GPU, against central differences of the oracle's own
    truncated sequential Schwarz (subdomain solves to 1e-14 on both sides)."""
    prob = gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0, seed=4, lx=10.0, ly=8.0, lz=3.0)
    st = gen.surface_stations(8, lx=10.0, ly=8.0, z=3.0)
    M = oracle.Misfit(prob.xc, prob.yc, prob.zc, st)
    g_obs = M.gravity(prob.drho * 1.1)
    N, p0 = 10, 2.0

    def J_oracle(p):
        S = oracle.Schwarz.from_problem(prob, p=p)
        for _ in range(N):
            S.iterate(inner_rtol=1e-14)
        phi, _ = S.residual()
        r = M.B @ phi[M.G.gnode] - g_obs
        return 0.5 * float(r @ r)

    sol = osm.Solver.from_problem(prob, p=p0, inner_rtol=1e-14, max_outer=400)   # the solve below needs 175
    sol.set_stations(st)
    J, dJdp = sol.grad_p(_t(g_obs), N)
    J_ref = J_oracle(p0)
    assert abs(J - J_ref) <= 1e-9 * J_ref
    h = 1e-5 * p0
    fd = (J_oracle(p0 + h) - J_oracle(p0 - h)) / (2 * h)
    assert abs(fd) > 1e-6 * J_ref / p0          # a genuinely p-dependent truncated misfit
    assert abs(dJdp - fd) <= 1e-5 * abs(fd), (dJdp, fd)
    # the handle is back in its zero state and solves like a fresh one
    _, n, rel = sol.solve(1e-10)
    _, n_ref, _, _ = oracle.Schwarz.from_problem(prob, p=p0).solve(inner_rtol=1e-14, rtol=1e-10, max_outer=400)
    assert rel <= 1e-10 and abs(n - n_ref) <= 1, (n, n_ref)
