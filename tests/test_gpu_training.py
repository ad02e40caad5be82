"""Adjoint gradients with device-resident angles, the autograd wrapper, finite-difference
checks at the adjoint-gradient workload sizes, and the on-device Adam loop.

Tolerances:
* gradient_dev vs gradient (host angles): 1e-12 max(1, sum|w|) (cos/sin of the angles
  are taken on the device instead of the host, 1 ulp apart);
* vs the oracle: 1e-10 max(1, sum|w|) as for every complex128 gradient;
* central differences with h = 1e-6: truncation h^2/6 |E'''| plus rounding 2 eps_E / h,
  below 1e-6 max(1, sum|w|) for these instances;
* Adam: the oracle-driven CPU Adam and the device loop agree to 1e-9 on the angles.
"""
import numpy as np
import pytest

import synth
from oracle import qaoa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402


def instance(n, seed, prob=0.2, weights="u01"):
    e, w, integer = synth.graph("gnp", n, seed, weights=weights, prob=prob)
    return q.Graph(n, e, w, integer), e, w, integer


def scale_of(w):
    return max(1.0, float(np.sum(np.abs(w))))


@pytest.mark.parametrize("n,p,dtype", [(9, 3, "c128"), (14, 4, "c128"), (14, 4, "c64")])
def test_gradient_dev_matches_host_angles_and_oracle(n, p, dtype):
    g, e, w, integer = instance(n, n, prob=0.5)
    cv = q.cost_vector(g, "f64")
    gam, bet = synth.angles(p, 3)
    psi, lam = q.new_state(n, dtype), q.new_state(n, dtype)
    host = q.gradient(psi, lam, cv, gam, bet).cpu().numpy()
    ang = torch.tensor(np.concatenate([gam, bet]), device="cuda")
    dev = q.gradient_dev(psi, lam, cv, ang).cpu().numpy()
    s = scale_of(w)
    tol = 1e-12 * s if dtype == "c128" else 1e-5 * s
    assert np.max(np.abs(host - dev)) <= tol
    C = qaoa.cut_values(n, e, w, integer=False)
    E, dg, db, _ = qaoa.adjoint_gradient(n, C, gam, bet)
    ref = np.concatenate([[E], dg, db])
    got = np.concatenate([dev[:1], dev[2:]])
    tol = 1e-10 * s if dtype == "c128" else 1e-4 * np.maximum(1.0, np.abs(ref))  # complex64: per value
    assert np.all(np.abs(got - ref) <= tol)


def test_autograd_function():
    n, p = 12, 3
    g, e, w, integer = instance(n, 4, prob=0.4)
    cv = q.cost_vector(g, "f64")
    gam, bet = synth.angles(p, 9)
    f = q.QAOAExpectation(cv)
    ang = torch.tensor(np.concatenate([gam, bet]), device="cuda", requires_grad=True)
    E = f(ang)
    (3.0 * E).backward()
    C = qaoa.cut_values(n, e, w, integer=False)
    E0, dg, db, _ = qaoa.adjoint_gradient(n, C, gam, bet)
    s = scale_of(w)
    assert abs(E.item() - E0) <= 1e-10 * s
    assert np.max(np.abs(ang.grad.cpu().numpy() - 3.0 * np.concatenate([dg, db]))) <= 3e-10 * s


@pytest.mark.parametrize("n", [24, 30])
def test_adjoint_vs_central_differences_p10(n):
    """G(n, 0.2), U(0,1) weights, p = 10, complex128: the 20-angle gradient against central
    differences of <C> (h = 1e-6), both on the device."""
    p, h = 10, 1e-6
    g, e, w, integer = instance(n, 1, prob=0.2)
    cv = q.cost_vector(g, "f64")
    gam, bet = synth.angles(p, 2)
    psi, lam = q.new_state(n, "c128"), q.new_state(n, "c128")
    out = q.gradient(psi, lam, cv, gam, bet).cpu().numpy()

    def E(gg, bb):
        return q.apply_layers(psi, cv, gg, bb, expect=True)[0].item()

    fd = np.zeros(2 * p)
    for l in range(p):
        d = np.zeros(p)
        d[l] = h
        fd[l] = (E(gam + d, bet) - E(gam - d, bet)) / (2 * h)
        fd[p + l] = (E(gam, bet + d) - E(gam, bet - d)) / (2 * h)
    assert np.max(np.abs(out[2:] - fd)) <= 1e-6 * scale_of(w)
    del psi, lam, cv
    torch.cuda.empty_cache()


def adam_reference(n, C, ang0, steps, lr, b1, b2, eps):
    """Adam ascent driven by the oracle's adjoint gradient (test reference)."""
    p = len(ang0) // 2
    ang = np.array(ang0, dtype=np.float64)
    m, v = np.zeros(2 * p), np.zeros(2 * p)
    rows = []
    for t in range(1, steps + 1):
        E, dg, db, _ = qaoa.adjoint_gradient(n, C, ang[:p], ang[p:])
        gr = np.concatenate([dg, db])
        rows.append(np.concatenate([[E], gr, ang]))
        m = b1 * m + (1 - b1) * gr
        v = b2 * v + (1 - b2) * gr * gr
        ang = ang + lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return ang, np.array(rows)


def test_adam_loop_matches_oracle_driven_adam():
    n, p, steps = 8, 2, 25
    g, e, w, integer = instance(n, 6, prob=0.5)
    cv = q.cost_vector(g, "f64")
    C = qaoa.cut_values(n, e, w, integer=False)
    gam, bet = synth.angles(p, 5)
    ang0 = np.concatenate([gam, bet])
    ang = torch.tensor(ang0, device="cuda")
    hist = q.optimize_adam(cv, ang, steps, lr=0.05).cpu().numpy()
    ref_ang, ref_rows = adam_reference(n, C, ang0, steps, 0.05, 0.9, 0.999, 1e-8)
    s = scale_of(w)
    assert np.max(np.abs(hist[:, 0] - ref_rows[:, 0])) <= 1e-9 * s
    assert np.max(np.abs(hist[:, 2:2 + 2 * p] - ref_rows[:, 1:1 + 2 * p])) <= 1e-9 * s
    assert np.max(np.abs(hist[:, 2 + 2 * p:] - ref_rows[:, 1 + 2 * p:])) <= 1e-9
    assert np.max(np.abs(ang.cpu().numpy() - ref_ang)) <= 1e-9


def test_adam_200_steps_improves_cut_n20():
    """A 200-step loop on the device raises <C> and never leaves the device inside the loop."""
    n, p = 20, 4
    g, e, w, integer = instance(n, 8, prob=0.2)
    cv = q.cost_vector(g, "f64")
    gam, bet = synth.angles(p, 1)
    ang = torch.tensor(np.concatenate(q.linear_ramp(p)), device="cuda") * 0.5
    launches0 = q.launch_count()
    hist = q.optimize_adam(cv, ang, 200, lr=0.02).cpu().numpy()
    assert hist.shape == (200, 4 * p + 2)
    assert hist[-1, 0] > hist[0, 0]
    assert abs(hist[-1, 1] - 1.0) < 1e-10
    # first step launched directly, the other 199 replay one captured graph
    assert q.launch_count() - launches0 < 200


def lbfgs_reference(n, C, ang0, max_evals, m, gtol, c1=1e-4):
    """The same L-BFGS rules on the CPU, driven by the oracle's adjoint gradient (minimising
    f = -E): Armijo backtracking with the safeguarded quadratic step, two-loop direction
    with H0 = s.y / y.y, restart on a non-descent direction.  Returns (rows, x_best, status)."""
    p = len(ang0) // 2
    pt = np.array(ang0, dtype=np.float64)
    x = g = d = None
    fk = alpha = gtd = 0.0
    S, Y, rho = [], [], []
    rows = []
    for ev in range(max_evals):
        E, dg, db, _ = qaoa.adjoint_gradient(n, C, pt[:p], pt[p:])
        grad = np.concatenate([dg, db])
        rows.append(np.concatenate([[E, 1.0], grad, pt]))
        ft, gt = -E, -grad
        if ev == 0 or ft <= fk + c1 * alpha * gtd:
            if ev > 0:
                s, yv = pt - x, gt - g
                sy = s @ yv
                if sy > 1e-12 * np.sqrt((s @ s) * (yv @ yv)) and sy > 0:
                    S.append(s), Y.append(yv), rho.append(1.0 / sy)
                    if len(S) > m:
                        S.pop(0), Y.pop(0), rho.pop(0)
            x, g, fk = pt.copy(), gt.copy(), ft
            if np.max(np.abs(g)) < gtol:
                return rows, x, "converged"
            q = g.copy()
            al = [0.0] * len(S)
            for k in range(len(S) - 1, -1, -1):
                al[k] = rho[k] * (S[k] @ q)
                q -= al[k] * Y[k]
            h0 = (1.0 / (rho[-1] * (Y[-1] @ Y[-1]))) if S else 1.0 / max(1.0, np.linalg.norm(g))
            r = h0 * q
            for k in range(len(S)):
                b = rho[k] * (Y[k] @ r)
                r += S[k] * (al[k] - b)
            d = -r
            gtd = g @ d
            if not gtd < 0:
                S, Y, rho = [], [], []
                d = -g / max(1.0, np.linalg.norm(g))
                gtd = g @ d
            alpha = 1.0
        else:
            den = 2.0 * (ft - fk - gtd * alpha)
            a = -gtd * alpha * alpha / den if den > 0 else 0.5 * alpha
            alpha = min(max(a, 0.1 * alpha), 0.5 * alpha)
            if alpha < 1e-12:
                return rows, x, "no progress"
        pt = x + alpha * d
    return rows, x, "evaluations used up"


def test_lbfgs_matches_oracle_driven_lbfgs():
    n, p = 8, 2
    g, e, w, integer = instance(n, 6, prob=0.5)
    cv = q.cost_vector(g, "f64")
    C = qaoa.cut_values(n, e, w, integer=False)
    gam, bet = synth.angles(p, 5)
    ang0 = np.concatenate([gam, bet])
    ang = torch.tensor(ang0, device="cuda")
    hist, info = q.optimize_lbfgs(cv, ang, max_evals=40, m=5, gtol=1e-7)
    rows, xbest, status = lbfgs_reference(n, C, ang0, 40, 5, 1e-7)
    rows = np.array(rows)
    hist = hist.cpu().numpy()
    s = scale_of(w)
    k = min(len(rows), len(hist), 25)  # the first evaluations, before rounding can flip a decision
    assert np.max(np.abs(hist[:k, 0] - rows[:k, 0])) <= 1e-9 * s
    assert np.max(np.abs(hist[:k, 2 + 2 * p:] - rows[:k, 2 + 2 * p:])) <= 1e-8
    if info["status"] == status == "converged":
        assert np.max(np.abs(ang.cpu().numpy() - xbest)) <= 1e-6


def test_lbfgs_converges_to_a_stationary_point():
    n, p = 12, 3
    g, e, w, integer = instance(n, 3, prob=0.4)
    cv = q.cost_vector(g, "f64")
    C = qaoa.cut_values(n, e, w, integer=False)
    ang = torch.tensor(np.concatenate(synth.angles(p, 8)), device="cuda")
    E0 = qaoa.adjoint_gradient(n, C, *np.split(ang.cpu().numpy(), 2))[0]
    hist, info = q.optimize_lbfgs(cv, ang, max_evals=300, m=10, gtol=1e-6)
    assert info["status"] == "converged", info
    a = ang.cpu().numpy()
    E, dg, db, _ = qaoa.adjoint_gradient(n, C, a[:p], a[p:])
    assert E >= E0 and abs(E - info["E"]) <= 1e-10 * scale_of(w)
    assert np.max(np.abs(np.concatenate([dg, db]))) <= 1e-5


def test_lbfgs_200_evaluations_n24_p10():
    """The adjoint-gradient workload's optimisation loop: G(24, 0.2), U(0,1), p = 10, up to 200
    evaluations on the device; accepted values never decrease and E rises."""
    n, p = 24, 10
    g, e, w, integer = instance(n, 1, prob=0.2)
    cv = q.cost_vector(g, "f64")
    ang = torch.tensor(np.concatenate(q.linear_ramp(p)), device="cuda") * 0.4
    launches0 = q.launch_count()
    hist, info = q.optimize_lbfgs(cv, ang, max_evals=200, m=10, gtol=1e-7)
    h = hist.cpu().numpy()
    assert len(h) == info["evaluations"] >= 2
    assert info["E"] > h[0, 0]
    assert np.all(np.abs(h[:, 1] - 1.0) <= 1e-10)
    assert q.launch_count() - launches0 < 60  # one direct evaluation, then graph replays


def test_adam_checkpoint_resume_is_exact():
    """12 steps, a checkpoint (angles + optimiser state to host and back), 8 more steps: the
    same trajectory, bit for bit, as 20 uninterrupted steps."""
    n, p = 10, 3
    g, e, w, integer = instance(n, 12, prob=0.5)
    cv = q.cost_vector(g, "f64")
    ang0 = np.concatenate(synth.angles(p, 14))
    a = torch.tensor(ang0, device="cuda")
    full = q.optimize_adam(cv, a, 20, lr=0.03).cpu().numpy()
    b = torch.tensor(ang0, device="cuda")
    st = q.optimizer_state("adam", p)
    h1 = q.optimize_adam(cv, b, 12, lr=0.03, state=st).cpu().numpy()
    saved_ang, saved_st = b.cpu().numpy(), st.cpu().numpy()
    b2, st2 = torch.tensor(saved_ang, device="cuda"), torch.tensor(saved_st, device="cuda")
    h2 = q.optimize_adam(cv, b2, 8, lr=0.03, state=st2, resume=True).cpu().numpy()
    assert np.array_equal(np.concatenate([h1, h2]), full)
    assert np.array_equal(b2.cpu().numpy(), a.cpu().numpy())


def test_lbfgs_checkpoint_resume_is_exact():
    n, p = 10, 3
    g, e, w, integer = instance(n, 13, prob=0.5)
    cv = q.cost_vector(g, "f64")
    ang0 = np.concatenate(synth.angles(p, 15))
    a = torch.tensor(ang0, device="cuda")
    full, info_full = q.optimize_lbfgs(cv, a, max_evals=30, m=6, gtol=1e-13)
    b = torch.tensor(ang0, device="cuda")
    st = q.optimizer_state("lbfgs", p)
    h1, _ = q.optimize_lbfgs(cv, b, max_evals=14, m=6, gtol=1e-13, state=st)
    saved_ang, saved_st = b.cpu().numpy(), st.cpu().numpy()
    b2, st2 = torch.tensor(saved_ang, device="cuda"), torch.tensor(saved_st, device="cuda")
    h2, info2 = q.optimize_lbfgs(cv, b2, max_evals=16, m=6, gtol=1e-13, state=st2, resume=True)
    assert np.array_equal(np.concatenate([h1.cpu().numpy(), h2.cpu().numpy()]), full.cpu().numpy())
    assert np.array_equal(b2.cpu().numpy(), a.cpu().numpy())
    assert info2 == info_full
