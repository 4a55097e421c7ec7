"""Pins for the IRLS/CGLS oracle (ch. 4) against closed forms, library
solvers (least squares, linear programming) and the paper's constants."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import brentq, linprog

from oracle import irls, stolt
from paper_1711_10214_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _const(name):
    with open(GOLDEN) as f:
        return json.load(f)[name]["value"]


def test_median_and_mad():
    assert irls.median([3.0, 1.0, 2.0]) == 2.0
    assert irls.median([4.0, 1.0, 2.0, 3.0]) == 2.5
    assert irls.mad([1.0, 2.0, 3.0, 4.0, 100.0]) == 1.0
    x = np.random.default_rng(0).standard_normal(1001)
    assert irls.median(x) == np.median(x)


def test_defaults_follow_paper_constants():
    import inspect
    sig = inspect.signature(irls.irls)
    assert sig.parameters["b_r"].default == _const("b_r")
    r = np.array([-3.0, -1.0, 0.0, 2.0, 10.0])
    assert irls.eps_residual(r) == pytest.approx(
        _const("b_r") * irls.mad(r) / _const("mad_normaliser"))
    assert irls.eps_model(np.array([0.0, -4.0, 2.0]), 1.0) == 4.0 / _const("eps_m_divisor")


def _dense_ops(A):
    return (lambda x: A @ x), (lambda r: A.T @ r)


def test_l2_first_outer_equals_least_squares():
    """p = q = 2: W = I, one outer iteration is CGLS, which reaches the
    least-squares solution in rank(A) iterations (exact arithmetic)."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 6))
    b = rng.standard_normal(30)
    f, t = _dense_ops(A)
    x, _ = irls.irls(f, t, b, n_outer=1, n_cg=12, p=2, q=2)
    np.testing.assert_allclose(x, np.linalg.lstsq(A, b, rcond=None)[0], atol=1e-10)


def test_constant_fit_is_huber_location():
    """Fitting a constant with p = 1 and eps_r = b_r MAD/0.6745 (Eq.
    ch4_epcilon_r): since MAD is shift invariant, the IRLS fixed point solves
    sum clip((y - x)/c, -1, 1) = 0 with c = 1.345 MAD(y)/0.6745 (Huber's
    location M-estimate), solved here independently by bracketing."""
    rng = np.random.default_rng(2)
    y = np.concatenate([rng.standard_normal(40), 8.0 + rng.standard_normal(9)])
    A = np.ones((y.size, 1))
    f, t = _dense_ops(A)
    x, rep = irls.irls(f, t, y, n_outer=120, n_cg=2, p=1, q=2)
    c = 1.345 * np.median(np.abs(y - np.median(y))) / 0.6745
    x_ref = brentq(lambda z: np.sum(np.clip((y - z) / c, -1, 1)), y.min(), y.max(), xtol=1e-14)
    assert abs(x[0] - x_ref) < 1e-8
    assert abs(x[0] - np.mean(y)) > 0.5        # far from the l2 answer


def test_l1_fit_of_constant_is_median():
    """l1 fit of a constant is the median (ch. 4 derivation): IRLS with a tiny
    fixed eps converges to it."""
    y = np.array([0.3, -1.2, 5.0, 0.9, 100.0, 0.1, -0.4])
    f, t = _dense_ops(np.ones((y.size, 1)))
    x, _ = irls.irls(f, t, y, n_outer=300, n_cg=2, p=1, q=2, eps_r_fixed=1e-12)
    assert abs(x[0] - np.median(y)) < 1e-6


def _lp_l1(A, b, mu=0.0):
    """min sum|A x - b| + mu sum|x| as an LP (scipy HiGHS)."""
    m, n = A.shape
    # variables: x+ (n), x- (n), e+ (m), e- (m);  A(x+ - x-) - e+ + e- = b
    c = np.concatenate([mu * np.ones(2 * n), np.ones(2 * m)])
    Aeq = np.hstack([A, -A, -np.eye(m), np.eye(m)])
    res = linprog(c, A_eq=Aeq, b_eq=b, bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_robust_irls_matches_lp(mu):
    """p = q = 1: the IRLS fixed point minimises ||Ax - b||_1 + mu ||x||_1
    (Eq. ch4_cost_fn via Eqs equ:10/equ:11); checked against an exact LP."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 5))
    x_true = rng.standard_normal(5)
    b = A @ x_true + 0.01 * rng.standard_normal(40)
    out = rng.choice(40, 4, replace=False)
    b[out] += rng.choice([-1, 1], 4) * 20.0
    f, t = _dense_ops(A)
    x, _ = irls.irls(f, t, b, n_outer=300, n_cg=10, p=1, q=1 if mu > 0 else 2, mu=mu,
                     eps_r_fixed=1e-9, eps_m_fixed=1e-9 if mu > 0 else None)
    obj = np.sum(np.abs(A @ x - b)) + mu * np.sum(np.abs(x))
    ref = _lp_l1(A, b, mu)
    assert abs(obj - ref) / ref < 1e-3


def test_q_closed_form():
    d = np.random.default_rng(4).standard_normal((8, 16))
    assert irls.q_db(d, 0.9 * d) == pytest.approx(20.0, abs=1e-10)
    assert irls.q_db(d, 0.99 * d) == pytest.approx(40.0, abs=1e-10)


def test_robust_beats_least_squares_on_blended_gather():
    """ch. 4 finding: with erratic blending noise the robust (p = 1) solve
    recovers the clean gather better than the l2 one (Q = Q_R - Q_PD > 0 for
    both, larger for p = 1)."""
    c = synth.config1(0)
    # a reduced copy of config 1 (every other trace / first 128 samples) keeps the test quick
    clean = c["clean"][::2, :128]
    blended = c["blended"][::2, :128]
    g = stolt.Geometry(128, 32, c["dt"], 2 * c["dx"], c["velocities"], wavelet_peak_hz=20.0)
    f = lambda m: stolt.forward(g, m)
    t = lambda d: stolt.adjoint(g, d)
    q = {}
    for p in (1, 2):
        m, rep = irls.irls(f, t, blended, n_outer=4, n_cg=10, p=p, q=1)
        q[p] = irls.q_db(clean, rep["d_model"]) - irls.q_db(clean, blended)
    assert q[2] > 0.0
    assert q[1] > q[2] + 1.0


def test_warm_start_at_the_solution_stays_there():
    """Starting from the l2 solution with p = q = 2 (W = I), CGLS has nothing
    left to do: the warm-started solve returns m0."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 6))
    b = rng.standard_normal(30)
    f, t = _dense_ops(A)
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    x, rep = irls.irls(f, t, b, n_outer=2, n_cg=10, p=2, q=2, m0=x_ls)
    np.testing.assert_allclose(x, x_ls, atol=1e-9)
    # wr0 = weights: a weighted l2 solve equals the weighted least squares
    w = rng.uniform(0.2, 2.0, 30)
    x_w, _ = irls.irls(f, t, b, n_outer=1, n_cg=12, p=2, q=2, wr0=w)
    ref = np.linalg.lstsq(w[:, None] * A, w * b, rcond=None)[0]
    np.testing.assert_allclose(x_w, ref, atol=1e-9)


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_robust_irls_on_restricted_stolt_matches_lp(mu):
    """The robust solve on the Stolt operator itself (ch. 4 Eq. ch4_cost_fn
    with p = q = 1; ch. 5 operator): L restricted to 12 active model
    coefficients of a 16-sample x 8-trace gather with two scan velocities,
    data = L x + small noise with 10% of the samples hit by large erratic
    spikes (blending-like outliers).  IRLS runs through the oracle's
    operator pair (forward / exact transpose, restricted and embedded), with
    a fixed tiny eps for 200 outer iterations; its objective
    ||L x - d||_1 + mu ||x||_1 must be within 1e-3 of the exact LP optimum
    (scipy HiGHS on the explicit 128 x 12 matrix, built column by column
    from unit models)."""
    nt, nx = 16, 8
    g = stolt.Geometry(nt, nx, 0.004, 12.5, [1500.0, 2500.0])
    rng = np.random.default_rng(21)
    n_model = int(np.prod(g.model_shape))
    active = np.sort(rng.choice(n_model, 12, replace=False))

    def embed(x):
        m = np.zeros(n_model)
        m[active] = x
        return m.reshape(g.model_shape)

    def fwd(x):
        return stolt.forward(g, embed(x))

    def adj(r):
        return stolt.adjoint(g, r).ravel()[active]

    A = np.stack([fwd(e).ravel() for e in np.eye(12)], axis=1)
    assert np.linalg.matrix_rank(A) == 12
    x_true = rng.standard_normal(12)
    b = A @ x_true + 1e-3 * rng.standard_normal(A.shape[0])
    out = rng.choice(b.size, b.size // 10, replace=False)
    b[out] += rng.choice([-1.0, 1.0], out.size) * 5.0 * np.max(np.abs(A @ x_true))
    x, rep = irls.irls(fwd, adj, b.reshape(nx, nt), n_outer=200, n_cg=24, p=1,
                       q=1 if mu > 0 else 2, mu=mu, eps_r_fixed=1e-9,
                       eps_m_fixed=1e-9 if mu > 0 else None)
    obj = np.sum(np.abs(A @ x - b)) + mu * np.sum(np.abs(x))
    ref = _lp_l1(A, b, mu)
    assert abs(obj - ref) / ref < 1e-3, (obj, ref)
    # the l2 fit of the same data is far from the l1 optimum
    x2 = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.sum(np.abs(A @ x2 - b)) > 1.05 * ref
