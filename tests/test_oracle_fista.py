"""Pins for the FISTA / power-method oracle (ch. 6, "Sparse inversion":
Eq. cost_fn with p = 2, q = 1).

Checked against things other than the oracle itself: hand values of the
soft threshold and of the momentum sequence, the eigenvalues of explicit
matrices (numpy's symmetric eigensolver), the closed-form minimiser for an
identity operator, the optimality (KKT) conditions of the convex problem,
and the O(1/k^2) bound of Beck and Teboulle's theorem.
"""
import numpy as np

from oracle import fista, stolt

DT, DX = 0.004, 12.5


def test_soft_threshold_hand_values():
    z = np.array([-3.0, -0.5, 0.0, 0.2, 2.5])
    assert np.array_equal(fista.soft(z, 1.0), np.array([-2.0, 0.0, 0.0, 0.0, 1.5]))
    assert np.array_equal(fista.soft(z, 0.0), z)


def test_momentum_sequence_hand_values():
    b = fista.momentum(3)
    t2 = (1.0 + np.sqrt(5.0)) / 2.0
    t3 = (1.0 + np.sqrt(1.0 + 4.0 * t2 * t2)) / 2.0
    t4 = (1.0 + np.sqrt(1.0 + 4.0 * t3 * t3)) / 2.0
    assert b[0] == 0.0
    assert abs(b[1] - (t2 - 1.0) / t3) < 1e-15
    assert abs(b[2] - (t3 - 1.0) / t4) < 1e-15


def test_power_method_finds_the_largest_eigenvalue():
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    ev = np.array([0.1, 0.5, 1.0, 2.0, 3.0, 3.5, 4.0, 5.0, 6.0, 6.5, 8.0, 10.0])
    A = Q @ np.diag(ev) @ Q.T
    lam = fista.power_method(lambda v: A @ v, rng.standard_normal(12), 200)
    assert abs(lam - 10.0) < 1e-9
    assert fista.power_method(lambda v: A @ v, np.zeros(12), 5) == 0.0


def test_identity_operator_gives_the_closed_form_minimiser():
    """min ||d - m||^2 + mu ||m||_1 is m = soft(d, mu / 2)."""
    rng = np.random.default_rng(1)
    d = rng.standard_normal(50)
    mu = 0.8
    x = fista.fista(lambda m: m, lambda r: r, d, mu, 25, 2.0, d.shape)
    assert np.allclose(x, fista.soft(d, mu / 2.0), atol=1e-14)


def _kkt_violation(A, d, x, mu):
    g = 2.0 * A.T @ (d - A @ x)          # -grad f: mu * subgradient at the optimum
    nz = x != 0.0
    v1 = np.abs(g[nz] - mu * np.sign(x[nz])).max(initial=0.0)
    v2 = np.maximum(np.abs(g[~nz]) - mu, 0.0).max(initial=0.0)
    return max(v1, v2)


def test_dense_lasso_meets_kkt_and_the_rate_bound():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 60))
    d = A @ (rng.standard_normal(60) * (rng.random(60) < 0.15)) + 0.01 * rng.standard_normal(30)
    mu = 0.5
    lf = 2.0 * np.linalg.eigvalsh(A.T @ A).max()
    x_star = fista.fista(lambda m: A @ m, lambda r: A.T @ r, d, mu, 20000, lf, (60,))
    assert _kkt_violation(A, d, x_star, mu) < 1e-6
    J = lambda x: float(np.sum((d - A @ x) ** 2) + mu * np.abs(x).sum())
    # Beck & Teboulle, Theorem 4.4: J(x_k) - J* <= 2 Lf ||x_0 - x*||^2 / (k + 1)^2
    # (their Lipschitz constant is that of grad f = our lf)
    for k in (5, 20, 100):
        xk = fista.fista(lambda m: A @ m, lambda r: A.T @ r, d, mu, k, lf, (60,))
        assert J(xk) - J(x_star) <= 2.0 * lf * np.sum(x_star ** 2) / (k + 1) ** 2 + 1e-12


def test_stolt_power_method_matches_the_explicit_normal_matrix():
    """lambda_max(L^T S^T S L) of a tiny Stolt geometry, the operator written
    out as a matrix column by column, against numpy's eigensolver."""
    g = stolt.Geometry(16, 4, DT, DX, [1800.0])
    mask = np.array([1.0, 0.0, 1.0, 1.0])
    n = int(np.prod(g.model_shape))
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(stolt.adjoint(g, stolt.forward(g, e.reshape(g.model_shape), mask), mask).ravel())
    N = np.array(cols).T
    assert np.allclose(N, N.T, atol=1e-12)
    lam_ref = np.linalg.eigvalsh(N).max()
    v0 = np.random.default_rng(3).standard_normal(g.model_shape)
    normal = lambda v: stolt.adjoint(g, stolt.forward(g, v, mask), mask)
    assert abs(fista.power_method(normal, v0, 300) - lam_ref) < 1e-8 * lam_ref


def test_stolt_fista_meets_kkt():
    g = stolt.Geometry(16, 4, DT, DX, [1800.0, 2600.0])
    rng = np.random.default_rng(4)
    d = rng.standard_normal(g.data_shape)
    mask = np.array([1.0, 1.0, 0.0, 1.0])
    mu = 0.05
    m, lf = fista.stolt_fista(g, d, mask, rng.standard_normal(g.model_shape), mu, 4000, 300)
    n = int(np.prod(g.model_shape))
    A = np.array([stolt.forward(g, np.eye(n)[i].reshape(g.model_shape), mask).ravel()
                  for i in range(n)]).T
    sd = (d * mask[:, None]).ravel()
    assert _kkt_violation(A, sd, m.ravel(), mu) < 1e-5 * max(1.0, np.abs(A.T @ sd).max())


def test_interpolation_of_decimated_traces():
    """The use of ch. 6: a gather of events that the velocity scan can
    represent, every other trace removed, is rebuilt on the missing traces far
    better than by leaving them empty."""
    nt, nx = 64, 32
    v = [1500.0, 2000.0]
    g = stolt.Geometry(nt, nx, DT, DX, v)
    m_true = np.zeros(g.model_shape)
    m_true[0, 0, 10, 20] = 1.0
    m_true[0, 1, 22, 35] = -0.8
    d_full = stolt.forward(g, m_true)
    mask = np.zeros(nx)
    mask[::2] = 1.0
    v0 = np.random.default_rng(5).standard_normal(g.model_shape)
    m, _ = fista.stolt_fista(g, d_full * mask[:, None], mask, v0, 1e-4, 200, 30)
    rec = stolt.forward(g, m)
    miss = mask == 0.0
    err = np.linalg.norm(rec[miss] - d_full[miss]) / np.linalg.norm(d_full[miss])
    assert err < 0.2, err
