"""l2-l1 sparse Radon inversion by FISTA with a power-method step, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows ch. 6, "Sparse inversion" (AASHRT interpolation):
  * cost J(m) = ||S (d - L m)||_2^2 + mu ||m||_1   (Eq. cost_fn with p = 2, q = 1;
    S the trace-sampling operator, a diagonal of per-trace weights)
  * minimised by FISTA (Beck and Teboulle 2009), whose step needs the largest
    eigenvalue of L^T S^T S L, estimated by Rayleigh's power method.

Steps, in the published algorithm's order (f(m) = ||S (d - L m)||^2, so
grad f(m) = 2 L^T S^T (S L m - S d) and its Lipschitz constant is
Lf = 2 lambda_max(L^T S^T S L)):
  power method: v = v0 / ||v0||; n_power times: w = L^T S^T S L v,
                lambda = ||w||, v = w / lambda
  FISTA:        x_0 = 0, y_1 = x_0, t_1 = 1; for k = 1 .. n_iter:
                x_k = soft(y_k - grad f(y_k) / Lf, mu / Lf)
                t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
                y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})
  soft(z, a) = sign(z) max(|z| - a, 0).
Readings where the thesis is silent: the starting model is zero; the
starting vector v0 of the power method is an input (the random draw is the
caller's); lambda = 0 (nothing sampled, or v0 in the null space) leaves the
model at zero.
"""
import numpy as np

from . import stolt


def soft(z, a):
    """Soft threshold (the proximal map of a ||.||_1)."""
    return np.sign(z) * np.maximum(np.abs(z) - a, 0.0)


def momentum(n_iter):
    """beta_k = (t_k - 1) / t_{k+1}, k = 1 .. n_iter, t_1 = 1."""
    t, out = 1.0, []
    for _ in range(n_iter):
        t1 = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        out.append((t - 1.0) / t1)
        t = t1
    return out


def power_method(normal_op, v0, n_power):
    """Largest eigenvalue of the symmetric positive semi-definite normal_op."""
    v = np.asarray(v0, dtype=np.float64)
    nv = np.linalg.norm(v)
    if nv == 0.0:
        return 0.0
    v = v / nv
    lam = 0.0
    for _ in range(n_power):
        w = normal_op(v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


def fista(fwd, adj, d, mu, n_iter, lf, model_shape):
    """FISTA on J(m) = ||d - A m||^2 + mu ||m||_1 with A = fwd, A^T = adj
    (any sampling is inside fwd / adj and d), step 1 / lf."""
    x = np.zeros(model_shape)
    if lf <= 0.0:
        return x
    y = x.copy()
    for beta in momentum(n_iter):
        grad = 2.0 * adj(fwd(y) - d)
        x_new = soft(y - grad / lf, mu / lf)
        y = x_new + beta * (x_new - x)
        x = x_new
    return x


def stolt_fista(g, d, mask, v0, mu, n_iter, n_power):
    """The Stolt ASHRT/AASHRT instance: A = S L with S = diag(mask) over the
    traces (mask None: every trace).  Returns (m, Lf)."""
    sd = d if mask is None else d * np.asarray(mask, dtype=np.float64)[:, None]

    def fwd(m):
        return stolt.forward(g, m, mask)

    def adj(r):
        return stolt.adjoint(g, r, mask)

    lam = power_method(lambda v: adj(fwd(v)), v0, n_power)
    lf = 2.0 * lam
    return fista(fwd, adj, sd, mu, n_iter, lf, g.model_shape), lf
